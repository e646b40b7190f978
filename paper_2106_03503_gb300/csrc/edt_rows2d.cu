// Row pass of the 2-D exact EDT (Sec. 3.3.1 of Strutz, "The Distance
// Transform and its Computation": lower envelope of the parabolas of Eq. (5)
// per row), fused with the end of the column pass and the optional sqrt.
//
// One block handles one band of 32 rows over the full width W: lane l of
// every warp works on row 32*band + l, and the warps split the columns into
// segments (band engine, edt_engine.cuh).  The prologue stages, per column,
// the band's source-bit word and the nearest source rows above and below the
// band (8 bytes per column, from the column-pass scratch) in shared memory.
// For row i the nearest source row g of column k then follows from a few bit
// operations (highest set bit at or above the row, lowest at or below), i.e.
// the squared vertical distance D_v(k) = (i - g)^2 of Fig. 18(b) is rebuilt on
// demand and never stored; all 32 rows read the same column word at once.
#include "edt_engine.cuh"
#include "edt_internal.h"

namespace edt {

// Encoded nearest source rows outside the band: up as int16 (-32768 = none),
// dn as uint16 (65535 = none), so that i - up and dn - i exceed any real
// distance (< 32768) when there is no source on that side.
constexpr uint32_t UP_NONE = 0x8000u;
constexpr uint32_t DN_NONE = 0xFFFFu;

struct BandRow2D {
    const uint32_t* bits;   // [W]: source bits of the band's 32 rows
    const uint32_t* updn;   // [W]: encoded up | dn << 16
    int base;               // first row of the band
    int i;                  // this lane's row
    int W;
    uint32_t mle, mge;      // bits at / above and at / below this row
    bool valid;

    __device__ __forceinline__ bool parts(int k, int& up, int& dn) const
    {
        const uint32_t w = bits[k];
        const uint32_t ud = updn[k];
        const uint32_t a = w & mle, b = w & mge;
        up = a ? base + 31 - __clz(a) : (int)(short)(ud & 0xFFFFu);
        dn = b ? base + __ffs(b) - 1 : (int)(ud >> 16);
        return valid;
    }
    __device__ __forceinline__ bool eval(int k, int& f) const
    {
        int up, dn;
        if (!parts(k, up, dn)) return false;
        const int d = min(i - up, dn - i);
        if (d >= 32768) return false;
        f = d * d;
        return true;
    }
    __device__ __forceinline__ int c(int k) const
    {
        int up, dn;
        parts(k, up, dn);
        const int d = min(i - up, dn - i);
        return d * d + k * k;
    }
    __device__ __forceinline__ int feature(int k) const
    {
        int up, dn;
        parts(k, up, dn);
        return ((i - up <= dn - i) ? up : dn) * W + k;
    }
};

struct BandOut2D {
    int32_t* D;
    int32_t* F;
    float* dist;
    int base, H, W;
    __device__ __forceinline__ void store(int ln, int j, int v, int f) const
    {
        const int row = base + ln;
        if (row >= H) return;
        const int64_t idx = (int64_t)row * W + j;
        if (D) D[idx] = v;
        if (F) F[idx] = f;
        if (dist) dist[idx] = sqrt_rn_int(v);
    }
};

// Shared memory of one band block: column data + band engine.
static size_t band2d_smem(int W, int lg, int NW)
{
    return (((size_t)8 * W + 15) & ~size_t(15)) + band_smem_bytes(NW, (1 << lg) >> 5, true);
}

__global__ void __launch_bounds__(1024)
k_rows2d(int H, int W, ColScratch s, int lg, int NW, int32_t* D, int32_t* F, float* dist)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t* sbits = reinterpret_cast<uint32_t*>(smem);
    uint32_t* supdn = sbits + W;
    const BandSmem sm = carve_band_smem(smem + (((size_t)8 * W + 15) & ~size_t(15)), NW,
                                        (1 << lg) >> 5, true);
    const int b = blockIdx.x;
    const int G = b >> 5;
    const uint32_t* Cb = s.C + (int64_t)b * W;
    const uint32_t* Ub = s.U + (int64_t)b * W;
    const uint32_t* GABg = s.GAB + (int64_t)G * W;
    for (int j = threadIdx.x; j < W; j += blockDim.x) {
        const uint32_t u = Ub[j];
        uint32_t up = u & 0xFFFFu, dn = u >> 16;
        if (up == (uint32_t)NONE16 || dn == (uint32_t)NONE16) {
            const uint32_t gab = GABg[j];
            if (up == (uint32_t)NONE16) up = gab & 0xFFFFu;
            if (dn == (uint32_t)NONE16) dn = gab >> 16;
        }
        sbits[j] = Cb[j];
        supdn[j] = (up == (uint32_t)NONE16 ? UP_NONE : up) | ((dn == (uint32_t)NONE16 ? DN_NONE : dn) << 16);
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    BandRow2D line;
    line.bits = sbits;
    line.updn = supdn;
    line.base = b * 32;
    line.i = b * 32 + lane;
    line.W = W;
    line.mle = FULL >> (31 - lane);
    line.mge = FULL << lane;
    line.valid = line.i < H;
    const BandOut2D out{D, F, dist, b * 32, H, W};
    band_envelope<true>(line, out, sm, W, lg, NW);
}

cudaError_t launch_rows2d(int H, int W, const ColGeom& g, const ColScratch& s,
                          int32_t* D, int32_t* F, float* dist, int sm_count,
                          cudaStream_t stream)
{
    (void)sm_count;
    int max_nw = 32, lg = 0, NW = 0;
    for (; max_nw >= 1; max_nw >>= 1) {
        lg = band_seg_log2(W, max_nw);
        NW = (W + (1 << lg) - 1) >> lg;
        if (band2d_smem(W, lg, NW) <= 227 * 1024) break;
    }
    const size_t smem = band2d_smem(W, lg, NW);
    k_rows2d<<<(unsigned)g.nb, NW * 32, smem, stream>>>(H, W, s, lg, NW, D, F, dist);
    return cudaGetLastError();
}

// --- batched row pass -------------------------------------------------------

// Row-pass geometry of a batch job of width W: segments of 2^lg columns, NW
// warps per band, `groups` bands side by side in one 16-warp block.
void batch_row_geometry(int W, int& lg, int& NW, int& groups)
{
    lg = band_seg_log2(W, BATCH_K2_WARPS);
    NW = (W + (1 << lg) - 1) >> lg;
    groups = BATCH_K2_WARPS / NW;
}

__host__ __device__ static size_t batch_group_bytes(int W, int lg, int NW)
{
    return (((size_t)8 * W + 15) & ~size_t(15)) + band_smem_bytes(NW, (1 << lg) >> 5, true);
}

size_t batch_rows_smem()
{
    size_t mx = 0;
    for (int W = 1; W <= BATCH_MAX_W; ++W) {
        int lg, NW, groups;
        batch_row_geometry(W, lg, NW, groups);
        const size_t b = (size_t)groups * batch_group_bytes(W, lg, NW);
        if (b > mx) mx = b;
    }
    return mx;
}

// Barrier of one band engine inside a block that runs several: a warp barrier
// for one-warp engines, else a named barrier (ids 1..8; 0 is __syncthreads).
struct DynSync {
    int id, nthreads;
    __device__ __forceinline__ void operator()() const
    {
        if (nthreads <= 32) __syncwarp();
        else asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
    }
};

__global__ void __launch_bounds__(BATCH_K2_WARPS * 32, 2)
k_batch_rows2d(const BatchHeader* __restrict__ hdr, const BatchJob* __restrict__ jobs,
               unsigned* __restrict__ work)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_item;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t total = hdr->k2_total;
    const int nj = hdr->njobs;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(work, 1u);
        __syncthreads();
        const int64_t item = s_item;
        if (item >= total) break;
        int lo = 0, hi = nj - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].k2_first <= item) lo = mid; else hi = mid - 1;
        }
        const BatchJob& J = jobs[lo];
        const int W = (int)J.g.cols, H = J.g.rows, lg = J.lg, NW = J.NW;
        const int grp = warp / NW, wg = warp - grp * NW;
        const int b = (int)((item - J.k2_first) * J.groups) + grp;
        if (grp < J.groups && b < J.g.nb) {
            unsigned char* base = smem + (size_t)grp * batch_group_bytes(W, lg, NW);
            uint32_t* sbits = reinterpret_cast<uint32_t*>(base);
            uint32_t* supdn = sbits + W;
            const BandSmem sm = carve_band_smem(base + (((size_t)8 * W + 15) & ~size_t(15)), NW,
                                                (1 << lg) >> 5, true);
            const DynSync sync{1 + grp, NW * 32};
            const uint32_t* Cb = J.s.C + (int64_t)b * W;
            const uint32_t* Ub = J.s.U + (int64_t)b * W;
            const uint32_t* GABg = J.s.GAB + (int64_t)(b >> 5) * W;
            for (int j = wg * 32 + lane; j < W; j += NW * 32) {
                const uint32_t u = Ub[j];
                uint32_t up = u & 0xFFFFu, dn = u >> 16;
                if (up == (uint32_t)NONE16 || dn == (uint32_t)NONE16) {
                    const uint32_t gab = GABg[j];
                    if (up == (uint32_t)NONE16) up = gab & 0xFFFFu;
                    if (dn == (uint32_t)NONE16) dn = gab >> 16;
                }
                sbits[j] = Cb[j];
                supdn[j] = (up == (uint32_t)NONE16 ? UP_NONE : up) |
                           ((dn == (uint32_t)NONE16 ? DN_NONE : dn) << 16);
            }
            sync();
            BandRow2D line;
            line.bits = sbits;
            line.updn = supdn;
            line.base = b * 32;
            line.i = b * 32 + lane;
            line.W = W;
            line.mle = FULL >> (31 - lane);
            line.mge = FULL << lane;
            line.valid = line.i < H;
            const BandOut2D out{J.D, J.F, J.dist, b * 32, H, W};
            band_envelope<true>(line, out, sm, W, lg, NW, wg, sync);
        }
        __syncthreads();
    }
}

cudaError_t launch_batch_rows2d(const BatchHeader* hdr, const BatchJob* jobs, unsigned* work,
                                int blocks, cudaStream_t stream)
{
    k_batch_rows2d<<<blocks, BATCH_K2_WARPS * 32, batch_rows_smem(), stream>>>(hdr, jobs, work);
    return cudaGetLastError();
}

cudaError_t set_batch_attributes()
{
    return cudaFuncSetAttribute(k_batch_rows2d, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)batch_rows_smem());
}

int batch_rows_blocks_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_rows2d, BATCH_K2_WARPS * 32,
                                                      batch_rows_smem()) != cudaSuccess || n < 1)
        n = 1;
    return n;
}

cudaError_t set_2d_attributes()
{
    return cudaFuncSetAttribute(k_rows2d, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

}  // namespace edt
