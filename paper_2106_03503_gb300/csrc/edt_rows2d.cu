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
// Bands of rows up to DIRECT_ROW_W wide first try an exact direct search
// (rows2d_direct: lanes on 32 consecutive columns of one row, giving up past
// DIRECT_ROW_CAP columns; in the batch rows2d_direct_patches: lanes on 4 rows
// x 8 columns, giving up past PATCH_ROW_CAP); a band in which some search
// gives up falls back to the band engine, which gives the same bits.
#include "edt_engine.cuh"
#include "edt_internal.h"

#include <cstring>

namespace edt {

// Encoded nearest source rows outside the band: up as int16 (-32768 = none),
// dn as uint16 (65535 = none), so that i - up and dn - i exceed any real
// distance (< 32768) when there is no source on that side.
constexpr uint32_t UP_NONE = 0x8000u;
constexpr uint32_t DN_NONE = 0xFFFFu;

struct BandRow2D {
    const uint32_t* bits;   // [W]: source bits of the band's 32 rows
    const uint32_t* updn;   // [W]: encoded up | dn << 16 (shared or global memory)
    int base;               // first row of the band
    int i;                  // this lane's row
    int W;
    uint32_t mle, mge;      // bits at / above and at / below this row
    uint32_t rbit;          // this row's bit
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
    __device__ __forceinline__ bool eval2(int k, int& f, int& g) const
    {
        int up, dn;
        if (!parts(k, up, dn)) return false;
        const int du = i - up, dd = dn - i;
        const int d = min(du, dd);
        if (d >= 32768) return false;
        f = d * d;
        g = ((du <= dd) ? up : dn) * W + k;
        return true;
    }
    __device__ __forceinline__ bool is_zero(int k) const { return (bits[k] & rbit) != 0u; }
    __device__ __forceinline__ bool chunk_has_source(int j0) const
    {
        // j0 is a multiple of 8 and bits 16-byte aligned
        const uint4 a = *reinterpret_cast<const uint4*>(bits + j0);
        const uint4 b = *reinterpret_cast<const uint4*>(bits + j0 + 4);
        return ((a.x | a.y | a.z | a.w | b.x | b.y | b.z | b.w) & rbit) != 0u;
    }
    __device__ __forceinline__ int self_feature(int k) const { return i * W + k; }
};

// Shared memory of one band block: column data (8 B per column), one flag per
// 32 columns (all 32 rows are sources there), then the band engine.
__host__ __device__ inline size_t band2d_col_bytes(int W)
{
    return (((size_t)8 * W + (size_t)(W + 31) / 32 + 15) & ~size_t(15));
}
// Direct row pass (rows2d_direct): rows up to DIRECT_ROW_W wide, one row's
// vertical offsets per warp in shared memory with DPAD entries of pad on both
// sides, searches give up after DIRECT_ROW_CAP columns.  OFF_NONE marks a
// column (or pad) without source: its cost 32767^2 exceeds that of any real
// candidate (offsets are at most 32766, searches at most DPAD long).
constexpr int DIRECT_ROW_W = 1024;
constexpr int DIRECT_ROW_CAP = 32;
constexpr int DPAD = DIRECT_ROW_CAP + 2;
constexpr short OFF_NONE = 32767;

__host__ __device__ inline size_t direct_row_bytes(int W, int NW)
{
    return W <= DIRECT_ROW_W ? (((size_t)NW * (W + 2 * DPAD) * 2 + 15) & ~size_t(15)) : 0;
}
// this warp's row of offsets (entry 0 = column 0; pads before and after)
__device__ __forceinline__ short* direct_rowbuf(void* base, int warp, int W)
{
    return reinterpret_cast<short*>(base) + (size_t)warp * (W + 2 * DPAD) + DPAD;
}

static size_t band2d_smem(int W, int lg, int NW)
{
    return band2d_col_bytes(W) + band_smem_bytes(NW, (1 << lg) >> 5) + direct_row_bytes(W, NW);
}

// Stage the band's column data: source word, encoded nearest source rows
// above / below, and the per-32-column "all rows are sources" flags.  Called
// by `nthreads` threads (a multiple of 32) with index tid.
__device__ __forceinline__ void stage_band(const ColScratch& s, int b, int H, int W, uint32_t* sbits,
                                           uint32_t* supdn, unsigned char* sfull, int tid, int nthreads,
                                           bool invert = false)
{
    const uint32_t* Cb = s.C + (int64_t)b * W;
    const uint32_t* Ub = s.U + (int64_t)b * W;
    const uint32_t* GABg = s.GAB + (int64_t)(b >> s.gs) * W;
    const int rows = min(32, H - b * 32);
    const uint32_t invalid = rows >= 32 ? 0u : (FULL << rows);
    const int Wr = (W + 31) & ~31;
    for (int j = tid; j < Wr; j += nthreads) {
        uint32_t w = 0u;
        if (j < W) {
            w = Cb[j];
            if (invert) w = ~w & ~invalid;   // the other class, rows inside the image
            const uint32_t u = Ub[j];
            uint32_t up = u & 0xFFFFu, dn = u >> 16;
            if (up == (uint32_t)NONE16 || dn == (uint32_t)NONE16) {
                const uint32_t gab = GABg[j];
                if (up == (uint32_t)NONE16) up = gab & 0xFFFFu;
                if (dn == (uint32_t)NONE16) dn = gab >> 16;
            }
            sbits[j] = w;
            supdn[j] = (up == (uint32_t)NONE16 ? UP_NONE : up) | ((dn == (uint32_t)NONE16 ? DN_NONE : dn) << 16);
            w |= invalid;
        }
        const uint32_t all = __reduce_and_sync(FULL, w);
        if ((j & 31) == 0) sfull[j >> 5] = (all == FULL) ? 1 : 0;
    }
}

// Direct row pass of band b (32 rows), for narrow rows: every pixel takes the
// minimum of Eq. (5) over the columns k of its row, D_v(k) + (j - k)^2, by an
// outward search from j that stops once r^2 reaches the best value found (the
// same exact search as band_direct), keeping the rightmost k at a tie, the
// hull walk's choice.  Here the lanes take 32 consecutive columns of one row:
// each warp first writes its row's vertical offsets (nearest source row minus
// the row, int16) into `rowbuf` from the staged column words, then searches
// and writes whole 128-byte lines of D, F and dist.  A search that reaches
// DIRECT_ROW_CAP columns with candidates left gives up for the whole band
// (abort flag): the caller then runs the hull engine, which rewrites every
// pixel with the same value.  Only the band's rows rlo .. rhi - 1 are done.
// Called by the nthr threads of one engine, which must have cleared *abort
// before their last barrier; returns true when those rows are done (the same
// answer in every thread).
template <class Sync>
__device__ bool rows2d_direct(const uint32_t* sbits, const uint32_t* supdn, int b, int H, int W, int32_t* D,
                              int32_t* F, float* dist, short* rowbuf, volatile int* abort, int lane, int warp,
                              int NW, Sync sync, int rlo = 0, int rhi = 32)
{
    const int base = b * 32, rows = min(rhi, H - base);
    for (int t = lane; t < DPAD; t += 32) {   // the pads: no source beyond the row's ends
        rowbuf[-1 - t] = OFF_NONE;
        rowbuf[W + t] = OFF_NONE;
    }
    for (int r = rlo + warp; r < rows; r += NW) {
        if (*abort) break;
        const int i = base + r;
        const uint32_t mle = FULL >> (31 - r), mge = FULL << r;
        for (int k = lane; k < W; k += 32) {
            const uint32_t w = sbits[k], ud = supdn[k];
            const uint32_t a = w & mle, bb = w & mge;
            const int up = a ? base + 31 - __clz(a) : (int)(short)(ud & 0xFFFFu);
            const int dn = bb ? base + __ffs(bb) - 1 : (int)(ud >> 16);
            const int du = i - up, dd = dn - i;
            rowbuf[k] = min(du, dd) >= 32768 ? OFF_NONE : (short)(du <= dd ? up - i : dn - i);
        }
        __syncwarp();
        bool gave_up = false;
        for (int c0 = 0; c0 < W; c0 += 32) {
            const int j = c0 + lane;
            bool unsettled = false;
            if (j < W) {
                // two steps per test of the stop rule (a step past the stop
                // costs at least its r^2, more than the best, and changes
                // nothing); the pads make bounds tests unneeded
                const int o = rowbuf[j];
                int best = o * o, bk = j;
                int rr = 1;
                for (int r2 = 1; rr <= DIRECT_ROW_CAP && r2 <= best; rr += 2, r2 += 4 * rr - 4) {
                    const int r2b = r2 + 2 * rr + 1;
                    const int ol = rowbuf[j - rr], orr = rowbuf[j + rr];
                    const int ol2 = rowbuf[j - rr - 1], orr2 = rowbuf[j + rr + 1];
                    const int cl = ol * ol + r2, cr = orr * orr + r2;
                    const int cl2 = ol2 * ol2 + r2b, cr2 = orr2 * orr2 + r2b;
                    if (cl < best) { best = cl; bk = j - rr; }
                    if (cr <= best) { best = cr; bk = j + rr; }
                    if (cl2 < best) { best = cl2; bk = j - rr - 1; }
                    if (cr2 <= best) { best = cr2; bk = j + rr + 1; }
                }
                // rr: the nearest distance not searched
                unsettled = rr * rr <= best && (j - rr >= 0 || j + rr < W);
                if (!unsettled) {
                    const int ob = rowbuf[bk];
                    const bool none = ob == OFF_NONE;   // the whole row has no source
                    const int64_t q = (int64_t)i * W + j;
                    const int v = none ? INT32_MAX : best;
                    if (D) D[q] = v;
                    if (F) F[q] = none ? -1 : (i + ob) * W + bk;
                    if (dist) dist[q] = sqrt_rn_int(v);
                }
            }
            if (__any_sync(FULL, unsettled)) {
                gave_up = true;
                break;
            }
        }
        __syncwarp();
        if (gave_up) {
            *abort = 1;
            break;
        }
    }
    sync();
    return *abort == 0;
}

// Direct row pass of band b on 4 x 8 patches (the batch's bands): the same
// exact search as rows2d_direct, but each warp takes 4 rows of the band at a
// time and its lanes a patch of 4 rows x 8 consecutive columns, so that the
// lanes of a warp, whose searches run as long as the farthest one, hold
// nearer distances than 32 columns of one row do.  The 4 rows' vertical
// offsets are int8: PATCH_NONE (-128) for a column without source, the
// others clamped to +-127.  A clamped or missing value costs at least 127^2,
// and never more than the true cost, so a search whose best is below 127^2
// chose an exact value and no clamped one could beat it; a best of 127^2 or
// more gives up (as a search still open at PATCH_ROW_CAP does).  Warp w's
// buffer is 4 rows of patch_pitch(W) bytes at buf + 4 w patch_pitch(W), each
// with PPAD bytes of pad (PATCH_NONE) before column 0 and after column W - 1;
// the pitch is 32 mod 128 bytes, so the 4 rows of a patch fall on disjoint
// banks.  Called and returning as rows2d_direct (all of the band's rows).
// The patch search stops at PATCH_ROW_CAP columns, further than the row-wise
// search: a patch's lanes hold more alike distances, so searching on costs
// less than handing the band to the hull engine.
constexpr int PATCH_NONE = -128;
constexpr int PATCH_ROW_CAP = 48;
constexpr int PPAD = PATCH_ROW_CAP + 2;
__host__ __device__ inline int patch_pitch(int W) { return ((W + 2 * PPAD + 127) & ~127) + 32; }
__host__ __device__ inline size_t patch_buf_bytes(int W, int NW)
{
    return W <= DIRECT_ROW_W ? (size_t)NW * 4 * patch_pitch(W) : 0;
}

template <class Sync>
__device__ bool rows2d_direct_patches(const uint32_t* sbits, const uint32_t* supdn, int b, int H, int W,
                                      int32_t* D, int32_t* F, float* dist, int8_t* buf, volatile int* abort,
                                      int lane, int warp, int NW, Sync sync)
{
    const int base = b * 32, rows = min(32, H - base), P = patch_pitch(W);
    int8_t* qb = buf + (size_t)warp * 4 * P + PPAD;   // row 0, column 0 of this warp's 4 rows
    for (int t = lane; t < 4 * PPAD; t += 32) {        // the pads: no source beyond the rows' ends
        const int rr = t / PPAD, e = t - rr * PPAD;
        qb[rr * P - 1 - e] = (int8_t)PATCH_NONE;
        qb[rr * P + W + e] = (int8_t)PATCH_NONE;
    }
    const int nq = (rows + 3) >> 2, nj = (W + 7) >> 3;
    const int8_t* rb = qb + (lane >> 3) * P;            // this lane's row of a patch
    for (int q = warp; q < nq; q += NW) {
        if (__any_sync(FULL, *abort != 0)) break;      // the same decision in every lane
        for (int rr = 0; rr < 4 && 4 * q + rr < rows; ++rr) {
            const int r = 4 * q + rr, i = base + r;
            const uint32_t mle = FULL >> (31 - r), mge = FULL << r;
            for (int k = lane; k < W; k += 32) {
                const uint32_t w = sbits[k], ud = supdn[k];
                const uint32_t a = w & mle, bb = w & mge;
                const int up = a ? base + 31 - __clz(a) : (int)(short)(ud & 0xFFFFu);
                const int dn = bb ? base + __ffs(bb) - 1 : (int)(ud >> 16);
                const int du = i - up, dd = dn - i;
                const int o = min(du, dd) >= 32768 ? PATCH_NONE : max(-127, min(127, du <= dd ? up - i : dn - i));
                qb[rr * P + k] = (int8_t)o;
            }
        }
        __syncwarp();
        const int r = 4 * q + (lane >> 3), i = base + r;
        bool gave_up = false;
        for (int jb = 0; jb < nj; ++jb) {
            const int j = 8 * jb + (lane & 7);
            bool unsettled = false;
            if (r < rows && j < W) {
                // two steps per test of the stop rule; the pads make bounds
                // tests unneeded
                const int o = rb[j];
                int best = o * o, bk = j;
                int rr = 1;
                for (int r2 = 1; rr <= PATCH_ROW_CAP && r2 <= best; rr += 2, r2 += 4 * rr - 4) {
                    const int r2b = r2 + 2 * rr + 1;
                    const int ol = rb[j - rr], orr = rb[j + rr];
                    const int ol2 = rb[j - rr - 1], orr2 = rb[j + rr + 1];
                    const int cl = ol * ol + r2, cr = orr * orr + r2;
                    const int cl2 = ol2 * ol2 + r2b, cr2 = orr2 * orr2 + r2b;
                    if (cl < best) { best = cl; bk = j - rr; }
                    if (cr <= best) { best = cr; bk = j + rr; }
                    if (cl2 < best) { best = cl2; bk = j - rr - 1; }
                    if (cr2 <= best) { best = cr2; bk = j + rr + 1; }
                }
                // rr: the nearest distance not searched
                unsettled = best >= 127 * 127 || (rr * rr <= best && (j - rr >= 0 || j + rr < W));
                if (!unsettled) {
                    const int ob = rb[bk];   // exact: |ob| <= 126
                    const int64_t qq = (int64_t)i * W + j;
                    if (D) D[qq] = best;
                    if (F) F[qq] = (i + ob) * W + bk;
                    if (dist) dist[qq] = sqrt_rn_int(best);
                }
            }
            if (__any_sync(FULL, unsettled)) {
                gave_up = true;
                break;
            }
        }
        __syncwarp();
        if (gave_up) {
            *abort = 1;
            break;
        }
    }
    sync();
    return *abort == 0;
}

// Tensor maps for TMA row stores: the output viewed as [rows][W] with an
// 8 x 32 box (8 columns, 32 rows).  Needs W % 4 == 0 (16-byte row pitch) and a
// 16-byte aligned base.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

bool make_row_map(CUtensorMap* m, void* base, bool is_float, int64_t rows, int W)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc || !base || W % 4 != 0 || W < OC || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)W * 4};
    const cuuint32_t box[2] = {(cuuint32_t)OC, 32};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, is_float ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_INT32, 2, base,
               dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Staging per warp for TMA stores: 3 arrays x 32 rows x 8 columns.
constexpr size_t TMA_STAGE_BYTES = 3 * 32 * OC * 4;

// One transform of the row kernel: its column-pass scratch, whether its
// sources are the complement of the stored column words, and its outputs.
struct RowJob {
    ColScratch s;
    int invert;
    int32_t* D;
    int32_t* F;
    float* dist;
};

// One block per band of 32 rows, bands band0 .. band0 + nbl - 1: blocks
// [0, nbl) run job 0, blocks [nbl, 2 nbl) job 1 (when two transforms of one
// mask are fused).  NARROW (rows up to DIRECT_ROW_W): the direct row pass
// first, the hull engine only for bands it gives up on; wider rows are
// compiled without it.
template <bool TMA, bool NARROW>
__global__ void __launch_bounds__(512, 2)
k_rows2d(int H, int W, int band0, int nbl, RowJob J0, RowJob J1, int lg, int NW, int split,
         const __grid_constant__ CUtensorMap mD0, const __grid_constant__ CUtensorMap mF0,
         const __grid_constant__ CUtensorMap mS0, const __grid_constant__ CUtensorMap mD1,
         const __grid_constant__ CUtensorMap mF1, const __grid_constant__ CUtensorMap mS1)
{
    extern __shared__ __align__(128) unsigned char smem[];
    uint32_t* sbits = reinterpret_cast<uint32_t*>(smem);
    uint32_t* supdn = sbits + W;
    unsigned char* sfull = reinterpret_cast<unsigned char*>(supdn + W);
    // TMA staging starts on a 128-byte boundary (the launch adds 128 bytes
    // of room for that); without TMA the engine follows the column data
    unsigned char* stage0 = smem + band2d_col_bytes(W);
    if (TMA) stage0 = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(stage0) + 127) & ~uintptr_t(127));
    const BandSmem sm = carve_band_smem(stage0 + (TMA ? NW * TMA_STAGE_BYTES : 0), NW, (1 << lg) >> 5);
    // `split` blocks share a band (small images: more blocks than bands),
    // block `part` of them doing rows part * 32 / split onwards
    const int bi = (int)blockIdx.x / split, part = (int)blockIdx.x - bi * split;
    const int rlo = part * (32 / split), rhi = rlo + 32 / split;
    const bool second = bi >= nbl;
    const RowJob& J = second ? J1 : J0;
    const int b = band0 + (second ? bi - nbl : bi);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    if constexpr (NARROW) {
        __shared__ int s_abort;
        if (threadIdx.x == 0) s_abort = 0;
        stage_band(J.s, b, H, W, sbits, supdn, sfull, threadIdx.x, blockDim.x, J.invert != 0);
        __syncthreads();
        // narrow rows: the direct search, unless some pixel's answer is far
        short* rowbuf = direct_rowbuf(reinterpret_cast<unsigned char*>(sm.ctr) + 16, warp, W);
        if (rows2d_direct(sbits, supdn, b, H, W, J.D, J.F, J.dist, rowbuf, &s_abort, lane, warp, NW, BlockSync(),
                          rlo, rhi))
            return;
        // the TMA stores below must land after the plain stores above
        if (TMA) asm volatile("fence.proxy.async.global;" ::: "memory");
    } else {
        stage_band(J.s, b, H, W, sbits, supdn, sfull, threadIdx.x, blockDim.x, J.invert != 0);
        __syncthreads();
    }
    BandRow2D line;
    line.bits = sbits;
    line.updn = supdn;
    line.base = b * 32;
    line.i = b * 32 + lane;
    line.W = W;
    line.mle = FULL >> (31 - lane);
    line.mge = FULL << lane;
    line.rbit = 1u << lane;
    line.valid = line.i < H;
    if (TMA) {
        const TmaRowOut out{J.D ? (second ? &mD1 : &mD0) : nullptr, J.F ? (second ? &mF1 : &mF0) : nullptr,
                            J.dist ? (second ? &mS1 : &mS0) : nullptr,
                            reinterpret_cast<int*>(stage0 + warp * TMA_STAGE_BYTES), b * 32, lane};
        band_envelope(line, out, sm, W, lg, NW, sfull);
    } else {
        const int vec = row_vec_width(W, J.D, J.F, J.dist);
        // with a split band, this block writes its own rows only
        const RowOut out{J.D, J.F, J.dist, (int64_t)line.i * W, line.valid && lane >= rlo && lane < rhi, vec};
        band_envelope(line, out, sm, W, lg, NW, sfull);
    }
}

// Row pass over bands [band0, band0 + nbl) for one transform (J1 unused) or
// two transforms of one mask.
static cudaError_t launch_rows(int H, int W, const RowJob& J0, const RowJob* J1, int band0, int nbl,
                               cudaStream_t stream)
{
    CUtensorMap m[6];
    memset(m, 0, sizeof(m));
    const RowJob* jobs[2] = {&J0, J1};
    // TMA stores where the shared memory still allows two blocks per SM
    // (widths up to 2048); per-lane 32-byte stores otherwise
    bool tma = W <= 2048;
    for (int k = 0; k < 2 && tma; ++k) {
        if (!jobs[k]) continue;
        if (jobs[k]->D) tma = tma && make_row_map(&m[3 * k + 0], jobs[k]->D, false, H, W);
        if (jobs[k]->F) tma = tma && make_row_map(&m[3 * k + 1], jobs[k]->F, false, H, W);
        if (jobs[k]->dist) tma = tma && make_row_map(&m[3 * k + 2], jobs[k]->dist, true, H, W);
    }
    const int shape2[2] = {H, W};
    const Tuning tu = tuning_lookup(2, shape2);
    int max_nw = tu.rows2d_nw > 0 ? tu.rows2d_nw : 16, lg = 0, NW = 0;
    size_t smem = 0;
    for (; max_nw >= 1; max_nw >>= 1) {
        lg = band_seg_log2(W, max_nw);
        NW = (W + (1 << lg) - 1) >> lg;
        smem = band2d_smem(W, lg, NW) + (tma ? NW * TMA_STAGE_BYTES + 128 : 0);
        if (smem <= 227 * 1024 - 64) break;   // room for the static shared flag
    }
    if (nbl <= 0) return cudaSuccess;
    const RowJob j1 = J1 ? *J1 : J0;
    const bool narrow = W <= DIRECT_ROW_W;
    // a small image's few bands are split over up to 4 blocks each (rows of a
    // band divided among them, plain stores), so that more SMs share the work
    int split = 1;
    const int bands = nbl * (J1 ? 2 : 1);
    if (narrow && device_sm_count() >= 2 * bands) {
        split = min(4, device_sm_count() / bands);
        split = split >= 4 ? 4 : (split >= 2 ? 2 : 1);
        tma = false;
    }
    const unsigned blocks = (unsigned)(bands * split);
    if (tma && narrow)
        k_rows2d<true, true><<<blocks, NW * 32, smem, stream>>>(H, W, band0, nbl, J0, j1, lg, NW, split, m[0],
                                                                m[1], m[2], m[3], m[4], m[5]);
    else if (tma)
        k_rows2d<true, false><<<blocks, NW * 32, smem, stream>>>(H, W, band0, nbl, J0, j1, lg, NW, split, m[0],
                                                                 m[1], m[2], m[3], m[4], m[5]);
    else if (narrow)
        k_rows2d<false, true><<<blocks, NW * 32, smem, stream>>>(H, W, band0, nbl, J0, j1, lg, NW, split, m[0],
                                                                 m[1], m[2], m[3], m[4], m[5]);
    else
        k_rows2d<false, false><<<blocks, NW * 32, smem, stream>>>(H, W, band0, nbl, J0, j1, lg, NW, split, m[0],
                                                                  m[1], m[2], m[3], m[4], m[5]);
    return cudaGetLastError();
}

cudaError_t launch_rows2d(int H, int W, const ColGeom& g, const ColScratch& s,
                          int32_t* D, int32_t* F, float* dist, int sm_count,
                          cudaStream_t stream, int band0, int nbl)
{
    (void)sm_count;
    const RowJob J{s, 0, D, F, dist};
    return launch_rows(H, W, J, nullptr, band0, nbl < 0 ? g.nb - band0 : nbl, stream);
}

cudaError_t launch_rows2d_pair(int H, int W, const ColGeom& g, const ColScratch& s_obj,
                               const ColScratch& s_bg, int32_t* D_obj, int32_t* F_obj,
                               int32_t* D_bg, int32_t* F_bg, cudaStream_t stream, int band0, int nbl)
{
    ColScratch sb = s_bg;
    sb.C = s_obj.C;   // the to-background sources are the complement of these words
    const RowJob J0{s_obj, 0, D_obj, F_obj, nullptr};
    const RowJob J1{sb, 1, D_bg, F_bg, nullptr};
    return launch_rows(H, W, J0, &J1, band0, nbl < 0 ? g.nb - band0 : nbl, stream);
}

// --- batched row pass -------------------------------------------------------

// Row-pass geometry of a batch job of width W <= BATCH_MAX_W: segments of
// 2^lg columns (at least 2^lgmin, built-in 2^8: narrow images get fewer warps
// per band and more bands per block instead of many short segments to merge),
// NW warps per band, `groups` bands side by side in one 16-warp block.
void batch_row_geometry(int W, int lgmin, int& lg, int& NW, int& groups)
{
    lg = band_seg_log2(W, BATCH_K2_WARPS);
    const int lo = lgmin > 0 ? lgmin : 8;
    if (lg < lo) lg = lo;
    NW = (W + (1 << lg) - 1) >> lg;
    groups = BATCH_K2_WARPS / NW;
}

// A batch band's shared memory: its column data, then the band engine, whose
// memory the direct search's patch buffers use first (the engine runs after
// the search, past a barrier, only on a band the search gave up).
__host__ __device__ static size_t batch_group_bytes(int W, int lg, int NW)
{
    const size_t eng = band_smem_bytes(NW, (1 << lg) >> 5), pb = patch_buf_bytes(W, NW);
    return band2d_col_bytes(W) + (eng > pb ? eng : pb);
}

// Segment minimums the autotuner may choose for the rows2d phase (the
// kernel's shared memory covers every one of them).
static const int kRowsLgmin[] = {6, 7, 8};

size_t batch_rows_smem()
{
    size_t mx = 0;
    for (int lgmin : kRowsLgmin)
        for (int W = 1; W <= BATCH_MAX_W; ++W) {
            int lg, NW, groups;
            batch_row_geometry(W, lgmin, lg, NW, groups);
            const size_t b = (size_t)groups * batch_group_bytes(W, lg, NW);
            if (b > mx) mx = b;
        }
    return mx;
}

// Rows wider than BATCH_MAX_W: one band per block, up to 16 warps.
size_t batch_wide_smem()
{
    const int W = 16384;
    const int lg = band_seg_log2(W, BATCH_K2_WARPS);
    return batch_group_bytes(W, lg, (W + (1 << lg) - 1) >> lg);
}

// Persistent row pass of phase PH (PH_ROWS: 2-D jobs up to BATCH_MAX_W wide,
// `groups` bands per work item; PH_WIDE: wider rows, one band per item).
template <int PH>
__global__ void __launch_bounds__(BATCH_K2_WARPS * 32, PH == PH_ROWS ? 2 : 1)
k_batch_rows2d(const BatchHeader* __restrict__ hdr, const BatchJob* __restrict__ jobs)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_item;
    __shared__ int s_abort[BATCH_K2_WARPS];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t total = hdr->k_total[PH];
    unsigned* work = hdr->cnt + PH;
    const int nj = hdr->njobs;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(work, 1u);
        __syncthreads();
        const int64_t item = s_item;
        if (item >= total) break;
        int lo = 0, hi = nj - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].k_first[PH] <= item) lo = mid; else hi = mid - 1;
        }
        const BatchJob& J = jobs[lo];
        const int W = J.W, H = J.H, lg = J.lg, NW = J.NW;
        const int grp = warp / NW, wg = warp - grp * NW;
        const int b = (int)((item - J.k_first[PH]) * J.groups) + grp;
        if (grp < J.groups && b < J.g.nb) {
            unsigned char* base = smem + (size_t)grp * batch_group_bytes(W, lg, NW);
            uint32_t* sbits = reinterpret_cast<uint32_t*>(base);
            uint32_t* supdn = sbits + W;
            unsigned char* sfull = reinterpret_cast<unsigned char*>(supdn + W);
            const BandSmem sm = carve_band_smem(base + band2d_col_bytes(W), NW, (1 << lg) >> 5);
            const GroupSync sync{1 + grp, NW * 32};
            if (wg == 0 && lane == 0) s_abort[grp] = 0;
            stage_band(J.s, b, H, W, sbits, supdn, sfull, wg * 32 + lane, NW * 32);
            sync();
            bool done = false;
            if (W <= DIRECT_ROW_W)
                done = rows2d_direct_patches(sbits, supdn, b, H, W, J.D, J.F, J.dist,
                                             reinterpret_cast<int8_t*>(sm.hb), &s_abort[grp], lane, wg, NW, sync);
            BandRow2D line;
            line.bits = sbits;
            line.updn = supdn;
            line.base = b * 32;
            line.i = b * 32 + lane;
            line.W = W;
            line.mle = FULL >> (31 - lane);
            line.mge = FULL << lane;
            line.rbit = 1u << lane;
            line.valid = line.i < H;
            const int vec = row_vec_width(W, J.D, J.F, J.dist);
            const RowOut out{J.D, J.F, J.dist, (int64_t)line.i * W, line.valid, vec};
            if (!done) band_envelope(line, out, sm, W, lg, NW, sfull, wg, sync);
        }
        __syncthreads();
    }
}

cudaError_t launch_batch_rows2d(const BatchHeader* hdr, const BatchJob* jobs, int blocks, cudaStream_t stream)
{
    k_batch_rows2d<PH_ROWS><<<blocks, BATCH_K2_WARPS * 32, batch_rows_smem(), stream>>>(hdr, jobs);
    return cudaGetLastError();
}

cudaError_t launch_batch_wide(const BatchHeader* hdr, const BatchJob* jobs, int blocks, cudaStream_t stream)
{
    k_batch_rows2d<PH_WIDE><<<blocks, BATCH_K2_WARPS * 32, batch_wide_smem(), stream>>>(hdr, jobs);
    return cudaGetLastError();
}

cudaError_t set_batch_row_attributes()
{
    cudaError_t e = cudaFuncSetAttribute(k_batch_rows2d<PH_ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)batch_rows_smem());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_batch_rows2d<PH_WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)batch_wide_smem());
}

int batch_rows_blocks_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_rows2d<PH_ROWS>, BATCH_K2_WARPS * 32,
                                                      batch_rows_smem()) != cudaSuccess || n < 1)
        n = 1;
    return n;
}

int batch_wide_blocks_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_rows2d<PH_WIDE>, BATCH_K2_WARPS * 32,
                                                      batch_wide_smem()) != cudaSuccess || n < 1)
        n = 1;
    return n;
}

// Opt a kernel in to all the dynamic shared memory a block may have beside
// its static shared memory (227 KB per block in all).
template <class K>
static cudaError_t allow_max_dynamic_smem(K kernel)
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(227 * 1024 - a.sharedSizeBytes));
}

cudaError_t set_2d_attributes()
{
    cudaError_t e = allow_max_dynamic_smem(k_rows2d<true, true>);
    if (e == cudaSuccess) e = allow_max_dynamic_smem(k_rows2d<true, false>);
    if (e == cudaSuccess) e = allow_max_dynamic_smem(k_rows2d<false, true>);
    if (e == cudaSuccess) e = allow_max_dynamic_smem(k_rows2d<false, false>);
    return e;
}

}  // namespace edt
