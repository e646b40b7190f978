// Row pass of the 2-D exact EDT (Sec. 3.3.1 of Strutz, "The Distance
// Transform and its Computation": lower envelope of the parabolas of Eq. (5)
// per row), fused with the end of the column pass and the optional sqrt.
//
// One block handles rows of one band of 32 rows over the full width W.  Its
// prologue stages, per column, the band's source-bit word and the nearest
// source rows above and below the band (8 bytes per column, from the column
// pass scratch) in shared memory.  For any row of the band the nearest source
// row g of column k then follows from a few bit operations (highest set bit at
// or above the row, lowest at or below), i.e. the squared vertical distance
// D_v(k) = (i - g)^2 of Fig. 18(b) is rebuilt on demand and never stored.
// Each warp then runs the lower-envelope engine on one row at a time and
// writes D, F (= g * W + k of the owning parabola) and optionally sqrt(D).
#include "edt_engine.cuh"
#include "edt_internal.h"

namespace edt {

struct Row2D {
    int n;                       // W
    const uint32_t* bits;        // padded [W]: source bits of the band
    const uint32_t* updn;        // padded [W]: nearest source above | below << 16
    int lg;                      // log2 of the lane segment length
    int base;                    // first row of the band
    int r;                       // row within the band
    int W;

    __device__ __forceinline__ int nearest(int k) const
    {
        const int idx = pad_index(k, lg);
        const uint32_t ud = updn[idx];
        return nearest_in_column(bits[idx], base, r, (int)(ud & 0xFFFFu), (int)(ud >> 16));
    }
    __device__ __forceinline__ bool eval(int k, int& f) const
    {
        const int g = nearest(k);
        if (g < 0) return false;
        const int d = base + r - g;
        f = d * d;
        return true;
    }
    __device__ __forceinline__ int c(int k) const
    {
        const int d = base + r - nearest(k);
        return d * d + k * k;
    }
    __device__ __forceinline__ int feature(int k) const { return nearest(k) * W + k; }
};

struct Out2D {
    int32_t* D;
    int32_t* F;
    float* dist;
    int64_t rowoff;
    __device__ __forceinline__ void store(int j, int v, int f) const
    {
        const int64_t i = rowoff + j;
        if (D) D[i] = v;
        if (F) F[i] = f;
        if (dist) dist[i] = sqrt_rn_int(v);
    }
};

__global__ void __launch_bounds__(256)
k_rows2d(int H, int W, ColScratch s, int rows_per_cta, int cpb, int32_t* D,
         int32_t* F, float* dist)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lg = seg_log2(W);
    const int S = 1 << lg;
    const int SW = (S + 31) / 32;
    const int np = padded_len(W);
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    uint32_t* sbits = reinterpret_cast<uint32_t*>(smem);
    uint32_t* supdn = sbits + np;
    const int col_bytes = ((2 * np * 4) + 15) & ~15;
    const WarpSmem sm = carve_warp_smem(smem + col_bytes + warp * warp_smem_bytes(SW), SW);

    const int b = blockIdx.x / cpb;
    const int chunk = blockIdx.x % cpb;
    const int G = b >> 5;
    const uint32_t* Cb = s.C + (int64_t)b * W;
    const uint32_t* Ub = s.U + (int64_t)b * W;
    const uint32_t* GABg = s.GAB + (int64_t)G * W;
    for (int j = threadIdx.x; j < W; j += blockDim.x) {
        const uint32_t w = Cb[j];
        const uint32_t u = Ub[j];
        uint32_t up = u & 0xFFFFu, dn = u >> 16;
        if (up == (uint32_t)NONE16 || dn == (uint32_t)NONE16) {
            const uint32_t gab = GABg[j];
            if (up == (uint32_t)NONE16) up = gab & 0xFFFFu;
            if (dn == (uint32_t)NONE16) dn = gab >> 16;
        }
        const int idx = pad_index(j, lg);
        sbits[idx] = w;
        supdn[idx] = up | (dn << 16);
    }
    __syncthreads();

    const int rbeg = chunk * rows_per_cta;
    const int rend = min(rbeg + rows_per_cta, min(32, H - b * 32));
    for (int r = rbeg + warp; r < rend; r += nwarps) {
        const Row2D line{W, sbits, supdn, lg, b * 32, r, W};
        const Out2D out{D, F, dist, (int64_t)(b * 32 + r) * W};
        warp_envelope(line, out, sm);
        __syncwarp();
    }
}

cudaError_t launch_rows2d(int H, int W, const ColGeom& g, const ColScratch& s,
                          int32_t* D, int32_t* F, float* dist, int sm_count,
                          cudaStream_t stream)
{
    int cpb = 1;  // blocks per band
    while (cpb < 8 && (int64_t)g.nb * cpb < 2 * (int64_t)sm_count) cpb *= 2;
    const int rows_per_cta = 32 / cpb;
    const int nwarps = rows_per_cta < 8 ? rows_per_cta : 8;
    const int lg = seg_log2(W);
    const int SW = ((1 << lg) + 31) / 32;
    const int np = padded_len(W);
    const size_t smem = (((size_t)2 * np * 4 + 15) & ~size_t(15)) +
                        (size_t)nwarps * warp_smem_bytes(SW);
    const unsigned blocks = (unsigned)(g.nb * cpb);
    k_rows2d<<<blocks, nwarps * 32, smem, stream>>>(H, W, s, rows_per_cta, cpb, D, F, dist);
    return cudaGetLastError();
}

cudaError_t set_2d_attributes()
{
    return cudaFuncSetAttribute(k_rows2d, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

}  // namespace edt
