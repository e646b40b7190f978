// City-block distance transform (Sec. 2.1 of Strutz, "The Distance
// Transform and its Computation").  The paper's second algorithm scans every
// column down and up, then every row forward and backward; here the column
// scans are the column-bit kernel (nearest source row above / below every
// band, shared with the Euclidean transform), and the row scans become two
// prefix minima per row: with a(k) the vertical distance of the row's pixel
// in column k to the nearest source in that column,
//     d(j) = min_k a(k) + |j - k|
//          = min( j + min_{k<=j} (a(k) - k),  -j + min_{k>=j} (a(k) + k) ),
// so every row is one forward and one backward min-scan, data-parallel over
// the columns.  A block takes 8 rows of one band; its threads hold CPT
// consecutive columns each (their column words in registers), scan them,
// and combine the threads' partial minima through shared memory; each thread
// writes its CPT results as whole 32-byte sectors.
#include "edt_engine.cuh"
#include "edt_internal.h"

namespace edt {

constexpr int CB_ROWS = 8;                 // rows per block
constexpr int CB_BIG = 1 << 29;            // "no source in this column"

__device__ __forceinline__ int warp_incl_min(int v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v = min(v, u);
    }
    return v;
}
__device__ __forceinline__ int warp_incl_min_rev(int v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_down_sync(FULL, v, o);
        if (lane + o < 32) v = min(v, u);
    }
    return v;
}

template <int CPT>
__global__ void __launch_bounds__(1024)
k_cityblock_rows(int H, int W, ColScratch s, int32_t* __restrict__ D, int vec)
{
    __shared__ int sx[32], sy[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarp = blockDim.x >> 5;
    const int b = blockIdx.x >> 2;                      // band
    const int r0 = (blockIdx.x & 3) * CB_ROWS;          // first row of the block inside the band
    const int base = b * 32;
    const int c0 = t * CPT;
    // column data of this thread's columns: source bits of the band and the
    // nearest source rows above / below it
    uint32_t w[CPT];
    int up_out[CPT], dn_out[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        const int col = c0 + c;
        w[c] = 0u;
        up_out[c] = -CB_BIG;
        dn_out[c] = CB_BIG;
        if (col < W) {
            w[c] = s.C[(int64_t)b * W + col];
            const uint32_t u = s.U[(int64_t)b * W + col];
            uint32_t up = u & 0xFFFFu, dn = u >> 16;
            if (up == (uint32_t)NONE16 || dn == (uint32_t)NONE16) {
                const uint32_t gab = s.GAB[(int64_t)(b >> s.gs) * W + col];
                if (up == (uint32_t)NONE16) up = gab & 0xFFFFu;
                if (dn == (uint32_t)NONE16) dn = gab >> 16;
            }
            if (up != (uint32_t)NONE16) up_out[c] = (int)up;
            if (dn != (uint32_t)NONE16) dn_out[c] = (int)dn;
        }
    }
    for (int rr = 0; rr < CB_ROWS; ++rr) {
        const int r = r0 + rr, i = base + r;
        if (i >= H) break;                               // uniform over the block
        const uint32_t mle = FULL >> (31 - r), mge = FULL << r;
        int px[CPT], sy_[CPT];
        int run = CB_BIG;
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const uint32_t a_ = w[c] & mle, b_ = w[c] & mge;
            const int up = a_ ? base + 31 - __clz(a_) : up_out[c];
            const int dn = b_ ? base + __ffs(b_) - 1 : dn_out[c];
            const int a = min(min(i - up, dn - i), CB_BIG);
            const int col = c0 + c;
            run = min(run, a - col);
            px[c] = run;                                  // prefix min of a(k) - k within the thread
            sy_[c] = a + col;
        }
        int suf = CB_BIG;
#pragma unroll
        for (int c = CPT - 1; c >= 0; --c) {
            suf = min(suf, sy_[c]);
            sy_[c] = suf;                                 // suffix min of a(k) + k within the thread
        }
        // exclusive prefix (over lower threads) of the forward minima and
        // exclusive suffix (over higher threads) of the backward minima
        const int ix = warp_incl_min(run, lane), iy = warp_incl_min_rev(suf, lane);
        if (lane == 31) sx[warp] = ix;
        if (lane == 0) sy[warp] = iy;
        __syncthreads();
        if (warp == 0) {
            const int vx = lane < nwarp ? sx[lane] : CB_BIG;
            const int vy = lane < nwarp ? sy[lane] : CB_BIG;
            const int ex = warp_incl_min(vx, lane), ey = warp_incl_min_rev(vy, lane);
            sx[lane] = ex;
            sy[lane] = ey;
        }
        __syncthreads();
        int carry_x = __shfl_up_sync(FULL, ix, 1), carry_y = __shfl_down_sync(FULL, iy, 1);
        if (lane == 0) carry_x = CB_BIG;
        if (lane == 31) carry_y = CB_BIG;
        if (warp > 0) carry_x = min(carry_x, sx[warp - 1]);
        if (warp + 1 < nwarp) carry_y = min(carry_y, sy[warp + 1]);
        int v[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int col = c0 + c;
            const int d = min(col + min(carry_x, px[c]), -col + min(carry_y, sy_[c]));
            v[c] = d >= CB_BIG / 2 ? INT32_MAX : d;
        }
        int32_t* row = D + (int64_t)i * W;
        if (vec == 2 && c0 + CPT <= W) {
#pragma unroll
            for (int c = 0; c < CPT; c += 8)
                st_v8(row + c0 + c, v[c], v[c + 1], v[c + 2], v[c + 3], v[c + 4], v[c + 5], v[c + 6], v[c + 7]);
        } else {
#pragma unroll
            for (int c = 0; c < CPT; ++c)
                if (c0 + c < W) row[c0 + c] = v[c];
        }
        __syncthreads();                                  // sx / sy reused by the next row
    }
}

cudaError_t launch_cityblock_rows(int H, int W, const ColGeom& g, const ColScratch& s, int32_t* D,
                                  cudaStream_t stream)
{
    const int vec = (W % 8 == 0 && (reinterpret_cast<uintptr_t>(D) & 31) == 0) ? 2 : 0;
    const unsigned blocks = (unsigned)(g.nb * 4);
    if (W <= 8 * 1024) {
        const int threads = ((W + 8 - 1) / 8 + 31) & ~31;
        k_cityblock_rows<8><<<blocks, threads, 0, stream>>>(H, W, s, D, vec);
    } else {
        const int threads = ((W + 16 - 1) / 16 + 31) & ~31;
        k_cityblock_rows<16><<<blocks, threads, 0, stream>>>(H, W, s, D, vec);
    }
    return cudaGetLastError();
}

}  // namespace edt
