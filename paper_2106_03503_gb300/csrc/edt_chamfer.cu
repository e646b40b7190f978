// Chamfer 4-3 distance transform (Sec. 2.2 of Strutz, "The Distance
// Transform and its Computation"): the cost of the cheapest path from the
// nearest source when a horizontal or vertical step costs 3 and a diagonal
// step 4, i.e. min over sources of 3 max(|dx|, |dy|) + min(|dx|, |dy|) -- the
// result of the paper's two raster scans.
//
// The raster scans are sequential; here the transform is split into passes
// that are data-parallel.  A cheapest path can always be ordered as its
// diagonal steps first and its straight steps after, and its straight steps
// are all horizontal or all vertical.  So with
//   E(r) = 4 x (number of diagonal steps from r to the nearest source on
//          either diagonal through r),
//   d(p) = min( min_{r in the row of p} E(r) + 3 |r - p|,
//               min_{r in the column of p} E(r) + 3 |r - p| ),
// where every candidate is the cost of a real path and the cheapest path is
// among them.  Passes:
//   (1) k_shear copies the sources into two sheared images (H x SW bytes):
//       the column v of the first is the diagonal j - i = v - (H - 1), the
//       column u of the second the anti-diagonal i + j = u;
//   (2) the column-bit kernel of the Euclidean transform runs on each, giving
//       the nearest source along every diagonal;
//   (3) k_chamfer_rows computes E for 8 rows per block (threads = columns)
//       and the row term as two prefix minima (as in the city-block pass,
//       weight 3), writing the row term to D and E to a scratch image;
//   (4) k_chamfer_cols_totals and k_chamfer_cols take the column term over
//       chunks of 128 rows (chunk minima first, then each chunk with the
//       minima of the chunks above and below it) and lower D to it.
#include "edt_engine.cuh"
#include "edt_internal.h"

namespace edt {

constexpr int CH_ROWS = 8;            // rows per block of the row kernel
constexpr int CH_BIG = 1 << 29;       // no source
constexpr int CH_CHUNK = 128;         // rows per chunk of the column kernels

size_t chamfer_sheared_width(int H, int W) { return ((size_t)W + H - 1 + 31) & ~size_t(31); }

// (1) 4 bytes of both sheared images per thread; 1 = source.
__global__ void k_shear(const uint8_t* __restrict__ mask, int H, int W, int SW, int mode,
                        uint8_t* __restrict__ Sd, uint8_t* __restrict__ Sa)
{
    const int64_t quads = (int64_t)H * (SW / 4);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < quads;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q / (SW / 4));
        const int v0 = (int)(q - (int64_t)i * (SW / 4)) * 4;
        uint32_t d = 0u, a = 0u;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int jd = v0 + t + i - (H - 1);      // diagonal j - i = v - (H - 1)
            const int ja = v0 + t - i;                // anti-diagonal i + j = u
            if (jd >= 0 && jd < W) {
                const uint8_t m = mask[(int64_t)i * W + jd];
                d |= (uint32_t)((mode == 0) ? (m != 0) : (m == 0)) << (8 * t);
            }
            if (ja >= 0 && ja < W) {
                const uint8_t m = mask[(int64_t)i * W + ja];
                a |= (uint32_t)((mode == 0) ? (m != 0) : (m == 0)) << (8 * t);
            }
        }
        *reinterpret_cast<uint32_t*>(Sd + (int64_t)i * SW + v0) = d;
        *reinterpret_cast<uint32_t*>(Sa + (int64_t)i * SW + v0) = a;
    }
}

// Steps from row i to the nearest source of column `col` of a sheared image,
// from its column-pass scratch (CH_BIG when the column has none).
__device__ __forceinline__ int diag_steps(const ColScratch& s, int64_t SW, int b, int r, int i, int col)
{
    const uint32_t w = s.C[(int64_t)b * SW + col];
    const uint32_t a_ = w & (FULL >> (31 - r)), b_ = w & (FULL << r);
    int up, dn;
    if (a_) {
        up = b * 32 + 31 - __clz(a_);
    } else {
        uint32_t u = s.U[(int64_t)b * SW + col] & 0xFFFFu;
        if (u == (uint32_t)NONE16) u = s.GAB[(int64_t)(b >> 5) * SW + col] & 0xFFFFu;
        up = (u == (uint32_t)NONE16) ? -CH_BIG : (int)u;
    }
    if (b_) {
        dn = b * 32 + __ffs(b_) - 1;
    } else {
        uint32_t u = s.U[(int64_t)b * SW + col] >> 16;
        if (u == (uint32_t)NONE16) u = s.GAB[(int64_t)(b >> 5) * SW + col] >> 16;
        dn = (u == (uint32_t)NONE16) ? CH_BIG : (int)u;
    }
    const int d = min(i - up, dn - i);
    return d < 32768 ? d : CH_BIG;     // real distances stay below 32768 rows
}

__device__ __forceinline__ int warp_incl_min_up(int v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v = min(v, u);
    }
    return v;
}
__device__ __forceinline__ int warp_incl_min_down(int v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_down_sync(FULL, v, o);
        if (lane + o < 32) v = min(v, u);
    }
    return v;
}

// (3) E and the row term for 8 rows of one band; CPT columns per thread.
template <int CPT>
__global__ void __launch_bounds__(1024)
k_chamfer_rows(int H, int W, int SW, ColScratch sd, ColScratch sa, int32_t* __restrict__ D,
               int32_t* __restrict__ E)
{
    __shared__ int sx[32], sy[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarp = blockDim.x >> 5;
    const int b = blockIdx.x >> 2;
    const int r0 = (blockIdx.x & 3) * CH_ROWS;
    const int c0 = t * CPT;
    for (int rr = 0; rr < CH_ROWS; ++rr) {
        const int r = r0 + rr, i = b * 32 + r;
        if (i >= H) break;                                // uniform over the block
        int e[CPT], px[CPT], sy_[CPT];
        int run = CH_BIG;
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int j = c0 + c;
            int ev = CH_BIG;
            if (j < W) {
                const int dd = diag_steps(sd, SW, b, r, i, j - i + H - 1);
                const int da = diag_steps(sa, SW, b, r, i, i + j);
                const int dm = min(dd, da);
                ev = dm >= CH_BIG ? CH_BIG : 4 * dm;
            }
            e[c] = ev;
            run = min(run, ev - 3 * j);
            px[c] = run;
            sy_[c] = ev + 3 * j;
        }
        int suf = CH_BIG;
#pragma unroll
        for (int c = CPT - 1; c >= 0; --c) {
            suf = min(suf, sy_[c]);
            sy_[c] = suf;
        }
        const int ix = warp_incl_min_up(run, lane), iy = warp_incl_min_down(suf, lane);
        if (lane == 31) sx[warp] = ix;
        if (lane == 0) sy[warp] = iy;
        __syncthreads();
        if (warp == 0) {
            const int vx = lane < nwarp ? sx[lane] : CH_BIG;
            const int vy = lane < nwarp ? sy[lane] : CH_BIG;
            const int ex = warp_incl_min_up(vx, lane), ey = warp_incl_min_down(vy, lane);
            sx[lane] = ex;
            sy[lane] = ey;
        }
        __syncthreads();
        int carry_x = __shfl_up_sync(FULL, ix, 1), carry_y = __shfl_down_sync(FULL, iy, 1);
        if (lane == 0) carry_x = CH_BIG;
        if (lane == 31) carry_y = CH_BIG;
        if (warp > 0) carry_x = min(carry_x, sx[warp - 1]);
        if (warp + 1 < nwarp) carry_y = min(carry_y, sy[warp + 1]);
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int j = c0 + c;
            if (j < W) {
                const int64_t o = (int64_t)i * W + j;
                D[o] = min(3 * j + min(carry_x, px[c]), -3 * j + min(carry_y, sy_[c]));
                E[o] = e[c];
            }
        }
        __syncthreads();
    }
}

// (4a) per chunk of CH_CHUNK rows and column: min of E(m) - 3m and E(m) + 3m.
__global__ void k_chamfer_cols_totals(int H, int W, const int32_t* __restrict__ E, int* __restrict__ Tf,
                                      int* __restrict__ Tb)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (j >= W) return;
    int f = CH_BIG, bk = CH_BIG;
    const int m1 = min(H, (q + 1) * CH_CHUNK);
    for (int m = q * CH_CHUNK; m < m1; ++m) {
        const int e = E[(int64_t)m * W + j];
        f = min(f, e - 3 * m);
        bk = min(bk, e + 3 * m);
    }
    Tf[(int64_t)q * W + j] = f;
    Tb[(int64_t)q * W + j] = bk;
}

// (4b) the column term of every pixel of a chunk, with the other chunks'
// minima as carries; D becomes min(row term, column term), INT32_MAX where
// no source exists.
__global__ void k_chamfer_cols(int H, int W, const int32_t* __restrict__ E, const int* __restrict__ Tf,
                               const int* __restrict__ Tb, int nq, int32_t* __restrict__ D)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (j >= W) return;
    int cf = CH_BIG, cb = CH_BIG;
    for (int k = 0; k < q; ++k) cf = min(cf, Tf[(int64_t)k * W + j]);
    for (int k = q + 1; k < nq; ++k) cb = min(cb, Tb[(int64_t)k * W + j]);
    const int m0 = q * CH_CHUNK, m1 = min(H, m0 + CH_CHUNK);
    for (int m = m1 - 1; m >= m0; --m) {              // from below: -3m + min_{k>=m} E(k) + 3k
        const int64_t o = (int64_t)m * W + j;
        cb = min(cb, E[o] + 3 * m);
        D[o] = min(D[o], -3 * m + cb);
    }
    for (int m = m0; m < m1; ++m) {                    // from above: 3m + min_{k<=m} E(k) - 3k
        const int64_t o = (int64_t)m * W + j;
        cf = min(cf, E[o] - 3 * m);
        const int d = min(D[o], 3 * m + cf);
        D[o] = d >= CH_BIG / 2 ? INT32_MAX : d;
    }
}

size_t chamfer_scratch_bytes(int H, int W)
{
    const size_t SW = chamfer_sheared_width(H, W);
    const ColGeom gs = col_geom(H, (int64_t)SW);
    const size_t nq = (H + CH_CHUNK - 1) / CH_CHUNK;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    return 2 * al((size_t)H * SW) + 2 * al(col_scratch_bytes(gs)) + al((size_t)H * W * 4) + 2 * al(nq * W * 4);
}

cudaError_t launch_chamfer(const uint8_t* mask, int H, int W, int mode, int32_t* D, void* scratch,
                           int sm_count, cudaStream_t stream)
{
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    const int SW = (int)chamfer_sheared_width(H, W);
    const ColGeom gs = col_geom(H, SW);
    const int nq = (H + CH_CHUNK - 1) / CH_CHUNK;
    char* p = static_cast<char*>(scratch);
    uint8_t* Sd = reinterpret_cast<uint8_t*>(p);
    p += al((size_t)H * SW);
    uint8_t* Sa = reinterpret_cast<uint8_t*>(p);
    p += al((size_t)H * SW);
    const ColScratch sd = col_scratch_carve(p, gs);
    p += al(col_scratch_bytes(gs));
    const ColScratch sa = col_scratch_carve(p, gs);
    p += al(col_scratch_bytes(gs));
    int32_t* E = reinterpret_cast<int32_t*>(p);
    p += al((size_t)H * W * 4);
    int* Tf = reinterpret_cast<int*>(p);
    p += al((size_t)nq * W * 4);
    int* Tb = reinterpret_cast<int*>(p);
    cudaError_t e;
    if ((e = cudaMemsetAsync(sd.cnt, 0, (size_t)gs.ntiles * 4, stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(sa.cnt, 0, (size_t)gs.ntiles * 4, stream)) != cudaSuccess) return e;
    k_shear<<<sm_count * 8, 256, 0, stream>>>(mask, H, W, SW, mode, Sd, Sa);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_colbits(Sd, gs, 0, sd, stream)) != cudaSuccess) return e;
    if ((e = launch_colbits(Sa, gs, 0, sa, stream)) != cudaSuccess) return e;
    const unsigned blocks = (unsigned)(((H + 31) / 32) * 4);
    if (W <= 8 * 1024)
        k_chamfer_rows<8><<<blocks, ((W + 7) / 8 + 31) & ~31, 0, stream>>>(H, W, SW, sd, sa, D, E);
    else
        k_chamfer_rows<16><<<blocks, ((W + 15) / 16 + 31) & ~31, 0, stream>>>(H, W, SW, sd, sa, D, E);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const dim3 grid((unsigned)((W + 127) / 128), (unsigned)nq);
    k_chamfer_cols_totals<<<grid, 128, 0, stream>>>(H, W, E, Tf, Tb);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_chamfer_cols<<<grid, 128, 0, stream>>>(H, W, E, Tf, Tb, nq, D);
    return cudaGetLastError();
}

}  // namespace edt
