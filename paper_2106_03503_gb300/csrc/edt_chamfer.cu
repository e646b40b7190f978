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
//   (1)+(2) the column-bit kernel of the Euclidean transform runs on two
//       sheared views of the mask (H x SW; the view's column v is the
//       diagonal j - i = v - (H - 1), resp. the anti-diagonal i + j = v),
//       reading the mask rows at shifted columns, and gives the nearest
//       source along every diagonal;
//   (3) k_chamfer_rows stages the sheared columns of 16 rows in shared
//       memory, computes E and the row term as two prefix minima (weight 3),
//       writes the row term to D and E to a scratch image, and per column
//       the minima of E(m) - 3m and E(m) + 3m over its 16 rows;
//   (4) k_chamfer_cols_carry turns those chunk minima into the minima over
//       all chunks above / below each chunk, and k_chamfer_cols takes the
//       column term of every 16-row chunk from its E values (in registers)
//       and those carries, lowering D to it: one read of E and D, one write
//       of D.
#include "edt_engine.cuh"
#include "edt_internal.h"

namespace edt {

constexpr int CH_ROWS = 16;           // rows per block of the row kernel
constexpr int CH_BIG = 1 << 29;       // no source
constexpr int CH_CHUNK = CH_ROWS;     // rows per chunk of the column kernels (one row block)

size_t chamfer_sheared_width(int H, int W) { return ((size_t)W + H - 1 + 31) & ~size_t(31); }

// Steps from row i (bit r of its band's word) to the nearest source of a
// staged sheared column {w, up | dn << 16}; CH_BIG when the column has none.
__device__ __forceinline__ int staged_steps(uint2 c, int base, int r, int i)
{
    const uint32_t a_ = c.x & (FULL >> (31 - r)), b_ = c.x & (FULL << r);
    const uint32_t uo = c.y & 0xFFFFu, dno = c.y >> 16;
    const int up = a_ ? base + 31 - __clz(a_) : (uo == (uint32_t)NONE16 ? -CH_BIG : (int)uo);
    const int dn = b_ ? base + __ffs(b_) - 1 : (dno == (uint32_t)NONE16 ? CH_BIG : (int)dno);
    const int d = min(i - up, dn - i);
    return d < 32768 ? d : CH_BIG;     // real distances stay below 32768 rows
}

// Column data {w, up | dn << 16} of column col of a sheared view's band b.
__device__ __forceinline__ uint2 sheared_column(const ColScratch& s, int64_t SW, int b, int64_t col)
{
    const uint32_t w = s.C[(int64_t)b * SW + col];
    const uint32_t u = s.U[(int64_t)b * SW + col];
    uint32_t up = u & 0xFFFFu, dn = u >> 16;
    if (up == (uint32_t)NONE16 || dn == (uint32_t)NONE16) {
        const uint32_t gab = s.GAB[(int64_t)(b >> s.gs) * SW + col];
        if (up == (uint32_t)NONE16) up = gab & 0xFFFFu;
        if (dn == (uint32_t)NONE16) dn = gab >> 16;
    }
    return make_uint2(w, up | (dn << 16));
}

// (3) E and the row term for CH_ROWS rows of one band.  The sheared columns
// these rows touch (W + CH_ROWS - 1 per direction) are staged in shared
// memory first.  Warp w holds columns [w * 32 SL, (w + 1) * 32 SL), lane l the
// columns w * 32 SL + 32 c + l (c < SL), so that loads and stores are
// coalesced; a row's prefix minima run slice by slice with warp shuffles,
// then across warps through shared memory.
template <int SL>
__global__ void __launch_bounds__(1024)
k_chamfer_rows(int H, int W, int SW, ColScratch sd, ColScratch sa, int32_t* __restrict__ D,
               int32_t* __restrict__ E, int* __restrict__ Tf, int* __restrict__ Tb)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int sx[32], sy[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarp = blockDim.x >> 5;
    const int nblk_band = 32 / CH_ROWS;
    const int b = blockIdx.x / nblk_band;
    const int base = b * 32;
    const int i0 = base + (blockIdx.x % nblk_band) * CH_ROWS;
    if (i0 >= H) return;                                  // whole block
    const int i1 = min(i0 + CH_ROWS, H);
    const int span = W + (i1 - 1 - i0);
    uint2* sD = reinterpret_cast<uint2*>(smem);           // diagonal columns H - i1 + x
    uint2* sA = sD + (W + CH_ROWS);                       // anti-diagonal columns i0 + x
    const int vbase = H - i1, ubase = i0;
    for (int x = t; x < span; x += blockDim.x) {
        sD[x] = sheared_column(sd, SW, b, vbase + x);
        sA[x] = sheared_column(sa, SW, b, ubase + x);
    }
    __syncthreads();
    const int jw = warp * 32 * SL;
    int tf[SL], tb[SL];                                   // chunk minima of E(m) -/+ 3m
#pragma unroll
    for (int c = 0; c < SL; ++c) tf[c] = tb[c] = CH_BIG;
    for (int i = i0; i < i1; ++i) {
        const int r = i - base;
        int e[SL], px[SL], sq[SL];
        int run = CH_BIG;
#pragma unroll
        for (int c = 0; c < SL; ++c) {
            const int j = jw + 32 * c + lane;
            int ev = CH_BIG;
            if (j < W) {
                const int dd = staged_steps(sD[j - i + H - 1 - vbase], base, r, i);
                const int da = staged_steps(sA[i + j - ubase], base, r, i);
                const int dm = min(dd, da);
                ev = dm >= CH_BIG ? CH_BIG : 4 * dm;
            }
            e[c] = ev;
            tf[c] = min(tf[c], ev - 3 * i);
            tb[c] = min(tb[c], ev + 3 * i);
            // slice prefix of E(k) - 3k, continued from the previous slices
            int v = ev - 3 * j;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(FULL, v, o);
                if (lane >= o) v = min(v, u);
            }
            v = min(v, run);
            px[c] = v;
            run = __shfl_sync(FULL, v, 31);
        }
        int suf = CH_BIG;
#pragma unroll
        for (int c = SL - 1; c >= 0; --c) {
            const int j = jw + 32 * c + lane;
            int v = e[c] + 3 * j;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_down_sync(FULL, v, o);
                if (lane + o < 32) v = min(v, u);
            }
            v = min(v, suf);
            sq[c] = v;
            suf = __shfl_sync(FULL, v, 0);
        }
        if (lane == 0) {
            sx[warp] = run;
            sy[warp] = suf;
        }
        __syncthreads();
        if (warp == 0) {
            int vx = lane < nwarp ? sx[lane] : CH_BIG, vy = lane < nwarp ? sy[lane] : CH_BIG;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int ux = __shfl_up_sync(FULL, vx, o), uy = __shfl_down_sync(FULL, vy, o);
                if (lane >= o) vx = min(vx, ux);
                if (lane + o < 32) vy = min(vy, uy);
            }
            sx[lane] = vx;
            sy[lane] = vy;
        }
        __syncthreads();
        const int cx = warp > 0 ? sx[warp - 1] : CH_BIG;
        const int cy = warp + 1 < nwarp ? sy[warp + 1] : CH_BIG;
#pragma unroll
        for (int c = 0; c < SL; ++c) {
            const int j = jw + 32 * c + lane;
            if (j < W) {
                const int64_t o = (int64_t)i * W + j;
                D[o] = min(3 * j + min(cx, px[c]), -3 * j + min(cy, sq[c]));
                E[o] = e[c];
            }
        }
        __syncthreads();
    }
    const int64_t q = i0 / CH_CHUNK;
#pragma unroll
    for (int c = 0; c < SL; ++c) {
        const int j = jw + 32 * c + lane;
        if (j < W) {
            Tf[q * W + j] = tf[c];
            Tb[q * W + j] = tb[c];
        }
    }
}

// (4a) per column, in place: Tf[q] becomes the minimum of E(m) - 3m over the
// chunks above chunk q, Tb[q] that of E(m) + 3m over the chunks below it.  A
// block of 32 warps takes 32 columns (lane x) and splits their chunks into 32
// consecutive runs (warp y): each thread reduces its run, the runs' minima are combined through
// shared memory, and each thread then rewrites its run with the carries.
__global__ void __launch_bounds__(1024)
k_chamfer_cols_carry(int W, int nq, int* __restrict__ Tf, int* __restrict__ Tb)
{
    __shared__ int sf[32][33], sb[32][33];
    const int x = threadIdx.x & 31, y = threadIdx.x >> 5;
    const int64_t j = (int64_t)blockIdx.x * 32 + x;
    const int q0 = (int)((int64_t)nq * y / 32), q1 = (int)((int64_t)nq * (y + 1) / 32);
    int f = CH_BIG, b = CH_BIG;
    if (j < W)
        for (int q = q0; q < q1; ++q) {
            f = min(f, Tf[q * (int64_t)W + j]);
            b = min(b, Tb[q * (int64_t)W + j]);
        }
    sf[y][x] = f;
    sb[y][x] = b;
    __syncthreads();
    int cf = CH_BIG, cb = CH_BIG;
    for (int k = 0; k < y; ++k) cf = min(cf, sf[k][x]);
    for (int k = y + 1; k < 32; ++k) cb = min(cb, sb[k][x]);
    if (j >= W) return;                                  // no barrier below
    for (int q = q0; q < q1; ++q) {
        const int t = Tf[q * (int64_t)W + j];
        Tf[q * (int64_t)W + j] = cf;
        cf = min(cf, t);
    }
    for (int q = q1 - 1; q >= q0; --q) {
        const int t = Tb[q * (int64_t)W + j];
        Tb[q * (int64_t)W + j] = cb;
        cb = min(cb, t);
    }
}

// (4b) the column term of every pixel of one chunk of CH_CHUNK rows: its E
// values in registers, the minima from below as a suffix over them plus the
// carry from the chunks below, the minima from above as a prefix plus the
// carry from the chunks above; D becomes min(row term, column term),
// INT32_MAX where no source exists.
__global__ void k_chamfer_cols(int H, int W, const int32_t* __restrict__ E, const int* __restrict__ Cf,
                               const int* __restrict__ Cb, int32_t* __restrict__ D)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (j >= W) return;
    const int m0 = q * CH_CHUNK;
    int e[CH_CHUNK], below[CH_CHUNK];
#pragma unroll
    for (int t = 0; t < CH_CHUNK; ++t) e[t] = (m0 + t < H) ? E[(int64_t)(m0 + t) * W + j] : CH_BIG;
    int cb = Cb[(int64_t)q * W + j];
#pragma unroll
    for (int t = CH_CHUNK - 1; t >= 0; --t) {          // -3m + min_{k>=m} E(k) + 3k
        cb = min(cb, e[t] + 3 * (m0 + t));
        below[t] = cb;
    }
    int cf = Cf[(int64_t)q * W + j];
#pragma unroll
    for (int t = 0; t < CH_CHUNK; ++t) {              // 3m + min_{k<=m} E(k) - 3k
        const int m = m0 + t;
        if (m < H) {
            const int64_t o = (int64_t)m * W + j;
            cf = min(cf, e[t] - 3 * m);
            const int d = min(D[o], min(3 * m + cf, -3 * m + below[t]));
            D[o] = d >= CH_BIG / 2 ? INT32_MAX : d;
        }
    }
}

size_t chamfer_scratch_bytes(int H, int W)
{
    const size_t SW = chamfer_sheared_width(H, W);
    const ColGeom gs = col_geom(H, (int64_t)SW);
    const size_t nq = (H + CH_CHUNK - 1) / CH_CHUNK;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    return 2 * al(col_scratch_bytes(gs)) + al((size_t)H * W * 4) + 2 * al(nq * W * 4);
}

cudaError_t launch_chamfer(const uint8_t* mask, int H, int W, int mode, int32_t* D, void* scratch,
                           int sm_count, cudaStream_t stream)
{
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    const int SW = (int)chamfer_sheared_width(H, W);
    const ColGeom gs = col_geom(H, SW);
    const int nq = (H + CH_CHUNK - 1) / CH_CHUNK;
    char* p = static_cast<char*>(scratch);
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
    (void)sm_count;
    if ((e = traced("k_colbits", stream, [&] { return launch_colbits_sheared(mask, gs, mode, sd, H, W, 1, stream); })) !=
        cudaSuccess)
        return e;
    if ((e = traced("k_colbits", stream, [&] { return launch_colbits_sheared(mask, gs, mode, sa, H, W, -1, stream); })) !=
        cudaSuccess)
        return e;
    const unsigned blocks = (unsigned)(((H + 31) / 32) * (32 / CH_ROWS));
    const size_t smem = 2 * (size_t)(W + CH_ROWS) * sizeof(uint2);
    if ((e = traced("k_chamfer_rows", stream, [&] {
             if (W <= 8 * 1024)
                 k_chamfer_rows<8><<<blocks, ((W + 255) / 256) * 32, smem, stream>>>(H, W, SW, sd, sa, D, E, Tf,
                                                                                     Tb);
             else
                 k_chamfer_rows<16><<<blocks, ((W + 511) / 512) * 32, smem, stream>>>(H, W, SW, sd, sa, D, E, Tf,
                                                                                      Tb);
             return cudaGetLastError();
         })) != cudaSuccess)
        return e;
    return traced("k_chamfer_cols", stream, [&] {
        k_chamfer_cols_carry<<<(unsigned)((W + 31) / 32), 1024, 0, stream>>>(W, nq, Tf, Tb);
        k_chamfer_cols<<<dim3((unsigned)((W + 127) / 128), (unsigned)nq), 128, 0, stream>>>(H, W, E, Tf, Tb, D);
        return cudaGetLastError();
    });
}

}  // namespace edt

namespace edt {
// The row kernel's dynamic shared memory: 2 x (W + CH_ROWS) x 8 bytes, at most
// 229,632 bytes for the widest row accepted (14336); its static shared memory
// (two 32-int arrays) has to fit beside it in the 227 KB of a block.
cudaError_t set_chamfer_attributes()
{
    const int bytes = 226 * 1024;
    cudaError_t e = cudaFuncSetAttribute(k_chamfer_rows<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_chamfer_rows<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}
}  // namespace edt
