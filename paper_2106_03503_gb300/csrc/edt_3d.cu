// 3-D exact EDT.  Sec. 3.1 of the paper handles a multi-dimensional image one
// axis at a time;
// for a [Dz][H][W] volume this library runs
//   (z) the column pass along z: the volume seen as a 2-D image with Dz rows
//       and H*W columns, handled by the same column-bit kernel as 2-D images;
//   (y) the lower envelope of Sec. 3.3.1 along y, over f(y') = (z - z')^2 with
//       z' the nearest source along z in column (y', x): for each voxel it
//       records the source (z', y') of its owning parabola, packed as
//       z' << 16 | y' (0xFFFFFFFF = no source in the whole x-slice);
//   (x) the lower envelope along x over f(x') = (z - z')^2 + (y - y')^2 read
//       from that record, writing D, F = z'*H*W + y'*W + x' and sqrt(D).
// The (z', y') record lives in the caller's F (or D) buffer: the x pass reads
// its rows into shared memory before it overwrites the same rows.
// Both envelope passes use the band engine (edt_engine.cuh) with 32 lines per
// block: 32 neighbouring x columns for the y pass (stores are coalesced across
// lanes), 32 consecutive rows for the x pass (stores go through the tile).
#include "edt_engine.cuh"
#include "edt_internal.h"

namespace edt {

constexpr uint32_t PNONE = 0xFFFFFFFFu;

// --- y pass ----------------------------------------------------------------

// y tile data: for each (y, x), d = nearest source z along z minus z (int16,
// YNONE when the column has no source), [YPAD + H + YPAD][32], the pads
// holding YNONE so that a search may step past either end.
constexpr short YNONE = 32767;
constexpr int YPAD = DIRECT_MAX_DIST;

struct LineY {
    const short* gz;         // row y' of this tile at gz[y' * 32] (pads around)
    int lane;
    int z;
    __device__ __forceinline__ bool eval(int k, int& f) const
    {
        const int d = gz[k * 32 + lane];
        if (d == YNONE) return false;
        f = d * d;
        return true;
    }
    __device__ __forceinline__ int c(int k) const
    {
        const int d = gz[k * 32 + lane];
        return d * d + k * k;
    }
    __device__ __forceinline__ bool eval2(int k, int& f, int& feat) const
    {
        const int d = gz[k * 32 + lane];
        if (d == YNONE) return false;
        f = d * d;
        feat = (int)(((uint32_t)(z + d) << 16) | (uint32_t)k);
        return true;
    }
    __device__ __forceinline__ bool is_zero(int k) const { return gz[k * 32 + lane] == 0; }
    __device__ __forceinline__ bool chunk_has_source(int j0) const
    {
        bool any = false;
#pragma unroll
        for (int t = 0; t < OC; ++t) any |= gz[(j0 + t) * 32 + lane] == 0;
        return any;
    }
    __device__ __forceinline__ int self_feature(int k) const
    {
        return (int)(((uint32_t)z << 16) | (uint32_t)k);
    }
};

struct OutY {
    uint32_t* P;             // record of voxel (z, y, x0 + lane) at P[y * W]
    int W;
    bool valid;
    __device__ __forceinline__ void finish() const {}
    __device__ __forceinline__ void store(int j0, int cnt, const int* v, const int* f) const
    {
        if (!valid) return;
#pragma unroll
        for (int t = 0; t < OC; ++t)
            if (t < cnt) P[(int64_t)(j0 + t) * W] = (v[t] == INT32_MAX) ? PNONE : (uint32_t)f[t];
    }
};

// y tile: z offsets of [YPAD + H + YPAD][32] (int16), per-warp maxima (32
// ints), engine
__host__ __device__ static inline size_t ytile_bytes(int H)
{
    return ((size_t)(H + 2 * YPAD) * 32 * 2 + 15) & ~size_t(15);
}
__host__ __device__ static inline size_t ypass_smem(int H, int lg, int NW)
{
    return ytile_bytes(H) + 128 + band_smem_bytes(NW, (1 << lg) >> 5);
}

size_t batch_ypass_group_bytes(int H, int lg, int NW) { return ypass_smem(H, lg, NW); }

// One y-pass tile: plane z, the 32 columns x0 .. x0+31 (one line per lane),
// NW warps = y segments.  Run by the nthr threads of one engine (tid = thread
// within it, warp = warp within it) over the shared memory at `base`.
template <class Sync>
__device__ void ypass_tile(int H, int W, const ColScratch& s, int lg, int NW, uint32_t* __restrict__ P,
                           int z, int x0, unsigned char* base, int tid, int nthr, int warp, Sync sync)
{
    short* gz = reinterpret_cast<short*>(base) + YPAD * 32;     // row 0 of the tile
    int* wmax = reinterpret_cast<int*>(base + ytile_bytes(H));
    const BandSmem sm = carve_band_smem(base + ytile_bytes(H) + 128, NW, (1 << lg) >> 5);
    const int lane = tid & 31;
    const int64_t plane = (int64_t)H * W;
    const int zb = z >> 5, zr = z & 31, zG = zb >> s.gs;

    // z offset of the nearest source along z of every (y, x) of the tile, and
    // the largest distance among them (columns past the volume's edge count
    // as 0); the pads hold YNONE
    int dmax = 0;
    for (int e = tid; e < (H + 2 * YPAD) * 32; e += nthr) {
        const int y = (e >> 5) - YPAD, xl = e & 31, x = x0 + xl;
        int d = YNONE;
        if (y >= 0 && y < H && x < W) {
            const int64_t p = (int64_t)y * W + x;
            const uint32_t w = s.C[(int64_t)zb * plane + p];
            const uint32_t u = s.U[(int64_t)zb * plane + p];
            uint32_t up = u & 0xFFFFu, dn = u >> 16;
            if (up == (uint32_t)NONE16 || dn == (uint32_t)NONE16) {
                const uint32_t gab = s.GAB[(int64_t)zG * plane + p];
                if (up == (uint32_t)NONE16) up = gab & 0xFFFFu;
                if (dn == (uint32_t)NONE16) dn = gab >> 16;
            }
            const int g = nearest_in_column(w, zb * 32, zr, (int)up, (int)dn);
            d = g < 0 ? YNONE : g - z;
            dmax = max(dmax, abs(d));
        }
        gz[e - YPAD * 32] = (short)d;
    }
    dmax = (int)__reduce_max_sync(FULL, (unsigned)dmax);
    if (lane == 0) wmax[warp] = dmax;
    sync();
    for (int w = 0; w < NW; ++w) dmax = max(dmax, wmax[w]);

    const OutY out{P + (int64_t)z * plane + x0 + lane, W, x0 + lane < W};
    if (dmax <= DIRECT_MAX_DIST) {
        // near answers: each position searches outward along y (Eq. (5)
        // minimised exactly, rightmost y' at a tie, as the hull walk); every
        // own offset is at most DIRECT_MAX_DIST = YPAD, so the search never
        // leaves the padded tile and needs no bounds or validity test (a pad
        // or a column without source costs 32767^2, more than any answer)
        const int nq = (H + OC - 1) / OC;
        for (int q = warp; q < nq; q += NW) {
            const int j0 = q * OC;
            int v[OC], ft[OC];
#pragma unroll
            for (int t = 0; t < OC; ++t) {
                const int j = j0 + t;
                v[t] = INT32_MAX;
                ft[t] = -1;
                if (j >= H || x0 + lane >= W) continue;   // not a voxel of the tile
                const short* col = gz + lane;
                const int d0 = col[j * 32];
                int best = d0 * d0, bk = j;
                for (int r = 1, r2 = 1; r2 <= best; ++r, r2 += 2 * r - 1) {
                    const int dl = col[(j - r) * 32], dr = col[(j + r) * 32];
                    const int cl = dl * dl + r2, cr = dr * dr + r2;
                    if (cl < best) { best = cl; bk = j - r; }
                    if (cr <= best) { best = cr; bk = j + r; }
                }
                v[t] = best;
                ft[t] = (int)(((uint32_t)(z + col[bk * 32]) << 16) | (uint32_t)bk);
            }
            out.store(j0, min(OC, H - j0), v, ft);
        }
    } else {
        const LineY line{gz, lane, z};
        band_envelope(line, out, sm, H, lg, NW, nullptr, warp, sync);
    }
}

// One block: one z, 32 consecutive x (one line per lane), warps = y segments.
__global__ void __launch_bounds__(1024)
k_ypass3d(int H, int W, ColScratch s, int lg, int NW, uint32_t* __restrict__ P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int xtiles = (W + 31) / 32;
    const int z = blockIdx.x / xtiles;
    const int x0 = (blockIdx.x % xtiles) * 32;
    ypass_tile(H, W, s, lg, NW, P, z, x0, smem, threadIdx.x, blockDim.x, threadIdx.x >> 5, BlockSync());
}

// --- x pass ----------------------------------------------------------------

struct LineX {
    const uint32_t* rec;     // this lane's row of (z', y') records (pitch odd)
    int z, y, H, W;
    uint32_t self;           // this row's own record, (z << 16) | y
    bool valid;
    __device__ __forceinline__ bool eval(int k, int& f) const
    {
        if (!valid) return false;
        const uint32_t p = rec[k];
        if (p == PNONE) return false;
        const int dz = z - (int)(p >> 16), dy = y - (int)(p & 0xFFFFu);
        f = dz * dz + dy * dy;
        return true;
    }
    __device__ __forceinline__ int c(int k) const
    {
        const uint32_t p = rec[k];
        const int dz = z - (int)(p >> 16), dy = y - (int)(p & 0xFFFFu);
        return dz * dz + dy * dy + k * k;
    }
    __device__ __forceinline__ bool eval2(int k, int& f, int& feat) const
    {
        if (!valid) return false;
        const uint32_t p = rec[k];
        if (p == PNONE) return false;
        const int zz = (int)(p >> 16), yy = (int)(p & 0xFFFFu);
        f = (z - zz) * (z - zz) + (y - yy) * (y - yy);
        feat = (zz * H + yy) * W + k;
        return true;
    }
    __device__ __forceinline__ bool is_zero(int k) const { return rec[k] == self; }
    __device__ __forceinline__ bool chunk_has_source(int j0) const
    {
        bool any = false;
#pragma unroll
        for (int t = 0; t < OC; ++t) any |= rec[j0 + t] == self;
        return any;
    }
    __device__ __forceinline__ int self_feature(int k) const { return (z * H + y) * W + k; }
};

__host__ __device__ static inline int xpass_pitch(int W) { return W | 1; }

// x unit: records of [32][pitch], per-warp maxima (32 ints), engine
__host__ __device__ static inline size_t xpass_smem(int W, int lg, int NW)
{
    return (((size_t)32 * xpass_pitch(W) * 4 + 15) & ~size_t(15)) + 128 +
           band_smem_bytes(NW, (1 << lg) >> 5);
}

size_t batch_xpass_group_bytes(int W, int lg, int NW) { return xpass_smem(W, lg, NW); }

// One x-pass unit: the 32 rows (z, y) starting at row0 of the Dz*H rows (one
// per lane), NW warps = x segments; run by one engine as ypass_tile.
template <class Sync>
__device__ void xpass_rows(int Dz, int H, int W, int lg, int NW, const uint32_t* P, int32_t* D, int32_t* F,
                           float* dist, int64_t row0, unsigned char* base, int tid, int nthr, int warp, Sync sync)
{
    const int pitch = W | 1;
    uint32_t* rec = reinterpret_cast<uint32_t*>(base);   // [32][pitch]
    int* wmax = reinterpret_cast<int*>(base + (((size_t)32 * pitch * 4 + 15) & ~size_t(15)));
    const BandSmem sm = carve_band_smem(base + (((size_t)32 * pitch * 4 + 15) & ~size_t(15)) + 128, NW,
                                        (1 << lg) >> 5);
    const int lane = tid & 31;
    const int64_t nrows = (int64_t)Dz * H;

    // the rows' (z', y') records, and the largest (z, y) distance among them
    // (rows past the volume's end count as 0); (z, y) of the unit's first row
    // once, then stepped row by row, so the loads need no divisions
    int dmax = 0;
    int zz = (int)(row0 / H), yy = (int)(row0 % H);
    for (int rl = 0; rl < 32; ++rl) {
        const int64_t row = row0 + rl;
        const bool live = row < nrows;
        const uint32_t* src = P + row * W;
        uint32_t* dst = rec + rl * pitch;
        for (int k = tid; k < W; k += nthr) {
            uint32_t p = PNONE;
            if (live) {
                p = src[k];
                const int dz = zz - (int)(p >> 16), dy = yy - (int)(p & 0xFFFFu);
                dmax = max(dmax, p == PNONE ? 32767 : max(abs(dz), abs(dy)));
            }
            dst[k] = p;
        }
        if (++yy == H) {
            yy = 0;
            ++zz;
        }
    }
    dmax = (int)__reduce_max_sync(FULL, (unsigned)dmax);
    if (lane == 0) wmax[warp] = dmax;
    sync();
    for (int w = 0; w < NW; ++w) dmax = max(dmax, wmax[w]);

    if (dmax <= DIRECT_MAX_DIST) {
        // near answers: each warp takes whole rows, its lanes 32 consecutive
        // x, and searches outward along the row (Eq. (5) minimised exactly,
        // rightmost x' at a tie, as the hull walk); every candidate at most
        // about 91 positions away, so the search stays short, neighbouring
        // lanes search about as far, and D, F, dist go out as 128-byte lines
        for (int rl = warp; rl < 32; rl += NW) {
            const int64_t row = row0 + rl;
            if (row >= nrows) break;
            const int zz = (int)(row / H), yy = (int)(row % H);
            uint32_t* rr = rec + rl * pitch;
            // the warp's own row, rewritten in place: bits 31..24 and 23..16
            // the z and y offsets of the record (each within +-64 here), bits
            // 15..0 their squared length (at most 2 * 64^2), so that a
            // candidate costs one load and a mask
            for (int k = lane; k < W; k += 32) {
                const uint32_t p = rr[k];
                const int dz = zz - (int)(p >> 16), dy = yy - (int)(p & 0xFFFFu);
                rr[k] = ((uint32_t)(dz & 0xFF) << 24) | ((uint32_t)(dy & 0xFF) << 16) | (uint32_t)(dz * dz + dy * dy);
            }
            __syncwarp();
            for (int c0 = 0; c0 < W; c0 += 32) {
                const int j = c0 + lane;
                if (j >= W) continue;
                int best = (int)(rr[j] & 0xFFFFu), bk = j;
                for (int r = 1, r2 = 1; r2 <= best; ++r, r2 += 2 * r - 1) {
                    if (j - r >= 0) {
                        const int c = (int)(rr[j - r] & 0xFFFFu) + r2;
                        if (c < best) {
                            best = c;
                            bk = j - r;
                        }
                    }
                    if (j + r < W) {
                        const int c = (int)(rr[j + r] & 0xFFFFu) + r2;
                        if (c <= best) {
                            best = c;
                            bk = j + r;
                        }
                    }
                }
                const uint32_t p = rr[bk];
                const int dz = (int)(int8_t)(p >> 24), dy = (int)(int8_t)((p >> 16) & 0xFFu);
                const int64_t q = row * W + j;
                if (D) D[q] = best;
                if (F) F[q] = ((zz - dz) * H + (yy - dy)) * W + bk;
                if (dist) dist[q] = sqrt_rn_int(best);
            }
        }
        return;
    }

    const int64_t row = row0 + lane;
    LineX line;
    line.rec = rec + lane * pitch;
    line.z = (int)(row / H);
    line.y = (int)(row % H);
    line.H = H;
    line.W = W;
    line.valid = row < nrows;
    line.self = ((uint32_t)line.z << 16) | (uint32_t)line.y;
    const int vec = row_vec_width(W, D, F, dist);
    const RowOut out{D, F, dist, row * W, row < nrows, vec};
    band_envelope(line, out, sm, W, lg, NW, nullptr, warp, sync);
}

// One block: 32 consecutive rows (z, y) of the volume (one per lane), warps =
// x segments.
__global__ void __launch_bounds__(1024)
k_xpass3d(int Dz, int H, int W, int lg, int NW, const uint32_t* P, int32_t* D,
          int32_t* F, float* dist)
{
    extern __shared__ __align__(16) unsigned char smem[];
    xpass_rows(Dz, H, W, lg, NW, P, D, F, dist, (int64_t)blockIdx.x * 32, smem, threadIdx.x, blockDim.x,
               threadIdx.x >> 5, BlockSync());
}

// --- batched 3-D passes ------------------------------------------------------

// Engine geometry of a 3-D line of n positions aiming at `pos` positions per
// warp (at most BATCH_3D_WARPS warps, segments of at least 32 positions).
void batch_line_geometry(int n, int pos, int& lg, int& NW)
{
    int want = (n + pos - 1) / pos;
    if (want < 1) want = 1;
    if (want > BATCH_3D_WARPS) want = BATCH_3D_WARPS;
    lg = band_seg_log2(n, want);
    NW = (n + (1 << lg) - 1) >> lg;
}

// Persistent y pass over every 3-D job of a batch: a work item is `groups`
// consecutive (z, x-tile) units of one job, one engine of NW warps each.
__global__ void __launch_bounds__(BATCH_3D_WARPS * 32)
k_batch_ypass3d(const BatchHeader* __restrict__ hdr, const BatchJob* __restrict__ jobs)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_item;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t total = hdr->k_total[PH_Y];
    unsigned* work = hdr->cnt + PH_Y;
    const int nj = hdr->njobs;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(work, 1u);
        __syncthreads();
        const int64_t item = s_item;
        if (item >= total) break;
        int lo = 0, hi = nj - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].k_first[PH_Y] <= item) lo = mid; else hi = mid - 1;
        }
        const BatchJob& J = jobs[lo];
        const int NW = J.NW;
        const int grp = warp / NW, wg = warp - grp * NW;
        const int xtiles = (J.W + 31) / 32;
        const int64_t unit = (item - J.k_first[PH_Y]) * J.groups + grp;
        if (grp < J.groups && unit < (int64_t)J.Dz * xtiles) {
            unsigned char* base = smem + (size_t)grp * ypass_smem(J.H, J.lg, NW);
            ypass_tile(J.H, J.W, J.s, J.lg, NW, reinterpret_cast<uint32_t*>(J.F), (int)(unit / xtiles),
                       (int)(unit % xtiles) * 32, base, wg * 32 + lane, NW * 32, wg, GroupSync{1 + grp, NW * 32});
        }
        __syncthreads();
    }
}

// Persistent x pass over every 3-D job of a batch: a work item is `xgroups`
// consecutive 32-row units of one job.
__global__ void __launch_bounds__(BATCH_3D_WARPS * 32)
k_batch_xpass3d(const BatchHeader* __restrict__ hdr, const BatchJob* __restrict__ jobs)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_item;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t total = hdr->k_total[PH_X];
    unsigned* work = hdr->cnt + PH_X;
    const int nj = hdr->njobs;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(work, 1u);
        __syncthreads();
        const int64_t item = s_item;
        if (item >= total) break;
        int lo = 0, hi = nj - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].k_first[PH_X] <= item) lo = mid; else hi = mid - 1;
        }
        const BatchJob& J = jobs[lo];
        const int NW = J.xNW;
        const int grp = warp / NW, wg = warp - grp * NW;
        const int64_t units = ((int64_t)J.Dz * J.H + 31) / 32;
        const int64_t unit = (item - J.k_first[PH_X]) * J.xgroups + grp;
        if (grp < J.xgroups && unit < units) {
            unsigned char* base = smem + (size_t)grp * xpass_smem(J.W, J.xlg, NW);
            xpass_rows(J.Dz, J.H, J.W, J.xlg, NW, reinterpret_cast<const uint32_t*>(J.F), J.D, J.F, J.dist,
                       unit * 32, base, wg * 32 + lane, NW * 32, wg, GroupSync{1 + grp, NW * 32});
        }
        __syncthreads();
    }
}

cudaError_t launch_batch_ypass3d(const BatchHeader* hdr, const BatchJob* jobs, int blocks, cudaStream_t stream)
{
    k_batch_ypass3d<<<blocks, BATCH_3D_WARPS * 32, BATCH_3D_SMEM, stream>>>(hdr, jobs);
    return cudaGetLastError();
}

cudaError_t launch_batch_xpass3d(const BatchHeader* hdr, const BatchJob* jobs, int blocks, cudaStream_t stream)
{
    k_batch_xpass3d<<<blocks, BATCH_3D_WARPS * 32, BATCH_3D_SMEM, stream>>>(hdr, jobs);
    return cudaGetLastError();
}

cudaError_t set_batch_3d_attributes()
{
    cudaError_t e = cudaFuncSetAttribute(k_batch_ypass3d, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)BATCH_3D_SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_batch_xpass3d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BATCH_3D_SMEM);
}

int batch_3d_blocks_per_sm()
{
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_batch_ypass3d, BATCH_3D_WARPS * 32, BATCH_3D_SMEM) !=
            cudaSuccess || a < 1)
        a = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_xpass3d, BATCH_3D_WARPS * 32, BATCH_3D_SMEM) !=
            cudaSuccess || b < 1)
        b = 1;
    return a < b ? a : b;
}

// Segments for lines of n positions: at most max_nw warps, fewer while the
// shared memory does not fit.
static void pick_band(int n, size_t (*smem_fn)(int, int, int), int max_nw, int& lg, int& NW)
{
    for (; max_nw >= 1; max_nw >>= 1) {
        lg = band_seg_log2(n, max_nw);
        NW = (n + (1 << lg) - 1) >> lg;
        if (smem_fn(n, lg, NW) <= 227 * 1024) return;
    }
}

cudaError_t launch_ypass3d(int Dz, int H, int W, const ColGeom& g,
                           const ColScratch& s, uint32_t* P, cudaStream_t stream)
{
    (void)g;
    // 8 warps: the y pass's shared memory is small (32 lines of 2-byte
    // nearest-z entries), so more blocks fit per SM and the merge tree is
    // shallower (measured on 512^3: 1.60 ms with 8, 1.88 ms with 16 warps)
    int lg, NW;
    const int shape3[3] = {Dz, H, W};
    const Tuning tu = tuning_lookup(3, shape3);
    pick_band(H, ypass_smem, tu.ypass_nw > 0 ? tu.ypass_nw : 8, lg, NW);
    const int xtiles = (W + 31) / 32;
    const unsigned blocks = (unsigned)((int64_t)Dz * xtiles);
    k_ypass3d<<<blocks, NW * 32, ypass_smem(H, lg, NW), stream>>>(H, W, s, lg, NW, P);
    return cudaGetLastError();
}

cudaError_t launch_xpass3d(int Dz, int H, int W, uint32_t* P, int32_t* D,
                           int32_t* F, float* dist, cudaStream_t stream)
{
    int lg, NW;
    const int shape3[3] = {Dz, H, W};
    const Tuning tu = tuning_lookup(3, shape3);
    pick_band(W, xpass_smem, tu.xpass_nw > 0 ? tu.xpass_nw : 32, lg, NW);
    const int64_t nrows = (int64_t)Dz * H;
    const unsigned blocks = (unsigned)((nrows + 31) / 32);
    k_xpass3d<<<blocks, NW * 32, xpass_smem(W, lg, NW), stream>>>(Dz, H, W, lg, NW, P, D, F, dist);
    return cudaGetLastError();
}

cudaError_t set_3d_attributes()
{
    cudaError_t e = cudaFuncSetAttribute(k_ypass3d, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_xpass3d, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

}  // namespace edt
