// Column pass of the exact EDT (Sec. 3.1 of Strutz, "The Distance Transform
// and its Computation"): for every column, where are the source pixels, and
// which source is nearest above and below each band of 32 rows.
//
// The paper's column pass propagates squared distances down and up each
// column (Listing 7, Fig. 19, Fig. 18(b)).  Its result at row i of column j is
// (i - g)^2 with g the nearest source row; here the same nearest row is
// produced in a compact form that the row kernel expands on the fly:
//   - one 32-bit word per (band of 32 rows, column) with the source bits,
//     built by a warp from a 32 x 32 byte tile (each lane loads 32
//     consecutive bytes of its own row and packs them into a row word; a
//     five-stage shuffle butterfly transposes the 32 row words into the 32
//     column words);
//   - per band, the nearest source row above and below it inside its group of
//     bands (32, or fewer for images too small to give 4096 warp units, never
//     more than 32 groups to a column), from a forward and a backward scan
//     over the group's words;
//   - per group, the nearest source above and below it over the whole column,
//     computed by whichever warp of a 32-column tile finishes last (an arrival
//     counter per tile; no warp ever waits for another).
// Where rows start on 16-byte boundaries (width a multiple of 16) every mask
// byte is loaded once, with 16-byte loads; otherwise a 32-byte row window is
// read as the aligned chunks or words that cover it, so the few bytes shared
// by two tiles' windows are loaded by both.
#include "edt_engine.cuh"
#include "edt_internal.h"

namespace edt {

constexpr int K1_WARPS = 4;

ColGeom col_geom(int rows, int64_t cols, bool coarse)
{
    ColGeom g;
    g.rows = rows;
    g.cols = cols;
    g.nb = (rows + 31) / 32;
    g.ntiles = (cols + 31) / 32;
    // smaller groups (more warps, each walking fewer bands) only while the
    // image gives fewer than 4096 warp units: finer groups also make the
    // consumers fall back to the group summaries more often
    g.gs = 5;
    auto groups = [&](int gs) { return (g.nb + (1 << gs) - 1) >> gs; };
    if (!coarse)
        while (g.gs > 0 && g.ntiles * groups(g.gs) < 4096 && groups(g.gs - 1) <= 32) --g.gs;
    g.nG = groups(g.gs);
    return g;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t col_scratch_bytes(const ColGeom& g)
{
    const size_t c = (size_t)g.cols * 4;
    return 2 * align256((size_t)g.nb * c) + 2 * align256((size_t)g.nG * c) +
           align256((size_t)g.ntiles * 4);
}

ColScratch col_scratch_carve(void* base, const ColGeom& g)
{
    const size_t c = (size_t)g.cols * 4;
    char* p = static_cast<char*>(base);
    ColScratch s;
    s.C = reinterpret_cast<uint32_t*>(p);
    p += align256((size_t)g.nb * c);
    s.U = reinterpret_cast<uint32_t*>(p);
    p += align256((size_t)g.nb * c);
    s.GFL = reinterpret_cast<uint32_t*>(p);
    p += align256((size_t)g.nG * c);
    s.GAB = reinterpret_cast<uint32_t*>(p);
    p += align256((size_t)g.nG * c);
    s.cnt = reinterpret_cast<unsigned*>(p);
    s.gs = g.gs;
    return s;
}

// Bit t of the result is set when byte t of v is nonzero (t < 4).  The
// per-byte compare gives 0xFF bytes; their top bits (7, 15, 23, 31) are moved
// to bits 28..31 by one multiply (no two partial products overlap).
__device__ __forceinline__ uint32_t nz_bits4(uint32_t v)
{
    const uint32_t x = __vcmpne4(v, 0u) & 0x80808080u;
    return (x * 0x00204081u) >> 28;
}

__device__ __forceinline__ uint32_t nz_bits16(uint4 a)
{
    return nz_bits4(a.x) | (nz_bits4(a.y) << 4) | (nz_bits4(a.z) << 8) |
           (nz_bits4(a.w) << 12);
}

// Source bits of the 32 bytes at p (only the first ncols are valid: the
// others may hold the bits of the bytes that follow, which the caller masks
// off).  VEC: p is 16-byte aligned.  al: bit 0 = the mask starts on a 4-byte
// boundary, bit 1 = on a 16-byte boundary, so the aligned word / 16-byte
// chunk holding byte p (and the bytes before p in it) lies inside the mask;
// end = one past the mask's last byte.  Aligned 16-byte loads of the window
// read each byte once and carry the evict-first hint.  An unaligned window,
// or one of fewer than 32 columns (a row's last tile), is read as the two or
// three aligned 16-byte chunks that cover 32 bytes from p while they end
// inside the mask (else as aligned words plus its last bytes one by one); the
// chunks that straddle two tiles are read by both, so these loads keep the
// default caching.
template <bool VEC>
__device__ __forceinline__ uint32_t load_row_bits(const uint8_t* __restrict__ p, int ncols, int al,
                                                  const uint8_t* end)
{
    if (VEC && ncols == 32) {
        const uint4 a = __ldcs(reinterpret_cast<const uint4*>(p));
        const uint4 b = __ldcs(reinterpret_cast<const uint4*>(p + 16));
        return nz_bits16(a) | (nz_bits16(b) << 16);
    }
    if (VEC && ncols == 16) {
        const uint4 a = __ldcs(reinterpret_cast<const uint4*>(p));
        return nz_bits16(a);
    }
    if (!VEC && (al & 2)) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(p) & ~uintptr_t(15);
        const int o = (int)(reinterpret_cast<uintptr_t>(p) & 15);
        if (a + (o ? 48 : 32) <= reinterpret_cast<uintptr_t>(end)) {
            const uint4* q = reinterpret_cast<const uint4*>(a);
            uint64_t bits = (uint64_t)(nz_bits16(__ldg(q)) | (nz_bits16(__ldg(q + 1)) << 16));
            if (o) bits |= (uint64_t)nz_bits16(__ldg(q + 2)) << 32;
            return (uint32_t)(bits >> o);
        }
    }
    if (!VEC && (al & 1) && ncols == 32) {
        // 8 aligned words from the word holding byte p, the last o = p mod 4
        // bytes one by one (never past byte 31), realigned by funnel shifts
        const uintptr_t a = reinterpret_cast<uintptr_t>(p) & ~uintptr_t(3);
        const int o = (int)(reinterpret_cast<uintptr_t>(p) & 3);
        const uint32_t* q = reinterpret_cast<const uint32_t*>(a);
        uint32_t w[9];
#pragma unroll
        for (int i = 0; i < 8; ++i) w[i] = __ldg(q + i);
        w[8] = 0u;
        for (int t = 0; t < o; ++t) w[8] |= (uint32_t)__ldg(p + 32 - o + t) << (8 * t);
        uint32_t bits = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) bits |= nz_bits4(__funnelshift_r(w[i], w[i + 1], 8 * o)) << (4 * i);
        return bits;
    }
    uint32_t bits = 0;
    for (int t = 0; t < ncols; ++t) bits |= (uint32_t)(__ldg(p + t) != 0) << t;
    return bits;
}

// Source bits of the 32 bytes of one image row at columns j0 .. j0+31 (a
// sheared view: some of them may lie outside the row; `valid` gets the bits
// of those inside).
__device__ __forceinline__ uint32_t sheared_row_bits(const uint8_t* __restrict__ row, int64_t W, int64_t j0,
                                                     int al, const uint8_t* end, uint32_t& valid)
{
    if (j0 >= 0 && j0 + 32 <= W) {
        valid = FULL;
        return load_row_bits<false>(row + j0, 32, al, end);
    }
    uint32_t bits = 0;
    valid = 0;
    if (j0 + 32 <= 0 || j0 >= W) return 0;  // wholly outside the row
    for (int t = 0; t < 32; ++t) {
        const int64_t j = j0 + t;
        if (j >= 0 && j < W) {
            valid |= 1u << t;
            bits |= (uint32_t)(__ldg(row + j) != 0) << t;
        }
    }
    return bits;
}

// 32 x 32 bit transpose across a warp: lane l holds row l (bit c = element
// (l, c)); the result in lane c is column c (bit l = element (l, c)).  Five
// butterfly stages: at distance j, lanes exchange words with lane l ^ j and
// swap the j-bit blocks that lie on the wrong side of the diagonal.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane)
{
#define EDT_TRANSPOSE_STAGE(j, m)                                                          \
    {                                                                                      \
        const uint32_t y = __shfl_xor_sync(FULL, x, j);                                    \
        x = (lane & (j)) ? ((x & ~(m)) | ((y >> (j)) & (m))) : ((x & (m)) | ((y << (j)) & ~(m))); \
    }
    EDT_TRANSPOSE_STAGE(16, 0x0000FFFFu)
    EDT_TRANSPOSE_STAGE(8, 0x00FF00FFu)
    EDT_TRANSPOSE_STAGE(4, 0x0F0F0F0Fu)
    EDT_TRANSPOSE_STAGE(2, 0x33333333u)
    EDT_TRANSPOSE_STAGE(1, 0x55555555u)
#undef EDT_TRANSPOSE_STAGE
    return x;
}

// Rows of band `band` that lie inside the image, as a bit mask.
__device__ __forceinline__ uint32_t band_rows_mask(const ColGeom& g, int band)
{
    const int rows = g.rows - band * 32;
    return rows >= 32 ? FULL : ((1u << rows) - 1u);
}

// Step (2) for one column: nearest source above / below each band of group G
// inside the group, and the group's first / last source row.  `invert` takes
// the complement of the words (the other class as sources) within the image.
__device__ __forceinline__ void group_scan(const ColGeom& g, const ColScratch& s, uint32_t (*cw)[32],
                                           uint32_t (*upS)[32], bool invert, int G, int64_t col)
{
    const int lane = threadIdx.x & 31;
    const int64_t W = g.cols;
    const int b0 = G << g.gs;
    const int nbg = min(1 << g.gs, g.nb - b0);
    int last = NONE16, first = NONE16;
    for (int bl = 0; bl < nbg; ++bl) {
        uint32_t w = cw[bl][lane];
        if (invert) w = ~w & band_rows_mask(g, b0 + bl);
        upS[bl][lane] = (uint32_t)last;
        if (w) {
            last = (b0 + bl) * 32 + 31 - __clz(w);
            if (first == NONE16) first = (b0 + bl) * 32 + __ffs(w) - 1;
        }
    }
    int nxt = NONE16;
    for (int bl = nbg - 1; bl >= 0; --bl) {
        uint32_t w = cw[bl][lane];
        if (invert) w = ~w & band_rows_mask(g, b0 + bl);
        s.U[(int64_t)(b0 + bl) * W + col] = upS[bl][lane] | ((uint32_t)nxt << 16);
        if (w) nxt = (b0 + bl) * 32 + __ffs(w) - 1;
    }
    s.GFL[(int64_t)G * W + col] = (uint32_t)first | ((uint32_t)last << 16);
}

// Step (3) for one column: nearest source above / below every group, over the
// whole column, from the groups' first / last rows.  tmp: 32 words of scratch.
__device__ __forceinline__ void link_groups(const ColGeom& g, const ColScratch& s, uint32_t (*tmp)[32],
                                            int64_t col)
{
    const int lane = threadIdx.x & 31;
    const int64_t W = g.cols;
    int above = NONE16;
    for (int G2 = 0; G2 < g.nG; ++G2) {
        const uint32_t v = __ldcg(s.GFL + (int64_t)G2 * W + col);
        tmp[G2][lane] = (uint32_t)above;
        if ((v >> 16) != (uint32_t)NONE16) above = (int)(v >> 16);
    }
    int below = NONE16;
    for (int G2 = g.nG - 1; G2 >= 0; --G2) {
        const uint32_t v = __ldcg(s.GFL + (int64_t)G2 * W + col);
        s.GAB[(int64_t)G2 * W + col] = tmp[G2][lane] | ((uint32_t)below << 16);
        if ((v & 0xFFFFu) != (uint32_t)NONE16) below = (int)(v & 0xFFFFu);
    }
}

// The work of one warp: columns [32*tile, 32*tile + 32) x bands of group G
// (bands G << gs .. (G + 1) << gs, at most 32).
// cw and upS are this warp's 32 x 32 shared scratch tiles.  With PAIR the
// warp serves both transforms from one read of the mask: s gets the summaries
// with the nonzero bytes as sources, s1 those with the zero bytes (the column
// words of the second are the complement of s.C inside the image and are not
// stored).
//
// SHEAR (+1 or -1) reads a sheared view of an imgH x imgW mask instead: the
// view's column v at row r is the image's column v + r - (imgH - 1) (SHEAR
// +1: the diagonals j - i = const become columns) or v - r (SHEAR -1: the
// anti-diagonals); pixels outside the image are no sources.
template <bool VEC, bool PAIR, int SHEAR = 0>
__device__ void colbits_warp(const uint8_t* __restrict__ mask, const ColGeom& g, int mode,
                             const ColScratch& s, const ColScratch& s1, int64_t tile, int G,
                             uint32_t (*cw)[32], uint32_t (*upS)[32], int imgH = 0, int64_t imgW = 0)
{
    const int lane = threadIdx.x & 31;
    const int64_t W = g.cols;
    const int64_t col0 = tile * 32;
    const int64_t col = col0 + lane;
    const int b0 = G << g.gs;
    const int nbg = min(1 << g.gs, g.nb - b0);
    const int ncols = (W - col0) < 32 ? (int)(W - col0) : 32;
    const uint32_t colvalid = ncols >= 32 ? FULL : ((1u << ncols) - 1u);
    const bool invert_in = !PAIR && mode == EDT_TO_BACKGROUND;
    const int al = ((reinterpret_cast<uintptr_t>(mask) & 3) == 0 ? 1 : 0) |
                   ((reinterpret_cast<uintptr_t>(mask) & 15) == 0 ? 2 : 0);
    const uint8_t* mask_end = mask + (SHEAR == 0 ? (int64_t)g.rows * W : (int64_t)imgH * imgW);

    // (1) source bits of 32 rows x 32 columns per band, transposed across the warp
    for (int bl = 0; bl < nbg; bl += 4) {
        uint32_t src[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int row = (b0 + bl + u) * 32 + lane;
            src[u] = 0;
            if (bl + u < nbg && row < g.rows) {
                if (SHEAR == 0) {
                    src[u] = load_row_bits<VEC>(mask + (int64_t)row * W + col0, ncols, al, mask_end);
                    if (invert_in) src[u] = ~src[u];
                    src[u] &= colvalid;
                } else {
                    const int64_t j0 = col0 + (SHEAR > 0 ? (int64_t)row - (imgH - 1) : -(int64_t)row);
                    uint32_t valid;
                    src[u] = sheared_row_bits(mask + (int64_t)row * imgW, imgW, j0, al, mask_end, valid);
                    if (invert_in) src[u] = ~src[u];
                    src[u] &= valid & colvalid;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (bl + u >= nbg) break;
            const uint32_t mine = transpose32(src[u], lane);
            cw[bl + u][lane] = mine;
            if (col < W) s.C[(int64_t)(b0 + bl + u) * W + col] = mine;
        }
    }
    __syncwarp();

    // (2) nearest source above / below each band inside the group
    if (col < W) {
        group_scan(g, s, cw, upS, false, G, col);
        if (PAIR) group_scan(g, s1, cw, upS, true, G, col);
    }

    // (3) the last group of this tile to finish links the groups; a column
    // of one group has nothing above or below it to link
    if (g.nG == 1) {
        if (col < W) {
            const uint32_t none = (uint32_t)NONE16 | ((uint32_t)NONE16 << 16);
            s.GAB[col] = none;
            if (PAIR) s1.GAB[col] = none;
        }
        return;
    }
    __threadfence();
    __syncwarp();
    unsigned old = 0;
    if (lane == 0) old = atomicAdd(&s.cnt[tile], 1u);
    old = __shfl_sync(FULL, old, 0);
    if (old != (unsigned)(g.nG - 1)) return;
    __threadfence();
    if (col < W) {
        link_groups(g, s, cw, col);
        if (PAIR) link_groups(g, s1, cw, col);
    }
    __syncwarp();
    if (lane == 0) s.cnt[tile] = 0u;  // ready for the next call
}

// Rows of a warp's two shared scratch tiles: the bands of a group, or the
// groups of a column when there are more of those.
__host__ __device__ inline int colbits_tile_rows(const ColGeom& g)
{
    return (1 << g.gs) > g.nG ? (1 << g.gs) : g.nG;
}

// Shared scratch per warp: two tiles of colbits_tile_rows(g) x 32 words
// (dynamic, so that small groups leave room for more resident blocks).
template <bool VEC, bool PAIR>
__global__ void __launch_bounds__(K1_WARPS * 32)
k_colbits(const uint8_t* __restrict__ mask, ColGeom g, int mode, ColScratch s, ColScratch s1)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    const int R = colbits_tile_rows(g);
    uint32_t (*cw)[32] =
        reinterpret_cast<uint32_t (*)[32]>(reinterpret_cast<uint32_t*>(smem) + (size_t)warp * 2 * R * 32);  // [band][column]
    uint32_t (*upS)[32] = cw + R;                                                                   // forward scans
    const int64_t gw = (int64_t)blockIdx.x * K1_WARPS + warp;
    if (gw >= g.ntiles * (int64_t)g.nG) return;  // whole warp; no block sync below
    colbits_warp<VEC, PAIR>(mask, g, mode, s, s1, gw % g.ntiles, (int)(gw / g.ntiles), cw, upS);
}

// Column pass over a sheared view (see colbits_warp) of an imgH x imgW mask;
// g is the view's geometry (imgH rows).
template <int SHEAR>
__global__ void __launch_bounds__(K1_WARPS * 32)
k_colbits_shear(const uint8_t* __restrict__ mask, ColGeom g, int mode, ColScratch s, int imgH, int64_t imgW)
{
    __shared__ uint32_t cw[K1_WARPS][32][32];
    __shared__ uint32_t upS[K1_WARPS][32][32];
    const int warp = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * K1_WARPS + warp;
    if (gw >= g.ntiles * (int64_t)g.nG) return;  // whole warp; no block sync below
    colbits_warp<false, false, SHEAR>(mask, g, mode, s, s, gw % g.ntiles, (int)(gw / g.ntiles), cw[warp],
                                      upS[warp], imgH, imgW);
}

cudaError_t launch_colbits_sheared(const uint8_t* mask, const ColGeom& g, int mode, const ColScratch& s,
                                   int imgH, int64_t imgW, int dir, cudaStream_t stream)
{
    const int64_t warps = g.ntiles * (int64_t)g.nG;
    const int64_t blocks = (warps + K1_WARPS - 1) / K1_WARPS;
    if (dir > 0)
        k_colbits_shear<1><<<(unsigned)blocks, K1_WARPS * 32, 0, stream>>>(mask, g, mode, s, imgH, imgW);
    else
        k_colbits_shear<-1><<<(unsigned)blocks, K1_WARPS * 32, 0, stream>>>(mask, g, mode, s, imgH, imgW);
    return cudaGetLastError();
}

// Persistent column pass over every job of a batch (for a 3-D job the z pass
// over its Dz x H*W view): warp units are numbered job by job
// (k_first[PH_COL]); warp w takes units w, w + (warps of the grid), ...,
// finding each unit's job by binary search from the previous one's.
__global__ void __launch_bounds__(K1_WARPS * 32)
k_batch_colbits(const BatchHeader* __restrict__ hdr, const BatchJob* __restrict__ jobs)
{
    __shared__ uint32_t cw[K1_WARPS][32][32];
    __shared__ uint32_t upS[K1_WARPS][32][32];
    const int warp = threadIdx.x >> 5;
    const int64_t total = hdr->k_total[PH_COL];
    const int nj = hdr->njobs;
    // units round-robin over the grid's warps: neighbouring tiles of a group
    // (whose rows share the 32-byte sectors their windows straddle) are read
    // at about the same time, so a shared sector comes from DRAM once
    const int64_t nw = (int64_t)gridDim.x * K1_WARPS, w = (int64_t)blockIdx.x * K1_WARPS + warp;
    int lo = 0;
    if (w < total) {
        int hi = nj - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].k_first[PH_COL] <= w) lo = mid; else hi = mid - 1;
        }
    }
    for (int64_t gw = w; gw < total; gw += nw) {
        // the unit's job: a step of nw units can pass many jobs, so a binary
        // search over the jobs after lo (each probe reads another job's entry)
        if (lo + 1 < nj && jobs[lo + 1].k_first[PH_COL] <= gw) {
            int a = lo + 1, b = nj - 1;
            while (a < b) {
                const int mid = (a + b + 1) >> 1;
                if (jobs[mid].k_first[PH_COL] <= gw) a = mid; else b = mid - 1;
            }
            lo = a;
        }
        const BatchJob& J = jobs[lo];
        const ColGeom g = J.g;
        const ColScratch s = J.s;
        const int64_t local = gw - J.k_first[PH_COL];
        if (J.vec)
            colbits_warp<true, false>(J.mask, g, J.mode, s, s, local % g.ntiles, (int)(local / g.ntiles),
                                      cw[warp], upS[warp]);
        else
            colbits_warp<false, false>(J.mask, g, J.mode, s, s, local % g.ntiles, (int)(local / g.ntiles),
                                       cw[warp], upS[warp]);
        __syncwarp();
    }
}

// Zero the batch's work and arrival counters (their number is in the table,
// so the graph node does not depend on the batch).
__global__ void __launch_bounds__(256) k_batch_clear(const BatchHeader* __restrict__ hdr)
{
    unsigned* c = hdr->cnt;
    const int64_t n = hdr->cnt_words;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c[i] = 0u;
}

cudaError_t launch_batch_clear(const BatchHeader* hdr, int blocks, cudaStream_t stream)
{
    k_batch_clear<<<blocks, 256, 0, stream>>>(hdr);
    return cudaGetLastError();
}

int batch_colbits_blocks_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_colbits, K1_WARPS * 32, 0) !=
            cudaSuccess || n < 1)
        n = 1;
    return n;
}

cudaError_t launch_batch_colbits(const BatchHeader* hdr, const BatchJob* jobs, int blocks,
                                 cudaStream_t stream)
{
    k_batch_colbits<<<blocks, K1_WARPS * 32, 0, stream>>>(hdr, jobs);
    return cudaGetLastError();
}

cudaError_t launch_colbits(const uint8_t* mask, const ColGeom& g, int mode,
                           const ColScratch& s, cudaStream_t stream)
{
    const int64_t warps = g.ntiles * (int64_t)g.nG;
    const int64_t blocks = (warps + K1_WARPS - 1) / K1_WARPS;
    const size_t smem = (size_t)K1_WARPS * 2 * colbits_tile_rows(g) * 32 * 4;
    const bool vec = (g.cols % 16 == 0) && ((reinterpret_cast<uintptr_t>(mask) & 15) == 0);
    if (vec)
        k_colbits<true, false><<<(unsigned)blocks, K1_WARPS * 32, smem, stream>>>(mask, g, mode, s, s);
    else
        k_colbits<false, false><<<(unsigned)blocks, K1_WARPS * 32, smem, stream>>>(mask, g, mode, s, s);
    return cudaGetLastError();
}

// Both transforms' summaries from one read of the mask (s: nonzero bytes are
// the sources, s1: zero bytes; s1.C is not written).
cudaError_t launch_colbits_pair(const uint8_t* mask, const ColGeom& g, const ColScratch& s,
                                const ColScratch& s1, cudaStream_t stream)
{
    const int64_t warps = g.ntiles * (int64_t)g.nG;
    const int64_t blocks = (warps + K1_WARPS - 1) / K1_WARPS;
    const size_t smem = (size_t)K1_WARPS * 2 * colbits_tile_rows(g) * 32 * 4;
    const bool vec = (g.cols % 16 == 0) && ((reinterpret_cast<uintptr_t>(mask) & 15) == 0);
    if (vec)
        k_colbits<true, true><<<(unsigned)blocks, K1_WARPS * 32, smem, stream>>>(mask, g, 0, s, s1);
    else
        k_colbits<false, true><<<(unsigned)blocks, K1_WARPS * 32, smem, stream>>>(mask, g, 0, s, s1);
    return cudaGetLastError();
}

}  // namespace edt
