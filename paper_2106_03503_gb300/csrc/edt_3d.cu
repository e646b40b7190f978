// 3-D exact EDT.  Sec. 3.1 of the paper handles a multi-dimensional image one
// axis at a time;
// for a [Dz][H][W] volume this library runs
//   (z) the column pass along z: the volume seen as a 2-D image with Dz rows
//       and H*W columns, handled by the same column-bit kernel as 2-D images,
//       then (plain transforms) k_zoffsets, which writes every voxel's int16
//       offset to its nearest source along z;
//   (y) the lower envelope of Sec. 3.3.1 along y, over f(y') = (z - z')^2 with
//       z' the nearest source along z in column (y', x): for each voxel it
//       records the source (z', y') of its owning parabola, encoded for
//       the x pass (offsets and squared length, see xrec_near);
//   (x) the lower envelope along x over f(x') = (z - z')^2 + (y - y')^2 read
//       from that record, writing D, F = z'*H*W + y'*W + x' and sqrt(D).
// The (z', y') record lives in the caller's F (or D) buffer: the x pass reads
// its rows into shared memory before it overwrites the same rows.
// A y tile (one z, 32 neighbouring x) or x unit (32 consecutive rows) whose
// own distances are all small takes an exact direct search; the others take
// the band engine (edt_engine.cuh) with one line per lane.
#include "edt_engine.cuh"
#include "edt_internal.h"

namespace edt {

constexpr uint32_t PNONE = 0xFFFFFFFFu;

// --- y pass ----------------------------------------------------------------

// y tile data: for each (y, x), d = nearest source z along z minus z (int16,
// YNONE when the column has no source), [YPAD + H + YPAD] rows of YP entries
// (32 used), the pads holding YNONE so that a search may step past either end.
// A row is YP = 40 entries (20 words) apart, so that the 4 x 8 (y, x) patch of
// a warp in the direct search reads 4 rows on disjoint groups of banks (rows
// y .. y+3 start at banks 20y + {0, 20, 8, 28} mod 32), and the 32 lanes of
// one row still read 16 consecutive words.
constexpr short YNONE = 32767;
constexpr int YPAD = DIRECT_MAX_DIST + 2;   // the search below looks one step past its stop
constexpr int YP = 40;

struct LineY {
    const short* gz;         // row y' of this tile at gz[y' * YP] (pads around)
    int lane;
    int z;
    __device__ __forceinline__ bool eval(int k, int& f) const
    {
        const int d = gz[k * YP + lane];
        if (d == YNONE) return false;
        f = d * d;
        return true;
    }
    __device__ __forceinline__ int c(int k) const
    {
        const int d = gz[k * YP + lane];
        return d * d + k * k;
    }
    __device__ __forceinline__ bool eval2(int k, int& f, int& feat) const
    {
        const int d = gz[k * YP + lane];
        if (d == YNONE) return false;
        f = d * d;
        feat = (int)(((uint32_t)(z + d) << 16) | (uint32_t)k);
        return true;
    }
    __device__ __forceinline__ bool is_zero(int k) const { return gz[k * YP + lane] == 0; }
    __device__ __forceinline__ bool chunk_has_source(int j0) const
    {
        bool any = false;
#pragma unroll
        for (int t = 0; t < OC; ++t) any |= gz[(j0 + t) * YP + lane] == 0;
        return any;
    }
    __device__ __forceinline__ int self_feature(int k) const
    {
        return (int)(((uint32_t)z << 16) | (uint32_t)k);
    }
};

// y-pass record of a voxel (z, y, x) whose source in its plane x is
// (z', y', x), written in the form the x pass reads: with dz = z - z', dy =
// y - y' and dz^2 + dy^2 < 128^2 (so both within +-127), bits 31..24 dz,
// 23..16 dy (two's complement), 15 clear and 14..0 dz^2 + dy^2, so that a
// direct search reads a candidate's squared length with one load and a mask;
// otherwise bit 15 set, z' in bits 31..16 and y' (< 2048) in bits 14..0;
// PNONE when the plane has no source.  The voxel's own position (dz = dy = 0)
// is record 0.
__device__ __forceinline__ uint32_t xrec_near(int dz, int dy, int len2)
{
    return ((uint32_t)dz << 24) | (((uint32_t)dy & 0xFFu) << 16) | (uint32_t)len2;
}

struct OutY {
    uint32_t* P;             // record of voxel (z, y, x0 + lane) at P[y * W]
    int W, z;
    bool valid;
    __device__ __forceinline__ void finish() const {}
    __device__ __forceinline__ void store(int j0, int cnt, const int* v, const int* f) const
    {
        if (!valid) return;
#pragma unroll
        for (int t = 0; t < OC; ++t) {
            if (t >= cnt) continue;
            const uint32_t src = (uint32_t)f[t];   // z' << 16 | y'
            uint32_t q = PNONE;
            if (v[t] < 128 * 128)
                q = xrec_near(z - (int)(src >> 16), j0 + t - (int)(src & 0xFFFFu), v[t]);
            else if (v[t] != INT32_MAX)
                q = src | 0x8000u;
            P[(int64_t)(j0 + t) * W] = q;
        }
    }
};

// y tile: z offsets of [YPAD + H + YPAD][YP] (int16), per-warp maxima and
// counts (2 x 32 ints), the direct search's give-up flag (16 bytes), engine
__host__ __device__ static inline size_t ytile_bytes(int H)
{
    return ((size_t)(H + 2 * YPAD) * YP * 2 + 15) & ~size_t(15);
}
__host__ __device__ static inline size_t ypass_smem(int H, int lg, int NW)
{
    return ytile_bytes(H) + 272 + band_smem_bytes(NW, (1 << lg) >> 5);
}

size_t batch_ypass_group_bytes(int H, int lg, int NW) { return ypass_smem(H, lg, NW); }

// z offsets of the nearest source along z of every voxel, written once for
// the y pass: d16[z][y][x] = z' - z (int16; YNONE when the column has no
// source).  A thread takes one column of one band of 32 planes: its word and
// band summary are read once, then one sweep over the planes follows the
// distance to the nearest source at or above each plane step by step and
// finds the one at or below from the word's remaining bits, the nearer taken
// as the column pass takes it (the one above at a tie).  A y tile staged from
// the words would read and decode them once per plane.
__global__ void __launch_bounds__(256)
k_zoffsets(int Dz, int64_t cols, ColScratch s, short* __restrict__ d16)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int zb = blockIdx.y;
    if (p >= cols) return;
    constexpr int BIG = 60000;   // beyond any distance (< 32768) even after 32 steps
    const uint32_t w = __ldg(s.C + (int64_t)zb * cols + p);
    const uint32_t u = __ldg(s.U + (int64_t)zb * cols + p);
    uint32_t up = u & 0xFFFFu, dn = u >> 16;
    if (up == (uint32_t)NONE16 || dn == (uint32_t)NONE16) {
        const uint32_t gab = __ldg(s.GAB + (int64_t)(zb >> s.gs) * cols + p);
        if (up == (uint32_t)NONE16) up = gab & 0xFFFFu;
        if (dn == (uint32_t)NONE16) dn = gab >> 16;
    }
    const int base = 32 * zb;
    const int rows = min(32, Dz - base);
    short* out = d16 + (int64_t)base * cols + p;
    if (w == 0u && up == (uint32_t)NONE16 && dn == (uint32_t)NONE16) {   // no source in the whole column
        for (int r = 0; r < rows; ++r) out[(int64_t)r * cols] = YNONE;
        return;
    }
    // with a source somewhere in the column, every plane has one above or
    // below it, closer than BIG; the one below comes from the word's bits at
    // and after the plane (their lowest), else from past the band
    const int ddout = dn == (uint32_t)NONE16 ? BIG : (int)dn - base;   // from the band's first plane
    int nu = up == (uint32_t)NONE16 ? -BIG : (int)up - (base - 1);    // minus the distance above
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        nu = (w & (1u << r)) ? 0 : nu - 1;
        const uint32_t rest = w >> r;
        const int dd = rest ? __ffs(rest) - 1 : ddout - r;
        if (r < rows) out[(int64_t)r * cols] = (short)(dd < -nu ? dd : nu);
    }
}

// 16-byte copy global -> shared that completes at cp_async_wait_all (the
// copies of a thread are all in flight together and need no registers)
__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    const uint32_t da = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(da), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// The items of one warp: item (jb, g) is rows 4 jb .. 4 jb + 3 and columns
// 8 g .. 8 g + 7 of the tile, and the warp takes items warp, warp + NW, ... of
// the order 4 jb + g.  FIXED (NW a multiple of 4): g is then the same in every
// item of the warp, so that what depends on it stays out of the loop.
// Returns false when a search gave up (CHECK).
template <bool CHECK, bool FIXED>
__device__ __forceinline__ bool ydirect_items(const short* gz, int H, int W, int x0, int z, int64_t plane,
                                              uint32_t* __restrict__ P, int lane, int warp, int NW,
                                              volatile int* abort)
{
    const int nyb = (H + 3) >> 2;
    const int end = FIXED ? nyb : 4 * nyb, step = FIXED ? NW >> 2 : NW;
    for (int it = FIXED ? warp >> 2 : warp; it < end; it += step) {
        if (CHECK && __any_sync(FULL, *abort != 0)) return false;   // the same decision in every lane
        const int jb = FIXED ? it : it >> 2, g = FIXED ? warp & 3 : it & 3;
        const int j = 4 * jb + (lane >> 3), xt = 8 * g + (lane & 7);
        const bool act = j < H && x0 + xt < W;   // a voxel of the tile
        const short* col = gz + xt;
        int best = 0, bk = j, rn2 = 1;
        if (act) {
            const int d0 = col[j * YP];
            best = d0 * d0;
            int r = 1, r2 = 1;
            for (; r2 <= best && (!CHECK || r < DIRECT_MAX_DIST); r += 2, r2 += 4 * r - 4) {
                const int r2b = r2 + 2 * r + 1;
                const int dl = col[(j - r) * YP], dr = col[(j + r) * YP];
                const int dl2 = col[(j - r - 1) * YP], dr2 = col[(j + r + 1) * YP];
                const int cl = dl * dl + r2, cr = dr * dr + r2;
                const int cl2 = dl2 * dl2 + r2b, cr2 = dr2 * dr2 + r2b;
                if (cl < best) { best = cl; bk = j - r; }
                if (cr <= best) { best = cr; bk = j + r; }
                if (cl2 < best) { best = cl2; bk = j - r - 1; }
                if (cr2 <= best) { best = cr2; bk = j + r + 1; }
            }
            rn2 = r2;   // r^2 of the nearest distance not searched
        }
        if (CHECK && __any_sync(FULL, act && rn2 <= best)) {
            *abort = 1;
            return false;
        }
        // a result kept has best < rn2 <= 65^2: |z' - z| <= 64 and |y' - y| <= 65
        if (act) P[(int64_t)z * plane + (int64_t)j * W + x0 + xt] = xrec_near(-col[bk * YP], j - bk, best);
    }
    return true;
}

// Direct search of a y tile: each position searches outward along y (Eq.
// (5) minimised exactly, rightmost y' at a tie, as the hull walk), two steps
// per test of the stop rule (a step past the stop costs at least its r^2,
// more than the best, and changes nothing).  A warp takes patches of 4 y x 8
// x: a search runs as far as the farthest lane of its warp, and neighbours in
// both directions need more alike distances than 32 along x alone.  Without
// CHECK every own offset is at most DIRECT_MAX_DIST, so a search stops by
// r = DIRECT_MAX_DIST + 1 < YPAD and never leaves the padded tile (a pad or a
// column without source costs 32767^2, more than any answer).  With CHECK
// (some own offset larger, or a column without source) the searches stop at
// that distance, and a search still open there makes the whole tile give up
// (returns false; the caller then runs the band engine, which rewrites every
// position with the same value).
template <bool CHECK, class Sync>
__device__ bool ydirect(const short* gz, int H, int W, int x0, int z, int64_t plane, uint32_t* __restrict__ P,
                        int lane, int warp, int NW, volatile int* abort, Sync sync)
{
    if ((NW & 3) == 0)
        ydirect_items<CHECK, true>(gz, H, W, x0, z, plane, P, lane, warp, NW, abort);
    else
        ydirect_items<CHECK, false>(gz, H, W, x0, z, plane, P, lane, warp, NW, abort);
    if (!CHECK) return true;
    sync();
    return *abort == 0;
}

// One y-pass tile: plane z, the 32 columns x0 .. x0+31 (one line per lane),
// NW warps = y segments.  Run by the nthr threads of one engine (tid = thread
// within it, warp = warp within it) over the shared memory at `base`.  The z
// offsets come from d16 (k_zoffsets) when it is given, else from the column
// pass's words and summaries.
template <class Sync>
__device__ void ypass_tile(int H, int W, const ColScratch& s, const short* __restrict__ d16, int lg, int NW,
                           uint32_t* __restrict__ P, int z, int x0, unsigned char* base, int tid, int nthr, int warp,
                           Sync sync)
{
    short* gz = reinterpret_cast<short*>(base) + YPAD * YP;     // row 0 of the tile
    int* wmax = reinterpret_cast<int*>(base + ytile_bytes(H));
    int* wfar = wmax + 32;
    volatile int* abort = wmax + 64;
    const BandSmem sm = carve_band_smem(base + ytile_bytes(H) + 272, NW, (1 << lg) >> 5);
    if (tid == 0) *abort = 0;   // seen by all after the barrier below
    const int lane = tid & 31;
    const int64_t plane = (int64_t)H * W;
    const int zb = z >> 5, zr = z & 31, zG = zb >> s.gs;

    // z offset of the nearest source along z of every (y, x) of the tile, the
    // largest distance among them and how many exceed DIRECT_MAX_DIST
    // (columns past the volume's edge count as 0); the pads hold YNONE.  The
    // offsets come from d16 (copied), or else are decoded from the column
    // pass's words: each thread first loads the words of SU elements, then
    // decodes them, so that SU pairs of loads are in flight at once.
    for (int e = tid; e < YPAD * YP; e += nthr) {
        gz[e - YPAD * YP] = YNONE;
        gz[H * YP + e] = YNONE;
    }
    const uint32_t* Cz = s.C + (int64_t)zb * plane;
    const uint32_t* Uz = s.U + (int64_t)zb * plane;
    const int total = H * 32;
    constexpr int SU = 4;
    int dmax = 0, far = 0;   // largest |offset|, and how many exceed DIRECT_MAX_DIST
    if (d16 && (W & 7) == 0) {
        // 8 offsets per 16-byte chunk (every row starts 16-byte aligned): all
        // of a thread's chunks copied asynchronously at once, chunks past the
        // volume's edge (whole chunks, W being a multiple of 8) set to YNONE;
        // then the largest |offset| over the in-volume chunks
        const short* src = d16 + (int64_t)z * plane + x0;
        const uint32_t none2 = (uint32_t)(uint16_t)YNONE * 0x10001u;
        for (int e = tid; e < H * 4; e += nthr) {
            const int y = e >> 2, xq = (e & 3) * 8;
            if (x0 + xq < W)
                cp_async16(gz + y * YP + xq, src + (int64_t)y * W + xq);
            else
                *reinterpret_cast<uint4*>(gz + y * YP + xq) = make_uint4(none2, none2, none2, none2);
        }
        cp_async_wait_all();
        sync();
        for (int e = tid; e < H * 4; e += nthr) {
            const int y = e >> 2, xq = (e & 3) * 8;
            if (x0 + xq >= W) continue;
            const uint4 v = *reinterpret_cast<const uint4*>(gz + y * YP + xq);
            const uint32_t a[4] = {__vabsss2(v.x), __vabsss2(v.y), __vabsss2(v.z), __vabsss2(v.w)};
            const uint32_t m = __vmaxs2(__vmaxs2(a[0], a[1]), __vmaxs2(a[2], a[3]));
            dmax = max(dmax, (int)max(m & 0xFFFFu, m >> 16));
#pragma unroll
            for (int t = 0; t < 4; ++t)
                far += (int)((a[t] & 0xFFFFu) > (uint32_t)DIRECT_MAX_DIST) + (int)((a[t] >> 16) > (uint32_t)DIRECT_MAX_DIST);
        }
    } else if (d16) {
        // W not a multiple of 8: offset by offset
        const short* src = d16 + (int64_t)z * plane + x0;
        for (int e = tid; e < total; e += nthr) {
            const int y = e >> 5, xl = e & 31;
            int d = YNONE;
            if (x0 + xl < W) {
                d = src[(int64_t)y * W + xl];
                dmax = max(dmax, abs(d));
                far += abs(d) > DIRECT_MAX_DIST;
            }
            gz[y * YP + xl] = (short)d;
        }
    }
    for (int e0 = d16 ? total : tid; e0 < total; e0 += SU * nthr) {
        uint32_t w[SU], u[SU];
#pragma unroll
        for (int i = 0; i < SU; ++i) {
            const int e = e0 + i * nthr, x = x0 + (e & 31);
            w[i] = 0u;
            u[i] = 0u;
            if (e < total && x < W) {
                const int64_t p = (int64_t)(e >> 5) * W + x;
                w[i] = __ldg(Cz + p);
                u[i] = __ldg(Uz + p);
            }
        }
#pragma unroll
        for (int i = 0; i < SU; ++i) {
            const int e = e0 + i * nthr, x = x0 + (e & 31);
            if (e >= total) break;
            int d = YNONE;
            if (x < W) {
                uint32_t up = u[i] & 0xFFFFu, dn = u[i] >> 16;
                if (up == (uint32_t)NONE16 || dn == (uint32_t)NONE16) {
                    const uint32_t gab = s.GAB[(int64_t)zG * plane + (int64_t)(e >> 5) * W + x];
                    if (up == (uint32_t)NONE16) up = gab & 0xFFFFu;
                    if (dn == (uint32_t)NONE16) dn = gab >> 16;
                }
                const int g = nearest_in_column(w[i], zb * 32, zr, (int)up, (int)dn);
                d = g < 0 ? YNONE : g - z;
                dmax = max(dmax, abs(d));
                far += abs(d) > DIRECT_MAX_DIST;
            }
            gz[(e >> 5) * YP + (e & 31)] = (short)d;
        }
    }
    dmax = (int)__reduce_max_sync(FULL, (unsigned)dmax);
    far = (int)__reduce_add_sync(FULL, (unsigned)far);
    if (lane == 0) {
        wmax[warp] = dmax;
        wfar[warp] = far;
    }
    sync();
    far = 0;
    for (int w = 0; w < NW; ++w) {
        dmax = max(dmax, wmax[w]);
        far += wfar[w];
    }

    // every own offset near: the direct search always ends inside the tile;
    // some far: it is tried while at most half of the tile's offsets are far
    // (beyond that the searches mostly run to their limit and give up)
    const int entries = H * min(32, W - x0);
    bool done = false;
    if (dmax <= DIRECT_MAX_DIST)
        done = ydirect<false>(gz, H, W, x0, z, plane, P, lane, warp, NW, abort, sync);
    else if (2 * far <= entries)
        done = ydirect<true>(gz, H, W, x0, z, plane, P, lane, warp, NW, abort, sync);
    if (!done) {
        const OutY out{P + (int64_t)z * plane + x0 + lane, W, z, x0 + lane < W};
        const LineY line{gz, lane, z};
        band_envelope(line, out, sm, H, lg, NW, nullptr, warp, sync);
    }
}

// One block: one z, 32 consecutive x (one line per lane), warps = y segments.
__global__ void __launch_bounds__(1024)
k_ypass3d(int H, int W, ColScratch s, const short* __restrict__ d16, int lg, int NW, uint32_t* __restrict__ P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int xtiles = (W + 31) / 32;
    const int z = blockIdx.x / xtiles;
    const int x0 = (blockIdx.x % xtiles) * 32;
    ypass_tile(H, W, s, d16, lg, NW, P, z, x0, smem, threadIdx.x, blockDim.x, threadIdx.x >> 5, BlockSync());
}

// --- x pass ----------------------------------------------------------------

// the source (z', y') of a record that is not PNONE
__device__ __forceinline__ void xrec_source(uint32_t q, int z, int y, int& zs, int& ys)
{
    if (q & 0x8000u) {
        zs = (int)(q >> 16);
        ys = (int)(q & 0x7FFFu);
    } else {
        zs = z - (int)(int8_t)(q >> 24);
        ys = y - (int)(int8_t)((q >> 16) & 0xFFu);
    }
}

struct LineX {
    const uint32_t* rec;     // this lane's row of records (xrec_near)
    int z, y, H, W;
    bool valid;
    __device__ __forceinline__ int sq(uint32_t q) const
    {
        if (!(q & 0x8000u)) return (int)(q & 0x7FFFu);
        const int dz = z - (int)(q >> 16), dy = y - (int)(q & 0x7FFFu);
        return dz * dz + dy * dy;
    }
    __device__ __forceinline__ bool eval(int k, int& f) const
    {
        if (!valid) return false;
        const uint32_t q = rec[k];
        if (q == PNONE) return false;
        f = sq(q);
        return true;
    }
    __device__ __forceinline__ int c(int k) const { return sq(rec[k]) + k * k; }
    __device__ __forceinline__ bool eval2(int k, int& f, int& feat) const
    {
        if (!valid) return false;
        const uint32_t q = rec[k];
        if (q == PNONE) return false;
        int zs, ys;
        xrec_source(q, z, y, zs, ys);
        f = sq(q);
        feat = (zs * H + ys) * W + k;
        return true;
    }
    __device__ __forceinline__ bool is_zero(int k) const { return rec[k] == 0u; }
    __device__ __forceinline__ bool chunk_has_source(int j0) const
    {
        bool any = false;
#pragma unroll
        for (int t = 0; t < OC; ++t) any |= rec[j0 + t] == 0u;
        return any;
    }
    __device__ __forceinline__ int self_feature(int k) const { return (z * H + y) * W + k; }
};

// x unit: the records of its 32 rows, row rl at xrow(rl) words: the pitch XP
// is a multiple of 32 of at least W + XPAD + 31 words and row rl is shifted by
// 8 (rl & 3) + (rl >> 2) words, so that at any column the 32 rows fall on 32
// distinct banks (lane = row reads of the hull engine) and the 4 rows of a
// group 8 banks apart (the 4 x 8 patches of the direct search).  At least
// XPAD words of pad lie before every row and after the last.  Then per-warp
// maxima (32 ints), the direct search's give-up flag (16 bytes) and the
// engine.
constexpr int XPAD = 96;
__host__ __device__ static inline int xpass_pitch(int W) { return (W + XPAD + 31 + 31) & ~31; }
__host__ __device__ static inline int xrow(int rl, int XP) { return XPAD + rl * XP + 8 * (rl & 3) + (rl >> 2); }
__host__ __device__ static inline size_t xpass_rec_bytes(int W)
{
    return ((size_t)(XPAD + 32 * xpass_pitch(W)) * 4 + 15) & ~size_t(15);
}
__host__ __device__ static inline size_t xpass_smem(int W, int lg, int NW)
{
    return xpass_rec_bytes(W) + 144 + band_smem_bytes(NW, (1 << lg) >> 5);
}

size_t batch_xpass_group_bytes(int W, int lg, int NW) { return xpass_smem(W, lg, NW); }

// The items of one warp: item (jb, g) is rows 4 g .. 4 g + 3 of the unit and
// columns 8 jb .. 8 jb + 7, and the warp takes items warp, warp + NW, ... of
// the order 8 jb + g.  FIXED (NW a multiple of 8): g is then the same in
// every item of the warp, so that the rows' pointers and output offsets stay
// out of the loop.  Returns false when a search gave up (CHECK).
template <bool CHECK, bool FIXED>
__device__ __forceinline__ bool xdirect_items(const uint32_t* rec, int XP, int H, int W, int64_t row0,
                                              int64_t nrows, int32_t* D, int32_t* F, float* dist, int lane,
                                              int warp, int NW, volatile int* abort)
{
    const int nj = (W + 7) >> 3;
    const int end = FIXED ? nj : 8 * nj, step = FIXED ? NW >> 3 : NW;
    for (int it = FIXED ? warp >> 3 : warp; it < end; it += step) {
        if (CHECK && __any_sync(FULL, *abort != 0)) return false;   // the same decision in every lane
        const int jb = FIXED ? it : it >> 3, g = FIXED ? warp & 7 : it & 7;
        const int rl = 4 * g + (lane >> 3), j = 8 * jb + (lane & 7);
        const int64_t row = row0 + rl;
        const bool act = row < nrows && j < W;
        const uint32_t* rr = rec + xrow(rl, XP);
        int best = 0, bk = j, rn2 = 1;
        const uint16_t* c16 = reinterpret_cast<const uint16_t*>(rr);   // bits 15..0 of record k at c16[2 k]
        if (act) {
            // one key per candidate k, cost * 256 + 128 - (k - j) (costs
            // below 2^17, |k - j| <= 91): the least key has the least cost
            // and, at a tie, the rightmost k; a step's four keys fold in a
            // tree of minimums
            int key = ((int)c16[2 * j] << 8) + 128;
            int r = 1, r2 = 1;
            for (; r2 <= (key >> 8) && (!CHECK || r < 90); r += 2, r2 += 4 * r - 4) {
                const int t = (r2 << 8) + 128, t2 = t + ((2 * r + 1) << 8);
                const int kl = ((int)c16[2 * (j - r)] << 8) + t + r, kr = ((int)c16[2 * (j + r)] << 8) + t - r;
                const int kl2 = ((int)c16[2 * (j - r - 1)] << 8) + t2 + r + 1;
                const int kr2 = ((int)c16[2 * (j + r + 1)] << 8) + t2 - r - 1;
                key = min(key, min(min(kl, kr), min(kl2, kr2)));
            }
            best = key >> 8;
            bk = j + 128 - (key & 0xFF);
            rn2 = r2;   // r^2 of the nearest distance not searched
        }
        if (CHECK && __any_sync(FULL, act && rn2 <= best)) {
            *abort = 1;
            return false;
        }
        if (act) {
            const uint32_t p = rr[bk];
            const int dz = (int)(int8_t)(p >> 24), dy = (int)(int8_t)((p >> 16) & 0xFFu);
            // row = z * H + y; every term below 2^31 (the volume has fewer
            // voxels, and |dz| < Dz, |dy| < H)
            const int rowW = (int)(row * W);
            const int64_t q = (int64_t)rowW + j;
            if (D) D[q] = best;
            if (F) F[q] = rowW + bk - (dz * H + dy) * W;
            if (dist) dist[q] = sqrt_rn_int(best);
        }
    }
    return true;
}

// Direct search of an x unit: each position searches outward along its row
// (Eq. (5) minimised exactly, rightmost x' at a tie, as the hull walk), two
// steps per test of the stop rule (a step past the stop costs at least its
// r^2, more than the best, and changes nothing), a candidate's cost being its
// record's bits 15..0 (xrec_near).  A warp takes patches of 4 rows x 8 x: a
// search runs as far as the farthest lane of its warp, and neighbours in both
// directions need more alike distances than 32 along x alone.  Without CHECK
// every record is one with offsets, its bits 15..0 the squared length and at
// most 2 * 64^2, so a search stops by r = 91 < XPAD and every look past a
// row's ends reads a pad.  With CHECK (longer records, escape records or
// planes without source) bits 15..0 of an escape record or of PNONE are 32768
// or more, and its true cost 128^2 or more; the searches stop at r = 91, and
// a search still open there (its best 91^2 or more, so any record whose bits
// 15..0 are not its true cost could still matter) makes the whole unit give
// up (returns false; the caller then runs the band engine).
template <bool CHECK, class Sync>
__device__ bool xdirect(const uint32_t* rec, int XP, int H, int W, int64_t row0, int64_t nrows, int32_t* D,
                        int32_t* F, float* dist, int lane, int warp, int NW, volatile int* abort, Sync sync)
{
    if ((NW & 7) == 0)
        xdirect_items<CHECK, true>(rec, XP, H, W, row0, nrows, D, F, dist, lane, warp, NW, abort);
    else
        xdirect_items<CHECK, false>(rec, XP, H, W, row0, nrows, D, F, dist, lane, warp, NW, abort);
    if (!CHECK) return true;
    sync();
    return *abort == 0;
}

// One x-pass unit: the 32 rows (z, y) starting at row0 of the Dz*H rows (one
// per lane), NW warps = x segments; run by one engine as ypass_tile.
template <class Sync>
__device__ void xpass_rows(int Dz, int H, int W, int lg, int NW, const uint32_t* P, int32_t* D, int32_t* F,
                           float* dist, int64_t row0, unsigned char* base, int tid, int nthr, int warp, Sync sync)
{
    const int XP = xpass_pitch(W);
    uint32_t* rec = reinterpret_cast<uint32_t*>(base);   // row rl at rec[xrow(rl, XP)]
    int* wmax = reinterpret_cast<int*>(base + xpass_rec_bytes(W));
    volatile int* abort = wmax + 32;
    const BandSmem sm = carve_band_smem(base + xpass_rec_bytes(W) + 144, NW, (1 << lg) >> 5);
    if (tid == 0) *abort = 0;   // seen by all after the barrier below
    const int lane = tid & 31;
    const int64_t nrows = (int64_t)Dz * H;

    // the pads (before row 0, between rows, after the last) cost 0xFFFF to
    // the direct search below, more than any answer it accepts
    for (int g = warp; g <= 32; g += NW) {
        const int st = g == 0 ? 0 : xrow(g - 1, XP) + W;
        const int en = g == 32 ? xrow(31, XP) + W + XPAD : xrow(g, XP);
        for (int a = st + lane; a < en; a += 32) rec[a] = 0xFFFFu;
    }
    // the rows' records, and the largest squared length among them (bits
    // 15..0: 32768 or more for an escape record or PNONE; rows past the
    // volume's end count as 0), RU loads in flight per thread
    constexpr int RU = 4;
    int dmax = 0;
    for (int rl0 = 0; rl0 < 32; rl0 += RU) {
        for (int k = tid; k < W; k += nthr) {
            uint32_t p[RU];
#pragma unroll
            for (int i = 0; i < RU; ++i) p[i] = row0 + rl0 + i < nrows ? P[(row0 + rl0 + i) * W + k] : PNONE;
#pragma unroll
            for (int i = 0; i < RU; ++i) {
                if (row0 + rl0 + i < nrows) dmax = max(dmax, (int)(p[i] & 0xFFFFu));
                rec[xrow(rl0 + i, XP) + k] = p[i];
            }
        }
    }
    dmax = (int)__reduce_max_sync(FULL, (unsigned)dmax);
    if (lane == 0) wmax[warp] = dmax;
    sync();
    for (int w = 0; w < NW; ++w) dmax = max(dmax, wmax[w]);

    const bool done = dmax <= 2 * DIRECT_MAX_DIST * DIRECT_MAX_DIST
                          ? xdirect<false>(rec, XP, H, W, row0, nrows, D, F, dist, lane, warp, NW, abort, sync)
                          : xdirect<true>(rec, XP, H, W, row0, nrows, D, F, dist, lane, warp, NW, abort, sync);
    if (done) return;

    const int64_t row = row0 + lane;
    LineX line;
    line.rec = rec + xrow(lane, XP);
    line.z = (int)(row / H);
    line.y = (int)(row % H);
    line.H = H;
    line.W = W;
    line.valid = row < nrows;
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
            ypass_tile(J.H, J.W, J.s, nullptr, J.lg, NW, reinterpret_cast<uint32_t*>(J.F), (int)(unit / xtiles),
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

cudaError_t launch_zoffsets(int Dz, int H, int W, const ColGeom& g, const ColScratch& s, short* d16,
                            cudaStream_t stream)
{
    const int64_t cols = (int64_t)H * W;
    const dim3 grid((unsigned)((cols + 255) / 256), (unsigned)g.nb);
    k_zoffsets<<<grid, 256, 0, stream>>>(Dz, cols, s, d16);
    return cudaGetLastError();
}

cudaError_t launch_ypass3d(int Dz, int H, int W, const ColGeom& g,
                           const ColScratch& s, const short* d16, uint32_t* P, cudaStream_t stream)
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
    k_ypass3d<<<blocks, NW * 32, ypass_smem(H, lg, NW), stream>>>(H, W, s, d16, lg, NW, P);
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
