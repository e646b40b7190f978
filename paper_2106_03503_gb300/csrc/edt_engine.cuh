// Device building blocks of libedt (sm_103a): the lower envelope of parabolas
// along many lines at once (Sec. 3.3.1 of Strutz, "The Distance Transform and
// its Computation"), the bit tricks of the column pass (Sec. 3.1) and the
// correctly rounded float32 square root.
//
// Lower envelope as a lower convex hull.  For one line, parabola k is
// D_k(j) = f(k) + (j - k)^2 (Eq. (5)).  Expanding, D_k(j) = j^2 - 2jk + c_k
// with c_k = f(k) + k^2, so the lower envelope over j is the lower convex
// hull of the points (k, c_k): parabola t is hidden between p < t < m exactly
// when the intersection of t and m (Eq. (6)) does not lie to the right of the
// intersection of p and t, i.e. slope(t, m) <= slope(p, t).  With positive
// denominators this is the integer test
//     (c_m - c_t) * (t - p) <= (c_t - c_p) * (m - t)
// evaluated in 64-bit, so no division and no rounding is needed.  (The
// paper's listing compares ceilings of the intersections instead; both give
// the same lower envelope at integer positions, ties aside.)
//
// Work split ("band engine").  A block processes 32 lines together, lane l
// of every warp working on line l, and the NW warps split the positions of
// the lines into NW segments of SEG = 2^lg positions.  So all lanes of a warp
// step through the same position k at the same time: data shared by the 32
// lines at position k (the column words of a band of 32 rows, say) is one
// broadcast shared-memory read, and only the per-line arithmetic differs.
//   (1) Each (segment, line) builds the hull of its own positions with the
//       paper's stack algorithm (pop while the top is hidden, then push); the
//       stack is a bit set in shared memory (bit = position is on the hull)
//       plus the top two entries in registers.
//   (2) log2(NW) rounds of pairwise merges join neighbouring segments' hulls,
//       every lane on its own line: for two x-separated lower hulls the joint
//       hull keeps a prefix of the left and a suffix of the right one, found
//       by the classic bridge walk (drop the left top while it is hidden
//       between its predecessor and the right bottom; drop the right bottom
//       while it is hidden between the left top and its successor).
//   (3) The warps fill the positions in units taken in turn from a shared
//       counter (so that costly parts of the lines are spread over all
//       warps): the owner of a position is the hull member with the smallest
//       value there; owners move right monotonically with the position, and
//       along the hull the values at a fixed position are unimodal, so a walk
//       finds them.  Each lane writes
//       its values 8 positions at a time: a row line as one 32-byte store
//       per array (a whole sector; 16-byte or single stores where the row
//       layout does not allow it) or, for rows up to 2048 wide, through a TMA
//       box of the warp's 32 rows; a column line as single stores that are
//       coalesced across the 32 neighbouring lines.
#pragma once

#include <cstdint>
#include <climits>
#include <cuda.h>
#include <cuda_runtime.h>

namespace edt {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int NONE16 = 0xFFFF;       // "no source" in 16-bit row fields
constexpr int OUT_CHUNK = 8;         // columns per lane per output round

// ---------------------------------------------------------------------------
// Correctly rounded float32 square root of a non-negative int32.
// The float estimate s = sqrtf((float)D) is within a couple of ulps; it is
// then moved to the float nearest to sqrt(D) with exact integer midpoint
// tests: for s = M * 2^E (M the 24-bit significand), the midpoint to the next
// float is (2M + 1) * 2^(E-1), and D >= mid^2 <=> D * 2^(2-2E) >= (2M+1)^2,
// both sides exact in 64 bits (about 4 M^2 < 2^52).  sqrt(D) is never a
// midpoint (it is an integer below 2^16 or irrational).  D = INT32_MAX means
// "no source" and maps to +infinity.
__device__ __forceinline__ float sqrt_rn_int(int32_t D)
{
    if (D == INT32_MAX) return __int_as_float(0x7F800000);
    if (D <= 0) return 0.0f;
    float s = sqrtf((float)D);
#pragma unroll 1
    for (int it = 0; it < 4; ++it) {
        const uint32_t bits = __float_as_uint(s);
        const int E = (int)(bits >> 23) - 150;                 // s = M * 2^E
        const uint64_t M = (uint64_t)((bits & 0x7FFFFFu) | 0x800000u);
        const uint64_t X = (uint64_t)(uint32_t)D << (2 - 2 * E);   // D*2^(2-2E)
        const uint64_t up = (2 * M + 1) * (2 * M + 1);
        if (X >= up) { s = __uint_as_float(bits + 1); continue; }
        bool below;
        if (M > 0x800000u) {
            below = X < (2 * M - 1) * (2 * M - 1);
        } else {  // s is a power of two: the float below is half an ulp away
            below = (X << 2) < (4 * M - 1) * (4 * M - 1);
        }
        if (below) { s = __uint_as_float(bits - 1); continue; }
        break;
    }
    return s;
}

// ---------------------------------------------------------------------------
// Column-pass helpers (Sec. 3.1).  A column-bit word holds 32 consecutive
// rows of one column (bit r = row base+r is a source).  The nearest source
// at or above row `r` of the word is its highest set bit among bits 0..r; at
// or below, its lowest set bit among r..31.

// Nearest source row to row i = base + r given the word and the nearest
// sources strictly above / below the word (NONE16 = none).  Returns the row,
// or -1 when the column has no source; ties go to the upper source.
__device__ __forceinline__ int nearest_in_column(uint32_t w, int base, int r,
                                                 int up_outside, int dn_outside)
{
    const uint32_t a = w & (FULL >> (31 - r));
    const int up = a ? base + 31 - __clz(a) : up_outside;
    const uint32_t b = w >> r;
    const int dn = b ? base + r + __ffs(b) - 1 : dn_outside;
    const int i = base + r;
    const int du = (up == NONE16) ? INT_MAX : i - up;
    const int dd = (dn == NONE16) ? INT_MAX : dn - i;
    if (du == INT_MAX && dd == INT_MAX) return -1;
    return (du <= dd) ? up : dn;
}

// ---------------------------------------------------------------------------
// Band engine.

constexpr int OC = 8;   // positions per fill round (tile width)

struct BandSmem {
    uint32_t* hb;   // [NW][SEGW][32] hull bits: segment, word, lane
    int* lo;        // [NW][32] first hull member of (segment, line), -1 none
    int* hi;        // [NW][32] last hull member
    int* ctr;       // next fill unit to hand out
};

__host__ __device__ inline size_t band_smem_bytes(int NW, int SEGW)
{
    return (size_t)NW * SEGW * 32 * 4 + (size_t)NW * 64 * 4 + 16;
}

__device__ __forceinline__ BandSmem carve_band_smem(unsigned char* base, int NW, int SEGW)
{
    BandSmem s;
    s.hb = reinterpret_cast<uint32_t*>(base);
    s.lo = reinterpret_cast<int*>(base + (size_t)NW * SEGW * 32 * 4);
    s.hi = s.lo + NW * 32;
    s.ctr = s.hi + NW * 32;
    return s;
}

// Positions per fill unit: about four units per warp, a multiple of 32
// between 32 and 256.
__host__ __device__ inline int band_fill_unit(int n, int NW)
{
    int u = (n / (4 * NW) + 31) & ~31;
    return u < 32 ? 32 : (u > 256 ? 256 : u);
}

// Segment length (power of two, >= 32) and segment count for a line of n
// positions split over at most max_nw warps.
__host__ __device__ inline int band_seg_log2(int n, int max_nw)
{
    int lg = 5;
    while ((((n + (1 << lg) - 1) >> lg)) > max_nw) ++lg;
    return lg;
}

// t is hidden between p < t < m on the hull of points (k, c_k).  With
// c_k = f(k) + k^2 and a = t - p, b = m - t, c = m - p this is
// c f(t) - b f(p) - a f(m) - abc >= 0: the separating-line test of Maurer et
// al. (the alternative the paper's Sec. 4 names), with >= in place of >.
// The two differ only where the three parabolas meet in one point, which
// changes a feature at a tie and never a distance.
__device__ __forceinline__ bool hidden(int p, int cp, int t, int ct, int m, int cm)
{
    return (long long)(cm - ct) * (long long)(t - p) <=
           (long long)(ct - cp) * (long long)(m - t);
}

// Previous / next hull member of (segment s, this lane) strictly before /
// after position x of that segment; -1 when none.
__device__ __forceinline__ int seg_prev(const uint32_t* hb, int s, int lg, int SEGW, int lane, int x)
{
    const int off = x - (s << lg);
    int w = off >> 5;
    const uint32_t* base = hb + (size_t)s * SEGW * 32 + lane;
    uint32_t m = base[w * 32] & ((1u << (off & 31)) - 1u);
    while (!m) {
        if (--w < 0) return -1;
        m = base[w * 32];
    }
    return (s << lg) + w * 32 + 31 - __clz(m);
}
__device__ __forceinline__ int seg_next(const uint32_t* hb, int s, int lg, int SEGW, int lane, int x)
{
    const int off = x - (s << lg);
    int w = off >> 5;
    const int b = off & 31;
    const uint32_t* base = hb + (size_t)s * SEGW * 32 + lane;
    uint32_t m = (b == 31) ? 0u : (base[w * 32] & (0xFFFFFFFEu << b));
    while (!m) {
        if (++w >= SEGW) return -1;
        m = base[w * 32];
    }
    return (s << lg) + w * 32 + __ffs(m) - 1;
}

// Join the hulls of segments [a0, b0) and [b0, b1) of this lane's line.
template <class Line>
__device__ void band_bridge(const Line& line, const BandSmem& sm, int lg, int SEGW, int lane,
                            int a0, int b0, int b1)
{
    int* lo = sm.lo + lane;
    int* hi = sm.hi + lane;
    int la = b0 - 1;
    while (la >= a0 && hi[la * 32] < 0) --la;
    int lb = b0;
    while (lb < b1 && lo[lb * 32] < 0) ++lb;
    while (la >= a0 && lb < b1) {
        const int x1 = hi[la * 32];
        const int y1 = lo[lb * 32];
        int x0 = seg_prev(sm.hb, la, lg, SEGW, lane, x1);
        int lx0 = la;
        if (x0 < 0) {
            int l = la - 1;
            while (l >= a0 && hi[l * 32] < 0) --l;
            if (l >= a0) { x0 = hi[l * 32]; lx0 = l; }
        }
        int y2 = seg_next(sm.hb, lb, lg, SEGW, lane, y1);
        const bool y2_same = (y2 >= 0);
        if (y2 < 0) {
            int l = lb + 1;
            while (l < b1 && lo[l * 32] < 0) ++l;
            if (l < b1) y2 = lo[l * 32];
        }
        const int cx1 = line.c(x1);
        const int cy1 = line.c(y1);
        if (x0 >= 0 && hidden(x0, line.c(x0), x1, cx1, y1, cy1)) {
            const int off = x1 - (la << lg);
            sm.hb[((size_t)la * SEGW + (off >> 5)) * 32 + lane] &= ~(1u << (off & 31));
            if (lx0 == la) {
                hi[la * 32] = x0;
            } else {
                hi[la * 32] = -1;
                lo[la * 32] = -1;
                la = lx0;
            }
            continue;
        }
        if (y2 >= 0 && hidden(x1, cx1, y1, cy1, y2, line.c(y2))) {
            const int off = y1 - (lb << lg);
            sm.hb[((size_t)lb * SEGW + (off >> 5)) * 32 + lane] &= ~(1u << (off & 31));
            if (y2_same) {
                lo[lb * 32] = y2;
            } else {
                lo[lb * 32] = -1;
                hi[lb * 32] = -1;
                ++lb;
                while (lb < b1 && lo[lb * 32] < 0) ++lb;
            }
            continue;
        }
        break;
    }
}

// Successor / predecessor of hull member x on this lane's merged line hull;
// nem = bit mask of segments holding members.
__device__ __forceinline__ int band_next(const BandSmem& sm, int lg, int SEGW, int lane,
                                         uint32_t nem, int x)
{
    const int s = x >> lg;
    const int y = seg_next(sm.hb, s, lg, SEGW, lane, x);
    if (y >= 0) return y;
    const uint32_t later = (s >= 31) ? 0u : (nem & (0xFFFFFFFEu << s));
    return later ? sm.lo[(__ffs(later) - 1) * 32 + lane] : -1;
}
__device__ __forceinline__ int band_prev(const BandSmem& sm, int lg, int SEGW, int lane,
                                         uint32_t nem, int x)
{
    const int s = x >> lg;
    const int y = seg_prev(sm.hb, s, lg, SEGW, lane, x);
    if (y >= 0) return y;
    const uint32_t earlier = nem & ((1u << s) - 1u);
    return earlier ? sm.hi[(31 - __clz(earlier)) * 32 + lane] : -1;
}

// Barrier of the NW warps that share one band engine (the whole block; a
// block running several engines side by side passes its own barrier).
struct BlockSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// Barrier of one band engine of a block that runs several side by side:
// named barrier `id` (1 + the engine's index; 0 is __syncthreads) over its
// nthreads threads, or a warp barrier for a one-warp engine.
struct GroupSync {
    int id, nthreads;
    __device__ __forceinline__ void operator()() const
    {
        if (nthreads <= 32) __syncwarp();
        else asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
    }
};

// Cursor over the merged hull of this lane's line, moving right: the hull
// word that holds the last returned member stays in a register.
struct HullCursor {
    int seg, word;     // position of `bits`
    uint32_t bits;     // remaining (not yet returned) members of that word
};

__device__ __forceinline__ void cursor_at(HullCursor& hc, const BandSmem& sm, int lg, int SEGW,
                                          int lane, int x)
{
    // position the cursor just after member (or position) x
    const int s = x >> lg;
    const int off = x - (s << lg);
    hc.seg = s;
    hc.word = off >> 5;
    const uint32_t w = sm.hb[((size_t)s * SEGW + hc.word) * 32 + lane];
    const int b = off & 31;
    hc.bits = (b == 31) ? 0u : (w & (0xFFFFFFFEu << b));
}

__device__ __forceinline__ int cursor_next(HullCursor& hc, const BandSmem& sm, int lg, int SEGW,
                                           int lane, uint32_t nem)
{
    for (;;) {
        if (hc.bits) {
            const int t = __ffs(hc.bits) - 1;
            hc.bits &= hc.bits - 1;
            return (hc.seg << lg) + hc.word * 32 + t;
        }
        if (++hc.word >= SEGW) {
            const uint32_t later = (hc.seg >= 31) ? 0u : (nem & (0xFFFFFFFEu << hc.seg));
            if (!later) return -1;
            hc.seg = __ffs(later) - 1;
            hc.word = 0;
        }
        hc.bits = sm.hb[((size_t)hc.seg * SEGW + hc.word) * 32 + lane];
    }
}

__device__ __forceinline__ bool aligned16(const void* p)
{
    return (reinterpret_cast<uintptr_t>(p) & 15) == 0;
}

// One 32-byte store (sm_100 and later): 8 consecutive words at a 32-byte
// aligned address, a whole sector in one instruction.
__device__ __forceinline__ void st_v8(void* q, int a0, int a1, int a2, int a3, int a4, int a5, int a6,
                                      int a7)
{
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                 :: "l"(q), "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(a4), "r"(a5), "r"(a6), "r"(a7)
                 : "memory");
}

// Widest vector store every row chunk of OC words of all arrays allows:
// 2 = 32-byte stores (W % 8 == 0, arrays 32-byte aligned), 1 = 16-byte stores
// (W % 4 == 0, 16-byte aligned), 0 = single words.  NULL arrays do not count.
__device__ __forceinline__ int row_vec_width(int W, const void* D, const void* F, const void* dist)
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(D) | reinterpret_cast<uintptr_t>(F) |
                        reinterpret_cast<uintptr_t>(dist);
    if (W % 8 == 0 && (a & 31) == 0) return 2;
    if (W % 4 == 0 && (a & 15) == 0) return 1;
    return 0;
}

// Output of one row (this lane's): 8 columns at a time, as one 32-byte or two
// 16-byte stores per array when the row layout allows it.
struct RowOut {
    int32_t* D;
    int32_t* F;
    float* dist;
    int64_t rowoff;          // row * W
    bool valid;              // row < H
    int vec;                 // row_vec_width of the arrays
    __device__ __forceinline__ void finish() const {}
    __device__ __forceinline__ void store(int j0, int cnt, const int* v, const int* f) const
    {
        if (!valid) return;
        const int64_t i = rowoff + j0;
        if (vec == 2 && cnt == OC) {
            if (D) st_v8(D + i, v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7]);
            if (F) st_v8(F + i, f[0], f[1], f[2], f[3], f[4], f[5], f[6], f[7]);
            if (dist) {
                int r[OC];
#pragma unroll
                for (int t = 0; t < OC; ++t) r[t] = __float_as_int(sqrt_rn_int(v[t]));
                st_v8(dist + i, r[0], r[1], r[2], r[3], r[4], r[5], r[6], r[7]);
            }
            return;
        }
        if (vec == 1 && cnt == OC) {
            if (D) {
                reinterpret_cast<int4*>(D + i)[0] = make_int4(v[0], v[1], v[2], v[3]);
                reinterpret_cast<int4*>(D + i)[1] = make_int4(v[4], v[5], v[6], v[7]);
            }
            if (F) {
                reinterpret_cast<int4*>(F + i)[0] = make_int4(f[0], f[1], f[2], f[3]);
                reinterpret_cast<int4*>(F + i)[1] = make_int4(f[4], f[5], f[6], f[7]);
            }
            if (dist) {
                reinterpret_cast<float4*>(dist + i)[0] =
                    make_float4(sqrt_rn_int(v[0]), sqrt_rn_int(v[1]), sqrt_rn_int(v[2]), sqrt_rn_int(v[3]));
                reinterpret_cast<float4*>(dist + i)[1] =
                    make_float4(sqrt_rn_int(v[4]), sqrt_rn_int(v[5]), sqrt_rn_int(v[6]), sqrt_rn_int(v[7]));
            }
            return;
        }
#pragma unroll
        for (int t = 0; t < OC; ++t) {
            if (t < cnt) {
                if (D) D[i + t] = v[t];
                if (F) F[i + t] = f[t];
                if (dist) dist[i + t] = sqrt_rn_int(v[t]);
            }
        }
    }
};

// Row output through the tensor memory accelerator: the warp's 32 rows x 8
// columns are staged in shared memory (1 KB per array) and written by one
// cp.async.bulk.tensor.2d store per array, so that the 32 row segments leave
// the SM as whole 32-byte sectors without going through the load/store unit.
// The tensor maps (D, F, dist; a NULL map pointer = array not written) view
// the output as [rows][W] int32 / float32 with a box of 8 x 32.
struct TmaRowOut {
    const CUtensorMap* mD;
    const CUtensorMap* mF;
    const CUtensorMap* mS;
    int* stage;              // this warp's 3 x 32 x 8 staging words
    int row0;                // first row of the box (the block's first line)
    int lane;
    __device__ __forceinline__ void issue(const CUtensorMap* m, const int* buf, int x) const
    {
        const uint32_t sa = (uint32_t)__cvta_generic_to_shared(buf);
        asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
                     :: "l"(m), "r"(x), "r"(row0), "r"(sa) : "memory");
    }
    __device__ __forceinline__ void store(int j0, int cnt, const int* v, const int* f) const
    {
        if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        __syncwarp();
        int* sD = stage;                       // arrays present, back to back
        int* sF = sD + (mD ? 32 * OC : 0);
        int* sS = sF + (mF ? 32 * OC : 0);
        if (mD) {
            reinterpret_cast<int4*>(sD + lane * OC)[0] = make_int4(v[0], v[1], v[2], v[3]);
            reinterpret_cast<int4*>(sD + lane * OC)[1] = make_int4(v[4], v[5], v[6], v[7]);
        }
        if (mF) {
            reinterpret_cast<int4*>(sF + lane * OC)[0] = make_int4(f[0], f[1], f[2], f[3]);
            reinterpret_cast<int4*>(sF + lane * OC)[1] = make_int4(f[4], f[5], f[6], f[7]);
        }
        if (mS) {
            reinterpret_cast<float4*>(sS + lane * OC)[0] =
                make_float4(sqrt_rn_int(v[0]), sqrt_rn_int(v[1]), sqrt_rn_int(v[2]), sqrt_rn_int(v[3]));
            reinterpret_cast<float4*>(sS + lane * OC)[1] =
                make_float4(sqrt_rn_int(v[4]), sqrt_rn_int(v[5]), sqrt_rn_int(v[6]), sqrt_rn_int(v[7]));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0 && cnt > 0) {   // never a box that starts past the row end
            if (mD) issue(mD, sD, j0);
            if (mF) issue(mF, sF, j0);
            if (mS) issue(mS, sS, j0);
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
    }
    __device__ __forceinline__ void finish() const
    {
        if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        __syncwarp();
    }
};

// Fill positions [a, b) of this lane's line from its merged hull.  cur = owner
// of the current position with value fo + (j - cur)^2 and feature featcur;
// nxt = the next hull member (fnxt, featnxt).  A source position owns itself
// (value 0); after a run of sources the walk resumes from the last source of
// the run.  Stores go out OC positions at a time (a is a multiple of OC).
template <class Line, class Out>
__device__ void band_fill(const Line& line, const Out& out, const BandSmem& sm, int lg, int SEGW,
                          int lane, uint32_t nem, const unsigned char* full, int a, int b)
{
    int cur = -1, fo = 0, featcur = -1, nxt = -1, fnxt = 0, featnxt = -1;
    bool need_next = false;
    HullCursor hc{0, 0, 0u};
    if (nem) {
        cur = band_prev(sm, lg, SEGW, lane, nem, a);   // last member before a
        if (cur < 0) cur = sm.lo[(__ffs(nem) - 1) * 32 + lane];
        line.eval(cur, fo);
        for (;;) {  // walk left while strictly better at a
            const int p = band_prev(sm, lg, SEGW, lane, nem, cur);
            if (p < 0) break;
            int fp;
            line.eval(p, fp);
            if ((long long)fp + (long long)(a - p) * (a - p) <
                (long long)fo + (long long)(a - cur) * (a - cur)) {
                cur = p;
                fo = fp;
            } else {
                break;
            }
        }
        line.eval2(cur, fo, featcur);
        need_next = true;
    }
    const int nq = (b - a + OC - 1) / OC;
    for (int q = 0; q < nq; ++q) {
        int v[OC], ft[OC];
        const int j0 = a + q * OC;
        const bool bulk = full && j0 + OC <= b && full[j0 >> 5] && cur >= 0;
        // whole chunk and no line (of those not in the bulk case) has a source
        // in it; every lane takes part in the vote
        const bool clear = j0 + OC <= b && !__any_sync(FULL, !bulk && cur >= 0 && line.chunk_has_source(j0));
        if (bulk) {
            // every line is a source at every position of this chunk
#pragma unroll
            for (int t = 0; t < OC; ++t) {
                v[t] = 0;
                ft[t] = line.self_feature(j0 + t);
            }
            cur = j0 + OC - 1;
            fo = 0;
            featcur = ft[OC - 1];
            need_next = true;
        } else if (clear) {
            // no line has a source in this chunk: start from the owner at j0
            // and take the minimum with every later hull member that beats
            // (or ties) its predecessor at the chunk's last position -- the
            // owners of the chunk's positions are exactly those members, and
            // visiting them left to right with "<=" keeps the rightmost owner
            // at a tie, as the walk below does
#pragma unroll
            for (int t = 0; t < OC; ++t) {
                v[t] = INT32_MAX;
                ft[t] = -1;
            }
            if (cur >= 0) {
                if (need_next) {
                    cursor_at(hc, sm, lg, SEGW, lane, cur);
                    nxt = cursor_next(hc, sm, lg, SEGW, lane, nem);
                    if (nxt >= 0) line.eval2(nxt, fnxt, featnxt);
                    need_next = false;
                }
#pragma unroll
                for (int t = 0; t < OC; ++t) {
                    const int d = j0 + t - cur;
                    v[t] = fo + d * d;
                    ft[t] = featcur;
                }
                const int je = j0 + OC - 1;
                while (nxt >= 0 && fnxt + (je - nxt) * (je - nxt) <= fo + (je - cur) * (je - cur)) {
#pragma unroll
                    for (int t = 0; t < OC; ++t) {
                        const int d = j0 + t - nxt;
                        const int val = fnxt + d * d;
                        if (val <= v[t]) {
                            v[t] = val;
                            ft[t] = featnxt;
                        }
                    }
                    cur = nxt;
                    fo = fnxt;
                    featcur = featnxt;
                    nxt = cursor_next(hc, sm, lg, SEGW, lane, nem);
                    if (nxt >= 0) line.eval2(nxt, fnxt, featnxt);
                }
            }
        } else {
#pragma unroll
            for (int t = 0; t < OC; ++t) {
                const int j = j0 + t;
                v[t] = INT32_MAX;
                ft[t] = -1;
                if (j < b && cur >= 0) {
                    if (line.is_zero(j)) {
                        cur = j;
                        fo = 0;
                        featcur = line.self_feature(j);
                        need_next = true;
                        v[t] = 0;
                        ft[t] = featcur;
                        continue;
                    }
                    if (need_next) {
                        cursor_at(hc, sm, lg, SEGW, lane, cur);
                        nxt = cursor_next(hc, sm, lg, SEGW, lane, nem);
                        if (nxt >= 0) line.eval2(nxt, fnxt, featnxt);
                        need_next = false;
                    }
                    while (nxt >= 0 && fnxt + (j - nxt) * (j - nxt) <= fo + (j - cur) * (j - cur)) {
                        cur = nxt;
                        fo = fnxt;
                        featcur = featnxt;
                        nxt = cursor_next(hc, sm, lg, SEGW, lane, nem);
                        if (nxt >= 0) line.eval2(nxt, fnxt, featnxt);
                    }
                    v[t] = fo + (j - cur) * (j - cur);
                    ft[t] = featcur;
                }
            }
        }
        out.store(j0, min(OC, b - j0), v, ft);
    }
}

// Direct minimum for lines whose answers are near: position j takes the
// minimum over k of f(k) + (j - k)^2 (Eq. (5)), searched outward from j,
// r = 0, 1, 2, ..., through the first r with r^2 above the best value found --
// every k farther away costs more, so the result is exact, and a k at r^2
// equal to the best (a source in the line itself) is still seen.  At a tie
// the rightmost k is kept (a candidate left of the current best must be
// strictly smaller, one right of it may tie), the same choice as the hull
// walk of band_fill.  Each warp takes every NW-th chunk of OC positions of the
// 32 lines; no barrier, no shared state.  Line and Out as for band_envelope.
template <class Line, class Out>
__device__ void band_direct(const Line& line, const Out& out, int n, int warp, int NW)
{
    const int nq = (n + OC - 1) / OC;
    for (int q = warp; q < nq; q += NW) {
        const int j0 = q * OC;
        int v[OC], ft[OC];
#pragma unroll
        for (int t = 0; t < OC; ++t) {
            const int j = j0 + t;
            v[t] = INT32_MAX;
            ft[t] = -1;
            if (j >= n) continue;
            int f, best = INT32_MAX, bk = -1;
            if (line.eval(j, f)) {
                best = f;
                bk = j;
            }
            for (int r = 1; r < n && r * r <= best; ++r) {
                if (j - r >= 0 && line.eval(j - r, f) && f + r * r < best) {
                    best = f + r * r;
                    bk = j - r;
                }
                if (j + r < n && line.eval(j + r, f) && f + r * r <= best) {
                    best = f + r * r;
                    bk = j + r;
                }
            }
            if (bk >= 0) {
                int g;
                line.eval2(bk, f, g);
                v[t] = best;
                ft[t] = g;
            }
        }
        out.store(j0, min(OC, n - j0), v, ft);
    }
    out.finish();
}

// Largest own value (as a distance, saturated at 2^15) at which an engine
// takes the direct search instead of the hull: the search from a position
// ends within sqrt of its answer, which is at most its own value.
constexpr int DIRECT_MAX_DIST = 64;

// The whole per-block computation, called by every thread of the block
// (blockDim.x = 32 * NW, or the NW warps of one group).  Line (per lane) must
// provide
//   bool eval(int k, int& f) const       f(k) of this lane's line, false = infinite
//   bool eval2(int k, int& f, int& g) const   f(k) and the feature of position k
//   int  c(int k) const                  f(k) + k*k for a finite position
//   bool is_zero(int k) const            f(k) == 0: position k is a source itself
//   bool chunk_has_source(int j0) const  is_zero(k) for some k in j0 .. j0+OC-1
//   int  self_feature(int k) const       feature of a source position k
// and Out must provide store(int j0, int cnt, const int* v, const int* f),
// called by every lane of the warp at the same time with the values of its
// line at positions j0 .. j0+cnt-1 (cnt <= OC, j0 a multiple of OC), and
// finish(), called once by every lane at the end.  v = INT32_MAX, f = -1 where
// the line has no finite value.
template <class Line, class Out, class Sync = BlockSync>
__device__ void band_envelope(const Line& line, const Out& out, const BandSmem& sm, int n,
                              int lg, int NW, const unsigned char* full = nullptr, int warp = -1,
                              Sync sync = Sync())
{
    if (warp < 0) warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int SEGW = (1 << lg) >> 5;
    const int s0 = warp << lg;
    const int s1 = min(s0 + (1 << lg), n);
    uint32_t* hbw = sm.hb + (size_t)warp * SEGW * 32 + lane;
    for (int w = 0; w < SEGW; ++w) hbw[w * 32] = 0u;

    // (1) hull of this segment of this lane's line.  A position lying on or
    // above the chord of its two neighbours (2 f(k) >= f(k-1) + f(k+1) + 2) is
    // no vertex of the line's hull and is skipped; the others go through the
    // stack algorithm, whose top three entries are kept in registers, as is
    // the hull word of the current position (cw, word index cwi).  Where all
    // 32 lines are sources at all 32 positions of a word (full[] set), every
    // position is a hull vertex owning itself (a source cannot be hidden), so
    // after the first one the word is filled at once.
    int top = -1, sec = -1, thr = -1, ctop = 0, csec = 0, cthr = 0;
    bool thr_known = true;
    int fprev = 0, fcur = 0, fnext = 0;
    bool iprev = (s0 > 0 && s0 - 1 < n) ? line.eval(s0 - 1, fprev) : false;
    bool icur = (s0 < s1) ? line.eval(s0, fcur) : false;
    uint32_t cw = 0u;
    int cwi = 0;
    // one hull word (32 positions) per outer step
    for (int c = s0; c < s1; c += 32) {
        cwi = (c - s0) >> 5;
        cw = 0u;
        const int ce = min(c + 32, s1);
        const bool bulk = full && ce == c + 32 && full[c >> 5];
        for (int k = c; k < ce; ++k) {
            const bool inext = (k + 1 < n) ? line.eval(k + 1, fnext) : false;
            const bool keep = icur && !(iprev && inext && 2 * fcur >= fprev + fnext + 2);
            if (keep) {
                const int ck = fcur + k * k;
                while (sec >= 0 && hidden(sec, csec, top, ctop, k, ck)) {
                    const int off = top - s0;
                    if ((off >> 5) == cwi) cw &= ~(1u << (off & 31));
                    else hbw[(off >> 5) * 32] &= ~(1u << (off & 31));
                    top = sec;
                    ctop = csec;
                    if (!thr_known) {
                        thr = -1;
                        const int so = sec - s0;
                        uint32_t m = ((so >> 5) == cwi ? cw : hbw[(so >> 5) * 32]) & ((1u << (so & 31)) - 1u);
                        int w = so >> 5;
                        while (!m && --w >= 0) m = hbw[w * 32];
                        if (m) {
                            thr = s0 + w * 32 + 31 - __clz(m);
                            cthr = line.c(thr);
                        }
                    }
                    sec = thr;
                    csec = cthr;
                    thr_known = false;
                }
                cw |= 1u << (k & 31);
                thr = sec;
                cthr = csec;
                thr_known = true;
                sec = top;
                csec = ctop;
                top = k;
                ctop = ck;
            }
            iprev = icur;
            fprev = fcur;
            icur = inext;
            fcur = fnext;
            if (bulk) {
                // every line is a source at positions c .. c+31: each is a hull
                // vertex owning itself (a source cannot be hidden)
                if (keep) {
                    cw = 0xFFFFFFFFu;
                    thr = c + 29;
                    cthr = thr * thr;
                    sec = c + 30;
                    csec = sec * sec;
                    top = c + 31;
                    ctop = top * top;
                    thr_known = true;
                }
                iprev = keep;
                fprev = 0;
                icur = (ce < n) ? line.eval(ce, fcur) : false;
                break;
            }
        }
        hbw[cwi * 32] = cw;
    }
    int first = -1;
    for (int w = 0; w < SEGW; ++w) {
        const uint32_t m = (w == cwi) ? cw : hbw[w * 32];
        if (m) {
            first = s0 + w * 32 + __ffs(m) - 1;
            break;
        }
    }
    sm.lo[warp * 32 + lane] = first;
    sm.hi[warp * 32 + lane] = top;
    if (warp == 0 && lane == 0) *sm.ctr = 0;
    sync();

    // (2) merge segments 1+1, 2+2, ...
    for (int half = 1; half < NW; half <<= 1) {
        if ((warp & (2 * half - 1)) == 0 && warp + half < NW)
            band_bridge(line, sm, lg, SEGW, lane, warp, warp + half, min(warp + 2 * half, NW));
        sync();
    }

    // (3) fill, in units of positions that the warps take in turn from a
    // shared counter, so that the costly parts of the lines do not leave the
    // other warps waiting.
    uint32_t nem = 0;
    for (int w = 0; w < NW; ++w) nem |= (uint32_t)(sm.lo[w * 32 + lane] >= 0) << w;
    const int UL = band_fill_unit(n, NW);
    const int nunits = (n + UL - 1) / UL;
    for (;;) {
        int u = 0;
        if (lane == 0) u = atomicAdd(sm.ctr, 1);
        u = __shfl_sync(FULL, u, 0);
        if (u >= nunits) break;
        band_fill(line, out, sm, lg, SEGW, lane, nem, full, u * UL, min(n, u * UL + UL));
    }
    out.finish();
}

}  // namespace edt
