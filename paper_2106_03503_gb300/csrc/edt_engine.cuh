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
//   (3) Each (segment, line) fills its positions: the owner of a position is
//       the hull member with the smallest value there; owners move right
//       monotonically with the position, and along the hull the values at a
//       fixed position are unimodal, so a walk finds them.  Values either go
//       straight to memory (lines adjacent in memory) or through a 32 x 8
//       shared tile that turns them into 32-byte row segments (lines are
//       rows, positions are columns).
#pragma once

#include <cstdint>
#include <climits>
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
    int* tileD;     // [NW][32][OC] staging of values (tiled output only)
    int* tileF;     // [NW][32][OC] staging of features
};

__host__ __device__ inline size_t band_smem_bytes(int NW, int SEGW, bool tiled)
{
    return (size_t)NW * SEGW * 32 * 4 + (size_t)NW * 64 * 4 +
           (tiled ? (size_t)NW * 32 * OC * 4 * 2 : 0);
}

__device__ __forceinline__ BandSmem carve_band_smem(unsigned char* base, int NW, int SEGW, bool tiled)
{
    BandSmem s;
    s.hb = reinterpret_cast<uint32_t*>(base);
    s.lo = reinterpret_cast<int*>(base + (size_t)NW * SEGW * 32 * 4);
    s.hi = s.lo + NW * 32;
    s.tileD = tiled ? s.hi + NW * 32 : nullptr;
    s.tileF = tiled ? s.tileD + NW * 32 * OC : nullptr;
    return s;
}

// Segment length (power of two, >= 32) and segment count for a line of n
// positions split over at most max_nw warps.
__host__ __device__ inline int band_seg_log2(int n, int max_nw)
{
    int lg = 5;
    while ((((n + (1 << lg) - 1) >> lg)) > max_nw) ++lg;
    return lg;
}

// t is hidden between p < t < m on the hull of points (k, c_k).
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

// The whole per-block computation, called by every thread of the block
// (blockDim.x = 32 * NW).  Line (per lane) must provide
//   bool eval(int k, int& f) const   f(k) of this lane's line, false = infinite
//   int  c(int k) const              f(k) + k*k for a finite position
//   int  feature(int k) const        output feature of position k
// and Out either (TILED) store(int line_lane, int j, int v, int f), called by
// any lane of the segment's warp, or (!TILED) the same called by the line's
// own lane.  v = INT32_MAX, f = -1 where the line has no finite value.
// Barrier of the NW warps that share one band engine: the whole block, or a
// named barrier when a block runs several engines side by side.
struct BlockSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct GroupSync {
    int id, nthreads;
    __device__ __forceinline__ void operator()() const
    {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
    }
};

template <bool TILED, class Line, class Out, class Sync = BlockSync>
__device__ void band_envelope(const Line& line, const Out& out, const BandSmem& sm, int n,
                              int lg, int NW, int warp = -1, Sync sync = Sync())
{
    if (warp < 0) warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int SEGW = (1 << lg) >> 5;
    const int s0 = warp << lg;
    const int s1 = min(s0 + (1 << lg), n);
    uint32_t* hbw = sm.hb + (size_t)warp * SEGW * 32 + lane;
    for (int w = 0; w < SEGW; ++w) hbw[w * 32] = 0u;

    // (1) hull of this segment of this lane's line
    int top = -1, sec = -1, ctop = 0, csec = 0, first = -1;
    for (int k = s0; k < s1; ++k) {
        int fk;
        if (!line.eval(k, fk)) continue;
        const int ck = fk + k * k;
        while (sec >= 0 && hidden(sec, csec, top, ctop, k, ck)) {
            const int off = top - s0;
            hbw[(off >> 5) * 32] &= ~(1u << (off & 31));
            top = sec;
            ctop = csec;
            sec = seg_prev(sm.hb, warp, lg, SEGW, lane, top);
            if (sec >= 0) csec = line.c(sec);
        }
        const int off = k - s0;
        hbw[(off >> 5) * 32] |= 1u << (off & 31);
        if (first < 0) first = k;
        sec = top;
        csec = ctop;
        top = k;
        ctop = ck;
    }
    sm.lo[warp * 32 + lane] = first;
    sm.hi[warp * 32 + lane] = top;
    sync();

    // (2) merge segments 1+1, 2+2, ...
    for (int half = 1; half < NW; half <<= 1) {
        if ((warp & (2 * half - 1)) == 0 && warp + half < NW)
            band_bridge(line, sm, lg, SEGW, lane, warp, warp + half, min(warp + 2 * half, NW));
        sync();
    }

    // (3) fill
    uint32_t nem = 0;
    for (int w = 0; w < NW; ++w) nem |= (uint32_t)(sm.lo[w * 32 + lane] >= 0) << w;
    int cur = -1, fcur = 0, featcur = -1, nxt = -1, fnxt = 0;
    bool stale = false;
    if (nem && s0 < s1) {
        const uint32_t before = nem & ((1u << warp) - 1u);
        cur = before ? sm.hi[(31 - __clz(before)) * 32 + lane] : sm.lo[(__ffs(nem) - 1) * 32 + lane];
        line.eval(cur, fcur);
        for (;;) {  // walk left while strictly better at s0
            const int p = band_prev(sm, lg, SEGW, lane, nem, cur);
            if (p < 0) break;
            int fp;
            line.eval(p, fp);
            if ((long long)fp + (long long)(s0 - p) * (s0 - p) <
                (long long)fcur + (long long)(s0 - cur) * (s0 - cur)) {
                cur = p;
                fcur = fp;
            } else {
                break;
            }
        }
        nxt = band_next(sm, lg, SEGW, lane, nem, cur);
        if (nxt >= 0) line.eval(nxt, fnxt);
        featcur = line.feature(cur);
    }
    const int nq = ((1 << lg) + OC - 1) / OC;
    for (int q = 0; q < nq; ++q) {
        int v[OC], ft[OC];
#pragma unroll
        for (int t = 0; t < OC; ++t) {
            const int j = s0 + q * OC + t;
            v[t] = INT32_MAX;
            ft[t] = -1;
            if (j < s1 && cur >= 0) {
                while (nxt >= 0 && fnxt + (j - nxt) * (j - nxt) <= fcur + (j - cur) * (j - cur)) {
                    cur = nxt;
                    fcur = fnxt;
                    stale = true;
                    nxt = band_next(sm, lg, SEGW, lane, nem, cur);
                    if (nxt >= 0) line.eval(nxt, fnxt);
                }
                if (stale) {
                    featcur = line.feature(cur);
                    stale = false;
                }
                v[t] = fcur + (j - cur) * (j - cur);
                ft[t] = featcur;
            }
        }
        if (TILED) {
            int4* td = reinterpret_cast<int4*>(sm.tileD + (warp * 32 + lane) * OC);
            int4* tf = reinterpret_cast<int4*>(sm.tileF + (warp * 32 + lane) * OC);
            td[0] = make_int4(v[0], v[1], v[2], v[3]);
            td[1] = make_int4(v[4], v[5], v[6], v[7]);
            tf[0] = make_int4(ft[0], ft[1], ft[2], ft[3]);
            tf[1] = make_int4(ft[4], ft[5], ft[6], ft[7]);
            __syncwarp();
            const int* tD = sm.tileD + warp * 32 * OC;
            const int* tF = sm.tileF + warp * 32 * OC;
#pragma unroll
            for (int p = 0; p < OC; ++p) {
                const int ln = p * (32 / OC) + lane / OC;
                const int t = lane % OC;
                const int j = s0 + q * OC + t;
                if (j < s1) out.store(ln, j, tD[ln * OC + t], tF[ln * OC + t]);
            }
            __syncwarp();
        } else {
#pragma unroll
            for (int t = 0; t < OC; ++t) {
                const int j = s0 + q * OC + t;
                if (j < s1) out.store(lane, j, v[t], ft[t]);
            }
        }
    }
}

}  // namespace edt
