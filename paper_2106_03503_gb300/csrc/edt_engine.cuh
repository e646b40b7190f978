// Device building blocks of libedt (sm_103a): the warp-level lower envelope
// of parabolas along one line (Sec. 3.3.1 of Strutz, "The Distance Transform
// and its Computation"), the bit tricks of the column pass (Sec. 3.1) and the
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
// Work split.  One warp handles one line of n values.  Lane l owns the
// contiguous segment [l*S, l*S + S).  (1) Each lane builds the hull of its
// segment with the paper's stack algorithm, the stack kept as a bit set in
// shared memory (bit = column is on the hull).  (2) Five rounds of pairwise
// merges join neighbouring lanes' hulls: for two x-separated lower hulls the
// joint hull keeps a prefix of the left one and a suffix of the right one,
// found by the classic bridge walk (drop the left top while it is hidden
// between its predecessor and the right bottom, drop the right bottom while it
// is hidden between the left top and its successor).  (3) Each lane fills its
// own columns: the owner of a column is the hull member with the smallest
// value there; owners move right monotonically with the column, and along
// the hull the values at a fixed column are unimodal, so a walk finds them.
// Results go through a small per-warp shared tile so that global stores are
// written in whole 32-byte sectors.
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
// Lower-envelope engine.

struct WarpSmem {
    uint32_t* hb;   // hull bits, layout [word][lane], SW words per lane
    int* lo;        // first hull member of each lane (-1 = none)
    int* hi;        // last hull member of each lane
    int* tileD;     // 32 x OUT_CHUNK staging tile for values
    int* tileF;     // 32 x OUT_CHUNK staging tile for features
};

// Bytes of shared memory one warp needs for a line with SW hull words/lane.
__host__ __device__ constexpr int warp_smem_bytes(int SW)
{
    return SW * 32 * 4 + 64 * 4 + 2 * 32 * OUT_CHUNK * 4;
}

__device__ __forceinline__ WarpSmem carve_warp_smem(unsigned char* base, int SW)
{
    WarpSmem s;
    s.hb = reinterpret_cast<uint32_t*>(base);
    s.lo = reinterpret_cast<int*>(base + SW * 32 * 4);
    s.hi = s.lo + 32;
    s.tileD = s.hi + 32;
    s.tileF = s.tileD + 32 * OUT_CHUNK;
    return s;
}

// Segment length per lane: the smallest power of two >= max(OUT_CHUNK,
// ceil(n / 32)), so that lane = column >> log2(S).  Hull words per lane: S/32.
__host__ __device__ inline int seg_log2(int n)
{
    int s = (n + 31) / 32;
    int l = 3;  // OUT_CHUNK = 8
    while ((1 << l) < s) ++l;
    return l;
}
__host__ __device__ inline int seg_len(int n) { return 1 << seg_log2(n); }
__host__ __device__ inline int seg_words(int n) { return (seg_len(n) + 31) / 32; }
// Shared-memory index of column k when lane segments of length S = 2^lg are
// stored back to back: one pad word per segment puts the 32 lanes' columns at
// the same offset into 32 different banks (S + 1 is odd).
__host__ __device__ __forceinline__ int pad_index(int k, int lg) { return k + (k >> lg); }
__host__ __device__ inline int padded_len(int n) { return n + (n >> seg_log2(n)) + 1; }

// t is hidden between p < t < m on the hull of points (k, c_k).
__device__ __forceinline__ bool hidden(int p, int cp, int t, int ct, int m, int cm)
{
    return (long long)(cm - ct) * (long long)(t - p) <=
           (long long)(ct - cp) * (long long)(m - t);
}

// Previous / next hull member of lane L strictly before / after column x
// (x must lie in L's segment).  -1 when none.
__device__ __forceinline__ int prev_in_lane(const uint32_t* hb, int L, int S, int x)
{
    const int off = x - L * S;
    int w = off >> 5;
    const int b = off & 31;
    uint32_t m = hb[w * 32 + L] & ((1u << b) - 1u);
    while (!m) {
        if (--w < 0) return -1;
        m = hb[w * 32 + L];
    }
    return L * S + w * 32 + 31 - __clz(m);
}
__device__ __forceinline__ int next_in_lane(const uint32_t* hb, int L, int S, int SW, int x)
{
    const int off = x - L * S;
    int w = off >> 5;
    const int b = off & 31;
    uint32_t m = (b == 31) ? 0u : (hb[w * 32 + L] & (0xFFFFFFFEu << b));
    while (!m) {
        if (++w >= SW) return -1;
        m = hb[w * 32 + L];
    }
    return L * S + w * 32 + __ffs(m) - 1;
}

// Join the hulls of lanes [a0, b0) and [b0, b1) (run by one lane).
template <class Line>
__device__ void bridge(const Line& line, uint32_t* hb, int* lo, int* hi, int S,
                       int SW, int a0, int b0, int b1)
{
    int la = b0 - 1;
    while (la >= a0 && hi[la] < 0) --la;
    int lb = b0;
    while (lb < b1 && lo[lb] < 0) ++lb;
    while (la >= a0 && lb < b1) {
        const int x1 = hi[la];
        const int y1 = lo[lb];
        int x0 = prev_in_lane(hb, la, S, x1);
        int lx0 = la;
        if (x0 < 0) {
            int l = la - 1;
            while (l >= a0 && hi[l] < 0) --l;
            if (l >= a0) { x0 = hi[l]; lx0 = l; }
        }
        int y2 = next_in_lane(hb, lb, S, SW, y1);
        const bool y2_same = (y2 >= 0);
        if (y2 < 0) {
            int l = lb + 1;
            while (l < b1 && lo[l] < 0) ++l;
            if (l < b1) y2 = lo[l];
        }
        const int cx1 = line.c(x1);
        const int cy1 = line.c(y1);
        if (x0 >= 0 && hidden(x0, line.c(x0), x1, cx1, y1, cy1)) {
            const int off = x1 - la * S;
            hb[(off >> 5) * 32 + la] &= ~(1u << (off & 31));
            if (lx0 == la) {
                hi[la] = x0;
            } else {
                hi[la] = -1;
                lo[la] = -1;
                la = lx0;
            }
            continue;
        }
        if (y2 >= 0 && hidden(x1, cx1, y1, cy1, y2, line.c(y2))) {
            const int off = y1 - lb * S;
            hb[(off >> 5) * 32 + lb] &= ~(1u << (off & 31));
            if (y2_same) {
                lo[lb] = y2;
            } else {
                lo[lb] = -1;
                hi[lb] = -1;
                ++lb;
                while (lb < b1 && lo[lb] < 0) ++lb;
            }
            continue;
        }
        break;
    }
}

// Global successor / predecessor of hull member x after the merge.
__device__ __forceinline__ int hull_next(const uint32_t* hb, const int* lo,
                                         uint32_t nonempty, int S, int SW, int x)
{
    const int L = x >> (31 - __clz(S));
    const int y = next_in_lane(hb, L, S, SW, x);
    if (y >= 0) return y;
    const uint32_t later = (L >= 31) ? 0u : (nonempty & (0xFFFFFFFEu << L));
    return later ? lo[__ffs(later) - 1] : -1;
}
__device__ __forceinline__ int hull_prev(const uint32_t* hb, const int* hi,
                                         uint32_t nonempty, int S, int x)
{
    const int L = x >> (31 - __clz(S));
    const int y = prev_in_lane(hb, L, S, x);
    if (y >= 0) return y;
    const uint32_t earlier = nonempty & ((1u << L) - 1u);
    return earlier ? hi[31 - __clz(earlier)] : -1;
}

// The whole per-line computation, executed by all 32 lanes of a warp.
//
// Line must provide:
//   int  n;                                 line length
//   bool eval(int k, int& f) const;         f(k) if finite (false = infinite)
//   int  c(int k) const;                    f(k) + k*k for a finite member
//   int  feature(int k) const;              output feature of source column k
// Out must provide:
//   void store(int j, int value, int feature) const;  value INT32_MAX and
//        feature -1 when the line has no finite value at all.
template <class Line, class Out>
__device__ void warp_envelope(const Line& line, const Out& out, const WarpSmem& sm)
{
    const int lane = threadIdx.x & 31;
    const int n = line.n;
    const int S = seg_len(n);
    const int SW = (S + 31) / 32;
    const int s0 = lane * S;
    const int s1 = min(s0 + S, n);
    for (int w = 0; w < SW; ++w) sm.hb[w * 32 + lane] = 0u;

    // (1) hull of the lane's own segment (stack algorithm of Sec. 3.3.1)
    int top = -1, sec = -1, ctop = 0, csec = 0, first = -1;
    for (int k = s0; k < s1; ++k) {
        int fk;
        if (!line.eval(k, fk)) continue;
        const int ck = fk + k * k;
        while (sec >= 0 && hidden(sec, csec, top, ctop, k, ck)) {
            const int off = top - s0;
            sm.hb[(off >> 5) * 32 + lane] &= ~(1u << (off & 31));
            top = sec;
            ctop = csec;
            sec = prev_in_lane(sm.hb, lane, S, top);
            if (sec >= 0) csec = line.c(sec);
        }
        const int off = k - s0;
        sm.hb[(off >> 5) * 32 + lane] |= 1u << (off & 31);
        if (first < 0) first = k;
        sec = top;
        csec = ctop;
        top = k;
        ctop = ck;
    }
    sm.lo[lane] = first;
    sm.hi[lane] = top;
    __syncwarp();

    // (2) merge neighbouring hulls, 1+1, 2+2, ..., 16+16 lanes
#pragma unroll 1
    for (int half = 1; half < 32; half <<= 1) {
        if ((lane & (2 * half - 1)) == 0)
            bridge(line, sm.hb, sm.lo, sm.hi, S, SW, lane, lane + half, lane + 2 * half);
        __syncwarp();
    }

    // (3) fill this lane's columns
    const uint32_t nonempty = __ballot_sync(FULL, sm.lo[lane] >= 0);
    int cur = -1, fcur = 0, featcur = -1, nxt = -1, fnxt = 0;
    bool feat_stale = false;
    if (nonempty && s0 < s1) {
        const uint32_t before = nonempty & ((1u << lane) - 1u);
        cur = before ? sm.hi[31 - __clz(before)] : sm.lo[__ffs(nonempty) - 1];
        line.eval(cur, fcur);
        // walk left while strictly better at s0
        for (;;) {
            const int p = hull_prev(sm.hb, sm.hi, nonempty, S, cur);
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
        nxt = hull_next(sm.hb, sm.lo, nonempty, S, SW, cur);
        if (nxt >= 0) line.eval(nxt, fnxt);
        featcur = line.feature(cur);
    }

    const int nch = S / OUT_CHUNK;
    for (int q = 0; q < nch; ++q) {
        int v[OUT_CHUNK], ft[OUT_CHUNK];
#pragma unroll
        for (int t = 0; t < OUT_CHUNK; ++t) {
            const int j = s0 + q * OUT_CHUNK + t;
            v[t] = INT32_MAX;
            ft[t] = -1;
            if (j < s1 && cur >= 0) {
                while (nxt >= 0 && fnxt + (j - nxt) * (j - nxt) <= fcur + (j - cur) * (j - cur)) {
                    cur = nxt;
                    fcur = fnxt;
                    feat_stale = true;
                    nxt = hull_next(sm.hb, sm.lo, nonempty, S, SW, cur);
                    if (nxt >= 0) line.eval(nxt, fnxt);
                }
                if (feat_stale) {
                    featcur = line.feature(cur);
                    feat_stale = false;
                }
                v[t] = fcur + (j - cur) * (j - cur);
                ft[t] = featcur;
            }
        }
        int4* td = reinterpret_cast<int4*>(sm.tileD + lane * OUT_CHUNK);
        int4* tf = reinterpret_cast<int4*>(sm.tileF + lane * OUT_CHUNK);
        td[0] = make_int4(v[0], v[1], v[2], v[3]);
        td[1] = make_int4(v[4], v[5], v[6], v[7]);
        tf[0] = make_int4(ft[0], ft[1], ft[2], ft[3]);
        tf[1] = make_int4(ft[4], ft[5], ft[6], ft[7]);
        __syncwarp();
#pragma unroll
        for (int p = 0; p < 32 / (32 / OUT_CHUNK); ++p) {
            const int L = p * (32 / OUT_CHUNK) + lane / OUT_CHUNK;
            const int t = lane % OUT_CHUNK;
            const int j = L * S + q * OUT_CHUNK + t;
            if (j < min(L * S + S, n))
                out.store(j, sm.tileD[L * OUT_CHUNK + t], sm.tileF[L * OUT_CHUNK + t]);
        }
        __syncwarp();
    }
}

}  // namespace edt
