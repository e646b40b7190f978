/*
 * Oracle for the exact Euclidean distance transform (EEDT) and its feature
 * (nearest source pixel) map, after T. Strutz, "The Distance Transform and its
 * Computation -- An Introduction", Section 3.  It is written from the
 * definitions the paper gives (the vertical distance to the nearest source of
 * a column, Sec. 3.1; the parabolas of Eq. (5) and their intersections,
 * Eq. (6), Sec. 3.3.1), not from the paper's program listings.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is plain, slow, single-threaded C that
 * exists to check the CUDA path.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the product never does.  It
 * shares no code, header, table or constant with the CUDA library.
 *
 * Arithmetic: all distances are held in int64_t, so no intermediate can
 * overflow for any image the CUDA path accepts.  Results are returned as
 * int32_t: D is the squared distance, F the 0-based row-major linear index of
 * the nearest source pixel.
 *
 * Readings of points on which the paper is silent or loose:
 *   - mode 0 ("to object"): sources are the nonzero mask bytes, every pixel
 *     receives its squared distance to the nearest nonzero pixel (Fig. 1c);
 *     mode 1 ("to background"): sources are the zero bytes (Fig. 1b).
 *   - only pixels inside the image count; there is no virtual border.
 *   - "infinity" is any value >= max_dist, where max_dist is one more than the
 *     largest squared distance inside the image (Sec. 3.1 asks for a value
 *     larger than (M-1)^2 + (L-1)^2).  The envelope only takes finite values
 *     as parabola vertices, so every finite result is a real distance; there
 *     is no dummy first parabola.
 *   - an image without any source pixel yields D = INT32_MAX, F = -1
 *     everywhere (the paper's algorithm would return a value derived from the
 *     initial infinity there).
 *   - the intersection of Eq. (6) is rounded up with exact integer ceiling
 *     division; no floating point is used.
 *   - ties: the column distances keep the upper source (the scans of Sec. 3.1
 *     replace a value only by a strictly smaller one), the envelope hands an
 *     integer intersection to the right-hand parabola (Fig. 21: the ties "2/5"
 *     and "5/8" go to 5 and 8); a returned feature is one valid nearest
 *     source, not the only one.
 *   - 3-D: the paper only says that the dimensions are processed separately
 *     (Sec. 3.1); here the scan runs along z, then the envelope along y, then
 *     along x.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORACLE_TO_OBJECT 0
#define ORACLE_TO_BACKGROUND 1

/* Sec. 3.1: the initial value must exceed the largest possible squared
 * distance in the image, sum over axes of (n_d - 1)^2. */
int64_t oracle_max_dist(int ndim, const int *shape)
{
    int64_t s = 1;
    for (int a = 0; a < ndim; ++a) {
        int64_t e = (int64_t)shape[a] - 1;
        s += e * e;
    }
    return s;
}

/* Sec. 3.1, Fig. 18(b) and Fig. 19: the squared vertical distance of a pixel
 * is the squared row difference to the nearest source pixel of its own column
 * (Eq. (5) restricted to one column).  Along one line of n values spaced by
 * `stride`, where a source holds d = 0, one sweep downwards records for every
 * position the nearest source at or above it, one sweep upwards the nearest
 * at or below it; the nearer of the two is kept, the upper one when both are
 * equally far (the scans of Sec. 3.1 replace a value only by a strictly
 * smaller one, so the value that arrived from above first stays).  With
 * down_only set, only sources at or above count (the state of Fig. 19).
 * Positions without a source in reach keep their value (infinity).  The
 * feature index of the chosen source travels with the distance.  `above` is
 * scratch space for n positions. */
static void column_nearest(int64_t *d, int32_t *feat, long n, long stride,
                           int down_only, long *above)
{
    long last = -1;
    for (long i = 0; i < n; ++i) {
        if (d[i * stride] == 0)
            last = i;
        above[i] = last;
    }
    long next = -1;
    for (long i = n - 1; i >= 0; --i) {
        if (d[i * stride] == 0)
            next = i;
        long up = above[i];
        long dn = down_only ? -1 : next;
        long g;
        if (up < 0 && dn < 0)
            continue;
        if (dn < 0 || (up >= 0 && i - up <= dn - i))
            g = up;
        else
            g = dn;
        d[i * stride] = (int64_t)(i - g) * (int64_t)(i - g);
        feat[i * stride] = feat[g * stride];
    }
}

/* Exact ceiling of num / den for den > 0 (reading of the rounding in Eq. (6)).
 * C division truncates toward zero, which already is the ceiling when the
 * quotient is negative. */
static int64_t ceil_div(int64_t num, int64_t den)
{
    int64_t q = num / den;
    if (num > 0 && num % den != 0)
        q += 1;
    return q;
}

/* Eq. (6) for the parabolas of Eq. (5) with vertices k < m: m is not worse
 * than k at position j exactly when
 *     2 j (m - k) >= f(m) - f(k) + m^2 - k^2,
 * so the first integer position where m is not worse is the ceiling of the
 * right-hand side over 2 (m - k).  At an integer intersection the two are
 * equal and m, the right-hand parabola, is taken. */
static int64_t first_not_worse(const int64_t *f, int64_t k, int64_t m)
{
    return ceil_div(f[m] - f[k] + m * m - k * k, 2 * (m - k));
}

/* Sec. 3.3.1, Eq. (5) and Eq. (6): along one line f[0..n-1] (values >=
 * max_dist are infinite), position j receives the minimum over k of
 * f(k) + (j - k)^2, taken at a minimising k that moves right as j grows.
 * The positions k that give the minimum somewhere form a list ordered by k,
 * each with the first position it takes, `start`; it keeps the positions up
 * to the next start.  Visiting the finite positions m from left to right:
 * while m is not worse than the last listed k already at k's start, k gives
 * the minimum nowhere and leaves the list; then m is listed from the first
 * position where it is not worse than the last remaining entry (position 0
 * when none remains), unless that position lies beyond the line.  Returns the
 * number of entries; site[] and start[] hold them, start[cnt] = n. */
static long lower_envelope(const int64_t *f, long n, int64_t max_dist,
                           int64_t *site, int64_t *start)
{
    long cnt = 0;
    for (long m = 0; m < n; ++m) {
        if (f[m] >= max_dist)
            continue;
        int64_t s = 0;
        while (cnt > 0) {
            s = first_not_worse(f, site[cnt - 1], m);
            if (s > start[cnt - 1])
                break;
            cnt -= 1;
            s = 0;
        }
        if (s > n - 1)
            continue;
        site[cnt] = m;
        start[cnt] = s;
        cnt += 1;
    }
    start[cnt] = n;
    return cnt;
}

/* Eq. (5) evaluated from the list: positions start[p] .. start[p+1]-1 take
 * f(site[p]) + (j - site[p])^2 and that site's feature.  A line without any
 * finite value stays infinite, feature -1. */
static void envelope_fill(const int64_t *f, const int32_t *feat_in, long n,
                          int64_t max_dist, const int64_t *site,
                          const int64_t *start, long cnt, int64_t *out,
                          int32_t *feat_out)
{
    if (cnt == 0) {
        for (long j = 0; j < n; ++j) {
            out[j] = max_dist;
            feat_out[j] = -1;
        }
        return;
    }
    for (long p = 0; p < cnt; ++p) {
        int64_t k = site[p];
        for (int64_t j = start[p]; j < start[p + 1]; ++j) {
            out[j] = f[k] + (j - k) * (j - k);
            feat_out[j] = feat_in[k];
        }
    }
}

/* Initialisation of Sec. 3.1, Fig. 18(a): 0 on source pixels, "infinity"
 * elsewhere; the feature of a source pixel is its own index. */
static void init_sources(const uint8_t *mask, long n, int mode,
                         int64_t max_dist, int64_t *d, int32_t *feat)
{
    for (long p = 0; p < n; ++p) {
        int is_src = (mode == ORACLE_TO_OBJECT) ? (mask[p] != 0) : (mask[p] == 0);
        d[p] = is_src ? 0 : max_dist;
        feat[p] = is_src ? (int32_t)p : -1;
    }
}

static void finish(const int64_t *d, const int32_t *feat, long n,
                   int64_t max_dist, int32_t *D, int32_t *F)
{
    for (long p = 0; p < n; ++p) {
        if (d[p] >= max_dist) {
            D[p] = INT32_MAX;
            if (F)
                F[p] = -1;
        } else {
            D[p] = (int32_t)d[p];
            if (F)
                F[p] = feat[p];
        }
    }
}

/* Working space of the line passes (one line at a time). */
typedef struct {
    int64_t *fv, *out, *site, *start;
    int32_t *featv, *featout;
    long *above;
} line_work;

static int work_alloc(line_work *w, long line)
{
    size_t n = (size_t)(line > 0 ? line : 1);
    w->fv = malloc(sizeof(int64_t) * n);
    w->out = malloc(sizeof(int64_t) * n);
    w->site = malloc(sizeof(int64_t) * (n + 1));
    w->start = malloc(sizeof(int64_t) * (n + 1));
    w->featv = malloc(sizeof(int32_t) * n);
    w->featout = malloc(sizeof(int32_t) * n);
    w->above = malloc(sizeof(long) * n);
    return (w->fv && w->out && w->site && w->start && w->featv && w->featout && w->above) ? 0 : -1;
}

static void work_free(line_work *w)
{
    free(w->fv); free(w->out); free(w->site); free(w->start);
    free(w->featv); free(w->featout); free(w->above);
}

/* One envelope pass along a strided line: gather, envelope, fill, scatter. */
static void envelope_pass(int64_t *d, int32_t *feat, long n, long stride,
                          int64_t max_dist, line_work *w)
{
    for (long j = 0; j < n; ++j) {
        w->fv[j] = d[j * stride];
        w->featv[j] = feat[j * stride];
    }
    long cnt = lower_envelope(w->fv, n, max_dist, w->site, w->start);
    envelope_fill(w->fv, w->featv, n, max_dist, w->site, w->start, cnt,
                  w->out, w->featout);
    for (long j = 0; j < n; ++j) {
        d[j * stride] = w->out[j];
        feat[j * stride] = w->featout[j];
    }
}

/* 2-D EEDT of an M x L image (Sec. 3.1 column distances, then the Sec. 3.3.1
 * envelope per row).  D and F are M*L int32 arrays; F may be NULL.
 * Returns 0, or -1 when memory runs out.  Columns, and then rows, are
 * independent of one another: built with -fopenmp (the all-core timing
 * build only; the checker is built without it and runs this single-threaded)
 * each thread takes whole columns, then whole rows, with its own line
 * buffers; the arithmetic is the same. */
int oracle_edt2d(const uint8_t *mask, int M, int L, int mode, int32_t *D,
                 int32_t *F)
{
    long n = (long)M * L;
    int shape[2] = {M, L};
    int64_t max_dist = oracle_max_dist(2, shape);
    int64_t *d = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int32_t *feat = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int rc = 0;
    if (!d || !feat) {
        free(d); free(feat);
        return -1;
    }
    init_sources(mask, n, mode, max_dist, d, feat);
#pragma omp parallel
    {
        line_work w;
        const int ok = work_alloc(&w, L > M ? L : M) == 0;
        if (!ok) {
#pragma omp atomic write
            rc = -1;
        }
#pragma omp for schedule(static)
        for (long j = 0; j < L; ++j)
            if (ok)
                column_nearest(d + j, feat + j, M, L, 0, w.above);
#pragma omp for schedule(dynamic, 8)
        for (long i = 0; i < M; ++i)
            if (ok)
                envelope_pass(d + i * L, feat + i * L, L, 1, max_dist, &w);
        work_free(&w);
    }
    if (rc == 0)
        finish(d, feat, n, max_dist, D, F);
    free(d); free(feat);
    return rc;
}

/* 3-D EEDT of a Dz x H x W volume: the column distances of Sec. 3.1 along z,
 * then the envelope of Sec. 3.3.1 along y and along x (lines independent, as
 * in 2-D). */
int oracle_edt3d(const uint8_t *mask, int Dz, int H, int W, int mode,
                 int32_t *D, int32_t *F)
{
    long n = (long)Dz * H * W;
    long plane = (long)H * W;
    int shape[3] = {Dz, H, W};
    int64_t max_dist = oracle_max_dist(3, shape);
    long line = Dz;
    if (H > line) line = H;
    if (W > line) line = W;
    int64_t *d = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int32_t *feat = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int rc = 0;
    if (!d || !feat) {
        free(d); free(feat);
        return -1;
    }
    init_sources(mask, n, mode, max_dist, d, feat);
#pragma omp parallel
    {
        line_work w;
        const int ok = work_alloc(&w, line) == 0;
        if (!ok) {
#pragma omp atomic write
            rc = -1;
        }
#pragma omp for schedule(static)
        for (long p = 0; p < plane; ++p)
            if (ok)
                column_nearest(d + p, feat + p, Dz, plane, 0, w.above);
#pragma omp for schedule(dynamic, 8)
        for (long zx = 0; zx < (long)Dz * W; ++zx)
            if (ok)
                envelope_pass(d + (zx / W) * plane + zx % W, feat + (zx / W) * plane + zx % W, H, W,
                              max_dist, &w);
#pragma omp for schedule(dynamic, 8)
        for (long zy = 0; zy < (long)Dz * H; ++zy)
            if (ok)
                envelope_pass(d + zy * W, feat + zy * W, W, 1, max_dist, &w);
        work_free(&w);
    }
    if (rc == 0)
        finish(d, feat, n, max_dist, D, F);
    free(d); free(feat);
    return rc;
}

/* The column distances alone on an M x L image (Fig. 19 when down_only != 0:
 * sources at or above only; Fig. 18(b) otherwise).  Dv receives the int64
 * squared vertical distances (max_dist = infinity), G the feature index. */
int oracle_column_pass2d(const uint8_t *mask, int M, int L, int mode,
                         int down_only, int64_t *Dv, int32_t *G)
{
    long n = (long)M * L;
    int shape[2] = {M, L};
    int64_t max_dist = oracle_max_dist(2, shape);
    long *above = malloc(sizeof(long) * (size_t)(M > 0 ? M : 1));
    if (!above)
        return -1;
    init_sources(mask, n, mode, max_dist, Dv, G);
    for (long j = 0; j < L; ++j)
        column_nearest(Dv + j, G + j, M, L, down_only, above);
    free(above);
    return 0;
}

/* The envelope list of Sec. 3.3.1 on one line f[0..n-1] (values >= max_dist
 * are infinite): the listed positions site[0..cnt-1] with their first
 * positions start[0..cnt] (0-based, start[cnt] = n).  Returns cnt. */
long oracle_envelope_state(const int64_t *f, long n, int64_t max_dist,
                           int64_t *site, int64_t *start)
{
    return lower_envelope(f, n, max_dist, site, start);
}

/* The basic O(M L^2) row processing of Sec. 3.1, after the same column
 * distances: each position starts from its own vertical distance and takes
 * any strictly smaller combination D_v(k) + (k - j)^2 (Eq. (5) minimised by
 * trying every k).  A second, independent row pass for cross-checks. */
int oracle_edt2d_basic(const uint8_t *mask, int M, int L, int mode,
                       int32_t *D, int32_t *F)
{
    long n = (long)M * L;
    int shape[2] = {M, L};
    int64_t max_dist = oracle_max_dist(2, shape);
    int64_t *d = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int32_t *feat = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t *v = malloc(sizeof(int64_t) * (size_t)(L > 0 ? L : 1));
    int32_t *fv = malloc(sizeof(int32_t) * (size_t)(L > 0 ? L : 1));
    long *above = malloc(sizeof(long) * (size_t)(M > 0 ? M : 1));
    int rc = 0;
    if (!d || !feat || !v || !fv || !above) {
        rc = -1;
        goto done;
    }
    init_sources(mask, n, mode, max_dist, d, feat);
    for (long j = 0; j < L; ++j)
        column_nearest(d + j, feat + j, M, L, 0, above);
    for (long i = 0; i < M; ++i) {
        for (long k = 0; k < L; ++k) {
            v[k] = d[i * L + k];
            fv[k] = feat[i * L + k];
        }
        for (long j = 0; j < L; ++j) {
            int64_t dist_min = v[j];
            int32_t f_min = fv[j];
            for (long k = 0; k < L; ++k) {
                int64_t dist = v[k] + (k - j) * (k - j);
                if (dist_min > dist) {
                    dist_min = dist;
                    f_min = fv[k];
                }
            }
            d[i * L + j] = dist_min;
            feat[i * L + j] = f_min;
        }
    }
    finish(d, feat, n, max_dist, D, F);
done:
    free(d); free(feat); free(v); free(fv); free(above);
    return rc;
}

/* Sec. 3.1 notes that the square root is only needed once, after all squared
 * distances are known.  Reading: the float32 nearest to sqrt(D).  The square
 * root is taken in double and rounded once to float; for integers below 2^31
 * this double rounding cannot differ from a single correct rounding (53 >=
 * 2*24 + 2).  D = INT32_MAX (no source) maps to +infinity. */
void oracle_sqrt_f32(const int32_t *D, long n, float *out)
{
    for (long p = 0; p < n; ++p) {
        if (D[p] == INT32_MAX)
            out[p] = (float)INFINITY;
        else
            out[p] = (float)sqrt((double)D[p]);
    }
}
