/*
 * Oracle for the exact Euclidean distance transform (EEDT) and its feature
 * (nearest source pixel) map, after T. Strutz, "The Distance Transform and its
 * Computation -- An Introduction", Section 3.
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
 *     larger than (M-1)^2 + (L-1)^2).  Values produced from an infinite input
 *     are clamped back to max_dist, with feature -1.
 *   - an image without any source pixel yields D = INT32_MAX, F = -1
 *     everywhere (the listings would return max_dist + (j-1)^2 there).
 *   - the intersection of Eq. (6) is rounded up with exact integer ceiling
 *     division; no floating point is used.
 *   - ties: the column scans keep the upper source (strict comparisons), the
 *     envelope hands an integer intersection to the right-hand parabola (the
 *     "j <= js" pop of the fast algorithm); a returned feature is one valid
 *     nearest source, not the only one.
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

/* Sec. 3.1, Fig. 19 and Fig. 18(b): the column scans of Listing 7 ("Simple
 * EEDT algorithm").  A downward scan then an upward scan
 * propagate squared distances along one line of n values spaced by `stride`;
 * the step to the next square is the odd number dist_step, which grows by 2
 * per propagated pixel and falls back to 1 where nothing is propagated, since
 * (x+1)^2 - x^2 = 2x + 1.  The feature index travels with the value. */
static void column_scan(int64_t *d, int32_t *feat, long n, long stride,
                        int down_only)
{
    int64_t dist_step = 1;
    for (long i = 1; i < n; ++i) {
        int64_t cand = d[(i - 1) * stride] + dist_step;
        if (d[i * stride] > cand) {
            d[i * stride] = cand;
            feat[i * stride] = feat[(i - 1) * stride];
            dist_step += 2;
        } else {
            dist_step = 1;
        }
    }
    if (down_only)
        return;
    dist_step = 1;
    for (long i = n - 2; i >= 0; --i) {
        int64_t cand = d[(i + 1) * stride] + dist_step;
        if (d[i * stride] > cand) {
            d[i * stride] = cand;
            feat[i * stride] = feat[(i + 1) * stride];
            dist_step += 2;
        } else {
            dist_step = 1;
        }
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

/* Eq. (6): the intersection j_s of the parabolas of Eq. (5) with vertices at
 * k < l, rounded up to the first integer position where l is not worse. */
static int64_t intersection_ceil(const int64_t *f, long stride, int64_t k,
                                 int64_t l)
{
    int64_t num = f[l * stride] - f[k * stride] - k * k + l * l;
    return ceil_div(num, 2 * (l - k));
}

/* Sec. 3.3.1 (Meijster et al.; Listing 9, "Fast algorithm for EEDT"): the
 * lower envelope of the parabolas D_k(j) = f(k) + (j - k)^2 of Eq. (5) along
 * one line of n values spaced by `stride`.
 *
 * First scan: walk the line left to right; each finite f(m) is a candidate
 * contributor.  Its intersection with the last stored contributor is computed
 * with Eq. (6); while it does not lie beyond that contributor's start, the
 * stored contributor is hidden and dropped.  A candidate whose intersection
 * lies beyond the end of the line is not stored.  ks[] holds the stored
 * contributors, js[] their first columns (0-based; js[0] is the stopping
 * point -max_dist during the scan and is closed to 0 afterwards, js[cnt] = n).
 * The first contributor is column 0, possibly a dummy with f = infinity,
 * exactly as in the paper.
 *
 * Returns the number of stored contributors cnt (ks[0..cnt-1], js[0..cnt]). */
static long envelope_scan(const int64_t *f, long n, long stride,
                          int64_t max_dist, int64_t *ks, int64_t *js)
{
    long idx = 0;
    js[0] = -max_dist;
    ks[0] = 0;
    for (long m = 1; m < n; ++m) {
        if (f[m * stride] >= max_dist)
            continue;
        int64_t k = ks[idx];
        int64_t j = intersection_ceil(f, stride, k, m);
        while (j <= js[idx]) {
            idx -= 1;
            k = ks[idx];
            j = intersection_ceil(f, stride, k, m);
        }
        if (j <= n - 1) {
            idx += 1;
            js[idx] = j > 0 ? j : 0;
            ks[idx] = m;
        }
    }
    js[0] = 0;
    js[idx + 1] = n;
    return idx + 1;
}

/* Second scan of Sec. 3.3.1: every position j in [js[p], js[p+1]) takes its
 * value from contributor ks[p] through Eq. (5), and its feature with it.
 * Values reached only from an infinite input are clamped to max_dist. */
static void envelope_fill(const int64_t *f, const int32_t *feat_in,
                          long stride, int64_t max_dist, const int64_t *ks,
                          const int64_t *js, long cnt, int64_t *out,
                          int32_t *feat_out)
{
    for (long p = 0; p < cnt; ++p) {
        int64_t k = ks[p];
        for (int64_t j = js[p]; j < js[p + 1]; ++j) {
            int64_t v = f[k * stride] + (j - k) * (j - k);
            if (f[k * stride] >= max_dist || v >= max_dist) {
                out[j * stride] = max_dist;
                feat_out[j * stride] = -1;
            } else {
                out[j * stride] = v;
                feat_out[j * stride] = feat_in[k * stride];
            }
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

/* Strided envelope pass: gather the line, run the two scans, scatter back. */
static void envelope_pass(int64_t *d, int32_t *feat, long n, long stride,
                          int64_t max_dist, int64_t *fv, int32_t *featv,
                          int64_t *out, int32_t *featout, int64_t *ks,
                          int64_t *js)
{
    for (long j = 0; j < n; ++j) {
        fv[j] = d[j * stride];
        featv[j] = feat[j * stride];
    }
    long cnt = envelope_scan(fv, n, 1, max_dist, ks, js);
    envelope_fill(fv, featv, 1, max_dist, ks, js, cnt, out, featout);
    for (long j = 0; j < n; ++j) {
        d[j * stride] = out[j];
        feat[j * stride] = featout[j];
    }
}

/* 2-D EEDT of an M x L image (Sec. 3.1 column scans, then the Sec. 3.3.1
 * envelope per row).  D and F are M*L int32 arrays; F may be NULL.
 * Returns 0, or -1 when memory runs out. */
int oracle_edt2d(const uint8_t *mask, int M, int L, int mode, int32_t *D,
                 int32_t *F)
{
    long n = (long)M * L;
    int shape[2] = {M, L};
    int64_t max_dist = oracle_max_dist(2, shape);
    int64_t *d = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int32_t *feat = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    long line = L > M ? L : M;
    int64_t *fv = malloc(sizeof(int64_t) * (size_t)line);
    int32_t *featv = malloc(sizeof(int32_t) * (size_t)line);
    int64_t *out = malloc(sizeof(int64_t) * (size_t)line);
    int32_t *featout = malloc(sizeof(int32_t) * (size_t)line);
    int64_t *ks = malloc(sizeof(int64_t) * (size_t)(line + 1));
    int64_t *js = malloc(sizeof(int64_t) * (size_t)(line + 2));
    int rc = 0;
    if (!d || !feat || !fv || !featv || !out || !featout || !ks || !js) {
        rc = -1;
        goto done;
    }
    init_sources(mask, n, mode, max_dist, d, feat);
    for (long j = 0; j < L; ++j)
        column_scan(d + j, feat + j, M, L, 0);
    for (long i = 0; i < M; ++i)
        envelope_pass(d + i * L, feat + i * L, L, 1, max_dist, fv, featv,
                      out, featout, ks, js);
    finish(d, feat, n, max_dist, D, F);
done:
    free(d); free(feat); free(fv); free(featv); free(out); free(featout);
    free(ks); free(js);
    return rc;
}

/* 3-D EEDT of a Dz x H x W volume: the column scans of Sec. 3.1 along z, then
 * the envelope of Sec. 3.3.1 along y and along x. */
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
    int64_t *fv = malloc(sizeof(int64_t) * (size_t)line);
    int32_t *featv = malloc(sizeof(int32_t) * (size_t)line);
    int64_t *out = malloc(sizeof(int64_t) * (size_t)line);
    int32_t *featout = malloc(sizeof(int32_t) * (size_t)line);
    int64_t *ks = malloc(sizeof(int64_t) * (size_t)(line + 1));
    int64_t *js = malloc(sizeof(int64_t) * (size_t)(line + 2));
    int rc = 0;
    if (!d || !feat || !fv || !featv || !out || !featout || !ks || !js) {
        rc = -1;
        goto done;
    }
    init_sources(mask, n, mode, max_dist, d, feat);
    for (long p = 0; p < plane; ++p)
        column_scan(d + p, feat + p, Dz, plane, 0);
    for (long z = 0; z < Dz; ++z)
        for (long x = 0; x < W; ++x)
            envelope_pass(d + z * plane + x, feat + z * plane + x, H, W,
                          max_dist, fv, featv, out, featout, ks, js);
    for (long z = 0; z < Dz; ++z)
        for (long y = 0; y < H; ++y)
            envelope_pass(d + z * plane + y * W, feat + z * plane + y * W, W,
                          1, max_dist, fv, featv, out, featout, ks, js);
    finish(d, feat, n, max_dist, D, F);
done:
    free(d); free(feat); free(fv); free(featv); free(out); free(featout);
    free(ks); free(js);
    return rc;
}

/* The column scans alone on an M x L image (Fig. 19 after the downward scan
 * when down_only != 0, Fig. 18(b) after both scans).  Dv receives the int64 squared
 * vertical distances (max_dist = infinity), G the feature index. */
int oracle_column_pass2d(const uint8_t *mask, int M, int L, int mode,
                         int down_only, int64_t *Dv, int32_t *G)
{
    long n = (long)M * L;
    int shape[2] = {M, L};
    int64_t max_dist = oracle_max_dist(2, shape);
    init_sources(mask, n, mode, max_dist, Dv, G);
    for (long j = 0; j < L; ++j)
        column_scan(Dv + j, G + j, M, L, down_only);
    return 0;
}

/* The first scan of Sec. 3.3.1 on one line f[0..n-1] (values >= max_dist are
 * infinite).  Writes the contributors ks[0..cnt-1] and the starts js[0..cnt]
 * (0-based) and returns cnt. */
long oracle_envelope_state(const int64_t *f, long n, int64_t max_dist,
                           int64_t *ks, int64_t *js)
{
    return envelope_scan(f, n, 1, max_dist, ks, js);
}

/* The basic O(M L^2) row processing of Sec. 3.1 (row part of Listing 7), after the same column scans: each position starts
 * from its own vertical distance and takes any strictly smaller combination
 * D_v(k) + (k - j)^2.  A second, independent row pass for cross-checks. */
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
    int rc = 0;
    if (!d || !feat || !v || !fv) {
        rc = -1;
        goto done;
    }
    init_sources(mask, n, mode, max_dist, d, feat);
    for (long j = 0; j < L; ++j)
        column_scan(d + j, feat + j, M, L, 0);
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
    free(d); free(feat); free(v); free(fv);
    return rc;
}

/* Sec. 3.1: "the square root can be drawn after all squared distances have
 * been determined".  Reading: the float32 nearest to sqrt(D).  The square
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
