/*
 * Oracle for the propagation transforms of T. Strutz, "The Distance
 * Transform and its Computation -- An Introduction", Section 2: the
 * city-block distance transform (Sec. 2.1), the chamfer 4-3 distance
 * transform (Sec. 2.2) and Danielsson's approximate Euclidean transform
 * (Sec. 2.3, at the end of this file).
 *
 * TEST INFRASTRUCTURE ONLY, like edt_oracle.c: plain single-threaded C that
 * the tests, the smoke check and the benchmark's CPU baseline may load; the
 * CUDA library never does, and the two share no code.
 *
 * Both transforms follow the paper's scans as its text states them:
 *   - initialisation (Sec. 2.1, Fig. 12(a)): 0 on source pixels, a value
 *     larger than any distance elsewhere;
 *   - city-block, sequential (Sec. 2.1): a forward raster scan (top-left to
 *     bottom-right) that lowers d(i,j) to d(i,j-1)+1 and then to d(i-1,j)+1,
 *     and a backward raster scan with d(i,j+1)+1 and d(i+1,j)+1 (Fig. 12);
 *   - city-block, four scans (Sec. 2.1): every column downward and upward,
 *     then every row forward and backward, one comparison per step (Fig. 13);
 *   - chamfer 4-3 (Sec. 2.2): the forward scan with weight 3 to the left and
 *     upper neighbours and 4 to the two upper diagonal neighbours, the
 *     backward scan mirrored (Fig. 15).
 * Readings (the paper is silent or its listing differs):
 *   - mode 0: sources are the nonzero bytes (Fig. 1c, the case Sec. 2
 *     treats); mode 1: sources are the zero bytes (Fig. 1b).
 *   - a neighbour outside the image is skipped.  (The city-block listing
 *     starts its inner loops at the second column, which leaves the first
 *     column without the downward comparison of the forward scan; the text
 *     asks for it "for all (i, j)", and only then is the result the
 *     city-block distance for sources in the first column.)
 *   - pixels still at the initial value when the scans end (an image without
 *     sources) get INT32_MAX; "stop" options return an intermediate state with
 *     INT32_MAX where the initial value is still present.
 * Distances are int64_t inside, int32_t out.
 */
#include <stdint.h>
#include <stdlib.h>

/* Initial value: larger than any distance of the image plus any step. */
static int64_t big_value(int M, int L) { return 4 * ((int64_t)M + L) + 16; }

static int is_source(const uint8_t *mask, long p, int mode)
{
    return mode == 0 ? mask[p] != 0 : mask[p] == 0;
}

static int64_t *init_grid(const uint8_t *mask, int M, int L, int mode, int64_t big)
{
    long n = (long)M * L;
    int64_t *d = (int64_t *)malloc(sizeof(int64_t) * (n ? n : 1));
    if (!d) return NULL;
    for (long p = 0; p < n; ++p) d[p] = is_source(mask, p, mode) ? 0 : big;
    return d;
}

/* lower d[p] to d[q] + w */
static void relax(int64_t *d, long p, long q, int64_t w)
{
    if (d[p] > d[q] + w) d[p] = d[q] + w;
}

static void put(const int64_t *d, long n, int64_t big, int32_t *D)
{
    for (long p = 0; p < n; ++p) D[p] = d[p] >= big ? INT32_MAX : (int32_t)d[p];
}

/* Sec. 2.1, sequential city-block transform (two raster scans); stop = 1
 * returns the state after the forward scan (Fig. 12(b)). */
int oracle_cityblock2d(const uint8_t *mask, int M, int L, int mode, int stop, int32_t *D)
{
    const int64_t big = big_value(M, L);
    int64_t *d = init_grid(mask, M, L, mode, big);
    if (!d) return 1;
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < L; ++j) {
            const long p = (long)i * L + j;
            if (j > 0) relax(d, p, p - 1, 1);
            if (i > 0) relax(d, p, p - L, 1);
        }
    if (!stop)
        for (int i = M - 1; i >= 0; --i)
            for (int j = L - 1; j >= 0; --j) {
                const long p = (long)i * L + j;
                if (j < L - 1) relax(d, p, p + 1, 1);
                if (i < M - 1) relax(d, p, p + L, 1);
            }
    put(d, (long)M * L, big, D);
    free(d);
    return 0;
}

/* Sec. 2.1, the four-scan variant: columns down and up, then rows forward and
 * backward; stop = 1 returns the state after the column scans (Fig. 13(b)). */
int oracle_cityblock2d_4scan(const uint8_t *mask, int M, int L, int mode, int stop, int32_t *D)
{
    const int64_t big = big_value(M, L);
    int64_t *d = init_grid(mask, M, L, mode, big);
    if (!d) return 1;
    for (int j = 0; j < L; ++j) {
        for (int i = 1; i < M; ++i) relax(d, (long)i * L + j, (long)(i - 1) * L + j, 1);
        for (int i = M - 2; i >= 0; --i) relax(d, (long)i * L + j, (long)(i + 1) * L + j, 1);
    }
    if (!stop)
        for (int i = 0; i < M; ++i) {
            for (int j = 1; j < L; ++j) relax(d, (long)i * L + j, (long)i * L + j - 1, 1);
            for (int j = L - 2; j >= 0; --j) relax(d, (long)i * L + j, (long)i * L + j + 1, 1);
        }
    put(d, (long)M * L, big, D);
    free(d);
    return 0;
}

/* Sec. 2.2, chamfer 4-3 transform (two raster scans, weights 3 for the
 * horizontal / vertical and 4 for the diagonal neighbours); stop = 1 returns
 * the state after the forward scan (Fig. 15(a)). */
int oracle_chamfer43_2d(const uint8_t *mask, int M, int L, int mode, int stop, int32_t *D)
{
    const int64_t big = big_value(M, L) * 4;
    int64_t *d = init_grid(mask, M, L, mode, big);
    if (!d) return 1;
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < L; ++j) {
            const long p = (long)i * L + j;
            if (j > 0) relax(d, p, p - 1, 3);
            if (i > 0) relax(d, p, p - L, 3);
            if (i > 0 && j > 0) relax(d, p, p - L - 1, 4);
            if (i > 0 && j < L - 1) relax(d, p, p - L + 1, 4);
        }
    if (!stop)
        for (int i = M - 1; i >= 0; --i)
            for (int j = L - 1; j >= 0; --j) {
                const long p = (long)i * L + j;
                if (j < L - 1) relax(d, p, p + 1, 3);
                if (i < M - 1) relax(d, p, p + L, 3);
                if (i < M - 1 && j > 0) relax(d, p, p + L - 1, 4);
                if (i < M - 1 && j < L - 1) relax(d, p, p + L + 1, 4);
            }
    put(d, (long)M * L, big, D);
    free(d);
    return 0;
}

/*
 * Sec. 2.3, Danielsson's approximate Euclidean transform in the form the
 * paper gives it (after Grevera): every pixel carries a relative position
 * (dy, dx) with non-negative components, (0, 0) on sources, none elsewhere.
 * Looking at a neighbour, a pixel takes the neighbour's position with dy
 * increased by one for a vertical step, dx for a horizontal one and both for
 * a diagonal one, when dy^2 + dx^2 of that is strictly below its own.
 * Forward scan, rows 1 .. M-1 (0-based; the first row is skipped), per row:
 *   (a) every column: the upper neighbour;
 *   (b) columns 1 .. L-1 left to right: the left, then the upper-left one;
 *   (c) columns L-2 .. 0 right to left: the upper-right, then the right one.
 * Backward scan, rows M-2 .. 0, mirrored vertically:
 *   (a) every column: the lower neighbour;
 *   (b) left to right: the left, then the lower-left one;
 *   (c) right to left: the right, then the lower-right one.
 * Readings: inside (c) of the forward scan the paper's listing looks at the
 * upper-right neighbour first and its text names the right neighbour first;
 * `order` selects the listing's order (0, the default reading) or the text's
 * (1).  Only ties of length between the two looks depend on it, and no mask
 * of up to 24 pixels tells them apart; the accuracy against the exact
 * transform is reported under both.  A single-row image is visited by
 * neither scan, so only its sources get a position.
 * Pins: Fig. 16(b) and 16(c) fix the passes, the increments and the strict
 * comparison (a plant of any of those fails them); a 4 x 4 mask derived by
 * hand from the text fixes the diagonal looks (without them one cell ends at
 * 9 instead of 8); the tests check the invariants below.  The order of the
 * two looks inside (b) and (c) is unpinned: no example within reach of a
 * hand derivation separates the orders.
 * stop = 1 returns the state after the forward scan (Fig. 16(b)).
 * Out: D = dy^2 + dx^2 (INT32_MAX without a position), DY, DX (-1 there).
 */
typedef struct {
    int64_t *dy, *dx;  /* -1 = no position yet */
    int L;
} RelPos;

static int64_t rel_len(const RelPos *r, long p)
{
    return r->dy[p] < 0 ? INT64_MAX : r->dy[p] * r->dy[p] + r->dx[p] * r->dx[p];
}

/* let pixel p look at neighbour q, with the step (sy, sx) in {0, 1}^2 */
static void take(RelPos *r, long p, long q, int sy, int sx)
{
    if (r->dy[q] < 0) return;
    const int64_t ny = r->dy[q] + sy, nx = r->dx[q] + sx;
    if (rel_len(r, p) > ny * ny + nx * nx) {
        r->dy[p] = ny;
        r->dx[p] = nx;
    }
}

/* one row of a scan; v = -1 looks at the row above, +1 at the row below;
 * order 1 looks right before upper-right in (c) of the forward scan */
static void danielsson_row(RelPos *r, int i, int v, int order)
{
    const int L = r->L;
    const long row = (long)i * L, nb = (long)(i + v) * L;
    for (int j = 0; j < L; ++j) take(r, row + j, nb + j, 1, 0);
    for (int j = 1; j < L; ++j) {
        take(r, row + j, row + j - 1, 0, 1);
        take(r, row + j, nb + j - 1, 1, 1);
    }
    for (int j = L - 2; j >= 0; --j) {
        if (v < 0 && order == 0) {
            take(r, row + j, nb + j + 1, 1, 1);
            take(r, row + j, row + j + 1, 0, 1);
        } else {
            take(r, row + j, row + j + 1, 0, 1);
            take(r, row + j, nb + j + 1, 1, 1);
        }
    }
}

int oracle_danielsson2d(const uint8_t *mask, int M, int L, int mode, int stop, int order, int32_t *D,
                        int32_t *DY, int32_t *DX)
{
    const long n = (long)M * L;
    RelPos r;
    r.L = L;
    r.dy = (int64_t *)malloc(sizeof(int64_t) * (n ? n : 1));
    r.dx = (int64_t *)malloc(sizeof(int64_t) * (n ? n : 1));
    if (!r.dy || !r.dx) {
        free(r.dy);
        free(r.dx);
        return 1;
    }
    for (long p = 0; p < n; ++p) r.dy[p] = r.dx[p] = is_source(mask, p, mode) ? 0 : -1;
    for (int i = 1; i < M; ++i) danielsson_row(&r, i, -1, order);
    if (!stop)
        for (int i = M - 2; i >= 0; --i) danielsson_row(&r, i, +1, order);
    for (long p = 0; p < n; ++p) {
        const int64_t len = rel_len(&r, p);
        D[p] = len == INT64_MAX || len > INT32_MAX ? INT32_MAX : (int32_t)len;
        DY[p] = (int32_t)r.dy[p];
        DX[p] = (int32_t)r.dx[p];
    }
    free(r.dy);
    free(r.dx);
    return 0;
}
