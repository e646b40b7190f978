// Driver of the host emulation of libedt's kernels (test infrastructure):
// runs the 2-D column and row kernels (single transforms and the fused pair),
// the 3-D passes, the city-block and chamfer passes and the persistent batch
// kernels on seeded random masks and compares the result with the
// CPU oracle: D exactly, F a source at squared distance D.
//   emu 2d PART NPARTS   2-D cases whose index is PART modulo NPARTS
//   emu 3d               3-D cases
//   emu batch            batches through the persistent kernels
//   emu maurer           the engine's hull test hidden() against Maurer's
//                        separating-line removal test on exhaustive triples
#include "shim.h"
#include "src/edt_internal.h"
#include "src/edt_engine.cuh"
extern "C" {
int oracle_edt2d(const uint8_t* mask, int M, int L, int mode, int32_t* D, int32_t* F);
int oracle_edt3d(const uint8_t* mask, int Z, int M, int L, int mode, int32_t* D, int32_t* F);
int oracle_cityblock2d(const uint8_t* mask, int M, int L, int mode, int stop, int32_t* D);
int oracle_chamfer43_2d(const uint8_t* mask, int M, int L, int mode, int stop, int32_t* D);
}
using namespace edt;

// The autotuner's table lives in a file the emulation does not build: the
// built-in geometry rules apply here.
Tuning edt::tuning_lookup(int, const int*) { return Tuning{}; }
BatchTuning edt::batch_tuning_lookup(int, const int*) { return BatchTuning{}; }
// As many SMs as a GB300 has: small images take the split row launch here too.
int edt::device_sm_count() { return 152; }

static uint64_t rng_state = 12345;
// features that are valid but name a different nearest source than the
// oracle's (both break ties the same way, so this should stay 0)
static long long g_f_differs = 0;
static void count_f(const int32_t* F, const std::vector<int32_t>& Fo, size_t n)
{
    for (size_t i = 0; i < n; ++i) g_f_differs += F[i] != Fo[i];
}
static double urand()
{
    rng_state = rng_state * 6364136223846793005ULL + 1442695040888963407ULL;
    return (rng_state >> 11) * (1.0 / 9007199254740992.0);
}

static int check_features(const std::vector<uint8_t>& mask, int H, int W, int mode, const int32_t* D,
                          const int32_t* F, const std::vector<int32_t>& Do)
{
    int bad = 0;
    const size_t n = (size_t)H * W;
    for (size_t i = 0; i < n && bad < 5; ++i) {
        if (D[i] != Do[i]) {
            fprintf(stderr, "D mismatch %dx%d mode %d at %zu: %d vs %d\n", H, W, mode, i, D[i], Do[i]);
            ++bad;
            continue;
        }
        if (Do[i] == INT32_MAX) {
            if (F[i] != -1) { fprintf(stderr, "F not -1 at %zu\n", i); ++bad; }
            continue;
        }
        const int64_t q = F[i];
        const bool src = q >= 0 && (size_t)q < n && (mode == 0 ? mask[q] != 0 : mask[q] == 0);
        const int64_t di = (int64_t)(i / W) - q / W, dj = (int64_t)(i % W) - q % W;
        if (!src || di * di + dj * dj != Do[i]) { fprintf(stderr, "F invalid %dx%d at %zu\n", H, W, i); ++bad; }
    }
    return bad;
}

static int32_t* alloc_words(size_t n) { return (int32_t*)aligned_alloc(256, (n * 4 + 255) / 256 * 256); }

static int run2d(int H, int W, double p, int mode, int align_off, bool pair)
{
    std::vector<uint8_t> mask((size_t)H * W);
    for (auto& m : mask) m = urand() < p;
    const ColGeom g = col_geom(H, W);
    std::vector<unsigned char> sa(col_scratch_bytes(g) + 256), sb(col_scratch_bytes(g) + 256);
    ColScratch s0 = col_scratch_carve((void*)(((uintptr_t)sa.data() + 255) & ~uintptr_t(255)), g);
    ColScratch s1 = col_scratch_carve((void*)(((uintptr_t)sb.data() + 255) & ~uintptr_t(255)), g);
    memset(s0.cnt, 0, g.ntiles * 4);
    memset(s1.cnt, 0, g.ntiles * 4);
    const size_t n = (size_t)H * W;
    // result arrays start align_off words after a 256-byte boundary
    int32_t* Db = alloc_words(n + align_off);
    int32_t* Fb = alloc_words(n + align_off);
    int32_t* Sb = alloc_words(n + align_off);
    int32_t* D1 = alloc_words(n);
    int32_t* F1 = alloc_words(n);
    int32_t *D = Db + align_off, *F = Fb + align_off;
    float* dist = reinterpret_cast<float*>(Sb + align_off);
    if (pair) {
        launch_colbits_pair(mask.data(), g, s0, s1, nullptr);
        launch_rows2d_pair(H, W, g, s0, s1, D, F, D1, F1, nullptr);
    } else {
        launch_colbits(mask.data(), g, mode, s0, nullptr);
        launch_rows2d(H, W, g, s0, D, F, dist, 0, nullptr);
    }
    int bad = 0;
    for (int k = 0; k < (pair ? 2 : 1); ++k) {
        const int mm = pair ? k : mode;
        std::vector<int32_t> Do(n), Fo(n);
        oracle_edt2d(mask.data(), H, W, mm, Do.data(), Fo.data());
        bad += check_features(mask, H, W, mm, k ? D1 : D, k ? F1 : F, Do);
        count_f(k ? F1 : F, Fo, (size_t)H * W);
        if (!pair)
            for (size_t i = 0; i < n && bad < 5; ++i) {
                const float want = Do[i] == INT32_MAX ? INFINITY : (float)std::sqrt((double)Do[i]);
                if (memcmp(&dist[i], &want, 4) != 0) { fprintf(stderr, "dist mismatch at %zu\n", i); ++bad; }
            }
    }
    free(Db); free(Fb); free(Sb); free(D1); free(F1);
    return bad;
}

static int run3d(int Dz, int H, int W, double p, int mode)
{
    std::vector<uint8_t> mask((size_t)Dz * H * W);
    for (auto& m : mask) m = urand() < p;
    const ColGeom g = col_geom(Dz, (int64_t)H * W);
    std::vector<unsigned char> scratch(col_scratch_bytes(g) + 256);
    ColScratch s = col_scratch_carve((void*)(((uintptr_t)scratch.data() + 255) & ~uintptr_t(255)), g);
    memset(s.cnt, 0, g.ntiles * 4);
    const size_t n = mask.size();
    int32_t* D = alloc_words(n);
    int32_t* F = alloc_words(n);
    float* dist = reinterpret_cast<float*>(alloc_words(n));
    short* d16 = reinterpret_cast<short*>(alloc_words((n + 1) / 2));   // the z offsets, as run_transform carves them
    launch_colbits(mask.data(), g, mode, s, nullptr);
    launch_zoffsets(Dz, H, W, g, s, d16, nullptr);
    launch_ypass3d(Dz, H, W, g, s, d16, reinterpret_cast<uint32_t*>(F), nullptr);
    launch_xpass3d(Dz, H, W, reinterpret_cast<uint32_t*>(F), D, F, dist, nullptr);
    std::vector<int32_t> Do(n), Fo(n);
    oracle_edt3d(mask.data(), Dz, H, W, mode, Do.data(), Fo.data());
    count_f(F, Fo, n);
    int bad = 0;
    for (size_t q = 0; q < n && bad < 5; ++q)
        if (D[q] != Do[q]) { fprintf(stderr, "3-D D mismatch %dx%dx%d at %zu: %d vs %d\n", Dz, H, W, q, D[q], Do[q]); ++bad; }
    free(D); free(F); free(dist); free(d16);
    return bad;
}

// D exactly and F a source at squared distance D, for a Dz x H x W volume.
static int check_features3d(const std::vector<uint8_t>& mask, int Dz, int H, int W, int mode, const int32_t* D,
                            const int32_t* F, const std::vector<int32_t>& Do)
{
    int bad = 0;
    const size_t n = (size_t)Dz * H * W;
    for (size_t i = 0; i < n && bad < 5; ++i) {
        if (D[i] != Do[i]) {
            fprintf(stderr, "3-D D mismatch %dx%dx%d mode %d at %zu: %d vs %d\n", Dz, H, W, mode, i, D[i], Do[i]);
            ++bad;
            continue;
        }
        if (Do[i] == INT32_MAX) {
            if (F[i] != -1) { fprintf(stderr, "3-D F not -1 at %zu\n", i); ++bad; }
            continue;
        }
        const int64_t q = F[i];
        const bool src = q >= 0 && (size_t)q < n && (mode == 0 ? mask[q] != 0 : mask[q] == 0);
        const int64_t plane = (int64_t)H * W;
        const int64_t dz = (int64_t)(i / plane) - q / plane, dy = (int64_t)((i % plane) / W) - (q % plane) / W,
                      dx = (int64_t)(i % W) - q % W;
        if (!src || dz * dz + dy * dy + dx * dx != Do[i]) {
            fprintf(stderr, "3-D F invalid %dx%dx%d at %zu\n", Dz, H, W, i);
            ++bad;
        }
    }
    return bad;
}

// A batch of mixed jobs (2-D up to 2048 wide, wider 2-D, 3-D) through the
// persistent kernels, with the table built by the library's batch_fill.
static int run_batch(int njobs, int blocks)
{
    struct Job {
        std::vector<uint8_t> mask;
        int ndim, shape[3], mode;
        int32_t *D, *F;
        size_t n;
    };
    std::vector<Job> js(njobs);
    const double ps[] = {0.0, 0.001, 0.02, 0.3, 1.0};
    for (int k = 0; k < njobs; ++k) {
        Job& j = js[k];
        const int kind = k % 4;
        if (kind == 3) {
            j.ndim = 3;
            j.shape[0] = 1 + (int)(urand() * 40);
            j.shape[1] = 1 + (int)(urand() * 70);
            j.shape[2] = 1 + (int)(urand() * 90);
        } else {
            j.ndim = 2;
            j.shape[0] = 1 + (int)(urand() * (kind == 2 ? 70 : 300));
            j.shape[1] = 1 + (int)(kind == 0 ? urand() * 2048 : kind == 2 ? 2049 + urand() * 3000 : urand() * 300);
            j.shape[2] = 0;
        }
        j.mode = k & 1;
        const double p = ps[k % 5];
        j.n = (size_t)j.shape[0] * j.shape[1] * (j.ndim == 3 ? j.shape[2] : 1);
        j.mask.resize(j.n);
        for (auto& m : j.mask) m = urand() < p;
        j.D = alloc_words(j.n);
        j.F = alloc_words(j.n);
    }
    // two 300 x 20 images with one source each (row 0, then row 1; column 5):
    // vertical offsets of 126, 127 and beyond in the same columns, on both
    // sides of the batch row search's int8 clamp
    for (int srow = 0; srow < 2; ++srow) {
        Job j;
        j.ndim = 2;
        j.shape[0] = 300;
        j.shape[1] = 20;
        j.shape[2] = 0;
        j.mode = 0;
        j.n = 300 * 20;
        j.mask.assign(j.n, 0);
        j.mask[(size_t)srow * 20 + 5] = 1;
        j.D = alloc_words(j.n);
        j.F = alloc_words(j.n);
        js.push_back(std::move(j));
    }
    njobs = (int)js.size();
    std::vector<edt_job> ej(njobs);
    for (int k = 0; k < njobs; ++k) {
        Job& j = js[k];
        ej[k] = edt_job{j.mask.data(), j.ndim, {j.shape[0], j.shape[1], j.shape[2]}, j.mode, j.D, j.F, nullptr};
        if (batch_kind(ej[k], nullptr) < 0) { fprintf(stderr, "job %d not batchable\n", k); return 1; }
    }
    size_t sb = 0;
    int64_t cw = 0;
    batch_layout(ej.data(), njobs, &sb, &cw);
    std::vector<unsigned char> scratch(sb + 256), cnt((size_t)cw * 4 + 256, 0xAB);
    std::vector<unsigned char> table(sizeof(BatchHeader) + (size_t)njobs * sizeof(BatchJob) + 256);
    auto* hdr = reinterpret_cast<BatchHeader*>(((uintptr_t)table.data() + 255) & ~uintptr_t(255));
    auto* tab = reinterpret_cast<BatchJob*>(hdr + 1);
    batch_fill(ej.data(), njobs, (char*)(((uintptr_t)scratch.data() + 255) & ~uintptr_t(255)),
               (unsigned*)(((uintptr_t)cnt.data() + 255) & ~uintptr_t(255)), hdr, tab);
    launch_batch_clear(hdr, blocks, nullptr);
    launch_batch_colbits(hdr, tab, blocks, nullptr);
    launch_batch_rows2d(hdr, tab, blocks, nullptr);
    launch_batch_wide(hdr, tab, blocks, nullptr);
    launch_batch_ypass3d(hdr, tab, blocks, nullptr);
    launch_batch_xpass3d(hdr, tab, blocks, nullptr);
    int bad = 0;
    for (Job& j : js) {
        std::vector<int32_t> Do(j.n), Fo(j.n);
        if (j.ndim == 2) {
            oracle_edt2d(j.mask.data(), j.shape[0], j.shape[1], j.mode, Do.data(), Fo.data());
            bad += check_features(j.mask, j.shape[0], j.shape[1], j.mode, j.D, j.F, Do);
            count_f(j.F, Fo, j.n);
        } else {
            oracle_edt3d(j.mask.data(), j.shape[0], j.shape[1], j.shape[2], j.mode, Do.data(), Fo.data());
            bad += check_features3d(j.mask, j.shape[0], j.shape[1], j.shape[2], j.mode, j.D, j.F, Do);
            count_f(j.F, Fo, j.n);
        }
        free(j.D);
        free(j.F);
    }
    return bad;
}

static int run_cityblock(int H, int W, double p, int mode, int align_off)
{
    std::vector<uint8_t> mask((size_t)H * W);
    for (auto& m : mask) m = urand() < p;
    const ColGeom g = col_geom(H, W);
    std::vector<unsigned char> sa(col_scratch_bytes(g) + 256);
    ColScratch s = col_scratch_carve((void*)(((uintptr_t)sa.data() + 255) & ~uintptr_t(255)), g);
    memset(s.cnt, 0, g.ntiles * 4);
    const size_t n = (size_t)H * W;
    int32_t* Db = alloc_words(n + align_off);
    int32_t* D = Db + align_off;
    launch_colbits(mask.data(), g, mode, s, nullptr);
    launch_cityblock_rows(H, W, g, s, D, nullptr);
    std::vector<int32_t> Do(n);
    oracle_cityblock2d(mask.data(), H, W, mode, 0, Do.data());
    int bad = 0;
    for (size_t i = 0; i < n && bad < 5; ++i)
        if (D[i] != Do[i]) { fprintf(stderr, "city-block mismatch %dx%d mode %d at %zu: %d vs %d\n", H, W, mode, i, D[i], Do[i]); ++bad; }
    free(Db);
    return bad;
}

static int run_chamfer(int H, int W, double p, int mode)
{
    std::vector<uint8_t> mask((size_t)H * W);
    for (auto& m : mask) m = urand() < p;
    std::vector<unsigned char> scratch(chamfer_scratch_bytes(H, W) + 256);
    void* sbase = (void*)(((uintptr_t)scratch.data() + 255) & ~uintptr_t(255));
    const size_t n = (size_t)H * W;
    int32_t* D = alloc_words(n);
    launch_chamfer(mask.data(), H, W, mode, D, sbase, 4, nullptr);
    std::vector<int32_t> Do(n);
    oracle_chamfer43_2d(mask.data(), H, W, mode, 0, Do.data());
    int bad = 0;
    for (size_t i = 0; i < n && bad < 5; ++i)
        if (D[i] != Do[i]) { fprintf(stderr, "chamfer mismatch %dx%d mode %d at %zu: %d vs %d\n", H, W, mode, i, D[i], Do[i]); ++bad; }
    free(D);
    return bad;
}

// Maurer, Qi and Raghavan (2003), "A linear time algorithm for computing exact
// Euclidean distance transforms of binary images in arbitrary dimensions",
// the removal test of their row pass: with sites at u < v < w on the line,
// squared distances f(u), f(v), f(w) from the line to them, a = v - u,
// b = w - v and c = a + b, site v is removed (its parabola never gives the
// minimum) when  c f(v) - b f(u) - a f(w) - a b c > 0.  The paper's Sec. 4
// names this approach as an alternative to the one of Sec. 3.3.1.
static long long maurer_lhs(long long u, long long fu, long long v, long long fv, long long w, long long fw)
{
    const long long a = v - u, b = w - v, c = a + b;
    return c * fv - b * fu - a * fw - a * b * c;
}

// For every triple u < v < w < n and every f in 0..fmax (plus a spread of
// larger values), the engine's hidden() must equal Maurer's removal test
// except where the three parabolas meet in one point (left-hand side 0),
// where hidden() removes v and Maurer keeps it; there the envelope's value
// at every integer position is the same with and without v.
static int run_maurer(int n, int fmax)
{
    std::vector<long long> fs;
    for (int f = 0; f <= fmax; ++f) fs.push_back(f);
    for (long long f : {20LL, 25LL, 49LL, 100LL, 101LL, 250LL, 1000LL, 4095LL, 65536LL, 1LL << 24}) fs.push_back(f);
    long long agree = 0, coincide = 0, bad = 0;
    for (int u = 0; u < n; ++u)
        for (int v = u + 1; v < n; ++v)
            for (int w = v + 1; w < n; ++w)
                for (long long fu : fs)
                    for (long long fv : fs)
                        for (long long fw : fs) {
                            const bool h = edt::hidden(u, (int)(fu + u * u), v, (int)(fv + v * v), w,
                                                       (int)(fw + w * w));
                            const long long lhs = maurer_lhs(u, fu, v, fv, w, fw);
                            const bool remove = lhs > 0;
                            if (h == remove) { ++agree; continue; }
                            if (lhs == 0 && h) {
                                ++coincide;
                                // v never lies strictly below both u and w
                                for (int j = -2 * n; j <= 3 * n; ++j) {
                                    const long long pu = fu + (long long)(j - u) * (j - u);
                                    const long long pv = fv + (long long)(j - v) * (j - v);
                                    const long long pw = fw + (long long)(j - w) * (j - w);
                                    if (pv < std::min(pu, pw)) { ++bad; break; }
                                }
                                continue;
                            }
                            if (bad < 5)
                                fprintf(stderr, "hidden %d vs Maurer %d at u %d v %d w %d f %lld %lld %lld\n", h,
                                        remove, u, v, w, fu, fv, fw);
                            ++bad;
                        }
    printf("maurer triples agree %lld coincide %lld bad %lld\n", agree, coincide, bad);
    return bad != 0;
}

int main(int argc, char** argv)
{
    if (argc > 1 && !strcmp(argv[1], "maurer")) {
        const int n = argc > 2 ? atoi(argv[2]) : 64, fmax = argc > 3 ? atoi(argv[3]) : 12;
        return run_maurer(n, fmax);
    }
    if (argc > 1 && !strcmp(argv[1], "chamfer")) {
        const int part = argc > 3 ? atoi(argv[2]) : 0, nparts = argc > 3 ? atoi(argv[3]) : 1;
        int bad = 0, cases = 0, run = 0;
        const int shapes[][2] = {{1, 1}, {1, 9}, {9, 1}, {5, 7}, {33, 31}, {64, 100}, {130, 70}, {40, 513},
                                 {3, 2048}, {2, 8200}, {300, 40}, {17, 14336}, {1100, 33}};
        for (auto& sh : shapes)
            for (double p : {0.0, 0.003, 0.05, 1.0}) {
                const int c = cases++;
                if (c % nparts != part) { for (long long i = 0; i < (long long)sh[0] * sh[1]; ++i) urand(); continue; }
                ++run;
                bad += run_chamfer(sh[0], sh[1], p, c & 1);
            }
        printf("chamfer cases %d bad %d\n", run, bad);
        return bad != 0;
    }
    if (argc > 1 && !strcmp(argv[1], "cityblock")) {
        const int part = argc > 3 ? atoi(argv[2]) : 0, nparts = argc > 3 ? atoi(argv[3]) : 1;
        int bad = 0, cases = 0, run = 0;
        const int shapes[][2] = {{1, 1}, {1, 9}, {9, 1}, {5, 7}, {33, 31}, {64, 100}, {40, 513}, {3, 2048},
                                 {2, 8192}, {9, 8200}, {2, 16384}, {1100, 33}};
        for (auto& sh : shapes)
            for (double p : {0.0, 0.003, 0.05, 1.0}) {
                const int c = cases++;
                if (c % nparts != part) { for (long long i = 0; i < (long long)sh[0] * sh[1]; ++i) urand(); continue; }
                ++run;
                bad += run_cityblock(sh[0], sh[1], p, c & 1, c % 3 == 0 ? 4 : 0);
            }
        printf("cityblock cases %d bad %d\n", run, bad);
        return bad != 0;
    }
    if (argc > 1 && !strcmp(argv[1], "batch")) {
        int bad = 0, cases = 0;
        for (int njobs : {1, 5, 17})
            for (int blocks : {1, 3}) {
                bad += run_batch(njobs, blocks);
                ++cases;
            }
        printf("batch cases %d bad %d f_differs %lld\n", cases, bad, g_f_differs);
        return bad != 0;
    }
    if (argc > 1 && !strcmp(argv[1], "3d")) {
        int bad = 0, cases = 0;
        const int shapes[][3] = {{1, 1, 1}, {3, 5, 7}, {1, 40, 50}, {40, 1, 50}, {40, 50, 1},
                                 {32, 33, 31}, {33, 32, 65}, {70, 17, 129}, {9, 17, 1000}, {5, 300, 40},
                                 {1100, 2, 3}};
        for (auto& sh : shapes)
            for (double p : {0.001, 0.05, 0.5})
                for (int mode = 0; mode < 2; ++mode) {
                    bad += run3d(sh[0], sh[1], sh[2], p, mode);
                    ++cases;
                }
        printf("3d cases %d bad %d f_differs %lld\n", cases, bad, g_f_differs);
        return bad != 0;
    }
    const int part = argc > 3 ? atoi(argv[2]) : 0, nparts = argc > 3 ? atoi(argv[3]) : 1;
    const int Hs[] = {1, 2, 33, 64, 100, 1100, 2100};
    const int Ws[] = {1, 5, 16, 31, 32, 48, 100, 513, 1024, 2048, 2052, 4100, 8192};
    const double ps[] = {0.0, 0.001, 0.02, 0.3, 1.0};
    int cases = 0, run = 0, bad = 0;
    for (int H : Hs)
        for (int W : Ws) {
            if ((long long)H * W > 300000) continue;
            for (double p : ps) {
                const int c = cases++;
                if (c % nparts != part) { for (long long i = 0; i < (long long)H * W; ++i) urand(); continue; }
                ++run;
                bad += run2d(H, W, p, c & 1, (c % 3 == 0) ? 4 : ((c % 7 == 0) ? 1 : 0), c % 5 == 0);
            }
        }
    printf("2d cases %d bad %d f_differs %lld\n", run, bad, g_f_differs);
    return bad != 0;
}
