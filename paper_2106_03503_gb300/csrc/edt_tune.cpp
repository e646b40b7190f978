// Autotuner for the band geometry (edt_autotune, edt_tune_get / _save /
// _load).  The envelope passes split each band of 32 lines into segments, one
// per warp; how many warps a band gets (and so how long the segments are)
// trades per-warp work against merge depth and resident blocks, and the best
// choice depends on the shape.  The built-in rules (16 warps for 2-D rows, 8
// for the 3-D y pass, 32 for the x pass, fewer when shared memory does not
// fit) were measured on the benchmark shapes; edt_autotune times the
// candidates on the caller's own mask and keeps the fastest for its shape
// class.  edt_autotune_batch does the same for the geometry of the batch
// kernels (the smallest row segment of narrow 2-D jobs, the positions per warp
// of the 3-D y and x passes), timing each shape class of the caller's batch
// on its own, then keeping those choices only if the whole batch runs faster
// with them than with the built-in geometry.  A choice never changes a
// result: every segmentation gives the same D and F, bit for bit.
#include <algorithm>
#include <array>
#include <cstdio>
#include <map>
#include <mutex>
#include <vector>

#include "edt_internal.h"

namespace edt {
edt_status fail(edt_status st, const char* fmt, ...);
edt_status cuda_fail(cudaError_t e, const char* what);
void clear_error();
edt_status device_setup(int* sm_count);
edt_status check_shape(int ndim, const int* shape, int mode);
size_t scratch_bytes(int ndim, const int* shape);
edt_status run_transform(const uint8_t* mask, int ndim, const int* shape, int mode,
                         int32_t* D, int32_t* F, float* dist, void* scratch,
                         int sm_count, cudaStream_t stream);

namespace {

using Key = std::array<int, 4>;   // ndim, then ceil(log2(side)) per axis

std::mutex g_tune_mu;
std::map<Key, Tuning> g_tune;
std::map<Key, BatchTuning> g_btune;    // batch geometry per shape class

int ceil_log2(int v)
{
    int l = 0;
    while ((1 << l) < v && l < 30) ++l;
    return l;
}

Key key_of(int ndim, const int* shape)
{
    Key k{ndim, 0, 0, 0};
    for (int a = 0; a < ndim && a < 3; ++a) k[1 + a] = ceil_log2(shape[a]);
    return k;
}

}  // namespace

Tuning tuning_lookup(int ndim, const int* shape)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_tune.empty()) return Tuning{};
    auto it = g_tune.find(key_of(ndim, shape));
    return it == g_tune.end() ? Tuning{} : it->second;
}

void tuning_store(int ndim, const int* shape, const Tuning& t)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key_of(ndim, shape)] = t;
}

BatchTuning batch_tuning_lookup(int ndim, const int* shape)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (g_btune.empty()) return BatchTuning{};
    auto it = g_btune.find(key_of(ndim, shape));
    return it == g_btune.end() ? BatchTuning{} : it->second;
}

void batch_tuning_store(int ndim, const int* shape, const BatchTuning& t)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_btune[key_of(ndim, shape)] = t;
}

edt_status batch_enqueue(edt_plan* p, const edt_job* jobs, int n, char* scratch, cudaStream_t stream);
int plan_n_max(const edt_plan* p);

}  // namespace edt

using namespace edt;

extern "C" edt_status edt_autotune(const uint8_t* mask, int ndim, const int* shape, int mode,
                                   edt_stream_t stream_)
{
    if (!mask) return fail(EDT_ERR_INVALID, "mask is NULL");
    edt_status st = check_shape(ndim, shape, mode);
    if (st != EDT_OK) return st;
    int sms = 0;
    if ((st = device_setup(&sms)) != EDT_OK) return st;
    cudaStream_t stream = (cudaStream_t)stream_;
    int64_t n = 1;
    for (int a = 0; a < ndim; ++a) n *= shape[a];
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t sb = al(scratch_bytes(ndim, shape));
    char* dev = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&dev, 2 * al((size_t)n * 4) + sb, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    int32_t* D = reinterpret_cast<int32_t*>(dev);
    int32_t* F = reinterpret_cast<int32_t*>(dev + al((size_t)n * 4));
    void* scratch = dev + 2 * al((size_t)n * 4);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    for (auto& x : ev)
        if (st == EDT_OK && (e = cudaEventCreate(&x)) != cudaSuccess) st = cuda_fail(e, "cudaEventCreate");

    // milliseconds per transform with tuning t (one untimed run, then two)
    auto time_with = [&](const Tuning& t) -> float {
        tuning_store(ndim, shape, t);
        if (run_transform(mask, ndim, shape, mode, D, F, nullptr, scratch, sms, stream) != EDT_OK) return -1.f;
        cudaEventRecord(ev[0], stream);
        for (int r = 0; r < 2; ++r)
            if (run_transform(mask, ndim, shape, mode, D, F, nullptr, scratch, sms, stream) != EDT_OK) return -1.f;
        cudaEventRecord(ev[1], stream);
        if (cudaEventSynchronize(ev[1]) != cudaSuccess) return -1.f;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        return ms / 2;
    };
    Tuning best{};
    if (st == EDT_OK) {
        if (ndim == 2) {
            float best_ms = -1.f;
            for (int nw : {16, 8, 4}) {
                Tuning t;
                t.rows2d_nw = nw;
                const float ms = time_with(t);
                if (ms < 0) { st = fail(EDT_ERR_CUDA, "autotune: a candidate failed"); break; }
                if (best_ms < 0 || ms < best_ms) { best_ms = ms; best = t; }
            }
        } else {
            // the y pass first with the x pass at its rule, then the x pass
            float best_ms = -1.f;
            for (int nw : {8, 4, 16, 32}) {
                Tuning t;
                t.ypass_nw = nw;
                const float ms = time_with(t);
                if (ms < 0) { st = fail(EDT_ERR_CUDA, "autotune: a candidate failed"); break; }
                if (best_ms < 0 || ms < best_ms) { best_ms = ms; best = t; }
            }
            for (int nw : {16, 8}) {
                if (st != EDT_OK) break;
                Tuning t = best;
                t.xpass_nw = nw;
                const float ms = time_with(t);
                if (ms < 0) { st = fail(EDT_ERR_CUDA, "autotune: a candidate failed"); break; }
                if (ms < best_ms) { best_ms = ms; best = t; }
            }
            if (st == EDT_OK && best.xpass_nw == 0) best.xpass_nw = 32;
        }
    }
    if (st == EDT_OK) tuning_store(ndim, shape, best);
    else tuning_store(ndim, shape, Tuning{});   // back to the rules after a failure
    cudaFreeAsync(dev, stream);
    e = cudaStreamSynchronize(stream);
    if (st == EDT_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize");
    for (auto& x : ev)
        if (x) cudaEventDestroy(x);
    if (st == EDT_OK) clear_error();
    return st;
}

extern "C" edt_status edt_autotune_batch(edt_plan* plan, const edt_job* jobs, int n, edt_stream_t stream_)
{
    if (!plan || !jobs || n <= 0) return fail(EDT_ERR_INVALID, "plan, jobs and n > 0 are required");
    const int n_max = plan_n_max(plan);
    if (n > n_max) return fail(EDT_ERR_INVALID, "%d jobs exceed the plan's %d", n, n_max);
    const int chunk = std::min(256, n_max);   // jobs per timed replay
    cudaStream_t stream = (cudaStream_t)stream_;
    for (int i = 0; i < n; ++i) {
        edt_status st = check_shape(jobs[i].ndim, jobs[i].shape, jobs[i].mode);
        if (st != EDT_OK) return st;
        const char* why = "";
        if (!jobs[i].mask || !jobs[i].F) return fail(EDT_ERR_INVALID, "job %d: mask and F must not be NULL", i);
        if (batch_kind(jobs[i], &why) < 0) return fail(EDT_ERR_TOO_LARGE, "job %d: %s", i, why);
    }
    // the jobs of each shape class, timed on their own
    std::map<Key, std::vector<edt_job>> classes;
    for (int i = 0; i < n; ++i) classes[key_of(jobs[i].ndim, jobs[i].shape)].push_back(jobs[i]);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    edt_status st = EDT_OK;
    cudaError_t e;
    for (auto& x : ev)
        if (st == EDT_OK && (e = cudaEventCreate(&x)) != cudaSuccess) st = cuda_fail(e, "cudaEventCreate");
    for (auto& kv : classes) {
        if (st != EDT_OK) break;
        std::vector<edt_job>& cj = kv.second;
        const edt_job& j0 = cj[0];
        const int kind = batch_kind(j0, nullptr);
        if (kind == BATCH_2D_WIDE) continue;   // no knob
        auto time_with = [&](const BatchTuning& t) -> float {
            batch_tuning_store(j0.ndim, j0.shape, t);
            float total = 0.f;
            for (size_t off = 0; off < cj.size(); off += (size_t)chunk) {
                const int cnt = (int)std::min<size_t>((size_t)chunk, cj.size() - off);
                if (batch_enqueue(plan, cj.data() + off, cnt, nullptr, stream) != EDT_OK) return -1.f;
                cudaEventRecord(ev[0], stream);
                for (int r = 0; r < 3; ++r)
                    if (batch_enqueue(plan, cj.data() + off, cnt, nullptr, stream) != EDT_OK) return -1.f;
                cudaEventRecord(ev[1], stream);
                if (cudaEventSynchronize(ev[1]) != cudaSuccess) return -1.f;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[0], ev[1]);
                total += ms / 3;
            }
            return total;
        };
        BatchTuning best{};
        float best_ms = -1.f;
        auto consider = [&](const BatchTuning& t) {
            const float ms = time_with(t);
            if (ms < 0) { st = fail(EDT_ERR_CUDA, "autotune_batch: a candidate failed"); return; }
            if (best_ms < 0 || ms < best_ms) { best_ms = ms; best = t; }
        };
        if (kind == BATCH_2D) {
            for (int lgmin : {8, 7, 6}) {
                BatchTuning t;
                t.rows2d_lgmin = lgmin;
                consider(t);
                if (st != EDT_OK) break;
            }
        } else {
            for (int pos : {64, 32, 128}) {      // y pass, x pass at its rule
                BatchTuning t;
                t.y_pos = pos;
                t.x_pos = 32;
                consider(t);
                if (st != EDT_OK) break;
            }
            const int ybest = best.y_pos;
            for (int pos : {64, 128}) {
                if (st != EDT_OK) break;
                BatchTuning t;
                t.y_pos = ybest;
                t.x_pos = pos;
                consider(t);
            }
        }
        batch_tuning_store(j0.ndim, j0.shape, st == EDT_OK ? best : BatchTuning{});
    }
    // the classes were timed alone, where a replay's fixed costs weigh more
    // than in the whole batch: keep the choices only if the whole batch is
    // faster with them than with the built-in geometry
    if (st == EDT_OK) {
        auto time_all = [&]() -> float {
            if (batch_enqueue(plan, jobs, n, nullptr, stream) != EDT_OK) return -1.f;   // warm
            cudaEventRecord(ev[0], stream);
            for (int r = 0; r < 3; ++r)
                if (batch_enqueue(plan, jobs, n, nullptr, stream) != EDT_OK) return -1.f;
            cudaEventRecord(ev[1], stream);
            if (cudaEventSynchronize(ev[1]) != cudaSuccess) return -1.f;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[0], ev[1]);
            return ms;
        };
        // the two alternated twice, the better time of each kept; the choices
        // stay only when they are faster by more than 1 %, so that timing
        // noise does not decide
        std::map<Key, BatchTuning> chosen;
        for (auto& kv : classes) chosen[kv.first] = batch_tuning_lookup(kv.second[0].ndim, kv.second[0].shape);
        auto use = [&](bool builtin) {
            for (auto& kv : classes)
                batch_tuning_store(kv.second[0].ndim, kv.second[0].shape, builtin ? BatchTuning{} : chosen[kv.first]);
        };
        float t_chosen = -1.f, t_builtin = -1.f;
        bool ok = true;
        for (int round = 0; round < 2 && ok; ++round)
            for (int builtin = 0; builtin < 2 && ok; ++builtin) {
                use(builtin != 0);
                const float t = time_all();
                float& best = builtin ? t_builtin : t_chosen;
                ok = t >= 0.f;
                if (ok && (best < 0.f || t < best)) best = t;
            }
        if (!ok) {
            use(true);
            st = fail(EDT_ERR_CUDA, "autotune_batch: timing the whole batch failed");
        } else {
            use(!(t_chosen < 0.99f * t_builtin));
        }
    }
    e = cudaStreamSynchronize(stream);
    if (st == EDT_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize");
    for (auto& x : ev)
        if (x) cudaEventDestroy(x);
    if (st == EDT_OK) clear_error();
    return st;
}

extern "C" edt_status edt_batch_tune_get(int ndim, const int* shape, int* values)
{
    if (!shape || !values) return fail(EDT_ERR_INVALID, "NULL argument");
    if (ndim != 2 && ndim != 3) return fail(EDT_ERR_INVALID, "ndim must be 2 or 3, got %d", ndim);
    for (int a = 0; a < ndim; ++a)
        if (shape[a] <= 0) return fail(EDT_ERR_INVALID, "shape[%d] = %d must be positive", a, shape[a]);
    const BatchTuning t = batch_tuning_lookup(ndim, shape);
    values[0] = t.rows2d_lgmin;
    values[1] = t.y_pos;
    values[2] = t.x_pos;
    clear_error();
    return EDT_OK;
}

extern "C" edt_status edt_tune_get(int ndim, const int* shape, int* warps)
{
    if (!shape || !warps) return fail(EDT_ERR_INVALID, "NULL argument");
    if (ndim != 2 && ndim != 3) return fail(EDT_ERR_INVALID, "ndim must be 2 or 3, got %d", ndim);
    for (int a = 0; a < ndim; ++a)
        if (shape[a] <= 0) return fail(EDT_ERR_INVALID, "shape[%d] = %d must be positive", a, shape[a]);
    const Tuning t = tuning_lookup(ndim, shape);
    warps[0] = t.rows2d_nw;
    warps[1] = t.ypass_nw;
    warps[2] = t.xpass_nw;
    clear_error();
    return EDT_OK;
}

extern "C" edt_status edt_tune_save(const char* path)
{
    if (!path) return fail(EDT_ERR_INVALID, "path is NULL");
    FILE* f = std::fopen(path, "w");
    if (!f) return fail(EDT_ERR_INVALID, "cannot write %s", path);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        std::fprintf(f, "# libedt tuning: ndim log2-sides(3) rows2d_warps ypass_warps xpass_warps\n");
        for (const auto& kv : g_tune)
            std::fprintf(f, "%d %d %d %d %d %d %d\n", kv.first[0], kv.first[1], kv.first[2], kv.first[3],
                         kv.second.rows2d_nw, kv.second.ypass_nw, kv.second.xpass_nw);
        std::fprintf(f, "# batch: b ndim log2-sides(3) rows2d_min_segment_log2 ypass_positions xpass_positions\n");
        for (const auto& kv : g_btune)
            std::fprintf(f, "b %d %d %d %d %d %d %d\n", kv.first[0], kv.first[1], kv.first[2], kv.first[3],
                         kv.second.rows2d_lgmin, kv.second.y_pos, kv.second.x_pos);
    }
    const bool ok = std::fclose(f) == 0;
    if (!ok) return fail(EDT_ERR_INVALID, "cannot write %s", path);
    clear_error();
    return EDT_OK;
}

extern "C" edt_status edt_tune_load(const char* path)
{
    if (!path) return fail(EDT_ERR_INVALID, "path is NULL");
    FILE* f = std::fopen(path, "r");
    if (!f) return fail(EDT_ERR_INVALID, "cannot read %s", path);
    std::map<Key, Tuning> loaded;
    std::map<Key, BatchTuning> bloaded;
    char line[256];
    edt_status st = EDT_OK;
    while (std::fgets(line, sizeof(line), f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        Key k;
        if (line[0] == 'b') {
            BatchTuning b;
            if (std::sscanf(line + 1, "%d %d %d %d %d %d %d", &k[0], &k[1], &k[2], &k[3], &b.rows2d_lgmin, &b.y_pos,
                            &b.x_pos) != 7 ||
                (k[0] != 2 && k[0] != 3)) {
                st = fail(EDT_ERR_INVALID, "malformed line in %s: %s", path, line);
                break;
            }
            auto ok_pos = [](int v) { return v == 0 || v == 32 || v == 64 || v == 128; };
            if (!(b.rows2d_lgmin == 0 || (b.rows2d_lgmin >= 6 && b.rows2d_lgmin <= 8)) || !ok_pos(b.y_pos) ||
                !ok_pos(b.x_pos)) {
                st = fail(EDT_ERR_INVALID, "batch geometry out of range in %s: %s", path, line);
                break;
            }
            bloaded[k] = b;
            continue;
        }
        Tuning t;
        if (std::sscanf(line, "%d %d %d %d %d %d %d", &k[0], &k[1], &k[2], &k[3], &t.rows2d_nw, &t.ypass_nw,
                        &t.xpass_nw) != 7 ||
            (k[0] != 2 && k[0] != 3)) {
            st = fail(EDT_ERR_INVALID, "malformed line in %s: %s", path, line);
            break;
        }
        auto ok_nw = [](int v, int hi) { return v == 0 || (v >= 1 && v <= hi && (v & (v - 1)) == 0); };
        if (!ok_nw(t.rows2d_nw, 16) || !ok_nw(t.ypass_nw, 32) || !ok_nw(t.xpass_nw, 32)) {
            st = fail(EDT_ERR_INVALID, "warp counts out of range in %s: %s", path, line);
            break;
        }
        loaded[k] = t;
    }
    std::fclose(f);
    if (st != EDT_OK) return st;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (const auto& kv : loaded) g_tune[kv.first] = kv.second;
        for (const auto& kv : bloaded) g_btune[kv.first] = kv.second;
    }
    clear_error();
    return EDT_OK;
}
