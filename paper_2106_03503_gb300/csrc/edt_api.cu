// C ABI of libedt: validation, scratch management and dispatch of the plain
// (one transform per call) entry points declared in include/edt.h.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "edt_internal.h"

namespace edt {

static thread_local std::string g_err;

edt_status fail(edt_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

edt_status cuda_fail(cudaError_t e, const char* what)
{
    return fail(e == cudaErrorMemoryAllocation ? EDT_ERR_NOMEM : EDT_ERR_CUDA,
                "%s: %s", what, cudaGetErrorString(e));
}

void clear_error() { g_err.clear(); }

// Per-device one-time setup: dynamic shared-memory opt-in of the kernels and
// the SM count used to size grids.
struct DeviceInfo {
    std::atomic<int> ready{0};
    int sm_count = 0;
};
static DeviceInfo g_dev[64];
static std::mutex g_dev_mu;

edt_status device_setup(int* sm_count)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(EDT_ERR_CUDA, "device index %d out of range", dev);
    DeviceInfo& d = g_dev[dev];
    if (!d.ready.load(std::memory_order_acquire)) {
        std::lock_guard<std::mutex> lk(g_dev_mu);
        if (!d.ready.load(std::memory_order_relaxed)) {
            int sms = 0;
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
            if ((e = set_2d_attributes()) != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
            if ((e = set_3d_attributes()) != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
            // keep freed scratch in this process's default pool instead of
            // returning it to the driver at every synchronisation
            cudaMemPool_t pool = nullptr;
            if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
                uint64_t keep = UINT64_MAX;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            }
            d.sm_count = sms;
            d.ready.store(1, std::memory_order_release);
        }
    }
    *sm_count = d.sm_count;
    return EDT_OK;
}

// Shape checks shared by every entry point (limits documented in edt.h).
edt_status check_shape(int ndim, const int* shape, int mode)
{
    if (!shape) return fail(EDT_ERR_INVALID, "shape is NULL");
    if (ndim != 2 && ndim != 3) return fail(EDT_ERR_INVALID, "ndim must be 2 or 3, got %d", ndim);
    if (mode != EDT_TO_OBJECT && mode != EDT_TO_BACKGROUND)
        return fail(EDT_ERR_INVALID, "mode must be EDT_TO_OBJECT or EDT_TO_BACKGROUND, got %d", mode);
    int64_t n = 1, maxsq = 0;
    for (int a = 0; a < ndim; ++a) {
        if (shape[a] <= 0) return fail(EDT_ERR_INVALID, "shape[%d] = %d must be positive", a, shape[a]);
        if (shape[a] > 32767) return fail(EDT_ERR_TOO_LARGE, "shape[%d] = %d exceeds 32767", a, shape[a]);
        n *= shape[a];
        maxsq += (int64_t)(shape[a] - 1) * (shape[a] - 1);
    }
    if (n >= ((int64_t)1 << 31)) return fail(EDT_ERR_TOO_LARGE, "%lld pixels exceed 2^31 - 1", (long long)n);
    if (maxsq >= INT32_MAX)
        return fail(EDT_ERR_TOO_LARGE, "largest squared distance %lld does not fit int32", (long long)maxsq);
    const int W = shape[ndim - 1];
    if (W > 16384) return fail(EDT_ERR_TOO_LARGE, "row width %d exceeds 16384", W);
    if (ndim == 3 && shape[1] > 2048) return fail(EDT_ERR_TOO_LARGE, "3-D height %d exceeds 2048", shape[1]);
    if (ndim == 3 && W > 1024) return fail(EDT_ERR_TOO_LARGE, "3-D row width %d exceeds 1024", W);
    return EDT_OK;
}

// Bytes of device scratch one transform needs.
size_t scratch_bytes(int ndim, const int* shape)
{
    const ColGeom g = (ndim == 2) ? col_geom(shape[0], shape[1])
                                  : col_geom(shape[0], (int64_t)shape[1] * shape[2]);
    return col_scratch_bytes(g);
}

// Enqueue one transform using `scratch` (scratch_bytes() bytes, device).
edt_status run_transform(const uint8_t* mask, int ndim, const int* shape, int mode,
                         int32_t* D, int32_t* F, float* dist, void* scratch,
                         int sm_count, cudaStream_t stream)
{
    cudaError_t e;
    if (ndim == 2) {
        const int H = shape[0], W = shape[1];
        const ColGeom g = col_geom(H, W);
        const ColScratch s = col_scratch_carve(scratch, g);
        if ((e = cudaMemsetAsync(s.cnt, 0, (size_t)g.ntiles * 4, stream)) != cudaSuccess)
            return cuda_fail(e, "cudaMemsetAsync");
        if ((e = traced("k_colbits", stream, [&] { return launch_colbits(mask, g, mode, s, stream); })) != cudaSuccess)
            return cuda_fail(e, "column pass launch");
        if ((e = traced("k_rows2d", stream,
                        [&] { return launch_rows2d(H, W, g, s, D, F, dist, sm_count, stream); })) != cudaSuccess)
            return cuda_fail(e, "row pass launch");
        return EDT_OK;
    }
    const int Dz = shape[0], H = shape[1], W = shape[2];
    const ColGeom g = col_geom(Dz, (int64_t)H * W);
    const ColScratch s = col_scratch_carve(scratch, g);
    uint32_t* P = reinterpret_cast<uint32_t*>(F ? F : D);
    if ((e = cudaMemsetAsync(s.cnt, 0, (size_t)g.ntiles * 4, stream)) != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync");
    if ((e = traced("k_colbits", stream, [&] { return launch_colbits(mask, g, mode, s, stream); })) != cudaSuccess)
        return cuda_fail(e, "z pass launch");
    if ((e = traced("k_ypass3d", stream, [&] { return launch_ypass3d(Dz, H, W, g, s, P, stream); })) != cudaSuccess)
        return cuda_fail(e, "y pass launch");
    if ((e = traced("k_xpass3d", stream,
                    [&] { return launch_xpass3d(Dz, H, W, P, D, F, dist, stream); })) != cudaSuccess)
        return cuda_fail(e, "x pass launch");
    return EDT_OK;
}

// --- kernel tracing ---------------------------------------------------------

struct TraceRec {
    const char* kernel;
    cudaEvent_t start, stop;
};
static std::mutex g_trace_mu;
static std::atomic<bool> g_trace_on{false};
static std::vector<TraceRec> g_trace;        // recorded launches
static std::vector<cudaEvent_t> g_event_pool;

static cudaEvent_t pooled_event()
{
    if (!g_event_pool.empty()) {
        cudaEvent_t ev = g_event_pool.back();
        g_event_pool.pop_back();
        return ev;
    }
    cudaEvent_t ev = nullptr;
    cudaEventCreate(&ev);
    return ev;
}

bool trace_on() { return g_trace_on.load(std::memory_order_relaxed); }

int trace_begin(const char* kernel, cudaStream_t stream)
{
    std::lock_guard<std::mutex> lk(g_trace_mu);
    TraceRec r{kernel, pooled_event(), pooled_event()};
    cudaEventRecord(r.start, stream);
    g_trace.push_back(r);
    return (int)g_trace.size() - 1;
}

void trace_end(int slot, cudaStream_t stream)
{
    std::lock_guard<std::mutex> lk(g_trace_mu);
    if (slot >= 0 && slot < (int)g_trace.size()) cudaEventRecord(g_trace[slot].stop, stream);
}

static void trace_reset_locked()
{
    for (auto& r : g_trace) {
        cudaEventSynchronize(r.stop);
        g_event_pool.push_back(r.start);
        g_event_pool.push_back(r.stop);
    }
    g_trace.clear();
}

// One transform with scratch from the stream-ordered pool.
edt_status plain_call(const uint8_t* mask, int ndim, const int* shape, int mode,
                      int32_t* D, int32_t* F, float* dist, cudaStream_t stream)
{
    edt_status st = check_shape(ndim, shape, mode);
    if (st != EDT_OK) return st;
    if (!mask) return fail(EDT_ERR_INVALID, "mask is NULL");
    if (!D && !F) return fail(EDT_ERR_INVALID, "D and F are both NULL");
    int sms = 0;
    if ((st = device_setup(&sms)) != EDT_OK) return st;
    const size_t bytes = scratch_bytes(ndim, shape);
    void* scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, bytes, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (scratch)");
    st = run_transform(mask, ndim, shape, mode, D, F, dist, scratch, sms, stream);
    e = cudaFreeAsync(scratch, stream);
    if (st == EDT_OK && e != cudaSuccess) return cuda_fail(e, "cudaFreeAsync");
    if (st == EDT_OK) clear_error();
    return st;
}

}  // namespace edt

using namespace edt;

extern "C" {

edt_status edt_sq2d(const uint8_t* mask, int H, int W, int mode, int32_t* D,
                    edt_stream_t stream)
{
    if (!D) return fail(EDT_ERR_INVALID, "D is NULL");
    const int shape[2] = {H, W};
    return plain_call(mask, 2, shape, mode, D, nullptr, nullptr, (cudaStream_t)stream);
}

edt_status edt_sq3d(const uint8_t* mask, int Dz, int H, int W, int mode,
                    int32_t* D, edt_stream_t stream)
{
    if (!D) return fail(EDT_ERR_INVALID, "D is NULL");
    const int shape[3] = {Dz, H, W};
    return plain_call(mask, 3, shape, mode, D, nullptr, nullptr, (cudaStream_t)stream);
}

edt_status edt_feature(const uint8_t* mask, int ndim, const int* shape, int mode,
                       int32_t* D, int32_t* F, float* dist, edt_stream_t stream)
{
    if (!F) return fail(EDT_ERR_INVALID, "F is NULL");
    return plain_call(mask, ndim, shape, mode, D, F, dist, (cudaStream_t)stream);
}

edt_status edt_feature_pair(const uint8_t* mask, int ndim, const int* shape, int32_t* D_obj,
                            int32_t* F_obj, int32_t* D_bg, int32_t* F_bg, edt_stream_t stream_)
{
    cudaStream_t stream = (cudaStream_t)stream_;
    edt_status st = check_shape(ndim, shape, EDT_TO_OBJECT);
    if (st != EDT_OK) return st;
    if (!mask || !F_obj || !F_bg) return fail(EDT_ERR_INVALID, "mask, F_obj and F_bg must not be NULL");
    if (ndim == 3) {
        st = plain_call(mask, 3, shape, EDT_TO_OBJECT, D_obj, F_obj, nullptr, stream);
        if (st != EDT_OK) return st;
        return plain_call(mask, 3, shape, EDT_TO_BACKGROUND, D_bg, F_bg, nullptr, stream);
    }
    int sms = 0;
    if ((st = device_setup(&sms)) != EDT_OK) return st;
    const int H = shape[0], W = shape[1];
    const ColGeom g = col_geom(H, W);
    const size_t one = col_scratch_bytes(g);
    char* scratch = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&scratch, 2 * one, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (scratch)");
    const ColScratch s0 = col_scratch_carve(scratch, g);
    const ColScratch s1 = col_scratch_carve(scratch + one, g);
    st = EDT_OK;
    if ((e = cudaMemsetAsync(s0.cnt, 0, (size_t)g.ntiles * 4, stream)) != cudaSuccess)
        st = cuda_fail(e, "cudaMemsetAsync");
    if (st == EDT_OK &&
        (e = traced("k_colbits", stream, [&] { return launch_colbits_pair(mask, g, s0, s1, stream); })) !=
            cudaSuccess)
        st = cuda_fail(e, "column pass launch");
    if (st == EDT_OK &&
        (e = traced("k_rows2d", stream, [&] {
             return launch_rows2d_pair(H, W, g, s0, s1, D_obj, F_obj, D_bg, F_bg, stream);
         })) != cudaSuccess)
        st = cuda_fail(e, "row pass launch");
    e = cudaFreeAsync(scratch, stream);
    if (st == EDT_OK && e != cudaSuccess) st = cuda_fail(e, "cudaFreeAsync");
    if (st == EDT_OK) clear_error();
    return st;
}

edt_status edt_feature_host(const uint8_t* mask, int ndim, const int* shape,
                            int mode, int32_t* D, int32_t* F, float* dist,
                            edt_stream_t stream_)
{
    cudaStream_t stream = (cudaStream_t)stream_;
    edt_status st = check_shape(ndim, shape, mode);
    if (st != EDT_OK) return st;
    if (!mask || !F) return fail(EDT_ERR_INVALID, "mask and F must not be NULL");
    int64_t n = 1;
    for (int a = 0; a < ndim; ++a) n *= shape[a];
    int sms = 0;
    if ((st = device_setup(&sms)) != EDT_OK) return st;
    // one device block: mask | D | F | dist | scratch, 256-byte aligned parts
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t bm = al((size_t)n), bd = D ? al((size_t)n * 4) : 0, bf = al((size_t)n * 4),
                 bs = dist ? al((size_t)n * 4) : 0, bx = scratch_bytes(ndim, shape);
    char* dev = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&dev, bm + bd + bf + bs + bx, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    uint8_t* dmask = reinterpret_cast<uint8_t*>(dev);
    int32_t* dD = D ? reinterpret_cast<int32_t*>(dev + bm) : nullptr;
    int32_t* dF = reinterpret_cast<int32_t*>(dev + bm + bd);
    float* dS = dist ? reinterpret_cast<float*>(dev + bm + bd + bf) : nullptr;
    void* scratch = dev + bm + bd + bf + bs;
    st = EDT_OK;
    if ((e = cudaMemcpyAsync(dmask, mask, (size_t)n, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
        st = cuda_fail(e, "cudaMemcpyAsync H2D");
    if (st == EDT_OK)
        st = run_transform(dmask, ndim, shape, mode, dD, dF, dS, scratch, sms, stream);
    if (st == EDT_OK && D &&
        (e = cudaMemcpyAsync(D, dD, (size_t)n * 4, cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
        st = cuda_fail(e, "cudaMemcpyAsync D2H");
    if (st == EDT_OK &&
        (e = cudaMemcpyAsync(F, dF, (size_t)n * 4, cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
        st = cuda_fail(e, "cudaMemcpyAsync D2H");
    if (st == EDT_OK && dist &&
        (e = cudaMemcpyAsync(dist, dS, (size_t)n * 4, cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
        st = cuda_fail(e, "cudaMemcpyAsync D2H");
    cudaFreeAsync(dev, stream);
    e = cudaStreamSynchronize(stream);
    if (st == EDT_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize");
    if (st == EDT_OK) clear_error();
    return st;
}

edt_status edt_trace_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_trace_mu);
    trace_reset_locked();
    g_trace_on.store(on != 0);
    return EDT_OK;
}

edt_status edt_trace_read(const char* kernel, double* total_ms, int64_t* launches)
{
    if (!kernel || !total_ms || !launches) return fail(EDT_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(g_trace_mu);
    double ms = 0.0;
    int64_t n = 0;
    for (auto& r : g_trace) {
        if (strcmp(r.kernel, kernel) != 0) continue;
        cudaError_t e = cudaEventSynchronize(r.stop);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
        float t = 0.f;
        e = cudaEventElapsedTime(&t, r.start, r.stop);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
        ms += t;
        ++n;
    }
    *total_ms = ms;
    *launches = n;
    return EDT_OK;
}

const char* edt_last_error(void) { return g_err.c_str(); }

const char* edt_version(void) { return "libedt 0.1 (sm_103a)"; }

}  // extern "C"
