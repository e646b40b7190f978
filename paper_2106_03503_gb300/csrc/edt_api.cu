// C ABI of libedt: validation, scratch management and dispatch of the plain
// (one transform per call) entry points declared in include/edt.h.
#include <algorithm>
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
    cudaStream_t copy = nullptr;   // device-to-host copies of the host-buffer calls
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
            if ((e = set_chamfer_attributes()) != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
            // keep freed scratch in this process's default pool instead of
            // returning it to the driver at every synchronisation
            cudaMemPool_t pool = nullptr;
            if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
                uint64_t keep = UINT64_MAX;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            }
            if ((e = cudaStreamCreateWithFlags(&d.copy, cudaStreamNonBlocking)) != cudaSuccess)
                return cuda_fail(e, "cudaStreamCreate");
            d.sm_count = sms;
            d.ready.store(1, std::memory_order_release);
        }
    }
    *sm_count = d.sm_count;
    return EDT_OK;
}

int device_sm_count()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    return g_dev[dev].ready.load(std::memory_order_acquire) ? g_dev[dev].sm_count : 0;
}

// Shape checks shared by every entry point (limits documented in edt.h).
// Copy stream of the current device (device_setup must have run).
static cudaStream_t copy_stream()
{
    int dev = 0;
    cudaGetDevice(&dev);
    return g_dev[dev].copy;
}

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
    if (ndim == 2) return col_scratch_bytes(col_geom(shape[0], shape[1]));
    // 3-D: the z pass's scratch, then the int16 z offsets of every voxel
    const ColGeom g = col_geom(shape[0], (int64_t)shape[1] * shape[2]);
    return ((col_scratch_bytes(g) + 255) & ~size_t(255)) + (size_t)shape[0] * shape[1] * shape[2] * 2;
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
    short* d16 = reinterpret_cast<short*>(static_cast<char*>(scratch) + ((col_scratch_bytes(g) + 255) & ~size_t(255)));
    uint32_t* P = reinterpret_cast<uint32_t*>(F ? F : D);
    if ((e = cudaMemsetAsync(s.cnt, 0, (size_t)g.ntiles * 4, stream)) != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync");
    if ((e = traced("k_colbits", stream, [&] { return launch_colbits(mask, g, mode, s, stream); })) != cudaSuccess)
        return cuda_fail(e, "z pass launch");
    if ((e = traced("k_zoffsets", stream, [&] { return launch_zoffsets(Dz, H, W, g, s, d16, stream); })) !=
        cudaSuccess)
        return cuda_fail(e, "z offsets launch");
    if ((e = traced("k_ypass3d", stream, [&] { return launch_ypass3d(Dz, H, W, g, s, d16, P, stream); })) !=
        cudaSuccess)
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

// --- host-buffer calls --------------------------------------------------------

// One transform's host result buffers (D and dist may be NULL).
struct HostOut {
    int mode;
    int32_t* D;
    int32_t* F;
    float* dist;
};

// Copy the mask to the device, run one transform (nout = 1) or both
// transforms of the mask (nout = 2, modes 0 and 1), copy the results back
// and wait for them.  For 2-D images the row pass runs in up to four launches
// over consecutive band ranges, and the rows of each range go back to the
// host on the device's copy stream as soon as its launch has finished, so
// that the device-to-host copy -- the bottleneck: 4 to 12 bytes per pixel and
// transform over the host link -- overlaps the rest of the row pass.
edt_status host_call(const uint8_t* mask, int ndim, const int* shape, const HostOut* outs, int nout,
                     cudaStream_t stream)
{
    int64_t n = 1;
    for (int a = 0; a < ndim; ++a) n *= shape[a];
    int sms = 0;
    edt_status st = device_setup(&sms);
    if (st != EDT_OK) return st;
    // one device block: mask | per transform D, F, dist | scratch per transform
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t bx = al(scratch_bytes(ndim, shape));
    size_t total = al((size_t)n) + nout * bx;
    for (int k = 0; k < nout; ++k)
        total += (outs[k].D ? al((size_t)n * 4) : 0) + al((size_t)n * 4) + (outs[k].dist ? al((size_t)n * 4) : 0);
    char* dev = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&dev, total, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    char* p = dev;
    uint8_t* dmask = reinterpret_cast<uint8_t*>(p);
    p += al((size_t)n);
    int32_t* dD[2] = {nullptr, nullptr};
    int32_t* dF[2] = {nullptr, nullptr};
    float* dS[2] = {nullptr, nullptr};
    void* scr[2] = {nullptr, nullptr};
    for (int k = 0; k < nout; ++k) {
        if (outs[k].D) { dD[k] = reinterpret_cast<int32_t*>(p); p += al((size_t)n * 4); }
        dF[k] = reinterpret_cast<int32_t*>(p);
        p += al((size_t)n * 4);
        if (outs[k].dist) { dS[k] = reinterpret_cast<float*>(p); p += al((size_t)n * 4); }
        scr[k] = p;
        p += bx;
    }
    cudaStream_t cs = copy_stream();
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    for (auto& x : ev)
        if (st == EDT_OK && (e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming)) != cudaSuccess)
            st = cuda_fail(e, "cudaEventCreate");
    if (st == EDT_OK && (e = cudaMemcpyAsync(dmask, mask, (size_t)n, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
        st = cuda_fail(e, "cudaMemcpyAsync H2D");
    // rows [r0, r1) of every result, device to host, on `on`
    auto copy_rows = [&](int64_t r0, int64_t r1, int64_t row, cudaStream_t on) {
        const size_t off = (size_t)(r0 * row), cnt = (size_t)((r1 - r0) * row) * 4;
        for (int k = 0; k < nout && st == EDT_OK; ++k) {
            if (outs[k].D && (e = cudaMemcpyAsync(outs[k].D + off, dD[k] + off, cnt, cudaMemcpyDeviceToHost, on)) != cudaSuccess)
                st = cuda_fail(e, "cudaMemcpyAsync D2H");
            if (st == EDT_OK &&
                (e = cudaMemcpyAsync(outs[k].F + off, dF[k] + off, cnt, cudaMemcpyDeviceToHost, on)) != cudaSuccess)
                st = cuda_fail(e, "cudaMemcpyAsync D2H");
            if (st == EDT_OK && outs[k].dist &&
                (e = cudaMemcpyAsync(outs[k].dist + off, dS[k] + off, cnt, cudaMemcpyDeviceToHost, on)) != cudaSuccess)
                st = cuda_fail(e, "cudaMemcpyAsync D2H");
        }
    };
    bool used_cs = false, joined = false;
    if (st == EDT_OK && ndim == 2) {
        const int H = shape[0], W = shape[1];
        const ColGeom g = col_geom(H, W);
        const ColScratch s0 = col_scratch_carve(scr[0], g);
        const ColScratch s1 = nout == 2 ? col_scratch_carve(scr[1], g) : s0;
        if ((e = cudaMemsetAsync(s0.cnt, 0, (size_t)g.ntiles * 4, stream)) != cudaSuccess)
            st = cuda_fail(e, "cudaMemsetAsync");
        if (st == EDT_OK &&
            (e = traced("k_colbits", stream, [&] {
                 return nout == 2 ? launch_colbits_pair(dmask, g, s0, s1, stream)
                                  : launch_colbits(dmask, g, outs[0].mode, s0, stream);
             })) != cudaSuccess)
            st = cuda_fail(e, "column pass launch");
        const int nchunk = g.nb >= 16 ? 4 : 1;
        for (int c = 0; c < nchunk && st == EDT_OK; ++c) {
            const int b0 = (int)((int64_t)g.nb * c / nchunk), b1 = (int)((int64_t)g.nb * (c + 1) / nchunk);
            e = traced("k_rows2d", stream, [&] {
                return nout == 2 ? launch_rows2d_pair(H, W, g, s0, s1, dD[0], dF[0], dD[1], dF[1], stream, b0, b1 - b0)
                                 : launch_rows2d(H, W, g, s0, dD[0], dF[0], dS[0], sms, stream, b0, b1 - b0);
            });
            if (e != cudaSuccess) { st = cuda_fail(e, "row pass launch"); break; }
            if ((e = cudaEventRecord(ev[c], stream)) != cudaSuccess || (e = cudaStreamWaitEvent(cs, ev[c], 0)) != cudaSuccess) {
                st = cuda_fail(e, "event");
                break;
            }
            used_cs = true;
            copy_rows((int64_t)b0 * 32, std::min<int64_t>((int64_t)b1 * 32, H), W, cs);
        }
        // order the free below after the copies
        if (st == EDT_OK) {
            if ((e = cudaEventRecord(ev[4], cs)) != cudaSuccess || (e = cudaStreamWaitEvent(stream, ev[4], 0)) != cudaSuccess)
                st = cuda_fail(e, "event");
            else
                joined = true;
        }
    } else if (st == EDT_OK) {
        for (int k = 0; k < nout && st == EDT_OK; ++k)
            st = run_transform(dmask, ndim, shape, outs[k].mode, dD[k], dF[k], dS[k], scr[k], sms, stream);
        if (st == EDT_OK) copy_rows(0, n / shape[ndim - 1], shape[ndim - 1], stream);
    }
    if (used_cs && !joined) cudaStreamSynchronize(cs);   // after an error: no copy may outlive the block
    cudaFreeAsync(dev, stream);
    e = cudaStreamSynchronize(stream);
    if (st == EDT_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize");
    for (auto& x : ev)
        if (x) cudaEventDestroy(x);
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

edt_status edt_cityblock2d(const uint8_t* mask, int H, int W, int mode, int32_t* D, edt_stream_t stream_)
{
    cudaStream_t stream = (cudaStream_t)stream_;
    const int shape[2] = {H, W};
    edt_status st = check_shape(2, shape, mode);
    if (st != EDT_OK) return st;
    if (!mask || !D) return fail(EDT_ERR_INVALID, "mask and D must not be NULL");
    int sms = 0;
    if ((st = device_setup(&sms)) != EDT_OK) return st;
    const ColGeom g = col_geom(H, W);
    void* scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, col_scratch_bytes(g), stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (scratch)");
    const ColScratch s = col_scratch_carve(scratch, g);
    if ((e = cudaMemsetAsync(s.cnt, 0, (size_t)g.ntiles * 4, stream)) != cudaSuccess)
        st = cuda_fail(e, "cudaMemsetAsync");
    if (st == EDT_OK &&
        (e = traced("k_colbits", stream, [&] { return launch_colbits(mask, g, mode, s, stream); })) != cudaSuccess)
        st = cuda_fail(e, "column pass launch");
    if (st == EDT_OK &&
        (e = traced("k_cityblock_rows", stream, [&] { return launch_cityblock_rows(H, W, g, s, D, stream); })) !=
            cudaSuccess)
        st = cuda_fail(e, "row pass launch");
    e = cudaFreeAsync(scratch, stream);
    if (st == EDT_OK && e != cudaSuccess) st = cuda_fail(e, "cudaFreeAsync");
    if (st == EDT_OK) clear_error();
    return st;
}

edt_status edt_chamfer43_2d(const uint8_t* mask, int H, int W, int mode, int32_t* D, edt_stream_t stream_)
{
    cudaStream_t stream = (cudaStream_t)stream_;
    const int shape[2] = {H, W};
    edt_status st = check_shape(2, shape, mode);
    if (st != EDT_OK) return st;
    if (!mask || !D) return fail(EDT_ERR_INVALID, "mask and D must not be NULL");
    if (W > 14336) return fail(EDT_ERR_TOO_LARGE, "chamfer rows are limited to 14336 columns (got %d)", W);
    int sms = 0;
    if ((st = device_setup(&sms)) != EDT_OK) return st;
    void* scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, chamfer_scratch_bytes(H, W), stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (scratch)");
    if ((e = launch_chamfer(mask, H, W, mode, D, scratch, sms, stream)) != cudaSuccess)
        st = cuda_fail(e, "chamfer launches");
    e = cudaFreeAsync(scratch, stream);
    if (st == EDT_OK && e != cudaSuccess) st = cuda_fail(e, "cudaFreeAsync");
    if (st == EDT_OK) clear_error();
    return st;
}

edt_status edt_feature_host(const uint8_t* mask, int ndim, const int* shape,
                            int mode, int32_t* D, int32_t* F, float* dist,
                            edt_stream_t stream)
{
    edt_status st = check_shape(ndim, shape, mode);
    if (st != EDT_OK) return st;
    if (!mask || !F) return fail(EDT_ERR_INVALID, "mask and F must not be NULL");
    const HostOut out{mode, D, F, dist};
    return host_call(mask, ndim, shape, &out, 1, (cudaStream_t)stream);
}

edt_status edt_feature_pair_host(const uint8_t* mask, int ndim, const int* shape, int32_t* D_obj,
                                 int32_t* F_obj, int32_t* D_bg, int32_t* F_bg, edt_stream_t stream)
{
    edt_status st = check_shape(ndim, shape, EDT_TO_OBJECT);
    if (st != EDT_OK) return st;
    if (!mask || !F_obj || !F_bg) return fail(EDT_ERR_INVALID, "mask, F_obj and F_bg must not be NULL");
    const HostOut outs[2] = {{EDT_TO_OBJECT, D_obj, F_obj, nullptr}, {EDT_TO_BACKGROUND, D_bg, F_bg, nullptr}};
    return host_call(mask, ndim, shape, outs, 2, (cudaStream_t)stream);
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
