// Allocation-free 2-D entry point: the column pass scratch lives in a fixed,
// file-scope device array instead of the stream-ordered pool.
//
// Who needs it: callers that are not allowed to allocate device memory on the
// call path -- a plugin inside a host framework that owns every device
// allocation (inference servers, game engines, medical-imaging pipelines with
// a fixed memory plan), or latency-critical code that cannot risk the
// implicit device synchronisation and global locking that cudaMalloc and
// cudaFree may take.  This entry point calls no cudaMalloc, cudaFree or
// allocating library routine; the caller passes the mask and the outputs.
//
// The price: the scratch array (EDT_NOALLOC_SCRATCH_BYTES) is reserved on every
// GPU that loads the library, until the process exits, and it is shared by all
// calls: calls that overlap on the GPU (different streams, or different host
// threads without ordering) race on it and must be serialised by the caller.
#include <atomic>
#include <mutex>

#include "edt_internal.h"

namespace edt {

// 32 MiB: enough for 2-D images up to 8192 x 8192 (about 16.5 MiB of column
// words and band summaries) and any image whose scratch fits.
constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)32 << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

edt_status fail(edt_status st, const char* fmt, ...);
edt_status cuda_fail(cudaError_t e, const char* what);
void clear_error();
edt_status device_setup(int* sm_count);
edt_status check_shape(int ndim, const int* shape, int mode);
size_t scratch_bytes(int ndim, const int* shape);
edt_status run_transform(const uint8_t* mask, int ndim, const int* shape, int mode,
                         int32_t* D, int32_t* F, float* dist, void* scratch,
                         int sm_count, cudaStream_t stream);

// Device address of the scratch array, resolved once per device with that
// device current (the host-side symbol is only a stand-in, not an address).
// After the first call on a device the address is read without the lock.
static std::atomic<void*> g_noalloc_ptr[64];
static std::mutex g_noalloc_mu;

static edt_status noalloc_scratch(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(EDT_ERR_CUDA, "device index %d out of range", dev);
    void* p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        p = g_noalloc_ptr[dev].load(std::memory_order_relaxed);
        if (!p) {
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress (static scratch)");
            g_noalloc_ptr[dev].store(p, std::memory_order_release);
        }
    }
    *out = p;
    return EDT_OK;
}

}  // namespace edt

using namespace edt;

extern "C" edt_status edt_feature2d_noalloc(const uint8_t* mask, int H, int W, int mode,
                                            int32_t* D, int32_t* F, float* dist,
                                            edt_stream_t stream)
{
    const int shape[2] = {H, W};
    edt_status st = check_shape(2, shape, mode);
    if (st != EDT_OK) return st;
    if (!mask || !F) return fail(EDT_ERR_INVALID, "mask and F must not be NULL");
    const size_t need = scratch_bytes(2, shape);
    if (need > NOALLOC_SCRATCH_BYTES)
        return fail(EDT_ERR_TOO_LARGE,
                    "a %d x %d image needs %zu bytes of scratch; the static scratch of "
                    "edt_feature2d_noalloc holds %zu bytes",
                    H, W, need, NOALLOC_SCRATCH_BYTES);
    int sms = 0;
    if ((st = device_setup(&sms)) != EDT_OK) return st;
    void* scratch = nullptr;
    if ((st = noalloc_scratch(&scratch)) != EDT_OK) return st;
    // run_transform clears the arrival counters before the column pass; every
    // other scratch word is written before it is read.
    st = run_transform(mask, 2, shape, mode, D, F, dist, scratch, sms, (cudaStream_t)stream);
    if (st == EDT_OK) clear_error();
    return st;
}
