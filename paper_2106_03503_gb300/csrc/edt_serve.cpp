// Continuous-batching server (edt_serve_create / _submit / _poll / _destroy).
//
// Jobs arrive with HOST buffers.  A scheduler thread keeps a FIFO of submitted
// jobs and a set of CUDA streams, each owning a batch plan.  Whenever a stream
// is idle and the head of the FIFO fits the device-memory budget, it admits
// jobs in arrival order while they fit, allocates their device buffers from
// the server's memory pool, and enqueues on that stream: the mask copies in,
// one batched launch for the 2-D jobs a plan accepts (width <= 2048) and plain
// transforms for the others (wider 2-D images, 3-D volumes), the result copies
// out, the buffer frees, and a host callback that completes the tickets and
// returns their bytes to the budget.  Batches on different streams overlap on
// the device; requests that arrive while batches run are admitted as soon as
// a stream and enough budget are free.  Every result is the same as a plain
// edt_feature call on the same mask (the kernels do not depend on batch
// membership), which the tests check alone and in the mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
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
}  // namespace edt

using namespace edt;

namespace {

using Clock = std::chrono::steady_clock;

constexpr int SERVE_PLAN_JOBS = 512;          // jobs per batched launch
// pixels admitted to one stream at a time (beyond the first job): a batch's
// tickets complete together, so a long backlog is split over the streams in
// batches of a few milliseconds of work instead of going to one stream whole
constexpr int64_t SERVE_BATCH_PIXELS = (int64_t)1 << 25;

struct Pending {
    uint64_t ticket;
    edt_job job;             // host pointers
    int64_t n;               // pixels
    size_t bytes;            // device footprint
    Clock::time_point t_submit;
};

struct Ticket {
    int state = 0;           // 0 queued, 1 running, 2 done
    edt_status status = EDT_OK;
    double latency = 0.0;
    Clock::time_point t_submit;
};

struct StreamSlot {
    cudaStream_t stream = nullptr;
    edt_plan* plan = nullptr;
    bool busy = false;
};

struct Completion;

}  // namespace

struct edt_server {
    int device = 0;
    int sm_count = 0;
    cudaMemPool_t pool = nullptr;   // job buffers: the server's own pool, grown to the budget at creation
    size_t budget = 0;       // bytes available to job buffers
    size_t in_use = 0;
    int64_t plan_pixels = 0;
    std::vector<StreamSlot> slots;
    std::deque<Pending> queue;
    std::unordered_map<uint64_t, Ticket> tickets;
    uint64_t next_ticket = 1;
    int outstanding = 0;     // submitted, not yet completed
    bool stopping = false;
    std::mutex mu;
    std::condition_variable cv;
    std::thread sched;
};

namespace {

struct Completion {
    edt_server* srv;
    int slot;
    size_t bytes;
    std::vector<uint64_t> tickets;
    edt_status status;
};

// Runs on a CUDA callback thread once the stream reached the end of a batch;
// must not call CUDA.
void CUDART_CB on_batch_done(void* arg)
{
    Completion* c = static_cast<Completion*>(arg);
    edt_server* s = c->srv;
    const auto now = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (uint64_t t : c->tickets) {
            auto it = s->tickets.find(t);
            if (it == s->tickets.end()) continue;
            it->second.state = 2;
            it->second.status = c->status;
            it->second.latency = std::chrono::duration<double>(now - it->second.t_submit).count();
        }
        s->in_use -= c->bytes;
        s->outstanding -= (int)c->tickets.size();
        s->slots[c->slot].busy = false;
    }
    s->cv.notify_all();
    delete c;
}

size_t job_bytes(const edt_job& j, int64_t n)
{
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t b = al((size_t)n) + al((size_t)n * 4);           // mask, F
    if (j.D) b += al((size_t)n * 4);
    if (j.dist) b += al((size_t)n * 4);
    b += scratch_bytes(j.ndim, j.shape);                     // column-pass scratch
    return b;
}

// Enqueue one admitted batch on slot `si` (called by the scheduler thread
// without the lock held).
void launch_batch(edt_server* s, int si, std::vector<Pending>& batch, size_t bytes)
{
    StreamSlot& slot = s->slots[si];
    cudaStream_t st = slot.stream;
    edt_status status = EDT_OK;
    struct Dev {
        uint8_t* mask;
        int32_t* D;
        int32_t* F;
        float* dist;
        void* scratch;
    };
    std::vector<Dev> dev(batch.size());
    std::vector<edt_job> bj;
    bj.reserve(batch.size());
    for (size_t k = 0; k < batch.size() && status == EDT_OK; ++k) {
        const Pending& p = batch[k];
        Dev d{};
        cudaError_t e = cudaSuccess;
        const size_t n = (size_t)p.n;
        const bool batched = p.job.ndim == 2 && p.job.shape[1] <= BATCH_MAX_W &&
                             (int64_t)n <= s->plan_pixels;
        if ((e = cudaMallocFromPoolAsync((void**)&d.mask, n, s->pool, st)) != cudaSuccess ||
            (e = cudaMallocFromPoolAsync((void**)&d.F, n * 4, s->pool, st)) != cudaSuccess ||
            (p.job.D && (e = cudaMallocFromPoolAsync((void**)&d.D, n * 4, s->pool, st)) != cudaSuccess) ||
            (p.job.dist && (e = cudaMallocFromPoolAsync((void**)&d.dist, n * 4, s->pool, st)) != cudaSuccess) ||
            (!batched &&
             (e = cudaMallocFromPoolAsync(&d.scratch, scratch_bytes(p.job.ndim, p.job.shape), s->pool, st)) != cudaSuccess)) {
            status = cuda_fail(e, "serve: device buffers");
            dev[k] = d;
            break;
        }
        dev[k] = d;
        if ((e = cudaMemcpyAsync(d.mask, p.job.mask, n, cudaMemcpyHostToDevice, st)) != cudaSuccess) {
            status = cuda_fail(e, "serve: mask copy");
            break;
        }
        if (batched) {
            edt_job j = p.job;
            j.mask = d.mask;
            j.D = d.D;
            j.F = d.F;
            j.dist = d.dist;
            bj.push_back(j);
        } else {
            status = run_transform(d.mask, p.job.ndim, p.job.shape, p.job.mode, d.D, d.F,
                                   d.dist, d.scratch, s->sm_count, st);
        }
    }
    // batched 2-D jobs: one or more plan replays
    for (size_t off = 0; off < bj.size() && status == EDT_OK;) {
        size_t cnt = 0;
        int64_t px = 0;
        while (off + cnt < bj.size() && cnt < (size_t)SERVE_PLAN_JOBS) {
            const int64_t q = (int64_t)bj[off + cnt].shape[0] * bj[off + cnt].shape[1];
            if (cnt > 0 && px + q > s->plan_pixels) break;
            px += q;
            ++cnt;
        }
        status = edt_batch(slot.plan, bj.data() + off, (int)cnt, (edt_stream_t)st);
        off += cnt;
    }
    for (size_t k = 0; k < batch.size(); ++k) {
        const Pending& p = batch[k];
        const Dev& d = dev[k];
        const size_t n = (size_t)p.n;
        if (status == EDT_OK) {
            cudaError_t e = cudaSuccess;
            if (p.job.D) e = cudaMemcpyAsync(p.job.D, d.D, n * 4, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(p.job.F, d.F, n * 4, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess && p.job.dist)
                e = cudaMemcpyAsync(p.job.dist, d.dist, n * 4, cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) status = cuda_fail(e, "serve: result copy");
        }
        if (d.mask) cudaFreeAsync(d.mask, st);
        if (d.D) cudaFreeAsync(d.D, st);
        if (d.F) cudaFreeAsync(d.F, st);
        if (d.dist) cudaFreeAsync(d.dist, st);
        if (d.scratch) cudaFreeAsync(d.scratch, st);
    }
    Completion* c = new Completion{s, si, bytes, {}, status};
    for (const Pending& p : batch) c->tickets.push_back(p.ticket);
    if (cudaLaunchHostFunc(st, on_batch_done, c) != cudaSuccess) {
        // the stream is broken: complete the tickets from here
        cudaStreamSynchronize(st);
        c->status = EDT_ERR_CUDA;
        on_batch_done(c);
    }
}

void scheduler(edt_server* s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        int si = -1;
        s->cv.wait(lk, [&] {
            if (s->stopping && s->queue.empty()) return true;
            if (s->queue.empty()) return false;
            si = -1;
            for (int k = 0; k < (int)s->slots.size(); ++k)
                if (!s->slots[k].busy) { si = k; break; }
            return si >= 0 && s->in_use + s->queue.front().bytes <= s->budget;
        });
        if (s->queue.empty()) {
            if (s->stopping) break;
            continue;
        }
        // admit in arrival order while the budget allows
        std::vector<Pending> batch;
        size_t bytes = 0;
        int64_t px = 0;
        while (!s->queue.empty() && s->in_use + bytes + s->queue.front().bytes <= s->budget &&
               batch.size() < (size_t)4 * SERVE_PLAN_JOBS &&
               (batch.empty() || px + s->queue.front().n <= SERVE_BATCH_PIXELS)) {
            bytes += s->queue.front().bytes;
            px += s->queue.front().n;
            batch.push_back(s->queue.front());
            s->queue.pop_front();
        }
        s->in_use += bytes;
        s->slots[si].busy = true;
        for (const Pending& p : batch) s->tickets[p.ticket].state = 1;
        lk.unlock();
        launch_batch(s, si, batch, bytes);
        lk.lock();
    }
}

}  // namespace

extern "C" edt_status edt_serve_create(edt_server** out, size_t mem_budget_bytes, int n_streams)
{
    if (!out) return fail(EDT_ERR_INVALID, "server pointer is NULL");
    *out = nullptr;
    if (n_streams <= 0 || n_streams > 16) return fail(EDT_ERR_INVALID, "n_streams must be in 1..16");
    int sms = 0;
    edt_status st = device_setup(&sms);
    if (st != EDT_OK) return st;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return fail(EDT_ERR_CUDA, "cudaMemGetInfo failed");
    if (mem_budget_bytes > free_b)
        return fail(EDT_ERR_BUDGET, "budget of %zu bytes exceeds the %zu bytes free on the device", mem_budget_bytes,
                    free_b);
    edt_server* s = new edt_server();
    cudaGetDevice(&s->device);
    s->sm_count = sms;
    // each stream's plan takes about 0.26 B/pixel of scratch for plan_pixels
    s->plan_pixels = (int64_t)std::min<double>((double)mem_budget_bytes / 9.5 / n_streams, 1.5e9);
    if (s->plan_pixels < 4096) s->plan_pixels = 4096;
    size_t reserved = 0;
    for (int k = 0; k < n_streams; ++k) {
        StreamSlot slot;
        cudaError_t e = cudaStreamCreateWithFlags(&slot.stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { st = cuda_fail(e, "cudaStreamCreate"); break; }
        st = edt_plan_create(&slot.plan, SERVE_PLAN_JOBS, s->plan_pixels);
        if (st != EDT_OK) { cudaStreamDestroy(slot.stream); break; }
        reserved += (size_t)(0.26 * (double)s->plan_pixels) + (size_t)SERVE_PLAN_JOBS * (16 * BATCH_MAX_W + 1024);
        s->slots.push_back(slot);
    }
    if (st != EDT_OK || reserved >= mem_budget_bytes) {
        for (auto& slot : s->slots) {
            edt_plan_destroy(slot.plan);
            cudaStreamDestroy(slot.stream);
        }
        delete s;
        if (st == EDT_OK) return fail(EDT_ERR_BUDGET, "budget of %zu bytes is below the plans' %zu", mem_budget_bytes, reserved);
        return st;
    }
    s->budget = mem_budget_bytes - reserved;
    // job buffers come from a pool of the server's own that keeps what is
    // freed, takes no cross-stream dependencies to reuse it, and is grown to
    // the budget here, so that no admitted job waits for the pool to map new
    // memory
    {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = s->device;
        cudaError_t e = cudaMemPoolCreate(&s->pool, &props);
        uint64_t keep = UINT64_MAX;
        int no = 0;
        if (e == cudaSuccess) e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e == cudaSuccess) e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolReuseAllowInternalDependencies, &no);
        void* warm = nullptr;
        cudaStream_t st0 = s->slots[0].stream;
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&warm, s->budget, s->pool, st0);
        if (e == cudaSuccess) e = cudaFreeAsync(warm, st0);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st0);
        if (e != cudaSuccess) {
            const edt_status err = cuda_fail(e, "serve: memory pool");
            if (s->pool) cudaMemPoolDestroy(s->pool);
            for (auto& slot : s->slots) {
                edt_plan_destroy(slot.plan);
                cudaStreamDestroy(slot.stream);
            }
            delete s;
            return err;
        }
    }
    s->sched = std::thread(scheduler, s);
    *out = s;
    clear_error();
    return EDT_OK;
}

extern "C" edt_status edt_serve_submit(edt_server* s, const edt_job* job, uint64_t* ticket)
{
    if (!s || !job || !ticket) return fail(EDT_ERR_INVALID, "NULL argument");
    edt_status st = check_shape(job->ndim, job->shape, job->mode);
    if (st != EDT_OK) return st;
    if (!job->mask || !job->F) return fail(EDT_ERR_INVALID, "mask and F must not be NULL");
    int64_t n = 1;
    for (int a = 0; a < job->ndim; ++a) n *= job->shape[a];
    Pending p;
    p.job = *job;
    p.n = n;
    p.bytes = job_bytes(*job, n);
    p.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) return fail(EDT_ERR_INVALID, "server is shutting down");
        if (p.bytes > s->budget)
            return fail(EDT_ERR_BUDGET, "job needs %zu device bytes; the budget is %zu", p.bytes, s->budget);
        p.ticket = s->next_ticket++;
        Ticket t;
        t.t_submit = p.t_submit;
        s->tickets[p.ticket] = t;
        s->queue.push_back(p);
        ++s->outstanding;
        *ticket = p.ticket;
    }
    s->cv.notify_all();
    clear_error();
    return EDT_OK;
}

extern "C" edt_status edt_serve_poll(edt_server* s, uint64_t ticket, double* latency_s)
{
    if (!s) return fail(EDT_ERR_INVALID, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(EDT_ERR_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
    if (it->second.state != 2) return EDT_ERR_NOT_READY;
    const edt_status st = it->second.status;
    if (latency_s) *latency_s = it->second.latency;
    s->tickets.erase(it);
    if (st != EDT_OK) return fail(st, "served job failed");
    return EDT_OK;
}

extern "C" edt_status edt_serve_destroy(edt_server* s)
{
    if (!s) return EDT_OK;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->stopping = true;
        s->cv.notify_all();
        s->cv.wait(lk, [&] { return s->outstanding == 0; });
    }
    s->cv.notify_all();
    if (s->sched.joinable()) s->sched.join();
    for (auto& slot : s->slots) {
        cudaStreamSynchronize(slot.stream);
        edt_plan_destroy(slot.plan);
        cudaStreamDestroy(slot.stream);
    }
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
    return EDT_OK;
}
