// Continuous-batching server (edt_serve_create / _submit / _poll / _destroy).
//
// Jobs arrive with HOST buffers.  A scheduler thread keeps a FIFO of submitted
// jobs and a set of CUDA streams, each owning a batch plan.  Whenever a stream
// is idle and the head of the FIFO fits the device-memory budget, it admits
// jobs in arrival order while they fit, allocates their device buffers (and
// the batch's column-pass scratch) from the server's memory pool, and
// enqueues on that stream: the mask copies in, batched replays for every job
// the batch kernels cover (2-D of any width, 3-D volumes up to the batch
// limits) and plain transforms for the rest (larger volumes), each job's
// result copies out followed by an event of that job, the buffer frees, and
// a last event.  A completion thread per stream waits for the jobs' events in
// turn and completes each ticket as soon as its job's results are on the
// host, with the status the device reports (an error raised by the GPU after
// enqueueing fails the tickets), returning the job's bytes to the budget; the
// last event frees the stream.  Batches on different streams
// overlap on the device; requests that arrive while batches run are admitted
// as soon as a stream and enough budget are free.  Every result is the same as
// a plain edt_feature call on the same mask (the kernels do not depend on
// batch membership), which the tests check alone and in the mix.
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
edt_status batch_enqueue(edt_plan* p, const edt_job* jobs, int n, char* scratch, cudaStream_t stream);
}  // namespace edt

using namespace edt;

namespace {

using Clock = std::chrono::steady_clock;

constexpr int SERVE_PLAN_JOBS = 512;          // jobs per batched launch
// pixels admitted to one stream at a time (beyond the first job): a stream
// is busy until its whole batch is done, so a long backlog is split over the streams in
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
    double latency = 0.0;    // submission -> completion
    double wait = 0.0;       // submission -> admission to a stream
    Clock::time_point t_submit, t_admit;
};

struct Completion {
    size_t bytes;            // budget bytes of the batch not yet given back
    std::vector<uint64_t> tickets;
    std::vector<size_t> job_bytes;
    int recorded = 0;        // jobs 0 .. recorded-1 have their own event
    edt_status status;       // of the enqueueing
};

// One stream with its batch plan and the thread that completes its batches.
struct StreamSlot {
    cudaStream_t stream = nullptr;
    edt_plan* plan = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<cudaEvent_t> job_done;   // one per job of a batch: its results are on the host
    bool busy = false;
    Completion* pending = nullptr;   // enqueued, waiting for `done`
    std::thread completer;
};

}  // namespace

struct edt_server {
    int device = 0;
    int sm_count = 0;
    cudaMemPool_t pool = nullptr;   // job buffers: the server's own pool, grown to the budget at creation
    size_t budget = 0;       // bytes available to job buffers
    size_t in_use = 0;
    int64_t plan_pixels = 0;
    std::vector<StreamSlot> slots;     // fixed once created (threads keep indices)
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

// Completion thread of stream slot `si`: for each enqueued batch, completes
// every job's ticket as soon as that job's results are on the host (its own
// event, recorded after its copies back), with the device's status, and gives
// its bytes back to the budget; then waits for the batch's last event and
// frees the stream.
void completer(edt_server* s, int si)
{
    cudaSetDevice(s->device);
    StreamSlot& slot = s->slots[si];
    std::unique_lock<std::mutex> lk(s->mu);
    auto finish = [&](uint64_t t, edt_status status, size_t bytes) {   // with the lock held
        auto it = s->tickets.find(t);
        if (it != s->tickets.end()) {
            it->second.state = 2;
            it->second.status = status;
            it->second.latency = std::chrono::duration<double>(Clock::now() - it->second.t_submit).count();
        }
        s->in_use -= bytes;
        --s->outstanding;
    };
    for (;;) {
        s->cv.wait(lk, [&] { return slot.pending != nullptr || (s->stopping && !slot.busy); });
        if (!slot.pending) break;
        Completion* c = slot.pending;
        lk.unlock();
        size_t given = 0;
        for (int k = 0; k < c->recorded; ++k) {
            const cudaError_t e = cudaEventSynchronize(slot.job_done[k]);
            edt_status status = c->status;
            if (status == EDT_OK && e != cudaSuccess) status = EDT_ERR_CUDA;
            lk.lock();
            finish(c->tickets[k], status, c->job_bytes[k]);
            given += c->job_bytes[k];
            s->cv.notify_all();
            lk.unlock();
        }
        const cudaError_t e = cudaEventSynchronize(slot.done);
        edt_status status = c->status;
        if (status == EDT_OK && e != cudaSuccess) status = EDT_ERR_CUDA;
        lk.lock();
        for (size_t k = (size_t)c->recorded; k < c->tickets.size(); ++k) {
            finish(c->tickets[k], status, c->job_bytes[k]);
            given += c->job_bytes[k];
        }
        s->in_use -= c->bytes - given;   // the rest of the batch's bytes (none when every job was counted)
        slot.pending = nullptr;
        slot.busy = false;
        delete c;
        s->cv.notify_all();
    }
}

bool served_in_batch(const edt_job& j) { return batch_kind(j, nullptr) >= 0; }

size_t job_bytes(const edt_job& j, int64_t n)
{
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t b = al((size_t)n) + al((size_t)n * 4);           // mask, F
    if (j.D) b += al((size_t)n * 4);
    if (j.dist) b += al((size_t)n * 4);
    b += al(served_in_batch(j) ? batch_job_scratch_bytes(j) : scratch_bytes(j.ndim, j.shape));   // column pass
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
        const bool batched = served_in_batch(p.job);
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
    // batched jobs: one or more plan replays, each with its column-pass
    // scratch from the pool (counted in the jobs' bytes)
    std::vector<void*> bscratch;
    for (size_t off = 0; off < bj.size() && status == EDT_OK;) {
        const int cnt = (int)std::min<size_t>(bj.size() - off, (size_t)SERVE_PLAN_JOBS);
        size_t sb = 0;
        int64_t words = 0;
        batch_layout(bj.data() + off, cnt, &sb, &words);
        void* sc = nullptr;
        cudaError_t e = cudaMallocFromPoolAsync(&sc, sb > 0 ? sb : 256, s->pool, st);
        if (e != cudaSuccess) {
            status = cuda_fail(e, "serve: batch scratch");
            break;
        }
        bscratch.push_back(sc);
        status = batch_enqueue(slot.plan, bj.data() + off, cnt, static_cast<char*>(sc), st);
        off += cnt;
    }
    for (void* sc : bscratch) cudaFreeAsync(sc, st);
    // results back job by job, each followed by its own event, so that a
    // job's ticket completes when its own results are on the host
    int recorded = 0;
    while (slot.job_done.size() < batch.size()) {
        cudaEvent_t ev = nullptr;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) break;
        slot.job_done.push_back(ev);
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
            if (status == EDT_OK && (size_t)recorded == k && k < slot.job_done.size() &&
                cudaEventRecord(slot.job_done[k], st) == cudaSuccess)
                ++recorded;
        }
        if (d.mask) cudaFreeAsync(d.mask, st);
        if (d.D) cudaFreeAsync(d.D, st);
        if (d.F) cudaFreeAsync(d.F, st);
        if (d.dist) cudaFreeAsync(d.dist, st);
        if (d.scratch) cudaFreeAsync(d.scratch, st);
    }
    Completion* c = new Completion{bytes, {}, {}, status == EDT_OK ? recorded : 0, status};
    for (const Pending& p : batch) {
        c->tickets.push_back(p.ticket);
        c->job_bytes.push_back(p.bytes);
    }
    cudaError_t e = cudaEventRecord(slot.done, st);
    if (e != cudaSuccess) {
        // the stream is broken: wait for what was enqueued, fail the tickets
        cudaStreamSynchronize(st);
        c->status = cuda_fail(e, "serve: cudaEventRecord");
        cudaEventRecord(slot.done, 0);
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        slot.pending = c;
    }
    s->cv.notify_all();
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
        const auto now = Clock::now();
        for (const Pending& p : batch) {
            Ticket& t = s->tickets[p.ticket];
            t.state = 1;
            t.t_admit = now;
            t.wait = std::chrono::duration<double>(now - t.t_submit).count();
        }
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
    // the batches' column-pass scratch comes from the pool with the jobs; a
    // plan keeps its job tables, its counters and a small scratch of its own
    s->plan_pixels = 4096;
    size_t reserved = 0;
    s->slots.reserve((size_t)n_streams);
    for (int k = 0; k < n_streams; ++k) {
        s->slots.emplace_back();
        StreamSlot& slot = s->slots.back();
        cudaError_t e = cudaStreamCreateWithFlags(&slot.stream, cudaStreamNonBlocking);
        // the completion thread spins on this event (no interrupt wake-up): it
        // frees the stream for the next batch as soon as the device is done
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&slot.done, cudaEventDisableTiming);
        if (e != cudaSuccess) { st = cuda_fail(e, "cudaStreamCreate / cudaEventCreate"); break; }
        st = edt_plan_create(&slot.plan, SERVE_PLAN_JOBS, s->plan_pixels);
        if (st != EDT_OK) break;
        reserved += (size_t)SERVE_PLAN_JOBS * (16 * BATCH_MAX_W + 1024 + sizeof(BatchJob)) + ((size_t)1 << 20);
    }
    if (st != EDT_OK || reserved >= mem_budget_bytes) {
        for (auto& slot : s->slots) {
            if (slot.plan) edt_plan_destroy(slot.plan);
            if (slot.done) cudaEventDestroy(slot.done);
            if (slot.stream) cudaStreamDestroy(slot.stream);
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
                cudaEventDestroy(slot.done);
                cudaStreamDestroy(slot.stream);
            }
            delete s;
            return err;
        }
    }
    for (int k = 0; k < (int)s->slots.size(); ++k) s->slots[k].completer = std::thread(completer, s, k);
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

extern "C" edt_status edt_serve_poll_detail(edt_server* s, uint64_t ticket, double* latency_s, double* wait_s)
{
    if (!s) return fail(EDT_ERR_INVALID, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return fail(EDT_ERR_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
    if (it->second.state != 2) return EDT_ERR_NOT_READY;
    const edt_status st = it->second.status;
    if (latency_s) *latency_s = it->second.latency;
    if (wait_s) *wait_s = it->second.wait;
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
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->cv.notify_all();
    }
    for (auto& slot : s->slots)
        if (slot.completer.joinable()) slot.completer.join();
    for (auto& slot : s->slots) {
        cudaStreamSynchronize(slot.stream);
        edt_plan_destroy(slot.plan);
        cudaEventDestroy(slot.done);
        for (cudaEvent_t ev : slot.job_done) cudaEventDestroy(ev);
        cudaStreamDestroy(slot.stream);
    }
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
    return EDT_OK;
}
