// Batched 2-D transforms (edt_plan_create / edt_batch / edt_plan_destroy).
//
// A plan owns: the device scratch of the column pass for all jobs of a batch,
// the arrival counters (one contiguous block, cleared by one memset), a device
// job table, two pinned host copies of that table and two CUDA graphs.  Each
// graph is [copy table host->device, clear counters, persistent column-pass
// kernel, persistent row-pass kernel]; the kernels read the job count and all
// per-job geometry from the table, so one instantiated graph serves every
// batch.  edt_batch fills a pinned table (jobs sorted widest first, so that
// the row pass hands out the most expensive work items first) and replays the
// graph on the caller's stream; the two tables alternate so that the host can
// prepare batch n+1 while batch n still copies.
#include <algorithm>
#include <cstring>
#include <vector>

#include "edt_internal.h"

namespace edt {
edt_status fail(edt_status st, const char* fmt, ...);
edt_status cuda_fail(cudaError_t e, const char* what);
void clear_error();
edt_status device_setup(int* sm_count);
edt_status check_shape(int ndim, const int* shape, int mode);
}  // namespace edt

using namespace edt;

struct edt_plan {
    int device = 0;
    int n_max = 0;
    int64_t max_pixels = 0;
    int sm_count = 0;
    size_t scratch_bytes = 0;
    size_t counter_words = 0;
    size_t table_bytes = 0;
    char* scratch = nullptr;          // device
    unsigned* counters = nullptr;     // device: [0] row-pass work counter, then tiles
    char* dtable = nullptr;           // device: BatchHeader + BatchJob[n_max]
    char* htable[2] = {nullptr, nullptr};   // pinned host copies
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaEvent_t done[2] = {nullptr, nullptr};
    int next = 0;
};

static size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// Bytes of column-pass scratch (without counters) of one H x W job.
static size_t job_scratch_bytes(const ColGeom& g)
{
    const size_t c = (size_t)g.cols * 4;
    return 2 * al256((size_t)g.nb * c) + 2 * al256((size_t)g.nG * c);
}

static void plan_free(edt_plan* p)
{
    if (!p) return;
    for (int b = 0; b < 2; ++b) {
        if (p->exec[b]) cudaGraphExecDestroy(p->exec[b]);
        if (p->done[b]) cudaEventDestroy(p->done[b]);
        if (p->htable[b]) cudaFreeHost(p->htable[b]);
    }
    if (p->scratch) cudaFree(p->scratch);
    if (p->counters) cudaFree(p->counters);
    if (p->dtable) cudaFree(p->dtable);
    delete p;
}

extern "C" edt_status edt_plan_create(edt_plan** out, int n_max, int64_t max_pixels)
{
    if (!out) return fail(EDT_ERR_INVALID, "plan pointer is NULL");
    *out = nullptr;
    if (n_max <= 0 || max_pixels <= 0) return fail(EDT_ERR_INVALID, "n_max and max_pixels must be positive");
    int sms = 0;
    edt_status st = device_setup(&sms);
    if (st != EDT_OK) return st;
    cudaError_t e;
    if ((e = set_batch_attributes()) != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    edt_plan* p = new edt_plan();
    cudaGetDevice(&p->device);
    p->n_max = n_max;
    p->max_pixels = max_pixels;
    p->sm_count = sms;
    // per job at most (2*ceil(H/32) + 2*ceil(H/1024)) * W * 4 bytes + alignment
    p->scratch_bytes = (size_t)(0.26 * (double)max_pixels) + (size_t)n_max * (16 * BATCH_MAX_W + 1024);
    p->counter_words = 1 + (size_t)n_max * ((BATCH_MAX_W + 31) / 32);
    p->table_bytes = sizeof(BatchHeader) + (size_t)n_max * sizeof(BatchJob);
    if ((e = cudaMalloc(&p->scratch, p->scratch_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&p->counters, p->counter_words * 4)) != cudaSuccess ||
        (e = cudaMalloc(&p->dtable, p->table_bytes)) != cudaSuccess) {
        plan_free(p);
        return cuda_fail(e, "cudaMalloc (batch plan)");
    }
    cudaStream_t cs = nullptr;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) {
        plan_free(p);
        return cuda_fail(e, "cudaStreamCreate");
    }
    const auto* hdr = reinterpret_cast<const BatchHeader*>(p->dtable);
    const auto* jobs = reinterpret_cast<const BatchJob*>(p->dtable + sizeof(BatchHeader));
    const int k1_blocks = sms * batch_colbits_blocks_per_sm();
    const int k2_blocks = sms * batch_rows_blocks_per_sm();
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        if ((e = cudaMallocHost(&p->htable[b], p->table_bytes)) != cudaSuccess) break;
        memset(p->htable[b], 0, p->table_bytes);
        if ((e = cudaEventCreateWithFlags(&p->done[b], cudaEventDisableTiming)) != cudaSuccess) break;
        cudaGraph_t graph = nullptr;
        if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) break;
        cudaMemcpyAsync(p->dtable, p->htable[b], p->table_bytes, cudaMemcpyHostToDevice, cs);
        cudaMemsetAsync(p->counters, 0, p->counter_words * 4, cs);
        launch_batch_colbits(hdr, jobs, k1_blocks, cs);
        launch_batch_rows2d(hdr, jobs, p->counters, k2_blocks, cs);
        e = cudaStreamEndCapture(cs, &graph);
        if (e != cudaSuccess) break;
        e = cudaGraphInstantiate(&p->exec[b], graph, 0);
        cudaGraphDestroy(graph);
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        plan_free(p);
        return cuda_fail(e, "building the batch graph");
    }
    *out = p;
    clear_error();
    return EDT_OK;
}

extern "C" edt_status edt_plan_destroy(edt_plan* p)
{
    if (!p) return EDT_OK;
    for (int b = 0; b < 2; ++b)
        if (p->done[b]) cudaEventSynchronize(p->done[b]);
    plan_free(p);
    return EDT_OK;
}

extern "C" edt_status edt_batch(edt_plan* p, const edt_job* jobs, int n, edt_stream_t stream)
{
    if (!p) return fail(EDT_ERR_INVALID, "plan is NULL");
    if (n < 0 || n > p->n_max) return fail(EDT_ERR_INVALID, "batch of %d jobs exceeds the plan's %d", n, p->n_max);
    if (n == 0) return EDT_OK;
    if (!jobs) return fail(EDT_ERR_INVALID, "jobs is NULL");
    int64_t px = 0;
    for (int i = 0; i < n; ++i) {
        const edt_job& j = jobs[i];
        if (j.ndim != 2) return fail(EDT_ERR_INVALID, "batch job %d: only 2-D jobs are batched", i);
        edt_status st = check_shape(2, j.shape, j.mode);
        if (st != EDT_OK) return st;
        if (j.shape[1] > BATCH_MAX_W)
            return fail(EDT_ERR_TOO_LARGE, "batch job %d: width %d exceeds %d", i, j.shape[1], BATCH_MAX_W);
        if (!j.mask || !j.F) return fail(EDT_ERR_INVALID, "batch job %d: mask and F must not be NULL", i);
        px += (int64_t)j.shape[0] * j.shape[1];
    }
    if (px > p->max_pixels)
        return fail(EDT_ERR_TOO_LARGE, "batch of %lld pixels exceeds the plan's %lld",
                    (long long)px, (long long)p->max_pixels);

    const int b = p->next;
    cudaError_t e = cudaEventSynchronize(p->done[b]);   // table b no longer being copied
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    // widest jobs first
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return jobs[a].shape[1] > jobs[c].shape[1];
    });
    auto* hdr = reinterpret_cast<BatchHeader*>(p->htable[b]);
    auto* tab = reinterpret_cast<BatchJob*>(p->htable[b] + sizeof(BatchHeader));
    size_t off = 0, cnt_off = 1;
    int64_t k1 = 0, k2 = 0;
    for (int t = 0; t < n; ++t) {
        const edt_job& j = jobs[order[t]];
        BatchJob& J = tab[t];
        const int H = j.shape[0], W = j.shape[1];
        J.mask = j.mask;
        J.D = j.D;
        J.F = j.F;
        J.dist = j.dist;
        J.g = col_geom(H, W, true);
        J.mode = j.mode;
        J.vec = (W % 16 == 0) && ((reinterpret_cast<uintptr_t>(j.mask) & 15) == 0);
        const size_t need = job_scratch_bytes(J.g);
        if (off + need > p->scratch_bytes)
            return fail(EDT_ERR_TOO_LARGE, "batch scratch exhausted at job %d", order[t]);
        const size_t c = (size_t)W * 4;
        char* base = p->scratch + off;
        J.s.C = reinterpret_cast<uint32_t*>(base);
        J.s.U = reinterpret_cast<uint32_t*>(base + al256((size_t)J.g.nb * c));
        J.s.GFL = reinterpret_cast<uint32_t*>(base + 2 * al256((size_t)J.g.nb * c));
        J.s.GAB = reinterpret_cast<uint32_t*>(base + 2 * al256((size_t)J.g.nb * c) + al256((size_t)J.g.nG * c));
        J.s.cnt = p->counters + cnt_off;
        J.s.gs = J.g.gs;
        off += need;
        cnt_off += (size_t)J.g.ntiles;
        batch_row_geometry(W, J.lg, J.NW, J.groups);
        J.pad0 = 0;
        J.k1_first = k1;
        J.k2_first = k2;
        k1 += J.g.ntiles * (int64_t)J.g.nG;
        k2 += (J.g.nb + J.groups - 1) / J.groups;
    }
    hdr->njobs = n;
    hdr->pad0 = 0;
    hdr->k1_total = k1;
    hdr->k2_total = k2;
    if ((e = cudaGraphLaunch(p->exec[b], (cudaStream_t)stream)) != cudaSuccess)
        return cuda_fail(e, "cudaGraphLaunch");
    if ((e = cudaEventRecord(p->done[b], (cudaStream_t)stream)) != cudaSuccess)
        return cuda_fail(e, "cudaEventRecord");
    p->next ^= 1;
    clear_error();
    return EDT_OK;
}
