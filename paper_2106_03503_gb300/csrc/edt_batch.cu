// Batched transforms (edt_plan_create / edt_batch / edt_plan_destroy).
//
// A plan owns: the device scratch of the column pass for all jobs of a batch,
// the work and arrival counters, a device job table, two pinned host copies of
// that table and two CUDA graphs.  Each graph is
//   [copy table host->device, clear counters, column pass, 2-D row pass,
//    wide 2-D row pass, 3-D y pass, 3-D x pass],
// every kernel persistent (a fixed grid that takes work items from the
// table), so one instantiated graph serves every batch: 2-D jobs of any
// accepted width and 3-D jobs, mixed.  The kernels find the counters and the
// job count through the table, so the scratch and counters may be
// reallocated between batches without touching the graph.  edt_batch fills a
// pinned table (edt_batch_table.cu) and replays the graph on the caller's
// stream; the two tables alternate so that the host can prepare batch n+1
// while batch n still copies.
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

cudaError_t set_batch_attributes()
{
    cudaError_t e = set_batch_row_attributes();
    if (e != cudaSuccess) return e;
    return set_batch_3d_attributes();
}
}  // namespace edt

using namespace edt;

struct edt_plan {
    int device = 0;
    int n_max = 0;
    int sm_count = 0;
    size_t scratch_bytes = 0;
    int64_t cnt_words = 0;
    size_t table_bytes = 0;
    char* scratch = nullptr;          // device
    unsigned* cnt = nullptr;          // device: work counters, then arrival counters
    char* dtable = nullptr;           // device: BatchHeader + BatchJob[n_max]
    char* htable[2] = {nullptr, nullptr};   // pinned host copies
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaEvent_t done[2] = {nullptr, nullptr};
    int next = 0;
};

static void plan_free(edt_plan* p)
{
    if (!p) return;
    for (int b = 0; b < 2; ++b) {
        if (p->exec[b]) cudaGraphExecDestroy(p->exec[b]);
        if (p->done[b]) cudaEventDestroy(p->done[b]);
        if (p->htable[b]) cudaFreeHost(p->htable[b]);
    }
    if (p->scratch) cudaFree(p->scratch);
    if (p->cnt) cudaFree(p->cnt);
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
    p->sm_count = sms;
    // enough for 2-D jobs up to BATCH_MAX_W wide totalling max_pixels (about
    // 0.26 B/pixel, plus the rounding of each job to whole bands); a batch
    // that needs more grows it
    p->scratch_bytes = (size_t)(0.26 * (double)max_pixels) + (size_t)n_max * (16 * BATCH_MAX_W + 1024);
    p->cnt_words = PH_COUNT + (int64_t)n_max * ((BATCH_MAX_W + 31) / 32);
    p->table_bytes = sizeof(BatchHeader) + (size_t)n_max * sizeof(BatchJob);
    if ((e = cudaMalloc(&p->scratch, p->scratch_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&p->cnt, (size_t)p->cnt_words * 4)) != cudaSuccess ||
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
    const int kw_blocks = sms * batch_wide_blocks_per_sm();
    const int k3_blocks = sms * batch_3d_blocks_per_sm();
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        if ((e = cudaMallocHost(&p->htable[b], p->table_bytes)) != cudaSuccess) break;
        memset(p->htable[b], 0, p->table_bytes);
        if ((e = cudaEventCreateWithFlags(&p->done[b], cudaEventDisableTiming)) != cudaSuccess) break;
        cudaGraph_t graph = nullptr;
        if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) break;
        cudaMemcpyAsync(p->dtable, p->htable[b], p->table_bytes, cudaMemcpyHostToDevice, cs);
        launch_batch_clear(hdr, sms * 2, cs);
        launch_batch_colbits(hdr, jobs, k1_blocks, cs);
        launch_batch_rows2d(hdr, jobs, k2_blocks, cs);
        launch_batch_wide(hdr, jobs, kw_blocks, cs);
        launch_batch_ypass3d(hdr, jobs, k3_blocks, cs);
        launch_batch_xpass3d(hdr, jobs, k3_blocks, cs);
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

// Grow the plan's scratch or counters to what a batch needs (after the
// plan's earlier batches have finished with them).
static edt_status plan_reserve(edt_plan* p, size_t scratch_bytes, int64_t cnt_words)
{
    if (scratch_bytes <= p->scratch_bytes && cnt_words <= p->cnt_words) return EDT_OK;
    cudaError_t e;
    for (int b = 0; b < 2; ++b)
        if ((e = cudaEventSynchronize(p->done[b])) != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    if (scratch_bytes > p->scratch_bytes) {
        const size_t want = std::max(scratch_bytes, p->scratch_bytes + p->scratch_bytes / 4);
        cudaFree(p->scratch);
        p->scratch = nullptr;
        p->scratch_bytes = 0;
        if ((e = cudaMalloc(&p->scratch, want)) != cudaSuccess) return cuda_fail(e, "cudaMalloc (batch scratch)");
        p->scratch_bytes = want;
    }
    if (cnt_words > p->cnt_words) {
        const int64_t want = std::max(cnt_words, p->cnt_words + p->cnt_words / 4);
        cudaFree(p->cnt);
        p->cnt = nullptr;
        p->cnt_words = 0;
        if ((e = cudaMalloc(&p->cnt, (size_t)want * 4)) != cudaSuccess) return cuda_fail(e, "cudaMalloc (batch counters)");
        p->cnt_words = want;
    }
    return EDT_OK;
}

// Validate a batch: every job a transform edt_feature accepts, of a shape the
// batch kernels cover.
static edt_status check_batch(const edt_job* jobs, int n)
{
    for (int i = 0; i < n; ++i) {
        const edt_job& j = jobs[i];
        edt_status st = check_shape(j.ndim, j.shape, j.mode);
        if (st != EDT_OK) return st;
        if (!j.mask || !j.F) return fail(EDT_ERR_INVALID, "batch job %d: mask and F must not be NULL", i);
        const char* why = "";
        if (batch_kind(j, &why) < 0) return fail(EDT_ERR_TOO_LARGE, "batch job %d: %s", i, why);
    }
    return EDT_OK;
}

namespace edt {

int plan_n_max(const edt_plan* p) { return p->n_max; }

// Enqueue a validated batch; scratch: the column-pass scratch to use (device,
// at least batch_layout's bytes), or NULL for the plan's own.
edt_status batch_enqueue(edt_plan* p, const edt_job* jobs, int n, char* scratch, cudaStream_t stream)
{
    size_t need = 0;
    int64_t words = 0;
    batch_layout(jobs, n, &need, &words);
    edt_status st = plan_reserve(p, scratch ? 0 : need, words);
    if (st != EDT_OK) return st;
    const int b = p->next;
    cudaError_t e = cudaEventSynchronize(p->done[b]);   // table b no longer being copied
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    auto* hdr = reinterpret_cast<BatchHeader*>(p->htable[b]);
    auto* tab = reinterpret_cast<BatchJob*>(p->htable[b] + sizeof(BatchHeader));
    batch_fill(jobs, n, scratch ? scratch : p->scratch, p->cnt, hdr, tab);
    if ((e = cudaGraphLaunch(p->exec[b], stream)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    if ((e = cudaEventRecord(p->done[b], stream)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    p->next ^= 1;
    return EDT_OK;
}

}  // namespace edt

extern "C" edt_status edt_batch(edt_plan* p, const edt_job* jobs, int n, edt_stream_t stream)
{
    if (!p) return fail(EDT_ERR_INVALID, "plan is NULL");
    if (n < 0 || n > p->n_max) return fail(EDT_ERR_INVALID, "batch of %d jobs exceeds the plan's %d", n, p->n_max);
    if (n == 0) return EDT_OK;
    if (!jobs) return fail(EDT_ERR_INVALID, "jobs is NULL");
    edt_status st = check_batch(jobs, n);
    if (st != EDT_OK) return st;
    st = batch_enqueue(p, jobs, n, nullptr, (cudaStream_t)stream);
    if (st == EDT_OK) clear_error();
    return st;
}
