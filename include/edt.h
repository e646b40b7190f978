/*
 * libedt -- exact squared Euclidean distance transform and feature map for
 * NVIDIA GB300 (sm_103a).
 *
 * The operation (T. Strutz, "The Distance Transform and its Computation",
 * Sec. 1.1 and Sec. 3): for a binary image or volume, every pixel p receives
 *     D(p) = min over source pixels q of |p - q|^2          (Eq. (4))
 * and F(p) = the 0-based row-major linear index of one source pixel q that
 * attains D(p) (the Voronoi / feature map of Fig. 2 and Fig. 21's k*).
 * Optionally dist(p) = the float32 nearest to sqrt(D(p)) (Sec. 3.1: the square
 * root is drawn after all squared distances are known).
 *
 * Which pixels are sources is chosen by `mode` (Sec. 1.1, Fig. 1):
 *     EDT_TO_OBJECT      sources are the nonzero mask bytes; background pixels
 *                        get their distance to the nearest object (Fig. 1c),
 *                        object pixels get 0;
 *     EDT_TO_BACKGROUND  sources are the zero mask bytes; object pixels get
 *                        their distance to the nearest background (Fig. 1b).
 * Only pixels inside the image count (no virtual border).  An image without
 * any source pixel yields D = INT32_MAX, F = -1 and dist = +inf everywhere.
 * D is exact (bit-identical to the definition); where several sources are
 * equally near, F names one of them.
 *
 * Conventions for every entry point:
 *   - Masks are uint8, any nonzero byte is an object pixel, C order: a 2-D
 *     mask is [H][W], a 3-D mask [Dz][H][W], unit isotropic spacing.
 *   - Unless an entry point says otherwise, every pointer is DEVICE memory
 *     owned by the caller; outputs must not overlap inputs or each other.
 *   - Calls are asynchronous on the given CUDA stream (0 = legacy default
 *     stream); results are ready when the stream reaches that point.
 *   - Every call returns an edt_status; nothing throws or aborts across the
 *     ABI.  edt_last_error() describes the last failure on the calling thread.
 *   - Size limits (EDT_ERR_TOO_LARGE beyond them): every side <= 32767; a 2-D
 *     row width W <= 16384; a 3-D volume H <= 2048 and W <= 1024 (a block
 *     holds 32 whole lines of y resp. x in shared memory); fewer than 2^31
 *     pixels in total; and the largest squared distance inside the image,
 *     sum of (side - 1)^2, must stay below 2^31 - 1 so that D fits int32.
 *   - Scratch memory: the plain calls draw their scratch from the device's
 *     stream-ordered memory pool (cudaMallocAsync on the given stream, freed on
 *     the same stream): about 0.26 byte per pixel for 2-D images, 2.26 bytes
 *     per voxel for 3-D volumes (the column pass's words plus every voxel's
 *     int16 offset to its nearest source along z); batch plans and servers own
 *     theirs.
 *   - Threads: the plain, pair, host-buffer, city-block and chamfer calls may
 *     be made from several host threads at once (on separate streams, with
 *     separate buffers); a plan is used from one thread at a time and
 *     edt_feature2d_noalloc calls must be ordered by the caller (see there).
 */
#ifndef LIBEDT_EDT_H
#define LIBEDT_EDT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *edt_stream_t; /* same type as cudaStream_t */

typedef enum {
    EDT_OK = 0,
    EDT_ERR_INVALID = 1,    /* null pointer, side <= 0, bad ndim or mode     */
    EDT_ERR_TOO_LARGE = 2,  /* a size limit above is exceeded                 */
    EDT_ERR_NOMEM = 3,      /* device or host allocation failed               */
    EDT_ERR_CUDA = 4,       /* a CUDA runtime call or kernel launch failed    */
    EDT_ERR_TIMEOUT = 5,    /* a bounded wait gave up                         */
    EDT_ERR_BUDGET = 6,     /* a served job can never fit the memory budget   */
    EDT_ERR_NOT_READY = 7   /* a served job has not finished yet              */
} edt_status;

enum { EDT_TO_OBJECT = 0, EDT_TO_BACKGROUND = 1 };

/* Squared 2-D EDT (Sec. 3.1 column scans + Sec. 3.3.1 row envelope).
 * mask: [H][W] uint8 (device); D: [H][W] int32 output (device). */
edt_status edt_sq2d(const uint8_t *mask, int H, int W, int mode, int32_t *D,
                    edt_stream_t stream);

/* Squared 3-D EDT of a [Dz][H][W] volume (the same method applied along z,
 * y and x; Sec. 3.1 treats the axes one after another). */
edt_status edt_sq3d(const uint8_t *mask, int Dz, int H, int W, int mode,
                    int32_t *D, edt_stream_t stream);

/* Squared EDT plus feature map, 2-D (ndim = 2, shape = {H, W}) or 3-D
 * (ndim = 3, shape = {Dz, H, W}).  F is required; D and dist may be NULL
 * (dist = correctly rounded float32 sqrt(D), Sec. 3.1).  shape is a host
 * pointer. */
edt_status edt_feature(const uint8_t *mask, int ndim, const int *shape,
                       int mode, int32_t *D, int32_t *F, float *dist,
                       edt_stream_t stream);

/* Both transforms of one mask (Sec. 1.1, Fig. 1(b) and 1(c)) from a single
 * read of it: EDT_TO_OBJECT results (distances of background pixels to the
 * nearest object) into D_obj / F_obj and EDT_TO_BACKGROUND results (distances
 * of object pixels to the nearest background) into D_bg / F_bg.  Each result
 * is bit-identical to the corresponding edt_feature call.  For 2-D images
 * the column pass runs once for both and one row launch covers both; 3-D
 * volumes run the two transforms one after the other.  F_obj and F_bg are
 * required, D_obj and D_bg may be NULL.  Device pointers. */
edt_status edt_feature_pair(const uint8_t *mask, int ndim, const int *shape,
                            int32_t *D_obj, int32_t *F_obj, int32_t *D_bg,
                            int32_t *F_bg, edt_stream_t stream);

/* The same as edt_feature with HOST buffers: mask, D, F, dist are host
 * pointers (pinned memory gives the fastest copies; pageable works).  The
 * call copies the mask to the device, runs the transform, copies the
 * results back and returns when they are in the host buffers.  Device
 * buffers come from the stream-ordered pool of the current device.  For 2-D
 * images the row pass runs in up to four launches over consecutive bands and
 * the rows of each go back to the host (on a copy stream of libedt's own)
 * while the next launch runs. */
edt_status edt_feature_host(const uint8_t *mask, int ndim, const int *shape,
                            int mode, int32_t *D, int32_t *F, float *dist,
                            edt_stream_t stream);

/* edt_feature_pair with HOST buffers (the mask is copied to the device once
 * for both transforms), in the manner of edt_feature_host.  F_obj and F_bg
 * are required, D_obj and D_bg may be NULL. */
edt_status edt_feature_pair_host(const uint8_t *mask, int ndim, const int *shape,
                                 int32_t *D_obj, int32_t *F_obj, int32_t *D_bg,
                                 int32_t *F_bg, edt_stream_t stream);

/* City-block distance transform of a 2-D image (Sec. 2.1): D[i][j] = the
 * smallest |i - a| + |j - b| over the source pixels (a, b) of `mode`,
 * INT32_MAX when the image has no source.  The same result as the paper's
 * sequential two-scan and four-scan algorithms.  Device pointers; D is
 * H x W int32, row-major.  Errors as edt_sq2d. */
edt_status edt_cityblock2d(const uint8_t *mask, int H, int W, int mode,
                           int32_t *D, edt_stream_t stream);

/* Chamfer 4-3 distance transform of a 2-D image (Sec. 2.2): D[i][j] = the
 * smallest 3 max(|i - a|, |j - b|) + min(|i - a|, |j - b|) over the source
 * pixels (a, b) of `mode` -- the cost of the cheapest path with steps of 3
 * (horizontal, vertical) and 4 (diagonal), the result of the paper's two
 * raster scans -- INT32_MAX when the image has no source.  Device pointers;
 * D is H x W int32, row-major; scratch (about 4 bytes per pixel plus
 * about 0.25 byte per position of each of the two sheared H x (W + H - 1)
 * views the column passes run over) comes from the stream-ordered pool.  Errors as edt_sq2d; rows wider than 14336 columns return
 * EDT_ERR_TOO_LARGE (a block keeps two sheared column records of 8 bytes per
 * column of its rows in shared memory). */
edt_status edt_chamfer43_2d(const uint8_t *mask, int H, int W, int mode,
                            int32_t *D, edt_stream_t stream);

/* One transform in a batch.  Pointers are device memory; F required, D and
 * dist may be NULL; shape[2] is ignored for ndim = 2. */
typedef struct {
    const uint8_t *mask;
    int ndim;
    int shape[3];
    int mode;
    int32_t *D;
    int32_t *F;
    float *dist;
} edt_job;

typedef struct edt_plan edt_plan;

/* A batch plan owns the device scratch, a device job table and the CUDA graph
 * that run up to n_max jobs in one replay: 2-D jobs of any width edt_feature
 * accepts and 3-D jobs whose y and x lines fit the batched 3-D kernels'
 * shared memory (height up to about 1150, row width up to about 670; larger
 * volumes: edt_feature).  `max_pixels` sizes the column-pass scratch the plan
 * allocates up front (about 0.26 bytes per pixel of 2-D jobs up to 2048 wide);
 * a batch that needs more grows it, which allocates and waits for the plan's
 * earlier batches.  Not thread-safe: use one plan from one thread and one
 * stream; plan creation allocates and may synchronise.  (Sec. 3: every job is
 * the same column pass and envelope passes as edt_feature.) */
edt_status edt_plan_create(edt_plan **plan, int n_max, int64_t max_pixels);
edt_status edt_plan_destroy(edt_plan *plan);

/* Run n jobs (n <= n_max; 2-D and 3-D mixed; pointers are device memory, F
 * required) as one graph replay on `stream`: the job table is copied to the
 * device and persistent kernels cover every job, one phase after the other
 * (column pass of all jobs, 2-D row passes, 3-D y passes, 3-D x passes).
 * Results are bit-identical to n separate edt_feature calls.  Returns after
 * enqueueing; the host may then reuse `jobs`.  EDT_ERR_TOO_LARGE for a 3-D
 * job the batch does not cover, EDT_ERR_INVALID for n > n_max or a NULL mask
 * or F. */
edt_status edt_batch(edt_plan *plan, const edt_job *jobs, int n,
                     edt_stream_t stream);

/* Autotuning of the batch geometry.  Times, for each shape class (the
 * rounded-up log2 of each side) among `jobs`, the candidate geometries of the
 * batch kernels on those jobs -- narrow 2-D jobs: the smallest row segment,
 * 2^8, 2^7 or 2^6 columns; 3-D jobs: 64, 32 or 128 positions per warp for the
 * y pass, then 32, 64 or 128 for the x pass -- and keeps the fastest in the
 * process-wide table that every later batch uses (saved and loaded with
 * edt_tune_save / edt_tune_load), provided the whole batch then runs more
 * than 1 % faster than with the built-in geometry (the two timed alternately,
 * twice each, the better time of each compared; else the built-in geometry is
 * stored for those classes).  Rows wider than 2048 have no knob.  n must not exceed the
 * plan's n_max (EDT_ERR_INVALID).  Runs the jobs (device pointers, as
 * edt_batch) several times on `stream`, which overwrites their outputs with
 * the same bits; synchronous.  Results never depend on the choice. */
edt_status edt_autotune_batch(edt_plan *plan, const edt_job *jobs, int n,
                              edt_stream_t stream);
/* The batch geometry in the table for a shape: values[0] = smallest row
 * segment log2 (0 = built-in 8), values[1] / values[2] = y / x positions per
 * warp (0 = built-in 64 / 32). */
edt_status edt_batch_tune_get(int ndim, const int *shape, int *values);

/* Continuous-batching server.  Jobs carry HOST pointers (mask in, D/F/dist
 * out).  A scheduler thread admits jobs while their device footprint fits
 * mem_budget_bytes, copies them in, groups the admitted jobs into batches
 * (edt_batch's kernels; 3-D volumes beyond the batch limits run as plain
 * transforms), runs them on n_streams streams so that batches overlap, copies
 * results out job by job and completes each ticket once that job's results
 * are on the host, with the device's status (a GPU error after enqueueing
 * fails the ticket).  Each result is identical to a plain edt_feature
 * call on the same mask.  The budget is taken from the device when the
 * server is created (a memory pool of its own, grown to the budget less the
 * batch plans' scratch) and given back by edt_serve_destroy; EDT_ERR_BUDGET
 * when it exceeds the device's free memory or does not cover the plans,
 * EDT_ERR_CUDA if the device still cannot provide it. */
typedef struct edt_server edt_server;

edt_status edt_serve_create(edt_server **server, size_t mem_budget_bytes,
                            int n_streams);
/* Queue one job; its host buffers must stay valid until the ticket is
 * polled as done.  EDT_ERR_BUDGET when the job alone exceeds the budget. */
edt_status edt_serve_submit(edt_server *server, const edt_job *job,
                            uint64_t *ticket);
/* EDT_OK when done (latency_s = seconds from submit to completion, may be
 * NULL), EDT_ERR_NOT_READY while queued or running, another status when the
 * job failed.  A finished ticket is forgotten after it was reported once. */
edt_status edt_serve_poll(edt_server *server, uint64_t ticket,
                          double *latency_s);
/* edt_serve_poll that also reports wait_s, the seconds from submission to
 * admission to a stream (latency_s - wait_s is the time on the stream:
 * copies, transform, copies back).  Either pointer may be NULL. */
edt_status edt_serve_poll_detail(edt_server *server, uint64_t ticket,
                                 double *latency_s, double *wait_s);
/* Wait until every submitted job has finished, then stop the scheduler and
 * free everything. */
edt_status edt_serve_destroy(edt_server *server);

/* Kernel timing for diagnostics and benchmarks.  While enabled, every kernel
 * this library launches is bracketed by two CUDA events recorded on the
 * stream it is launched on.  edt_trace_read waits for the recorded events and
 * returns, for the kernel named `kernel` (e.g. "k_rows2d"), the summed elapsed
 * milliseconds and the number of launches since tracing was last enabled.
 * Enabling resets the record.  Costs two event records per launch. */
edt_status edt_trace_enable(int on);
edt_status edt_trace_read(const char *kernel, double *total_ms,
                          int64_t *launches);

/* Allocation-free variant of edt_feature for 2-D images.  The paper has no
 * counterpart: this is an interface for callers that may not allocate device
 * memory on the call path -- plugins whose host framework owns every device
 * allocation, or latency-critical code that cannot risk the implicit device
 * synchronisation of cudaMalloc / cudaFree.  It calls no allocator: the
 * column-pass scratch is a fixed 32 MiB static device array (enough for
 * 8192 x 8192), reserved on every GPU that loads libedt until the process
 * exits; images whose scratch does not fit return EDT_ERR_TOO_LARGE.
 * Arguments as for edt_feature with ndim = 2 (device pointers; F required, D
 * and dist may be NULL); results are bit-identical to edt_feature.
 * The first call on a device resolves the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array: calls that
 * overlap on the GPU (other streams, other threads) race on it, so the caller
 * must order them (e.g. one stream). */
edt_status edt_feature2d_noalloc(const uint8_t *mask, int H, int W, int mode,
                                 int32_t *D, int32_t *F, float *dist,
                                 edt_stream_t stream);

/* Autotuning of the band geometry.  The envelope passes give each band of
 * 32 lines (rows for 2-D, y and x lines for 3-D) several warps, each taking
 * one segment of the lines, and merge the segments' envelopes; the number of
 * warps per band trades per-warp work against merge depth and resident
 * blocks.  edt_autotune times the candidates (2-D rows: 16, 8, 4 warps; 3-D
 * y pass: 8, 4, 16, 32, then x pass: 32, 16, 8) on `mask` (DEVICE, the given
 * shape and mode) and keeps the fastest for the shape's class -- the
 * rounded-up log2 of each side -- in a process-wide table that every later
 * call of that class uses (plain, pair and host-buffer calls; batches are
 * tuned by edt_autotune_batch).  Results do not depend on the choice: D and F are the same
 * bits for every candidate.  Synchronous; device scratch from the stream's
 * pool.  Without tuning, the built-in rule applies (16, 8, 32). */
edt_status edt_autotune(const uint8_t *mask, int ndim, const int *shape,
                        int mode, edt_stream_t stream);
/* The tuned warps per band of a shape's class: warps[0] = 2-D rows,
 * warps[1] = 3-D y pass, warps[2] = 3-D x pass; 0 = the built-in rule.
 * Host-only (no device needed). */
edt_status edt_tune_get(int ndim, const int *shape, int *warps);
/* Write the table to a text file / merge a file into the table (lines of
 * "ndim log2(side0) log2(side1) log2(side2) rows2d ypass xpass", '#' starts
 * a comment; warp counts are powers of two up to 16, 32, 32, or 0; batch
 * geometry lines "b ndim log2(side0) log2(side1) log2(side2) lgmin ypos
 * xpos" with lgmin 0 or 6..8 and positions 0, 32, 64 or 128).
 * Host-only; EDT_ERR_INVALID for unreadable or malformed files (the table is
 * then unchanged). */
edt_status edt_tune_save(const char *path);
edt_status edt_tune_load(const char *path);

/* Message of the last failure on the calling thread ("" when none). */
const char *edt_last_error(void);

/* Library version string. */
const char *edt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LIBEDT_EDT_H */
