// Internal declarations shared by the libedt translation units (host side).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/edt.h"

namespace edt {

// Scratch of the column pass for an image of `rows` x `cols` (rows = the
// scanned axis).  All arrays are uint32 in device memory, `cols` wide:
//   C    [nb][cols]  column-bit words, bit r = row 32*band + r is a source
//   U    [nb][cols]  nearest source row above | below << 16 of each band,
//                    looking only inside the band's group (1 << gs bands)
//                    (0xFFFF = none in the group)
//   GFL  [nG][cols]  first | last << 16 source row of each group
//   GAB  [nG][cols]  nearest source row above | below << 16 of each group,
//                    over the whole column (0xFFFF = none)
//   cnt  [ntiles]    arrival counters of the groups of one 32-column tile
struct ColScratch {
    uint32_t* C;
    uint32_t* U;
    uint32_t* GFL;
    uint32_t* GAB;
    unsigned* cnt;
    int gs;        // bands per group = 1 << gs (the group of band b is b >> gs)
};

struct ColGeom {
    int rows;
    int64_t cols;
    int nb;        // bands of 32 rows
    int gs;        // bands per group = 1 << gs
    int nG;        // groups of 1 << gs bands (at most 32)
    int64_t ntiles;  // tiles of 32 columns
};

// Geometry of an image of `rows` x `cols` for the column pass.  Groups have
// 32 bands, or fewer (down to 1) while the image gives fewer than 4096 warp
// units and a column keeps at most 32 groups; `coarse` keeps 32 bands per
// group (the batch plans size their scratch for that).
ColGeom col_geom(int rows, int64_t cols, bool coarse = false);
size_t col_scratch_bytes(const ColGeom& g);
ColScratch col_scratch_carve(void* base, const ColGeom& g);

// Launchers (asynchronous on `stream`; return cudaGetLastError()).
cudaError_t launch_colbits(const uint8_t* mask, const ColGeom& g, int mode,
                           const ColScratch& s, cudaStream_t stream);
// Row pass over bands [band0, band0 + nbl) (nbl < 0: to the last band).
cudaError_t launch_rows2d(int H, int W, const ColGeom& g, const ColScratch& s,
                          int32_t* D, int32_t* F, float* dist, int sm_count,
                          cudaStream_t stream, int band0 = 0, int nbl = -1);
cudaError_t launch_colbits_pair(const uint8_t* mask, const ColGeom& g, const ColScratch& s,
                                const ColScratch& s1, cudaStream_t stream);
cudaError_t launch_rows2d_pair(int H, int W, const ColGeom& g, const ColScratch& s_obj,
                               const ColScratch& s_bg, int32_t* D_obj, int32_t* F_obj,
                               int32_t* D_bg, int32_t* F_bg, cudaStream_t stream, int band0 = 0,
                               int nbl = -1);
// City-block row pass (Sec. 2.1): D from the column-pass scratch of the
// chosen sources.
cudaError_t launch_cityblock_rows(int H, int W, const ColGeom& g, const ColScratch& s, int32_t* D,
                                  cudaStream_t stream);
// Column pass over a sheared view of an imgH x imgW mask (g: the view's
// geometry): dir +1 turns the diagonals j - i = const into columns (view
// column v = j - i + imgH - 1), dir -1 the anti-diagonals (v = i + j).
cudaError_t launch_colbits_sheared(const uint8_t* mask, const ColGeom& g, int mode, const ColScratch& s,
                                   int imgH, int64_t imgW, int dir, cudaStream_t stream);

// Chamfer 4-3 transform (Sec. 2.2): scratch size and the whole pass sequence.
size_t chamfer_scratch_bytes(int H, int W);
cudaError_t launch_chamfer(const uint8_t* mask, int H, int W, int mode, int32_t* D, void* scratch,
                           int sm_count, cudaStream_t stream);
// 3-D: the z offset of every voxel's nearest source along z (int16,
// Dz*H*W entries) from the z column pass's scratch, then the y pass over
// them (d16 NULL: the y pass decodes the column words itself) and the x pass.
cudaError_t launch_zoffsets(int Dz, int H, int W, const ColGeom& g, const ColScratch& s, short* d16,
                            cudaStream_t stream);
cudaError_t launch_ypass3d(int Dz, int H, int W, const ColGeom& g,
                           const ColScratch& s, const short* d16, uint32_t* P, cudaStream_t stream);
cudaError_t launch_xpass3d(int Dz, int H, int W, uint32_t* P, int32_t* D,
                           int32_t* F, float* dist, cudaStream_t stream);

// Batched transforms.  A device job table (header + jobs) drives persistent
// kernels that each cover one phase of every job in the batch:
//   clear    zero the work and arrival counters (their number is in the header)
//   colbits  the column pass of every job (for 3-D the z pass over Dz x H*W)
//   rows2d   2-D row pass, widths up to BATCH_MAX_W (several bands side by side)
//   wide     2-D row pass, wider rows (one band per block)
//   ypass    3-D y pass (several (z, x-tile) units side by side)
//   xpass    3-D x pass (several 32-row units side by side)
// Each phase numbers its work items job by job (k_first[phase]); a job of
// another kind has none in that phase.
enum BatchKind { BATCH_2D = 0, BATCH_2D_WIDE = 1, BATCH_3D = 2 };
enum BatchPhase { PH_COL = 0, PH_ROWS = 1, PH_WIDE = 2, PH_Y = 3, PH_X = 4, PH_COUNT = 5 };

struct BatchJob {
    const uint8_t* mask;
    int32_t* D;
    int32_t* F;
    float* dist;
    ColScratch s;
    ColGeom g;             // column pass: rows = H (2-D) or Dz (3-D), cols = W or H*W
    int kind, mode, vec;   // vec: 16-byte mask loads allowed
    int Dz, H, W;          // image shape (Dz = 1 for 2-D)
    int lg, NW, groups;    // rows2d / wide / ypass: segment log2, warps per engine, engines per item
    int xlg, xNW, xgroups; // xpass
    int64_t k_first[PH_COUNT];   // first work item of this job in each phase
};

struct BatchHeader {
    int njobs;
    int pad0;
    int64_t k_total[PH_COUNT];   // work items per phase
    unsigned* cnt;               // [0, PH_COUNT): work counters; then arrival counters
    int64_t cnt_words;           // words of cnt the clear kernel zeroes
};

constexpr int BATCH_MAX_W = 2048;      // widest image of the rows2d phase
constexpr int BATCH_K2_WARPS = 16;     // threads per row-pass block / 32
constexpr int BATCH_3D_WARPS = 16;     // threads per y / x pass block / 32
constexpr size_t BATCH_3D_SMEM = (size_t)108 << 10;   // dynamic shared memory of a y / x pass block
int batch_colbits_blocks_per_sm();
int batch_rows_blocks_per_sm();
int batch_wide_blocks_per_sm();
int batch_3d_blocks_per_sm();

// Geometry overrides of the batch phases (edt_autotune_batch), 0 = built-in:
// rows2d_lgmin = smallest segment log2 of the rows2d phase (built-in 8, i.e.
// segments of at least 256 columns); y_pos / x_pos = positions per warp the
// y / x pass aims at (built-in 64 / 32).
struct BatchTuning {
    int rows2d_lgmin = 0;
    int y_pos = 0;
    int x_pos = 0;
};
BatchTuning batch_tuning_lookup(int ndim, const int* shape);
void batch_tuning_store(int ndim, const int* shape, const BatchTuning& t);

void batch_row_geometry(int W, int lgmin, int& lg, int& NW, int& groups);
size_t batch_rows_smem();
size_t batch_wide_smem();
// 3-D engine geometry of a line of n positions aiming at `pos` positions per
// warp, and its shared memory per engine (y: H positions; x: W positions)
void batch_line_geometry(int n, int pos, int& lg, int& NW);
size_t batch_ypass_group_bytes(int H, int lg, int NW);
size_t batch_xpass_group_bytes(int W, int lg, int NW);

// Job table of one batch (edt_batch_table.cu).  batch_kind: the job's kind,
// or -1 when it cannot be batched (`why` then says so).  batch_layout: the
// column-pass scratch bytes and counter words a batch needs.  batch_fill: the
// table (jobs ordered by kind, the heaviest first within a kind), with the
// scratch carved from `scratch` and the counters from `cnt` (device
// addresses, at least batch_layout's sizes).  Shapes must have passed
// check_shape and batch_kind.
int batch_kind(const edt_job& j, const char** why);
size_t batch_job_scratch_bytes(const edt_job& j);
void batch_layout(const edt_job* jobs, int n, size_t* scratch_bytes, int64_t* cnt_words);
void batch_fill(const edt_job* jobs, int n, char* scratch, unsigned* cnt, BatchHeader* hdr, BatchJob* tab);

cudaError_t launch_batch_clear(const BatchHeader* hdr, int blocks, cudaStream_t stream);
cudaError_t launch_batch_colbits(const BatchHeader* hdr, const BatchJob* jobs, int blocks,
                                 cudaStream_t stream);
cudaError_t launch_batch_rows2d(const BatchHeader* hdr, const BatchJob* jobs, int blocks, cudaStream_t stream);
cudaError_t launch_batch_wide(const BatchHeader* hdr, const BatchJob* jobs, int blocks, cudaStream_t stream);
cudaError_t launch_batch_ypass3d(const BatchHeader* hdr, const BatchJob* jobs, int blocks, cudaStream_t stream);
cudaError_t launch_batch_xpass3d(const BatchHeader* hdr, const BatchJob* jobs, int blocks, cudaStream_t stream);
cudaError_t set_batch_attributes();
cudaError_t set_batch_row_attributes();
cudaError_t set_batch_3d_attributes();

// Kernel tracing (see edt_trace_enable): trace_begin records the start event
// of a launch on `stream` and returns a slot, trace_end its stop event.
bool trace_on();
int trace_begin(const char* kernel, cudaStream_t stream);
void trace_end(int slot, cudaStream_t stream);

// Enqueue `launch` (a callable returning cudaError_t) bracketed by trace
// events when tracing is on.
template <class F>
cudaError_t traced(const char* kernel, cudaStream_t stream, F&& launch)
{
    if (!trace_on()) return launch();
    const int slot = trace_begin(kernel, stream);
    const cudaError_t e = launch();
    trace_end(slot, stream);
    return e;
}

// Tuned geometry (edt_autotune) per shape class: the upper bound on warps per
// band -- hence the segment length along the lines -- of the 2-D row pass and
// of the 3-D y and x passes; 0 = the built-in rule (16, 8, 32).  The class of
// a shape is the rounded-up log2 of each side.
struct Tuning {
    int rows2d_nw = 0;
    int ypass_nw = 0;
    int xpass_nw = 0;
};
Tuning tuning_lookup(int ndim, const int* shape);
void tuning_store(int ndim, const int* shape, const Tuning& t);

cudaError_t set_2d_attributes();
// SM count of the current device (cached by the per-device set-up; 0 before it)
int device_sm_count();
cudaError_t set_chamfer_attributes();
cudaError_t set_3d_attributes();

}  // namespace edt
