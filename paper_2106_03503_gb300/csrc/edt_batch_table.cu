// Job table of a batch (host side): which persistent kernel covers each job,
// the geometry of its engines, its share of the column-pass scratch and of
// the counters, and where its work items start in every phase.  Kept apart
// from the plan code so that the kernel emulation in the tests builds exactly
// the tables the library builds.
#include <algorithm>
#include <cstring>
#include <vector>

#include "edt_engine.cuh"
#include "edt_internal.h"

namespace edt {

static size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

static ColGeom job_geom(const edt_job& j)
{
    return j.ndim == 2 ? col_geom(j.shape[0], j.shape[1], true)
                       : col_geom(j.shape[0], (int64_t)j.shape[1] * j.shape[2], true);
}

// Column-pass scratch of one job: C, U ([nb][cols]) and GFL, GAB ([nG][cols]).
static size_t geom_scratch_bytes(const ColGeom& g)
{
    const size_t c = (size_t)g.cols * 4;
    return 2 * al256((size_t)g.nb * c) + 2 * al256((size_t)g.nG * c);
}

size_t batch_job_scratch_bytes(const edt_job& j) { return geom_scratch_bytes(job_geom(j)); }

// The y / x positions per warp the 3-D passes may be tuned to: a 3-D job is
// batched only if every candidate fits the block's shared memory.
static const int kPosCandidates[] = {32, 64, 128};

int batch_kind(const edt_job& j, const char** why)
{
    if (j.ndim == 2) return j.shape[1] <= BATCH_MAX_W ? BATCH_2D : BATCH_2D_WIDE;
    if (j.ndim != 3) {
        if (why) *why = "ndim must be 2 or 3";
        return -1;
    }
    const int H = j.shape[1], W = j.shape[2];
    for (int pos : kPosCandidates) {
        int lg, NW;
        batch_line_geometry(H, pos, lg, NW);
        if (batch_ypass_group_bytes(H, lg, NW) > BATCH_3D_SMEM) {
            if (why) *why = "3-D height too large for the batched y pass (about 1150 at most)";
            return -1;
        }
        batch_line_geometry(W, pos, lg, NW);
        if (batch_xpass_group_bytes(W, lg, NW) > BATCH_3D_SMEM) {
            if (why) *why = "3-D row width too large for the batched x pass (about 670 at most)";
            return -1;
        }
    }
    return BATCH_3D;
}

void batch_layout(const edt_job* jobs, int n, size_t* scratch_bytes, int64_t* cnt_words)
{
    size_t sb = 0;
    int64_t cw = PH_COUNT;
    for (int i = 0; i < n; ++i) {
        const ColGeom g = job_geom(jobs[i]);
        sb += geom_scratch_bytes(g);
        cw += g.ntiles;
    }
    *scratch_bytes = sb;
    *cnt_words = cw;
}

// Work of a job for ordering inside its kind: pixels per row pass item.
static int64_t job_weight(const edt_job& j)
{
    return j.ndim == 2 ? (int64_t)j.shape[1] : (int64_t)j.shape[1] * j.shape[2];
}

void batch_fill(const edt_job* jobs, int n, char* scratch, unsigned* cnt, BatchHeader* hdr, BatchJob* tab)
{
    std::vector<int> order(n);
    std::vector<int> kind(n);
    for (int i = 0; i < n; ++i) {
        order[i] = i;
        kind[i] = batch_kind(jobs[i], nullptr);
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        if (kind[a] != kind[c]) return kind[a] < kind[c];
        return job_weight(jobs[a]) > job_weight(jobs[c]);
    });
    size_t off = 0;
    int64_t cnt_off = PH_COUNT;
    int64_t k[PH_COUNT] = {0, 0, 0, 0, 0};
    for (int t = 0; t < n; ++t) {
        const edt_job& j = jobs[order[t]];
        BatchJob& J = tab[t];
        memset(&J, 0, sizeof(J));
        J.kind = kind[order[t]];
        J.mask = j.mask;
        J.D = j.D;
        J.F = j.F;
        J.dist = j.dist;
        J.mode = j.mode;
        J.Dz = j.ndim == 3 ? j.shape[0] : 1;
        J.H = j.ndim == 3 ? j.shape[1] : j.shape[0];
        J.W = j.ndim == 3 ? j.shape[2] : j.shape[1];
        J.g = job_geom(j);
        J.vec = (J.g.cols % 16 == 0) && ((reinterpret_cast<uintptr_t>(j.mask) & 15) == 0);
        const size_t c = (size_t)J.g.cols * 4;
        char* base = scratch + off;
        J.s.C = reinterpret_cast<uint32_t*>(base);
        J.s.U = reinterpret_cast<uint32_t*>(base + al256((size_t)J.g.nb * c));
        J.s.GFL = reinterpret_cast<uint32_t*>(base + 2 * al256((size_t)J.g.nb * c));
        J.s.GAB = reinterpret_cast<uint32_t*>(base + 2 * al256((size_t)J.g.nb * c) + al256((size_t)J.g.nG * c));
        J.s.cnt = cnt + cnt_off;
        J.s.gs = J.g.gs;
        off += geom_scratch_bytes(J.g);
        cnt_off += J.g.ntiles;
        for (int ph = 0; ph < PH_COUNT; ++ph) J.k_first[ph] = k[ph];
        k[PH_COL] += J.g.ntiles * (int64_t)J.g.nG;
        const BatchTuning tu = batch_tuning_lookup(j.ndim, j.shape);
        if (J.kind == BATCH_2D) {
            batch_row_geometry(J.W, tu.rows2d_lgmin, J.lg, J.NW, J.groups);
            k[PH_ROWS] += (J.g.nb + J.groups - 1) / J.groups;
        } else if (J.kind == BATCH_2D_WIDE) {
            J.lg = band_seg_log2(J.W, BATCH_K2_WARPS);
            J.NW = (J.W + (1 << J.lg) - 1) >> J.lg;
            J.groups = 1;
            k[PH_WIDE] += J.g.nb;
        } else {
            const int ypos = tu.y_pos > 0 ? tu.y_pos : 64, xpos = tu.x_pos > 0 ? tu.x_pos : 32;
            batch_line_geometry(J.H, ypos, J.lg, J.NW);
            J.groups = std::max<int>(1, std::min<int>(BATCH_3D_WARPS / J.NW,
                                                      (int)(BATCH_3D_SMEM / batch_ypass_group_bytes(J.H, J.lg, J.NW))));
            batch_line_geometry(J.W, xpos, J.xlg, J.xNW);
            J.xgroups = std::max<int>(1, std::min<int>(BATCH_3D_WARPS / J.xNW,
                                                       (int)(BATCH_3D_SMEM / batch_xpass_group_bytes(J.W, J.xlg, J.xNW))));
            const int64_t yunits = (int64_t)J.Dz * ((J.W + 31) / 32);
            const int64_t xunits = ((int64_t)J.Dz * J.H + 31) / 32;
            k[PH_Y] += (yunits + J.groups - 1) / J.groups;
            k[PH_X] += (xunits + J.xgroups - 1) / J.xgroups;
        }
    }
    hdr->njobs = n;
    hdr->pad0 = 0;
    for (int ph = 0; ph < PH_COUNT; ++ph) hdr->k_total[ph] = k[ph];
    hdr->cnt = cnt;
    hdr->cnt_words = cnt_off;
}

}  // namespace edt
