// reduce.cuh -- the caller-provided workspace of the fixed-order FP64
// reductions (grid_reduce in fpm_common.cuh): a completion counter at offset
// 0 and per-block partial sums from byte 256.
#pragma once

#include "fpm_common.cuh"

namespace fpm {

// Workspace layout: [0] grid_reduce completion counter, [16] and [32] the
// ticket and completion counters of a persistent sweep, partial sums from
// byte 256 (one slot of 8 doubles per block or per tile ticket).
struct RedWs {
    unsigned *counter;
    double *part;
    unsigned *work;
    unsigned *done;
};

inline fpm_status red_ws(int n, const fpm_grid *grid, void *ws, size_t bytes, const char *who, RedWs &r)
{
    size_t need = 0;
    fpm_reduce_workspace(n, grid, &need);
    if (!ws || bytes < need) return fpm_fail(FPM_ERR_WORKSPACE, "%s: workspace %zu < %zu bytes", who, bytes, need);
    if (((uintptr_t)ws & 15u) != 0) return fpm_fail(FPM_ERR_WORKSPACE, "%s: workspace not 16-B aligned", who);
    r.counter = (unsigned *)ws;
    r.work = (unsigned *)((char *)ws + 16);
    r.done = (unsigned *)((char *)ws + 32);
    r.part = (double *)((char *)ws + 256);
    return FPM_OK;
}

}  // namespace fpm
