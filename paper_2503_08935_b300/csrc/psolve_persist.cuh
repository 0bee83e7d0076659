// psolve_persist.cuh -- host interface of the persistent (single-launch)
// solve; the kernel itself is in psolve_persist.cu.
#pragma once
#include "psolve_engine.cuh"

namespace psolve {

// Grid-barrier state of one persistent launch (zeroed before each launch).
struct GridSync {
    uint32_t count; // barrier arrivals so far
    int32_t err;    // nonzero: a wait gave up (1 grid barrier, 2 tensor copy)
    int32_t pad_[2];
};

struct PersistArgs {
    const Desc *descs;
    const int32_t *list; // launch list (ListHdr + entries)
    GridSync *gs;
    int32_t degree;      // Chebyshev degree d
    int32_t iters;       // outer iterations at most (each problem also stops at its maxit)
    int32_t init;        // 1: compute r0 and the norms first
    int32_t use_x0;      // init from x0 (r0 = b - A x0) instead of x0 = 0
    int32_t true_res;    // 1: ||b - A x||^2 after the loop
    int32_t pad_;
};

// Set the persistent kernel of `plan` up (shared memory, occupancy) and return
// its grid size: resident CTAs per SM x SMs, at most the list's units.  Call
// outside stream capture.
psolve_status persist_configure(const Plan &plan, int sms, long long units, int *grid_out);
// Enqueue the barrier reset and the cooperative launch on stream s
// (capturable into a CUDA graph).
psolve_status persist_enqueue(cudaStream_t s, const Plan &plan, int grid, const PersistArgs &args);

} // namespace psolve
