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

// One phase of the persistent kernel: which operation of the kernel's list
// runs, with which arguments (descs/list are filled in on the device).
struct PhaseRec {
    int32_t kind;
    int32_t pad_;
    KArgs a;
};

// r0 + one outer iteration at the largest degree + the true residual.
constexpr int MAX_PHASES = 2 * MAX_DEGREE + 8;

// Device state of the persistent solve of one context or batch: the barrier
// words and the phase table.  The table is uploaded before each launch, the
// barrier words are reset by the launch's own memset node.
struct PersistState {
    GridSync gs;
    int32_t n_init, n_iter, n_tail, pad_;
    PhaseRec ph[MAX_PHASES];
};

struct PersistArgs {
    const Desc *descs;
    const int32_t *list; // launch list (ListHdr + entries)
    PersistState *st;    // device
    int32_t iters;       // outer iterations at most (each problem also stops at its maxit)
    int32_t n_init, n_iter, n_tail; // phases: [0, n_init) once, the next n_iter per iteration, then n_tail
};

// Fill st_host's phase table for `plan` (r0 from x0 or x0 = 0, the outer
// iteration, the exit true residual when true_res).
void persist_table(const Plan &plan, bool use_x0, bool true_res, PersistState *st_host);
// Set the persistent kernel of `plan` up (shared memory, occupancy) and return
// its grid size: resident CTAs per SM x SMs, at most the list's units.  Call
// outside stream capture.
psolve_status persist_configure(const Plan &plan, int sms, long long units, int *grid_out);
// Enqueue the barrier reset and the cooperative launch on stream s
// (capturable into a CUDA graph).  The phase table must already be on the
// device.
psolve_status persist_enqueue(cudaStream_t s, const Plan &plan, int grid, const PersistArgs &args);

} // namespace psolve
