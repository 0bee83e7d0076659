// psolve_tune.cuh -- the slab-depth / stencil-engine autotuner (psolve_tune.cu).
#pragma once
#include "psolve_engine.cuh"

namespace psolve {

struct TuneChoice {
    int zc = 0;         // planes per work unit
    int engine = 0;     // 1: TMA ring, 0: general engine
    double us = 0.0;    // probe time of the choice (microseconds)
    int from_cache = 0; // 1: read from the on-disk cache, not measured here
};

// The choice for P's grid shape and Chebyshev precision on a GPU with `sms`
// SMs: from the cache, else measured on P's bound workspace (whose contents
// it overwrites) with stream s.  Thread-safe.
psolve_status tune_problem(const Problem &P, int sms, cudaStream_t s, TuneChoice *out);

} // namespace psolve
