// psolve_persist_f32.cu -- the persistent kernels with FP32 Chebyshev vectors
// (one translation unit per precision, so that they compile in parallel).
#include "psolve_persist_kernel.cuh"

namespace psolve {

PersistKernel persist_kernel_f32(const Plan &plan)
{
    const bool blk = plan.precond != PSOLVE_PC_CHEB;
    return blk ? kernel_cheb<float, true>(plan.exact_bounds) : kernel_cheb<float, false>(plan.exact_bounds);
}

} // namespace psolve
