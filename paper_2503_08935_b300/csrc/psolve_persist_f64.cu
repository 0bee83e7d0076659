// psolve_persist_f64.cu -- the persistent kernels with FP64 Chebyshev vectors
// and the unpreconditioned one (one translation unit per precision, so that
// they compile in parallel).
#include "psolve_persist_kernel.cuh"

namespace psolve {

PersistKernel persist_kernel_f64(const Plan &plan)
{
    if (plan.precond == PSOLVE_PC_NONE) return kernel_of<0, double, false, false>();
    const bool blk = plan.precond != PSOLVE_PC_CHEB;
    return blk ? kernel_cheb<double, true>(plan.exact_bounds) : kernel_cheb<double, false>(plan.exact_bounds);
}

} // namespace psolve
