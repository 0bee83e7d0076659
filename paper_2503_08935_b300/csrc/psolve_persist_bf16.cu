// psolve_persist_bf16.cu -- the persistent kernels with BF16 Chebyshev vectors
// (one translation unit per precision, so that they compile in parallel).
#include "psolve_persist_kernel.cuh"

namespace psolve {

PersistKernel persist_kernel_bf16(const Plan &plan)
{
    const bool blk = plan.precond != PSOLVE_PC_CHEB;
    return blk ? kernel_cheb<__nv_bfloat16, true>(plan.exact_bounds) : kernel_cheb<__nv_bfloat16, false>(plan.exact_bounds);
}

} // namespace psolve
