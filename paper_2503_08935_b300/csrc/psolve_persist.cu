// psolve_persist.cu -- host side of the persistent (single-launch) solve:
// kernel selection, phase table, launch configuration and the cooperative
// launch.  The kernels are in psolve_persist_kernel.cuh, instantiated one
// precision per translation unit (psolve_persist_{f64,f32,bf16}.cu).
#include "psolve_persist_kernel.cuh"

namespace psolve {

static PersistKernel kernel_for(const Plan &plan)
{
    if (plan.precond == PSOLVE_PC_NONE) return persist_kernel_f64(plan);
    switch (plan.prec) {
    case PSOLVE_FP32: return persist_kernel_f32(plan);
    case PSOLVE_BF16: return persist_kernel_bf16(plan);
    default: return persist_kernel_f64(plan);
    }
}

void persist_table(const Plan &plan, bool use_x0, bool true_res, PersistState *st_host)
{
    kernel_for(plan).table(plan, use_x0, true_res, st_host);
}

psolve_status persist_configure(const Plan &plan, int sms, long long units, int *grid_out)
{
    const PersistKernel k = kernel_for(plan);
    PS_CK(cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, k.smem));
    int occ = 0;
    PS_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k.fn, NTHREADS, k.smem));
    if (occ < 1) {
        set_error("persistent kernel does not fit on an SM");
        return PSOLVE_E_CUDA;
    }
    long long g = (long long)occ * sms;
    if (units < g) g = units;
    if (g < 1) g = 1;
    *grid_out = (int)g;
    return PSOLVE_OK;
}

psolve_status persist_enqueue(cudaStream_t s, const Plan &plan, int grid, const PersistArgs &args)
{
    const PersistKernel k = kernel_for(plan);
    PS_CK(cudaMemsetAsync(&args.st->gs, 0, sizeof(GridSync), s));
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = (size_t)k.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    PersistArgs a = args;
    PS_CK(cudaLaunchKernelEx(&cfg, k.fn, a));
    return PSOLVE_OK;
}

} // namespace psolve
