// psolve_persist.cu -- the whole solve of a launch list as ONE cooperative
// kernel launch: the initial residual, every outer iteration of Algorithm 1
// (with the Chebyshev sweeps of Algorithm 2) and the exit true residual, each
// phase followed by a grid-wide barrier.  The phase order is the same program
// the per-kernel path launches (psolve_program.cuh), and each phase runs the
// same engine code (engine_body) with the same unit-to-CTA assignment, so the
// two paths give bitwise identical results.
//
// Grid barrier.  A monotonically increasing arrival counter in device memory
// (zeroed by a memset node before each launch): barrier number n waits until
// the counter reaches n * gridDim.x.  The wait is bounded (GRID_WAIT_NS of
// wall time from %globaltimer); a CTA that gives up raises the launch's error
// word, every other CTA sees it in its own wait and leaves, and the host
// reports PSOLVE_TIMEOUT.  Co-residency of all CTAs is guaranteed by the
// cooperative launch attribute (the launch fails instead of deadlocking when
// the grid does not fit).
//
// Memory ordering across phases.  Vector loads go through L2 (gld), scalar
// blocks are read with L2 loads or volatile accesses, the barrier is a
// release/acquire pair at GPU scope, and a proxy fence on both sides orders
// the generic-proxy stores of one phase before the tensor copies (async
// proxy) of the next.  The TMA ring's mbarriers are re-initialised at each
// phase because the ring's stage count differs between operations.
#include "psolve_engine.cuh"
#include "psolve_persist.cuh"

namespace psolve {

constexpr unsigned long long GRID_WAIT_NS = 4000000000ull; // 4 s per barrier wait

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u32(uint32_t *p, uint32_t v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// All CTAs of the launch meet here.  Returns false when the launch is being
// abandoned (this CTA or another gave up waiting).
__device__ bool grid_sync(GridSync *gs, uint32_t &target, int *s_flag)
{
    fence_proxy_async_global();
    __syncthreads();
    target += gridDim.x;
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        red_release_add_u32(&gs->count, 1u);
        const unsigned long long t0 = globaltimer_ns();
        unsigned ns = 32;
        while ((int)(ld_acquire_u32(&gs->count) - target) < 0) {
            if (*(volatile int32_t *)&gs->err) {
                ok = 0;
                break;
            }
            if (globaltimer_ns() - t0 > GRID_WAIT_NS) {
                atomicExch(&gs->err, 1);
                ok = 0;
                break;
            }
            __nanosleep(ns);
            if (ns < 512) ns *= 2;
        }
        __threadfence();
        fence_proxy_async_global();
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

// Re-arm the TMA ring for the next phase (no copies are in flight: every
// march waits for each plane it issued).
__device__ __forceinline__ void engine_rearm(EngineShared &sh)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int b = 0; b < MAX_STAGES; ++b) {
            asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&sh.bars[b])) : "memory");
            mbar_init(&sh.bars[b], 1);
        }
        mbar_init_fence();
    }
    sh.seq = 0;
    __syncthreads();
}

// One phase, compiled as a function of its own so that each operation gets
// the full register budget instead of sharing it with the state the kernel
// keeps across phases (the call costs nothing next to a phase).
template <class Op>
__device__ __noinline__ void engine_phase(const KArgs &a, EngineShared &sh)
{
    engine_body<Op>(a, sh);
}

// The device-side visitor of the phase programs.
struct PhaseRunner {
    const PersistArgs *pa;
    EngineShared *sh;
    int *s_flag;
    uint32_t target;
    bool ok;

    template <class Op>
    __device__ __forceinline__ void go(int, int, KArgs a, double, double = 0.0, int = 0)
    {
        if (!ok) return;
        a.descs = pa->descs;
        a.list = pa->list;
        engine_rearm(*sh);
        engine_phase<Op>(a, *sh);
        if (threadIdx.x == 0 && *sh->s_dead) atomicExch(&pa->gs->err, 2); // a tensor-copy wait gave up
        ok = grid_sync(pa->gs, target, s_flag);
    }
};

// Whether every listed problem has stopped.  Read right after a barrier; the
// first phase of an iteration never writes `stop`, so every CTA sees the same
// flags and takes the same decision.
__device__ bool list_all_stopped(const PersistArgs &pa, int *s_all)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const ListHdr hdr = *reinterpret_cast<const ListHdr *>(pa.list);
        const int2 *ent = reinterpret_cast<const int2 *>(pa.list + 2);
        int all = 1;
        for (int e = 0; e < hdr.n && all; ++e)
            if (!ld_flag(&pa.descs[ent[e].x].sc->stop)) all = 0;
        *s_all = all;
    }
    __syncthreads();
    return *s_all != 0;
}

template <int KIND, class T, bool BLK, bool WY>
__global__ void __launch_bounds__(NTHREADS, 4) k_persist(PersistArgs pa)
{
    __shared__ double sred[(NTHREADS / 32) * MAX_DOTS];
    __shared__ alignas(8) uint64_t bars[MAX_STAGES];
    __shared__ int s_last, s_dead, s_flag, s_all;
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    EngineShared sh;
    engine_setup(sh, sred, bars, &s_last, &s_dead, dyn_smem);
    PhaseRunner v{&pa, &sh, &s_flag, 0u, true};
    if (pa.init) prog_init(v, pa.use_x0 != 0);
    for (int it = 1; it <= pa.iters && v.ok; ++it) {
        if (list_all_stopped(pa, &s_all)) break;
        if constexpr (KIND == 0) prog_iteration_none(v, it);
        else prog_iteration_cheb<T, BLK, WY>(v, pa.degree, it);
    }
    if (pa.true_res) prog_true_residual(v);
}

// ------------------------------------------------------------------ host --
namespace {

// Largest dynamic shared memory over the operations of a program.
struct SmemMax {
    int bytes = 0;
    template <class Op>
    void go(int, int, KArgs, double, double = 0.0, int = 0)
    {
        const int b = engine_dyn_smem<Op>();
        if (b > bytes) bytes = b;
    }
};

struct PersistKernel {
    void (*fn)(PersistArgs) = nullptr;
    int smem = 0;
};

template <int KIND, class T, bool BLK, bool WY>
PersistKernel kernel_of()
{
    SmemMax m;
    prog_init(m, false);
    prog_init(m, true);
    if constexpr (KIND == 0) prog_iteration_none(m, 1);
    else prog_iteration_cheb<T, BLK, WY>(m, 3, 1);
    prog_true_residual(m);
    return PersistKernel{k_persist<KIND, T, BLK, WY>, m.bytes};
}

template <class T, bool BLK>
PersistKernel kernel_cheb(bool eb)
{
    return eb ? kernel_of<1, T, BLK, false>() : kernel_of<1, T, BLK, true>();
}

PersistKernel kernel_for(const Plan &plan)
{
    if (plan.precond == PSOLVE_PC_NONE) return kernel_of<0, double, false, false>();
    const bool blk = plan.precond != PSOLVE_PC_CHEB;
    switch (plan.prec) {
    case PSOLVE_FP32: return blk ? kernel_cheb<float, true>(plan.exact_bounds) : kernel_cheb<float, false>(plan.exact_bounds);
    case PSOLVE_BF16:
        return blk ? kernel_cheb<__nv_bfloat16, true>(plan.exact_bounds)
                   : kernel_cheb<__nv_bfloat16, false>(plan.exact_bounds);
    default: return blk ? kernel_cheb<double, true>(plan.exact_bounds) : kernel_cheb<double, false>(plan.exact_bounds);
    }
}

} // namespace

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
    PS_CK(cudaMemsetAsync(args.gs, 0, sizeof(GridSync), s));
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
