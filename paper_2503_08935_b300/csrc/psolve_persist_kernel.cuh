// psolve_persist_kernel.cuh -- the whole solve of a launch list as ONE cooperative
// kernel launch: the initial residual, every outer iteration of Algorithm 1
// (with the Chebyshev sweeps of Algorithm 2) and the exit true residual, each
// phase followed by a grid-wide barrier.  The phases are those of the program
// the per-kernel path launches (psolve_program.cuh), recorded by the host into
// a table of (operation, arguments); each phase runs the same engine code
// (engine_body) as that operation's own kernel, and every reduction is summed
// per unit in unit order, so the two paths give bitwise identical results.
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
#pragma once
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
static __device__ bool grid_sync(GridSync *gs, uint32_t &target, int *s_flag,
                                 unsigned long long limit_ns = GRID_WAIT_NS)
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
            if (globaltimer_ns() - t0 > limit_ns) {
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

// Type lists of the operations one persistent kernel can run; a phase's
// `kind` is the index of its operation in the list.
template <class... Ops>
struct TypeList {};

template <class Op, class L>
struct IndexOf;
template <class Op, class... R>
struct IndexOf<Op, TypeList<Op, R...>> {
    static constexpr int value = 0;
};
template <class Op, class H, class... R>
struct IndexOf<Op, TypeList<H, R...>> {
    static constexpr int value = 1 + IndexOf<Op, TypeList<R...>>::value;
};

// The persistent kernels carry one sweep kind, the one with Neumann-face
// handling (with no Neumann face it computes exactly what the sweep compiled
// without it computes); phases recorded with the latter run as the former.
template <class Op>
struct PersistAlias {
    using type = Op;
};
template <class T, class TB, bool BLK, bool WY, bool UNIT, bool K2>
struct PersistAlias<OpCiSweep<T, TB, BLK, WY, false, UNIT, K2>> {
    using type = OpCiSweep<T, TB, BLK, WY, true, UNIT, K2>;
};

template <class L, class Op>
struct Append;
template <class... Ops, class Op>
struct Append<TypeList<Ops...>, Op> {
    using type = TypeList<Ops..., Op>;
};

template <int KIND, class T, bool BLK, bool WY>
struct PersistOps { // Chebyshev-preconditioned iteration
    using TB = typename std::conditional<is_mixed<T>(), T, double>::type;
    using Common = TypeList<OpInit0, OpResidual<true>, OpResidual<false>, OpCiSweep<T, TB, BLK, WY>,
                            OpStencilDot<T>, OpStencil2Dot<T>, OpUpdate<T>, OpReplace>;
    // FP64: CI sweep 1 fused with its right-hand side; sweep 1 and the sweeps
    // before the last one in the scaled-iterate form
    using Fused = typename Append<typename Append<Common, OpCiFirst<T, BLK, SIDE_P>>::type,
                                  OpCiFirst<T, BLK, SIDE_S>>::type;
    using Scaled = typename Append<
        typename Append<typename Append<typename Append<Fused, OpCiSweep<T, TB, BLK, WY, true, true>>::type,
                                        OpCiSweep<T, TB, BLK, WY, true, true, true>>::type,
                        OpCiFirst<T, BLK, SIDE_P, true>>::type,
        OpCiFirst<T, BLK, SIDE_S, true>>::type;
    // mixed precision: the pointwise right-hand sides and sweep 1 on b_c
    using Mixed = typename Append<typename Append<typename Append<Common, OpDirUpdate<T>>::type,
                                                  OpHalfStep<T>>::type,
                                  OpCiFirstC<T, BLK>>::type;
    using List = typename std::conditional<is_mixed<T>(), Mixed, Scaled>::type;
};
template <class T, bool BLK, bool WY>
struct PersistOps<0, T, BLK, WY> { // unpreconditioned iteration
    using List = TypeList<OpInit0, OpResidual<true>, OpResidual<false>, OpPUpdate, OpStencilDot<double>, OpSUpdate,
                          OpStencil2Dot<double>, OpUpdate<double>, OpReplace>;
};

// Runs operation number `kind` of the list.  The phase's arguments come from
// device memory, so each operation is compiled exactly as in its own kernel
// (nothing is specialised on the phase), and runs the same arithmetic.
template <class L>
struct Dispatch;
template <class Op, class... R>
struct Dispatch<TypeList<Op, R...>> {
    static __device__ __forceinline__ void run(int kind, const KArgs &a, EngineShared &sh)
    {
        if (kind == 0) engine_body<Op>(a, sh);
        else if constexpr (sizeof...(R) > 0) Dispatch<TypeList<R...>>::run(kind - 1, a, sh);
    }
};

// Whether every listed problem has stopped.  Read right after a barrier; the
// first phase of an iteration never writes `stop`, so every CTA sees the same
// flags and takes the same decision.
static __device__ bool list_all_stopped(const Desc *descs, const int32_t *list, int *s_all)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const ListHdr hdr = *reinterpret_cast<const ListHdr *>(list);
        const int2 *ent = reinterpret_cast<const int2 *>(list + LIST_HDR_INTS);
        int all = 1;
        for (int e = 0; e < hdr.n && all; ++e)
            if (!ld_flag(&descs[ent[e].x].sc->stop)) all = 0;
        *s_all = all;
    }
    __syncthreads();
    return *s_all != 0;
}

// One phase on every CTA, then the grid barrier; false: abandon the launch.
// The phase's arguments are staged in shared memory (like a kernel's
// parameters, they hold no registers while the operation runs).
template <class L>
__device__ __forceinline__ bool run_phase(const PhaseRec *ph, int i, const Desc *descs, const int32_t *list,
                                          GridSync *gs, KArgs &s_a, int &s_kind, EngineShared &sh,
                                          uint32_t &target, int *s_flag)
{
    __syncthreads(); // the previous phase is done with the ring and with s_a
    if (threadIdx.x == 0) {
        // re-arm the TMA ring (no copies are in flight: every march waits for
        // each plane it issued) and stage this phase's arguments
        for (int b = 0; b < MAX_STAGES; ++b) {
            asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&sh.bars[b])) : "memory");
            mbar_init(&sh.bars[b], 1);
        }
        mbar_init_fence();
        s_a = ph[i].a;
        s_a.descs = descs;
        s_a.list = list;
        s_kind = ph[i].kind;
    }
    sh.seq = 0;
    __syncthreads();
    Dispatch<L>::run(s_kind, s_a, sh);
    if (threadIdx.x == 0 && *sh.s_dead) atomicExch(&gs->err, 2); // a tensor-copy wait gave up
    return grid_sync(gs, target, s_flag);
}

template <int KIND, class T, bool BLK, bool WY>
__global__ void __launch_bounds__(NTHREADS, 4) k_persist(PersistArgs pa)
{
    using L = typename PersistOps<KIND, T, BLK, WY>::List;
    __shared__ double sred[(NTHREADS / 32) * MAX_DOTS];
    __shared__ alignas(8) uint64_t bars[MAX_STAGES];
    __shared__ int s_last, s_dead, s_flag, s_all, s_kind, s_unit;
    __shared__ KArgs s_a;
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    EngineShared sh;
    engine_setup(sh, sred, bars, &s_last, &s_dead, &s_unit, dyn_smem);
    uint32_t target = 0;
    bool ok = true;
    for (int i = 0; i < pa.n_init && ok; ++i)
        ok = run_phase<L>(pa.st->ph, i, pa.descs, pa.list, &pa.st->gs, s_a, s_kind, sh, target, &s_flag);
    for (int it = 1; it <= pa.iters && ok; ++it) {
        if (list_all_stopped(pa.descs, pa.list, &s_all)) break;
        for (int i = 0; i < pa.n_iter && ok; ++i)
            ok = run_phase<L>(pa.st->ph, pa.n_init + i, pa.descs, pa.list, &pa.st->gs, s_a, s_kind, sh, target,
                              &s_flag);
    }
    for (int i = 0; i < pa.n_tail && ok; ++i)
        ok = run_phase<L>(pa.st->ph, pa.n_init + pa.n_iter + i, pa.descs, pa.list, &pa.st->gs, s_a, s_kind, sh,
                          target, &s_flag);
}

// ------------------------------------------------------- host-side helpers --
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

// Records the phases of a program as (operation index, arguments).
template <class L>
struct TableBuilder {
    PhaseRec *out;
    int n = 0;
    template <class Op>
    void go(int, int, KArgs a, double, double = 0.0, int = 0)
    {
        if (n >= MAX_PHASES) return; // cannot happen: degree <= MAX_DEGREE
        out[n].kind = IndexOf<typename PersistAlias<Op>::type, L>::value;
        out[n].pad_ = 0;
        out[n].a = a;
        ++n;
    }
};

template <int KIND, class T, bool BLK, bool WY>
void table_of(const Plan &plan, bool use_x0, bool true_res, PersistState *st)
{
    using L = typename PersistOps<KIND, T, BLK, WY>::List;
    TableBuilder<L> tb{st->ph};
    prog_init(tb, use_x0);
    st->n_init = tb.n;
    if constexpr (KIND == 0) prog_iteration_none(tb, 2, plan.rr_every > 0);
    else prog_iteration_cheb<T, BLK, WY>(tb, plan.degree, 2, plan.rr_every > 0, true,
                                         plan.split); // one sweep kind for every grid
    st->n_iter = tb.n - st->n_init;
    if (true_res) prog_true_residual(tb);
    st->n_tail = tb.n - st->n_init - st->n_iter;
}

struct PersistKernel {
    void (*fn)(PersistArgs) = nullptr;
    int smem = 0;
    void (*table)(const Plan &, bool, bool, PersistState *) = nullptr;
};

template <int KIND, class T, bool BLK, bool WY>
PersistKernel kernel_of()
{
    SmemMax m;
    prog_init(m, false);
    prog_init(m, true);
    if constexpr (KIND == 0) prog_iteration_none(m, 1, true);
    else prog_iteration_cheb<T, BLK, WY>(m, 3, 1, true, true);
    prog_true_residual(m);
    return PersistKernel{k_persist<KIND, T, BLK, WY>, m.bytes, table_of<KIND, T, BLK, WY>};
}

template <class T, bool BLK>
inline PersistKernel kernel_cheb(bool eb)
{
    return eb ? kernel_of<1, T, BLK, false>() : kernel_of<1, T, BLK, true>();
}

// The persistent kernels of one precision (each in its own translation unit).
PersistKernel persist_kernel_f64(const Plan &plan);
PersistKernel persist_kernel_f32(const Plan &plan);
PersistKernel persist_kernel_bf16(const Plan &plan);

} // namespace psolve
