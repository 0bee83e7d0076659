// psolve_program.cuh -- the ordered phases of one outer Bi-CGSTAB iteration
// (Algorithm 1, preconditioned by the Chebyshev iteration of Algorithm 2),
// written once and run two ways:
//   * on the host, V = Launcher: each phase becomes one kernel launch (plain
//     or captured into a CUDA graph);
//   * on the host, V = the persistent kernel's table builder: the phases are
//     recorded as (operation, arguments), and one cooperative launch runs
//     them on every CTA with a grid barrier after each.
// V::go<Op>(cls, side, args, bytes_per_point, half_bytes_per_point, is_update)
// takes one phase; the byte figures feed the host's traffic model.  `iter` (1-based) only selects the first-iteration
// byte figure.
#pragma once
#include <type_traits>

#include "psolve_kernels.cuh"

namespace psolve {

template <class T>
__host__ __device__ constexpr bool is_mixed()
{
    return !std::is_same<T, double>::value;
}

// Residual replacement after the update: r = b - A x for the problems whose
// outer iteration count is a multiple of their rr_every (side 2: the byte
// model counts it only on those iterations).
#pragma nv_exec_check_disable
template <class V>
__host__ __device__ void prog_replace(V &v)
{
    KArgs a{};
    a.skip = SKIP_STOP | SKIP_NOT_RR;
    v.template go<OpReplace>(PSOLVE_K_OTHER, 2, a, 32.0);
}

// Whether a program runner V launches wide sweeps (OpCiSweepW, 128-thread
// CTAs): the per-kernel launcher does; the persistent kernel, whose CTAs all
// have 256 threads, does not.
template <class V, class = void>
struct RunsWide {
    static constexpr bool value = false;
};
template <class V>
struct RunsWide<V, std::void_t<decltype(V::WIDE_SWEEPS)>> {
    static constexpr bool value = V::WIDE_SWEEPS;
};

// One sweep of kind (NEU, UNIT) chosen at run time; `wide`: the launch list
// allows the two-points-per-thread form (FP32/BF16 vectors, whole grid, no
// Neumann face, TMA ring), which computes the same values.
#pragma nv_exec_check_disable
template <class T, class TB, bool BLK, bool WY, class V>
__host__ __device__ void prog_sweep(V &v, int cls, int side, const KArgs &a, double bytes, bool neu, bool unit,
                                    bool wide = false)
{
    constexpr bool U = !is_mixed<T>(); // the scaled-iterate form exists for FP64 vectors
    if constexpr (RunsWide<V>::value && is_mixed<T>() && !BLK) {
        if (wide && !neu) {
            v.template go<OpCiSweepW<T, WY>>(cls, side, a, bytes);
            return;
        }
    }
    if constexpr (U) {
        if (unit && a.k == 2) { // FP64 pipe bound: the form without the y_{k-2} term
            if (neu) v.template go<OpCiSweep<T, TB, BLK, WY, true, true, true>>(cls, side, a, bytes);
            else v.template go<OpCiSweep<T, TB, BLK, WY, false, true, true>>(cls, side, a, bytes);
            return;
        }
    }
    if (neu && unit) v.template go<OpCiSweep<T, TB, BLK, WY, true, U>>(cls, side, a, bytes);
    else if (neu) v.template go<OpCiSweep<T, TB, BLK, WY, true, false>>(cls, side, a, bytes);
    else if (unit) v.template go<OpCiSweep<T, TB, BLK, WY, false, U>>(cls, side, a, bytes);
    else v.template go<OpCiSweep<T, TB, BLK, WY, false, false>>(cls, side, a, bytes);
}

// CI sweep 1 of the mixed-precision forms on the rounded right-hand side b_c
// (OpCiFirstC; two points per thread where the launch list allows it).
#pragma nv_exec_check_disable
template <class T, bool BLK, class V>
__host__ __device__ void prog_sweep1(V &v, int side, const KArgs &a, double bytes, bool neu, bool wide)
{
    if constexpr (RunsWide<V>::value && !BLK) {
        if (wide && !neu) {
            v.template go<OpCiFirstCW<T>>(PSOLVE_K_CI_FIRST, side, a, bytes);
            return;
        }
    }
    v.template go<OpCiFirstC<T, BLK>>(PSOLVE_K_CI_FIRST, side, a, bytes);
}

// Chebyshev sweeps k = 2..d (Algorithm 2 loop).  y_k overwrites y_{k-2}'s
// buffer (read only at the same point), and the last sweep writes `final_role`.
// neu: the grid has Neumann faces (else the sweeps compiled without them run).
// split: sub-units per work unit (KArgs::split).
// With FP64 vectors every sweep stores its iterate scaled (OpCiSweep; the
// last one p^ or r^, divided by Desc::hat); the descriptor's coefficients
// must be those of degree d.
// Sweeps k = 2..d two per pass (OpCiSweepPairW) on a wide launch list; an odd
// last sweep runs alone (OpCiSweepW).  y_1 is in y_a; a pair reads its inputs
// with a halo, so its outputs go to two of the four work vectors y_a..y_d
// that hold neither input (the last sweep writes final_role).
#pragma nv_exec_check_disable
template <class T, class TB, bool WY, class V>
__host__ __device__ void prog_sweeps_paired(V &v, int d, int side, int brole, int final_role, int skip)
{
    const double c = sizeof(T), cb = sizeof(TB);
    const int bufs[4] = {ROLE_YA, ROLE_YB, ROLE_YC, ROLE_YD};
    auto pick = [&](int x0, int x1, int x2) -> int {
        for (int q = 0; q < 4; ++q)
            if (bufs[q] != x0 && bufs[q] != x1 && bufs[q] != x2) return bufs[q];
        return ROLE_YD; // not reached: at most three of the four are excluded
    };
    int cur = ROLE_YA, prev = -1; // y_{k-1}, y_{k-2} (none before sweep 2)
    int k = 2;
    while (k <= d) {
        KArgs a{};
        a.k = k;
        a.skip = skip;
        a.in = cur;
        a.z = prev >= 0 ? prev : ROLE_YB; // unused by sweep 2
        a.b = brole;
        const int cls = (k == 2) ? PSOLVE_K_CI_SWEEP3 : PSOLVE_K_CI_SWEEP4;
        if (k + 1 <= d) {
            a.out = pick(cur, prev, -1);
            a.aux = (k + 1 == d) ? final_role : pick(cur, prev, a.out);
            const double bytes = c + cb + (k >= 3 ? c : 0.0) + 2.0 * c;
            v.template go<OpCiSweepPairW<T, WY>>(cls, side, a, bytes);
            prev = a.out;
            cur = a.aux;
            k += 2;
        } else {
            a.out = final_role;
            const double bytes = c + cb + (k >= 3 ? c : 0.0) + c;
            v.template go<OpCiSweepW<T, WY>>(cls, side, a, bytes);
            k += 1;
        }
    }
}

#pragma nv_exec_check_disable
template <class T, class TB, bool BLK, bool WY, class V>
__host__ __device__ void prog_sweeps(V &v, int d, int side, int brole, int final_role, int skip, bool neu,
                                     int split = 1, bool wide = false)
{
    const double c = sizeof(T), cb = sizeof(TB);
    if constexpr (RunsWide<V>::value && is_mixed<T>() && !BLK) {
        if (wide && !neu) {
            prog_sweeps_paired<T, TB, WY>(v, d, side, brole, final_role, skip);
            return;
        }
    }
    for (int k = 2; k <= d; ++k) {
        KArgs a{};
        a.k = k;
        a.skip = skip;
        a.split = split;
        a.in = (k % 2 == 0) ? ROLE_YA : ROLE_YB;
        a.z = (k % 2 == 0) ? ROLE_YB : ROLE_YA;
        a.out = (k == d) ? final_role : a.z;
        a.b = brole;
        const int cls = (k == 2) ? PSOLVE_K_CI_SWEEP3 : PSOLVE_K_CI_SWEEP4;
        const double bytes = (k == 2) ? c + cb + c : c + cb + c + c;
        prog_sweep<T, TB, BLK, WY>(v, cls, side, a, bytes, neu, !is_mixed<T>(), wide);
    }
}

// One preconditioned outer iteration: direction update + M^-1 p, w = A p^
// with r~.w (alpha), s = r - alpha w + M^-1 s with ||s||^2 (half-step test),
// t = A r^ with t.s, t.t (omega), then x, r with r~.r, r.r (beta, stop test),
// then, when rr, the residual replacement.
#pragma nv_exec_check_disable
template <class T, bool BLK, bool WY, class V>
__host__ __device__ void prog_iteration_cheb(V &v, int d, int iter, bool rr, bool neu, int split = 1,
                                             bool wide = false)
{
    using TB = typename std::conditional<is_mixed<T>(), T, double>::type;
    constexpr bool MIX = is_mixed<T>();
    constexpr bool U = !MIX; // FP64 vectors: y_1 stored scaled when d >= 2 (OpCiFirst)
    const double c = sizeof(T);
    {
        // p side: p_{i-1} = r + beta (p_{i-2} - omega w) and CI sweep 1 on it:
        // fused (FP64, the stencil forms p stencil-wise), or a pointwise pass
        // that also stores p rounded (b_c) and sweep 1 on b_c (mixed)
        KArgs a{};
        a.skip = SKIP_STOP;
        a.in = ROLE_PCUR;
        a.out = (d <= 1) ? ROLE_PH : ROLE_YA;
        const double rd = (iter == 1) ? 8.0 : 24.0;
        if constexpr (MIX) {
            v.template go<OpDirUpdate<T>>(PSOLVE_K_CI_FIRST, 0, a, rd + 8.0 + c);
            prog_sweep1<T, BLK>(v, 0, a, 2.0 * c, neu, wide);
        } else {
            const double bytes = rd + 8.0 + c;
            if (U && d >= 2) v.template go<OpCiFirst<T, BLK, SIDE_P, U>>(PSOLVE_K_CI_FIRST, 0, a, bytes);
            else v.template go<OpCiFirst<T, BLK, SIDE_P>>(PSOLVE_K_CI_FIRST, 0, a, bytes);
        }
    }
    prog_sweeps<T, TB, BLK, WY>(v, d, 0, MIX ? ROLE_BC : ROLE_PCUR, ROLE_PH, SKIP_STOP, neu, split, wide);
    {
        KArgs a{};
        a.skip = SKIP_STOP;
        a.in = ROLE_PH;
        v.template go<OpStencilDot<T>>(PSOLVE_K_STENCIL_DOT, 0, a, c + 16.0);
    }
    {
        // s side: s = r - alpha w with ||s||^2 and CI sweep 1 on it (fused, or
        // two passes as on the p side; sweep 1 is skipped after a passed
        // half-step test, like the sweeps after it)
        KArgs a{};
        a.skip = SKIP_STOP;
        a.in = ROLE_S;
        a.out = (d <= 1) ? ROLE_RH : ROLE_YA;
        if constexpr (MIX) {
            v.template go<OpHalfStep<T>>(PSOLVE_K_CI_FIRST, 0, a, 24.0 + c);
            KArgs b = a;
            b.skip = SKIP_STOP | SKIP_HALF;
            prog_sweep1<T, BLK>(v, 1, b, 2.0 * c, neu, wide);
        } else {
            const double bytes = 24.0 + c;
            if (U && d >= 2) v.template go<OpCiFirst<T, BLK, SIDE_S, U>>(PSOLVE_K_CI_FIRST, 0, a, bytes);
            else v.template go<OpCiFirst<T, BLK, SIDE_S>>(PSOLVE_K_CI_FIRST, 0, a, bytes);
        }
    }
    prog_sweeps<T, TB, BLK, WY>(v, d, 1, MIX ? ROLE_BC : ROLE_S, ROLE_RH, SKIP_STOP | SKIP_HALF, neu, split,
                                wide);
    {
        KArgs a{};
        a.skip = SKIP_STOP | SKIP_HALF;
        a.in = ROLE_RH;
        v.template go<OpStencil2Dot<T>>(PSOLVE_K_STENCIL_2DOT, 1, a, c + 16.0);
    }
    {
        KArgs a{};
        a.skip = SKIP_STOP;
        a.in = ROLE_PH;
        a.aux = ROLE_RH;
        v.template go<OpUpdate<T>>(PSOLVE_K_UPDATE, 0, a, 48.0 + 2 * c, 16.0 + c, 1);
    }
    if (rr) prog_replace(v);
}

// One unpreconditioned outer iteration (M = I).
#pragma nv_exec_check_disable
template <class V>
__host__ __device__ void prog_iteration_none(V &v, int iter, bool rr)
{
    {
        KArgs a{};
        a.skip = SKIP_STOP;
        v.template go<OpPUpdate>(PSOLVE_K_OTHER, 0, a, iter == 1 ? 16.0 : 32.0);
    }
    {
        KArgs a{};
        a.skip = SKIP_STOP;
        a.in = ROLE_P;
        v.template go<OpStencilDot<double>>(PSOLVE_K_STENCIL_DOT, 0, a, 24.0);
    }
    {
        KArgs a{};
        a.skip = SKIP_STOP;
        v.template go<OpSUpdate>(PSOLVE_K_OTHER, 0, a, 24.0);
    }
    {
        KArgs a{};
        a.skip = SKIP_STOP | SKIP_HALF;
        a.in = ROLE_S;
        v.template go<OpStencil2Dot<double>>(PSOLVE_K_STENCIL_2DOT, 1, a, 16.0);
    }
    {
        KArgs a{};
        a.skip = SKIP_STOP;
        a.in = ROLE_P;
        a.aux = ROLE_S;
        v.template go<OpUpdate<double>>(PSOLVE_K_UPDATE, 0, a, 56.0, 24.0, 1);
    }
    if (rr) prog_replace(v);
}

// r0 = b - A x0 (or r0 = b for x0 = 0) with ||b||^2 and ||r0||^2.
#pragma nv_exec_check_disable
template <class V>
__host__ __device__ void prog_init(V &v, bool use_x0)
{
    KArgs a{};
    a.skip = 0;
    if (use_x0) v.template go<OpResidual<true>>(PSOLVE_K_INIT, 0, a, 32.0);
    else v.template go<OpInit0>(PSOLVE_K_INIT, 0, a, 24.0);
}

// ||b - A x||^2 at exit.
#pragma nv_exec_check_disable
template <class V>
__host__ __device__ void prog_true_residual(V &v)
{
    KArgs a{};
    a.skip = 0;
    v.template go<OpResidual<false>>(PSOLVE_K_OTHER, 0, a, 16.0);
}

} // namespace psolve
