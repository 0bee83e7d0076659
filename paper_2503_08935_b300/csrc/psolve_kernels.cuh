// psolve_kernels.cuh -- CUDA kernels of the Bi-CGSTAB / Chebyshev hot path
// (sm_103a).  No tensor cores: the 7-point operator is a streaming stencil,
// bound by HBM bandwidth.
//
// Engine.  A CTA of TILE_X x TILE_Y threads owns an xy tile; each thread owns
// one z column and marches along z keeping u(k-1), u(k), u(k+1) in registers.
// The x/y neighbours of plane k come from a shared-memory copy of the plane
// (tile plus a one-cell halo, double-buffered), so every input value is read
// from HBM once per sweep; the next planes (own column, halo and pointwise
// operands) are prefetched into registers one step ahead.  Zero Dirichlet
// ghosts (Eq. 4) are zero-filled halo cells; the block-restricted operator
// R_s A R_s^T of Eq. 14 zeroes neighbours across block faces.
//
// Work is split into units (tile x z-chunk); a launch covers every unit of
// every problem in the launch list, each CTA taking one contiguous range.
// Fused dot products are summed per unit (warp shuffle -> shared memory ->
// one partial per unit), and the CTA that completes a problem's last unit
// (atomic ticket) adds that problem's partials in unit order and updates its
// scalars (alpha, omega, beta, convergence flags) on the device.  The result
// is deterministic and independent of the launch size and batch mix.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "psolve_types.cuh"

namespace psolve {

// ------------------------------------------------------------------------
// Storage types of the Chebyshev vectors and their arithmetic type.
// ------------------------------------------------------------------------
template <class T> struct Elem;
template <> struct Elem<double> {
    using C = double;
    static __device__ __forceinline__ double ld(const void *p, int i) { return __ldg((const double *)p + i); }
    static __device__ __forceinline__ void st(void *p, int i, double v) { ((double *)p)[i] = v; }
    static __device__ __forceinline__ double round(double v) { return v; }
};
template <> struct Elem<float> {
    using C = float;
    static __device__ __forceinline__ float ld(const void *p, int i) { return __ldg((const float *)p + i); }
    static __device__ __forceinline__ void st(void *p, int i, float v) { ((float *)p)[i] = v; }
    static __device__ __forceinline__ float round(double v) { return (float)v; }
};
template <> struct Elem<__nv_bfloat16> {
    using C = float;
    static __device__ __forceinline__ float ld(const void *p, int i)
    {
        return __bfloat162float(__ldg((const __nv_bfloat16 *)p + i));
    }
    static __device__ __forceinline__ void st(void *p, int i, float v)
    {
        ((__nv_bfloat16 *)p)[i] = __float2bfloat16_rn(v);
    }
    static __device__ __forceinline__ float round(double v)
    {
        return __bfloat162float(__float2bfloat16_rn((float)v));
    }
};

// ------------------------------------------------------------------------
// Deterministic reductions.
// ------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
    // xor butterfly: every lane ends with the same, order-fixed value
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums v over the CTA; the result is valid in thread 0.  All threads call.
template <int ND>
__device__ __forceinline__ void block_sum(double (&v)[ND], double *sred)
{
    constexpr int NW = NTHREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < ND; ++j) v[j] = warp_sum(v[j]);
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < ND; ++j) sred[warp * ND + j] = v[j];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int j = 0; j < ND; ++j) v[j] = warp_sum(lane < NW ? sred[lane * ND + j] : 0.0);
    }
    __syncthreads();
}

__device__ __forceinline__ int ld_flag(const int32_t *p) { return __ldcg(p); }
__device__ __forceinline__ double ld_scal(const double *p) { return __ldcg(p); }

__device__ __forceinline__ int resolve_role(int role, int iter)
{
    if (role == ROLE_PCUR) return ROLE_P + (iter & 1);
    if (role == ROLE_POLD) return ROLE_P + 1 - (iter & 1);
    return role;
}

// ------------------------------------------------------------------------
// Scalar updates done once per problem by the last CTA of a reduction.
// Status codes match psolve_status.
// ------------------------------------------------------------------------
enum Epi {
    EPI_NONE = 0,
    EPI_INIT0,   // v0 = ||b||^2                        (x0 = 0: r = b, r~ = b)
    EPI_INITX0,  // v0 = ||b||^2, v1 = ||r0||^2          (r~ = r0)
    EPI_ALPHA,   // v0 = r~ . w        -> alpha = rho / v0           (Alg. 1)
    EPI_SNORM,   // v0 = ||s||^2       -> half-step test             (Alg. 1)
    EPI_OMEGA,   // v0 = t . s, v1 = t . t -> omega = v0 / v1       (Alg. 1)
    EPI_UPDATE,  // v0 = r~ . r, v1 = ||r||^2 -> test, beta, rho     (Alg. 1)
    EPI_TRUE,    // v0 = ||b - A x||^2
    EPI_RAW      // store v in red[]
};

constexpr int ST_OK = 0, ST_NOT_CONVERGED = 4, ST_BREAKDOWN = 5, ST_NONFINITE = 6;

__device__ __forceinline__ void stop_with(Scal *sc, int status)
{
    sc->status = status;
    sc->stop = 1;
}

template <int EPI, int ND>
__device__ void epilogue(const Desc &D, Scal *sc, const double (&v)[ND])
{
    if constexpr (EPI == EPI_INIT0 || EPI == EPI_INITX0) {
        const double nb2 = v[0];
        const double rr = (EPI == EPI_INITX0) ? v[ND - 1] : v[0];
        sc->nb2 = nb2;
        sc->rr = rr;
        sc->rho = rr; // r~ = r0
        sc->thr2 = D.rtol * D.rtol * nb2;
        sc->iter = 0;
        sc->first = 1;
        sc->half = 0;
        sc->half_exit = 0;
        sc->zero_x = 0;
        sc->maxit = D.maxit;
        sc->alpha = sc->omega = sc->beta = 0.0;
        sc->ss = 0.0;
        sc->stop = 0;
        sc->status = ST_NOT_CONVERGED;
        if (!isfinite(nb2) || !isfinite(rr)) {
            stop_with(sc, ST_NONFINITE);
        } else if (nb2 == 0.0) { // b = 0: x = 0 is the solution
            sc->rr = 0.0;
            sc->zero_x = (EPI == EPI_INITX0);
            stop_with(sc, ST_OK);
        } else if (rr <= sc->thr2) {
            stop_with(sc, ST_OK);
        } else if (D.maxit <= 0) {
            stop_with(sc, ST_NOT_CONVERGED);
        }
    } else if constexpr (EPI == EPI_ALPHA) {
        const double sig = v[0];
        sc->red[0] = sig;
        if (!isfinite(sig)) stop_with(sc, ST_NONFINITE);
        else if (sig == 0.0) stop_with(sc, ST_BREAKDOWN);
        else sc->alpha = sc->rho / sig;
    } else if constexpr (EPI == EPI_SNORM) {
        const double ss = v[0];
        sc->ss = ss;
        sc->half = 0;
        if (!isfinite(ss)) stop_with(sc, ST_NONFINITE);
        else if (D.half_check && ss <= sc->thr2) sc->half = 1;
    } else if constexpr (EPI == EPI_OMEGA) {
        const double ts = v[0], tt = v[1];
        if (!isfinite(ts) || !isfinite(tt)) stop_with(sc, ST_NONFINITE);
        else if (tt == 0.0) stop_with(sc, ST_BREAKDOWN);
        else {
            const double om = ts / tt;
            sc->omega = om;
            if (om == 0.0) stop_with(sc, ST_BREAKDOWN);
        }
    } else if constexpr (EPI == EPI_UPDATE) {
        sc->iter += 1;
        if (sc->half) { // x += alpha p^ was the whole update
            sc->rr = sc->ss;
            sc->half_exit = 1;
            stop_with(sc, ST_OK);
        } else {
            const double rho_new = v[0], rr = v[1];
            sc->rr = rr;
            if (!isfinite(rr) || !isfinite(rho_new)) stop_with(sc, ST_NONFINITE);
            else if (rr <= sc->thr2) stop_with(sc, ST_OK);
            else if (rho_new == 0.0) stop_with(sc, ST_BREAKDOWN);
            else {
                sc->beta = (rho_new / sc->rho) * (sc->alpha / sc->omega);
                sc->rho = rho_new;
                sc->first = 0;
                if (sc->iter >= sc->maxit) stop_with(sc, ST_NOT_CONVERGED);
            }
        }
    } else if constexpr (EPI == EPI_TRUE) {
        sc->true_rr = v[0];
    } else if constexpr (EPI == EPI_RAW) {
#pragma unroll
        for (int j = 0; j < ND; ++j) sc->red[j] = v[j];
    }
}

// ------------------------------------------------------------------------
// Per-unit partial flush.
// ------------------------------------------------------------------------
template <int ND>
__device__ __forceinline__ void flush_unit(double (&acc)[ND], double *sred, double *partials, int unit)
{
    block_sum<ND>(acc, sred);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < ND; ++j) partials[unit * MAX_DOTS + j] = acc[j];
    }
#pragma unroll
    for (int j = 0; j < ND; ++j) acc[j] = 0.0;
}

// ------------------------------------------------------------------------
// Stencil march over chunks [c0, c1) of one tile.
// Op provides: types C (arithmetic), U (own-column value), PW (pointwise
// operands); ND; BLOCKED; U load(idx); C sv(U); PW pw(bool, idx);
// void emit(idx, C au, U uc, PW, acc).
// ------------------------------------------------------------------------
template <class Op>
__device__ __forceinline__ void march_stencil(Op &op, const Desc &D, int tile, int c0, int c1,
                                              typename Op::C *sp, double *sred)
{
    using C = typename Op::C;
    using U = typename Op::U;
    using PW = typename Op::PW;
    constexpr int ND = Op::ND;
    constexpr int NDA = ND > 0 ? ND : 1;
    constexpr int SW = TILE_X + 2;
    constexpr int SPL = SW * (TILE_Y + 2);

    const int nx = D.nx, ny = D.ny, nz = D.nz, zc = D.zc;
    const int plane = nx * ny;
    const int tid = threadIdx.x, tx = tid % TILE_X, ty = tid / TILE_X;
    const int i0 = (tile % D.tiles_x) * TILE_X, j0 = (tile / D.tiles_x) * TILE_Y;
    const int i = i0 + tx, j = j0 + ty;
    const bool in = (i < nx) && (j < ny);
    const int col = in ? j * nx + i : 0;

    // halo cell owned by this thread (rows above/below, columns left/right)
    int hs = -1, hi = 0, hj = 0;
    if (tid < TILE_X) {
        hs = tid + 1; hi = i0 + tid; hj = j0 - 1;
    } else if (tid < 2 * TILE_X) {
        hs = (TILE_Y + 1) * SW + (tid - TILE_X) + 1; hi = i0 + tid - TILE_X; hj = j0 + TILE_Y;
    } else if (tid < 2 * TILE_X + TILE_Y) {
        const int r = tid - 2 * TILE_X;
        hs = (r + 1) * SW; hi = i0 - 1; hj = j0 + r;
    } else if (tid < 2 * TILE_X + 2 * TILE_Y) {
        const int r = tid - 2 * TILE_X - TILE_Y;
        hs = (r + 1) * SW + TILE_X + 1; hi = i0 + TILE_X; hj = j0 + r;
    }
    const bool hv = hs >= 0 && hi >= 0 && hi < nx && hj >= 0 && hj < ny;
    const int hcol = hv ? hj * nx + hi : 0;
    const int me = (ty + 1) * SW + tx + 1;

    bool okw = true, oke = true, oks = true, okn = true;
    if constexpr (Op::BLOCKED) {
        okw = (i % D.bx) != 0;
        oke = (i % D.bx) != D.bx - 1;
        oks = (j % D.by) != 0;
        okn = (j % D.by) != D.by - 1;
    }
    const C cx = (C)D.cx, cy = (C)D.cy, cz = (C)D.cz, cc = (C)D.cc;

    const int kb = c0 * zc;
    const int ke = min(nz, c1 * zc);

    __syncthreads(); // the previous run's readers of sp are done
    U um = (in && kb >= 1) ? op.load(col + (kb - 1) * plane) : U(0);
    U uc = in ? op.load(col + kb * plane) : U(0);
    U up = (in && kb + 1 < nz) ? op.load(col + (kb + 1) * plane) : U(0);
    C hn = (hv && kb + 1 < nz) ? op.sv(op.load(hcol + (kb + 1) * plane)) : C(0);
    sp[me] = op.sv(uc);
    if (hs >= 0) sp[hs] = hv ? op.sv(op.load(hcol + kb * plane)) : C(0);
    PW pw = op.pw(in, col + kb * plane);

    int kk = 0;
    if constexpr (Op::BLOCKED) kk = kb % D.bz;
    double acc[NDA];
#pragma unroll
    for (int q = 0; q < NDA; ++q) acc[q] = 0.0;
    int unit = tile * D.nzc + c0;
    int cend = min(nz, (c0 + 1) * zc);
    int buf = 0;

    for (int k = kb; k < ke; ++k) {
        // prefetch: own column and halo of plane k+2, pointwise operands of plane k+1
        const U upp = (in && k + 2 < nz) ? op.load(col + (k + 2) * plane) : U(0);
        const C hnn = (hv && k + 2 < nz) ? op.sv(op.load(hcol + (k + 2) * plane)) : C(0);
        const PW pwn = op.pw(in && k + 1 < ke, col + (k + 1) * plane);
        __syncthreads();
        const C *s = sp + buf * SPL;
        if (in) {
            C w = s[me - 1], e = s[me + 1], so = s[me - SW], no = s[me + SW];
            C dn = op.sv(um), un = op.sv(up);
            if constexpr (Op::BLOCKED) {
                if (!okw) w = C(0);
                if (!oke) e = C(0);
                if (!oks) so = C(0);
                if (!okn) no = C(0);
                if (kk == 0) dn = C(0);
                if (kk == D.bz - 1) un = C(0);
            }
            const C au = cc * op.sv(uc) - cx * (w + e) - cy * (so + no) - cz * (dn + un);
            op.emit(col + k * plane, au, uc, pw, acc);
        }
        C *sn = sp + (buf ^ 1) * SPL;
        sn[me] = op.sv(up);
        if (hs >= 0) sn[hs] = hn;
        um = uc;
        uc = up;
        up = upp;
        hn = hnn;
        pw = pwn;
        buf ^= 1;
        if constexpr (Op::BLOCKED) {
            if (++kk == D.bz) kk = 0;
        }
        if constexpr (ND > 0) {
            if (k + 1 == cend) {
                flush_unit<ND>(acc, sred, D.partials, unit);
                ++unit;
                cend = min(nz, cend + zc);
            }
        }
    }
}

// Pointwise march (no stencil) over chunks [c0, c1) of one tile.
template <class Op>
__device__ __forceinline__ void march_point(Op &op, const Desc &D, int tile, int c0, int c1, double *sred)
{
    constexpr int ND = Op::ND;
    constexpr int NDA = ND > 0 ? ND : 1;
    const int nx = D.nx, ny = D.ny, nz = D.nz, zc = D.zc;
    const int plane = nx * ny;
    const int tid = threadIdx.x, tx = tid % TILE_X, ty = tid / TILE_X;
    const int i = (tile % D.tiles_x) * TILE_X + tx, j = (tile / D.tiles_x) * TILE_Y + ty;
    const bool in = (i < nx) && (j < ny);
    const int col = in ? j * nx + i : 0;
    const int kb = c0 * zc;
    const int ke = min(nz, c1 * zc);
    double acc[NDA];
#pragma unroll
    for (int q = 0; q < NDA; ++q) acc[q] = 0.0;
    int unit = tile * D.nzc + c0;
    int cend = min(nz, (c0 + 1) * zc);
    for (int k = kb; k < ke; ++k) {
        if (in) op.emit(col + k * plane, acc);
        if constexpr (ND > 0) {
            if (k + 1 == cend) {
                flush_unit<ND>(acc, sred, D.partials, unit);
                ++unit;
                cend = min(nz, cend + zc);
            }
        }
    }
}

// ------------------------------------------------------------------------
// The generic kernel: walk this CTA's unit range over the launch list.
// ------------------------------------------------------------------------
template <class Op>
__global__ void __launch_bounds__(NTHREADS, 4) k_engine(KArgs a)
{
    using C = typename Op::C;
    constexpr int SPL = (TILE_X + 2) * (TILE_Y + 2);
    __shared__ C sp[Op::STENCIL ? 2 * SPL : 1];
    __shared__ double sred[(NTHREADS / 32) * MAX_DOTS];
    __shared__ int s_last;

    const ListHdr hdr = *reinterpret_cast<const ListHdr *>(a.list);
    const int2 *ent = reinterpret_cast<const int2 *>(a.list + 2);
    const long long total = hdr.total;
    int u0 = (int)(total * blockIdx.x / gridDim.x);
    const int u1 = (int)(total * (blockIdx.x + 1) / gridDim.x);
    if (u0 >= u1) return;

    int lo = 0, hi = hdr.n - 1; // last entry whose first unit <= u0
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ent[mid].y <= u0) lo = mid;
        else hi = mid - 1;
    }
    for (int e = lo; e < hdr.n && u0 < u1; ++e) {
        const int2 en = ent[e];
        const Desc &D = a.descs[en.x];
        const int units = D.units;
        const int pu0 = u0 - en.y;
        const int pu1 = min(u1 - en.y, units);
        u0 = en.y + pu1;
        if (pu0 >= pu1) continue;
        Scal *sc = D.sc;
        if ((a.skip & SKIP_STOP) && ld_flag(&sc->stop)) continue;
        if ((a.skip & SKIP_HALF) && ld_flag(&sc->half)) continue;

        Op op(D, a, sc);
        const int nzc = D.nzc;
        for (int pu = pu0; pu < pu1;) {
            const int tile = pu / nzc;
            const int c0 = pu - tile * nzc;
            const int run_end = min(pu1, (tile + 1) * nzc);
            const int c1 = c0 + (run_end - pu);
            if constexpr (Op::STENCIL) march_stencil<Op>(op, D, tile, c0, c1, sp, sred);
            else march_point<Op>(op, D, tile, c0, c1, sred);
            pu = run_end;
        }
        if constexpr (Op::ND > 0) {
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                const unsigned n = (unsigned)(pu1 - pu0);
                const unsigned prev = atomicAdd(&sc->ticket, n);
                s_last = (prev + n == (unsigned)units);
            }
            __syncthreads();
            if (s_last) {
                __threadfence();
                double v[Op::ND];
#pragma unroll
                for (int q = 0; q < Op::ND; ++q) v[q] = 0.0;
                for (int u = threadIdx.x; u < units; u += NTHREADS) {
#pragma unroll
                    for (int q = 0; q < Op::ND; ++q) v[q] += __ldcg(D.partials + u * MAX_DOTS + q);
                }
                block_sum<Op::ND>(v, sred);
                if (threadIdx.x == 0) {
                    epilogue<Op::EPI, Op::ND>(D, sc, v);
                    sc->ticket = 0;
                    __threadfence();
                }
            }
        }
    }
}

// ------------------------------------------------------------------------
// Operations.
// ------------------------------------------------------------------------
struct NoPW {};

// Chebyshev sweep 1 (Algorithm 2, first two steps) on a right-hand side u
// that is itself formed point by point from FP64 vectors:
//   SIDE_P: u = p_{i-1} = r + beta (p_{i-2} - omega w)   (Alg. 1, last line;
//           u = r on the first iteration)
//   SIDE_S: u = s = r - alpha w                          (Alg. 1) and ||s||^2
// It writes u (FP64), the CI copy of u rounded to T (mixed precision only),
// and z = u/theta (degree 0) or y_1 = (2 rho_1/delta)(2u - A u/theta).
constexpr int SIDE_P = 0, SIDE_S = 1;
template <class T, bool BLK, int SIDE>
struct OpCiFirst {
    using E = Elem<T>;
    using C = typename E::C;
    using U = double;
    using PW = NoPW;
    static constexpr int ND = SIDE == SIDE_S ? 1 : 0;
    static constexpr int EPI = SIDE == SIDE_S ? EPI_SNORM : EPI_NONE;
    static constexpr bool STENCIL = true, BLOCKED = BLK;
    static constexpr bool MIXED = !std::is_same<T, double>::value;
    const double *r, *pold, *w;
    double *uout;
    void *bc, *out;
    double beta, omega, alpha;
    int first, degree;
    C tinv, coef1;
    __device__ OpCiFirst(const Desc &D, const KArgs &a, Scal *sc)
    {
        const int iter = ld_flag(&sc->iter);
        r = (const double *)D.vec[ROLE_R];
        w = (const double *)D.vec[ROLE_W];
        pold = (const double *)D.vec[resolve_role(ROLE_POLD, iter)];
        uout = (double *)D.vec[resolve_role(a.in, iter)];
        bc = D.vec[ROLE_BC];
        out = D.vec[a.out];
        beta = ld_scal(&sc->beta);
        omega = ld_scal(&sc->omega);
        alpha = ld_scal(&sc->alpha);
        first = ld_flag(&sc->first);
        degree = D.degree;
        tinv = (C)D.theta_inv;
        coef1 = (C)(D.two_over_delta * D.rho[1]);
    }
    __device__ __forceinline__ double load(int idx) const
    {
        if constexpr (SIDE == SIDE_S) {
            return r[idx] - alpha * w[idx];
        } else {
            if (first) return r[idx];
            return r[idx] + beta * (pold[idx] - omega * w[idx]);
        }
    }
    __device__ __forceinline__ C sv(double u) const { return (C)E::round(u); }
    __device__ __forceinline__ PW pw(bool, int) const { return PW{}; }
    template <int NA>
    __device__ __forceinline__ void emit(int idx, C au, double uc, const PW &, double (&acc)[NA]) const
    {
        uout[idx] = uc;
        if constexpr (SIDE == SIDE_S) acc[0] += uc * uc;
        const C b = sv(uc);
        if constexpr (MIXED) E::st(bc, idx, b);
        if (degree == 0) E::st(out, idx, b * tinv);
        else E::st(out, idx, coef1 * (C(2) * b - au * tinv));
    }
};

// Chebyshev sweep k >= 2 (Algorithm 2 loop body):
//   w = rho_k (2 sigma y + (2/delta)(b - A y) - rho_{k-1} z),
// y = y_{k-1} (stencil input), z = y_{k-2} (z = b/theta when k = 2).
// TB is the storage type of the CI right-hand side b.
template <class T, class TB, bool BLK>
struct OpCiSweep {
    using E = Elem<T>;
    using EB = Elem<TB>;
    using C = typename E::C;
    using U = C;
    struct PW { C b, z; };
    static constexpr int ND = 0, EPI = EPI_NONE;
    static constexpr bool STENCIL = true, BLOCKED = BLK;
    const void *y, *bv, *zv;
    void *out;
    C tinv, tod, tsig, rk, rk1;
    int k;
    __device__ OpCiSweep(const Desc &D, const KArgs &a, Scal *sc)
    {
        const int iter = ld_flag(&sc->iter);
        y = D.vec[a.in];
        bv = D.vec[resolve_role(a.b, iter)];
        zv = D.vec[a.z];
        out = D.vec[a.out];
        k = a.k;
        tinv = (C)D.theta_inv;
        tod = (C)D.two_over_delta;
        tsig = (C)D.two_sigma;
        rk = (C)D.rho[a.k];
        rk1 = (C)D.rho[a.k - 1];
    }
    __device__ __forceinline__ C load(int idx) const { return E::ld(y, idx); }
    __device__ __forceinline__ C sv(C u) const { return u; }
    __device__ __forceinline__ PW pw(bool valid, int idx) const
    {
        PW p{C(0), C(0)};
        if (valid) {
            p.b = (C)EB::ld(bv, idx);
            if (k >= 3) p.z = E::ld(zv, idx);
        }
        return p;
    }
    template <int NA>
    __device__ __forceinline__ void emit(int idx, C au, C yc, const PW &p, double (&)[NA]) const
    {
        const C z = (k == 2) ? p.b * tinv : p.z;
        E::st(out, idx, rk * (tsig * yc + tod * (p.b - au) - rk1 * z));
    }
};

// w = A p^ and r~ . w  (Algorithm 3, first stencil kernel); T = type of p^.
template <class T>
struct OpStencilDot {
    using C = double;
    using U = double;
    using PW = double;
    static constexpr int ND = 1, EPI = EPI_ALPHA;
    static constexpr bool STENCIL = true, BLOCKED = false;
    const void *ph;
    const double *rt;
    double *w;
    __device__ OpStencilDot(const Desc &D, const KArgs &a, Scal *)
    {
        ph = D.vec[a.in];
        rt = (const double *)D.vec[ROLE_RT];
        w = (double *)D.vec[ROLE_W];
    }
    __device__ __forceinline__ double load(int idx) const { return (double)Elem<T>::ld(ph, idx); }
    __device__ __forceinline__ double sv(double u) const { return u; }
    __device__ __forceinline__ double pw(bool valid, int idx) const { return valid ? __ldg(rt + idx) : 0.0; }
    template <int NA>
    __device__ __forceinline__ void emit(int idx, double au, double, double rtv, double (&acc)[NA]) const
    {
        w[idx] = au;
        acc[0] += rtv * au;
    }
};

// t = A r^, t . s and t . t (Algorithm 3, second stencil kernel).
template <class T>
struct OpStencil2Dot {
    using C = double;
    using U = double;
    using PW = double;
    static constexpr int ND = 2, EPI = EPI_OMEGA;
    static constexpr bool STENCIL = true, BLOCKED = false;
    const void *rh;
    const double *s;
    double *t;
    __device__ OpStencil2Dot(const Desc &D, const KArgs &a, Scal *)
    {
        rh = D.vec[a.in];
        s = (const double *)D.vec[ROLE_S];
        t = (double *)D.vec[ROLE_T];
    }
    __device__ __forceinline__ double load(int idx) const { return (double)Elem<T>::ld(rh, idx); }
    __device__ __forceinline__ double sv(double u) const { return u; }
    __device__ __forceinline__ double pw(bool valid, int idx) const { return valid ? s[idx] : 0.0; }
    template <int NA>
    __device__ __forceinline__ void emit(int idx, double au, double, double sv_, double (&acc)[NA]) const
    {
        t[idx] = au;
        acc[0] += au * sv_;
        acc[1] += au * au;
    }
};

// Plain out = A u (optionally block-restricted); building block.
template <bool BLK>
struct OpApplyA {
    using C = double;
    using U = double;
    using PW = NoPW;
    static constexpr int ND = 0, EPI = EPI_NONE;
    static constexpr bool STENCIL = true, BLOCKED = BLK;
    const double *u;
    double *v;
    __device__ OpApplyA(const Desc &D, const KArgs &a, Scal *)
    {
        u = (const double *)D.vec[a.in];
        v = (double *)D.vec[a.out];
    }
    __device__ __forceinline__ double load(int idx) const { return __ldg(u + idx); }
    __device__ __forceinline__ double sv(double x) const { return x; }
    __device__ __forceinline__ PW pw(bool, int) const { return PW{}; }
    template <int NA>
    __device__ __forceinline__ void emit(int idx, double au, double, const PW &, double (&)[NA]) const
    {
        v[idx] = au;
    }
};

// r = b - A x with ||b||^2 and ||r||^2 (initial residual for a given x0,
// r~ = r0), or only ||b - A x||^2 (true residual at exit).
template <bool INIT>
struct OpResidual {
    using C = double;
    using U = double;
    using PW = double;
    static constexpr int ND = INIT ? 2 : 1;
    static constexpr int EPI = INIT ? EPI_INITX0 : EPI_TRUE;
    static constexpr bool STENCIL = true, BLOCKED = false;
    const double *x, *b;
    double *r, *rt;
    __device__ OpResidual(const Desc &D, const KArgs &, Scal *)
    {
        x = (const double *)D.vec[ROLE_X];
        b = (const double *)D.vec[ROLE_B];
        r = (double *)D.vec[ROLE_R];
        rt = (double *)D.vec[ROLE_RT];
    }
    __device__ __forceinline__ double load(int idx) const { return x[idx]; }
    __device__ __forceinline__ double sv(double u) const { return u; }
    __device__ __forceinline__ double pw(bool valid, int idx) const { return valid ? __ldg(b + idx) : 0.0; }
    template <int NA>
    __device__ __forceinline__ void emit(int idx, double au, double, double bv, double (&acc)[NA]) const
    {
        const double rv = bv - au;
        if constexpr (INIT) {
            r[idx] = rv;
            rt[idx] = rv;
            acc[0] += bv * bv;
            acc[1] += rv * rv;
        } else {
            acc[0] += rv * rv;
        }
    }
};

// x0 = 0: r = b, x = 0, ||b||^2 (r~ aliases b).
struct OpInit0 {
    using C = double;
    static constexpr int ND = 1, EPI = EPI_INIT0;
    static constexpr bool STENCIL = false;
    const double *b;
    double *r, *x;
    __device__ OpInit0(const Desc &D, const KArgs &, Scal *)
    {
        b = (const double *)D.vec[ROLE_B];
        r = (double *)D.vec[ROLE_R];
        x = (double *)D.vec[ROLE_X];
    }
    template <int NA>
    __device__ __forceinline__ void emit(int idx, double (&acc)[NA]) const
    {
        const double bv = __ldg(b + idx);
        r[idx] = bv;
        x[idx] = 0.0;
        acc[0] += bv * bv;
    }
};

// x += alpha p^ + omega r^; r = s - omega t; r~ . r, ||r||^2
// (Algorithm 3, KernelBiCGS4+5).  After a passed half-step test only
// x += alpha p^ (Algorithm 1).  T = type of p^ and r^.
template <class T>
struct OpUpdate {
    using C = double;
    static constexpr int ND = 2, EPI = EPI_UPDATE;
    static constexpr bool STENCIL = false;
    double *x, *r;
    const void *ph, *rh;
    const double *s, *t, *rt;
    double alpha, omega;
    int half;
    __device__ OpUpdate(const Desc &D, const KArgs &a, Scal *sc)
    {
        x = (double *)D.vec[ROLE_X];
        r = (double *)D.vec[ROLE_R];
        ph = D.vec[a.in];
        rh = D.vec[a.aux];
        s = (const double *)D.vec[ROLE_S];
        t = (const double *)D.vec[ROLE_T];
        rt = (const double *)D.vec[ROLE_RT];
        alpha = ld_scal(&sc->alpha);
        omega = ld_scal(&sc->omega);
        half = ld_flag(&sc->half);
    }
    template <int NA>
    __device__ __forceinline__ void emit(int idx, double (&acc)[NA]) const
    {
        const double pv = (double)Elem<T>::ld(ph, idx);
        if (half) {
            x[idx] = x[idx] + alpha * pv;
            return;
        }
        const double rv = (double)Elem<T>::ld(rh, idx);
        const double sv = __ldg(s + idx), tv = __ldg(t + idx), rtv = __ldg(rt + idx);
        x[idx] = x[idx] + alpha * pv + omega * rv;
        const double rn = sv - omega * tv;
        r[idx] = rn;
        acc[0] += rtv * rn;
        acc[1] += rn * rn;
    }
};

// Unpreconditioned direction update p = r + beta (p - omega w), in place
// (pointwise; p = r on the first iteration).
struct OpPUpdate {
    using C = double;
    static constexpr int ND = 0, EPI = EPI_NONE;
    static constexpr bool STENCIL = false;
    const double *r, *w;
    double *p;
    double beta, omega;
    int first;
    __device__ OpPUpdate(const Desc &D, const KArgs &, Scal *sc)
    {
        r = (const double *)D.vec[ROLE_R];
        w = (const double *)D.vec[ROLE_W];
        p = (double *)D.vec[ROLE_P];
        beta = ld_scal(&sc->beta);
        omega = ld_scal(&sc->omega);
        first = ld_flag(&sc->first);
    }
    template <int NA>
    __device__ __forceinline__ void emit(int idx, double (&)[NA]) const
    {
        if (first) p[idx] = __ldg(r + idx);
        else p[idx] = __ldg(r + idx) + beta * (p[idx] - omega * __ldg(w + idx));
    }
};

// Unpreconditioned half step s = r - alpha w with ||s||^2 (pointwise).
struct OpSUpdate {
    using C = double;
    static constexpr int ND = 1, EPI = EPI_SNORM;
    static constexpr bool STENCIL = false;
    const double *r, *w;
    double *s;
    double alpha;
    __device__ OpSUpdate(const Desc &D, const KArgs &, Scal *sc)
    {
        r = (const double *)D.vec[ROLE_R];
        w = (const double *)D.vec[ROLE_W];
        s = (double *)D.vec[ROLE_S];
        alpha = ld_scal(&sc->alpha);
    }
    template <int NA>
    __device__ __forceinline__ void emit(int idx, double (&acc)[NA]) const
    {
        const double v = __ldg(r + idx) - alpha * __ldg(w + idx);
        s[idx] = v;
        acc[0] += v * v;
    }
};

// a . b (building block).
struct OpDot {
    using C = double;
    static constexpr int ND = 1, EPI = EPI_RAW;
    static constexpr bool STENCIL = false;
    const double *a, *b;
    __device__ OpDot(const Desc &D, const KArgs &k, Scal *)
    {
        a = (const double *)D.vec[k.in];
        b = (const double *)D.vec[k.aux];
    }
    template <int NA>
    __device__ __forceinline__ void emit(int idx, double (&acc)[NA]) const
    {
        acc[0] += __ldg(a + idx) * __ldg(b + idx);
    }
};

// out (FP64) = in (type T), exact widening (building block).
template <class T>
struct OpWiden {
    using C = double;
    static constexpr int ND = 0, EPI = EPI_NONE;
    static constexpr bool STENCIL = false;
    const void *in;
    double *out;
    __device__ OpWiden(const Desc &D, const KArgs &k, Scal *)
    {
        in = D.vec[k.in];
        out = (double *)D.vec[k.out];
    }
    template <int NA>
    __device__ __forceinline__ void emit(int idx, double (&)[NA]) const
    {
        out[idx] = (double)Elem<T>::ld(in, idx);
    }
};

} // namespace psolve
