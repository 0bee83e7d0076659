// psolve_kernels.cuh -- CUDA kernels of the Bi-CGSTAB / Chebyshev hot path
// (sm_103a).  No tensor cores: the 7-point operator is a streaming stencil,
// bound by HBM bandwidth.
//
// Engines.  A CTA of TILE_X x TILE_Y threads owns an xy tile; each thread owns
// one z column and marches along z.  Two engines compute bitwise the same
// values (same thread mapping, same expressions):
//  * the TMA ring (march_tma, used when the row pitch is a multiple of 8 and
//    the vectors are 16-byte aligned): one thread stages whole plane tiles, halo included,
//    several planes ahead with cp.async.bulk.tensor into a shared-memory ring
//    tracked by mbarriers, so the bytes in flight do not depend on registers;
//  * the general engine (march_stencil, any size): u(k-1), u(k), u(k+1) in
//    registers, the x/y neighbours of plane k from a double-buffered shared
//    copy of the plane, the next planes prefetched one step ahead.
// Either way every input value is read from HBM once per sweep.  Zero
// Dirichlet ghosts (Eq. 4) are zero-filled halo cells; the block-restricted
// operator R_s A R_s^T of Eq. 14 zeroes neighbours across block faces.
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
// Exact conversions on the integer pipe.  B300 executes FP64 conversions on
// its narrow FP64 pipe (2 instructions per clock per SM), where they compete
// with the FP64 arithmetic of the outer iteration; these IEEE-754 bit
// manipulations give the same results with integer instructions only.
// ------------------------------------------------------------------------
// float -> double, exact.  Normal: re-bias the exponent (1023 - 127 = 896)
// and move the 23-bit mantissa to the top of the 52-bit field.  Subnormal:
// normalise with a leading-zero count.  Zero, Inf and NaN keep their class.
__device__ __forceinline__ double f2d_exact(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t sign = u & 0x80000000u;
    const uint32_t e = (u >> 23) & 0xffu;
    const uint32_t man = u & 0x7fffffu;
    uint32_t ed = e + 896u, m = man;
    if (e == 0u) {
        if (man == 0u) {
            ed = 0u;
        } else { // value man * 2^-149 = 1.f * 2^(31 - clz - 149)
            const uint32_t lz = (uint32_t)__clz((int)man);
            ed = 905u - lz;
            m = (man << (lz - 8u)) & 0x7fffffu;
        }
    } else if (e == 0xffu) {
        ed = 0x7ffu;
    }
    const uint32_t hi = sign | (ed << 20) | (m >> 3);
    const uint32_t lo = m << 29;
    return __hiloint2double((int)hi, (int)lo);
}

// double -> float, round to nearest even (IEEE-754).  Normal results keep 23
// of the 52 mantissa bits and round on the 29 dropped bits; a carry out of the
// mantissa moves into the exponent (and to infinity at the top).  Subnormal
// results shift the 53-bit significand right by (926 - e) and round the same
// way; results below half the smallest subnormal are zero, values beyond the
// float range are infinity, NaN stays NaN.
__device__ __forceinline__ float d2f_rn(double d)
{
    const uint32_t hi = (uint32_t)__double2hiint(d);
    const uint32_t lo = (uint32_t)__double2loint(d);
    const uint32_t sign = hi & 0x80000000u;
    const uint32_t e = (hi >> 20) & 0x7ffu;
    uint32_t r;
    if (e >= 897u && e <= 1150u) {
        const uint32_t m23 = ((hi & 0xfffffu) << 3) | (lo >> 29);
        const uint32_t rest = lo & 0x1fffffffu;
        r = sign | ((e - 896u) << 23) | m23;
        if (rest > 0x10000000u || (rest == 0x10000000u && (m23 & 1u))) r += 1u;
    } else if (e > 1150u) {
        const bool nan = e == 0x7ffu && ((hi & 0xfffffu) | lo) != 0u;
        r = sign | (nan ? 0x7fc00000u : 0x7f800000u);
    } else if (e == 0u || 926u - e > 63u) {
        r = sign; // +-0
    } else {
        const uint64_t m = (((uint64_t)(hi & 0xfffffu) | 0x100000u) << 32) | lo; // 53-bit significand
        const uint32_t sh = 926u - e;                                           // 30..63
        const uint64_t q = m >> sh;
        const uint64_t rest = m & ((1ull << sh) - 1ull);
        const uint64_t half = 1ull << (sh - 1u);
        r = sign | (uint32_t)q;
        if (rest > half || (rest == half && (q & 1ull))) r += 1u;
    }
    return __uint_as_float(r);
}

// ------------------------------------------------------------------------
// Global loads of solver vectors.  They go through L2 only (ld.global.cg):
// the persistent kernel reads, after a grid barrier, vectors that other SMs
// rewrote since this SM last read them, so neither the read-only path nor a
// possibly stale L1 line may serve them.  Each vector element is read once
// per kernel, so L1 would not help the streaming kernels either.
// ------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T gld(const T *p)
{
    return __ldcg(p);
}

// ------------------------------------------------------------------------
// Storage types of the Chebyshev vectors and their arithmetic type.
// ------------------------------------------------------------------------
template <class T> struct Elem;
template <> struct Elem<double> {
    using C = double;
    static __device__ __forceinline__ double ld(const void *p, int i) { return gld((const double *)p + i); }
    static __device__ __forceinline__ double lds(const void *p, int i) { return ((const double *)p)[i]; }
    static __device__ __forceinline__ double wide(const void *p, int i) { return ld(p, i); }
    static __device__ __forceinline__ double wides(const void *p, int i) { return lds(p, i); }
    static __device__ __forceinline__ void st(void *p, int i, double v) { ((double *)p)[i] = v; }
    static __device__ __forceinline__ double round(double v) { return v; }
};
template <> struct Elem<float> {
    using C = float;
    static __device__ __forceinline__ float ld(const void *p, int i) { return gld((const float *)p + i); }
    static __device__ __forceinline__ float lds(const void *p, int i) { return ((const float *)p)[i]; }
    static __device__ __forceinline__ double wide(const void *p, int i) { return f2d_exact(ld(p, i)); }
    static __device__ __forceinline__ double wides(const void *p, int i) { return f2d_exact(lds(p, i)); }
    static __device__ __forceinline__ void st(void *p, int i, float v) { ((float *)p)[i] = v; }
    static __device__ __forceinline__ float round(double v) { return d2f_rn(v); }
};
template <> struct Elem<__nv_bfloat16> {
    using C = float;
    static __device__ __forceinline__ float ld(const void *p, int i)
    {
        return __bfloat162float(gld((const __nv_bfloat16 *)p + i));
    }
    static __device__ __forceinline__ float lds(const void *p, int i)
    {
        return __bfloat162float(((const __nv_bfloat16 *)p)[i]);
    }
    static __device__ __forceinline__ double wide(const void *p, int i) { return f2d_exact(ld(p, i)); }
    static __device__ __forceinline__ double wides(const void *p, int i) { return f2d_exact(lds(p, i)); }
    static __device__ __forceinline__ void st(void *p, int i, float v)
    {
        ((__nv_bfloat16 *)p)[i] = __float2bfloat16_rn(v);
    }
    static __device__ __forceinline__ float round(double v)
    {
        return __bfloat162float(__float2bfloat16_rn(d2f_rn(v)));
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
    EPI_RAW,     // store v in red[]
    EPI_REPLACE  // v0 = r~ . r, v1 = ||r||^2 of r = b - A x -> rescale beta, rho; test
};

constexpr int ST_OK = 0, ST_INTERNAL = 3 /* PSOLVE_E_CUDA */, ST_NOT_CONVERGED = 4, ST_BREAKDOWN = 5,
              ST_NONFINITE = 6;

__device__ __forceinline__ void stop_with(volatile Scal *sc, int status)
{
    sc->status = status;
    sc->stop = 1;
}

// Runs in one thread of the CTA that finished a reduction last.  The scalar
// block is accessed through volatile (L2) loads and stores: in the persistent
// kernel another SM may have rewritten it since this SM's L1 last held it.
template <int EPI, int ND>
__device__ void epilogue(const Desc &D, Scal *sc_mem, const double (&v)[ND])
{
    volatile Scal *sc = sc_mem;
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
        sc->alpha = 0.0;
        sc->omega = 0.0;
        sc->beta = 0.0;
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
        if (D.hist && sc->iter < D.hist_cap) D.hist[2 * sc->iter] = ss; // iteration iter + 1
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
        sc->iter = sc->iter + 1;
        if (sc->half) { // x += alpha p^ was the whole update
            sc->rr = sc->ss;
            sc->half_exit = 1;
            stop_with(sc, ST_OK);
        } else {
            const double rho_new = v[0], rr = v[1];
            sc->rr = rr;
            if (D.hist && sc->iter <= D.hist_cap) D.hist[2 * sc->iter - 1] = rr;
            if (!isfinite(rr) || !isfinite(rho_new)) stop_with(sc, ST_NONFINITE);
            else if (rr <= sc->thr2) stop_with(sc, ST_OK);
            else if (rr > 1e16 * sc->nb2) stop_with(sc, ST_NOT_CONVERGED); // diverged: ||r|| > 1e8 ||b||
            else if (rho_new == 0.0) stop_with(sc, ST_BREAKDOWN);
            else {
                sc->beta = (rho_new / sc->rho) * (sc->alpha / sc->omega);
                sc->rho = rho_new;
                sc->first = 0;
                if (sc->iter >= sc->maxit) stop_with(sc, ST_NOT_CONVERGED);
            }
        }
    } else if constexpr (EPI == EPI_REPLACE) {
        // beta = (rho_i / rho_{i-1})(alpha / omega) is proportional to rho_i:
        // rescale it to rho_i = r~ . r of the replaced residual
        const double rho_new = v[0], rr = v[1];
        sc->rr = rr;
        if (D.hist && sc->iter <= D.hist_cap) D.hist[2 * sc->iter - 1] = rr; // replaces the recursive norm
        if (!isfinite(rr) || !isfinite(rho_new)) stop_with(sc, ST_NONFINITE);
        else if (rr <= sc->thr2) stop_with(sc, ST_OK);
        else if (rho_new == 0.0) stop_with(sc, ST_BREAKDOWN);
        else {
            sc->beta = sc->beta * (rho_new / sc->rho);
            sc->rho = rho_new;
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

// Zero-flux Neumann faces (matrix N, Eq. 5): the outside neighbour of a
// boundary unknown equals its inside neighbour, so the pair sum across that
// face is twice the inside value.  neumann_mask() gives, once per march, the
// faces this thread's column touches (bits 0-3: x-, x+, y-, y+; bits 4-5: z-,
// z+, which apply on the first / last plane); apply_neumann() runs after the
// zero ghosts of the block restriction, which never remove the inside
// neighbour (a Neumann face needs two unknowns per block on its axis).
// Whether an operation handles Neumann faces (all do, except sweeps compiled
// for grids without them).
template <class Op, class = void>
struct HasNeumann {
    static constexpr bool value = true;
};
template <class Op>
struct HasNeumann<Op, std::void_t<decltype(Op::NEUMANN)>> {
    static constexpr bool value = Op::NEUMANN;
};

__device__ __forceinline__ int neumann_mask(int bcm, int i, int j, int nx, int ny)
{
    int m = bcm & 48;
    if (i == 0) m |= bcm & 1;
    if (i == nx - 1) m |= bcm & 2;
    if (j == 0) m |= bcm & 4;
    if (j == ny - 1) m |= bcm & 8;
    return m;
}

template <class C>
__device__ __forceinline__ void apply_neumann(int m, bool first_plane, bool last_plane, C &w, C &e, C &so, C &no,
                                              C &dn, C &un)
{
    if (m & 1) w = e;
    if (m & 2) e = w;
    if (m & 4) so = no;
    if (m & 8) no = so;
    if ((m & 16) && first_plane) dn = un;
    if ((m & 32) && last_plane) un = dn;
}

// ------------------------------------------------------------------------
// Stencil march over planes [kb, ke) of chunk c0 of one tile.
// Op provides: types C (arithmetic), U (own-column value), PW (pointwise
// operands); ND; BLOCKED; U load(idx); C sv(U); PW pw(bool, idx);
// void emit(idx, C u, C sx, C sy, C sz, U uc, PW, acc) with u the centre value
// and sx, sy, sz the sums of its two neighbours along x, y, z, so that
// (A u) = cc u - cx sx - cy sy - cz sz (Eq. 3 / Eq. 6).  Each operation folds
// its own constants into these terms: on B300 the FP64 pipe (2 FMA per clock
// per SM), not HBM, bounds the FP64 kernels, so every FP64 instruction counts.
// ------------------------------------------------------------------------
template <class Op>
__device__ __forceinline__ void march_stencil(Op &op, const Desc &D, int tile, int c0, int kb, int ke,
                                              typename Op::C *sp, double *sred)
{
    using C = typename Op::C;
    using U = typename Op::U;
    using PW = typename Op::PW;
    constexpr int ND = Op::ND;
    constexpr int NDA = ND > 0 ? ND : 1;
    constexpr int SW = TILE_X + 2;
    constexpr int SPL = SW * (TILE_Y + 2);

    const int nx = D.nx, ny = D.ny, nz = D.nz, px = D.px;
    const int plane = px * ny;
    const int tid = threadIdx.x, tx = tid % TILE_X, ty = tid / TILE_X;
    const int i0 = (tile % D.tiles_x) * TILE_X, j0 = (tile / D.tiles_x) * TILE_Y;
    const int i = i0 + tx, j = j0 + ty;
    const bool in = (i < nx) && (j < ny);
    const int col = in ? j * px + i : 0;

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
    const int hcol = hv ? hj * px + hi : 0;
    const int me = (ty + 1) * SW + tx + 1;

    bool okw = true, oke = true, oks = true, okn = true;
    if constexpr (Op::BLOCKED) {
        okw = (i % D.bx) != 0;
        oke = (i % D.bx) != D.bx - 1;
        oks = (j % D.by) != 0;
        okn = (j % D.by) != D.by - 1;
    }
    const int nbm = (HasNeumann<Op>::value && D.bcm) ? neumann_mask(D.bcm, i, j, nx, ny) : 0;

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
    const int ntiles = D.tiles_x * D.tiles_y;
    const int unit = c0 * ntiles + tile; // units are numbered chunk-major
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
            if (nbm) apply_neumann(nbm, k == 0, k == nz - 1, w, e, so, no, dn, un);
            op.emit(col + k * plane, op.sv(uc), w + e, so + no, dn + un, uc, pw, acc);
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
    }
    if constexpr (ND > 0) flush_unit<ND>(acc, sred, D.partials, unit);
}

// Planes a pointwise operation keeps in flight ahead of the one it computes
// (2, or the operation's PREFETCH: 1 where three planes of inputs would not
// fit in the registers; 0: load two planes, then compute both).
template <class Op, class = void>
struct PointDepth {
    static constexpr int value = 2;
};
template <class Op>
struct PointDepth<Op, std::void_t<decltype(Op::PREFETCH)>> {
    static constexpr int value = Op::PREFETCH;
};

// Pointwise march (no stencil) over chunks [c0, c1) of one tile, software
// pipelined: while plane k is computed, the loads of planes k+1 and k+2 are
// in flight (different planes never alias).  A warp that has computed a plane
// therefore finds the next one arriving instead of issuing its loads only
// then, which keeps loads in flight during the FP64 work (the update with 6
// inputs per point is bound by both).  Planes are applied in order, so the
// per-thread partial sums are the same as with one plane at a time.
// Op provides: struct In (raw loaded values; narrow types are widened in
// apply); In load(idx); void apply(idx, const In&, acc).
template <class Op>
__device__ __forceinline__ void march_point(Op &op, const Desc &D, int tile, int c0, int c1, double *sred)
{
    constexpr int ND = Op::ND;
    constexpr int NDA = ND > 0 ? ND : 1;
    using In = typename Op::In;
    const int nx = D.nx, ny = D.ny, nz = D.nz, zc = D.zc;
    const int plane = D.px * ny;
    const int tid = threadIdx.x, tx = tid % TILE_X, ty = tid / TILE_X;
    const int i = (tile % D.tiles_x) * TILE_X + tx, j = (tile / D.tiles_x) * TILE_Y + ty;
    const bool in = (i < nx) && (j < ny);
    const int col = in ? j * D.px + i : 0;
    const int ntiles = D.tiles_x * D.tiles_y;
    double acc[NDA];
#pragma unroll
    for (int q = 0; q < NDA; ++q) acc[q] = 0.0;
    for (int c = c0; c < c1; ++c) {
        const int kb = c * zc, ke = min(nz, (c + 1) * zc);
        if constexpr (PointDepth<Op>::value >= 2) {
            In a{}, b{};
            if (in) a = op.load(col + kb * plane);
            if (in && kb + 1 < ke) b = op.load(col + (kb + 1) * plane);
            for (int k = kb; k < ke; ++k) {
                In n{};
                if (in && k + 2 < ke) n = op.load(col + (k + 2) * plane);
                if (in) op.apply(col + k * plane, a, acc);
                a = b;
                b = n;
            }
        } else if constexpr (PointDepth<Op>::value == 1) { // one plane ahead (many inputs: registers)
            In a{};
            if (in) a = op.load(col + kb * plane);
            for (int k = kb; k < ke; ++k) {
                In n{};
                if (in && k + 1 < ke) n = op.load(col + (k + 1) * plane);
                if (in) op.apply(col + k * plane, a, acc);
                a = n;
            }
        } else { // two planes loaded, then both computed
            for (int k = kb; k < ke; k += 2) {
                const bool two = k + 1 < ke;
                In v0{}, v1{};
                if (in) v0 = op.load(col + k * plane);
                if (in && two) v1 = op.load(col + (k + 1) * plane);
                if (in) op.apply(col + k * plane, v0, acc);
                if (in && two) op.apply(col + (k + 1) * plane, v1, acc);
            }
        }
        if constexpr (ND > 0) flush_unit<ND>(acc, sred, D.partials, c * ntiles + tile);
    }
}

// ------------------------------------------------------------------------
// TMA ring engine (problems with desc.tma = 1).
//
// Thread 0 stages plane q of every operand with one cp.async.bulk.tensor per
// array: the stencil input as a (TILE_X + 2 HX) x (TILE_Y + 2) halo box
// starting at (i0 - HX, j0 - 1) with HX = 16 / sizeof(element) (so the x start
// is 16-byte aligned), the pointwise operands as TILE_X x TILE_Y boxes.  Out of
// range elements are zero-filled by the copy engine: those zeros are exactly
// the Dirichlet ghosts of Eq. 4, including planes -1 and nz.  A ring of
// STAGES planes, one mbarrier each, keeps STAGES - 3 planes in flight ahead of
// the three (k-1, k, k+1) the stencil reads.  Every wait is bounded; on
// time-out the problem stops with status TIMEOUT and the CTA stops waiting.
// ------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Bounded wait for the completion of phase `parity`: gives up after about
// 2^31 clock cycles (about a second).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit = 1LL << 31)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
                 "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
                 : "memory");
}

constexpr int align128(int b) { return (b + 127) & ~127; }

// Ring stages an operation asks for (0: as many as fit in 48 KB, 4..8).
template <class Op, class = void>
struct RingStages {
    static constexpr int value = 0;
};
template <class Op>
struct RingStages<Op, std::void_t<decltype(Op::RING_STAGES)>> {
    static constexpr int value = Op::RING_STAGES;
};

// Shared-memory geometry of one ring stage for an operation.
template <class Op>
struct Ring {
    using TH = typename Op::TH;
    using TP = typename Op::TP;
    using C = typename Op::C;
    static constexpr int HX = 16 / (int)sizeof(TH);      // halo columns each side
    static constexpr int W = TILE_X + 2 * HX;            // halo box width
    static constexpr int HBOX = W * (TILE_Y + 2);        // halo box elements
    static constexpr int HBYTES = HBOX * (int)sizeof(TH);
    static constexpr int PBYTES = TILE_X * TILE_Y * (int)sizeof(TP);
    static constexpr int HSTRIDE = align128(HBYTES);
    static constexpr int PSTRIDE = align128(PBYTES);
    static constexpr int STAGE = Op::NH * HSTRIDE + Op::NP * PSTRIDE;
    using U = typename Op::U;
    // transformed planes: the stencil value (C) and, when it differs, the centre value (U)
    static constexpr bool UX = Op::XFORM && !std::is_same<U, C>::value;
    static constexpr int XBYTES = Op::XFORM ? align128(HBOX * (int)sizeof(C)) + (UX ? align128(HBOX * (int)sizeof(U)) : 0) : 0;
    static constexpr int STAGES_RAW = (48 * 1024 - 3 * XBYTES) / (STAGE > 0 ? STAGE : 1);
    static constexpr int STAGES_FIT = STAGES_RAW < 4 ? 4 : (STAGES_RAW > 8 ? 8 : STAGES_RAW);
    static constexpr int STAGES = RingStages<Op>::value > 0 ? RingStages<Op>::value : STAGES_FIT; // <= MAX_STAGES
    static constexpr int BYTES = STAGES * STAGE + 3 * XBYTES; // dynamic shared memory
};

// Issue the copies of plane q into stage `st` (thread 0 only).
template <class Op>
__device__ __forceinline__ void ring_issue(const Op &op, const Desc &D, unsigned char *stage, uint64_t *bar,
                                           int i0, int j0, int q, bool with_pw)
{
    using R = Ring<Op>;
    const uint32_t bytes = op.nh * R::HBYTES + (with_pw ? op.np * R::PBYTES : 0);
    mbar_expect_tx(bar, bytes);
    for (int a = 0; a < op.nh; ++a)
        tma_load_3d(stage + a * R::HSTRIDE, D.tmap + TMAPS_PER_ROLE * op.hrole[a] + TMAP_HALO, i0 - R::HX, j0 - 1, q,
                    bar);
    if (with_pw)
        for (int a = 0; a < op.np; ++a)
            tma_load_3d(stage + Op::NH * R::HSTRIDE + a * R::PSTRIDE, D.tmap + TMAPS_PER_ROLE * op.prole[a] + TMAP_PLAIN,
                        i0, j0, q,
                        bar);
}

template <class Op>
__device__ __forceinline__ void stage_ptrs(unsigned char *stage, const void *(&h)[Op::NH > 0 ? Op::NH : 1],
                                           const void *(&p)[Op::NP > 0 ? Op::NP : 1])
{
    using R = Ring<Op>;
#pragma unroll
    for (int a = 0; a < Op::NH; ++a) h[a] = stage + a * R::HSTRIDE;
#pragma unroll
    for (int a = 0; a < Op::NP; ++a) p[a] = stage + Op::NH * R::HSTRIDE + a * R::PSTRIDE;
}

// Stencil march over planes [kb, ke) of chunk c0 of one tile, operands staged by TMA.
// `seq` counts the planes this CTA has staged so far (all threads agree); plane
// number n lives in stage n % STAGES and completes phase (n / STAGES) & 1.
// The stages (and mbarrier parities) of planes k-1, k, k+1 are carried as
// rolling indices, and each thread keeps the centre values of those three
// planes in registers (a z-queue), so a point costs four in-plane neighbour
// reads from shared memory plus one for the next plane's centre.
template <class Op>
__device__ __forceinline__ void march_tma(Op &op, const Desc &D, int tile, int c0, int kb, int ke,
                                          unsigned char *ring, uint64_t *bars, uint32_t &seq,
                                          double *sred, int *s_dead)
{
    using R = Ring<Op>;
    using C = typename Op::C;
    using U = typename Op::U;
    using PW = typename Op::PW;
    constexpr int S = R::STAGES;
    constexpr int W = R::W;
    constexpr int ND = Op::ND;
    constexpr int NDA = ND > 0 ? ND : 1;
    constexpr int NHA = Op::NH > 0 ? Op::NH : 1;
    constexpr int NPA = Op::NP > 0 ? Op::NP : 1;

    const int nx = D.nx, ny = D.ny, nz = D.nz, px = D.px;
    const int plane = px * ny;
    const int tid = threadIdx.x, tx = tid % TILE_X, ty = tid / TILE_X;
    const int i0 = (tile % D.tiles_x) * TILE_X, j0 = (tile / D.tiles_x) * TILE_Y;
    const int i = i0 + tx, j = j0 + ty;
    const bool in = (i < nx) && (j < ny);
    const int col = in ? j * px + i : 0;
    const int me = (ty + 1) * W + tx + R::HX; // this point in a halo box
    const int mp = ty * TILE_X + tx;          // this point in a plain box

    bool okw = true, oke = true, oks = true, okn = true;
    if constexpr (Op::BLOCKED) {
        okw = (i % D.bx) != 0;
        oke = (i % D.bx) != D.bx - 1;
        oks = (j % D.by) != 0;
        okn = (j % D.by) != D.by - 1;
    }
    const int nbm = (HasNeumann<Op>::value && D.bcm) ? neumann_mask(D.bcm, i, j, nx, ny) : 0;
    const int q0 = kb - 1, q1 = ke; // stencil-input planes q0..q1, pointwise planes kb..ke-1
    const int nplanes = q1 - q0 + 1;
    const uint32_t seq0 = seq;
    unsigned char *xbase = ring + S * R::STAGE; // transformed u planes (XFORM only)
    C *xring = reinterpret_cast<C *>(xbase);
    U *uring = reinterpret_cast<U *>(xbase + 3 * align128(R::HBOX * (int)sizeof(C))); // when U != C

    // rolling stage index and mbarrier parity of a plane, advanced plane by plane
    struct Slot {
        int st;
        uint32_t par;
        __device__ __forceinline__ void next()
        {
            if (++st == R::STAGES) {
                st = 0;
                par ^= 1u;
            }
        }
    };
    Slot sm{(int)(seq0 % S), (seq0 / S) & 1u}; // plane k-1 (starts at q0)
    Slot smm = sm;                              // plane k-2 (used from the second step on)
    Slot sc = sm;
    sc.next(); // plane k
    Slot sn = sc;
    sn.next(); // plane k+1
    int xm = 0, xc = 1, xn = 2; // transformed-plane slots of k-1, k, k+1 (XFORM only)

    auto stage = [&](int st) { return ring + st * R::STAGE; };
    auto wait = [&](const Slot &sl) {
        if (*s_dead) return;
        if (!mbar_wait(bars + sl.st, sl.par)) {
            *s_dead = 1;
            D.sc->status = ST_TIMEOUT;
            D.sc->stop = 1;
        }
    };
    auto transform = [&](int st, int slot) {
        if constexpr (Op::XFORM) {
            const void *h[NHA], *p[NPA];
            stage_ptrs<Op>(stage(st), h, p);
            for (int x = tid; x < R::HBOX; x += NTHREADS) {
                const U v = op.load_s(h, x);
                xring[slot * R::HBOX + x] = op.sv(v);
                if constexpr (R::UX) uring[slot * R::HBOX + x] = v;
            }
        }
    };
    // this thread's centre value of the plane in stage `st` / slot `slot`
    auto centre = [&](int st, int slot) -> U {
        if constexpr (!Op::XFORM) {
            const void *h[NHA], *p[NPA];
            stage_ptrs<Op>(stage(st), h, p);
            return op.load_s(h, me);
        } else if constexpr (R::UX) {
            return uring[slot * R::HBOX + me];
        } else {
            return xring[slot * R::HBOX + me];
        }
    };

    __syncthreads(); // the previous run's readers of the ring are done
    if (tid == 0) {
        Slot si = sm;
        for (int n = 0; n < S && n < nplanes; ++n) {
            const int q = q0 + n;
            ring_issue<Op>(op, D, stage(si.st), bars + si.st, i0, j0, q, q >= kb && q < ke);
            si.next();
        }
    }
    wait(sm);
    wait(sc);
    transform(sm.st, xm);
    transform(sc.st, xc);
    if constexpr (Op::XFORM) __syncthreads();
    U zdn = in ? centre(sm.st, xm) : U(0); // centre values of planes k-1 and k
    U zc_ = in ? centre(sc.st, xc) : U(0);

    double acc[NDA];
#pragma unroll
    for (int a = 0; a < NDA; ++a) acc[a] = 0.0;
    int kk = 0;
    if constexpr (Op::BLOCKED) kk = kb % D.bz;
    const int ntiles = D.tiles_x * D.tiles_y;
    const int unit = c0 * ntiles + tile;

    for (int k = kb; k < ke; ++k) {
        wait(sn);
        transform(sn.st, xn);
        if constexpr (Op::XFORM) __syncthreads();
        const bool live = in && !*s_dead;
        U zup = U(0);
        if (live) {
            zup = centre(sn.st, xn);
            C w, e, so, no;
            if constexpr (Op::XFORM) {
                const C *xs = xring + xc * R::HBOX;
                w = xs[me - 1], e = xs[me + 1], so = xs[me - W], no = xs[me + W];
            } else {
                const void *h[NHA], *p[NPA];
                stage_ptrs<Op>(stage(sc.st), h, p);
                w = op.sv(op.load_s(h, me - 1)), e = op.sv(op.load_s(h, me + 1));
                so = op.sv(op.load_s(h, me - W)), no = op.sv(op.load_s(h, me + W));
            }
            C dn = op.sv(zdn), un = op.sv(zup);
            if constexpr (Op::BLOCKED) {
                if (!okw) w = C(0);
                if (!oke) e = C(0);
                if (!oks) so = C(0);
                if (!okn) no = C(0);
                if (kk == 0) dn = C(0);
                if (kk == D.bz - 1) un = C(0);
            }
            if (nbm) apply_neumann(nbm, k == 0, k == nz - 1, w, e, so, no, dn, un);
            const void *h[NHA], *p[NPA];
            stage_ptrs<Op>(stage(sc.st), h, p);
            const PW pw = op.pw_s(p, mp);
            op.emit(col + k * plane, op.sv(zc_), w + e, so + no, dn + un, zc_, pw, acc);
        }
        // the Chebyshev sweeps (no transform, no dots) take one CTA barrier per
        // two planes below (measured 241 -> 234 us per FP64 sweep at 256^3);
        // the stencil kernels with dots measured no better that way
        if constexpr (Op::XFORM || S < 6 || ND > 0) {
            __syncthreads(); // stage of plane k-1 (and its transformed plane) is free
            if (tid == 0 && k - 1 + S <= q1 && !*s_dead) {
                const int q = k - 1 + S;
                ring_issue<Op>(op, D, stage(sm.st), bars + sm.st, i0, j0, q, q >= kb && q < ke);
            }
        } else if ((k - kb) & 1) {
            // one CTA barrier per two planes: the stages of planes k-2 and k-1
            // are free, and both refills go out in plane order.  Plane k+1,
            // waited for at the top of step k, went out at the barrier after
            // step k-S+2 or k-S+3, at least three planes ahead with S >= 6.
            __syncthreads();
            if (tid == 0 && !*s_dead) {
                if (k - 2 + S <= q1) {
                    const int q = k - 2 + S;
                    ring_issue<Op>(op, D, stage(smm.st), bars + smm.st, i0, j0, q, q >= kb && q < ke);
                }
                if (k - 1 + S <= q1) {
                    const int q = k - 1 + S;
                    ring_issue<Op>(op, D, stage(sm.st), bars + sm.st, i0, j0, q, q >= kb && q < ke);
                }
            }
        }
        // rotate: plane k becomes k-1, k+1 becomes k
        smm = sm;
        sm = sc;
        sc = sn;
        sn.next();
        const int xt = xm;
        xm = xc;
        xc = xn;
        xn = xt;
        zdn = zc_;
        zc_ = zup;
        if constexpr (Op::BLOCKED) {
            if (++kk == D.bz) kk = 0;
        }
    }
    if constexpr (ND > 0) flush_unit<ND>(acc, sred, D.partials, unit);
    // every issued plane was waited for (q1 in the last step; planes beyond q1
    // are never issued), so nothing is left in flight
    seq = seq0 + nplanes;
}

// ------------------------------------------------------------------------
// Wide Chebyshev sweeps (OpCiSweepW): the same TMA ring, with each of
// TILE_X * TILE_Y / 2 threads computing two x-adjacent points of a plane.
// Per plane a thread reads its centre pair from the z-queue, the two outer x
// neighbours as single values, the y neighbours, the next plane's centre and
// the pointwise operands b and y_{k-2} as pairs, and stores one pair: seven
// shared-memory reads and one store for two points, where the one-point march
// spends seven reads and one store per point, and the per-plane work (ring
// waits, stage bookkeeping, barriers) is shared by two points.  The sweep is
// limited by instruction issue at one point per thread; the arithmetic and
// its order are those of the one-point sweep (OpCiSweep::combine), so the
// results are bitwise the same.  Needs the TMA ring (row pitch a multiple of
// 8): pair addresses are 2-element aligned, and a pair that straddles the
// grid's x end (nx odd) writes its right value into the row's padding.
// ------------------------------------------------------------------------
template <class Op>
__device__ __forceinline__ void march_tma_wide(Op &op, const Desc &D, int tile, int kb, int ke,
                                               unsigned char *ring, uint64_t *bars, uint32_t &seq, int *s_dead)
{
    using R = Ring<Op>;
    constexpr int S = R::STAGES;
    constexpr int W = R::W;
    constexpr int PX = TILE_X / 2; // point pairs along x
    static_assert(S >= 6, "one CTA barrier per two planes needs six or more stages");
    static_assert(Op::NH == 1 && (Op::NP == 0 || Op::NP == 2) && (R::HX % 2) == 0 && (W % 2) == 0,
                  "one halo operand, pair alignment");

    const int nx = D.nx, ny = D.ny;
    const int plane = D.px * ny;
    const int tid = threadIdx.x, tx = tid % PX, ty = tid / PX;
    const int i0 = (tile % D.tiles_x) * TILE_X, j0 = (tile / D.tiles_x) * TILE_Y;
    const int i = i0 + 2 * tx, j = j0 + ty;
    // with nx odd the pair (nx - 1, nx) stores its right value into column
    // nx, which the pitch (a multiple of 8) holds as padding and no one reads
    // as a grid value (the tensor maps end at nx and read zeros beyond it)
    const bool in = (i < nx) && (j < ny);
    const int col = in ? j * D.px + i : 0;
    const int me = (ty + 1) * W + R::HX + 2 * tx; // left point of the pair in a halo box (even)
    const int mp = ty * TILE_X + 2 * tx;          // the same in a plain box (even)
    const int q0 = kb - 1, q1 = ke;
    const int nplanes = q1 - q0 + 1;
    const uint32_t seq0 = seq;

    struct Slot {
        int st;
        uint32_t par;
        __device__ __forceinline__ void next()
        {
            if (++st == S) {
                st = 0;
                par ^= 1u;
            }
        }
    };
    Slot sm{(int)(seq0 % S), (seq0 / S) & 1u}; // plane k-1
    Slot sc = sm;
    sc.next(); // plane k
    Slot sn = sc;
    sn.next(); // plane k+1
    auto stage = [&](int st) { return ring + st * R::STAGE; };
    auto wait = [&](const Slot &sl) {
        if (*s_dead) return;
        if (!mbar_wait(bars + sl.st, sl.par)) {
            *s_dead = 1;
            D.sc->status = ST_TIMEOUT;
            D.sc->stop = 1;
        }
    };
    // Thread 0, after a CTA barrier that ends every read of the stages of
    // planes nref..p: refill each with the plane S further on (planes beyond
    // q1 are never issued).  Plane n of this march lives in stage (seq0 + n -
    // q0) % S.  Step k reads plane k's stage and the centre pair of plane k+1,
    // so the stages of the planes up to k are free after step k, and S - 2
    // planes are in flight ahead of the one waited for.
    int nref = q0;
    auto refill_upto = [&](int p) {
        for (; nref <= p; ++nref) {
            const int q = nref + S;
            const int st = (int)((seq0 + (uint32_t)(nref - q0)) % S);
            if (q <= q1 && !*s_dead) ring_issue<Op>(op, D, stage(st), bars + st, i0, j0, q, q >= kb && q < ke);
        }
    };

    __syncthreads(); // the previous run's readers of the ring are done
    if (tid == 0) {
        Slot si = sm;
        for (int n = 0; n < S && n < nplanes; ++n) {
            const int q = q0 + n;
            ring_issue<Op>(op, D, stage(si.st), bars + si.st, i0, j0, q, q >= kb && q < ke);
            si.next();
        }
    }
    wait(sm);
    wait(sc);
    float2 zdn = in ? op.ld2(stage(sm.st), me) : make_float2(0.f, 0.f); // centre pairs of planes k-1, k
    float2 zc = in ? op.ld2(stage(sc.st), me) : make_float2(0.f, 0.f);

    for (int k = kb; k < ke; ++k) {
        wait(sn);
        float2 zup = make_float2(0.f, 0.f);
        if (in && !*s_dead) {
            const unsigned char *hs = stage(sc.st);
            const unsigned char *ps = hs + R::HSTRIDE;
            zup = op.ld2(stage(sn.st), me);
            const float w = op.ld1(hs, me - 1), e = op.ld1(hs, me + 2);
            const float2 so = op.ld2(hs, me - W), no = op.ld2(hs, me + W);
            float2 b = make_float2(0.f, 0.f), z = b;
            if constexpr (Op::NP == 2) { // sweeps k >= 2: b and y_(k-2)
                b = op.ld2(ps, mp);
                if (op.k >= 3) z = op.ld2(ps + R::PSTRIDE, mp);
            }
            op.emit2(col + k * plane, zc, make_float2(w + zc.y, zc.x + e), make_float2(so.x + no.x, so.y + no.y),
                     make_float2(zdn.x + zup.x, zdn.y + zup.y), b, z);
        }
        if ((k - kb) & 1) {
            // one CTA barrier per two planes: the stages of the planes up to k
            // are free and their refills go out in plane order; plane k+1,
            // waited for at the top of step k, went out at the barrier after
            // step k-S+1 or k-S+2, at least four planes ahead with S = 6
            // (measured 59.7 -> 57.4 us per 256^3 FP32 sweep against refilling
            // one step later; the one-point FP64 sweep measured slower that
            // way, 234 -> 242 us, and keeps the later refill)
            __syncthreads();
            if (tid == 0) refill_upto(k);
        }
        sm = sc;
        sc = sn;
        sn.next();
        zdn = zc;
        zc = zup;
    }
    seq = seq0 + nplanes;
}

// Whether an operation is a wide sweep, and the CTA size of its kernel.
template <class Op, class = void>
struct IsWide {
    static constexpr bool value = false;
};
template <class Op>
struct IsWide<Op, std::void_t<decltype(Op::WIDE)>> {
    static constexpr bool value = Op::WIDE;
};
template <class Op>
constexpr int op_threads()
{
    return IsWide<Op>::value ? NTHREADS / 2 : NTHREADS;
}

// Whether an operation is a pair of Chebyshev sweeps in one pass
// (OpCiSweepPairW, march_pair_wide, defined with the operations below).
template <class Op, class = void>
struct IsPair {
    static constexpr bool value = false;
};
template <class Op>
struct IsPair<Op, std::void_t<decltype(Op::PAIR)>> {
    static constexpr bool value = Op::PAIR;
};
template <class Op>
__device__ __forceinline__ void march_pair_wide(Op &op, const Desc &D, int tile, int kb, int ke,
                                                unsigned char *ring, uint64_t *bars, uint32_t &seq, int *s_dead);

// ------------------------------------------------------------------------
// The generic kernel: take units from the launch list until it is exhausted.
// ------------------------------------------------------------------------
// Shared-memory state of a CTA, reused by every phase a CTA runs.
struct EngineShared {
    double *sred;          // block-reduction scratch
    uint64_t *bars;        // TMA ring mbarriers (MAX_STAGES)
    int *s_last, *s_dead;
    int *s_unit;           // the unit thread 0 took
    unsigned char *dyn;    // TMA ring / general-engine planes
    uint32_t seq;          // planes this CTA has staged so far (all threads agree)
};

constexpr int MAX_STAGES = 8;

// One phase.  Each CTA starts with the unit of its own index and then takes
// units one at a time from the list's counter, so a unit goes to whichever
// CTA is free first and no SM idles while another still holds a queue of
// units; units are handed out in increasing order,
// chunk-major within a problem, so the CTAs running at one time cover
// neighbouring tiles at nearby z and the halo rows one CTA reads are still
// in L2 when its neighbours read them.  A problem's dot products are summed
// per unit, and the CTA that completes its last unit (atomic ticket) reduces
// the per-unit partials in unit order, so results do not depend on which CTA
// took which unit.
template <class Op>
__device__ __forceinline__ void engine_body(const KArgs &a, EngineShared &sh)
{
    using C = typename Op::C;
    C *sp = reinterpret_cast<C *>(sh.dyn);

    const ListHdr hdr = *reinterpret_cast<const ListHdr *>(a.list);
    const int2 *ent = reinterpret_cast<const int2 *>(a.list + LIST_HDR_INTS);
    uint32_t *sched = reinterpret_cast<uint32_t *>(const_cast<int32_t *>(a.list)) + 2; // next, done
    const int G = gridDim.x;
    // A stencil operation without dot products may split every work unit into
    // S sub-units of consecutive planes (finer scheduling at the end of a
    // launch); dot products keep whole units (their partials are per unit).
    const int S = (Op::STENCIL && Op::ND == 0 && a.split > 1) ? a.split : 1;
    const int total = hdr.total * S;
    // the first unit of a CTA is its index; the rest come from the counter
    // (never touched when the list has no more units than the launch has CTAs)
    const bool dynamic = total > G;
    int u = blockIdx.x;
    int e = 0; // list entry of the last unit taken
    while (u < total) {
        const int ub = S > 1 ? u / S : u; // the work unit
        if (e + 1 < hdr.n && ent[e + 1].y <= ub) { // the last entry whose first unit <= ub
            int lo = e + 1, hi = hdr.n - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (ent[mid].y <= ub) lo = mid;
                else hi = mid - 1;
            }
            e = lo;
        }
        const int2 en = ent[e];
        const Desc &D = a.descs[en.x];
        Scal *sc = D.sc;
        const bool skip = ((a.skip & SKIP_STOP) && ld_flag(&sc->stop)) ||
                          ((a.skip & SKIP_HALF) && ld_flag(&sc->half)) ||
                          ((a.skip & SKIP_NOT_RR) && (D.rr_every <= 0 || ld_flag(&sc->iter) % D.rr_every != 0));
        if (!skip) {
            Op op(D, a, sc);
            const int ntiles = D.tiles_x * D.tiles_y;
            const int l = ub - en.y; // problem-local unit, chunk-major
            const int c0 = l / ntiles;
            const int tile = l - c0 * ntiles;
            if constexpr (Op::STENCIL) {
                int kb = c0 * D.zc, ke = min(D.nz, kb + D.zc);
                if (S > 1) { // sub-unit u - ub S of the unit's planes
                    const int part = (D.zc + S - 1) / S;
                    kb += (u - ub * S) * part;
                    ke = min(ke, kb + part);
                }
                if (kb < ke) {
                    if constexpr (IsPair<Op>::value) {
                        // the host runs paired sweeps only on lists of TMA problems
                        if (D.tma) march_pair_wide<Op>(op, D, tile, kb, ke, sh.dyn, sh.bars, sh.seq, sh.s_dead);
                        else if (threadIdx.x == 0) stop_with(sc, ST_INTERNAL);
                    } else if constexpr (IsWide<Op>::value) {
                        // the host runs wide sweeps only on lists of TMA problems
                        if (D.tma) march_tma_wide<Op>(op, D, tile, kb, ke, sh.dyn, sh.bars, sh.seq, sh.s_dead);
                        else if (threadIdx.x == 0) stop_with(sc, ST_INTERNAL);
                    } else if (D.tma) {
                        march_tma<Op>(op, D, tile, c0, kb, ke, sh.dyn, sh.bars, sh.seq, sh.sred, sh.s_dead);
                    } else {
                        march_stencil<Op>(op, D, tile, c0, kb, ke, sp, sh.sred);
                    }
                }
            } else {
                march_point<Op>(op, D, tile, c0, c0 + 1, sh.sred);
            }
            if constexpr (Op::ND > 0) {
                const int units = D.units;
                __syncthreads();
                if (threadIdx.x == 0) {
                    __threadfence();
                    const unsigned prev = atomicAdd(&sc->ticket, 1u);
                    *sh.s_last = (prev + 1u == (unsigned)units);
                }
                __syncthreads();
                if (*sh.s_last) {
                    __threadfence();
                    double v[Op::ND];
#pragma unroll
                    for (int q = 0; q < Op::ND; ++q) v[q] = 0.0;
                    for (int w = threadIdx.x; w < units; w += NTHREADS) {
#pragma unroll
                        for (int q = 0; q < Op::ND; ++q) v[q] += __ldcg(D.partials + w * MAX_DOTS + q);
                    }
                    block_sum<Op::ND>(v, sh.sred);
                    if (threadIdx.x == 0) {
                        epilogue<Op::EPI, Op::ND>(D, sc, v);
                        sc->ticket = 0;
                        __threadfence();
                    }
                }
                __syncthreads(); // s_last is reused by the next unit
            }
        }
        if (!dynamic) break;
        if (threadIdx.x == 0) *sh.s_unit = G + (int)atomicAdd(&sched[0], 1u);
        __syncthreads();
        u = *sh.s_unit;
        __syncthreads(); // every thread has read s_unit before thread 0 takes the next unit
    }
    // The last CTA to finish resets the counters for the next launch on this
    // list (no CTA of this launch touches them after its own last take).
    if (dynamic && threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&sched[1], 1u) == (unsigned)G - 1u) {
            atomicExch(&sched[0], 0u);
            atomicExch(&sched[1], 0u);
            __threadfence();
        }
    }
}

// Initialise the CTA's shared state (mbarriers of the TMA ring).
__device__ __forceinline__ void engine_setup(EngineShared &sh, double *sred, uint64_t *bars, int *s_last,
                                             int *s_dead, int *s_unit, unsigned char *dyn)
{
    sh.sred = sred;
    sh.bars = bars;
    sh.s_last = s_last;
    sh.s_dead = s_dead;
    sh.s_unit = s_unit;
    sh.dyn = dyn;
    sh.seq = 0;
    if (threadIdx.x == 0) {
        for (int b = 0; b < MAX_STAGES; ++b) mbar_init(&bars[b], 1);
        mbar_init_fence();
        *s_dead = 0;
    }
    __syncthreads();
}

// Resident CTAs per SM a kernel is compiled for: 4 (64 registers a thread),
// or the operation's MIN_BLOCKS when it fits in fewer registers without
// spilling (more warps to hide the ring's latency).
template <class Op, class = void>
struct MinBlocks {
    static constexpr int value = 4;
};
template <class Op>
struct MinBlocks<Op, std::void_t<decltype(Op::MIN_BLOCKS)>> {
    static constexpr int value = Op::MIN_BLOCKS;
};

template <class Op>
__global__ void __launch_bounds__(op_threads<Op>(), MinBlocks<Op>::value) k_engine(KArgs a)
{
    __shared__ double sred[(NTHREADS / 32) * MAX_DOTS];
    __shared__ alignas(8) uint64_t bars[MAX_STAGES];
    __shared__ int s_last, s_dead, s_unit;
    // the TMA ring, or the general engine's double-buffered plane: a CTA runs
    // one engine at a time, and each march starts with a barrier
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    EngineShared sh;
    engine_setup(sh, sred, bars, &s_last, &s_dead, &s_unit, dyn_smem);
    engine_body<Op>(a, sh);
}

// Dynamic shared memory a launch of k_engine<Op> needs.
template <class Op>
constexpr int engine_dyn_smem()
{
    if constexpr (IsPair<Op>::value) {
        return Op::DYN_BYTES; // its stages and the y_k planes
    } else if constexpr (IsWide<Op>::value) {
        return Ring<Op>::BYTES; // TMA ring only
    } else if constexpr (Op::STENCIL) {
        constexpr int lsu = 2 * (TILE_X + 2) * (TILE_Y + 2) * (int)sizeof(typename Op::C);
        return Ring<Op>::BYTES > lsu ? Ring<Op>::BYTES : lsu;
    } else {
        return 0;
    }
}

// ------------------------------------------------------------------------
// Operations.
// ------------------------------------------------------------------------
struct NoPW {};

// A u = cc u - cx sx - cy sy - cz sz: 1 multiply + 3 fused multiply-adds.
template <class C>
__device__ __forceinline__ C apply_A_terms(C cc, C cx, C cy, C cz, C u, C sx, C sy, C sz)
{
    return fma(-cz, sz, fma(-cy, sy, fma(-cx, sx, cc * u)));
}

// Chebyshev sweep 1 (Algorithm 2, first two steps) on a right-hand side u
// that is itself formed point by point from FP64 vectors:
//   SIDE_P: u = p_{i-1} = r + beta (p_{i-2} - omega w)   (Alg. 1, last line;
//           u = r on the first iteration)
//   SIDE_S: u = s = r - alpha w                          (Alg. 1) and ||s||^2
// It writes u (FP64), the CI copy of u rounded to T (mixed precision only),
// and z = u/theta (degree 0) or y_1 = (2 rho_1/delta)(2u - A u/theta).
// UNIT (FP64, degree >= 2): y_1 is stored divided by its (positive)
// coefficient of the x-pair sum, which then enters with coefficient 1 (6
// FP64 instructions instead of 7; the sweeps take the scale into account,
// see OpCiSweep).
constexpr int SIDE_P = 0, SIDE_S = 1;
template <class T, bool BLK, int SIDE, bool UNIT = false>
struct OpCiFirst {
    using E = Elem<T>;
    using C = typename E::C;
    using U = double;
    using PW = NoPW;
    static constexpr int ND = SIDE == SIDE_S ? 1 : 0;
    static constexpr int EPI = SIDE == SIDE_S ? EPI_SNORM : EPI_NONE;
    static constexpr bool STENCIL = true, BLOCKED = BLK;
    static constexpr bool MIXED = !std::is_same<T, double>::value;
    static_assert(!UNIT || !MIXED, "scaled iterates are FP64 only");
    // staged form: halo boxes of r (and w, p_{i-2}); u is formed once per plane
    using TH = double;
    using TP = double;
    static constexpr int NH = SIDE == SIDE_S ? 2 : 3, NP = 0;
    static constexpr bool XFORM = true;
    int nh, np, hrole[NH], prole[1];
    const double *r, *pold, *w;
    double *uout;
    void *bc, *out;
    double beta, omega, alpha;
    int first, degree;
    C tinv, a_u, a_x, a_y, a_z;
    __device__ OpCiFirst(const Desc &D, const KArgs &a, Scal *sc)
    {
        const int iter = ld_flag(&sc->iter);
        r = (const double *)D.vec[ROLE_R];
        w = (const double *)D.vec[ROLE_W];
        pold = (const double *)D.vec[resolve_role(ROLE_POLD, iter)];
        first = ld_flag(&sc->first);
        np = 0;
        prole[0] = 0;
        hrole[0] = ROLE_R;
        if constexpr (SIDE == SIDE_S) {
            nh = 2;
            hrole[1] = ROLE_W;
        } else {
            nh = first ? 1 : 3;
            hrole[1] = resolve_role(ROLE_POLD, iter);
            hrole[2] = ROLE_W;
        }
        uout = (double *)D.vec[resolve_role(a.in, iter)];
        bc = D.vec[ROLE_BC];
        out = D.vec[a.out];
        beta = ld_scal(&sc->beta);
        omega = ld_scal(&sc->omega);
        alpha = ld_scal(&sc->alpha);
        degree = D.degree;
        tinv = (C)D.theta_inv;
        // y_1 = (2 rho_1/delta)(2u - A u / theta)
        //     = c (2 - cc/theta) u + (c/theta)(cx sx + cy sy + cz sz),  c = 2 rho_1/delta
        // (folded on the host)
        a_u = (C)D.ci1[0];
        a_x = (C)D.ci1[1];
        a_y = (C)D.ci1[2];
        a_z = (C)D.ci1[3];
    }
    __device__ __forceinline__ double load(int idx) const
    {
        if constexpr (SIDE == SIDE_S) {
            return gld(r + idx) - alpha * gld(w + idx);
        } else {
            if (first) return gld(r + idx);
            return gld(r + idx) + beta * (gld(pold + idx) - omega * gld(w + idx));
        }
    }
    __device__ __forceinline__ double load_s(const void *const *h, int x) const
    {
        if constexpr (SIDE == SIDE_S) {
            return Elem<double>::lds(h[0], x) - alpha * Elem<double>::lds(h[1], x);
        } else {
            if (first) return Elem<double>::lds(h[0], x);
            return Elem<double>::lds(h[0], x) +
                   beta * (Elem<double>::lds(h[1], x) - omega * Elem<double>::lds(h[2], x));
        }
    }
    __device__ __forceinline__ C sv(double u) const { return (C)E::round(u); }
    __device__ __forceinline__ PW pw(bool, int) const { return PW{}; }
    __device__ __forceinline__ PW pw_s(const void *const *, int) const { return PW{}; }
    template <int NA>
    __device__ __forceinline__ void emit(int idx, C b, C sx, C sy, C sz, double uc, const PW &,
                                         double (&acc)[NA]) const
    {
        uout[idx] = uc;
        if constexpr (SIDE == SIDE_S) acc[0] += uc * uc;
        if constexpr (MIXED) E::st(bc, idx, b);
        if constexpr (UNIT) E::st(out, idx, fma(a_z, sz, fma(a_y, sy, fma(a_u, b, sx))));
        else if (degree == 0) E::st(out, idx, b * tinv);
        else E::st(out, idx, fma(a_z, sz, fma(a_y, sy, fma(a_x, sx, a_u * b))));
    }
};

// Mixed precision (FP32 / BF16 Chebyshev vectors): CI sweep 1 in two passes.
// The fused OpCiFirst forms the FP64 right-hand side u on every cell of its
// halo box (40 % more FP64 work than points) and rounds it there; in the
// mixed solve that FP64 work and the transform pass bound it.  Here a
// pointwise pass forms u once per point in FP64 and stores it together with
// its rounding to the Chebyshev type (the CI right-hand side b_c the sweeps
// read anyway), and sweep 1 then reads b_c as its stencil input.  The values
// are those of OpCiFirst: the same expression for u, the same rounding, and
// the same FP32 expression for y_1 on the rounded values; the extra traffic is
// one read of b_c.

// p_{i-1} = r + beta (p_{i-2} - omega w)  (p = r on the first iteration) into
// the current p buffer, and b_c = p_{i-1} rounded (Algorithm 1, last line).
template <class T>
struct OpDirUpdate {
    using C = double;
    using E = Elem<T>;
    static constexpr int ND = 0, EPI = EPI_NONE;
    static constexpr bool STENCIL = false;
    const double *r, *pold, *w;
    double *p;
    void *bc;
    double beta, omega;
    int first;
    __device__ OpDirUpdate(const Desc &D, const KArgs &a, Scal *sc)
    {
        const int iter = ld_flag(&sc->iter);
        r = (const double *)D.vec[ROLE_R];
        w = (const double *)D.vec[ROLE_W];
        pold = (const double *)D.vec[resolve_role(ROLE_POLD, iter)];
        p = (double *)D.vec[resolve_role(a.in, iter)];
        bc = D.vec[ROLE_BC];
        beta = ld_scal(&sc->beta);
        omega = ld_scal(&sc->omega);
        first = ld_flag(&sc->first);
    }
    struct In { double r, p, w; };
    __device__ __forceinline__ In load(int idx) const
    {
        In v{};
        v.r = gld(r + idx);
        if (!first) {
            v.p = gld(pold + idx);
            v.w = gld(w + idx);
        }
        return v;
    }
    template <int NA>
    __device__ __forceinline__ void apply(int idx, const In &v, double (&)[NA]) const
    {
        // the expression OpCiFirst<T, BLK, SIDE_P>::load evaluates
        const double u = first ? v.r : v.r + beta * (v.p - omega * v.w);
        p[idx] = u;
        E::st(bc, idx, E::round(u));
    }
};

// s = r - alpha w with ||s||^2 (Algorithm 1, half step) and b_c = s rounded.
template <class T>
struct OpHalfStep {
    using C = double;
    using E = Elem<T>;
    static constexpr int ND = 1, EPI = EPI_SNORM;
    static constexpr bool STENCIL = false;
    const double *r, *w;
    double *s;
    void *bc;
    double alpha;
    __device__ OpHalfStep(const Desc &D, const KArgs &, Scal *sc)
    {
        r = (const double *)D.vec[ROLE_R];
        w = (const double *)D.vec[ROLE_W];
        s = (double *)D.vec[ROLE_S];
        bc = D.vec[ROLE_BC];
        alpha = ld_scal(&sc->alpha);
    }
    struct In { double r, w; };
    __device__ __forceinline__ In load(int idx) const { return In{gld(r + idx), gld(w + idx)}; }
    template <int NA>
    __device__ __forceinline__ void apply(int idx, const In &v, double (&acc)[NA]) const
    {
        const double u = v.r - alpha * v.w; // as OpCiFirst<T, BLK, SIDE_S>::load
        s[idx] = u;
        acc[0] += u * u;
        E::st(bc, idx, E::round(u));
    }
};

// CI sweep 1 (Algorithm 2, first two steps) on the rounded right-hand side
// b_c written by OpDirUpdate / OpHalfStep: y_1 = (2 rho_1/delta)(2u - A u/theta)
// in the Chebyshev type's arithmetic, or z = u/theta for degree 0, with the
// coefficients OpCiFirst uses (folded on the host).  One point per thread,
// either engine, block restriction and Neumann faces as the sweeps.
template <class T, bool BLK>
struct OpCiFirstC {
    using E = Elem<T>;
    using C = typename E::C;
    using U = C;
    using PW = NoPW;
    static constexpr int ND = 0, EPI = EPI_NONE;
    static constexpr bool STENCIL = true, BLOCKED = BLK;
    static_assert(!std::is_same<T, double>::value, "the two-pass sweep 1 is the mixed-precision form");
    using TH = T;
    using TP = T;
    static constexpr int NH = 1, NP = 0;
    static constexpr bool XFORM = false;
    int nh = 1, np = 0, hrole[NH], prole[1];
    const void *u;
    void *out;
    int degree;
    C tinv, a_u, a_x, a_y, a_z;
    __device__ OpCiFirstC(const Desc &D, const KArgs &a, Scal *)
    {
        u = D.vec[ROLE_BC];
        out = D.vec[a.out];
        hrole[0] = ROLE_BC;
        prole[0] = 0;
        degree = D.degree;
        tinv = D.theta_inv_f; // FP32 copies rounded on the host
        a_u = D.ci1f[0];
        a_x = D.ci1f[1];
        a_y = D.ci1f[2];
        a_z = D.ci1f[3];
    }
    __device__ __forceinline__ C load(int idx) const { return E::ld(u, idx); }
    __device__ __forceinline__ C load_s(const void *const *h, int x) const { return E::lds(h[0], x); }
    __device__ __forceinline__ C sv(C v) const { return v; }
    __device__ __forceinline__ PW pw(bool, int) const { return PW{}; }
    __device__ __forceinline__ PW pw_s(const void *const *, int) const { return PW{}; }
    // the expression of OpCiFirst::emit (non-scaled form)
    __device__ __forceinline__ C combine(C b, C sx, C sy, C sz) const
    {
        if (degree == 0) return b * tinv;
        return fma(a_z, sz, fma(a_y, sy, fma(a_x, sx, a_u * b)));
    }
    template <int NA>
    __device__ __forceinline__ void emit(int idx, C b, C sx, C sy, C sz, C, const PW &, double (&)[NA]) const
    {
        E::st(out, idx, combine(b, sx, sy, sz));
    }
};

// Chebyshev sweep k >= 2 (Algorithm 2 loop body):
//   w = rho_k (2 sigma y + (2/delta)(b - A y) - rho_{k-1} z),
// y = y_{k-1} (stencil input), z = y_{k-2} (z = b/theta when k = 2).
// TB is the storage type of the CI right-hand side b.
//
// Scaled iterates (FP64 vectors only).  Written out, w is a combination of
// b, z and the three neighbour-pair sums of y; each coefficient costs one
// FP64 instruction, and the FP64 pipe bounds this kernel.  The intermediate
// iterates are therefore stored as yhat_j = y_j / s_j with s_j = the
// coefficient of b in sweep j (2 <= j <= d), so that b enters with
// coefficient exactly 1 and the sweep saves its multiply (UNIT); y_1 is
// stored divided by its x-pair coefficient (OpCiFirst).  The last iterate
// y_d (p^ or r^) is stored the same way, divided by Desc::hat, which its
// readers never need (see OpStencilDot), so every sweep is in the
// 7-instruction form.  The other coefficients take the ratios of the scales
// (problem_set_cheb folds them), and s_j > 0 is a fixed per-sweep number (no
// accumulated product), so the iterates stay in range.
// A sweep compiled without UNIT computes the same values (its b coefficient
// is then c/c = 1).
// K2: the sweep k = 2 only, compiled without the y_{k-2} term (its coefficient
// and operand are zero at k = 2, but with k known only at run time the term
// costs an FMA on the FP64 pipe per point: 7 FP64 instructions instead of 6).
template <class T, class TB, bool BLK, bool WITH_Y = true, bool NEU = true, bool UNIT = false, bool K2 = false>
struct OpCiSweep {
    using E = Elem<T>;
    using EB = Elem<TB>;
    using C = typename E::C;
    using U = C;
    struct PW { C b, z; };
    static constexpr int ND = 0, EPI = EPI_NONE;
    static constexpr bool STENCIL = true, BLOCKED = BLK;
    static_assert(sizeof(TB) == sizeof(T), "CI right-hand side and iterates share one type");
    // without block restriction the FP32/BF16 sweep fits 40 registers: 6 CTAs
    // per SM hide more of the ring's latency (FP32 sweep 79 -> 71 us at 256^3);
    // the FP64 sweep is bound by the FP64 pipe and measured slower at 5 (48
    // registers), so it keeps 4
    static constexpr int MIN_BLOCKS = (BLK || sizeof(T) == 8) ? 4 : 6;
    // NEU = false: the grid has no Neumann face, and the sweep is compiled
    // without the face handling (the FP64 sweep is at its register budget)
    static constexpr bool NEUMANN = NEU;
    static constexpr bool SCALED = std::is_same<T, double>::value;
    static_assert(SCALED || !UNIT, "scaled iterates are FP64 only");
    // staged form: halo box of y_{k-1}, plain boxes of b and y_{k-2}
    using TH = T;
    using TP = T;
    static constexpr int NH = 1, NP = 2;
    static constexpr bool XFORM = false;
    int nh, np, hrole[NH], prole[NP];
    const void *y, *bv, *zv;
    void *out;
    C c_y, c_b, c_z, c_x, c_yy, c_zz;
    int k;
    __device__ OpCiSweep(const Desc &D, const KArgs &a, Scal *sc)
    {
        const int iter = ld_flag(&sc->iter);
        y = D.vec[a.in];
        bv = D.vec[resolve_role(a.b, iter)];
        zv = D.vec[a.z];
        out = D.vec[a.out];
        k = a.k;
        nh = 1;
        hrole[0] = a.in;
        np = (!K2 && a.k >= 3) ? 2 : 1;
        prole[0] = resolve_role(a.b, iter);
        prole[1] = a.z;
        // w = rho_k (2 sigma y + (2/delta)(b - A y) - rho_{k-1} z) with A y expanded:
        //   = rho_k (2 sigma - (2/delta) cc) y + rho_k (2/delta) b - rho_k rho_{k-1} z
        //     + rho_k (2/delta)(cx sx + cy sy + cz sz);  z = b/theta when k = 2
        // the coefficients, scaled as above, come folded from the host (the
        // operation is built per work unit by every thread: computing them
        // here cost the FP64 pipe several percent of the sweep).  WITH_Y =
        // false: exact closed-form bounds, where lambda_min + lambda_max = 2 cc
        // (Eq. 9: sin^2 a + cos^2 a = 1 per axis, for the grid and for every
        // block), so theta = cc and the y coefficient vanishes; the kernel
        // then skips its multiply.
        if constexpr (std::is_same<C, float>::value) { // rounded on the host (Desc::cikf)
            const float *ck = D.cikf[a.k];
            c_y = ck[0];
            c_b = ck[1];
            c_z = ck[2];
            c_x = ck[3];
            c_yy = ck[4];
            c_zz = ck[5];
        } else {
            const double *ck = D.cik[a.k];
            c_y = ck[0];
            c_b = ck[1];
            c_z = ck[2];
            c_x = ck[3];
            c_yy = ck[4];
            c_zz = ck[5];
        }
    }
    __device__ __forceinline__ C load(int idx) const { return E::ld(y, idx); }
    __device__ __forceinline__ C load_s(const void *const *h, int x) const { return E::lds(h[0], x); }
    __device__ __forceinline__ C sv(C u) const { return u; }
    __device__ __forceinline__ PW pw(bool valid, int idx) const
    {
        PW p{C(0), C(0)};
        if (valid) {
            p.b = (C)EB::ld(bv, idx);
            if (!K2 && k >= 3) p.z = E::ld(zv, idx);
        }
        return p;
    }
    __device__ __forceinline__ PW pw_s(const void *const *p, int x) const
    {
        PW v{(C)EB::lds(p[0], x), C(0)};
        if (!K2 && k >= 3) v.z = E::lds(p[1], x);
        return v;
    }
    // the new iterate at one point from its centre value, neighbour-pair sums,
    // b and z
    __device__ __forceinline__ C combine(C yc, C sx, C sy, C sz, C b, C z) const
    {
        C v;
        if constexpr (UNIT && WITH_Y) v = fma(c_y, yc, b);
        else if constexpr (UNIT) v = b;
        else if constexpr (WITH_Y) v = fma(c_b, b, c_y * yc);
        else v = c_b * b;
        if constexpr (!K2)
            if (k >= 3) v = fma(c_z, z, v);
        return fma(c_zz, sz, fma(c_yy, sy, fma(c_x, sx, v)));
    }
    template <int NA>
    __device__ __forceinline__ void emit(int idx, C yc, C sx, C sy, C sz, C, const PW &p, double (&)[NA]) const
    {
        E::st(out, idx, combine(yc, sx, sy, sz, p.b, p.z));
    }
};

// Pairs of x-adjacent Chebyshev-vector elements (wide sweeps): FP32 math on
// FP32 or BF16 storage, element index even.
template <class T> struct Pair;
template <> struct Pair<float> {
    static __device__ __forceinline__ float2 lds(const void *p, int x)
    {
        return *reinterpret_cast<const float2 *>(reinterpret_cast<const float *>(p) + x);
    }
    static __device__ __forceinline__ float lds1(const void *p, int x) { return reinterpret_cast<const float *>(p)[x]; }
    static __device__ __forceinline__ void st(void *p, int x, float2 v)
    {
        *reinterpret_cast<float2 *>(reinterpret_cast<float *>(p) + x) = v;
    }
};
template <> struct Pair<__nv_bfloat16> {
    static __device__ __forceinline__ float2 lds(const void *p, int x)
    {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(reinterpret_cast<const __nv_bfloat16 *>(p) + x));
    }
    static __device__ __forceinline__ float lds1(const void *p, int x)
    {
        return __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(p)[x]);
    }
    static __device__ __forceinline__ void st(void *p, int x, float2 v)
    {
        // each element rounded to nearest even, as Elem<__nv_bfloat16>::st does
        *reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<__nv_bfloat16 *>(p) + x) = __floats2bfloat162_rn(v.x, v.y);
    }
};

// Chebyshev sweep k >= 2 with FP32 or BF16 vectors on the whole grid (no block
// restriction, no Neumann face), two x-adjacent points per thread
// (march_tma_wide; 128 threads per CTA).  Same coefficients, arithmetic and
// results as OpCiSweep<T, T, false, WY, false>.
template <class T, bool WY>
struct OpCiSweepW : OpCiSweep<T, T, false, WY, false, false> {
    using Base = OpCiSweep<T, T, false, WY, false, false>;
    static_assert(std::is_same<typename Base::C, float>::value, "wide sweeps are the FP32-math forms");
    static constexpr bool WIDE = true;
    // 64 registers a thread at 8 CTAs of 128 threads per SM; six ring stages
    // (22 KB with FP32 vectors) let that many CTAs fit in shared memory
    static constexpr int MIN_BLOCKS = 8;
    static constexpr int RING_STAGES = 6;
    __device__ OpCiSweepW(const Desc &D, const KArgs &a, Scal *sc) : Base(D, a, sc) {}
    __device__ __forceinline__ float2 ld2(const void *p, int x) const { return Pair<T>::lds(p, x); }
    __device__ __forceinline__ float ld1(const void *p, int x) const { return Pair<T>::lds1(p, x); }
    __device__ __forceinline__ void emit2(int idx, float2 yc, float2 sx, float2 sy, float2 sz, float2 b,
                                          float2 z) const
    {
        Pair<T>::st(this->out, idx,
                    make_float2(this->combine(yc.x, sx.x, sy.x, sz.x, b.x, z.x),
                                this->combine(yc.y, sx.y, sy.y, sz.y, b.y, z.y)));
    }
};

// CI sweep 1 on b_c with two x-adjacent points per thread (march_tma_wide;
// whole grid, no Neumann face, TMA ring): the values of OpCiFirstC.
template <class T>
struct OpCiFirstCW : OpCiFirstC<T, false> {
    using Base = OpCiFirstC<T, false>;
    static constexpr bool WIDE = true;
    static constexpr bool NEUMANN = false;
    // one FP32 halo box per stage (1.7 KB): eight stages, and 8 CTAs of 128
    // threads per SM at 64 registers
    static constexpr int MIN_BLOCKS = 8;
    static constexpr int RING_STAGES = 8;
    __device__ OpCiFirstCW(const Desc &D, const KArgs &a, Scal *sc) : Base(D, a, sc) {}
    __device__ __forceinline__ float2 ld2(const void *p, int x) const { return Pair<T>::lds(p, x); }
    __device__ __forceinline__ float ld1(const void *p, int x) const { return Pair<T>::lds1(p, x); }
    __device__ __forceinline__ void emit2(int idx, float2 yc, float2 sx, float2 sy, float2 sz, float2, float2) const
    {
        Pair<T>::st(this->out, idx,
                    make_float2(this->combine(yc.x, sx.x, sy.x, sz.x), this->combine(yc.y, sx.y, sy.y, sz.y)));
    }
};

// A value of FP32 arithmetic as the storage type T holds it (read back as FP32).
template <class T>
__device__ __forceinline__ float E_round(float v)
{
    if constexpr (std::is_same<T, float>::value) return v;
    else return __bfloat162float(__float2bfloat16_rn(v));
}
// ------------------------------------------------------------------------
// Temporal blocking of the Chebyshev sweeps (FP32/BF16 vectors, G(CI) on the
// TMA ring): sweeps k and k+1 in one pass over the grid.  Algorithm 2's
// recurrence is reduction-free, so sweep k+1 can follow sweep k plane by
// plane: y_k is computed on the tile and a one-cell ring around it (34 x 10
// cells), from y_{k-1} staged with a two-cell halo in y (and the aligned
// four-cell halo in x), then y_{k+1} on the tile from the last three planes
// of y_k held in shared memory.  One pass reads y_{k-1}, b and y_{k-2} and
// writes y_k and y_{k+1}: 5 vector accesses for two sweeps instead of 8.  The
// values are those of two single sweeps: each y_k is rounded to the storage
// type before sweep k+1 reads it, outside-grid cells of y_k are the zero
// ghosts, and every expression is OpCiSweep::combine.  y_k and y_{k+1} go to
// buffers that neither input occupies (the inputs are read with a halo by
// neighbouring tiles, so nothing is overwritten in place).
// KArgs: k (the first sweep), in = y_{k-1}, z = y_{k-2} (k >= 3), b = b_c,
// out = y_k, aux = y_{k+1}.
// ------------------------------------------------------------------------
template <class T, bool WY>
struct OpCiSweepPairW {
    using E = Elem<T>;
    using C = float;
    using U = C;
    using PW = NoPW;
    static_assert(!std::is_same<T, double>::value, "paired sweeps are the FP32-arithmetic forms");
    static constexpr int ND = 0, EPI = EPI_NONE;
    static constexpr bool STENCIL = true, BLOCKED = false, NEUMANN = false, WIDE = true, PAIR = true;
    static constexpr int MIN_BLOCKS = 6;
    // shared-memory geometry: per stage the y_{k-1} box (W x (TILE_Y + 4)),
    // the b box and the y_{k-2} box (W x (TILE_Y + 2)); the y_k ring of four
    // planes (W x (TILE_Y + 2) floats each); the same x origin i0 - HX
    static constexpr int HX = 16 / (int)sizeof(T);
    static constexpr int W = TILE_X + 2 * HX;
    static constexpr int AROWS = TILE_Y + 4, BROWS = TILE_Y + 2;
    static constexpr int ABYTES = W * AROWS * (int)sizeof(T), BBYTES = W * BROWS * (int)sizeof(T);
    static constexpr int AST = align128(ABYTES), BST = align128(BBYTES);
    static constexpr int STAGE = AST + 2 * BST;
    static constexpr int STAGES = 6;
    static constexpr int YPLANE = W * BROWS; // floats per y_k ring plane
    static constexpr int DYN_BYTES = STAGES * STAGE + 4 * YPLANE * (int)sizeof(float);
    static constexpr int EX = TILE_X + 2, EY = TILE_Y + 2; // the tile and its one-cell ring
    const void *ym1, *bv, *zv;
    void *out1, *out2;
    int k, rin, rb, rz;
    float c1[6], c2[6];
    __device__ OpCiSweepPairW(const Desc &D, const KArgs &a, Scal *sc)
    {
        const int iter = ld_flag(&sc->iter);
        k = a.k;
        rin = a.in;
        rb = resolve_role(a.b, iter);
        rz = a.z;
        ym1 = D.vec[rin];
        bv = D.vec[rb];
        zv = D.vec[rz];
        out1 = D.vec[a.out];
        out2 = D.vec[a.aux];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            c1[q] = D.cikf[a.k][q];
            c2[q] = D.cikf[a.k + 1][q];
        }
    }
    // OpCiSweep::combine with the coefficients of sweep kk
    static __device__ __forceinline__ float combine(const float (&c)[6], int kk, float yc, float sx, float sy,
                                                    float sz, float b, float z)
    {
        float v;
        if constexpr (WY) v = fma(c[1], b, c[0] * yc);
        else v = c[1] * b;
        if (kk >= 3) v = fma(c[2], z, v);
        return fma(c[5], sz, fma(c[4], sy, fma(c[3], sx, v)));
    }
    static __device__ __forceinline__ float lds(const unsigned char *p, int x) { return E::lds(p, x); }
};

// The march of a pair over output planes [kb, ke) of one tile.  Stencil
// input planes q0 = kb - 2 .. q1 = ke + 1 are staged (b and y_{k-2} for kb - 1
// .. ke); step p (kb - 2 <= p < ke) computes y_k on plane p+1 over the tile
// and its ring, then, after one CTA barrier, y_{k+1} on plane p over the
// tile.  Plane q's stage is last read in step q, so it is refilled (with
// plane q + S) after the barrier of step q+1; the y_k ring keeps four planes,
// so the plane written in step p+1 never overlaps one read in step p.
template <class Op>
__device__ __forceinline__ void march_pair_wide(Op &op, const Desc &D, int tile, int kb, int ke,
                                                unsigned char *ring, uint64_t *bars, uint32_t &seq, int *s_dead)
{
    using T = typename std::conditional<Op::HX == 4, float, __nv_bfloat16>::type;
    constexpr int S = Op::STAGES, W = Op::W, HX = Op::HX;
    constexpr int PX = TILE_X / 2;
    static_assert(S >= 5 && S <= MAX_STAGES, "stages");
    const int nx = D.nx, ny = D.ny, nz = D.nz;
    const int plane = D.px * ny;
    const int tid = threadIdx.x;
    const int i0 = (tile % D.tiles_x) * TILE_X, j0 = (tile / D.tiles_x) * TILE_Y;
    const int q0 = kb - 2, q1 = ke + 1;
    const int nplanes = q1 - q0 + 1;
    const uint32_t seq0 = seq;
    float *yring = reinterpret_cast<float *>(ring + S * Op::STAGE);
    const bool with_z = op.k >= 3;
    const CUtensorMap *mA = D.tmap + TMAPS_PER_ROLE * op.rin + TMAP_HALO2;
    const CUtensorMap *mB = D.tmap + TMAPS_PER_ROLE * op.rb + TMAP_HALO;
    const CUtensorMap *mZ = D.tmap + TMAPS_PER_ROLE * op.rz + TMAP_HALO;
    // rolling stage index and mbarrier parity of a plane (plane n of this
    // march lives in stage (seq0 + n - q0) % S), advanced plane by plane
    struct Slot {
        int st;
        uint32_t par;
        __device__ __forceinline__ void next()
        {
            if (++st == S) {
                st = 0;
                par ^= 1u;
            }
        }
    };
    auto stage = [&](const Slot &sl) { return ring + sl.st * Op::STAGE; };
    auto issue = [&](const Slot &sl, int q) { // thread 0: plane q into the stage of slot sl
        unsigned char *st = stage(sl);
        uint64_t *b = bars + sl.st;
        const bool bz = q >= kb - 1 && q <= ke;
        const uint32_t bytes = Op::ABYTES + (bz ? Op::BBYTES * (with_z ? 2 : 1) : 0);
        mbar_expect_tx(b, bytes);
        tma_load_3d(st, mA, i0 - HX, j0 - 2, q, b);
        if (bz) {
            tma_load_3d(st + Op::AST, mB, i0 - HX, j0 - 1, q, b);
            if (with_z) tma_load_3d(st + Op::AST + Op::BST, mZ, i0 - HX, j0 - 1, q, b);
        }
    };
    auto wait = [&](const Slot &sl) {
        if (*s_dead) return;
        if (!mbar_wait(bars + sl.st, sl.par)) {
            *s_dead = 1;
            D.sc->status = ST_TIMEOUT;
            D.sc->stop = 1;
        }
    };
    Slot s0{(int)(seq0 % S), (seq0 / S) & 1u}; // plane p
    Slot s1 = s0;
    s1.next(); // plane p + 1
    Slot s2 = s1;
    s2.next(); // plane p + 2
    Slot sr = s0;   // thread 0: the stage of plane nref, the lowest not yet refilled
    int nref = q0;

    __syncthreads(); // the previous run's readers of the ring are done
    if (tid == 0) {
        Slot si = s0;
        for (int n = 0; n < S && n < nplanes; ++n) {
            issue(si, q0 + n);
            si.next();
        }
    }
    wait(s0);
    wait(s1);
    // the pair mapping of the tile for y_{k+1}
    const int tx = tid % PX, ty = tid / PX;
    const int gi = i0 + 2 * tx, gj = j0 + ty;
    const bool tin = gi < nx && gj < ny; // nx odd: gi + 1 may be the padding column nx (above)
    const int col = tin ? gj * D.px + gi : 0;
    const int me = (ty + 1) * W + HX + 2 * tx;
    // the ring cell of this thread (the first NRING threads): the rows above
    // and below the tile (EX cells each), then the columns left and right of
    // it (TILE_Y cells each), as an index into a W-wide, EY-row plane
    constexpr int NRING = 2 * Op::EX + 2 * TILE_Y;
    static_assert(NRING <= NTHREADS / 2, "one ring cell per thread");
    int rcell = -1;
    bool rin_grid = false;
    if (tid < NRING) {
        int ex, ey;
        if (tid < Op::EX) {
            ex = tid;
            ey = 0;
        } else if (tid < 2 * Op::EX) {
            ex = tid - Op::EX;
            ey = Op::EY - 1;
        } else if (tid < 2 * Op::EX + TILE_Y) {
            ex = 0;
            ey = 1 + tid - 2 * Op::EX;
        } else {
            ex = Op::EX - 1;
            ey = 1 + tid - 2 * Op::EX - TILE_Y;
        }
        rcell = ey * W + HX - 1 + ex;
        const int ci = i0 - 1 + ex, cj = j0 - 1 + ey;
        rin_grid = ci >= 0 && ci < nx && cj >= 0 && cj < ny;
    }

    for (int p = q0; p < ke; ++p) {
        wait(s2);
        const bool dead = *s_dead;
        // y_k on plane p+1: the tile by the pair mapping, its one-cell ring by
        // the first NRING threads
        const int qk = p + 1;
        if (!dead) {
            const unsigned char *A0 = stage(s0), *A1 = stage(s1), *A2 = stage(s2);
            const unsigned char *B1 = A1 + Op::AST, *Z1 = A1 + Op::AST + Op::BST;
            float *Y = yring + (qk & 3) * Op::YPLANE;
            const bool zin = qk >= 0 && qk < nz;
            {
                const int ia = me + W; // the y_{k-1} box has one more halo row on top
                float2 v = make_float2(0.f, 0.f);
                if (zin && tin) {
                    const float2 yc = Pair<T>::lds(A1, ia);
                    const float w = Op::lds(A1, ia - 1), e = Op::lds(A1, ia + 2);
                    const float2 so = Pair<T>::lds(A1, ia - W), no = Pair<T>::lds(A1, ia + W);
                    const float2 dn = Pair<T>::lds(A0, ia), up = Pair<T>::lds(A2, ia);
                    const float2 b = Pair<T>::lds(B1, me);
                    const float2 z = with_z ? Pair<T>::lds(Z1, me) : make_float2(0.f, 0.f);
                    v.x = E_round<T>(Op::combine(op.c1, op.k, yc.x, w + yc.y, so.x + no.x, dn.x + up.x, b.x, z.x));
                    v.y = E_round<T>(Op::combine(op.c1, op.k, yc.y, yc.x + e, so.y + no.y, dn.y + up.y, b.y, z.y));
                    // nx odd: the right point of the last pair is the ghost
                    // column nx, which y_{k+1} reads as zero (Eq. 4)
                    if (gi + 1 >= nx) v.y = 0.f;
                    if (qk >= kb && qk < ke) Pair<T>::st(op.out1, col + qk * plane, v);
                }
                *reinterpret_cast<float2 *>(Y + me) = v;
            }
            if (rcell >= 0) {
                float v = 0.f;
                if (zin && rin_grid) {
                    const int ia = rcell + W;
                    const float yc = Op::lds(A1, ia);
                    const float sx = Op::lds(A1, ia - 1) + Op::lds(A1, ia + 1);
                    const float sy = Op::lds(A1, ia - W) + Op::lds(A1, ia + W);
                    const float sz = Op::lds(A0, ia) + Op::lds(A2, ia);
                    const float b = Op::lds(B1, rcell);
                    const float z = with_z ? Op::lds(Z1, rcell) : 0.f;
                    v = E_round<T>(Op::combine(op.c1, op.k, yc, sx, sy, sz, b, z));
                }
                Y[rcell] = v;
            }
        }
        __syncthreads();
        if (tid == 0) // stages of the planes up to p - 1 are free
            for (; nref <= p - 1; ++nref) {
                if (nref + S <= q1 && !*s_dead) issue(sr, nref + S);
                sr.next();
            }
        // y_{k+1} on plane p over the tile
        if (p >= kb && tin && !dead) {
            const float *Y0 = yring + ((p - 1) & 3) * Op::YPLANE, *Y1 = yring + (p & 3) * Op::YPLANE,
                        *Y2 = yring + ((p + 1) & 3) * Op::YPLANE;
            const unsigned char *Ap = stage(s0), *Bp = Ap + Op::AST;
            const float2 yc = *reinterpret_cast<const float2 *>(Y1 + me);
            const float w = Y1[me - 1], e = Y1[me + 2];
            const float2 so = *reinterpret_cast<const float2 *>(Y1 + me - W);
            const float2 no = *reinterpret_cast<const float2 *>(Y1 + me + W);
            const float2 dn = *reinterpret_cast<const float2 *>(Y0 + me);
            const float2 up = *reinterpret_cast<const float2 *>(Y2 + me);
            const float2 b = Pair<T>::lds(Bp, me);
            const float2 z = Pair<T>::lds(Ap, me + W); // y_{k-1} on plane p (rows shifted by the extra halo row)
            const int kk = op.k + 1;
            Pair<T>::st(op.out2, col + p * plane,
                        make_float2(Op::combine(op.c2, kk, yc.x, w + yc.y, so.x + no.x, dn.x + up.x, b.x, z.x),
                                    Op::combine(op.c2, kk, yc.y, yc.x + e, so.y + no.y, dn.y + up.y, b.y, z.y)));
        }
        s0 = s1; // plane p+1 becomes p, p+2 becomes p+1
        s1 = s2;
        s2.next();
    }
    seq = seq0 + nplanes;
}

// w = A p^ and r~ . w  (Algorithm 3, first stencil kernel); T = type of p^.
// w is stored as w' = A q / cc, q = p^ as stored (p^ / Desc::hat): the centre
// then enters with coefficient 1 (6 FP64 instructions for A instead of 7).
// Nothing downstream needs the factor kappa = hat cc (w = kappa w'): alpha =
// rho / (r~ . w') comes out as kappa alpha, so s = r - alpha w and the
// direction update read w' with it unchanged, beta uses alpha / omega (both
// scaled alike, see OpStencil2Dot), and x += (alpha / cc) q (OpUpdate).
template <class T>
struct OpStencilDot {
    using C = double;
    using U = double;
    using PW = double;
    static constexpr int ND = 1, EPI = EPI_ALPHA;
    static constexpr bool STENCIL = true, BLOCKED = false;
    using TH = T;
    using TP = double;
    static constexpr int NH = 1, NP = 1;
    // a narrower p^ is widened once per staged cell instead of at all 7 reads
    static constexpr bool XFORM = !std::is_same<T, double>::value;
    int nh = 1, np = 1, hrole[NH], prole[NP];
    const void *ph;
    const double *rt;
    double *w;
    double wx, wy, wz; // -cx/cc, -cy/cc, -cz/cc
    __device__ OpStencilDot(const Desc &D, const KArgs &a, Scal *)
    {
        ph = D.vec[a.in];
        rt = (const double *)D.vec[ROLE_RT];
        w = (double *)D.vec[ROLE_W];
        hrole[0] = a.in;
        prole[0] = ROLE_RT;
        wx = D.wcx, wy = D.wcy, wz = D.wcz;
    }
    __device__ __forceinline__ double load(int idx) const { return Elem<T>::wide(ph, idx); }
    __device__ __forceinline__ double load_s(const void *const *h, int x) const { return Elem<T>::wides(h[0], x); }
    __device__ __forceinline__ double pw_s(const void *const *p, int x) const { return Elem<double>::lds(p[0], x); }
    __device__ __forceinline__ double sv(double u) const { return u; }
    __device__ __forceinline__ double pw(bool valid, int idx) const { return valid ? gld(rt + idx) : 0.0; }
    template <int NA>
    __device__ __forceinline__ void emit(int idx, double u, double sx, double sy, double sz, double, double rtv,
                                         double (&acc)[NA]) const
    {
        const double au = fma(wz, sz, fma(wy, sy, fma(wx, sx, u))); // A u / cc
        w[idx] = au;
        acc[0] += rtv * au;
    }
};

// t = A r^, t . s and t . t (Algorithm 3, second stencil kernel).  t is
// stored as t' = A q / cc, q = r^ as stored, like w (OpStencilDot): omega =
// (t' . s) / (t' . t') comes out as kappa omega, r = s - omega t' is then
// exact, and x += (omega / cc) q (OpUpdate).
template <class T>
struct OpStencil2Dot {
    using C = double;
    using U = double;
    using PW = double;
    static constexpr int ND = 2, EPI = EPI_OMEGA;
    static constexpr bool STENCIL = true, BLOCKED = false;
    using TH = T;
    using TP = double;
    static constexpr int NH = 1, NP = 1;
    static constexpr bool XFORM = !std::is_same<T, double>::value;
    int nh = 1, np = 1, hrole[NH], prole[NP];
    const void *rh;
    const double *s;
    double *t;
    double wx, wy, wz; // -cx/cc, -cy/cc, -cz/cc
    __device__ OpStencil2Dot(const Desc &D, const KArgs &a, Scal *)
    {
        rh = D.vec[a.in];
        s = (const double *)D.vec[ROLE_S];
        t = (double *)D.vec[ROLE_T];
        hrole[0] = a.in;
        prole[0] = ROLE_S;
        wx = D.wcx, wy = D.wcy, wz = D.wcz;
    }
    __device__ __forceinline__ double load(int idx) const { return Elem<T>::wide(rh, idx); }
    __device__ __forceinline__ double load_s(const void *const *h, int x) const { return Elem<T>::wides(h[0], x); }
    __device__ __forceinline__ double pw_s(const void *const *p, int x) const { return Elem<double>::lds(p[0], x); }
    __device__ __forceinline__ double sv(double u) const { return u; }
    __device__ __forceinline__ double pw(bool valid, int idx) const { return valid ? gld(s + idx) : 0.0; }
    template <int NA>
    __device__ __forceinline__ void emit(int idx, double u, double sx, double sy, double sz, double, double sv_,
                                         double (&acc)[NA]) const
    {
        const double au = fma(wz, sz, fma(wy, sy, fma(wx, sx, u))); // A u / cc
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
    using TH = double;
    using TP = double;
    static constexpr int NH = 1, NP = 0;
    static constexpr bool XFORM = false;
    int nh = 1, np = 0, hrole[NH], prole[1];
    const double *u;
    double *v;
    double cc, cx, cy, cz;
    __device__ OpApplyA(const Desc &D, const KArgs &a, Scal *)
    {
        u = (const double *)D.vec[a.in];
        v = (double *)D.vec[a.out];
        hrole[0] = a.in;
        prole[0] = 0;
        cc = D.cc, cx = D.cx, cy = D.cy, cz = D.cz;
    }
    __device__ __forceinline__ double load(int idx) const { return gld(u + idx); }
    __device__ __forceinline__ double load_s(const void *const *h, int x) const { return Elem<double>::lds(h[0], x); }
    __device__ __forceinline__ double sv(double x) const { return x; }
    __device__ __forceinline__ PW pw(bool, int) const { return PW{}; }
    __device__ __forceinline__ PW pw_s(const void *const *, int) const { return PW{}; }
    template <int NA>
    __device__ __forceinline__ void emit(int idx, double uu, double sx, double sy, double sz, double, const PW &,
                                         double (&)[NA]) const
    {
        v[idx] = apply_A_terms(cc, cx, cy, cz, uu, sx, sy, sz);
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
    using TH = double;
    using TP = double;
    static constexpr int NH = 1, NP = 1;
    static constexpr bool XFORM = false;
    int nh = 1, np = 1, hrole[NH], prole[NP];
    const double *x, *b;
    double *r, *rt;
    double cc, cx, cy, cz;
    __device__ OpResidual(const Desc &D, const KArgs &, Scal *)
    {
        x = (const double *)D.vec[ROLE_X];
        b = (const double *)D.vec[ROLE_B];
        r = (double *)D.vec[ROLE_R];
        rt = (double *)D.vec[ROLE_RT];
        hrole[0] = ROLE_X;
        prole[0] = ROLE_B;
        cc = D.cc, cx = D.cx, cy = D.cy, cz = D.cz;
    }
    __device__ __forceinline__ double load(int idx) const { return gld(x + idx); }
    __device__ __forceinline__ double load_s(const void *const *h, int x_) const { return Elem<double>::lds(h[0], x_); }
    __device__ __forceinline__ double pw_s(const void *const *p, int x_) const { return Elem<double>::lds(p[0], x_); }
    __device__ __forceinline__ double sv(double u) const { return u; }
    __device__ __forceinline__ double pw(bool valid, int idx) const { return valid ? gld(b + idx) : 0.0; }
    template <int NA>
    __device__ __forceinline__ void emit(int idx, double u, double sx, double sy, double sz, double, double bv,
                                         double (&acc)[NA]) const
    {
        const double rv = bv - apply_A_terms(cc, cx, cy, cz, u, sx, sy, sz);
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

// Residual replacement: r = b - A x replaces the recursive residual, with
// r~.r and ||r||^2 (the epilogue rescales beta and rho to the new r).  Runs
// after the update of outer iterations that are multiples of rr_every.
struct OpReplace {
    using C = double;
    using U = double;
    struct PW {
        double b, rt;
    };
    static constexpr int ND = 2, EPI = EPI_REPLACE;
    static constexpr bool STENCIL = true, BLOCKED = false;
    using TH = double;
    using TP = double;
    static constexpr int NH = 1, NP = 2;
    static constexpr bool XFORM = false;
    int nh = 1, np = 2, hrole[NH], prole[NP];
    const double *x, *b, *rt;
    double *r;
    double cc, cx, cy, cz;
    __device__ OpReplace(const Desc &D, const KArgs &, Scal *)
    {
        x = (const double *)D.vec[ROLE_X];
        b = (const double *)D.vec[ROLE_B];
        rt = (const double *)D.vec[ROLE_RT];
        r = (double *)D.vec[ROLE_R];
        hrole[0] = ROLE_X;
        prole[0] = ROLE_B;
        prole[1] = ROLE_RT;
        cc = D.cc, cx = D.cx, cy = D.cy, cz = D.cz;
    }
    __device__ __forceinline__ double load(int idx) const { return gld(x + idx); }
    __device__ __forceinline__ double load_s(const void *const *h, int x_) const { return Elem<double>::lds(h[0], x_); }
    __device__ __forceinline__ PW pw_s(const void *const *p, int x_) const
    {
        return PW{Elem<double>::lds(p[0], x_), Elem<double>::lds(p[1], x_)};
    }
    __device__ __forceinline__ double sv(double u) const { return u; }
    __device__ __forceinline__ PW pw(bool valid, int idx) const
    {
        return valid ? PW{gld(b + idx), gld(rt + idx)} : PW{0.0, 0.0};
    }
    template <int NA>
    __device__ __forceinline__ void emit(int idx, double u, double sx, double sy, double sz, double, const PW &p,
                                         double (&acc)[NA]) const
    {
        const double rv = p.b - apply_A_terms(cc, cx, cy, cz, u, sx, sy, sz);
        r[idx] = rv;
        acc[0] += p.rt * rv;
        acc[1] += rv * rv;
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
    struct In { double b; };
    __device__ __forceinline__ In load(int idx) const { return In{gld(b + idx)}; }
    template <int NA>
    __device__ __forceinline__ void apply(int idx, const In &v, double (&acc)[NA]) const
    {
        r[idx] = v.b;
        x[idx] = 0.0;
        acc[0] += v.b * v.b;
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
    double alpha, omega, alpha_h, omega_h;
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
        // w, t and p^, r^ are stored scaled (OpStencilDot): the true alpha p^
        // is (alpha / cc) times p^ as stored, and the same for omega r^
        alpha_h = alpha * D.inv_cc;
        omega_h = omega * D.inv_cc;
    }
    // six inputs per point: one plane ahead with FP32/BF16 p^ and r^ (256^3
    // update 289 -> 236 us); with FP64 ones the two-planes-then-compute loop
    // measured faster (227 against 239 us)
    static constexpr int PREFETCH = std::is_same<T, double>::value ? 0 : 1;
    using Raw = typename std::conditional<std::is_same<T, double>::value, double, typename Elem<T>::C>::type;
    struct In { double x; Raw p, r; double s, t, rt; };
    __device__ __forceinline__ In load(int idx) const
    {
        In v{};
        v.x = gld(x + idx);
        v.p = Elem<T>::ld(ph, idx);
        if (!half) {
            v.r = Elem<T>::ld(rh, idx);
            v.s = gld(s + idx);
            v.t = gld(t + idx);
            v.rt = gld(rt + idx);
        }
        return v;
    }
    // narrow p^, r^ are widened here, when their loads have arrived
    static __device__ __forceinline__ double widen(Raw v)
    {
        if constexpr (std::is_same<Raw, double>::value) return v;
        else return f2d_exact(v);
    }
    template <int NA>
    __device__ __forceinline__ void apply(int idx, const In &v, double (&acc)[NA]) const
    {
        const double p = widen(v.p);
        if (half) {
            x[idx] = v.x + alpha_h * p;
            return;
        }
        x[idx] = v.x + alpha_h * p + omega_h * widen(v.r);
        const double rn = v.s - omega * v.t;
        r[idx] = rn;
        acc[0] += v.rt * rn;
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
    struct In { double r, p, w; };
    __device__ __forceinline__ In load(int idx) const
    {
        In v{};
        v.r = gld(r + idx);
        if (!first) {
            v.p = gld(p + idx);
            v.w = gld(w + idx);
        }
        return v;
    }
    template <int NA>
    __device__ __forceinline__ void apply(int idx, const In &v, double (&)[NA]) const
    {
        if (first) p[idx] = v.r;
        else p[idx] = v.r + beta * (v.p - omega * v.w);
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
    struct In { double r, w; };
    __device__ __forceinline__ In load(int idx) const { return In{gld(r + idx), gld(w + idx)}; }
    template <int NA>
    __device__ __forceinline__ void apply(int idx, const In &u, double (&acc)[NA]) const
    {
        const double v = u.r - alpha * u.w;
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
    struct In { double a, b; };
    __device__ __forceinline__ In load(int idx) const { return In{gld(a + idx), gld(b + idx)}; }
    template <int NA>
    __device__ __forceinline__ void apply(int, const In &v, double (&acc)[NA]) const
    {
        acc[0] += v.a * v.b;
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
    double hat; // p^ is stored divided by it
    __device__ OpWiden(const Desc &D, const KArgs &k, Scal *)
    {
        in = D.vec[k.in];
        out = (double *)D.vec[k.out];
        hat = D.hat;
    }
    using Raw = typename std::conditional<std::is_same<T, double>::value, double, typename Elem<T>::C>::type;
    struct In { Raw v; };
    __device__ __forceinline__ In load(int idx) const { return In{Elem<T>::ld(in, idx)}; }
    template <int NA>
    __device__ __forceinline__ void apply(int idx, const In &v, double (&)[NA]) const
    {
        if constexpr (std::is_same<Raw, double>::value) out[idx] = v.v * hat;
        else out[idx] = f2d_exact(v.v) * hat;
    }
};

} // namespace psolve
