"""GPU parity of the CUDA path against the FP64 CPU oracle, through the C ABI.

Tolerances (FP64 path):
* stencil: |A u (GPU) - A u (oracle)| <= 1e-14 * (2 cc) * max|u|, i.e. a few
  units in the last place of the largest term (cc = 2 sum 1/h_d^2);
* dot: |error| <= N * 2^-53 * sum|a_i b_i| (recursive-summation bound);
* Chebyshev preconditioner: max error <= 1e-11 * max|M^-1 v| for degree <= 16
  (the three-term recurrence is stable; errors grow ~linearly with degree);
* solves at rtol 1e-10: relative L2 of x <= 1e-8 and iterations within +-2
  (the 256^3 benchmark problem, whose stopping point is decided by rounding,
  is compared in distribution in test_gpu_full_256.py);
  at a fixed iteration count (rtol = 0) the iterates agree to 1e-10, which is
  what "the same computation" means given a condition number up to ~1e4.
Mixed precision changes the preconditioner, so it is compared to the FP64
oracle solution at the same rtol by relative L2 (reported, bounded loosely)
and by the true residual.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_08935_b300 import binding as B
from paper_2503_08935_b300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = "cuda:0"

# ragged shapes (nz, ny, nx): partial x tiles (32), partial y tiles (8), short z
# engine=0 runs the TMA ring on every size (rows padded to a multiple of 8 when
# nx is not one); engine=1 forces the general engine
SHAPES = [(1, 1, 1), (2, 3, 5), (7, 9, 33), (19, 24, 37), (16, 16, 16), (33, 18, 5), (5, 40, 70),
          (64, 64, 64), (3, 17, 40), (9, 5, 8), (13, 11, 72)]


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()


def stencil_tol(h, u):
    cc = 2.0 * sum(1.0 / v ** 2 for v in h)
    return 1e-14 * 2 * cc * max(np.max(np.abs(u)), 1e-300)


# ------------------------------------------------------------- conversions --
@pytest.mark.parametrize("seed", [1, 2])
def test_integer_pipe_conversions_match_hardware(seed):
    assert B.selfcheck_conversions(seed=seed, count=1 << 27) == 0


def test_bounded_wait_gives_up_and_reports_timeout():
    """The TMA ring's waits are bounded: a wait on a barrier nothing completes
    returns TIMEOUT after the limit instead of hanging."""
    assert B.selfcheck_wait_timeout(1 << 20) == B.TIMEOUT


@pytest.mark.parametrize("kind", [0, 1])
def test_measured_fp64_rate_is_plausible(kind):
    """The FP64 roofline's denominator: a B300 SM runs a few FP64 instructions
    per clock (the fma and add rates agree), so the measured rate per SM per
    clock lies well inside (0.5, 64), and the run is long enough to time."""
    r = B.measure_fp64_rate(kind=kind, iters=4096)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert r["ms"] > 1.0 and 500.0 < r["sm_mhz"] < 4000.0
    per_clk_sm = r["instr_per_s"] / (sms * r["sm_mhz"] * 1e6)
    assert 0.5 < per_clk_sm < 64.0, per_clk_sm


# ---------------------------------------------------------------- stencil --
@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("shape", SHAPES)
def test_apply_A_matches_oracle(shape, engine):
    h = (0.7 / (shape[2] + 1), 1.3 / (shape[1] + 1), 1.0 / (shape[0] + 1))
    u = I.rhs_uniform(shape, seed=3)
    out = torch.empty(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape, h, engine=engine) as s:
        s.apply_A(dev(u), out)
    ref = O.apply_A(u, h)
    assert np.max(np.abs(host(out) - ref)) <= stencil_tol(h, u)


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("shape,blocks", [((8, 6, 4), (2, 3, 2)), ((16, 24, 40), (5, 3, 4)),
                                          ((32, 32, 64), (4, 4, 2)), ((9, 9, 9), (3, 3, 3)),
                                          ((4, 4, 4), (4, 4, 4)), ((12, 16, 48), (2, 4, 3))])
def test_block_restricted_apply_A_matches_oracle(shape, blocks, engine):
    h = I.default_h(shape)
    u = I.rhs_uniform(shape, seed=4)
    out = torch.empty(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape, h, blocks=blocks, engine=engine) as s:
        s.apply_A(dev(u), out, block_restricted=True)
    ref = O.apply_A(u, h, blocks)
    assert np.max(np.abs(host(out) - ref)) <= stencil_tol(h, u)


def test_apply_A_full_size_256():
    shape = (256, 256, 256)
    h = I.default_h(shape)
    u = I.rhs_uniform(shape, seed=1)
    out = torch.empty(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape, h) as s:
        s.apply_A(dev(u), out)
    ref = O.apply_A(u, h)
    assert np.max(np.abs(host(out) - ref)) <= stencil_tol(h, u)


# -------------------------------------------------------------------- dot --
@pytest.mark.parametrize("shape", [(1, 1, 1), (19, 24, 37), (64, 64, 64), (128, 128, 130)])
def test_dot_matches_oracle(shape):
    a = I.rhs_uniform(shape, seed=5)
    b = I.rhs_uniform(shape, seed=6)
    with B.Solver(shape) as s:
        got = s.dot(dev(a), dev(b))
    ref = O.dot(a, b)
    n = a.size
    assert abs(got - ref) <= n * 2.0 ** -53 * float(np.sum(np.abs(a * b)))


def test_dot_is_deterministic():
    shape = (40, 50, 60)
    a, b = dev(I.rhs_uniform(shape, seed=7)), dev(I.rhs_uniform(shape, seed=8))
    with B.Solver(shape) as s:
        vals = {s.dot(a, b) for _ in range(5)}
    assert len(vals) == 1


# ---------------------------------------------------------- preconditioner --
@pytest.mark.parametrize("shape", [(20, 24, 38), (20, 24, 40)])
@pytest.mark.parametrize("precond,blocks", [(B.PC_CHEB, (1, 1, 1)), (B.PC_BJ_CHEB, (2, 3, 2)),
                                            (B.PC_GNOCOMM_CHEB, (2, 3, 2))])
@pytest.mark.parametrize("degree", [0, 1, 2, 3, 8, 16])
def test_precond_fp64_matches_oracle(shape, precond, blocks, degree):
    h = I.default_h(shape)
    v = I.rhs_uniform(shape, seed=9)
    out = torch.empty(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape, h, blocks=blocks) as s:
        s.precond_apply(dev(v), out, precond, degree)
    ref = O.precond_apply(v, h, precond, degree, blocks)
    assert np.max(np.abs(host(out) - ref)) <= 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("scales,degree", [((100.0, 1 - 1e-4), 2), ((100.0, 1 - 1e-4), 3), ((100.0, 1 - 1e-4), 24),
                                           ((100.0, 1 - 1e-4), 64), ((2.0, 0.9), 2), ((2.0, 0.9), 3),
                                           ((1.0, 0.6), 2), ((1.0, 0.6), 3)])
@pytest.mark.parametrize("precond,blocks", [(B.PC_CHEB, (1, 1, 1)), (B.PC_GNOCOMM_CHEB, (2, 3, 2))])
def test_precond_fp64_rescaled_bounds_any_degree(scales, degree, precond, blocks):
    """Rescaled bounds (the y term of every sweep present), anisotropic h and
    degrees up to the largest accepted: the FP64 sweeps store their
    intermediate iterates scaled, and the result must still be M^-1 v of
    Algorithm 2 as the oracle computes it.  (An interval that cuts off the top
    of the spectrum is only taken at low degree: there the polynomial grows
    like T_d outside it, to 1e31 at degree 64.)"""
    shape = (20, 24, 40)
    h = (0.05, 0.04, 0.03)
    v = I.rhs_uniform(shape, seed=11)
    out = torch.empty(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape, h, blocks=blocks, lmin_scale=scales[0], lmax_scale=scales[1]) as s:
        s.precond_apply(dev(v), out, precond, degree)
    ref = O.precond_apply(v, h, precond, degree, blocks, lmin_scale=scales[0], lmax_scale=scales[1])
    assert np.all(np.isfinite(host(out)))
    assert np.max(np.abs(host(out) - ref)) <= 1e-11 * max(1.0, degree / 16) * np.max(np.abs(ref))


@pytest.mark.parametrize("shape", [(24, 24, 40), (24, 24, 37)])
@pytest.mark.parametrize("prec,tol", [(B.FP32, 2e-5), (B.BF16, 3e-2)])
@pytest.mark.parametrize("degree", [1, 4, 8])
def test_precond_mixed_close_to_oracle(shape, prec, tol, degree):
    h = I.default_h(shape)
    v = I.rhs_uniform(shape, seed=10)
    out = torch.empty(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape, h, cheb_prec=prec) as s:
        s.precond_apply(dev(v), out, B.PC_CHEB, degree)
    ref = O.precond_apply(v, h, O.PC_CHEB, degree)
    assert rel(host(out), ref) <= tol


@pytest.mark.parametrize("shape", [(24, 24, 40), (24, 24, 38)])
@pytest.mark.parametrize("prec,tol", [(B.FP32, 2e-5), (B.BF16, 3e-2)])
@pytest.mark.parametrize("precond", [B.PC_BJ_CHEB, B.PC_GNOCOMM_CHEB])
def test_block_precond_mixed_close_to_oracle(shape, prec, tol, precond):
    h = I.default_h(shape)
    v = I.rhs_uniform(shape, seed=10)
    out = torch.empty(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape, h, cheb_prec=prec, blocks=(2, 3, 2)) as s:
        s.precond_apply(dev(v), out, precond, 6)
    ref = O.precond_apply(v, h, precond, 6, (2, 3, 2))
    assert rel(host(out), ref) <= tol


def test_cheb_interval_matches_oracle():
    shape = (20, 24, 36)
    h = (0.05, 0.04, 0.03)
    with B.Solver(shape, h, blocks=(3, 2, 4), lmin_scale=2.0, lmax_scale=0.9) as s:
        for pc in (B.PC_CHEB, B.PC_BJ_CHEB, B.PC_GNOCOMM_CHEB):
            a, b = s.cheb_interval(pc)
            ra, rb = O.cheb_interval(shape, h, pc, (3, 2, 4), 2.0, 0.9)
            assert abs(a - ra) <= 1e-13 * rb and abs(b - rb) <= 1e-13 * rb


# ------------------------------------------------------------------ solves --
SOLVE_CASES = [
    # (shape, precond, degree, blocks, scales)
    ((24, 20, 36), B.PC_NONE, 0, (1, 1, 1), (1.0, 1.0)),
    ((24, 20, 36), B.PC_CHEB, 4, (1, 1, 1), (1.0, 1.0)),
    ((24, 20, 36), B.PC_CHEB, 8, (1, 1, 1), (1.0, 1.0)),
    ((24, 20, 40), B.PC_CHEB, 8, (1, 1, 1), (1.0, 1.0)),
    ((24, 20, 40), B.PC_NONE, 0, (1, 1, 1), (1.0, 1.0)),
    ((24, 20, 40), B.PC_BJ_CHEB, 3, (2, 2, 2), (1.0, 1.0)),
    ((24, 20, 36), B.PC_CHEB, 0, (1, 1, 1), (1.0, 1.0)),
    ((24, 20, 36), B.PC_CHEB, 1, (1, 1, 1), (1.0, 1.0)),
    ((24, 20, 36), B.PC_BJ_CHEB, 3, (2, 2, 2), (1.0, 1.0)),
    ((24, 20, 36), B.PC_GNOCOMM_CHEB, 4, (2, 2, 3), (1.0, 1.0)),
    ((33, 17, 45), B.PC_CHEB, 5, (1, 1, 1), (3.0, 1.0 - 1e-4)),
    ((40, 40, 40), B.PC_GNOCOMM_CHEB, 8, (2, 2, 2), (10.0, 1.0 - 1e-4)),
    ((1, 7, 1), B.PC_CHEB, 2, (1, 1, 1), (1.0, 1.0)),
]


def _solve_both(shape, precond, degree, blocks, scales, rtol=1e-10, maxit=500, x0=None, **opt_kw):
    h = I.default_h(shape)
    b = I.rhs_uniform(shape, seed=11)
    x = dev(x0) if x0 is not None else torch.zeros(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape, h, blocks=blocks, lmin_scale=scales[0], lmax_scale=scales[1],
                  use_x0=1 if x0 is not None else 0, **opt_kw) as s:
        info = s.solve(dev(b), x, rtol=rtol, maxit=maxit, precond=precond, degree=degree)
    xo, ro = O.bicgstab(b, h, rtol=rtol, maxit=maxit, precond=precond, degree=degree, blocks=blocks,
                        lmin_scale=scales[0], lmax_scale=scales[1], x0=x0)
    return host(x), info, xo, ro


def iter_slack(case, oracle_iters):
    """Allowed difference in iteration count at free stopping.  G(CI) converges
    smoothly and gets +-2.  With BJ/GNoComm blocks or no preconditioner the
    residual history of these small grids is erratic (plateaus just above
    rtol), so rounding differences move the stopping point: the iterates agree
    to 1e-15 for 10 iterations and drift to ~1e-9 by 30 (see
    test_fixed_iterations_match_oracle), and the BJ(CI) 24x20x36 case stopped at
    43 and 45 iterations in two equally valid reduction orders against the
    oracle's 40.  Bound: +-max(2, 15 %).  G(CI) of degree 0 or 1 (M a scaled
    identity, or one stencil) is no better: over 12 right-hand sides perturbed
    by 1e-15 relative noise the oracle alone takes 85..96 iterations at degree
    0 and 46..58 at degree 1 on the 24x20x36 grid."""
    if case[1] == B.PC_CHEB and case[2] >= 2:
        return 2
    return max(2, math.ceil(0.15 * oracle_iters))


@pytest.mark.parametrize("case", SOLVE_CASES)
def test_solve_matches_oracle(case):
    x, info, xo, ro = _solve_both(*case)
    assert info.status == B.OK and ro.status == O.OK
    assert abs(info.iterations - ro.iterations) <= iter_slack(case, ro.iterations)
    assert rel(x, xo) <= 1e-8
    assert info.rel_res_recursive <= 1e-10 and info.rel_res_true <= 2e-10
    assert abs(info.rel_res_true - info.rel_res_recursive) <= 0.1 * 1e-10


@pytest.mark.parametrize("case", SOLVE_CASES[:11])
@pytest.mark.parametrize("its,tol", [(4, 1e-12), (12, 1e-10)])
def test_fixed_iterations_match_oracle(case, its, tol):
    """rtol = 0: both sides run exactly `its` iterations of the same recurrence."""
    x, info, xo, ro = _solve_both(*case, rtol=0.0, maxit=its)
    assert info.status == B.NOT_CONVERGED and info.iterations == its == ro.iterations
    assert rel(x, xo) <= tol


ENGINE_CASES = [(p, pc, blk) for p in (B.FP64, B.FP32, B.BF16)
                for pc, blk in ((B.PC_CHEB, (1, 1, 1)), (B.PC_GNOCOMM_CHEB, (2, 2, 2)), (B.PC_NONE, (1, 1, 1)))
                # BF16 storage with a block-restricted preconditioner does not converge (the
                # rounding makes the preconditioner inconsistent; both engines agree on that)
                if not (p == B.BF16 and pc == B.PC_GNOCOMM_CHEB)]


@pytest.mark.parametrize("prec,precond,blocks", ENGINE_CASES)
def test_engines_agree(prec, precond, blocks):
    """The TMA ring and the general engine compute the same values with the same
    thread mapping and expressions; a whole solve must agree to rounding."""
    shape = (32, 24, 48)
    h = I.default_h(shape)
    b = dev(I.rhs_uniform(shape, seed=16))
    outs = []
    for engine in (0, 1):
        x = torch.zeros(shape, dtype=torch.float64, device=DEV)
        with B.Solver(shape, h, engine=engine, cheb_prec=prec, blocks=blocks) as s:
            info = s.solve(b, x, rtol=1e-10, maxit=400, precond=precond, degree=6)
        assert info.status == B.OK and info.engine == (1 if engine == 0 else 0)
        outs.append((host(x), info.iterations))
    assert outs[0][1] == outs[1][1]
    assert np.max(np.abs(outs[0][0] - outs[1][0])) <= 1e-12 * np.max(np.abs(outs[1][0]))


@pytest.mark.parametrize("prec", [B.FP32, B.BF16])
@pytest.mark.parametrize("shape", [(37, 20, 40), (33, 16, 64), (5, 9, 8), (21, 17, 37), (12, 9, 22)])
def test_wide_sweeps_bitwise_equal_to_one_point_sweeps(prec, shape):
    """With FP32/BF16 Chebyshev vectors, G(CI) on the TMA ring runs its sweeps
    two per pass and two x-adjacent points per thread (CI sweep 1 on the
    rounded right-hand side, then pairs of sweeps, an odd last one alone); the
    general engine runs them one sweep and one point at a time with the same
    expressions.  M^-1 v (degrees 1..5, 8 and 16: sweep 2 without y_{k-2},
    pairs ending on the last sweep or followed by a single one) and a whole
    solve agree bit for bit, on grids with a partial x tile, ragged y tiles and
    odd plane counts, and on grids whose rows are padded for the tensor copies
    (nx = 37: the last point pair straddles the grid edge; nx = 22)."""
    h = I.default_h(shape)
    v = dev(I.rhs_uniform(shape, seed=21))
    for deg in (1, 2, 3, 4, 5, 8, 16):
        outs = []
        for engine in (0, 1):
            out = torch.empty_like(v)
            with B.Solver(shape, h, engine=engine, cheb_prec=prec) as s:
                s.precond_apply(v, out, B.PC_CHEB, deg)
            outs.append(out)
        assert torch.equal(outs[0], outs[1]), f"degree {deg}"
    sols = []
    for engine in (0, 1):
        x = torch.zeros(shape, dtype=torch.float64, device=DEV)
        with B.Solver(shape, h, engine=engine, cheb_prec=prec) as s:
            info = s.solve(v, x, rtol=1e-9, maxit=300, precond=B.PC_CHEB, degree=8, raise_on_error=False)
        assert info.engine == (1 if engine == 0 else 0)
        sols.append((x, info.iterations, info.status))
    assert sols[0][1] == sols[1][1] and sols[0][2] == sols[1][2]
    assert torch.equal(sols[0][0], sols[1][0])


# ------------------------------------------------------------ padded rows --
@pytest.mark.parametrize("shape", [(21, 17, 37), (12, 9, 22)])
def test_padded_rows_every_entry_point(shape):
    """A grid whose nx is not a multiple of 8 is laid out with its rows padded
    to one, so that it runs on the TMA ring (info.engine == 1) while the
    caller's b and x are copied through padded staging vectors.  Every entry
    point gives bitwise the values of a context on the general engine with
    unpadded rows (engine = 1): A u, M^-1 v, u . b, a solve from x0 = 0, from
    host buffers and from an initial guess; a batch and a served request of
    the grid give bitwise the solo solve (FP32 Chebyshev vectors for the
    server, so its paired sweeps run over the padded rows too)."""
    h = I.default_h(shape)
    b = dev(I.rhs_uniform(shape, seed=31))
    u = dev(I.rhs_uniform(shape, seed=32))
    x0 = dev(I.rhs_uniform(shape, seed=33))
    res = {}
    for engine in (0, 1):
        r = {}
        with B.Solver(shape, h, engine=engine) as s:
            r["Au"] = host(s.apply_A(u, torch.empty_like(u)))
            r["Mv"] = host(s.precond_apply(u, torch.empty_like(u), B.PC_CHEB, 5))
            r["dot"] = np.array([s.dot(u, b)])
            x = torch.zeros_like(b)
            info = s.solve(b, x, rtol=1e-10, maxit=300, precond=B.PC_CHEB, degree=4)
            assert info.status == B.OK and info.engine == (1 if engine == 0 else 0)
            r["x"], r["it"] = host(x), np.array([info.iterations])
            xh = torch.zeros(shape, dtype=torch.float64).pin_memory()
            s.solve_host(torch.from_numpy(host(b)).pin_memory(), xh, rtol=1e-10, maxit=300, precond=B.PC_CHEB,
                         degree=4)
            r["x_host"] = xh.numpy().copy()
        with B.Solver(shape, h, engine=engine, use_x0=1) as s:
            x = x0.clone()
            info = s.solve(b, x, rtol=1e-10, maxit=300, precond=B.PC_CHEB, degree=4)
            assert info.status == B.OK
            r["x_from_x0"] = host(x)
        res[engine] = r
    for k in res[0]:
        assert np.array_equal(res[0][k], res[1][k]), k
    assert np.array_equal(res[0]["x"], res[0]["x_host"])
    xo, ro = O.bicgstab(host(b), h, rtol=1e-10, maxit=300, precond=O.PC_CHEB, degree=4)
    assert rel(res[0]["x"], xo) <= 1e-8
    # a batch with the padded grid and an unpadded one, and a served request
    xb = [torch.zeros_like(b), torch.zeros((8, 8, 16), dtype=torch.float64, device=DEV)]
    infos = B.solve_batch([b, dev(I.rhs_uniform((8, 8, 16), seed=34))], xb, rtol=1e-10, maxit=300,
                          precond=B.PC_CHEB, degree=4, slab_share=1)  # decomposed as a grid alone
    assert infos[0].engine == 1 and np.array_equal(host(xb[0]), res[0]["x"])
    with B.Solver(shape, h, cheb_prec=B.FP32, slab_share=B.SHARED_SLAB_SHARE) as s:
        xs = torch.zeros_like(b)
        solo = s.solve(b, xs, rtol=1e-9, maxit=300, precond=B.PC_CHEB, degree=8)
    with B.Server(4e9, max_slots=4) as srv:
        xv = torch.zeros_like(b)
        served = srv.wait(srv.submit(b, xv, rtol=1e-9, maxit=300, precond=B.PC_CHEB, degree=8, cheb_prec=B.FP32))
    assert served.status == B.OK and served.iterations == solo.iterations and served.engine == 1
    assert torch.equal(xv, xs)


@pytest.mark.parametrize("prec", [B.FP64, B.FP32])
@pytest.mark.parametrize("shape", [(40, 50, 99), (24, 33, 130)])
def test_padded_rows_larger_grids_bitwise(prec, shape):
    """Padded rows on grids of several x tiles (nx = 99: the straddling pair
    in the fourth tile; nx = 130: pitch 136, a last tile of two columns):
    solves on the TMA ring equal the general engine's bit for bit."""
    h = I.default_h(shape)
    b = dev(I.rhs_uniform(shape, seed=35))
    out = []
    for engine in (0, 1):
        x = torch.zeros(shape, dtype=torch.float64, device=DEV)
        with B.Solver(shape, h, engine=engine, cheb_prec=prec) as s:
            info = s.solve(b, x, rtol=1e-10, maxit=400, precond=B.PC_CHEB, degree=8)
        assert info.status == B.OK and info.engine == (1 if engine == 0 else 0)
        out.append((x, info.iterations))
    assert out[0][1] == out[1][1] and torch.equal(out[0][0], out[1][0])


def test_solve_with_initial_guess():
    shape = (18, 21, 34)
    x0 = I.rhs_uniform(shape, seed=12)
    x, info, xo, ro = _solve_both(shape, B.PC_CHEB, 4, (1, 1, 1), (1.0, 1.0), x0=x0)
    assert info.status == B.OK and abs(info.iterations - ro.iterations) <= 2
    assert rel(x, xo) <= 1e-8


def test_config_32cubed_manufactured_half_step():
    """32^3, h = 1/33, f = 3 pi^2 sin sin sin, no preconditioner: the RHS is a
    discrete eigenvector, so the first half step converges; x = f / lambda_111."""
    shape = (32, 32, 32)
    h = I.default_h(shape)
    f = I.rhs_manufactured(shape)
    x = torch.zeros(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape, h) as s:
        info = s.solve(dev(f), x, rtol=1e-10, maxit=2000, precond=B.PC_NONE)
    lam111 = 3 * 4.0 / h[0] ** 2 * math.sin(math.pi * h[0] / 2) ** 2
    assert info.status == B.OK and info.iterations == 1 and info.half_step_exit
    assert rel(host(x), f / lam111) <= 1e-12


def test_graph_eager_and_timing_are_bitwise_equal():
    shape = (30, 26, 44)
    h = I.default_h(shape)
    b = dev(I.rhs_uniform(shape, seed=13))
    outs = []
    for kw in (dict(use_graph=1), dict(use_graph=0), dict(timing=1), dict(poll_every=3)):
        x = torch.zeros(shape, dtype=torch.float64, device=DEV)
        with B.Solver(shape, h, **kw) as s:
            info = s.solve(b, x, rtol=1e-10, maxit=300, precond=B.PC_CHEB, degree=6)
        outs.append((host(x), info))
    for x, info in outs[1:]:
        assert np.array_equal(x, outs[0][0]) and info.iterations == outs[0][1].iterations
    tm = outs[2][1].kclass
    assert tm["ci_sweep4"]["launches"] > 0 and tm["ci_sweep4"]["ms"] > 0
    assert tm["stencil_dot"]["launches"] == outs[2][1].iterations


def test_solve_host_equals_device_solve():
    shape = (20, 22, 24)
    h = I.default_h(shape)
    b = I.rhs_uniform(shape, seed=14)
    x = torch.zeros(shape, dtype=torch.float64, device=DEV)
    xh = torch.zeros(shape, dtype=torch.float64).pin_memory()
    bh = torch.from_numpy(b).pin_memory()
    with B.Solver(shape, h) as s:
        i1 = s.solve(dev(b), x, rtol=1e-10, maxit=300, precond=B.PC_CHEB, degree=4)
        i2 = s.solve_host(bh, xh, rtol=1e-10, maxit=300, precond=B.PC_CHEB, degree=4)
    assert i1.iterations == i2.iterations and np.array_equal(host(x), xh.numpy())


@pytest.mark.parametrize("prec", [B.FP32, B.BF16])
def test_mixed_precision_reaches_rtol(prec):
    """Both sides stop at ||r||/||b|| <= 1e-10; their solutions may differ by up to
    kappa * 1e-10 (kappa ~ 700 here), so the bound on x is 1e-7."""
    shape = (32, 30, 40)
    h = I.default_h(shape)
    b = I.rhs_uniform(shape, seed=15)
    x = torch.zeros(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape, h, cheb_prec=prec) as s:
        info = s.solve(dev(b), x, rtol=1e-10, maxit=500, precond=B.PC_CHEB, degree=8)
    xo, ro = O.bicgstab(b, h, rtol=1e-10, maxit=500, precond=O.PC_CHEB, degree=8)
    assert info.status == B.OK and info.rel_res_true <= 2e-10
    assert rel(host(x), xo) <= 1e-7


# ------------------------------------------------------------- edge cases --
def test_zero_rhs():
    shape = (8, 9, 10)
    x = torch.ones(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape) as s:
        info = s.solve(torch.zeros(shape, dtype=torch.float64, device=DEV), x, precond=B.PC_CHEB, degree=3)
    assert info.status == B.OK and info.iterations == 0 and not host(x).any()


def test_zero_rhs_with_initial_guess_returns_zero():
    shape = (8, 9, 10)
    x = torch.ones(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape, use_x0=1) as s:
        info = s.solve(torch.zeros(shape, dtype=torch.float64, device=DEV), x, precond=B.PC_CHEB, degree=3)
    assert info.status == B.OK and info.iterations == 0 and not host(x).any()


def test_nonfinite_rhs():
    shape = (8, 9, 10)
    b = I.rhs_uniform(shape)
    b[3, 4, 5] = np.inf
    x = torch.zeros(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape) as s:
        info = s.solve(dev(b), x, precond=B.PC_CHEB, degree=3)
    assert info.status == B.NONFINITE


def test_maxit_and_zero_maxit():
    shape = (16, 16, 16)
    b = dev(I.rhs_uniform(shape))
    with B.Solver(shape) as s:
        x = torch.zeros(shape, dtype=torch.float64, device=DEV)
        assert s.solve(b, x, rtol=1e-14, maxit=0, precond=B.PC_CHEB, degree=2).status == B.NOT_CONVERGED
        info = s.solve(b, x, rtol=1e-14, maxit=2, precond=B.PC_CHEB, degree=2)
        assert info.status == B.NOT_CONVERGED and info.iterations == 2


def test_argument_errors():
    shape = (10, 12, 14)
    b = dev(I.rhs_uniform(shape))
    x = torch.zeros(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape, blocks=(3, 1, 1)) as s:
        with pytest.raises(B.PsolveError):  # 3 blocks do not divide nx = 14
            s.solve(b, x, precond=B.PC_BJ_CHEB, degree=2)
        with pytest.raises(B.PsolveError):
            s.solve(b, x, precond=B.PC_CHEB, degree=65)
        with pytest.raises(B.PsolveError):
            s.solve(b, x, rtol=-1.0)
    with B.Solver((4, 4, 4), lmin_scale=100.0, lmax_scale=1 - 1e-4) as s:
        with pytest.raises(B.PsolveError):  # empty interval on a tiny grid
            s.solve(torch.ones((4, 4, 4), dtype=torch.float64, device=DEV),
                    torch.zeros((4, 4, 4), dtype=torch.float64, device=DEV), precond=B.PC_CHEB, degree=2)


@pytest.mark.parametrize("prec", [B.FP64, B.FP32])
def test_repeated_solves_reuse_context(prec):
    """One context across solves on different buffers, with A u and M^-1 v
    calls in between (they bind other vectors to the descriptor): every result
    is bitwise that of a fresh context, so the tensor maps and the descriptor
    a context keeps from one call to the next always describe the buffers of
    the current call."""
    shape = (20, 24, 32)  # nx % 8 == 0: the TMA engine, whose maps are cached
    h = I.default_h(shape)
    bs = [dev(I.rhs_uniform(shape, seed=seed)) for seed in (1, 2, 3)]  # all alive: distinct addresses
    xs = [torch.zeros(shape, dtype=torch.float64, device=DEV) for _ in range(3)]
    u = dev(I.rhs_uniform(shape, seed=9))
    ref_x, outs = {}, {}
    for q in range(3):
        with B.Solver(shape, h, cheb_prec=prec) as f:
            xr = torch.zeros(shape, dtype=torch.float64, device=DEV)
            f.solve(bs[q], xr, precond=B.PC_CHEB, degree=4)
            ref_x[q] = host(xr)
    with B.Solver(shape, h, cheb_prec=prec) as f:
        ref_au = host(f.apply_A(u, torch.empty_like(u)))
        ref_mv = host(f.precond_apply(u, torch.empty_like(u), B.PC_CHEB, 4))
    with B.Solver(shape, h, cheb_prec=prec) as s:
        for k, (q, j) in enumerate([(0, 0), (1, 1), (0, 2), (2, 0), (0, 0), (1, 2)]):
            xs[j].zero_()
            s.solve(bs[q], xs[j], precond=B.PC_CHEB, degree=4)
            assert np.array_equal(host(xs[j]), ref_x[q]), (k, q, j)
            outs.setdefault(k % 2, torch.empty_like(u))
            if k % 2 == 0:
                assert np.array_equal(host(s.apply_A(u, outs[0])), ref_au), k
            else:
                assert np.array_equal(host(s.precond_apply(u, outs[1], B.PC_CHEB, 4)), ref_mv), k
    assert not np.array_equal(ref_x[0], ref_x[1])


# ------------------------------------------------------------------ batch --
def test_batch_bitwise_equals_alone_and_matches_oracle():
    shapes = [(16, 24, 40), (32, 16, 16), (9, 33, 17), (24, 24, 24), (8, 8, 64)]
    bs = [I.rhs_uniform(sh, seed=20 + q) for q, sh in enumerate(shapes)]
    xs = [torch.zeros(sh, dtype=torch.float64, device=DEV) for sh in shapes]
    infos = B.solve_batch([dev(b) for b in bs], xs, rtol=1e-10, maxit=300, precond=B.PC_CHEB, degree=4)
    for q, sh in enumerate(shapes):
        xa = torch.zeros(sh, dtype=torch.float64, device=DEV)
        with B.Solver(sh, slab_share=B.SHARED_SLAB_SHARE) as s:  # the batch's default slab share
            ia = s.solve(dev(bs[q]), xa, rtol=1e-10, maxit=300, precond=B.PC_CHEB, degree=4)
        assert infos[q].status == B.OK and infos[q].iterations == ia.iterations
        assert np.array_equal(host(xs[q]), host(xa))
        xo, ro = O.bicgstab(bs[q], I.default_h(sh), rtol=1e-10, maxit=300, precond=O.PC_CHEB, degree=4)
        assert rel(host(xs[q]), xo) <= 1e-8
        assert abs(ro.iterations - ia.iterations) <= max(2, math.ceil(0.1 * ro.iterations))


# ------------------------------------------------------ full-size configs --
def test_full_size_256_cheb8_fixed_iterations_and_residual():
    """256^3, Chebyshev degree 8, in the benchmark's launch configuration:
    two fixed iterations against the oracle, then a full solve whose true and
    recursive residuals must agree."""
    shape = (256, 256, 256)
    h = I.default_h(shape)
    b = I.rhs_uniform(shape, seed=1)
    bt = dev(b)
    x = torch.zeros(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape, h) as s:
        info = s.solve(bt, x, rtol=0.0, maxit=2, precond=B.PC_CHEB, degree=8)
        assert info.iterations == 2
        xo, ro = O.bicgstab(b, h, rtol=0.0, maxit=2, precond=O.PC_CHEB, degree=8)
        assert rel(host(x), xo) <= 1e-10
        info = s.solve(bt, x, rtol=1e-10, maxit=500, precond=B.PC_CHEB, degree=8)
    assert info.status == B.OK
    assert info.rel_res_true <= 2e-10 and abs(info.rel_res_true - info.rel_res_recursive) <= 1e-11
