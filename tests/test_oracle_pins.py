"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Nothing here re-types the oracle's own formulas.  Each check compares the
oracle against an independent object:

* the dense Kronecker-sum matrix P of Eq. 6 built from the 1-D matrix D of
  Eq. 4 with numpy (and its block-diagonal restriction, Eq. 12-14);
* the golden matrix D and the Dirichlet eigenvalues of Eq. 4 / Eq. 9 for n = 5
  written out in closed form (tests/golden/);
* LAPACK's symmetric eigen-solver and dense LU solve on P;
* the Chebyshev residual polynomial T_{d+1}((theta-lambda)/delta)/T_{d+1}(sigma)
  evaluated through the cos / cosh closed form of T_m;
* Krylov finite termination, the minimal-residual property of omega, and the
  exact discrete solution for the manufactured right-hand side;
* exact rational arithmetic (fractions) for the compensated dot product.

A plausible slip in the oracle (a wrong h_d on an axis, a dropped neighbour, a
sign, an off-by-one in a Chebyshev coefficient, a wrong beta or omega, a missing
x-update term) fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2503_08935_b300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ---------------------------------------------------------------- helpers --
def D1(n):
    """Eq. 4, built independently of the oracle."""
    return 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)


def dense_P(shape, h, blocks=None):
    """Eq. 6: P = I_z x I_y x D_x/hx^2 + I_z x D_y/hy^2 x I_x + D_z/hz^2 x I_y x I_x.
    With ``blocks`` (x, y, z counts): keep only entries inside one block (R_s A R_s^T)."""
    nz, ny, nx = shape
    hx, hy, hz = h
    M = (np.kron(np.eye(nz), np.kron(np.eye(ny), D1(nx) / hx ** 2))
         + np.kron(np.eye(nz), np.kron(D1(ny) / hy ** 2, np.eye(nx)))
         + np.kron(D1(nz) / hz ** 2, np.kron(np.eye(ny), np.eye(nx))))
    if blocks is not None:
        bx, by, bz = blocks
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        lab = (((k // (nz // bz)) * by + (j // (ny // by))) * bx + (i // (nx // bx))).ravel()
        M = M * (lab[:, None] == lab[None, :])
    return M


def cheb_T(m, x):
    """Chebyshev polynomial of the first kind via its trigonometric closed form."""
    if abs(x) <= 1.0:
        return math.cos(m * math.acos(x))
    if x > 1.0:
        return math.cosh(m * math.acosh(x))
    return (-1) ** m * math.cosh(m * math.acosh(-x))


def cheb_q(lam, a, b, d):
    """Degree-d Chebyshev iterate from x0 = 0 acting on an eigenvector of eigenvalue lam:
    x = (1 - T_{d+1}((theta - lam)/delta) / T_{d+1}(sigma)) / lam."""
    th, de = 0.5 * (b + a), 0.5 * (b - a)
    return (1.0 - cheb_T(d + 1, (th - lam) / de) / cheb_T(d + 1, th / de)) / lam


def sine_mode(shape, kx, ky, kz):
    nz, ny, nx = shape
    sx = np.sin(kx * math.pi * np.arange(1, nx + 1) / (nx + 1))
    sy = np.sin(ky * math.pi * np.arange(1, ny + 1) / (ny + 1))
    sz = np.sin(kz * math.pi * np.arange(1, nz + 1) / (nz + 1))
    return sz[:, None, None] * sy[None, :, None] * sx[None, None, :]


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append([float(eval(t, {"sqrt": math.sqrt})) for t in line.split()])
    return np.array(rows)


# ------------------------------------------------------------------- dots --
def _exact_dot(a, b):
    return sum((Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b)), Fraction(0))


@pytest.mark.parametrize("cond", ["plain", "cancelling"])
def test_dot2_near_correctly_rounded(cond):
    rng = np.random.default_rng(7)
    n = 400
    a = rng.standard_normal(n)
    b = rng.standard_normal(n)
    if cond == "cancelling":
        # Each pair (a_i 2^e_i, b_i) and (a_i 2^e_i, -b_i (1 + 2^-20)) nearly cancels, but the two
        # products round differently, so the sum is ~2^-20 of the products' magnitude and a
        # dot product that drops the products' rounding errors misses the bound by ~2^20.
        e = np.ldexp(1.0, rng.integers(-30, 30, n))
        a = np.concatenate([a * e, a * e])
        b = np.concatenate([b, -b * (1.0 + 2.0 ** -20)])
    got = O.dot(a, b)
    exact = _exact_dot(a, b)
    eps = 2.0 ** -53
    n = a.size
    gam = n * eps / (1 - n * eps)
    bound = eps * abs(float(exact)) + gam * gam * float(sum(abs(x * y) for x, y in zip(a, b)))
    assert abs(Fraction(got) - exact) <= Fraction(bound) * 2


def test_dot_empty_and_single():
    assert O.dot(np.zeros(0), np.zeros(0)) == 0.0
    assert O.dot(np.array([3.0]), np.array([-2.5])) == -7.5


# ---------------------------------------------------------------- stencil --
def test_D_matrix_golden_eq4():
    """Columns of A on a 5x1x1 grid with h = 1 equal D_5 (Eq. 4, golden) plus the
    1x1 Dirichlet matrices [2] of the y and z axes on the diagonal."""
    Dg = read_golden("dirichlet_D_n5.txt")
    assert Dg.shape == (5, 5)
    cols = []
    for q in range(5):
        e = np.zeros((1, 1, 5))
        e[0, 0, q] = 1.0
        cols.append(O.apply_A(e, (1.0, 1.0, 1.0)).ravel())
    A = np.array(cols).T
    assert np.array_equal(A, Dg + 4.0 * np.eye(5))


@pytest.mark.parametrize("shape,h", [((5, 4, 3), (0.3, 0.7, 1.1)), ((4, 4, 4), (0.5, 0.25, 0.125)),
                                     ((2, 7, 1), (1.0, 0.2, 0.9)), ((1, 1, 1), (0.5, 0.5, 0.5))])
def test_stencil_equals_dense_kronecker(shape, h):
    u = np.random.default_rng(11).standard_normal(shape)
    ref = dense_P(shape, h) @ u.ravel()
    got = O.apply_A(u, h).ravel()
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(np.abs(ref))


@pytest.mark.parametrize("shape,blocks", [((4, 6, 4), (2, 3, 2)), ((6, 4, 8), (4, 2, 3)),
                                          ((3, 3, 3), (1, 1, 1)), ((4, 4, 4), (4, 4, 4))])
def test_block_stencil_equals_block_diagonal(shape, blocks):
    h = (0.2, 0.3, 0.25)
    u = np.random.default_rng(12).standard_normal(shape)
    ref = dense_P(shape, h, blocks) @ u.ravel()
    got = O.apply_A(u, h, blocks).ravel()
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_block_sizes_must_divide():
    with pytest.raises(ValueError):
        O.apply_A(np.zeros((4, 4, 5)), (1, 1, 1), (2, 2, 2))


# ------------------------------------------------------------ eigenvalues --
def test_dirichlet_eigs_golden_eq9():
    """Eq. 9 for n = 5 in closed form: {2 - sqrt3, 1, 2, 3, 2 + sqrt3} (golden)."""
    ev = read_golden("dirichlet_eigs_n5.txt").ravel()
    lam = np.linalg.eigvalsh(D1(5))
    assert np.allclose(np.sort(lam), ev, rtol=0, atol=1e-14)
    lo, hi = O.eig_bounds((5, 1, 1), (1.0, 1.0, 1.0))
    assert abs(lo - (ev[0] + 4.0)) <= 1e-14 and abs(hi - (ev[-1] + 4.0)) <= 1e-14


@pytest.mark.parametrize("shape", [(6, 5, 4), (3, 7, 2), (1, 1, 9)])
def test_sine_modes_are_eigenvectors(shape):
    h = (0.31, 0.17, 0.23)
    nz, ny, nx = shape
    for kx, ky, kz in [(1, 1, 1), (nx, ny, nz), (max(1, nx // 2), 1, nz)]:
        v = sine_mode(shape, kx, ky, kz)
        lam = sum(4.0 / hd ** 2 * math.sin(k * math.pi / (2 * (n + 1))) ** 2
                  for k, n, hd in [(kx, nx, h[0]), (ky, ny, h[1]), (kz, nz, h[2])])
        Av = O.apply_A(v, h)
        assert rel(Av, lam * v) <= 1e-13


@pytest.mark.parametrize("shape,h", [((3, 5, 4), (0.4, 0.2, 0.3)), ((6, 6, 6), None)])
def test_eig_bounds_match_dense_spectrum(shape, h):
    h = I.default_h(shape) if h is None else h
    lam = np.linalg.eigvalsh(dense_P(shape, h))
    nz, ny, nx = shape
    lo, hi = O.eig_bounds((nx, ny, nz), h)
    assert abs(lo - lam[0]) <= 1e-12 * lam[-1]
    assert abs(hi - lam[-1]) <= 1e-12 * lam[-1]


# -------------------------------------------------------------- Chebyshev --
@pytest.mark.parametrize("scales", [(1.0, 1.0), (3.0, 0.9), (0.5, 1.2)])
@pytest.mark.parametrize("d", [0, 1, 2, 3, 5, 8, 12])
def test_cheb_matches_spectral_closed_form(d, scales):
    shape = (6, 5, 4)
    h = I.default_h(shape)
    P = dense_P(shape, h)
    lam, V = np.linalg.eigh(P)
    a0, b0 = O.eig_bounds((4, 5, 6), h)
    a, b = a0 * scales[0], b0 * scales[1]
    rhs = np.random.default_rng(3).standard_normal(shape)
    q = np.array([cheb_q(l, a, b, d) for l in lam])
    ref = V @ (q * (V.T @ rhs.ravel()))
    got = O.cheb(rhs, h, a, b, d).ravel()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("precond", [O.PC_BJ_CHEB, O.PC_GNOCOMM_CHEB])
def test_block_cheb_matches_block_spectrum(precond):
    shape, blocks = (4, 6, 8), (2, 3, 2)
    h = (0.11, 0.13, 0.17)
    Pb = dense_P(shape, h, blocks)
    lam, V = np.linalg.eigh(Pb)
    a, b = O.cheb_interval(shape, h, precond, blocks)
    if precond == O.PC_BJ_CHEB:  # interval of one block (all blocks equal)
        assert abs(a - lam[0]) <= 1e-12 * lam[-1] and abs(b - lam[-1]) <= 1e-12 * lam[-1]
    else:  # GNoComm: whole-grid interval, strictly wider than any block's spectrum
        g0, g1 = np.linalg.eigvalsh(dense_P(shape, h))[[0, -1]]
        assert abs(a - g0) <= 1e-12 * g1 and abs(b - g1) <= 1e-12 * g1
    rhs = np.random.default_rng(4).standard_normal(shape)
    for d in (0, 1, 4):
        q = np.array([cheb_q(l, a, b, d) for l in lam])
        ref = V @ (q * (V.T @ rhs.ravel()))
        got = O.precond_apply(rhs, h, precond, d, blocks).ravel()
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_cheb_degree0_is_b_over_theta_and_linear():
    shape = (5, 6, 7)
    h = I.default_h(shape)
    a, b = O.eig_bounds((7, 6, 5), h)
    u = I.rhs_uniform(shape, seed=5)
    v = I.rhs_uniform(shape, seed=6)
    assert np.array_equal(O.cheb(u, h, a, b, 0), u / (0.5 * (a + b)))
    lhs = O.cheb(2.5 * u + v, h, a, b, 6)
    rhs = 2.5 * O.cheb(u, h, a, b, 6) + O.cheb(v, h, a, b, 6)
    assert rel(lhs, rhs) <= 1e-13


def test_cheb_error_decay_exact_bounds():
    """With exact bounds, ||CI_d(b) - A^{-1} b||_A <= 2 ((sqrt k - 1)/(sqrt k + 1))^{d+1} ||A^{-1} b||_A."""
    shape = (8, 8, 8)
    h = I.default_h(shape)
    P = dense_P(shape, h)
    a, b = O.eig_bounds((8, 8, 8), h)
    rhs = I.rhs_uniform(shape, seed=9)
    xs = np.linalg.solve(P, rhs.ravel())
    kap = b / a
    c = (math.sqrt(kap) - 1) / (math.sqrt(kap) + 1)

    def anorm(e):
        return math.sqrt(e @ P @ e)

    for d in (1, 4, 8, 16):
        e = O.cheb(rhs, h, a, b, d).ravel() - xs
        assert anorm(e) <= 2 * c ** (d + 1) * anorm(xs) * (1 + 1e-9)


# -------------------------------------------------------------- Bi-CGSTAB --
PCS = [(O.PC_NONE, 0, (1, 1, 1)), (O.PC_CHEB, 3, (1, 1, 1)), (O.PC_BJ_CHEB, 2, (2, 1, 2)),
       (O.PC_GNOCOMM_CHEB, 2, (2, 1, 2)), (O.PC_CHEB, 0, (1, 1, 1))]


@pytest.mark.parametrize("shape", [(4, 4, 4), (6, 6, 6), (6, 5, 4)])
@pytest.mark.parametrize("pc", PCS)
@pytest.mark.parametrize("with_x0", [False, True])
def test_bicgstab_matches_dense_solve(shape, pc, with_x0):
    h = I.default_h(shape)
    P = dense_P(shape, h)
    b = I.rhs_uniform(shape, seed=21)
    x0 = I.rhs_uniform(shape, seed=22) if with_x0 else None
    x, res = O.bicgstab(b, h, rtol=1e-13, maxit=1000, precond=pc[0], degree=pc[1], blocks=pc[2], x0=x0)
    assert res.status == O.OK
    xs = np.linalg.solve(P, b.ravel())
    kappa = np.linalg.cond(P)
    assert rel(x, xs) <= 10 * kappa * 1e-13
    assert res.rel_res_true <= 1e-12


def test_finite_termination_on_m_modes():
    """b in the span of m eigenvectors with distinct eigenvalues: the Krylov space has
    dimension m, BiCG ends at step m, so Bi-CGSTAB's half-step residual s_m vanishes."""
    shape = (7, 6, 5)
    h = I.default_h(shape)
    modes = [(1, 1, 1), (2, 3, 1), (5, 6, 7), (3, 2, 4)]
    for m in range(1, len(modes) + 1):
        b = sum((0.7 + q) * sine_mode(shape, *modes[q]) for q in range(m))
        for pc in (O.PC_NONE, O.PC_CHEB):
            x, res = O.bicgstab(b, h, rtol=1e-11, maxit=50, precond=pc, degree=2 if pc else 0)
            assert res.status == O.OK and res.iterations <= m, (m, pc, res)
            assert res.rel_res_true <= 1e-10


@pytest.mark.parametrize("pc", PCS[:4])
def test_omega_minimises_residual(pc):
    """omega = t.s / t.t minimises ||s - omega t||, so ||r_i|| <= ||s_i|| each iteration."""
    shape = (10, 9, 8)
    h = I.default_h(shape)
    b = I.rhs_uniform(shape, seed=31)
    x, res = O.bicgstab(b, h, rtol=0.0, maxit=6, precond=pc[0], degree=pc[1], blocks=pc[2])
    assert res.iterations == 6
    hs, hr = res.hist_s, res.hist_r
    assert np.all(np.isfinite(hr)) and np.all(hr <= hs * (1 + 1e-13))


@pytest.mark.parametrize("pc", PCS[:4])
def test_true_and_recursive_residual_agree(pc):
    shape = (16, 16, 16)
    h = I.default_h(shape)
    b = I.rhs_uniform(shape, seed=41)
    rtol = 1e-10
    x, res = O.bicgstab(b, h, rtol=rtol, maxit=2000, precond=pc[0], degree=pc[1] + 2, blocks=pc[2])
    assert res.status == O.OK
    assert res.rel_res_recursive <= rtol
    assert abs(res.rel_res_true - res.rel_res_recursive) <= 0.1 * rtol


@pytest.mark.parametrize("n", [15, 32])
def test_manufactured_exact_discrete_solution_and_half_step(n):
    """f = 3 pi^2 prod sin(pi x_d) is the (1,1,1) sine mode, so A^{-1} f = f / lambda_111
    exactly, and the first half-step already converges (s = f - alpha A f = 0)."""
    shape = (n, n, n)
    h = I.default_h(shape)
    f = I.rhs_manufactured(shape)
    x, res = O.bicgstab(f, h, rtol=1e-10, maxit=2000)
    lam111 = 3 * 4.0 / h[0] ** 2 * math.sin(math.pi * h[0] / 2) ** 2
    assert res.status == O.OK and res.iterations == 1 and res.half_step_exit
    assert rel(x, f / lam111) <= 1e-12


def test_manufactured_second_order_convergence():
    """Discretisation error against the continuous solution sin sin sin: O(h^2), ratio ~4."""
    errs = []
    for n in (15, 31, 63):
        shape = (n, n, n)
        h = I.default_h(shape)
        f = I.rhs_manufactured(shape)
        x, res = O.bicgstab(f, h, rtol=1e-12, maxit=100)
        exact = f / (3 * math.pi ** 2)
        errs.append(np.max(np.abs(x - exact)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.8 < r1 < 4.2 and 3.9 < r2 < 4.1


# --------------------------------------------------------- special cases --
def test_zero_rhs_gives_zero():
    b = np.zeros((3, 4, 5))
    x, res = O.bicgstab(b, (1, 1, 1), rtol=1e-10, maxit=10, x0=np.ones_like(b))
    assert res.status == O.OK and res.iterations == 0 and not np.any(x)


def test_nonfinite_rhs_is_reported():
    b = I.rhs_uniform((4, 4, 4))
    b[1, 2, 3] = np.nan
    x, res = O.bicgstab(b, I.default_h(b.shape), rtol=1e-10, maxit=10)
    assert res.status == O.NONFINITE


def test_maxit_exhaustion():
    shape = (12, 12, 12)
    b = I.rhs_uniform(shape)
    x, res = O.bicgstab(b, I.default_h(shape), rtol=1e-14, maxit=2)
    assert res.status == O.NOT_CONVERGED and res.iterations == 2


def test_exact_initial_guess_returns_immediately():
    shape = (5, 5, 5)
    h = I.default_h(shape)
    xs = I.rhs_uniform(shape, seed=8)
    b = O.apply_A(xs, h)
    x, res = O.bicgstab(b, h, rtol=1e-10, maxit=10, x0=xs)
    assert res.status == O.OK and res.iterations == 0 and np.array_equal(x, xs)


def test_rescaled_interval_inverted_is_rejected():
    """lambda_min x 100 exceeds lambda_max on a tiny grid: the interval is empty."""
    with pytest.raises(ValueError):
        O.cheb_interval((4, 4, 4), I.default_h((4, 4, 4)), O.PC_CHEB, (1, 1, 1), 100.0, 1 - 1e-4)


# ------------------------------------------- residual replacement (added form) --
# Not part of the paper's method: every rr_every iterations r is recomputed as
# b - A x and beta, rho are rescaled to it.  In exact arithmetic the recursive
# and the true residual coincide, so the iteration is unchanged.
@pytest.mark.parametrize("shape", [(4, 4, 4), (6, 5, 4)])
@pytest.mark.parametrize("rr", [1, 2])
def test_residual_replacement_matches_dense_solve(shape, rr):
    h = I.default_h(shape)
    P = dense_P(shape, h)
    b = I.rhs_uniform(shape, seed=23)
    x, res = O.bicgstab(b, h, rtol=1e-13, maxit=1000, precond=O.PC_CHEB, degree=3, rr_every=rr)
    assert res.status == O.OK
    xs = np.linalg.solve(P, b.ravel())
    assert rel(x, xs) <= 10 * np.linalg.cond(P) * 1e-13
    assert res.rel_res_true <= 1e-12


def test_residual_replacement_that_never_triggers_is_algorithm_1():
    shape = (12, 10, 9)
    h = I.default_h(shape)
    b = I.rhs_uniform(shape, seed=24)
    x0, r0 = O.bicgstab(b, h, rtol=1e-10, maxit=500, precond=O.PC_CHEB, degree=4)
    x1, r1 = O.bicgstab(b, h, rtol=1e-10, maxit=500, precond=O.PC_CHEB, degree=4, rr_every=r0.iterations + 1)
    assert r1.iterations == r0.iterations and np.array_equal(x0, x1)


@pytest.mark.parametrize("pc", PCS[:2])
def test_residual_replacement_every_iteration_closes_the_residual_gap(pc):
    """With rr_every = 1 the recursive residual at exit is one update away from a
    true one, so it agrees with the recomputed true residual far below rtol, and the
    iteration count stays within a few of Algorithm 1's."""
    shape = (16, 16, 16)
    h = I.default_h(shape)
    b = I.rhs_uniform(shape, seed=42)
    rtol = 1e-10
    xa, ra = O.bicgstab(b, h, rtol=rtol, maxit=2000, precond=pc[0], degree=pc[1] + 2)
    x, res = O.bicgstab(b, h, rtol=rtol, maxit=2000, precond=pc[0], degree=pc[1] + 2, rr_every=1)
    assert res.status == O.OK and res.rel_res_recursive <= rtol
    assert abs(res.rel_res_true - res.rel_res_recursive) <= 1e-3 * rtol
    assert abs(res.iterations - ra.iterations) <= 2
    assert rel(x, xa) <= 1e-8


def test_residual_replacement_rejects_negative_period():
    b = I.rhs_uniform((4, 4, 4), seed=1)
    with pytest.raises(ValueError):
        O.bicgstab(b, I.default_h((4, 4, 4)), rr_every=-1)


# ------------------------------------------------ Neumann faces (Eq. 5) --
# Face conditions x-, x+, y-, y+, z-, z+: 0 Dirichlet (D, Eq. 4), 1 zero-flux
# Neumann (N, Eq. 5: first row (2, -2) for a Neumann minus face, last row
# (-2, 2) for a Neumann plus face).
def N1(n, fm, fp):
    M = D1(n)
    if fm:
        M[0, 1] = -2.0
    if fp:
        M[n - 1, n - 2] = -2.0
    return M


def axis_matrix(n, fm, fp, nblocks=1):
    """1-D operator of one axis, block-diagonal over `nblocks` equal blocks: the
    domain's faces keep their condition, faces between blocks are Dirichlet (Eq. 14)."""
    m = n // nblocks
    M = np.zeros((n, n))
    for b in range(nblocks):
        M[b * m:(b + 1) * m, b * m:(b + 1) * m] = N1(m, fm if b == 0 else 0, fp if b == nblocks - 1 else 0)
    return M


def dense_P_bc(shape, h, bc, blocks=(1, 1, 1)):
    """Eq. 6 with each O_d the D or N matrix its faces call for."""
    nz, ny, nx = shape
    hx, hy, hz = h
    Ox = axis_matrix(nx, bc[0], bc[1], blocks[0]) / hx ** 2
    Oy = axis_matrix(ny, bc[2], bc[3], blocks[1]) / hy ** 2
    Oz = axis_matrix(nz, bc[4], bc[5], blocks[2]) / hz ** 2
    return (np.kron(np.eye(nz), np.kron(np.eye(ny), Ox)) + np.kron(np.eye(nz), np.kron(Oy, np.eye(nx)))
            + np.kron(Oz, np.kron(np.eye(ny), np.eye(nx))))


BCS = [I.PAPER_BC, (1, 0, 0, 1, 0, 1), (1, 1, 0, 0, 0, 1), (0, 0, 0, 1, 0, 0)]


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("blocks", [None, (2, 1, 2)])
def test_neumann_stencil_equals_dense_kronecker(bc, blocks):
    shape = (4, 6, 8)
    h = (0.25, 0.2, 0.3)
    u = I.rhs_uniform(shape, seed=81)
    P = dense_P_bc(shape, h, bc, blocks if blocks else (1, 1, 1))
    assert np.allclose(O.apply_A(u, h, blocks=blocks, bc=bc).ravel(), P @ u.ravel(), rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("bc", BCS)
def test_neumann_eig_bounds_match_dense_spectrum(bc):
    shape = (5, 6, 7)
    h = (0.3, 0.2, 0.25)
    ev = np.linalg.eigvals(dense_P_bc(shape, h, bc))
    assert np.max(np.abs(ev.imag)) < 1e-8  # N is similar to a symmetric matrix
    lo, hi = O.eig_bounds((shape[2], shape[1], shape[0]), h, bc=bc)
    assert lo == pytest.approx(ev.real.min(), rel=1e-10) and hi == pytest.approx(ev.real.max(), rel=1e-10)


@pytest.mark.parametrize("bc", [I.PAPER_BC, (1, 1, 0, 0, 0, 1)])
def test_neumann_bj_interval_covers_every_block(bc):
    shape = (6, 6, 9)
    h = (0.2, 0.25, 0.3)
    blocks = (3, 2, 3)
    ev = np.linalg.eigvals(dense_P_bc(shape, h, bc, blocks)).real
    a, b = O.cheb_interval(shape, h, O.PC_BJ_CHEB, blocks=blocks, bc=bc)
    assert a == pytest.approx(ev.min(), rel=1e-10) and b == pytest.approx(ev.max(), rel=1e-10)
    # G(CI) / GNoComm(CI): the whole grid's bounds
    ev_g = np.linalg.eigvals(dense_P_bc(shape, h, bc)).real
    for pc in (O.PC_CHEB, O.PC_GNOCOMM_CHEB):
        a, b = O.cheb_interval(shape, h, pc, blocks=blocks, bc=bc)
        assert a == pytest.approx(ev_g.min(), rel=1e-10) and b == pytest.approx(ev_g.max(), rel=1e-10)


@pytest.mark.parametrize("bc", BCS[:2])
def test_neumann_chebyshev_matches_spectral_closed_form(bc):
    """Algorithm 2 applies p_d(A) b with p_d the Chebyshev residual polynomial's
    companion (x = (1 - T_{d+1}-shaped residual) / lambda); checked through the
    eigen-decomposition of the (nonsymmetric, diagonalisable) dense operator."""
    shape = (4, 5, 6)
    h = (0.2, 0.3, 0.25)
    P = dense_P_bc(shape, h, bc)
    lam, V = np.linalg.eig(P)
    lam, V = lam.real, V.real
    a, b = O.cheb_interval(shape, h, O.PC_CHEB, bc=bc)
    rhs = I.rhs_uniform(shape, seed=82)
    for d in (1, 3, 6):
        x = O.cheb(rhs, h, a, b, d, bc=bc).ravel()
        theta, delta = (b + a) / 2, (b - a) / 2
        t = (theta - lam) / delta
        s = theta / delta
        Tk = lambda k, z: np.cosh(k * np.arccosh(z)) if np.all(z >= 1) else np.cos(k * np.arccos(np.clip(z, -1, 1)))
        res_poly = Tk(d + 1, t) / np.cosh((d + 1) * np.arccosh(s))  # residual polynomial on the spectrum
        coef = np.linalg.solve(V, rhs.ravel())
        expect = V @ ((1 - res_poly) / lam * coef)
        assert rel(x, expect) <= 1e-9, d


@pytest.mark.parametrize("bc", BCS[:3])
@pytest.mark.parametrize("pc", [(O.PC_NONE, 0, (1, 1, 1)), (O.PC_CHEB, 4, (1, 1, 1)),
                                (O.PC_BJ_CHEB, 3, (2, 1, 2)), (O.PC_GNOCOMM_CHEB, 3, (2, 1, 2))])
def test_neumann_bicgstab_matches_dense_solve(bc, pc):
    shape = (4, 6, 8)
    h = (0.25, 0.2, 0.3)
    P = dense_P_bc(shape, h, bc)
    b = I.rhs_uniform(shape, seed=83)
    x, res = O.bicgstab(b, h, rtol=1e-12, maxit=2000, precond=pc[0], degree=pc[1], blocks=pc[2], bc=bc)
    assert res.status == O.OK
    assert rel(x, np.linalg.solve(P, b.ravel())) <= 10 * np.linalg.cond(P) * 1e-12
    assert res.rel_res_true <= 1e-11


def test_neumann_manufactured_second_order_convergence():
    """u = sin(pi x/2) cos(pi y/2) cos(pi z/2) meets the set-up's face conditions
    (Dirichlet at x = 0, y = 1, z = 1; Neumann at x = 1, y = 0, z = 0); the
    discrete solution converges to it at second order."""
    errs = []
    for n in (8, 16, 32):
        shape = (n, n, n)
        f, u = I.rhs_manufactured_bc(shape, I.PAPER_BC)
        h = I.default_h_bc(shape, I.PAPER_BC)
        x, res = O.bicgstab(f, h, rtol=1e-12, maxit=4000, precond=O.PC_CHEB, degree=6, bc=I.PAPER_BC)
        assert res.status == O.OK
        errs.append(np.max(np.abs(x - u)))
    assert 3.3 < errs[0] / errs[1] < 4.7 and 3.3 < errs[1] / errs[2] < 4.7, errs


def test_neumann_rejects_bad_faces():
    u = I.rhs_uniform((4, 4, 4), seed=1)
    with pytest.raises(ValueError):
        O.apply_A(u, (0.1, 0.1, 0.1), bc=(2, 0, 0, 0, 0, 0))
    with pytest.raises(ValueError):  # a Neumann face needs two points per block on its axis
        O.apply_A(u, (0.1, 0.1, 0.1), blocks=(4, 1, 1), bc=(1, 0, 0, 0, 0, 0))
    with pytest.raises(ValueError):  # Neumann on every face: singular, no Chebyshev interval
        O.cheb_interval((4, 4, 4), (0.1, 0.1, 0.1), O.PC_CHEB, bc=(1, 1, 1, 1, 1, 1))


# ------------------------- flexible preconditioners G(BiCGS), BJ(BiCGS) --
# M_i^-1 v is an inner Bi-CGSTAB solve of A z = v (whole grid, or each block
# with Dirichlet ghosts towards its neighbours) from z = 0, stopped at an
# inner tolerance; the outer iteration is Algorithm 1 with that M_i.
@pytest.mark.parametrize("bc", [None, I.PAPER_BC])
def test_inner_solve_preconditioners_approach_exact_inverses(bc):
    shape = (4, 6, 8)
    h = (0.25, 0.2, 0.3)
    bcs = bc if bc is not None else (0,) * 6
    v = I.rhs_uniform(shape, seed=91)
    z = O.precond_apply(v, h, O.PC_G_BICGS, 0, bc=bc, inner_rtol=1e-13, inner_maxit=1000)
    assert rel(z, np.linalg.solve(dense_P_bc(shape, h, bcs), v.ravel())) <= 1e-10
    blocks = (2, 1, 2)
    zb = O.precond_apply(v, h, O.PC_BJ_BICGS, 0, blocks=blocks, bc=bc, inner_rtol=1e-13, inner_maxit=1000)
    assert rel(zb, np.linalg.solve(dense_P_bc(shape, h, bcs, blocks), v.ravel())) <= 1e-10


def test_exact_inner_solve_makes_the_outer_iteration_stop_at_the_first_half_step():
    """With M = A (inner solve to round-off), p^ = A^-1 r0, w = r0, alpha = 1 and s = 0."""
    shape = (5, 6, 7)
    h = I.default_h(shape)
    b = I.rhs_uniform(shape, seed=92)
    x, res = O.bicgstab(b, h, rtol=1e-10, maxit=50, precond=O.PC_G_BICGS, inner_rtol=1e-14, inner_maxit=2000)
    assert res.status == O.OK and res.iterations == 1 and res.half_step_exit
    assert rel(x, np.linalg.solve(dense_P(shape, h), b.ravel())) <= 1e-11


@pytest.mark.parametrize("pc,blocks,tol", [(O.PC_G_BICGS, (1, 1, 1), 1e-2), (O.PC_BJ_BICGS, (2, 2, 2), 1e-6)])
@pytest.mark.parametrize("bc", [None, I.PAPER_BC])
def test_flexible_bicgstab_matches_dense_solve(pc, blocks, tol, bc):
    shape = (8, 8, 12)
    h = (0.1, 0.12, 0.09)
    bcs = bc if bc is not None else (0,) * 6
    b = I.rhs_uniform(shape, seed=93)
    x, res = O.bicgstab(b, h, rtol=1e-10, maxit=500, precond=pc, blocks=blocks, bc=bc, inner_rtol=tol,
                        inner_maxit=500)
    P = dense_P_bc(shape, h, bcs)
    assert res.status == O.OK and res.rel_res_true <= 1.1e-10
    assert rel(x, np.linalg.solve(P, b.ravel())) <= 10 * np.linalg.cond(P) * 1e-10


# ------------------------------------------------- the OpenMP build ---------
# The same source compiled with -fopenmp: loops spread over threads, dot
# products as the Dot2 recurrence over 64 fixed index ranges joined in order.
# It runs the long stored 256^3 reference solves and the timed CPU baseline;
# these pins hold it to the same facts as the serial build and to the serial
# build itself.
@pytest.fixture
def omp_build():
    prev = O.use_build("omp")
    yield
    O.use_build(prev)


@pytest.mark.parametrize("cond", ["plain", "cancelling"])
def test_omp_dot2_near_correctly_rounded(omp_build, cond):
    test_dot2_near_correctly_rounded(cond)
    test_dot_empty_and_single()


def test_omp_dot_does_not_depend_on_thread_count(omp_build):
    rng = np.random.default_rng(8)
    a, b = rng.standard_normal(100_003), rng.standard_normal(100_003)
    vals = []
    for t in (1, 3, 8):
        O.threads(t)
        vals.append(O.dot(a, b))
    O.threads(os.cpu_count() or 1)
    assert vals[0] == vals[1] == vals[2]


@pytest.mark.parametrize("shape", [(6, 5, 4), (6, 6, 6)])
@pytest.mark.parametrize("pc", PCS[:3])
def test_omp_bicgstab_matches_dense_solve(omp_build, shape, pc):
    test_bicgstab_matches_dense_solve(shape, pc, False)


def test_omp_build_follows_the_serial_build():
    """G(CI) d=8 on 40x36x44 (three threads): the OpenMP build's solve agrees
    with the serial build's to rounding (same iteration count, solutions and
    residual histories within 1e-12)."""
    shape = (44, 36, 40)
    h = I.default_h(shape)
    b = I.rhs_uniform(shape, seed=5)
    xs, rs = O.bicgstab(b, h, rtol=1e-10, maxit=300, precond=O.PC_CHEB, degree=8)
    prev = O.use_build("omp")
    try:
        O.threads(3)
        xo, ro = O.bicgstab(b, h, rtol=1e-10, maxit=300, precond=O.PC_CHEB, degree=8)
        O.threads(os.cpu_count() or 1)
    finally:
        O.use_build(prev)
    assert rs.status == ro.status == O.OK and rs.iterations == ro.iterations
    assert rel(xo, xs) <= 1e-12
    np.testing.assert_allclose(ro.hist_s, rs.hist_s, rtol=1e-12)


def test_snapshots_equal_runs_stopped_there():
    """x copied out after iteration k of a longer solve is the iterate of a
    solve with maxit = k; slots past the exit stay NaN."""
    shape = (12, 10, 14)
    h = I.default_h(shape)
    b = I.rhs_uniform(shape, seed=3)
    x, r = O.bicgstab(b, h, rtol=1e-10, maxit=100, precond=O.PC_CHEB, degree=4, snapshots=(2, 5, 1000))
    for k in (2, 5):
        xk, rk = O.bicgstab(b, h, rtol=0.0, maxit=k, precond=O.PC_CHEB, degree=4)
        assert rk.iterations == k and np.array_equal(xk, r.snapshots[k])
    assert np.isnan(r.snapshots[1000]).all()
