"""Zero-flux Neumann faces (matrix N, Eq. 5) on the GPU against the oracle:
the operator on both stencil engines, with and without the block restriction,
the Chebyshev preconditioner, whole solves for every preconditioner, the
persistent form, and the experimental set-up's problem (mixed faces, its
right-hand side, GNoComm(CI) with 24 Chebyshev iterations and rescaled
bounds)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_08935_b300 import binding as B
from paper_2503_08935_b300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
BCS = [I.PAPER_BC, (1, 0, 0, 1, 0, 1), (1, 1, 0, 0, 0, 1)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("shape", [(12, 16, 40), (11, 13, 21)])  # TMA ring, unpadded and padded rows
@pytest.mark.parametrize("blocked", [0, 1])
def test_neumann_apply_A_matches_oracle(bc, shape, blocked):
    h = (0.07, 0.05, 0.09)
    blocks = (2, 1, 1) if shape[2] % 2 == 0 else (1, 1, 1)
    u = I.rhs_uniform(shape, seed=801)
    out = torch.empty(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape, h, bc=bc, blocks=blocks) as s:
        s.apply_A(dev(u), out, block_restricted=blocked)
    torch.cuda.synchronize()
    ref = O.apply_A(u, h, blocks=blocks if blocked else None, bc=bc)
    assert rel(out.cpu().numpy(), ref) <= 1e-14


@pytest.mark.parametrize("bc", BCS[:2])
@pytest.mark.parametrize("precond,blocks", [(B.PC_CHEB, (1, 1, 1)), (B.PC_BJ_CHEB, (2, 2, 2)),
                                            (B.PC_GNOCOMM_CHEB, (2, 2, 2))])
def test_neumann_preconditioner_matches_oracle(bc, precond, blocks):
    shape = (16, 16, 24)
    h = (0.05, 0.06, 0.07)
    v = I.rhs_uniform(shape, seed=802)
    out = torch.empty(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape, h, bc=bc, blocks=blocks) as s:
        a, b = s.cheb_interval(precond)
        s.precond_apply(dev(v), out, precond=precond, degree=7)
    torch.cuda.synchronize()
    ao, bo = O.cheb_interval(shape, h, precond, blocks=blocks, bc=bc)
    assert a == pytest.approx(ao, rel=1e-13) and b == pytest.approx(bo, rel=1e-13)
    ref = O.precond_apply(v, h, precond, 7, blocks=blocks, bc=bc)
    assert rel(out.cpu().numpy(), ref) <= 1e-12


SOLVES = [
    (B.PC_CHEB, 8, (1, 1, 1), {}),
    (B.PC_CHEB, 8, (1, 1, 1), dict(lmin_scale=100.0, lmax_scale=1 - 1e-4)),
    (B.PC_GNOCOMM_CHEB, 6, (2, 2, 2), {}),
    (B.PC_BJ_CHEB, 6, (2, 2, 2), {}),
    (B.PC_NONE, 0, (1, 1, 1), {}),
]


@pytest.mark.parametrize("bc", BCS[:2])
@pytest.mark.parametrize("precond,degree,blocks,kw", SOLVES)
def test_neumann_solve_matches_oracle(bc, precond, degree, blocks, kw):
    shape = (16, 24, 32)
    h = (0.05, 0.06, 0.07)
    bn = I.rhs_uniform(shape, seed=803)
    x = torch.zeros(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape, h, bc=bc, blocks=blocks, **kw) as s:
        info = s.solve(dev(bn), x, rtol=1e-10, maxit=3000, precond=precond, degree=degree)
    torch.cuda.synchronize()
    xo, ro = O.bicgstab(bn, h, rtol=1e-10, maxit=3000, precond=precond, degree=degree, blocks=blocks, bc=bc,
                        **kw)
    assert info.status == B.OK and ro.status == O.OK
    slack = 2 if precond == B.PC_CHEB else max(2, int(0.15 * ro.iterations))
    assert abs(info.iterations - ro.iterations) <= slack, (info.iterations, ro.iterations)
    assert rel(x.cpu().numpy(), xo) <= 1e-8
    assert info.rel_res_true <= 1.1e-10


@pytest.mark.parametrize("bc", BCS[:2])
def test_neumann_engines_and_persistent_agree_bitwise(bc):
    shape = (16, 24, 32)
    h = (0.05, 0.06, 0.07)
    b = dev(I.rhs_uniform(shape, seed=804))
    outs = []
    for kw in ({}, dict(engine=1), dict(persistent=1)):
        x = torch.zeros(shape, dtype=torch.float64, device=DEV)
        with B.Solver(shape, h, bc=bc, **kw) as s:
            info = s.solve(b, x, rtol=1e-10, maxit=500, precond=B.PC_CHEB, degree=6)
        torch.cuda.synchronize()
        outs.append((info.iterations, x.cpu().numpy()))
    assert outs[0][0] == outs[1][0] == outs[2][0]
    assert np.array_equal(outs[0][1], outs[1][1]) and np.array_equal(outs[0][1], outs[2][1])


def test_neumann_mixed_precision_reaches_the_fp64_residual():
    shape = (32, 32, 32)
    h = I.default_h_bc(shape, I.PAPER_BC)
    f, _ = I.rhs_manufactured_bc(shape, I.PAPER_BC)
    x = torch.zeros(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape, h, bc=I.PAPER_BC, cheb_prec=B.FP32) as s:
        info = s.solve(dev(f), x, rtol=1e-10, maxit=500, precond=B.PC_CHEB, degree=8)
    torch.cuda.synchronize()
    xo, ro = O.bicgstab(f, h, rtol=1e-10, maxit=500, precond=O.PC_CHEB, degree=8, bc=I.PAPER_BC)
    assert info.status == B.OK and info.rel_res_true <= 1.5e-10
    assert rel(x.cpu().numpy(), xo) <= 1e-7


def test_paper_problem_64_gnocomm_matches_oracle():
    """The set-up's single-device case: 64^3 unknowns on its box (h = 0.4), Dirichlet
    faces x-, y+, z+, Neumann faces x+, y-, z-, f = sin x + cos y + 3 sin z - 2yz + 2
    normalised, GNoComm(CI) without subdivision, 24 Chebyshev iterations, bounds
    lambda_min x 10, lambda_max x (1 - 1e-4), rtol 1e-10."""
    shape = (64, 64, 64)
    h = (0.4, 0.4, 0.4)
    bn = I.rhs_paper_problem(shape, h=h)
    kw = dict(lmin_scale=10.0, lmax_scale=1 - 1e-4)
    x = torch.zeros(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape, h, bc=I.PAPER_BC, **kw) as s:
        info = s.solve(dev(bn), x, rtol=1e-10, maxit=500, precond=B.PC_GNOCOMM_CHEB, degree=24)
    torch.cuda.synchronize()
    xo, ro = O.bicgstab(bn, h, rtol=1e-10, maxit=500, precond=O.PC_GNOCOMM_CHEB, degree=24, bc=I.PAPER_BC, **kw)
    assert info.status == B.OK and ro.status == O.OK
    assert abs(info.iterations - ro.iterations) <= 2, (info.iterations, ro.iterations)
    assert rel(x.cpu().numpy(), xo) <= 1e-8
