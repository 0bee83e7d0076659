"""The persistent solve (opts.persistent = 1): the whole solve of a launch
list as one cooperative kernel launch with grid barriers between phases.  It
runs the same phase program and engine code as the per-kernel path, so its
results must be bitwise those of that path, for every preconditioner,
precision, stencil engine and for uneven batches."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_08935_b300 import binding as B
from paper_2503_08935_b300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()


def run(shape, b, precond, degree, rtol=1e-10, maxit=500, x0=None, **kw):
    x = torch.zeros(shape, dtype=torch.float64, device=DEV) if x0 is None else x0.clone()
    with B.Solver(shape, **kw) as s:
        info = s.solve(b, x, rtol=rtol, maxit=maxit, precond=precond, degree=degree)
    torch.cuda.synchronize()
    return x.cpu().numpy(), info


CASES = [
    # (shape (nz, ny, nx), precond, degree, opts)
    ((24, 32, 40), B.PC_CHEB, 8, {}),                                   # TMA ring, exact bounds
    ((23, 19, 37), B.PC_CHEB, 6, {}),                                   # TMA ring on padded rows (nx % 8 != 0)
    ((23, 19, 37), B.PC_CHEB, 6, dict(engine=1)),                       # general engine
    ((24, 32, 40), B.PC_CHEB, 8, dict(lmin_scale=100.0, lmax_scale=1 - 1e-4)),  # rescaled bounds (y term)
    ((24, 32, 40), B.PC_CHEB, 8, dict(cheb_prec=B.FP32)),
    ((32, 32, 32), B.PC_BJ_CHEB, 6, dict(cheb_prec=B.FP32, blocks=(2, 2, 2))),
    ((32, 32, 32), B.PC_GNOCOMM_CHEB, 4, dict(cheb_prec=B.BF16, blocks=(2, 2, 2))),
    ((16, 24, 48), B.PC_CHEB, 1, {}),                                   # degree 1: no sweeps
    ((9, 10, 11), B.PC_NONE, 0, {}),
]


@pytest.mark.parametrize("shape,precond,degree,kw", CASES)
@pytest.mark.parametrize("use_graph", [1, 0])
def test_persistent_bitwise_equals_per_kernel(shape, precond, degree, kw, use_graph):
    b = torch.from_numpy(I.rhs_uniform(shape, seed=301)).to(DEV)
    xr, ir = run(shape, b, precond, degree, **kw)
    xp, ip = run(shape, b, precond, degree, persistent=1, use_graph=use_graph, **kw)
    assert ip.status == ir.status and ip.iterations == ir.iterations
    assert ip.half_step_exit == ir.half_step_exit
    assert ip.rel_res_recursive == ir.rel_res_recursive and ip.rel_res_true == ir.rel_res_true
    assert np.array_equal(xp, xr)
    assert ip.kernel_launches == 1
    assert ip.model_bytes == ir.model_bytes


def test_persistent_unpreconditioned_32cubed_manufactured_matches_oracle():
    """The 32^3 unpreconditioned manufactured-solution case, through one launch."""
    shape = (32, 32, 32)
    bn = I.rhs_manufactured(shape)
    b = torch.from_numpy(bn).to(DEV)
    xp, ip = run(shape, b, B.PC_NONE, 0, maxit=2000, persistent=1)
    xo, ro = O.bicgstab(bn, I.default_h(shape), rtol=1e-10, maxit=2000, precond=O.PC_NONE, degree=0)
    assert ip.status == B.OK
    assert abs(ip.iterations - ro.iterations) <= 2
    assert np.linalg.norm(xp - xo) / np.linalg.norm(xo) <= 1e-8


def test_persistent_with_initial_guess_and_repeat_calls():
    shape = (16, 16, 24)
    b = torch.from_numpy(I.rhs_uniform(shape, seed=302)).to(DEV)
    x0 = torch.from_numpy(0.01 * I.rhs_uniform(shape, seed=303)).to(DEV)
    xr, ir = run(shape, b, B.PC_CHEB, 5, x0=x0, use_x0=1)
    # the same context twice: the cached single-launch graph is replayed
    x = x0.clone()
    with B.Solver(shape, use_x0=1, persistent=1) as s:
        i1 = s.solve(b, x, rtol=1e-10, maxit=500, precond=B.PC_CHEB, degree=5)
        x1 = x.cpu().numpy()
        x.copy_(x0)
        i2 = s.solve(b, x, rtol=1e-10, maxit=500, precond=B.PC_CHEB, degree=5)
        x2 = x.cpu().numpy()
    assert i1.iterations == ir.iterations == i2.iterations
    assert np.array_equal(x1, xr) and np.array_equal(x2, xr)


def test_persistent_edge_cases():
    shape = (8, 8, 16)
    zero = torch.zeros(shape, dtype=torch.float64, device=DEV)
    # b = 0 with a nonzero initial guess: x = 0, status OK, no iterations
    x0 = torch.ones(shape, dtype=torch.float64, device=DEV)
    x, info = run(shape, zero, B.PC_CHEB, 4, x0=x0, use_x0=1, persistent=1)
    assert info.status == B.OK and info.iterations == 0 and not x.any()
    assert info.rel_res_true == 0.0
    # maxit = 0: not converged, nothing iterated
    b = torch.from_numpy(I.rhs_uniform(shape, seed=304)).to(DEV)
    x, info = run(shape, b, B.PC_CHEB, 4, maxit=0, persistent=1)
    assert info.status == B.NOT_CONVERGED and info.iterations == 0
    # a maxit that stops the solve early: same state as the per-kernel path
    xr, ir = run(shape, b, B.PC_CHEB, 4, maxit=3)
    xp, ip = run(shape, b, B.PC_CHEB, 4, maxit=3, persistent=1)
    assert ip.status == ir.status == B.NOT_CONVERGED and ip.iterations == ir.iterations == 3
    assert np.array_equal(xp, xr)
    # one point (unpreconditioned: one point has an empty Chebyshev interval)
    one = torch.ones((1, 1, 1), dtype=torch.float64, device=DEV)
    x1, i1 = run((1, 1, 1), one, B.PC_NONE, 0, persistent=1)
    xr1, ir1 = run((1, 1, 1), one, B.PC_NONE, 0)
    assert i1.status == ir1.status == B.OK and np.array_equal(x1, xr1)


def test_persistent_rejects_timing_mode():
    shape = (8, 8, 8)
    b = torch.ones(shape, dtype=torch.float64, device=DEV)
    x = torch.zeros_like(b)
    with B.Solver(shape, persistent=1, timing=1) as s:
        with pytest.raises(B.PsolveError) as e:
            s.solve(b, x, precond=B.PC_CHEB, degree=2)
    assert e.value.status == B.E_ARG


@pytest.mark.parametrize("prec", [B.FP64, B.FP32])
def test_persistent_batch_bitwise_equals_per_kernel_batch(prec):
    shapes = I.batch_shapes(10, seed=2, sides=(16, 24, 32, 40, 48)) + [(17, 9, 33), (5, 7, 3)]
    bs = [torch.from_numpy(I.rhs_uniform(sh, seed=400 + q)).to(DEV) for q, sh in enumerate(shapes)]
    xr = [torch.zeros(sh, dtype=torch.float64, device=DEV) for sh in shapes]
    xp = [torch.zeros(sh, dtype=torch.float64, device=DEV) for sh in shapes]
    ir = B.solve_batch(bs, xr, rtol=1e-10, maxit=500, precond=B.PC_CHEB, degree=8, cheb_prec=prec)
    ip = B.solve_batch(bs, xp, rtol=1e-10, maxit=500, precond=B.PC_CHEB, degree=8, cheb_prec=prec, persistent=1)
    torch.cuda.synchronize()
    for q in range(len(shapes)):
        assert ip[q].status == ir[q].status == B.OK
        assert ip[q].iterations == ir[q].iterations
        assert np.array_equal(xp[q].cpu().numpy(), xr[q].cpu().numpy())
    assert ip[0].kernel_launches == 1


def test_persistent_batch_mixed_stop_times():
    """Problems that stop early (b = 0, easy grids) idle while others iterate."""
    shapes = [(32, 32, 32), (4, 4, 8), (24, 24, 24), (8, 8, 8)]
    bs = [torch.from_numpy(I.rhs_uniform(sh, seed=500 + q)).to(DEV) for q, sh in enumerate(shapes)]
    bs[3].zero_()
    xr = [torch.zeros(sh, dtype=torch.float64, device=DEV) for sh in shapes]
    xp = [torch.zeros(sh, dtype=torch.float64, device=DEV) for sh in shapes]
    ir = B.solve_batch(bs, xr, rtol=1e-10, maxit=500, precond=B.PC_NONE, degree=0)
    ip = B.solve_batch(bs, xp, rtol=1e-10, maxit=500, precond=B.PC_NONE, degree=0, persistent=1)
    torch.cuda.synchronize()
    for q in range(len(shapes)):
        assert ip[q].status == ir[q].status and ip[q].iterations == ir[q].iterations
        assert np.array_equal(xp[q].cpu().numpy(), xr[q].cpu().numpy())
    assert ip[3].iterations == 0


def test_grid_barrier_gives_up_when_a_cta_never_arrives():
    """Failure detection without a GPU fault: one CTA of a cooperative launch
    skips the persistent kernel's grid barrier; every other CTA gives up after
    the (short) wait limit, raises the error word and returns."""
    import time
    ok = B.selfcheck_grid_timeout(limit_ns=20_000_000, absent_cta=-1)
    assert ok["passed"] == ok["ctas"] and ok["gave_up"] == 0 and ok["error_word"] == 0
    t0 = time.perf_counter()
    bad = B.selfcheck_grid_timeout(limit_ns=20_000_000, absent_cta=0)
    elapsed = time.perf_counter() - t0
    assert bad["passed"] == 0 and bad["gave_up"] == bad["ctas"] - 1 and bad["error_word"] == 1
    assert elapsed < 2.0
    # the context is still usable afterwards
    shape = (8, 8, 16)
    b = torch.from_numpy(I.rhs_uniform(shape, seed=305)).to(DEV)
    x, info = run(shape, b, B.PC_CHEB, 4, persistent=1)
    assert info.status == B.OK
