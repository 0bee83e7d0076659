"""Residual history (opts.record_history, psolve_history) against the oracle's
history of Algorithm 1, and the GNoComm(CI) degree warning (the paper's N_s/2
bound)."""
import math

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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def gpu_solve_hist(shape, b, rtol, maxit, precond, degree, **kw):
    x = torch.zeros(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape, record_history=1, **kw) as s:
        info = s.solve(dev(b), x, rtol=rtol, maxit=maxit, precond=precond, degree=degree)
        hs, hr = s.history()
    return x.cpu().numpy(), info, hs, hr


@pytest.mark.parametrize("prec", [B.FP64, B.FP32])
def test_history_tracks_oracle(prec):
    """G(CI) d=4 on a ragged grid: the recorded ||s_i||/||b|| and ||r_i||/||b||
    follow the oracle's.  The iterates agree to rounding for the first ~10
    iterations (1e-12 relative on the norms, FP64); FP32 Chebyshev vectors are
    a different preconditioner, compared only for the first iteration (the
    residual r0 = b is exact, and s_1 depends on M only through alpha)."""
    shape = (24, 20, 36)
    h = I.default_h(shape)
    b = I.rhs_uniform(shape, seed=11)
    x, info, hs, hr = gpu_solve_hist(shape, b, 1e-10, 300, B.PC_CHEB, 4, cheb_prec=prec)
    xo, ro = O.bicgstab(b, h, rtol=1e-10, maxit=300, precond=O.PC_CHEB, degree=4)
    assert info.status == B.OK
    assert len(hs) == len(hr) == info.iterations
    # the GPU stopped at the first iteration where its own recorded residual passed
    rtol = 1e-10
    passed = [i for i in range(len(hs)) if hs[i] <= rtol or (np.isfinite(hr[i]) and hr[i] <= rtol)]
    assert passed and passed[0] == info.iterations - 1
    if info.half_step_exit:
        assert hs[-1] <= rtol and np.isnan(hr[-1])
    else:
        assert hr[-1] <= rtol
    assert np.all(np.isfinite(hs)) and np.all(np.isfinite(hr[:-1]))
    if prec == B.FP64:
        k = min(10, len(hs), len(ro.hist_s))
        np.testing.assert_allclose(hs[:k], ro.hist_s[:k], rtol=1e-12)
        np.testing.assert_allclose(hr[:k], ro.hist_r[:k], rtol=1e-12)
        assert abs(info.iterations - ro.iterations) <= 2
    # the recorded last value is the result's recursive residual
    last = hs[-1] if info.half_step_exit else hr[-1]
    assert math.isclose(last, info.rel_res_recursive, rel_tol=1e-14)


def test_history_with_residual_replacement_matches_oracle():
    """With residual replacement the recorded r-norm of a replacement iteration
    is that of the true residual b - A x, as in the oracle."""
    shape = (20, 16, 24)
    h = I.default_h(shape)
    b = I.rhs_uniform(shape, seed=12)
    x, info, hs, hr = gpu_solve_hist(shape, b, 1e-10, 200, B.PC_CHEB, 4, rr_every=3)
    xo, ro = O.bicgstab(b, h, rtol=1e-10, maxit=200, precond=O.PC_CHEB, degree=4, rr_every=3)
    k = min(9, len(hr), len(ro.hist_r))
    np.testing.assert_allclose(hr[:k], ro.hist_r[:k], rtol=1e-11)
    np.testing.assert_allclose(hs[:k], ro.hist_s[:k], rtol=1e-11)


def test_history_persistent_equals_per_kernel():
    """The single-launch solve records the same history bitwise."""
    shape = (32, 24, 40)
    b = I.rhs_uniform(shape, seed=13)
    _, i1, hs1, hr1 = gpu_solve_hist(shape, b, 1e-10, 300, B.PC_CHEB, 6)
    _, i2, hs2, hr2 = gpu_solve_hist(shape, b, 1e-10, 300, B.PC_CHEB, 6, persistent=1)
    assert i1.iterations == i2.iterations
    assert np.array_equal(hs1, hs2, equal_nan=True) and np.array_equal(hr1, hr2, equal_nan=True)


def test_history_needs_the_option_and_a_solve():
    shape = (8, 8, 8)
    with B.Solver(shape) as s:
        with pytest.raises(B.PsolveError):
            s.history()
    with B.Solver(shape, record_history=1) as s:
        with pytest.raises(B.PsolveError):
            s.history()  # nothing solved yet
        b = dev(I.rhs_uniform(shape, seed=3))
        x = torch.zeros(shape, dtype=torch.float64, device=DEV)
        s.solve(b, x, rtol=1e-10, maxit=5, precond=B.PC_CHEB, degree=2)
        hs, hr = s.history()
        assert len(hs) <= 5
        # a longer solve than the buffer held grows it
        info = s.solve(b, x, rtol=0.0, maxit=40, precond=B.PC_NONE, degree=0)
        hs, hr = s.history()
        assert len(hs) == info.iterations == 40 and np.all(np.isfinite(hr))


def test_gnocomm_degree_above_half_block_side_warns():
    """GNoComm(CI) with 4x4x4 blocks of 6 points: degree 3 = N_s/2 runs
    silently, degree 4 runs with a warning (the paper's N_s/2 upper bound);
    the status is the solve's own."""
    shape = (24, 24, 24)
    b = dev(I.rhs_uniform(shape, seed=14))
    x = torch.zeros(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape, blocks=(4, 4, 4)) as s:
        info = s.solve(b, x, rtol=1e-8, maxit=500, precond=B.PC_GNOCOMM_CHEB, degree=3)
        assert info.status == B.OK and B.last_error() == ""
        info = s.solve(b, x, rtol=1e-8, maxit=500, precond=B.PC_GNOCOMM_CHEB, degree=4)
        assert info.status == B.OK
        assert B.last_error().startswith("warning:") and "GNoComm" in B.last_error()
