"""The 256^3 benchmark problem (h = 1/257, b ~ U[-1,1) seed 1, G(CI) degree 8
with exact bounds, rtol 1e-10) against the FP64 oracle's stored runs
(tests/golden/oracle_256_cheb8_history.json, written by
tests/golden/make_oracle_256_history.py from the oracle alone).

Every tolerance here comes from a measurement of the oracle itself: the same
oracle solve repeated on right-hand sides perturbed by 1e-15 relative noise
(Algorithm 1 is unchanged; only rounding-sized differences enter).  Those runs
agree to ~1e-15 for ten iterations, then rounding is amplified: from about
iteration 38 their residual histories differ by more than 1 %, after 60
iterations their iterates differ by ~7e-4, and they stop anywhere between 137
and 144 iterations, yet their solutions agree to ~1e-10.  The GPU computes the
same recurrence with different rounding in every operation (other summation
orders, fused multiply-adds, scaled Chebyshev iterates), which acts like a
perturbation of about 1e-13 rather than 1e-15.  So:

* before the amplification (histories) and at fixed iteration counts (iterates)
  the GPU may differ from the oracle by 100x the oracle's own response to a
  1e-15 perturbation (the response to ~1e-13), with a floor of 1e-13 (history)
  or 1e-12 (iterates) where that response is below rounding;
* the stopping iteration is compared as a distribution: the median over the
  unperturbed and eight perturbed right-hand sides on the GPU against the
  oracle's median over its six stored runs, within +-2, or half the oracle's
  interquartile range if that is larger;
* every GPU solve's solution is within rel-L2 1e-8 of the oracle's, and its
  true residual within 1.1 rtol.
"""
import json
import os

import numpy as np
import pytest
import torch

from paper_2503_08935_b300 import binding as B
from paper_2503_08935_b300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SHAPE = (256, 256, 256)
RTOL = 1e-10
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SEEDS = (1001, 1002, 1003, 1004, 1005, 1006, 1007, 1008)  # GPU perturbations (oracle: 1001..1004)


def _arr(values):
    return np.array([np.nan if v is None else v for v in values], dtype=np.float64)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def gold():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()
    g = json.load(open(os.path.join(GOLDEN, "oracle_256_cheb8_history.json")))
    serial = json.load(open(os.path.join(GOLDEN, "oracle_256_cheb8.json")))
    g["sample_index"] = serial["sample_index"]
    g["serial_iterations"] = serial["iterations"]
    return g


@pytest.fixture(scope="module")
def solver():
    with B.Solver(SHAPE, I.default_h(SHAPE), record_history=1) as s:
        yield s


def _samples(x, gold):
    idx = torch.tensor(gold["sample_index"], dtype=torch.int64, device=DEV)
    return x.reshape(-1)[idx].cpu().numpy()


@pytest.mark.parametrize("k", [10, 30, 60])
def test_fixed_iterations_within_oracle_rounding_response(gold, solver, k):
    """rtol = 0, exactly k outer iterations on both sides: the GPU iterate at the
    4096 sample points is within 100x the oracle's own change under 1e-15
    perturbations of b (at least 1e-12), as is its norm."""
    spread = max(r["fixed"][str(k)]["rel_l2_samples"] for r in gold["perturbed"]["runs"])
    tol = max(1e-12, 100.0 * spread)
    b = torch.from_numpy(I.rhs_uniform(SHAPE, seed=1)).to(DEV)
    x = torch.zeros(SHAPE, dtype=torch.float64, device=DEV)
    info = solver.solve(b, x, rtol=0.0, maxit=k, precond=B.PC_CHEB, degree=8, raise_on_error=False)
    assert info.status == B.NOT_CONVERGED and info.iterations == k
    ref = gold["fixed"][str(k)]
    err = _rel(_samples(x, gold), np.array(ref["sample_x"]))
    print(f"256^3 after {k} iterations: GPU vs oracle {err:.2e}, oracle's own spread {spread:.2e}, tol {tol:.2e}")
    assert err <= tol
    assert abs(float(torch.linalg.vector_norm(x)) - ref["x_norm2"]) <= tol * ref["x_norm2"]


def test_residual_history_tracks_oracle_until_rounding_takes_over(gold, solver):
    """The recorded ||r_i||/||b|| and ||s_i||/||b|| follow the oracle's history
    within max(1e-13, 100x the oracle's own relative change under 1e-15
    perturbations) for every iteration before the one where that change first
    exceeds 1 % (about iteration 38); the GPU stops at the first iteration
    where its own recorded residual passes rtol."""
    orr, ors = _arr(gold["hist_r"]), _arr(gold["hist_s"])
    env_r, env_s = np.zeros(len(orr)), np.zeros(len(ors))
    for run in gold["perturbed"]["runs"]:
        pr, ps = _arr(run["hist_r"]), _arr(run["hist_s"])
        m = min(len(pr), len(orr))
        env_r[:m] = np.fmax(env_r[:m], np.abs(pr[:m] - orr[:m]) / orr[:m])
        m = min(len(ps), len(ors))
        env_s[:m] = np.fmax(env_s[:m], np.abs(ps[:m] - ors[:m]) / ors[:m])
    istar = int(np.argmax(env_r > 0.01))
    assert 20 <= istar <= 60, istar  # the oracle's own amplification point
    b = torch.from_numpy(I.rhs_uniform(SHAPE, seed=1)).to(DEV)
    x = torch.zeros(SHAPE, dtype=torch.float64, device=DEV)
    info = solver.solve(b, x, rtol=RTOL, maxit=500, precond=B.PC_CHEB, degree=8)
    hs, hr = solver.history()
    hs, hr = np.asarray(hs), np.asarray(hr)
    assert info.status == B.OK and len(hs) == len(hr) == info.iterations
    for name, g_, o_, env in (("r", hr, orr, env_r), ("s", hs, ors, env_s)):
        dev_ = np.abs(g_[:istar] - o_[:istar]) / o_[:istar]
        tol = np.maximum(1e-13, 100.0 * env[:istar])
        worst = int(np.argmax(dev_ / tol))
        print(f"history {name}: worst deviation/tolerance {dev_[worst] / tol[worst]:.2f} at iteration {worst + 1}")
        assert np.all(dev_ <= tol), (worst + 1, dev_[worst], tol[worst])
    # the exit is the GPU's own first pass of the test (half step or full step)
    passed = [i for i in range(len(hs)) if hs[i] <= RTOL or (np.isfinite(hr[i]) and hr[i] <= RTOL)]
    assert passed and passed[0] == info.iterations - 1


def test_stopping_iteration_and_solution_in_distribution(gold, solver):
    """The convergence tail is erratic: at a fixed iteration the oracle's own
    perturbed runs differ by up to 5x in residual, and they stop anywhere in
    137..144.  The GPU is run on the same right-hand side and on eight
    1e-15-perturbed ones; the median of its stopping iterations must be within
    max(2, half the oracle's interquartile range) of the median of the
    oracle's six stored runs (four perturbed, the unperturbed OpenMP build and
    the serial build).  Every GPU solution is within rel-L2 1e-8 of the
    oracle's at the sample points, with a true residual within 1.1 rtol."""
    oracle_its = [gold["iterations"], gold["serial_iterations"]] + [r["iterations"] for r in
                                                                     gold["perturbed"]["runs"]]
    q1, med_o, q3 = np.percentile(oracle_its, [25, 50, 75])
    xo = np.array(gold["sample_x"])
    b0 = I.rhs_uniform(SHAPE, seed=1)
    x = torch.zeros(SHAPE, dtype=torch.float64, device=DEV)
    gpu_its, errs = [], []
    for seed in (None,) + SEEDS:
        bb = b0 if seed is None else I.perturb_relative(b0, seed, 1e-15)
        info = solver.solve(torch.from_numpy(bb).to(DEV), x, rtol=RTOL, maxit=500, precond=B.PC_CHEB, degree=8)
        assert info.status == B.OK and info.rel_res_true <= 1.1 * RTOL, (seed, info.rel_res_true)
        gpu_its.append(info.iterations)
        errs.append(_rel(_samples(x, gold), xo))
    med_g = float(np.median(gpu_its))
    slack = max(2.0, 0.5 * (q3 - q1))
    print(f"256^3 stopping iterations: GPU {gpu_its} (median {med_g}), oracle {sorted(oracle_its)} "
          f"(median {med_o}, IQR {q3 - q1}); rel-L2 vs oracle {min(errs):.1e}..{max(errs):.1e}")
    assert abs(med_g - med_o) <= slack
    assert max(errs) <= 1e-8
