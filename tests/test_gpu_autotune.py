"""The slab-depth / stencil-engine autotuner (opts.autotune): its choice is
valid, a tuned solve still matches the oracle, a tuned grid decomposes the
same way alone and in a batch (bitwise equal results), and the on-disk cache
named by PSOLVE_TUNE_CACHE is written and obeyed by a later process."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_08935_b300 import binding as B
from paper_2503_08935_b300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()


def run(shape, b, precond, degree, rtol=1e-10, maxit=500, **kw):
    x = torch.zeros(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape, **kw) as s:
        info = s.solve(b, x, rtol=rtol, maxit=maxit, precond=precond, degree=degree)
    torch.cuda.synchronize()
    return x.cpu().numpy(), info


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("shape,prec", [((24, 32, 40), B.FP64), ((23, 19, 37), B.FP64), ((64, 64, 64), B.FP32)])
def test_autotuned_solve_is_valid_and_matches_oracle(shape, prec):
    bn = I.rhs_uniform(shape, seed=701)
    b = torch.from_numpy(bn).to(DEV)
    x, info = run(shape, b, B.PC_CHEB, 8, autotune=1, cheb_prec=prec)
    assert info.tuned in (1, 2)
    zc = info.slab_planes
    assert 1 <= zc <= min(32, shape[0]) and zc & (zc - 1) == 0
    assert info.engine in (0, 1)  # nx = 37: padded rows, either engine may be chosen
    xo, ro = O.bicgstab(bn, I.default_h(shape), rtol=1e-10, maxit=500, precond=O.PC_CHEB, degree=8)
    assert info.status == B.OK and info.rel_res_true <= 1.1e-10
    if prec == B.FP64:
        assert abs(info.iterations - ro.iterations) <= 2 and rel(x, xo) <= 1e-8
    else:  # FP32 Chebyshev vectors: another preconditioner, so only the solution is compared
        assert rel(x, xo) <= 1e-6


def test_autotuned_batch_equals_autotuned_alone():
    shapes = [(24, 32, 40), (17, 9, 33), (32, 32, 32), (8, 40, 16)]
    bs = [torch.from_numpy(I.rhs_uniform(sh, seed=710 + q)).to(DEV) for q, sh in enumerate(shapes)]
    xs = [torch.zeros(sh, dtype=torch.float64, device=DEV) for sh in shapes]
    infos = B.solve_batch(bs, xs, rtol=1e-10, maxit=500, precond=B.PC_CHEB, degree=6, autotune=1)
    torch.cuda.synchronize()
    for q, sh in enumerate(shapes):
        xa, ia = run(sh, bs[q], B.PC_CHEB, 6, autotune=1)
        assert infos[q].tuned in (1, 2) and infos[q].slab_planes == ia.slab_planes
        assert infos[q].engine == ia.engine
        assert infos[q].status == B.OK and infos[q].iterations == ia.iterations
        assert np.array_equal(xs[q].cpu().numpy(), xa)


CHILD = r"""
import json, sys, torch
sys.path.insert(0, {root!r})
from paper_2503_08935_b300 import binding as B
from paper_2503_08935_b300 import inputs as I
shape = (24, 32, 40)
b = torch.from_numpy(I.rhs_uniform(shape, seed=720)).cuda()
x = torch.zeros_like(b)
with B.Solver(shape, autotune=1) as s:
    info = s.solve(b, x, rtol=1e-10, maxit=500, precond=B.PC_CHEB, degree=6)
print(json.dumps({{"zc": info.slab_planes, "engine": info.engine, "tuned": info.tuned, "status": info.status}}))
"""


def _child(cache):
    env = dict(os.environ, PSOLVE_TUNE_CACHE=str(cache))
    out = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_tune_cache_file_is_written_and_obeyed(tmp_path):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # a fresh cache: the child measures and appends its decision
    fresh = tmp_path / "fresh.txt"
    r = _child(fresh)
    assert r["status"] == B.OK and r["tuned"] == 1
    lines = fresh.read_text().splitlines()
    decisions = [ln.split() for ln in lines if ln.startswith("psolve-tune-1")]
    assert len(decisions) == 1 and list(map(int, decisions[0][1:8])) == [sms, 40, 32, 24, 0, r["zc"], r["engine"]]
    # every measured candidate is recorded as a comment line before it
    cands = [ln.split() for ln in lines if ln.startswith("# candidate")]
    assert len(cands) >= 6 and all(list(map(int, c[2:7])) == [sms, 40, 32, 24, 0] for c in cands)
    assert min(float(c[9]) for c in cands) == pytest.approx(float(decisions[0][8]), rel=1e-3)
    # a planted entry: the child takes it without measuring
    planted = tmp_path / "planted.txt"
    planted.write_text(f"garbage line\npsolve-tune-1 {sms} 40 32 24 0 2 0 1.0\npsolve-tune-1 {sms} 40 32 24 0 8 1 0.5\n")
    r = _child(planted)
    assert r == {"zc": 2, "engine": 0, "tuned": 2, "status": B.OK}
