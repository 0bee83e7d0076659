"""FP64 sweeps split 32-plane work units into two halves (sweep_split): a grid
forced to 32-plane slabs through a planted tune-cache entry, with a ragged
last slab (nz = 80: 32 + 32 + 16 planes, so one half-unit is empty), solved
against the oracle, and the persistent single-launch form bitwise equal to
the graph-replayed one."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_08935_b300 import inputs as I

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHAPE = (80, 24, 40)  # (nz, ny, nx)

CHILD = r"""
import json, sys, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_2503_08935_b300 import binding as B
from paper_2503_08935_b300 import inputs as I
shape = {shape!r}
b = torch.from_numpy(I.rhs_uniform(shape, seed=1201)).cuda()
out = {{}}
for name, kw in (("graph", {{}}), ("persistent", {{"persistent": 1}})):
    x = torch.zeros_like(b)
    with B.Solver(shape, autotune=1, **kw) as s:
        info = s.solve(b, x, rtol=1e-10, maxit=500, precond=B.PC_CHEB, degree=6)
    torch.cuda.synchronize()
    np.save({tmp!r} + "/x_" + name + ".npy", x.cpu().numpy())
    out[name] = {{"zc": info.slab_planes, "tuned": info.tuned, "status": info.status, "it": info.iterations,
                  "rt": info.rel_res_true}}
print(json.dumps(out))
"""


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_split_units_with_ragged_slab_match_oracle(tmp_path):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nz, ny, nx = SHAPE
    cache = tmp_path / "tune.txt"
    cache.write_text(f"psolve-tune-1 {sms} {nx} {ny} {nz} 0 32 1 1.0\n")  # 32-plane slabs, TMA ring
    env = dict(os.environ, PSOLVE_TUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, shape=SHAPE, tmp=str(tmp_path))], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    g, p = res["graph"], res["persistent"]
    assert g["zc"] == 32 and g["tuned"] == 2 and g["status"] == 0 and p["status"] == 0
    xg, xp = np.load(tmp_path / "x_graph.npy"), np.load(tmp_path / "x_persistent.npy")
    assert g["it"] == p["it"] and np.array_equal(xg, xp)
    bn = I.rhs_uniform(SHAPE, seed=1201)
    xo, ro = O.bicgstab(bn, I.default_h(SHAPE), rtol=1e-10, maxit=500, precond=O.PC_CHEB, degree=6)
    assert ro.status == O.OK and abs(g["it"] - ro.iterations) <= 2, (g["it"], ro.iterations)
    assert float(np.linalg.norm(xg - xo) / np.linalg.norm(xo)) <= 1e-8
    assert g["rt"] <= 1.1e-10
