"""Write tests/golden/oracle_256_cheb8.json: the FP64 oracle's solve of the
256^3 benchmark problem (h = 1/257, b ~ U[-1,1) splitmix64 seed 1, x0 = 0,
G(CI) degree 8 with exact closed-form bounds, rtol 1e-10), reduced to what a
test can compare: status, iterations, residuals, ||x||_2 and x at 4096 seeded
sample points.  Calls only oracle/ and the input generators.  Serial; takes
about ten minutes."""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle as O  # noqa: E402
from paper_2503_08935_b300 import inputs as I  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_256_cheb8.json")


def main():
    shape = (256, 256, 256)
    h = I.default_h(shape)
    b = I.rhs_uniform(shape, seed=1)
    t = time.time()
    x, r = O.bicgstab(b, h, rtol=1e-10, maxit=500, precond=O.PC_CHEB, degree=8)
    secs = time.time() - t
    idx = (I.splitmix64(99, 4096) % np.uint64(b.size)).astype(np.int64)
    out = {
        "what": "FP64 oracle, 256^3, h=1/257, b=U[-1,1) seed 1, G(CI) degree 8, scales (1,1), rtol 1e-10",
        "status": r.status, "iterations": r.iterations, "half_step_exit": r.half_step_exit,
        "rel_res_recursive": r.rel_res_recursive, "rel_res_true": r.rel_res_true,
        "x_norm2": float(np.linalg.norm(x)), "sample_seed": 99,
        "sample_index": idx.tolist(), "sample_x": x.ravel()[idx].tolist(),
        "oracle_seconds_serial": secs,
    }
    with open(OUT, "w") as f:
        json.dump(out, f)
    print(f"iterations {r.iterations}, {secs:.0f} s -> {OUT}")


if __name__ == "__main__":
    main()
