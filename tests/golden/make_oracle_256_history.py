"""Write tests/golden/oracle_256_cheb8_history.json: the FP64 oracle's view of
the 256^3 benchmark problem (h = 1/257, b ~ U[-1,1) splitmix64 seed 1, x0 = 0,
G(CI) degree 8 with exact closed-form bounds, rtol 1e-10) in the form the
fixed-iteration and history parity tests need:

  * the full solve's residual history ||s_i||/||b|| and ||r_i||/||b||
    (Algorithm 1) and its stopping point;
  * the solution after exactly 10, 30 and 60 iterations (rtol 0) at the 4096
    seeded sample points of oracle_256_cheb8.json, with ||x||_2;
  * the oracle's own sensitivity: the same runs for right-hand sides
    perturbed by 1e-15 relative noise (seeds 1001..), reduced to how far their
    solutions (whole vector and samples) and histories move from the
    unperturbed ones, and where they stop.

Calls only oracle/ and the input generators.  Runs the OpenMP build of the
oracle (the same arithmetic per point; dot products summed over fixed index
ranges, so its results do not depend on the thread count, but may differ in
the last bit from the serial build's single running sum).  The serial
build's stored solve (oracle_256_cheb8.json) is compared with the OpenMP one
as one more measurement of the oracle's own rounding spread.  Takes about an
hour on 8 cores."""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle as O  # noqa: E402
from paper_2503_08935_b300 import inputs as I  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "oracle_256_cheb8_history.json")
FIXED = (10, 30, 60)
PERTURB_SEEDS = (1001, 1002, 1003, 1004)
EPS = 1e-15


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def hist_list(h):
    return [None if not np.isfinite(v) else float(v) for v in h]


def solve(b, h, log):
    """Full solve of b with x snapshots after the FIXED iteration counts."""
    t = time.time()
    x, r = O.bicgstab(b, h, rtol=1e-10, maxit=500, precond=O.PC_CHEB, degree=8, snapshots=FIXED)
    log(f"  {r.iterations} iterations (half-step exit {r.half_step_exit}), {time.time() - t:.0f} s")
    assert r.status == O.OK and all(np.all(np.isfinite(r.snapshots[k])) for k in FIXED)
    return x, r


def main():
    log = lambda m: print(m, flush=True)  # noqa: E731
    O.use_build("omp")
    threads = O.threads()
    shape = (256, 256, 256)
    h = I.default_h(shape)
    b = I.rhs_uniform(shape, seed=1)
    serial = json.load(open(os.path.join(HERE, "oracle_256_cheb8.json")))
    idx = np.array(serial["sample_index"], dtype=np.int64)

    log(f"unperturbed ({threads} threads)")
    t0 = time.time()
    xb, rb = solve(b, h, log)
    out = {
        "what": "FP64 oracle (OpenMP build), 256^3, h=1/257, b=U[-1,1) seed 1, G(CI) degree 8, "
                "scales (1,1), rtol 1e-10",
        "threads": threads,
        "iterations": rb.iterations, "half_step_exit": rb.half_step_exit,
        "rel_res_recursive": rb.rel_res_recursive, "rel_res_true": rb.rel_res_true,
        "hist_s": hist_list(rb.hist_s), "hist_r": hist_list(rb.hist_r),
        "sample_seed": serial["sample_seed"], "sample_x": xb.ravel()[idx].tolist(),
        "x_norm2": float(np.linalg.norm(xb)),
        "serial_build": {"iterations": serial["iterations"], "half_step_exit": serial["half_step_exit"],
                         "rel_res_recursive": serial["rel_res_recursive"],
                         "final_rel_l2_samples_vs_omp": rel(np.array(serial["sample_x"]), xb.ravel()[idx])},
        "fixed": {},
        "perturbed": {"eps": EPS, "seeds": list(PERTURB_SEEDS), "runs": []},
    }
    for k in FIXED:
        xk = rb.snapshots[k]
        out["fixed"][str(k)] = {"sample_x": xk.ravel()[idx].tolist(), "x_norm2": float(np.linalg.norm(xk))}
    for seed in PERTURB_SEEDS:
        log(f"b perturbed by {EPS:g} relative noise, seed {seed}")
        xp, rp = solve(I.perturb_relative(b, seed, EPS), h, log)
        rec = {
            "seed": seed, "iterations": rp.iterations, "half_step_exit": rp.half_step_exit,
            "rel_res_recursive": rp.rel_res_recursive, "rel_res_true": rp.rel_res_true,
            "hist_s": hist_list(rp.hist_s), "hist_r": hist_list(rp.hist_r),
            "final_rel_l2": rel(xp, xb), "final_rel_l2_samples": rel(xp.ravel()[idx], xb.ravel()[idx]),
            "fixed": {str(k): {"rel_l2": rel(rp.snapshots[k], rb.snapshots[k]),
                               "rel_l2_samples": rel(rp.snapshots[k].ravel()[idx], rb.snapshots[k].ravel()[idx])}
                      for k in FIXED},
        }
        out["perturbed"]["runs"].append(rec)
        log(f"  final rel-L2 vs unperturbed {rec['final_rel_l2']:.3e}; after "
            + ", ".join(f"{k}: {rec['fixed'][str(k)]['rel_l2']:.2e}" for k in FIXED))
        del xp, rp
    out["oracle_seconds"] = time.time() - t0
    with open(OUT, "w") as f:
        json.dump(out, f)
    log(f"wrote {OUT} in {out['oracle_seconds']:.0f} s")


if __name__ == "__main__":
    main()
