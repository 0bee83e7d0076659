"""Benchmark: 256^3 Poisson solve, Bi-CGSTAB with the Chebyshev preconditioner.

One step = one complete solve of the 256^3 problem (h = 1/257, zero Dirichlet,
b ~ U[-1, 1) splitmix64 seed 1, x0 = 0, G(CI) degree 8 with exact closed-form
eigenvalue bounds, FP64, rtol 1e-10): every row of the hot path (initial
residual, fused direction update + Chebyshev sweep 1, sweeps 2..8, stencil +
dot, half-step update + sweeps, stencil + 2 dots, x/r update + 2 dots, true
residual) runs in the library's CUDA kernels.  `value` is solves per second
with b resident in HBM; `e2e` is the same through psolve_solve_host with the
host->device copy of b and the device->host copy of x inside the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With torchrun (N > 1) every rank solves its own replica (no collective on the
data path: the solve does not shard without a halo exchange), timing is the
max over ranks and `value` is the total solves/s.  `--impl reference` times
the FP64 CPU oracle on this host on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "256³ time-to-rtol 1e-10 & HBM GB/s; batched solves/s; p50/p99 serve latency"
SHAPE = (256, 256, 256)
RTOL = 1e-10
MAXIT = 500
DEGREE = 8
WORKLOAD = "poisson 256^3 FP64, Bi-CGSTAB + G(CI) Chebyshev degree 8, exact bounds, rtol 1e-10"
GOLDEN_256 = os.path.join(ROOT, "tests", "golden", "oracle_256_cheb8.json")
# ncu summaries of the dominant kernel per Chebyshev precision (the FP32/BF16 sweeps run two points per thread)
NCU_SUMMARY = {"fp64": os.path.join(ROOT, "profiles", "ncu_ci_sweep4_256_fp64.md"),
               "fp32": os.path.join(ROOT, "profiles", "ncu_ci_sweep_pair_256_fp32.md"),
               "bf16": os.path.join(ROOT, "profiles", "ncu_ci_sweep_pair_256_bf16.md")}
KERNEL_SRC = os.path.join(ROOT, "paper_2503_08935_b300", "csrc", "psolve_kernels.cuh")
# FP64 instructions per point of a Chebyshev sweep k >= 3 (exact bounds, where the
# y coefficient vanishes; see OpCiSweep): b, y_{k-2} and the six neighbours of
# y_{k-1} are combined with three neighbour-pair sums and four fused multiply-adds
# (7, the least for eight inputs); every iterate, p^ and r^ included, is stored
# scaled so that b enters with coefficient 1.


def sweep4_fp64_ops_per_point(degree):
    """Mean FP64 instructions per point over the sweeps k = 3..degree."""
    return 7.0


# FP64 instructions per grid point of each kernel class of the FP64 solve
# (exact bounds, Chebyshev degree >= 2, TMA ring, 32-plane work units).  CI
# sweep 1 forms its right-hand side u on every cell of its 36 x 10 halo box
# per 32 x 8 tile and on the unit's two halo planes (the direction update
# p = r + beta (p - omega w): 2 fused multiply-adds per cell; the half step
# s = r - alpha w: 1), then 3 pair sums and 3 fused multiply-adds per point,
# plus ||s||^2 on the s side; the two sides alternate, so the class mean is
# their average.  The others: sweep k = 2: 3 adds + 3 fmas; k >= 3: 3 adds +
# 4 fmas; stencil + dot: A u / cc (3 adds + 3 fmas) + 1; stencil + 2 dots:
# 6 + 2; update: x (2 fmas), r (1 fma), 2 dots.  ncu's per-opcode counters
# (DADD + DFMA executed per point) agree: 9.0 for the p side of sweep 1, 6.0
# and 7.0 for the sweeps; the dot kernels execute 0.15-0.45 more in their
# per-unit reductions, which the counts below leave out.
HALO_CELLS_PER_POINT_FP64 = (32 + 2 * 2) * (8 + 2) / (32 * 8) * (32 + 2) / 32
FP64_OPS_PER_POINT = {
    "ci_first": 0.5 * ((2 * HALO_CELLS_PER_POINT_FP64 + 6) + (HALO_CELLS_PER_POINT_FP64 + 6 + 1)),
    "ci_sweep3": 6.0, "ci_sweep4": 7.0, "stencil_dot": 7.0, "stencil_2dot": 8.0, "update": 5.0,
}


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(ms, dist, device):
    """The step time of the slowest rank (every rank gets it); ms itself on one rank."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(world, ms_per_step):
    """Whole-job solves/s: every rank solves one problem per step (replicas)."""
    return world * 1e3 / ms_per_step


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def kernel_source_hash():
    with open(KERNEL_SRC, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def ncu_traffic_per_point(prec):
    """DRAM bytes per algorithmic byte of the captured ci_sweep4 launch in the
    committed ncu summary, or None if there is none or the kernel source
    changed since."""
    try:
        txt = open(NCU_SUMMARY[prec]).read()
    except OSError:
        return None
    vals = {}
    for line in txt.splitlines():
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_point"]) / float(vals["algorithmic_bytes_per_point"])
    except (KeyError, ValueError, ZeroDivisionError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples go where PSOLVE_CLOCKS_DIR says (kept for inspection), else to /tmp
        out_dir = os.environ.get("PSOLVE_CLOCKS_DIR") or "/tmp"
        self.path = os.path.join(out_dir, f"psolve_clocks_rank{index}_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        power = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": num(rows[0][2]),
                "power_w_max": max(power) if power else None, "samples": len(rows), "reasons": reasons}


# ------------------------------------------------------------- reference --
def cpu_info():
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def _oracle(threads):
    """The OpenMP build of the oracle with `threads` threads (0: every core);
    returns the module and the thread count in use.  Its arithmetic per point
    is the serial oracle's; dot products are summed over fixed index ranges."""
    import oracle as O
    O.use_build("omp")
    n = O.threads(threads if threads > 0 else (os.cpu_count() or 1))
    return O, n


def oracle_sample(shape=SHAPE, threads=0):
    """Bounded oracle sample on the full problem: the oracle's solve with
    maxit = 0 (set-up + true residual) and maxit = 1 (one more outer
    iteration).  Returns (t_setup, t_iteration, threads) in seconds."""
    from paper_2503_08935_b300 import inputs as I
    O, n = _oracle(threads)
    h = I.default_h(shape)
    b = I.rhs_uniform(shape, seed=1)
    t = time.perf_counter()
    O.bicgstab(b, h, rtol=0.0, maxit=0, precond=O.PC_CHEB, degree=DEGREE)
    t0 = time.perf_counter() - t
    t = time.perf_counter()
    O.bicgstab(b, h, rtol=0.0, maxit=1, precond=O.PC_CHEB, degree=DEGREE)
    t1 = time.perf_counter() - t
    return t0, max(t1 - t0, 1e-9), n


def oracle_full_solve(shape, threads, precond_name):
    """A complete oracle solve to rtol 1e-10: 32^3 is the manufactured-sine
    configuration (no preconditioner, converges at the first half step); other
    sizes the benchmark's recipe (U[-1,1) seed 1, G(CI) degree 8, exact bounds)."""
    from paper_2503_08935_b300 import inputs as I
    O, n = _oracle(threads)
    h = I.default_h(shape)
    if precond_name == "none":
        b, pc, deg = I.rhs_manufactured(shape), O.PC_NONE, 0
    else:
        b, pc, deg = I.rhs_uniform(shape, seed=1), O.PC_CHEB, DEGREE
    t = time.perf_counter()
    _, r = O.bicgstab(b, h, rtol=RTOL, maxit=2000, precond=pc, degree=deg)
    return {"grid": "x".join(map(str, shape[::-1])), "precond": precond_name, "threads": n,
            "seconds": time.perf_counter() - t, "iterations": r.iterations, "status": r.status,
            "rel_res_true": r.rel_res_true}


def oracle_iterations(default):
    try:
        with open(GOLDEN_256) as f:
            return int(json.load(f)["iterations"]), "stored oracle run (tests/golden/oracle_256_cheb8.json)"
    except Exception:
        return default, "iteration count of the GPU solve"


def cpu_baseline_record(iters_gpu):
    """The oracle timed on this host's cores: the 256^3 solve extrapolated from
    its set-up and one outer iteration (every core), plus the 32^3 and 64^3
    configurations solved to completion on every core and on one."""
    t_setup, t_iter, n = oracle_sample()
    iters, src = oracle_iterations(iters_gpu)
    t_solve = t_setup + iters * t_iter
    full = [oracle_full_solve((32, 32, 32), 0, "none"), oracle_full_solve((64, 64, 64), 0, "cheb8"),
            oracle_full_solve((64, 64, 64), 1, "cheb8")]
    rec = {"value": 1.0 / t_solve, "unit": "solves/s", "cores": n, "kind": "oracle",
           "sample": (f"OpenMP build of the FP64 oracle on {n} threads, full 256^3 problem: set-up + true "
                      f"residual ({t_setup:.2f} s) and one outer iteration ({t_iter:.2f} s); the solve is "
                      f"extrapolated to set-up + {iters} iterations ({src})"),
           "extrapolated": True, "seconds_per_solve_extrapolated": t_solve, "threads": n,
           "complete_solves": full}
    rec.update(cpu_info())
    return rec


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    # warm-up steps on a small sample (code and page cache), timed steps on the full problem
    for _ in range(args.warmup):
        oracle_sample((64, 64, 64))
    times = []
    iters, src = oracle_iterations(30)
    n = 1
    for _ in range(args.steps):
        t_setup, t_iter, n = oracle_sample()
        times.append(t_setup + iters * t_iter)
    t = statistics.mean(times)
    value = 1.0 / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": gpu_config(world, "fp64"),
        "cpu_baseline": dict({"value": value, "unit": "solves/s", "cores": n, "kind": "oracle",
                              "sample": (f"each step: OpenMP build of the FP64 oracle on {n} threads, set-up + "
                                         f"one outer iteration on the full 256^3 problem, extrapolated to "
                                         f"set-up + {iters} iterations ({src})")}, **cpu_info()),
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def gpu_config(world, prec):
    """The workload description both arms print (the same keys and values)."""
    return {"workload": WORKLOAD if prec == "fp64" else WORKLOAD + f", Chebyshev vectors {prec}",
            "grid": "256x256x256", "h": "1/257", "rhs": "U[-1,1) splitmix64 seed 1",
            "precond": "G(CI) degree 8, bounds (1,1)", "rtol": RTOL,
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": "inputs larger than L2: ~10 FP64 vectors of 134 MB each"}


# ------------------------------------------------------------------ GPU --
def run_gpu(args):
    import numpy as np
    import torch

    from paper_2503_08935_b300 import binding as B
    from paper_2503_08935_b300 import inputs as I

    rank, world, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)

    h = I.default_h(SHAPE)
    b_host = torch.from_numpy(I.rhs_uniform(SHAPE, seed=1)).pin_memory()
    b = b_host.to(dev)
    x = torch.zeros(SHAPE, dtype=torch.float64, device=dev)
    x_host = torch.empty(SHAPE, dtype=torch.float64).pin_memory()
    npts = b.numel()

    prec = {"fp64": B.FP64, "fp32": B.FP32, "bf16": B.BF16}[args.prec]
    # the headline solve as a caller runs it (the iteration loop replayed from a
    # CUDA graph); a second context with CUDA events around every kernel launch
    # (plain launches, 2-3% slower) gives the per-kernel times of the roofline
    solver = B.Solver(SHAPE, h, timing=0, stream=stream, cheb_prec=prec)
    ksolver = B.Solver(SHAPE, h, timing=1, stream=stream, cheb_prec=prec) if args.kernel_timing else None

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()

    def timed(fn, steps):
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        infos = [fn() for _ in range(steps)]
        ev1.record(stream)
        barrier()
        ms = max_over_ranks(ev0.elapsed_time(ev1), dist, dev)
        return ms, infos

    def solve_dev():
        info = solver.solve(b, x, rtol=RTOL, maxit=MAXIT, precond=B.PC_CHEB, degree=DEGREE)
        if info.status != B.OK:
            raise RuntimeError(f"solve status {info.status_name}")
        return info

    def solve_timed_kernels():
        info = ksolver.solve(b, x, rtol=RTOL, maxit=MAXIT, precond=B.PC_CHEB, degree=DEGREE)
        if info.status != B.OK:
            raise RuntimeError(f"solve status {info.status_name}")
        return info

    def solve_e2e():
        info = solver.solve_host(b_host, x_host, rtol=RTOL, maxit=MAXIT, precond=B.PC_CHEB, degree=DEGREE)
        if info.status != B.OK:
            raise RuntimeError(f"solve status {info.status_name}")
        return info

    for _ in range(args.warmup):
        solve_dev()
    with ClockSampler(dev.index) as clk:
        ms, infos = timed(solve_dev, args.steps)
    clocks = clk.summary()
    for _ in range(max(1, args.warmup // 2)):
        solve_e2e()
    ms_e2e, infos_e2e = timed(solve_e2e, args.steps)
    if ksolver is not None:
        for _ in range(max(1, args.warmup // 2)):
            solve_timed_kernels()
        ms_k, kinfos = timed(solve_timed_kernels, args.steps)

    per_step = ms / args.steps
    value = aggregate_value(world, per_step)
    iters = infos[-1].iterations
    model_bytes = statistics.mean(i.model_bytes for i in infos)
    launches = sum(i.kernel_launches for i in infos)

    # dominant kernel: Chebyshev sweep k >= 3 (reads y_{k-1}, b, y_{k-2}; writes y_k)
    peak, peak_kind = measured_peaks()
    roof = None
    breakdown = {}
    if args.kernel_timing:
        k = "ci_sweep4"
        kms = sum(i.kclass[k]["ms"] for i in kinfos)
        kn = sum(i.kclass[k]["launches"] for i in kinfos)
        kbytes = sum(i.kclass[k]["bytes"] for i in kinfos)
        avg_ms = kms / max(kn, 1)
        per_launch = kbytes / max(kn, 1)
        gbs = per_launch / (avg_ms * 1e-3) / 1e9
        ratio = ncu_traffic_per_point(args.prec)
        ctype = {"fp64": "double", "fp32": "float", "bf16": "__nv_bfloat16"}[args.prec]
        kname = ("k_engine<OpCiSweep<double,double,...>> (Chebyshev sweeps k>=3, scaled-iterate form)"
                 if args.prec == "fp64" else
                 f"k_engine<OpCiSweepPairW<{ctype},...>> (Chebyshev sweeps k>=4 two per pass, two points per "
                 f"thread) with OpCiSweepW (an odd last sweep alone)")
        roof = {"kernel": kname,
                # the captured launch's DRAM bytes per algorithmic byte times this class's algorithmic bytes
                "traffic": (ratio * kbytes / max(kn, 1)) if ratio is not None else None,
                "algorithmic_bytes_per_launch": per_launch, "avg_launch_ms": avg_ms, "launches": kn,
                "share_of_step": kms / ms_k if ms_k > 0 else None,
                "hbm_view": {"achieved_GBps": gbs, "peak_GBps": peak, "frac": gbs / peak,
                             "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, copy test)"}}
        if args.prec == "fp64":
            # the FP64 kernels are bound by the FP64 pipe: the peak is the FP64
            # instruction rate measured on this GPU by the library's own kernel
            # (independent fused multiply-add chains), in this process
            fma = B.measure_fp64_rate(kind=0, iters=8192, stream=stream)
            add = B.measure_fp64_rate(kind=1, iters=8192, stream=stream)
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            peak_ops = fma["instr_per_s"]
            opp = sweep4_fp64_ops_per_point(DEGREE)
            ops = opp * npts / (avg_ms * 1e-3)
            roof.update({"bound": "alu", "achieved": ops / 1e12, "peak": peak_ops / 1e12, "unit": "TFP64op/s",
                         "frac": ops / peak_ops,
                         "peak_kind": ("measured: psolve_measure_fp64_rate, independent FP64 fma chains on every "
                                       f"SM, {fma['ms']:.1f} ms run at {fma['sm_mhz']:.0f} MHz SM clock"),
                         "peak_fp64_add_Tinstr_s": add["instr_per_s"] / 1e12,
                         "peak_per_clock_per_sm": peak_ops / (sms * fma["sm_mhz"] * 1e6),
                         "ops_per_point": opp})
            floors = {}
            for name, opp_k in FP64_OPS_PER_POINT.items():
                kms_c = sum(i.kclass[name]["ms"] for i in kinfos)
                kn_c = sum(i.kclass[name]["launches"] for i in kinfos)
                if kn_c:
                    live_us = kms_c / kn_c * 1e3
                    floor_us = opp_k * npts / peak_ops * 1e6
                    floors[name] = {"fp64_instr_per_point": round(opp_k, 3), "floor_us": floor_us,
                                    "live_us_per_launch": live_us, "frac_of_fp64_peak": floor_us / live_us}
            roof["fp64_floor_per_kernel"] = floors
        else:
            roof.update({"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, copy test)"})
        for name in B.K_NAMES:
            kms_c = sum(i.kclass[name]["ms"] for i in kinfos)
            kb_c = sum(i.kclass[name]["bytes"] for i in kinfos)
            kn_c = sum(i.kclass[name]["launches"] for i in kinfos)
            if kn_c:
                breakdown[name] = {"ms_per_step": kms_c / args.steps, "launches_per_step": kn_c / args.steps,
                                   "GB/s": kb_c / (kms_c * 1e-3) / 1e9 if kms_c > 0 else None}
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.prec == "fp64" else f"f64 outer / {args.prec} Chebyshev",
        "data": "synthetic",
        "config": gpu_config(world, args.prec),
        "iterations": iters, "time_to_rtol_ms": per_step,
        "hbm_gbs_solve": model_bytes / (per_step * 1e-3) / 1e9,
        "model_bytes_per_solve": model_bytes,
        "rel_res_true": infos[-1].rel_res_true,
        "rel_l2_vs_oracle": rel_vs_oracle(x, oracle_samples(dev, torch), torch),
        "roofline": roof,
        "e2e": {"value": aggregate_value(world, ms_e2e / args.steps), "unit": "solves/s",
                "h2d_bytes_per_step": 8 * npts, "d2h_bytes_per_step": 8 * npts,
                "ms_per_step": ms_e2e / args.steps},
        "gpu_launches": launches,
        "clocks": clocks,
        "timing": ("value: the solve as a caller runs it, iteration loop replayed from a CUDA graph; roofline and "
                   "kernel_breakdown: a second timed loop of the same solves with CUDA events around every kernel "
                   "launch (plain launches)" if args.kernel_timing else "CUDA-graph replay; no per-kernel timing"),
    }
    if ksolver is not None:
        line["kernel_timing_ms_per_step"] = ms_k / args.steps
    if breakdown:
        line["kernel_breakdown"] = breakdown
    if args.variants and rank == 0:
        x_ref = x.clone()
        line["variants"] = run_variants(args, b, x_ref, stream, B, torch)
    if args.extras != "none" and rank == 0:
        line["configs"] = run_extras(args, B, I, torch, stream)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_record(iters)
    solver.close()
    if ksolver is not None:
        ksolver.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_variants(args, b, x_ref, stream, B, torch):
    """The same 256^3 problem with the Chebyshev vectors in FP32 and in BF16
    (FP64 outer iteration), and with the rescaled bounds of the experimental
    set-up (lambda_min x 100, lambda_max x (1 - 1e-4)), with residual
    replacement every 5 iterations, and the persistent single-launch form of
    the solve; each reports time to
    rtol 1e-10 (CUDA events, graph replay), iterations, the true residual and
    the relative L2 difference from the FP64 solution of the headline run."""
    out = {}
    cases = [("fp32_cheb8", dict(cheb_prec=B.FP32), B.PC_CHEB, 8),
             ("bf16_cheb8", dict(cheb_prec=B.BF16), B.PC_CHEB, 8),
             ("fp32_cheb16", dict(cheb_prec=B.FP32), B.PC_CHEB, 16),
             ("fp64_cheb8_paper_scaled", dict(lmin_scale=100.0, lmax_scale=1 - 1e-4), B.PC_CHEB, 8),
             ("fp32_cheb8_paper_scaled", dict(cheb_prec=B.FP32, lmin_scale=100.0, lmax_scale=1 - 1e-4),
              B.PC_CHEB, 8),
             ("fp64_gnocomm8_4x4x4", dict(blocks=(4, 4, 4)), B.PC_GNOCOMM_CHEB, 8),
             ("fp64_bj8_4x4x4", dict(blocks=(4, 4, 4)), B.PC_BJ_CHEB, 8),
             ("fp64_none", dict(), B.PC_NONE, 0),
             ("fp32_cheb8_rr5", dict(cheb_prec=B.FP32, rr_every=5), B.PC_CHEB, 8),
             ("bf16_cheb8_rr5", dict(cheb_prec=B.BF16, rr_every=5), B.PC_CHEB, 8),
             ("fp64_cheb8_persistent", dict(persistent=1), B.PC_CHEB, 8),
             ("fp32_cheb8_persistent", dict(cheb_prec=B.FP32, persistent=1), B.PC_CHEB, 8)]
    h = (1.0 / 257,) * 3
    x = torch.zeros_like(b)
    gold = oracle_samples(b.device, torch)
    for name, kw, pc, deg in cases:
        with B.Solver(SHAPE, h, stream=stream, **kw) as s:
            maxit = 5000 if pc == B.PC_NONE else MAXIT
            s.solve(b, x, rtol=RTOL, maxit=maxit, precond=pc, degree=deg)  # warm-up (graph capture)
            steps = max(1, min(args.steps, 3))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                info = s.solve(b, x, rtol=RTOL, maxit=maxit, precond=pc, degree=deg)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
        rel = float(torch.linalg.vector_norm(x - x_ref) / torch.linalg.vector_norm(x_ref))
        out[name] = {"status": info.status_name, "time_to_rtol_ms": ms, "iterations": info.iterations,
                     "rel_res_true": info.rel_res_true, "rel_l2_vs_fp64_solution": rel,
                     "rel_l2_vs_oracle": rel_vs_oracle(x, gold, torch),
                     "model_gb_per_s": info.model_bytes / (ms * 1e-3) / 1e9, "engine": info.engine}
    return out


def oracle_samples(device, torch):
    """The stored FP64 oracle solve of this problem (serial oracle, G(CI) degree
    8, exact bounds, rtol 1e-10) at its 4096 seeded sample points, or None."""
    try:
        with open(GOLDEN_256) as f:
            g = json.load(f)
    except OSError:
        return None
    return (torch.tensor(g["sample_index"], dtype=torch.int64, device=device),
            torch.tensor(g["sample_x"], dtype=torch.float64, device=device))


def rel_vs_oracle(x, gold, torch):
    """Relative L2 difference from the oracle's solution at its sample points."""
    if gold is None:
        return None
    idx, xo = gold
    return float(torch.linalg.vector_norm(x.reshape(-1)[idx] - xo) / torch.linalg.vector_norm(xo))


# --------------------------------------------------------------- extras --
def _timed_cuda(fn, stream, torch, reps=1):
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def extra_small_latency(B, I, torch, stream, reps=200):
    """32^3, h = 1/33, f = 3 pi^2 sin sin sin, no preconditioner, rtol 1e-10:
    the first half step converges, so this measures per-solve latency (median
    of five blocks of reps/5 solves; every block's mean is reported too)."""
    import math
    shape = (32, 32, 32)
    h = I.default_h(shape)
    f = I.rhs_manufactured(shape)
    b = torch.from_numpy(f).cuda()
    x = torch.zeros_like(b)
    per_mode, blocks = {}, {}
    for mode, kw in (("graph", {}), ("persistent", {"persistent": 1})):
        with B.Solver(shape, h, stream=stream, **kw) as s:
            for _ in range(10):
                info = s.solve(b, x, rtol=1e-10, maxit=2000, precond=B.PC_NONE)
            # the solve is host-bound at this size, and the host is shared:
            # five blocks of reps/5 solves, the median block reported
            runs = [_timed_cuda(lambda: s.solve(b, x, rtol=1e-10, maxit=2000, precond=B.PC_NONE), stream,
                                torch, max(1, reps // 5)) for _ in range(5)]
        blocks[mode] = sorted(r[0] * 1e3 for r in runs)
        per_mode[mode] = (sorted(r[0] for r in runs)[2], runs[-1][1])
    best = min(per_mode, key=lambda m: per_mode[m][0])
    ms, info = per_mode[best]
    xh = x.cpu().numpy()
    lam111 = 3 * 4.0 / h[0] ** 2 * math.sin(math.pi * h[0] / 2) ** 2
    exact_discrete = f / lam111
    exact_cont = f / (3 * math.pi ** 2)
    import numpy as np
    return {"workload": "32^3 manufactured sine, no preconditioner, rtol 1e-10", "us_per_solve": ms * 1e3,
            "solves_per_s": 1e3 / ms, "mode": best,
            "us_per_solve_graph": per_mode["graph"][0] * 1e3,
            "us_per_solve_persistent": per_mode["persistent"][0] * 1e3,
            "blocks_us_per_solve": blocks,
            "iterations": info.iterations, "half_step_exit": info.half_step_exit,
            "rel_err_vs_exact_discrete": float(np.linalg.norm(xh - exact_discrete) / np.linalg.norm(exact_discrete)),
            "max_err_vs_continuous": float(np.max(np.abs(xh - exact_cont))),
            "kernel_launches_per_solve": info.kernel_launches}


def extra_batch(B, I, torch, stream, count=64):
    """64 independent grids, sides drawn (seed 2) from {32, 48, 64, 96, 128},
    G(CI) degree 8, FP64, rtol 1e-10: one batched solve (every launch covers
    all unfinished grids, iterations replayed from one CUDA graph; the batch's
    default slab share) against a sequential loop of single solves of the same
    grids on the same GPU (contexts created beforehand, slab share 1)."""
    shapes = I.batch_shapes(count=count, seed=2)
    bs = [torch.from_numpy(I.rhs_uniform(sh, seed=1 + q)).cuda() for q, sh in enumerate(shapes)]
    xs = [torch.zeros_like(b) for b in bs]
    npts = sum(b.numel() for b in bs)
    run = lambda: B.solve_batch(bs, xs, rtol=1e-10, maxit=500, precond=B.PC_CHEB, degree=8, stream=stream)
    run()
    ms_b, infos = _timed_cuda(run, stream, torch, 2)
    xg = [x.clone() for x in xs]
    # the same batch as ONE persistent cooperative launch in a CUDA graph
    run_p = lambda: B.solve_batch(bs, xs, rtol=1e-10, maxit=500, precond=B.PC_CHEB, degree=8, stream=stream,
                                  persistent=1)
    run_p()
    ms_p, infos_p = _timed_cuda(run_p, stream, torch, 2)
    same_p = all(bool(torch.equal(a, c)) for a, c in zip(xs, xg))
    # with the slab depth and engine of each grid shape picked by the autotuner
    # (the first call tunes and is not timed)
    tuned = {}
    for name, kw in (("graph", {}), ("persistent", {"persistent": 1})):
        run_t = lambda: B.solve_batch(bs, xs, rtol=1e-10, maxit=500, precond=B.PC_CHEB, degree=8, stream=stream,
                                      autotune=1, **kw)
        run_t()
        ms_t, infos_t = _timed_cuda(run_t, stream, torch, 2)
        tuned[name] = {"ms": ms_t, "solves_per_s": count * 1e3 / ms_t, "all_ok": all(i.status == B.OK for i in infos_t),
                       "max_iterations": max(i.iterations for i in infos_t)}
    tuned["slab_planes"] = sorted({(i.slab_planes, i.engine) for i in infos_t})
    solvers = [B.Solver(sh, stream=stream) for sh in shapes]

    def seq():
        out = []
        for s_, b, x in zip(solvers, bs, xs):
            out.append(s_.solve(b, x, rtol=1e-10, maxit=500, precond=B.PC_CHEB, degree=8))
        return out
    seq()
    ms_s, infos_s = _timed_cuda(seq, stream, torch, 1)
    for s_ in solvers:
        s_.close()
    # the batch decomposes its grids with the shared slab share, the single
    # solves as grids alone: other reduction orders, iteration counts may differ
    diff = max(abs(a.iterations - c.iterations) for a, c in zip(infos, infos_s))
    return {"workload": f"batch of {count} grids, sides from {{32,48,64,96,128}} (seed 2), G(CI) d=8 FP64, rtol 1e-10",
            "points_total": npts, "batched_ms": ms_b, "batched_solves_per_s": count * 1e3 / ms_b,
            "persistent_ms": ms_p, "persistent_solves_per_s": count * 1e3 / ms_p,
            "persistent_launches": infos_p[0].kernel_launches, "persistent_bitwise_equal_to_graph": same_p,
            "autotuned": tuned,
            "sequential_ms": ms_s, "sequential_solves_per_s": count * 1e3 / ms_s, "speedup": ms_s / ms_b,
            "all_ok": all(i.status == B.OK for i in infos), "max_iteration_difference_vs_solo": diff,
            "max_iterations": max(i.iterations for i in infos)}


def extra_serve(B, I, torch, stream, n_req, factors=(0.8,), budget=120e9, max_slots=128):
    """Serving stream: n_req requests, sides log-uniform on [16, 256] (seed 3),
    Poisson arrivals, FP64 outer / FP32 Chebyshev degree 8, rtol 1e-8, HBM
    admission budget 120 GB.  The service rate mu is calibrated by submitting
    a burst at once; the stream then runs at factor * mu.  Latency is submit
    to result-ready, measured by the server."""
    import time
    import numpy as np
    shapes, gaps = I.serving_stream(count=n_req, seed=3)
    bs = [torch.from_numpy(I.rhs_uniform(sh, seed=4 + q)).cuda() for q, sh in enumerate(shapes)]
    xs = [torch.zeros_like(b) for b in bs]
    torch.cuda.synchronize()
    out = {"workload": f"{n_req} requests, sides log-uniform [16,256] (seed 3), FP32 Chebyshev d=8, rtol 1e-8, "
                       f"budget {budget / 1e9:.0f} GB", "mean_points": float(np.mean([b.numel() for b in bs]))}
    with B.Server(budget, max_slots=max_slots,
                  stream=stream) as srv:
        ncal = min(200, n_req)
        t0 = time.perf_counter()
        ts = [srv.submit(bs[q], xs[q], rtol=1e-8, maxit=2000, precond=B.PC_CHEB, degree=8, cheb_prec=B.FP32) for q in range(ncal)]
        for t in ts:
            srv.wait(t)
        mu = ncal / (time.perf_counter() - t0)
        out["calibrated_mu_solves_per_s"] = mu
        for f in factors:
            lam = f * mu
            arrivals = np.cumsum(gaps) / lam
            tickets = []
            start = time.perf_counter()
            for q in range(n_req):
                delay = start + arrivals[q] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                tickets.append(srv.submit(bs[q], xs[q], rtol=1e-8, maxit=2000, precond=B.PC_CHEB, degree=8, cheb_prec=B.FP32))
            infos = [srv.wait(t, timeout=600) for t in tickets]
            wall = time.perf_counter() - start
            lat = np.array([i.seconds for i in infos]) * 1e3
            pts = np.array([b.numel() for b in bs], dtype=np.float64)
            # latency by request size: thirds of the stream by grid points
            cuts = np.percentile(pts, [100 / 3, 200 / 3])
            thirds = {}
            for name, sel in (("small", pts <= cuts[0]), ("medium", (pts > cuts[0]) & (pts <= cuts[1])),
                              ("large", pts > cuts[1])):
                if sel.any():
                    thirds[name] = {"max_points": float(pts[sel].max()), "p50_ms": float(np.percentile(lat[sel], 50)),
                                    "p99_ms": float(np.percentile(lat[sel], 99))}
            out[f"at_{f:.1f}_mu"] = {"offered_rate": lam, "solves_per_s": n_req / wall,
                                     "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                                     "mean_ms": float(lat.mean()),
                                     "by_size": thirds,
                                     # algorithmic bytes of every served solve over the wall time
                                     "model_GBps": float(sum(i.model_bytes for i in infos) / wall / 1e9),
                                     "all_ok": all(i.status == B.OK for i in infos),
                                     "max_true_residual": max(i.rel_res_true for i in infos)}
    # the same requests solved one after another on the same GPU, same settings:
    # (a) each with its own context (create, solve, destroy: a loop of plain
    # solves); (b) with one context per grid shape created beforehand and its
    # graphs captured by a first solve, so only the solves are timed
    ncal = min(200, n_req)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for q in range(ncal):
        with B.Solver(tuple(bs[q].shape), cheb_prec=B.FP32, stream=stream) as s_:
            s_.solve(bs[q], xs[q], rtol=1e-8, maxit=2000, precond=B.PC_CHEB, degree=8)
    torch.cuda.synchronize()
    seq = ncal / (time.perf_counter() - t0)
    ctxs = {}
    for q in range(ncal):
        shp = tuple(bs[q].shape)
        if shp not in ctxs:
            ctxs[shp] = B.Solver(shp, cheb_prec=B.FP32, stream=stream)
            ctxs[shp].solve(bs[q], xs[q], rtol=1e-8, maxit=2000, precond=B.PC_CHEB, degree=8)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for q in range(ncal):
        ctxs[tuple(bs[q].shape)].solve(bs[q], xs[q], rtol=1e-8, maxit=2000, precond=B.PC_CHEB, degree=8)
    torch.cuda.synchronize()
    seq_pre = ncal / (time.perf_counter() - t0)
    for c in ctxs.values():
        c.close()
    out["sequential_solves_per_s"] = seq
    out["sequential_precreated_solves_per_s"] = seq_pre
    out["served_burst_vs_sequential_precreated"] = out["calibrated_mu_solves_per_s"] / seq_pre
    # the served throughput under Poisson arrivals: at the highest offered rate
    # the server is saturated, so its solves/s is the sustained service rate
    top = max(factors)
    sustained = out[f"at_{top:.1f}_mu"]["solves_per_s"]
    out["served_poisson_solves_per_s"] = sustained
    out["served_poisson_vs_sequential_precreated"] = sustained / seq_pre
    return out


def extra_512_mixed(B, I, torch, stream, with_bf16=True):
    """512^3, RHS = manufactured sine + 1e-3 U[-1,1) (seed 1), FP64 outer with
    the Chebyshev vectors in FP64 (reference), FP32 and (with_bf16) BF16,
    degree 8 and 16, rtol 1e-10; the error of each is stated against the GPU's
    FP64-vector solve of the same problem (no oracle solve is stored at this
    size: it would take the FP64 oracle hours)."""
    shape = (512, 512, 512)
    h = I.default_h(shape)
    b = torch.from_numpy(I.rhs_manufactured_noisy(shape, seed=1)).cuda()
    res = {"error_reference": "GPU FP64 solve (fp64_d8) of the same problem, not the oracle"}
    x_ref = None
    cases = [("fp64_d8", B.FP64, 8), ("fp32_d8", B.FP32, 8), ("fp32_d16", B.FP32, 16)]
    if with_bf16:
        cases += [("bf16_d8", B.BF16, 8), ("bf16_d16", B.BF16, 16)]
    for name, prec, deg in cases:
        x = torch.zeros_like(b)
        with B.Solver(shape, h, stream=stream, cheb_prec=prec) as s:
            maxit = 300 if prec == B.BF16 else 1000  # BF16 storage does not converge here (see DESIGN)
            ms, info = _timed_cuda(lambda: s.solve(b, x, rtol=1e-10, maxit=maxit, precond=B.PC_CHEB, degree=deg),
                                   stream, torch, 1)
        if x_ref is None:
            x_ref = x.clone()
        rel = float(torch.linalg.vector_norm(x - x_ref) / torch.linalg.vector_norm(x_ref))
        res[name] = {"status": info.status_name, "time_to_rtol_ms": ms, "iterations": info.iterations,
                     "rel_res_true": info.rel_res_true, "rel_l2_vs_gpu_fp64": rel,
                     "model_gb_per_s": info.model_bytes / (ms * 1e-3) / 1e9}
        del x
    return res


def extra_paper_problem(B, I, torch, stream, full=False):
    """The experimental set-up's own problem: Dirichlet faces x-, y+, z+ and
    zero-flux Neumann faces x+, y-, z- (Eq. 5), f = sin x + cos y + 3 sin z - 2yz + 2
    (normalised) on its box at h = 0.1 (256^3) or h = 0.4 (64^3), rtol 1e-10,
    24 Chebyshev iterations, the paper's bound rescaling for G(CI) and GNoComm(CI).
    One GPU and no subdivision of the domain across devices; the paper's iteration
    counts (Table 2: 64 MI250X GCDs, 4x4x4 subdomains; single device: 14) are
    context for the iteration counts, not for the times.  The flexible forms
    (FBiCGS-G(BiCGS), inner tolerance 1e-2; FBiCGS-BJ(BiCGS), 1e-6; at most 500
    inner iterations) run at 64^3 always and at 256^3 with ``full`` (one timed
    solve after a one-iteration warm-up: they take seconds)."""
    out = {}
    scaled = dict(lmin_scale=100.0, lmax_scale=1 - 1e-4)
    cases = [("256_g_ci24_scaled", (256,) * 3, 0.1, B.PC_CHEB, 24, (1, 1, 1), scaled, "50+-2"),
             ("256_gnocomm_ci24_scaled_4x4x4", (256,) * 3, 0.1, B.PC_GNOCOMM_CHEB, 24, (4, 4, 4), scaled, "140+-12"),
             ("256_bj_ci24_4x4x4", (256,) * 3, 0.1, B.PC_BJ_CHEB, 24, (4, 4, 4), {}, "172+-20"),
             ("256_none", (256,) * 3, 0.1, B.PC_NONE, 0, (1, 1, 1), {}, "1543+-245"),
             ("64_gnocomm_ci24_x10", (64,) * 3, 0.4, B.PC_GNOCOMM_CHEB, 24, (1, 1, 1),
              dict(lmin_scale=10.0, lmax_scale=1 - 1e-4), "14 (single device)")]
    for name, shape, hv, pc, deg, blocks, kw, paper in cases:
        h = (hv, hv, hv)
        b = torch.from_numpy(I.rhs_paper_problem(shape, h=h)).cuda()
        x = torch.zeros_like(b)
        with B.Solver(shape, h, bc=I.PAPER_BC, blocks=blocks, stream=stream, **kw) as s:
            s.solve(b, x, rtol=1e-10, maxit=5000, precond=pc, degree=deg)  # warm-up
            ms, info = _timed_cuda(lambda: s.solve(b, x, rtol=1e-10, maxit=5000, precond=pc, degree=deg), stream,
                                   torch, 1)
        out[name] = {"status": info.status_name, "iterations": info.iterations, "time_ms": ms,
                     "rel_res_true": info.rel_res_true, "paper_iterations": paper}
    flex = [("64_fbicgs_g_bicgs", (64,) * 3, 0.4, B.PC_G_BICGS, (1, 1, 1), 1e-2, "-"),
            ("64_fbicgs_bj_bicgs_2x2x2", (64,) * 3, 0.4, B.PC_BJ_BICGS, (2, 2, 2), 1e-6, "-")]
    if full:
        flex += [("256_fbicgs_g_bicgs", (256,) * 3, 0.1, B.PC_G_BICGS, (1, 1, 1), 1e-2, "13+-3 (950+-10 inner)"),
                 ("256_fbicgs_bj_bicgs_4x4x4", (256,) * 3, 0.1, B.PC_BJ_BICGS, (4, 4, 4), 1e-6,
                  "125+-12 (370+-2 inner)")]
    for name, shape, hv, pc, blocks, irt, paper in flex:
        h = (hv, hv, hv)
        b = torch.from_numpy(I.rhs_paper_problem(shape, h=h)).cuda()
        x = torch.zeros_like(b)
        with B.Solver(shape, h, bc=I.PAPER_BC, blocks=blocks, stream=stream, inner_rtol=irt, inner_maxit=500) as s:
            s.solve(b, x, rtol=1e-10, maxit=1, precond=pc, raise_on_error=False)  # inner set-up and graphs
            ms, info = _timed_cuda(lambda: s.solve(b, x, rtol=1e-10, maxit=1000, precond=pc), stream, torch, 1)
        out[name] = {"status": info.status_name, "iterations": info.iterations, "time_ms": ms,
                     "inner_iterations_per_outer": info.inner_iterations / max(1, info.iterations),
                     "rel_res_true": info.rel_res_true, "paper_iterations": paper}
    return out


def run_extras(args, B, I, torch, stream):
    """quick: 32^3, the batch, the set-up's problem (64^3 flexible forms) and
    300 served requests.  std (the default): the same with the 512^3 FP64 and
    FP32 runs and the 2000-request stream at 0.8 and 1.2 of the calibrated
    rate.  full: also the 512^3 BF16 runs and the 256^3 flexible solves."""
    full = args.extras == "full"
    out = {"config1_32cubed": extra_small_latency(B, I, torch, stream),
           "config4_batch64": extra_batch(B, I, torch, stream),
           "paper_problem": extra_paper_problem(B, I, torch, stream, full=full)}
    if args.extras in ("std", "full"):
        out["config3_512_mixed"] = extra_512_mixed(B, I, torch, stream, with_bf16=full)
        out["config5_serving"] = extra_serve(B, I, torch, stream, 2000, factors=(0.8, 1.2))
    else:
        out["config5_serving"] = extra_serve(B, I, torch, stream, 300, factors=(0.8, 1.2))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--kernel-timing", type=int, default=1,
                    help="1: plain launches with CUDA events per kernel (roofline); 0: graph replay")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32", "bf16"],
                    help="storage of the Chebyshev vectors in the timed solve (default FP64 throughout)")
    ap.add_argument("--extras", default="std", choices=["none", "quick", "std", "full"],
                    help="also measure the other configurations: 32^3 latency, batch of 64, the set-up's "
                         "problem and serving (quick: 300 requests; std: 2000 requests at 0.8 and 1.2 mu "
                         "and the 512^3 FP64/FP32 runs; full: also 512^3 BF16 and the 256^3 flexible solves)")
    ap.add_argument("--variants", type=int, default=1,
                    help="1: also time FP32/BF16 Chebyshev and other preconditioners on the same problem")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
