"""Thin ctypes binding of libpsolve (include/psolve.h).

Argument marshalling only: every step of the solver runs in the CUDA library.
Device vectors are torch tensors (float64, contiguous, on the CUDA device) and
are passed as raw pointers; streams are torch streams passed as handles.  If
the compiled library is missing the import fails loudly; there is no CPU path.

The C entry points keep their names (``psolve_create``, ``psolve_solve``, ...);
``Solver`` and ``solve_batch`` wrap them for tensors.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpsolve.so")

OK, E_ARG, E_OOM, E_CUDA, NOT_CONVERGED, BREAKDOWN, NONFINITE, TIMEOUT, PENDING, REJECTED = range(10)
STATUS_NAMES = ["OK", "E_ARG", "E_OOM", "E_CUDA", "NOT_CONVERGED", "BREAKDOWN", "NONFINITE", "TIMEOUT",
                "PENDING", "REJECTED"]
PC_NONE, PC_CHEB, PC_BJ_CHEB, PC_GNOCOMM_CHEB, PC_G_BICGS, PC_BJ_BICGS = 0, 1, 2, 3, 4, 5
FP64, FP32, BF16 = 0, 1, 2
SHARED_SLAB_SHARE = 16  # PSOLVE_SHARED_SLAB_SHARE: the batch's and the server's default opts.slab_share
K_INIT, K_CI_FIRST, K_CI_SWEEP3, K_CI_SWEEP4, K_STENCIL_DOT, K_STENCIL_2DOT, K_UPDATE, K_OTHER = range(8)
K_NCLASS = 8
K_NAMES = ["init", "ci_first", "ci_sweep3", "ci_sweep4", "stencil_dot", "stencil_2dot", "update", "other"]

EXPORTS = [
    "psolve_opts_default", "psolve_create", "psolve_solve", "psolve_solve_host", "psolve_destroy",
    "psolve_apply_A", "psolve_precond_apply", "psolve_dot", "psolve_cheb_interval", "psolve_solve_batch",
    "psolve_server_create", "psolve_submit", "psolve_poll", "psolve_server_destroy", "psolve_last_error",
    "psolve_version", "psolve_dot_noalloc", "psolve_selfcheck_conversions", "psolve_selfcheck_wait_timeout",
    "psolve_selfcheck_grid_timeout", "psolve_history", "psolve_measure_fp64_rate",
]


class Opts(ctypes.Structure):
    _fields_ = [
        ("lmin_scale", ctypes.c_double),
        ("lmax_scale", ctypes.c_double),
        ("blocks", ctypes.c_int32 * 3),
        ("cheb_prec", ctypes.c_int32),
        ("half_step_check", ctypes.c_int32),
        ("use_x0", ctypes.c_int32),
        ("poll_every", ctypes.c_int32),
        ("use_graph", ctypes.c_int32),
        ("timing", ctypes.c_int32),
        ("true_residual", ctypes.c_int32),
        ("rr_every", ctypes.c_int32),
        ("engine", ctypes.c_int32),
        ("persistent", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("inner_maxit", ctypes.c_int32),
        ("record_history", ctypes.c_int32),
        ("slab_share", ctypes.c_int32),
        ("inner_rtol", ctypes.c_double),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("iterations", ctypes.c_int32),
        ("half_step_exit", ctypes.c_int32),
        ("engine", ctypes.c_int32),
        ("slab_planes", ctypes.c_int32),
        ("tuned", ctypes.c_int32),
        ("rel_res_recursive", ctypes.c_double),
        ("rel_res_true", ctypes.c_double),
        ("seconds", ctypes.c_double),
        ("model_bytes", ctypes.c_double),
        ("kernel_launches", ctypes.c_int64),
        ("inner_iterations", ctypes.c_int64),
        ("kclass_ms", ctypes.c_double * K_NCLASS),
        ("kclass_launches", ctypes.c_int64 * K_NCLASS),
        ("kclass_bytes", ctypes.c_double * K_NCLASS),
    ]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("kclass_ms", "kclass_launches",
                                                                        "kclass_bytes")}
        d["status_name"] = STATUS_NAMES[self.status] if 0 <= self.status < len(STATUS_NAMES) else "?"
        d["kclass"] = {K_NAMES[c]: {"ms": self.kclass_ms[c], "launches": self.kclass_launches[c],
                                    "bytes": self.kclass_bytes[c]} for c in range(K_NCLASS)}
        return d


_lib = None


def lib():
    """Load libpsolve.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libpsolve.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        I64P = ctypes.POINTER(ctypes.c_int64)
        DP = ctypes.POINTER(ctypes.c_double)
        I32P = ctypes.POINTER(ctypes.c_int32)
        L.psolve_opts_default.argtypes = [ctypes.POINTER(Opts)]
        L.psolve_opts_default.restype = None
        L.psolve_create.argtypes = [I64P, DP, I32P, ctypes.POINTER(Opts), ctypes.c_void_p, ctypes.POINTER(P)]
        L.psolve_solve.argtypes = [P, P, P, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.POINTER(Result)]
        L.psolve_solve_host.argtypes = L.psolve_solve.argtypes
        L.psolve_destroy.argtypes = [P]
        L.psolve_destroy.restype = None
        L.psolve_apply_A.argtypes = [P, P, P, ctypes.c_int32]
        L.psolve_precond_apply.argtypes = [P, P, P, ctypes.c_int32, ctypes.c_int32]
        L.psolve_dot.argtypes = [P, P, P, DP]
        L.psolve_cheb_interval.argtypes = [P, ctypes.c_int32, DP, DP]
        L.psolve_solve_batch.argtypes = [ctypes.c_int32, I64P, DP, ctypes.POINTER(P), ctypes.POINTER(P),
                                         ctypes.c_double, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(Opts), ctypes.c_void_p, ctypes.POINTER(Result)]
        L.psolve_server_create.argtypes = [ctypes.c_double, ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(P)]
        L.psolve_submit.argtypes = [P, I64P, DP, P, P, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_uint64)]
        L.psolve_history.argtypes = [P, ctypes.c_int32, DP, DP, I32P]
        L.psolve_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(Result)]
        L.psolve_server_destroy.argtypes = [P]
        L.psolve_server_destroy.restype = None
        L.psolve_selfcheck_conversions.argtypes = [ctypes.c_uint64, ctypes.c_int64, I64P]
        L.psolve_selfcheck_conversions.restype = ctypes.c_int32
        L.psolve_selfcheck_wait_timeout.argtypes = [ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)]
        L.psolve_selfcheck_wait_timeout.restype = ctypes.c_int32
        I32P = ctypes.POINTER(ctypes.c_int32)
        L.psolve_selfcheck_grid_timeout.argtypes = [ctypes.c_int64, ctypes.c_int32, I32P, I32P, I32P, I32P]
        L.psolve_selfcheck_grid_timeout.restype = ctypes.c_int32
        L.psolve_measure_fp64_rate.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, DP, DP, DP]
        L.psolve_measure_fp64_rate.restype = ctypes.c_int32
        L.psolve_dot_noalloc.argtypes = [I64P, P, P, ctypes.c_void_p, DP]
        L.psolve_dot_noalloc.restype = ctypes.c_int32
        L.psolve_last_error.restype = ctypes.c_char_p
        L.psolve_last_error.argtypes = []
        L.psolve_version.restype = ctypes.c_char_p
        L.psolve_version.argtypes = []
        for name in ("psolve_create", "psolve_solve", "psolve_solve_host", "psolve_apply_A",
                     "psolve_precond_apply", "psolve_dot", "psolve_cheb_interval", "psolve_solve_batch",
                     "psolve_server_create", "psolve_submit", "psolve_poll", "psolve_history"):
            getattr(L, name).restype = ctypes.c_int32
        _lib = L
    return _lib


class PsolveError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        msg = lib().psolve_last_error().decode()
        super().__init__(f"{what}: {STATUS_NAMES[status] if 0 <= status < 10 else status}: {msg}")


def last_error() -> str:
    return lib().psolve_last_error().decode()


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().psolve_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "blocks":
            for d in range(3):
                o.blocks[d] = int(v[d])
        else:
            setattr(o, k, v)
    return o


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def _ptr(t):
    return ctypes.c_void_p(int(t.data_ptr()))


def _check_vec(t, shape):
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and tuple(t.shape) == tuple(shape)):
        raise ValueError(f"expected a contiguous float64 CUDA tensor of shape {tuple(shape)}")


@dataclass
class SolveInfo:
    status: int
    iterations: int
    half_step_exit: bool
    rel_res_recursive: float
    rel_res_true: float
    seconds: float
    model_bytes: float
    kernel_launches: int
    kclass: dict
    engine: int = 0
    slab_planes: int = 0
    tuned: int = 0
    inner_iterations: int = 0

    @property
    def status_name(self):
        return STATUS_NAMES[self.status]


def _info(r: Result) -> SolveInfo:
    d = r.as_dict()
    return SolveInfo(r.status, r.iterations, bool(r.half_step_exit), r.rel_res_recursive, r.rel_res_true,
                     r.seconds, r.model_bytes, r.kernel_launches, d["kclass"], r.engine, r.slab_planes, r.tuned,
                     r.inner_iterations)


class Solver:
    """One grid (shape (nz, ny, nx)) with its device workspace (psolve_create)."""

    def __init__(self, shape_zyx, h=None, opts: Opts | None = None, stream=None, bc=None, **opt_kw):
        """``bc``: face conditions (x-, x+, y-, y+, z-, z+), 0 zero Dirichlet, 1 zero-flux
        Neumann; None = all Dirichlet."""
        nz, ny, nx = shape_zyx
        self.shape = (nz, ny, nx)
        if h is None:
            h = (1.0 / (nx + 1), 1.0 / (ny + 1), 1.0 / (nz + 1))
        self.h = tuple(float(v) for v in h)
        self.opts = opts if opts is not None else default_opts(**opt_kw)
        self._stream = _stream_handle(stream)
        grid = (ctypes.c_int64 * 3)(nx, ny, nz)
        hh = (ctypes.c_double * 3)(*self.h)
        ctx = ctypes.c_void_p()
        bcs = (ctypes.c_int32 * 6)(*[int(v) for v in bc]) if bc is not None else None
        st = lib().psolve_create(grid, hh, bcs, ctypes.byref(self.opts), self._stream, ctypes.byref(ctx))
        if st != OK:
            raise PsolveError(st, "psolve_create")
        self.ctx = ctx

    def close(self):
        if getattr(self, "ctx", None):
            lib().psolve_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, b, x, rtol=1e-10, maxit=2000, precond=PC_NONE, degree=0, raise_on_error=True) -> SolveInfo:
        _check_vec(b, self.shape)
        _check_vec(x, self.shape)
        r = Result()
        st = lib().psolve_solve(self.ctx, _ptr(b), _ptr(x), float(rtol), int(maxit), int(precond), int(degree),
                                ctypes.byref(r))
        if raise_on_error and st in (E_ARG, E_OOM, E_CUDA, TIMEOUT):
            raise PsolveError(st, "psolve_solve")
        if st in (E_ARG, E_OOM, E_CUDA, TIMEOUT):
            r.status = st
        return _info(r)

    def solve_host(self, b_host, x_host, rtol=1e-10, maxit=2000, precond=PC_NONE, degree=0) -> SolveInfo:
        """b_host / x_host: float64 C-contiguous CPU tensors or numpy arrays (pinned is faster)."""
        def hp(a):
            if hasattr(a, "data_ptr"):
                return ctypes.c_void_p(int(a.data_ptr()))
            return ctypes.c_void_p(a.ctypes.data)
        r = Result()
        st = lib().psolve_solve_host(self.ctx, hp(b_host), hp(x_host), float(rtol), int(maxit), int(precond),
                                     int(degree), ctypes.byref(r))
        if st in (E_ARG, E_OOM, E_CUDA, TIMEOUT):
            raise PsolveError(st, "psolve_solve_host")
        return _info(r)

    def history(self):
        """(rel_s, rel_r): ||s_i||/||b|| and ||r_i||/||b|| of each outer iteration of
        the last solve (psolve_history; needs record_history=1), numpy arrays with
        NaN where an iteration did not produce the value."""
        import numpy as np
        cnt = ctypes.c_int32()
        st = lib().psolve_history(self.ctx, 0, None, None, ctypes.byref(cnt))
        if st != OK:
            raise PsolveError(st, "psolve_history")
        n = cnt.value
        rs = np.full(max(n, 1), np.nan)
        rr = np.full(max(n, 1), np.nan)
        st = lib().psolve_history(self.ctx, n, rs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  rr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(cnt))
        if st != OK:
            raise PsolveError(st, "psolve_history")
        return rs[:n], rr[:n]

    def apply_A(self, u, out, block_restricted=False):
        _check_vec(u, self.shape)
        _check_vec(out, self.shape)
        st = lib().psolve_apply_A(self.ctx, _ptr(u), _ptr(out), 1 if block_restricted else 0)
        if st != OK:
            raise PsolveError(st, "psolve_apply_A")
        return out

    def precond_apply(self, v, out, precond, degree):
        _check_vec(v, self.shape)
        _check_vec(out, self.shape)
        st = lib().psolve_precond_apply(self.ctx, _ptr(v), _ptr(out), int(precond), int(degree))
        if st != OK:
            raise PsolveError(st, "psolve_precond_apply")
        return out

    def dot(self, a, b) -> float:
        _check_vec(a, self.shape)
        _check_vec(b, self.shape)
        res = ctypes.c_double()
        st = lib().psolve_dot(self.ctx, _ptr(a), _ptr(b), ctypes.byref(res))
        if st != OK:
            raise PsolveError(st, "psolve_dot")
        return res.value

    def cheb_interval(self, precond):
        a, b = ctypes.c_double(), ctypes.c_double()
        st = lib().psolve_cheb_interval(self.ctx, int(precond), ctypes.byref(a), ctypes.byref(b))
        if st != OK:
            raise PsolveError(st, "psolve_cheb_interval")
        return a.value, b.value


def solve_batch(bs, xs, hs=None, rtol=1e-10, maxit=2000, precond=PC_CHEB, degree=8, opts: Opts | None = None,
                stream=None, **opt_kw):
    """psolve_solve_batch over lists of (nz, ny, nx) float64 CUDA tensors."""
    n = len(bs)
    assert n == len(xs) and n > 0
    grids = (ctypes.c_int64 * (3 * n))()
    hh = (ctypes.c_double * (3 * n))()
    rp = (ctypes.c_void_p * n)()
    xp = (ctypes.c_void_p * n)()
    for q, (b, x) in enumerate(zip(bs, xs)):
        nz, ny, nx = b.shape
        _check_vec(b, b.shape)
        _check_vec(x, b.shape)
        grids[3 * q:3 * q + 3] = [nx, ny, nz]
        h = hs[q] if hs is not None else (1.0 / (nx + 1), 1.0 / (ny + 1), 1.0 / (nz + 1))
        hh[3 * q:3 * q + 3] = [float(v) for v in h]
        rp[q] = int(b.data_ptr())
        xp[q] = int(x.data_ptr())
    o = opts if opts is not None else default_opts(**opt_kw)
    res = (Result * n)()
    st = lib().psolve_solve_batch(n, grids, hh, rp, xp, float(rtol), int(maxit), int(precond), int(degree),
                                  ctypes.byref(o), _stream_handle(stream), res)
    if st in (E_ARG, E_OOM, E_CUDA, TIMEOUT):
        raise PsolveError(st, "psolve_solve_batch")
    return [_info(r) for r in res]


def selfcheck_conversions(seed=1, count=1 << 26) -> int:
    """Number of differences between the library's integer-pipe FP32<->FP64
    conversions and the hardware conversions on `count` bit patterns."""
    bad = ctypes.c_int64()
    st = lib().psolve_selfcheck_conversions(int(seed), int(count), ctypes.byref(bad))
    if st != OK:
        raise PsolveError(st, "psolve_selfcheck_conversions")
    return bad.value


def selfcheck_wait_timeout(limit_cycles=1 << 20) -> int:
    """Status of a bounded wait on a barrier nothing completes (TIMEOUT expected)."""
    st_out = ctypes.c_int32()
    st = lib().psolve_selfcheck_wait_timeout(int(limit_cycles), ctypes.byref(st_out))
    if st != OK:
        raise PsolveError(st, "psolve_selfcheck_wait_timeout")
    return st_out.value


def selfcheck_grid_timeout(limit_ns=20_000_000, absent_cta=0) -> dict:
    """One grid barrier of the persistent kernel with CTA `absent_cta` missing
    (-1: none); returns the CTA counts and the barrier's error word."""
    v = [ctypes.c_int32() for _ in range(4)]
    st = lib().psolve_selfcheck_grid_timeout(int(limit_ns), int(absent_cta), *[ctypes.byref(x) for x in v])
    if st != OK:
        raise PsolveError(st, "psolve_selfcheck_grid_timeout")
    return dict(zip(("ctas", "passed", "gave_up", "error_word"), (x.value for x in v)))


def measure_fp64_rate(kind=0, iters=4096, stream=None) -> dict:
    """psolve_measure_fp64_rate: FP64 instructions per second of this GPU
    (kind 0: fused multiply-add, 1: add), the timed run's ms and SM clock."""
    rate, ms, mhz = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    st = lib().psolve_measure_fp64_rate(int(kind), int(iters), _stream_handle(stream), ctypes.byref(rate),
                                        ctypes.byref(ms), ctypes.byref(mhz))
    if st != OK:
        raise PsolveError(st, "psolve_measure_fp64_rate")
    return {"instr_per_s": rate.value, "ms": ms.value, "sm_mhz": mhz.value}


def dot_noalloc(a, b, stream=None) -> float:
    """psolve_dot_noalloc on two float64 CUDA tensors of shape (nz, ny, nx):
    the library's deterministic dot product without a context or any device
    allocation (for callers that must not allocate)."""
    nz, ny, nx = a.shape
    _check_vec(a, a.shape)
    _check_vec(b, a.shape)
    grid = (ctypes.c_int64 * 3)(nx, ny, nz)
    res = ctypes.c_double()
    st = lib().psolve_dot_noalloc(grid, _ptr(a), _ptr(b), _stream_handle(stream), ctypes.byref(res))
    if st != OK:
        raise PsolveError(st, "psolve_dot_noalloc")
    return res.value


class Server:
    """Continuous-batching server (psolve_server_create / submit / poll / destroy).

    Requests of different grid sizes share every kernel launch; they are
    admitted at round boundaries while slots and the memory budget allow.
    The caller keeps b and x alive until the request's poll is final, and must
    make b ready on the server's stream before submitting.  Each request names
    its preconditioner (precond, degree, and opts.cheb_prec); requests that
    share one share every launch."""

    def __init__(self, budget_bytes, max_slots=64, stream=None):
        srv = ctypes.c_void_p()
        self._stream = _stream_handle(stream)
        st = lib().psolve_server_create(float(budget_bytes), int(max_slots), self._stream, ctypes.byref(srv))
        if st != OK:
            raise PsolveError(st, "psolve_server_create")
        self.srv = srv

    def submit(self, b, x, h=None, rtol=1e-10, maxit=2000, precond=PC_CHEB, degree=8, opts: Opts | None = None,
               **opt_kw) -> int:
        nz, ny, nx = b.shape
        _check_vec(b, b.shape)
        _check_vec(x, b.shape)
        if h is None:
            h = (1.0 / (nx + 1), 1.0 / (ny + 1), 1.0 / (nz + 1))
        grid = (ctypes.c_int64 * 3)(nx, ny, nz)
        hh = (ctypes.c_double * 3)(*[float(v) for v in h])
        o = opts if opts is not None else default_opts(**opt_kw)
        t = ctypes.c_uint64()
        st = lib().psolve_submit(self.srv, grid, hh, _ptr(b), _ptr(x), float(rtol), int(maxit), int(precond),
                                 int(degree), ctypes.byref(o), ctypes.byref(t))
        if st != OK:
            raise PsolveError(st, "psolve_submit")
        return t.value

    def poll(self, ticket):
        """(status, SolveInfo or None): status PENDING while the request runs."""
        r = Result()
        st = lib().psolve_poll(self.srv, ctypes.c_uint64(ticket), ctypes.byref(r))
        if st == PENDING:
            return st, None
        if st == E_ARG:
            raise PsolveError(st, "psolve_poll")
        return st, _info(r)

    def wait(self, ticket, timeout=120.0, interval=1e-4):
        import time
        t0 = time.monotonic()
        while True:
            st, info = self.poll(ticket)
            if st != PENDING:
                return info
            if time.monotonic() - t0 > timeout:
                raise TimeoutError(f"request {ticket} still pending after {timeout} s")
            time.sleep(interval)

    def close(self):
        if getattr(self, "srv", None):
            lib().psolve_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
