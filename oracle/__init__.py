"""FP64 CPU oracle for the preconditioned Bi-CGSTAB Poisson solver (arxiv 2503.08935).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` import this package.
The CUDA product path never imports, links or calls it.

Thin ctypes wrapper around ``psolve_oracle.c`` (plain serial C, FP64).  The
same source is also built with OpenMP (``use_build("omp")``, ``threads``) for
the timed CPU baseline and long stored reference runs; the serial build is the
default and the one the parity tests use.  Arrays
are numpy float64 of shape (nz, ny, nx), C-contiguous (x fastest), matching
the oracle's ``i + nx*(j + ny*k)`` layout.

What each function follows:
    apply_A          Eq. 3 / Eq. 6 (7-point operator, zero Dirichlet ghosts);
                     with ``blocks`` the block-diagonal restriction of Eq. 12-14.
    eig_bounds       Eq. 9-11 (closed-form Dirichlet spectrum, extreme sums).
    cheb             Eq. 15 and Algorithm 2 (Chebyshev iteration, degree d).
    precond_apply    the G(CI) / BJ(CI) / GNoComm(CI) preconditioners.
    bicgstab         Algorithm 1 with the half-step exit.
    dot              Ogita-Rump-Oishi Dot2 compensated dot product.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from .build_oracle import build as _build, build_omp as _build_omp, LIB_PATH, LIB_OMP_PATH

PC_NONE, PC_CHEB, PC_BJ_CHEB, PC_GNOCOMM_CHEB, PC_G_BICGS, PC_BJ_BICGS = 0, 1, 2, 3, 4, 5
OK, E_ARG, E_OOM, NOT_CONVERGED, BREAKDOWN, NONFINITE = 0, 1, 2, 4, 5, 6

_libs = {}
_active = "serial"


class _PC(ctypes.Structure):
    _fields_ = [
        ("type", ctypes.c_int32),
        ("degree", ctypes.c_int32),
        ("blocks", ctypes.c_int32 * 3),
        ("lmin_scale", ctypes.c_double),
        ("lmax_scale", ctypes.c_double),
        ("bc", ctypes.c_int32 * 6),
        ("inner_rtol", ctypes.c_double),
        ("inner_maxit", ctypes.c_int32),
        ("pad_", ctypes.c_int32),
    ]


class _Res(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("iterations", ctypes.c_int32),
        ("half_step_exit", ctypes.c_int32),
        ("pad_", ctypes.c_int32),
        ("rel_res_recursive", ctypes.c_double),
        ("rel_res_true", ctypes.c_double),
    ]


def use_build(kind: str) -> str:
    """Select the oracle build the functions below call: "serial" (default,
    the parity oracle) or "omp" (the OpenMP build).  Returns the previous one."""
    global _active
    if kind not in ("serial", "omp"):
        raise ValueError(kind)
    prev, _active = _active, kind
    return prev


def threads(n: int = 0) -> int:
    """Threads the OpenMP build uses (n > 0 sets them); 1 for the serial build."""
    return int(lib().oracle_threads(int(n)))


def lib():
    L = _libs.get(_active)
    if L is None:
        if _active == "omp":
            path = LIB_OMP_PATH
            if not os.path.exists(path):
                _build_omp()
        else:
            path = os.environ.get("PSOLVE_ORACLE_LIB")  # a mutant build, used by the mutation test
            if not path:
                path = LIB_PATH
                if not os.path.exists(path):
                    _build()
        L = ctypes.CDLL(path)
        D = ctypes.POINTER(ctypes.c_double)
        I64 = ctypes.POINTER(ctypes.c_int64)
        I32 = ctypes.POINTER(ctypes.c_int32)
        L.oracle_threads.restype = ctypes.c_int
        L.oracle_threads.argtypes = [ctypes.c_int32]
        L.oracle_dot.restype = ctypes.c_double
        L.oracle_dot.argtypes = [ctypes.c_int64, D, D]
        L.oracle_apply_A.argtypes = [I64, D, I32, D, D]
        L.oracle_eig_bounds.argtypes = [I64, D, D, D]
        L.oracle_cheb.argtypes = [I64, D, I32, ctypes.c_double, ctypes.c_double, ctypes.c_int32, D, D]
        L.oracle_cheb_interval.argtypes = [I64, D, ctypes.c_int32, I32, ctypes.c_double,
                                           ctypes.c_double, D, D]
        L.oracle_precond_apply.argtypes = [I64, D, ctypes.POINTER(_PC), D, D]
        L.oracle_apply_A_bc.argtypes = [I64, D, I32, I32, D, D]
        L.oracle_eig_bounds_bc.argtypes = [I64, D, I32, D, D]
        L.oracle_cheb_bc.argtypes = [I64, D, I32, I32, ctypes.c_double, ctypes.c_double, ctypes.c_int32, D, D]
        L.oracle_cheb_interval_bc.argtypes = [I64, D, I32, ctypes.c_int32, I32, ctypes.c_double,
                                              ctypes.c_double, D, D]
        L.oracle_bicgstab.argtypes = [I64, D, D, D, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                      ctypes.POINTER(_PC), ctypes.c_int32, ctypes.POINTER(_Res), D, D]
        L.oracle_bicgstab_rr.argtypes = [I64, D, D, D, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                         ctypes.POINTER(_PC), ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(_Res), D, D]
        L.oracle_bicgstab_snap.argtypes = [I64, D, D, D, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                           ctypes.POINTER(_PC), ctypes.c_int32, ctypes.c_int32,
                                           ctypes.POINTER(_Res), D, D, ctypes.c_int32, I32, D]
        _libs[_active] = L
    return L


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _n(shape):
    nz, ny, nx = shape
    return (ctypes.c_int64 * 3)(nx, ny, nz)


def _h(h):
    return (ctypes.c_double * 3)(*[float(v) for v in h])


def _blk(blocks):
    if blocks is None:
        return None
    return (ctypes.c_int32 * 3)(*[int(v) for v in blocks])


def _bc(bc):
    """Face conditions x-, x+, y-, y+, z-, z+ (0 Dirichlet, 1 Neumann) or None."""
    if bc is None:
        return None
    assert len(bc) == 6
    return (ctypes.c_int32 * 6)(*[int(v) for v in bc])


def _vec(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.ndim == 3
    return a


def _check(st, what):
    if st != OK:
        raise ValueError(f"oracle {what} failed with status {st}")


def dot(a, b) -> float:
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    b = np.ascontiguousarray(b, dtype=np.float64).ravel()
    assert a.size == b.size
    return lib().oracle_dot(a.size, _dp(a), _dp(b))


def apply_A(u, h, blocks=None, bc=None):
    """out = A u (Eq. 6).  ``h`` = (hx, hy, hz); ``blocks`` = blocks per axis (x, y, z);
    ``bc`` = face conditions (x-, x+, y-, y+, z-, z+), 0 Dirichlet / 1 Neumann (Eq. 4 / Eq. 5)."""
    u = _vec(u)
    out = np.empty_like(u)
    if bc is None:
        st = lib().oracle_apply_A(_n(u.shape), _h(h), _blk(blocks), _dp(u), _dp(out))
    else:
        st = lib().oracle_apply_A_bc(_n(u.shape), _h(h), _bc(bc), _blk(blocks), _dp(u), _dp(out))
    _check(st, "apply_A")
    return out


def eig_bounds(n_xyz, h, bc=None):
    """(lambda_min, lambda_max) of the grid operator, Eq. 10 / Eq. 11."""
    lo, hi = ctypes.c_double(), ctypes.c_double()
    n = (ctypes.c_int64 * 3)(*[int(v) for v in n_xyz])
    if bc is None:
        st = lib().oracle_eig_bounds(n, _h(h), ctypes.byref(lo), ctypes.byref(hi))
    else:
        st = lib().oracle_eig_bounds_bc(n, _h(h), _bc(bc), ctypes.byref(lo), ctypes.byref(hi))
    _check(st, "eig_bounds")
    return lo.value, hi.value


def cheb_interval(shape, h, precond, blocks=(1, 1, 1), lmin_scale=1.0, lmax_scale=1.0, bc=None):
    a, b = ctypes.c_double(), ctypes.c_double()
    if bc is None:
        st = lib().oracle_cheb_interval(_n(shape), _h(h), int(precond), _blk(blocks), float(lmin_scale),
                                        float(lmax_scale), ctypes.byref(a), ctypes.byref(b))
    else:
        st = lib().oracle_cheb_interval_bc(_n(shape), _h(h), _bc(bc), int(precond), _blk(blocks),
                                           float(lmin_scale), float(lmax_scale), ctypes.byref(a), ctypes.byref(b))
    _check(st, "cheb_interval")
    return a.value, b.value


def cheb(rhs, h, a, b, degree, blocks=None, bc=None):
    """Algorithm 2 on [a, b] for ``degree`` iterations (x = z if 0, x = y if 1)."""
    rhs = _vec(rhs)
    x = np.empty_like(rhs)
    if bc is None:
        st = lib().oracle_cheb(_n(rhs.shape), _h(h), _blk(blocks), float(a), float(b), int(degree),
                               _dp(rhs), _dp(x))
    else:
        st = lib().oracle_cheb_bc(_n(rhs.shape), _h(h), _bc(bc), _blk(blocks), float(a), float(b), int(degree),
                                  _dp(rhs), _dp(x))
    _check(st, "cheb")
    return x


def _pc(precond, degree, blocks, lmin_scale, lmax_scale, bc=None, inner_rtol=1e-2, inner_maxit=500):
    pc = _PC()
    pc.inner_rtol = float(inner_rtol)
    pc.inner_maxit = int(inner_maxit)
    pc.type = int(precond)
    pc.degree = int(degree)
    for d in range(3):
        pc.blocks[d] = int(blocks[d])
    pc.lmin_scale = float(lmin_scale)
    pc.lmax_scale = float(lmax_scale)
    for f in range(6):
        pc.bc[f] = int(bc[f]) if bc is not None else 0
    return pc


def precond_apply(v, h, precond, degree, blocks=(1, 1, 1), lmin_scale=1.0, lmax_scale=1.0, bc=None,
                  inner_rtol=1e-2, inner_maxit=500):
    v = _vec(v)
    out = np.empty_like(v)
    pc = _pc(precond, degree, blocks, lmin_scale, lmax_scale, bc, inner_rtol, inner_maxit)
    _check(lib().oracle_precond_apply(_n(v.shape), _h(h), ctypes.byref(pc), _dp(v), _dp(out)),
           "precond_apply")
    return out


@dataclass
class Result:
    status: int
    iterations: int
    half_step_exit: bool
    rel_res_recursive: float
    rel_res_true: float
    hist_s: np.ndarray
    hist_r: np.ndarray
    snapshots: dict = None


def bicgstab(b, h, rtol=1e-10, maxit=2000, precond=PC_NONE, degree=0, blocks=(1, 1, 1),
             lmin_scale=1.0, lmax_scale=1.0, x0=None, half_step_check=True, rr_every=0, bc=None,
             inner_rtol=1e-2, inner_maxit=500, snapshots=()):
    """Algorithm 1.  Returns (x, Result).  ``x0`` None means x0 = 0.
    ``rr_every`` > 0 adds residual replacement (not part of the paper's method).
    ``bc`` = face conditions of the operator (None: all zero Dirichlet).
    ``snapshots``: outer iterations after which x is copied out; the copies
    are returned in ``Result.snapshots`` ({iteration: x}, NaN if not reached)."""
    b = _vec(b)
    x = np.zeros_like(b) if x0 is None else _vec(x0).copy()
    hs = np.full(max(maxit, 1), np.nan)
    hr = np.full(max(maxit, 1), np.nan)
    pc = _pc(precond, degree, blocks, lmin_scale, lmax_scale, bc, inner_rtol, inner_maxit)
    r = _Res()
    snaps = {}
    if snapshots:
        at = (ctypes.c_int32 * len(snapshots))(*[int(k) for k in snapshots])
        buf = np.full((len(snapshots),) + b.shape, np.nan)
        lib().oracle_bicgstab_snap(_n(b.shape), _h(h), _dp(b), _dp(x), 1 if x0 is not None else 0, float(rtol),
                                   int(maxit), ctypes.byref(pc), 1 if half_step_check else 0, int(rr_every),
                                   ctypes.byref(r), _dp(hs), _dp(hr), len(snapshots), at, _dp(buf))
        snaps = {int(k): buf[j] for j, k in enumerate(snapshots)}
    elif rr_every:
        lib().oracle_bicgstab_rr(_n(b.shape), _h(h), _dp(b), _dp(x), 1 if x0 is not None else 0, float(rtol),
                                 int(maxit), ctypes.byref(pc), 1 if half_step_check else 0, int(rr_every),
                                 ctypes.byref(r), _dp(hs), _dp(hr))
    else:
        lib().oracle_bicgstab(_n(b.shape), _h(h), _dp(b), _dp(x), 1 if x0 is not None else 0, float(rtol),
                              int(maxit), ctypes.byref(pc), 1 if half_step_check else 0, ctypes.byref(r),
                              _dp(hs), _dp(hr))
    if r.status in (E_ARG, E_OOM):
        raise ValueError(f"oracle bicgstab failed with status {r.status}")
    it = r.iterations
    return x, Result(r.status, it, bool(r.half_step_exit), r.rel_res_recursive, r.rel_res_true,
                     hs[:it], hr[:it], snaps)
