"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds no arithmetic of the solver: it only produces right-hand
sides, grid spacings and workload mixes.  Both the CUDA path and the CPU oracle
are fed the identical arrays it returns.

Random values use splitmix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) as a counter-based generator:
value i of a stream with seed s is mix(s + (i + 1) * 0x9E3779B97F4A7C15), and a
uniform double in [0, 1) is (value >> 11) * 2**-53.

Arrays are numpy float64 with shape (nz, ny, nx), x fastest.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """uint64 values ``offset .. offset+count-1`` of the counter-based stream ``seed``."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, lo: float = -1.0, hi: float = 1.0, offset: int = 0) -> np.ndarray:
    """i.i.d. uniform[lo, hi) doubles from the splitmix64 stream ``seed``."""
    u = (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def default_h(shape_zyx) -> tuple:
    """Unit-cube spacing h_d = 1/(n_d + 1), returned as (hx, hy, hz)."""
    nz, ny, nx = shape_zyx
    return (1.0 / (nx + 1), 1.0 / (ny + 1), 1.0 / (nz + 1))


# Face conditions, ordered x-, x+, y-, y+, z-, z+: 0 zero Dirichlet, 1 zero-flux
# Neumann.  The experimental set-up's problem has Dirichlet faces at x-, y+, z+
# and Neumann faces at x+, y-, z-.
PAPER_BC = (0, 1, 1, 0, 1, 0)


def axis_coords(n: int, h: float, lo: float, bc_minus: int) -> np.ndarray:
    """Coordinates of the n unknowns along one axis whose domain starts at ``lo``:
    with a Dirichlet minus face the boundary node ``lo`` is known and the first
    unknown is ``lo + h``; with a Neumann minus face the boundary node is itself
    the first unknown."""
    return lo + (np.arange(n) + (0 if bc_minus == 1 else 1)) * h


def default_h_bc(shape_zyx, bc) -> tuple:
    """Unit-interval spacing per axis for face conditions ``bc``: 1/(n+1) with two
    Dirichlet faces (both boundary nodes known), 1/n with one Neumann face, 1/(n-1)
    with two (the boundary nodes are unknowns)."""
    nz, ny, nx = shape_zyx
    out = []
    for d, n in enumerate((nx, ny, nz)):
        k = bc[2 * d] + bc[2 * d + 1]
        out.append(1.0 / (n + 1 - k))
    return tuple(out)


def rhs_manufactured_bc(shape_zyx, bc) -> np.ndarray:
    """f = -Laplace(u) for u = prod_d g_d(x_d) on the unit cube, with g_d
    meeting the face conditions of axis d: sin(pi x) (Dirichlet both), sin(pi x/2)
    (Neumann at x = 1), cos(pi x/2) (Neumann at x = 0), cos(pi x) (Neumann both);
    f = (k_x^2 + k_y^2 + k_z^2) u.  Returns (f, u) at the unknowns."""
    nz, ny, nx = shape_zyx
    h = default_h_bc(shape_zyx, bc)
    gs, ks = [], []
    for d, n in enumerate((nx, ny, nz)):
        x = axis_coords(n, h[d], 0.0, bc[2 * d])
        fm, fp = bc[2 * d], bc[2 * d + 1]
        if not fm and not fp:
            k, g = math.pi, np.sin(math.pi * x)
        elif not fm:
            k, g = math.pi / 2, np.sin(math.pi * x / 2)
        elif not fp:
            k, g = math.pi / 2, np.cos(math.pi * x / 2)
        else:
            k, g = math.pi, np.cos(math.pi * x)
        gs.append(g)
        ks.append(k)
    u = gs[2][:, None, None] * gs[1][None, :, None] * gs[0][None, None, :]
    return (ks[0] ** 2 + ks[1] ** 2 + ks[2] ** 2) * u, u


def rhs_paper_problem(shape_zyx, h=(0.1, 0.1, 0.1), lo=(3.0, 2.5, 10.0), bc=PAPER_BC) -> np.ndarray:
    """The experimental set-up's right-hand side sin x + cos y + 3 sin z - 2 y z + 2
    on the box starting at ``lo`` (x in [3, 28.5], y in [2.5, 28], z in [10, 35.5] at
    h = 0.1), sampled at the unknowns of face conditions ``bc`` and normalised to
    unit 2-norm (the paper normalises the right-hand side)."""
    nz, ny, nx = shape_zyx
    x = axis_coords(nx, h[0], lo[0], bc[0])
    y = axis_coords(ny, h[1], lo[1], bc[2])
    z = axis_coords(nz, h[2], lo[2], bc[4])
    f = (np.sin(x)[None, None, :] + np.cos(y)[None, :, None] + 3.0 * np.sin(z)[:, None, None]
         - 2.0 * y[None, :, None] * z[:, None, None] + 2.0)
    return f / np.linalg.norm(f)


def rhs_uniform(shape_zyx, seed: int = 1) -> np.ndarray:
    """b ~ U[-1, 1) per point, linear index order (x fastest)."""
    n = int(np.prod(shape_zyx))
    return uniform(seed, n).reshape(shape_zyx)


def rhs_manufactured(shape_zyx, h=None) -> np.ndarray:
    """f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z) at interior points x_i = (i+1) h."""
    nz, ny, nx = shape_zyx
    hx, hy, hz = default_h(shape_zyx) if h is None else h
    sx = np.sin(math.pi * hx * np.arange(1, nx + 1))
    sy = np.sin(math.pi * hy * np.arange(1, ny + 1))
    sz = np.sin(math.pi * hz * np.arange(1, nz + 1))
    return 3.0 * math.pi ** 2 * sz[:, None, None] * sy[None, :, None] * sx[None, None, :]


def rhs_manufactured_noisy(shape_zyx, seed: int = 1, noise: float = 1e-3, h=None) -> np.ndarray:
    """Manufactured sine plus ``noise`` * U[-1, 1) (seeded)."""
    return rhs_manufactured(shape_zyx, h) + noise * rhs_uniform(shape_zyx, seed)


def batch_shapes(count: int = 64, seed: int = 2, sides=(32, 48, 64, 96, 128)) -> list:
    """``count`` grid shapes (nz, ny, nx), each side drawn independently from ``sides``."""
    v = splitmix64(seed, 3 * count)
    k = (v % np.uint64(len(sides))).astype(np.int64)
    out = []
    for g in range(count):
        nx, ny, nz = (sides[k[3 * g]], sides[k[3 * g + 1]], sides[k[3 * g + 2]])
        out.append((nz, ny, nx))
    return out


def serving_stream(count: int = 2000, seed: int = 3, lo: int = 16, hi: int = 256):
    """Per-request grid shapes with each side log-uniform on [lo, hi] (rounded),
    plus unit-rate exponential inter-arrival gaps (scale them by 1/lambda)."""
    u = uniform(seed, 3 * count, 0.0, 1.0)
    sides = np.rint(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
    sides = np.clip(sides, lo, hi)
    shapes = [(int(sides[3 * i + 2]), int(sides[3 * i + 1]), int(sides[3 * i])) for i in range(count)]
    g = uniform(seed + 1000, count, 0.0, 1.0)
    gaps = -np.log1p(-g)  # Exp(1)
    return shapes, gaps


def perturb_relative(v: np.ndarray, seed: int, eps: float) -> np.ndarray:
    """v * (1 + eps * u) with u i.i.d. uniform[-1, 1) from the splitmix64 stream
    ``seed``: a right-hand side that differs from v by rounding-sized noise."""
    u = uniform(seed, v.size).reshape(v.shape)
    return v * (1.0 + eps * u)
