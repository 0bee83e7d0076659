"""psolve_dot_noalloc: the dot product for callers that must not allocate
device memory (for instance while a framework's caching allocator or a
serving process owns the memory budget, or on host paths that cannot take the
synchronisation cudaMalloc/cudaFree may cause).  Its scratch is a fixed
device array inside the library, so it is checked here against the context
based psolve_dot, through the C ABI, on two calls in a row.  This file is
collected last so that a failure here does not hide the other GPU tests."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_08935_b300 import binding as B
from paper_2503_08935_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()


@pytest.mark.parametrize("shape", [(19, 24, 37), (64, 64, 64), (1, 1, 1), (100, 80, 130)])
def test_noalloc_dot_matches_context_dot_twice(shape):
    a_np = I.rhs_uniform(shape, seed=31)
    b_np = I.rhs_uniform(shape, seed=32)
    a = torch.from_numpy(a_np).cuda()
    b = torch.from_numpy(b_np).cuda()
    with B.Solver(shape) as s:
        ref = s.dot(a, b)
    tol = a_np.size * 2.0 ** -53 * float(np.sum(np.abs(a_np * b_np)))
    first = B.dot_noalloc(a, b)
    second = B.dot_noalloc(a, b)
    assert abs(first - ref) <= tol and abs(second - ref) <= tol
    # same units, same summation order as a context without the autotuner
    assert first == ref and second == ref
    assert abs(first - O.dot(a_np, b_np)) <= tol
    # a different pair right after: the shared scratch must not leak state
    c = torch.from_numpy(I.rhs_uniform(shape, seed=33)).cuda()
    with B.Solver(shape) as s:
        ref_c = s.dot(a, c)
    assert abs(B.dot_noalloc(a, c) - ref_c) <= a_np.size * 2.0 ** -53 * float(
        torch.sum(torch.abs(a * c)).item())


def test_noalloc_rejects_grids_beyond_its_scratch():
    """A flat 32768 x 4096 x 1 grid has 524288 xy tiles, hence at least that many
    work units whatever the chunk length, more than the 4 MiB scratch holds
    (262144).  The vectors are allocated at full size all the same, so that the
    call could not read out of bounds even if the size check were wrong."""
    import ctypes
    shape = (1, 4096, 32768)
    a = torch.zeros(shape, dtype=torch.float64, device="cuda")
    grid = (ctypes.c_int64 * 3)(32768, 4096, 1)
    res = ctypes.c_double()
    st = B.lib().psolve_dot_noalloc(grid, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(a.data_ptr()),
                                    ctypes.c_void_p(0), ctypes.byref(res))
    assert st == B.E_ARG and "scratch" in B.last_error()
    del a
    torch.cuda.empty_cache()
