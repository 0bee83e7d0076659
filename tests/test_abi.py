"""CPU-side checks of the C-ABI boundary: the library loads, exports every entry
point include/psolve.h declares, the ctypes structures match the C layout, and
argument validation rejects bad input before any CUDA call."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2503_08935_b300 import binding as B
from paper_2503_08935_b300 import build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "psolve.h")


@pytest.fixture(scope="module")
def L():
    if build_lib.needs_build():
        build_lib.build()
    return B.lib()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"PSOLVE_API[^;(]*?\b(psolve_\w+)\s*\(", text)))


def test_header_declares_the_binding_exports():
    assert declared_functions() == sorted(B.EXPORTS)


def test_library_exports_every_declared_symbol(L):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(psolve_\w+)", out))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(L, name)
    # nothing else leaks out of the library
    assert exported == set(declared_functions())


def test_struct_layout_matches_c(tmp_path):
    src = tmp_path / "probe.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "psolve.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(psolve_opts), sizeof(psolve_result),"
        " offsetof(psolve_result, kernel_launches), offsetof(psolve_result, kclass_bytes),"
        " offsetof(psolve_opts, engine), offsetof(psolve_opts, autotune), offsetof(psolve_result, tuned));"
        " printf(\"%zu %zu %zu %d\\n\", offsetof(psolve_opts, record_history), offsetof(psolve_opts, inner_rtol),"
        " offsetof(psolve_opts, slab_share), PSOLVE_SHARED_SLAB_SHARE);"
        " return 0;}\n")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    so, sr, okl, okb, orr, oat, otu, orh, oir, oss, sss = map(
        int, subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split())
    assert so == ctypes.sizeof(B.Opts) and sr == ctypes.sizeof(B.Result)
    assert okl == B.Result.kernel_launches.offset and okb == B.Result.kclass_bytes.offset
    assert orr == B.Opts.engine.offset and oat == B.Opts.autotune.offset and otu == B.Result.tuned.offset
    assert orh == B.Opts.record_history.offset and oir == B.Opts.inner_rtol.offset
    assert oss == B.Opts.slab_share.offset and sss == B.SHARED_SLAB_SHARE


def test_default_opts(L):
    o = B.default_opts()
    assert (o.lmin_scale, o.lmax_scale) == (1.0, 1.0)
    assert list(o.blocks) == [1, 1, 1]
    assert o.cheb_prec == B.FP64 and o.half_step_check == 1 and o.use_x0 == 0
    assert o.use_graph == 1 and o.true_residual == 1 and o.timing == 0
    assert o.record_history == 0 and o.slab_share == 0


def _create(L, grid, h, bc=None, opts=None):
    g = (ctypes.c_int64 * 3)(*grid)
    hh = (ctypes.c_double * 3)(*h)
    b = (ctypes.c_int32 * 6)(*bc) if bc is not None else None
    ctx = ctypes.c_void_p()
    st = L.psolve_create(g, hh, b, ctypes.byref(opts) if opts is not None else None, None, ctypes.byref(ctx))
    return st, ctx


@pytest.mark.parametrize("grid,h", [((0, 4, 4), (1, 1, 1)), ((4, -1, 4), (1, 1, 1)), ((4, 4, 4), (1, 0, 1)),
                                    ((4, 4, 4), (1, float("nan"), 1)), ((2048, 2048, 1024), (1, 1, 1))])
def test_create_rejects_bad_grids(L, grid, h):
    st, ctx = _create(L, grid, h)
    assert st == B.E_ARG and not ctx.value
    assert B.last_error()


def test_create_rejects_bad_faces_and_bad_opts(L):
    st, _ = _create(L, (4, 4, 4), (1, 1, 1), bc=(0, 2, 0, 0, 0, 0))
    assert st == B.E_ARG and "Neumann" in B.last_error()
    st, _ = _create(L, (4, 4, 4), (1, 1, 1), bc=(1, 1, 1, 1, 1, 1))
    assert st == B.E_ARG and "singular" in B.last_error()
    st, _ = _create(L, (1, 4, 4), (1, 1, 1), bc=(1, 0, 0, 0, 0, 0))
    assert st == B.E_ARG and "2 unknowns" in B.last_error()
    st, _ = _create(L, (4, 4, 4), (1, 1, 1), opts=B.default_opts(blocks=(0, 1, 1)))
    assert st == B.E_ARG
    st, _ = _create(L, (4, 4, 4), (1, 1, 1), opts=B.default_opts(cheb_prec=7))
    assert st == B.E_ARG
    for share in (-1, 4097):
        st, _ = _create(L, (4, 4, 4), (1, 1, 1), opts=B.default_opts(slab_share=share))
        assert st == B.E_ARG and "slab_share" in B.last_error()


def test_batch_rejects_a_bad_slab_share_before_touching_the_device(L):
    g = (ctypes.c_int64 * 3)(4, 4, 4)
    hh = (ctypes.c_double * 3)(1, 1, 1)
    ptrs = (ctypes.c_void_p * 1)(16)  # never dereferenced: the options are checked first
    res = (B.Result * 1)()
    o = B.default_opts(slab_share=-3)
    st = L.psolve_solve_batch(1, g, hh, ptrs, ptrs, 1e-10, 10, B.PC_CHEB, 8, ctypes.byref(o), None, res)
    assert st == B.E_ARG and "slab_share" in B.last_error()


def test_null_arguments_are_rejected(L):
    r = B.Result()
    assert L.psolve_solve(None, None, None, 1e-10, 10, 0, 0, ctypes.byref(r)) == B.E_ARG
    assert L.psolve_apply_A(None, None, None, 0) == B.E_ARG
    assert L.psolve_solve_batch(0, None, None, None, None, 1e-10, 10, 1, 8, None, None, None) == B.E_ARG
    cnt = ctypes.c_int32()
    assert L.psolve_history(None, 0, None, None, ctypes.byref(cnt)) == B.E_ARG
    t = ctypes.c_uint64()
    g = (ctypes.c_int64 * 3)(4, 4, 4)
    hh = (ctypes.c_double * 3)(1, 1, 1)
    assert L.psolve_submit(None, g, hh, None, None, 1e-10, 10, 1, 8, None, ctypes.byref(t)) == B.E_ARG
    srv = ctypes.c_void_p()
    assert L.psolve_server_create(0.0, 4, None, ctypes.byref(srv)) == B.E_ARG and not srv.value
    L.psolve_destroy(None)  # no-op
