"""Batched and served solves: each problem's result is bitwise the result of
solving it alone (in a context with the same slab_share, by default
PSOLVE_SHARED_SLAB_SHARE for batches and served requests), whatever else shares
the launches; the server admits work as memory frees up and rejects requests
that cannot fit."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_08935_b300 import binding as B
from paper_2503_08935_b300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()


def solo(shape, b, precond, degree, prec, rtol=1e-10, **kw):
    x = torch.zeros(shape, dtype=torch.float64, device=DEV)
    with B.Solver(shape, cheb_prec=prec, **kw) as s:
        info = s.solve(b, x, rtol=rtol, maxit=500, precond=precond, degree=degree)
    torch.cuda.synchronize()
    return x.cpu().numpy(), info


@pytest.mark.parametrize("share", [0, 1])
@pytest.mark.parametrize("prec", [B.FP64, B.FP32])
def test_served_results_bitwise_equal_alone(prec, share):
    """share 0: the server's default slab share, against contexts created with
    slab_share = SHARED_SLAB_SHARE; share 1: requests decomposed as a grid
    alone, against default contexts."""
    shapes = [(24, 16, 40), (17, 9, 33), (32, 32, 32), (8, 40, 16), (20, 20, 21), (48, 24, 64)]
    bs = [torch.from_numpy(I.rhs_uniform(sh, seed=50 + q)).to(DEV) for q, sh in enumerate(shapes)]
    xs = [torch.zeros(sh, dtype=torch.float64, device=DEV) for sh in shapes]
    torch.cuda.synchronize()
    with B.Server(budget_bytes=2 << 30, max_slots=4) as srv:
        tickets = [srv.submit(b, x, rtol=1e-10, maxit=500, precond=B.PC_CHEB, degree=6, cheb_prec=prec,
                              slab_share=share)
                   for b, x in zip(bs, xs)]
        infos = [srv.wait(t) for t in tickets]
    torch.cuda.synchronize()
    for q, sh in enumerate(shapes):
        xa, ia = solo(sh, bs[q], B.PC_CHEB, 6, prec, slab_share=share or B.SHARED_SLAB_SHARE)
        assert infos[q].slab_planes == ia.slab_planes
        assert infos[q].status == B.OK and infos[q].iterations == ia.iterations
        assert np.array_equal(xs[q].cpu().numpy(), xa)
        assert infos[q].rel_res_true <= 2e-10


def test_server_admits_under_a_tight_budget_and_rejects_oversized():
    shapes = [(32, 32, 40), (32, 32, 40), (24, 24, 24), (32, 32, 40)]
    bs = [torch.from_numpy(I.rhs_uniform(sh, seed=60 + q)).to(DEV) for q, sh in enumerate(shapes)]
    xs = [torch.zeros(sh, dtype=torch.float64, device=DEV) for sh in shapes]
    torch.cuda.synchronize()
    one = 12 * 8 * 32 * 32 * 40  # roughly one 32x32x40 workspace: forces one-at-a-time admission
    with B.Server(budget_bytes=1.6 * one, max_slots=8) as srv:
        tickets = [srv.submit(b, x, rtol=1e-10, precond=B.PC_CHEB, degree=4) for b, x in zip(bs, xs)]
        big = torch.zeros((64, 64, 64), dtype=torch.float64, device=DEV)
        with pytest.raises(B.PsolveError) as e:
            srv.submit(big, big, precond=B.PC_CHEB, degree=4)
        assert e.value.status == B.REJECTED
        with pytest.raises(B.PsolveError) as e:  # served requests share the exact bounds
            srv.submit(bs[0], xs[0], precond=B.PC_CHEB, degree=4, lmin_scale=100.0, lmax_scale=1 - 1e-4)
        assert e.value.status == B.E_ARG
        with pytest.raises(B.PsolveError) as e:  # the flexible forms are not served
            srv.submit(bs[0], xs[0], precond=B.PC_G_BICGS, degree=0)
        assert e.value.status == B.E_ARG
        infos = [srv.wait(t) for t in tickets]
    for q, sh in enumerate(shapes):
        assert infos[q].status == B.OK
        xo, ro = O.bicgstab(bs[q].cpu().numpy(), I.default_h(sh), rtol=1e-10, maxit=500, precond=O.PC_CHEB,
                            degree=4)
        x = xs[q].cpu().numpy()
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-8


def test_served_requests_join_while_others_run():
    """A request submitted while a large one is on the GPU finishes first."""
    big_shape, small_shape = (192, 192, 192), (16, 16, 16)
    bb = torch.from_numpy(I.rhs_uniform(big_shape, seed=70)).to(DEV)
    xb = torch.zeros(big_shape, dtype=torch.float64, device=DEV)
    bsm = torch.from_numpy(I.rhs_uniform(small_shape, seed=71)).to(DEV)
    xsm = torch.zeros(small_shape, dtype=torch.float64, device=DEV)
    torch.cuda.synchronize()
    with B.Server(budget_bytes=4 << 30, max_slots=8) as srv:
        tb = srv.submit(bb, xb, rtol=1e-12, maxit=2000, precond=B.PC_CHEB, degree=8)
        import time
        time.sleep(0.02)
        ts = srv.submit(bsm, xsm, rtol=1e-10, precond=B.PC_CHEB, degree=8)
        ism = srv.wait(ts)
        st_big, _ = srv.poll(tb)
        ib = srv.wait(tb)
    assert ism.status == B.OK and ib.status == B.OK
    assert st_big == B.PENDING  # the small one completed while the big one was still running
    xa, ia = solo(small_shape, bsm, B.PC_CHEB, 8, B.FP64, slab_share=B.SHARED_SLAB_SHARE)
    assert np.array_equal(xsm.cpu().numpy(), xa)


# (precond, degree, Chebyshev precision, blocks) of the mixed-preconditioner stream
MIXED_REQUESTS = [
    ((24, 16, 40), B.PC_CHEB, 8, B.FP64, (1, 1, 1)),
    ((32, 32, 32), B.PC_CHEB, 8, B.FP32, (1, 1, 1)),
    ((20, 24, 16), B.PC_BJ_CHEB, 6, B.FP64, (2, 2, 2)),
    ((17, 9, 33), B.PC_NONE, 0, B.FP64, (1, 1, 1)),
    ((32, 16, 24), B.PC_GNOCOMM_CHEB, 4, B.FP64, (2, 2, 2)),
    ((40, 24, 16), B.PC_CHEB, 8, B.FP64, (1, 1, 1)),
    ((16, 32, 24), B.PC_CHEB, 4, B.FP32, (1, 1, 1)),
    ((24, 24, 24), B.PC_BJ_CHEB, 6, B.FP64, (2, 2, 2)),
]


def test_served_mixed_preconditioners_bitwise_equal_alone():
    """Requests with different preconditioners (G(CI), BJ(CI), GNoComm(CI), none;
    FP64 and FP32 Chebyshev vectors; several degrees) in one server: each
    preconditioner is a launch group of its own in every round, and every
    result is bitwise the result of solving the request alone."""
    bs, xs = [], []
    for q, (sh, *_rest) in enumerate(MIXED_REQUESTS):
        bs.append(torch.from_numpy(I.rhs_uniform(sh, seed=80 + q)).to(DEV))
        xs.append(torch.zeros(sh, dtype=torch.float64, device=DEV))
    torch.cuda.synchronize()
    with B.Server(budget_bytes=2 << 30, max_slots=5) as srv:
        tickets = [srv.submit(bs[q], xs[q], rtol=1e-10, maxit=1000, precond=pc, degree=d, cheb_prec=prec,
                              blocks=blk)
                   for q, (sh, pc, d, prec, blk) in enumerate(MIXED_REQUESTS)]
        infos = [srv.wait(t) for t in tickets]
    torch.cuda.synchronize()
    for q, (sh, pc, d, prec, blk) in enumerate(MIXED_REQUESTS):
        x = torch.zeros(sh, dtype=torch.float64, device=DEV)
        with B.Solver(sh, cheb_prec=prec, blocks=blk, slab_share=B.SHARED_SLAB_SHARE) as s:
            ia = s.solve(bs[q], x, rtol=1e-10, maxit=1000, precond=pc, degree=d)
        torch.cuda.synchronize()
        assert infos[q].status == B.OK and ia.status == B.OK
        assert infos[q].iterations == ia.iterations, (q, infos[q].iterations, ia.iterations)
        assert np.array_equal(xs[q].cpu().numpy(), x.cpu().numpy()), q
        assert infos[q].rel_res_true <= 2e-10


def test_batch_of_mixed_sizes_config_shapes():
    """A smaller version of the 64-grid batch: sides from {32, 48, 64, 96, 128}."""
    shapes = I.batch_shapes(count=6, seed=2)
    bs = [torch.from_numpy(I.rhs_uniform(sh, seed=1 + q)).to(DEV) for q, sh in enumerate(shapes)]
    xs = [torch.zeros(sh, dtype=torch.float64, device=DEV) for sh in shapes]
    infos = B.solve_batch(bs, xs, rtol=1e-10, maxit=500, precond=B.PC_CHEB, degree=8)
    for q, sh in enumerate(shapes):
        xa, ia = solo(sh, bs[q], B.PC_CHEB, 8, B.FP64, slab_share=B.SHARED_SLAB_SHARE)
        assert infos[q].status == B.OK and infos[q].iterations == ia.iterations
        assert np.array_equal(xs[q].cpu().numpy(), xa)


def test_slab_share_picks_deeper_slabs_for_shared_launches():
    """A 32^3 grid alone is cut into one-plane units (parallelism for one
    grid); with slab_share = 16 the rule takes it to share every launch with
    15 more and picks deeper slabs.  Both decompositions solve to the oracle's
    solution, and a batch with slab_share = 16 is bitwise the solo solve with
    the same setting."""
    shape = (32, 32, 32)
    b = torch.from_numpy(I.rhs_uniform(shape, seed=90)).to(DEV)
    x1, i1 = solo(shape, b, B.PC_CHEB, 8, B.FP64)
    x16, i16 = solo(shape, b, B.PC_CHEB, 8, B.FP64, slab_share=16)
    assert i16.slab_planes > i1.slab_planes
    xo, ro = O.bicgstab(b.cpu().numpy(), I.default_h(shape), rtol=1e-10, maxit=500, precond=O.PC_CHEB, degree=8)
    for x, info in ((x1, i1), (x16, i16)):
        assert info.status == B.OK and abs(info.iterations - ro.iterations) <= 2
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-8
    xb = [torch.zeros(shape, dtype=torch.float64, device=DEV)]
    ib = B.solve_batch([b], xb, rtol=1e-10, maxit=500, precond=B.PC_CHEB, degree=8, slab_share=16)
    assert ib[0].slab_planes == i16.slab_planes and np.array_equal(xb[0].cpu().numpy(), x16)
