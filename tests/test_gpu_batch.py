"""Batched solves of independent problems of mixed size and order: every
problem's solution against the FP64 oracle, and against solving the same
problem alone."""
import numpy as np
import pytest

import oracle
from workloads import Box, batched_problems, rhs_global

pytestmark = pytest.mark.gpu

BOXES = [Box(2, 1, 1, 5, 0.0), Box(1, 2, 2, 7, 0.05), Box(2, 2, 1, 9, 0.05),
         Box(1, 1, 3, 11, 0.05), Box(3, 1, 1, 5, 0.05), Box(1, 1, 1, 3, 0.0),
         Box(2, 2, 2, 7, 0.05)]


@pytest.fixture(scope="module")
def nb():
    import __graft_entry__ as g
    g.build()
    import paper_2405_11065_gb300 as nb
    return nb


@pytest.fixture(scope="module")
def ctx(nb):
    return nb.Context(0)


def _batch_rhs(batch, boxes, seeds):
    import torch
    ug = np.concatenate([rhs_global(bx, s) for bx, s in zip(boxes, seeds)])
    ug_t = torch.from_numpy(ug).cuda()
    b = torch.empty(batch.n_local, dtype=torch.float64, device="cuda")
    batch.to_local(ug_t, b)
    return b


def test_batch_layout_and_rhs(nb, ctx):
    batch = nb.Batch(ctx, BOXES)
    assert batch.n_local == sum(bx.n_local for bx in BOXES)
    assert batch.n_global == sum(bx.n_global for bx in BOXES)
    # problems are grouped by order in the batch L-vector
    order = np.argsort(batch.l_off)
    Ns = [BOXES[p].N for p in order]
    assert Ns == sorted(Ns)
    b = _batch_rhs(batch, BOXES, range(len(BOXES))).cpu().numpy()
    for p, bx in enumerate(BOXES):
        P = oracle.Problem(bx)
        sl = b[batch.l_off[p]:batch.l_off[p] + bx.n_local]
        np.testing.assert_array_equal(sl, P.to_local(rhs_global(bx, p)))


@pytest.mark.parametrize("use_graph", [1, 0])
def test_batch_fp64_matches_oracle_and_single_solves(nb, ctx, use_graph):
    import torch
    batch = nb.Batch(ctx, BOXES)
    b = _batch_rhs(batch, BOXES, range(len(BOXES)))
    x = torch.zeros_like(b)
    out = batch.solve(b, x, nb.default_opts(prec=nb.NB_FP64, rtol=1e-12, use_graph=use_graph))
    assert out["status"] == 0, out
    xs = x.cpu().numpy()
    bs = b.cpu().numpy()
    for p, bx in enumerate(BOXES):
        P = oracle.Problem(bx)
        sl = slice(batch.l_off[p], batch.l_off[p] + bx.n_local)
        bp = bs[sl]
        if not np.any(bp):
            assert np.all(xs[sl] == 0)
            continue
        xo, ito, _, _ = P.pcg(bp, tol=1e-12, maxit=5000)
        assert np.linalg.norm(xs[sl] - xo) <= 1e-10 * np.linalg.norm(xo), p
        assert abs(out["problems"][p]["iters"] - ito) <= 1, (p, out["problems"][p], ito)
        # the same problem solved alone takes the same iterations
        mesh = nb.Mesh.from_box(ctx, bx)
        x1 = torch.zeros(bx.n_local, dtype=torch.float64, device="cuda")
        o1 = mesh.solve(b[sl].contiguous(), x1, nb.default_opts(prec=nb.NB_FP64, rtol=1e-12))
        assert abs(o1["iters"] - out["problems"][p]["iters"]) <= 1


def test_batch_mixed_refinement(nb, ctx):
    import torch
    batch = nb.Batch(ctx, BOXES)
    b = _batch_rhs(batch, BOXES, range(len(BOXES)))
    x = torch.zeros_like(b)
    out = batch.solve(b, x, nb.default_opts(prec=nb.NB_FP32, rtol=1e-10))
    assert out["status"] == 0, out
    xs, bs = x.cpu().numpy(), b.cpu().numpy()
    for p, bx in enumerate(BOXES):
        P = oracle.Problem(bx)
        sl = slice(batch.l_off[p], batch.l_off[p] + bx.n_local)
        if not np.any(bs[sl]):
            continue
        assert P.true_relres(bs[sl], xs[sl]) < 1.01e-10, p
        xo, _, _, _ = P.pcg(bs[sl], tol=1e-13, maxit=5000)
        assert np.linalg.norm(xs[sl] - xo) <= 1e-8 * np.linalg.norm(xo), p
    # graph and host-launched iterations give the same bits
    x2 = torch.zeros_like(b)
    batch.solve(b, x2, nb.default_opts(prec=nb.NB_FP32, rtol=1e-10, use_graph=0))
    assert torch.equal(x, x2)


def test_batch_from_the_batched_workload(nb, ctx):
    """Problems drawn like the 256-problem batched workload (E in 8..512,
    N in {5,7,9,11}), checked by the oracle's FP64 residual.  A prime E gives
    a 1 x 1 x E chain of elements whose condition number needs tens of
    thousands of Jacobi-PCG iterations, hence the iteration limit."""
    import torch
    probs = batched_problems(12)
    boxes = [bx for bx, _ in probs]
    batch = nb.Batch(ctx, boxes)
    batch.autotune(reps=2)
    b = _batch_rhs(batch, boxes, [s for _, s in probs])
    x = torch.zeros_like(b)
    out = batch.solve(b, x, nb.default_opts(prec=nb.NB_FP32, rtol=1e-10, maxiter=200000))
    assert out["status"] == 0, out
    xs, bs = x.cpu().numpy(), b.cpu().numpy()
    for p, bx in enumerate(boxes):
        P = oracle.Problem(bx)
        sl = slice(batch.l_off[p], batch.l_off[p] + bx.n_local)
        assert P.true_relres(bs[sl], xs[sl]) < 1.01e-10, (p, bx)
