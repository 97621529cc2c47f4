"""The slab-partitioned CG on the GPU: a box cut into z-slabs, each slab a
mesh of its own (nb_setup_slab) on the same GPU, the interface planes
handed over between slabs by device copies (the in-process communicator of
paper_2405_11065_gb300.slab) -- against the oracle's PCG of the undivided
box and the library's own single-mesh solve."""
import numpy as np
import pytest

import oracle
from workloads import Box, rhs_global

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    import __graft_entry__ as g
    g.build()
    import paper_2405_11065_gb300 as nb
    return nb


@pytest.fixture(scope="module")
def ctx(nb):
    return nb.Context(0)


def _run(nb, ctx, box, nslabs, prec, tol, seed=5):
    import torch
    from paper_2405_11065_gb300 import slab as S
    bounds = S.slab_bounds(box.nz, nslabs)
    slabs = [S.GpuSlab(ctx, box.nx, box.ny, box.nz, z0, z1, box.N, box.deform, prec=prec)
             for z0, z1 in bounds]
    comm = S.InProcessComm()
    S.setup_diagonal(slabs, comm)
    bg = torch.from_numpy(rhs_global(box, seed)).cuda()
    for s in slabs:
        s.set_rhs(bg)
    it, rel, hist = S.slab_pcg(slabs, comm, tol=tol, maxit=5000)
    xg = np.zeros(box.n_global)
    for s in slabs:
        a, b = s.global_range()
        xg[a:b] = s.solution().double().cpu().numpy()
    return it, rel, hist, xg


BOXES = [Box(4, 3, 6, 5, 0.05), Box(3, 3, 4, 9, 0.05)]


@pytest.mark.parametrize("box", BOXES, ids=lambda b: f"{b.nx}x{b.ny}x{b.nz}N{b.N}")
@pytest.mark.parametrize("nslabs", [2, 3])
def test_fp64_slabs_match_the_oracle(nb, ctx, box, nslabs):
    it, rel, hist, xg = _run(nb, ctx, box, nslabs, nb.NB_FP64, 1e-10)
    P = oracle.Problem(box)
    b = P.to_local(rhs_global(box, 5))
    xo, ito, _, histo = P.pcg(b, tol=1e-10, maxit=5000, history=True)
    assert abs(it - ito) <= 1, (it, ito)
    k = min(len(hist), len(histo), 20)
    np.testing.assert_allclose(hist[:k], histo[:k], rtol=1e-8)
    xL = P.to_local(xg)
    assert P.true_relres(b, xL) < 1.01e-10
    err = np.linalg.norm(xL - xo) / np.linalg.norm(xo)
    print(f"{nslabs} slabs FP64: {it} iterations (oracle {ito}), |x - x_oracle| {err:.2e}")
    assert err <= 1e-9


def test_fp32_slabs_reach_fp32_accuracy(nb, ctx):
    """The paper's single-precision CG loop on three slabs: the recursive
    residual reaches 1e-5 and the solution is within FP32 reach of the
    oracle's (error stated)."""
    box = BOXES[1]
    it, rel, hist, xg = _run(nb, ctx, box, 3, nb.NB_FP32, 1e-5)
    P = oracle.Problem(box)
    b = P.to_local(rhs_global(box, 5))
    xo, _, _, _ = P.pcg(b, tol=1e-13, maxit=5000)
    xL = P.to_local(xg)
    err = np.linalg.norm(xL - xo) / np.linalg.norm(xo)
    true_rel = P.true_relres(b, xL)
    print(f"3 slabs FP32: {it} iterations, true residual {true_rel:.2e}, |x - x_oracle| {err:.2e}")
    assert rel < 1e-5 and true_rel < 5e-5
    assert err < 1e-3


def test_slab_setup_errors(nb, ctx):
    with pytest.raises(nb.NbError):
        nb.Mesh(ctx, 2, 2, 4, 5, 0.0, slab=(3, 3))
    with pytest.raises(nb.NbError):
        nb.Mesh(ctx, 2, 2, 4, 5, 0.0, slab=(0, 5))
    m = nb.Mesh(ctx, 2, 2, 4, 5, 0.0, slab=(0, 2))
    import torch
    face = torch.zeros(m.plane_size(), dtype=torch.float64, device="cuda")
    with pytest.raises(nb.NbError):
        m.slab_diag_face(0, face)  # no interface below the lowest slab
