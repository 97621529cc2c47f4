"""Emulated reduced precision on the GPU against the oracle (Section 4.2):
the operator with every operation rounded to t bits, and the CG loop's
residual history for t = 52 (binary64), 23, 12 and 8."""
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


BOXES = [Box(2, 2, 1, 4, 0.05), Box(3, 2, 2, 7, 0.05)]


@pytest.mark.parametrize("box", BOXES, ids=lambda b: f"{b.nx}x{b.ny}x{b.nz}N{b.N}")
@pytest.mark.parametrize("t", [52, 23, 12, 8])
def test_apply_vprec_matches_oracle(nb, ctx, box, t):
    """Same operations in the same order per node and per global node; the
    GPU's own geometry and derivative matrix agree with the oracle's to about
    1e-15, which can move a value across a rounding boundary: the bar is
    identity for most entries and one unit in the t-th bit elsewhere."""
    import torch
    mesh = nb.Mesh.from_box(ctx, box)
    P = oracle.Problem(box)
    u = P.to_local(rhs_global(box, 3))
    ref = P.apply_vprec(u, t)
    w = torch.empty(box.n_local, dtype=torch.float64, device="cuda")
    mesh.apply_vprec(t, torch.from_numpy(u).cuda(), w)
    got = w.cpu().numpy()
    if t == 52:
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
        return
    same = np.mean(got == ref)
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max() / scale
    print(f"t={t}: {100 * same:.2f} % identical, max difference {err:.2e} of max |w|")
    assert same > 0.9
    assert err <= 2.0 ** -(t - 4)


@pytest.mark.parametrize("t", [52, 23, 12, 8])
def test_cg_vprec_history_matches_oracle(nb, ctx, t):
    """30 iterations without preconditioner (the paper's case): identical to
    binary64 CG at t = 52; at lower t the dot products are summed in another
    order, so the histories agree within what t bits allow, and the residual
    floor is the oracle's within a factor of 4."""
    import torch
    box = Box(3, 2, 2, 5, 0.05)
    mesh = nb.Mesh.from_box(ctx, box)
    P = oracle.Problem(box)
    b = P.to_local(rhs_global(box, 4))
    x_ref, h_ref = P.cg_vprec(b, 30, t)
    x = torch.zeros(box.n_local, dtype=torch.float64, device="cuda")
    h = mesh.cg_vprec(t, 30, torch.from_numpy(b).cuda(), x)
    if t == 52:
        np.testing.assert_allclose(h, h_ref, rtol=1e-9)
        np.testing.assert_allclose(x.cpu().numpy(), x_ref, rtol=0,
                                   atol=1e-9 * np.abs(x_ref).max())
        return
    # early iterations: relative differences at the level of 2^-t times the
    # loop's conditioning; later the two runs settle on floors of the same size
    np.testing.assert_allclose(h[:5], h_ref[:5], rtol=2.0 ** -(t - 12))
    ratio = h[-1] / h_ref[-1]
    print(f"t={t}: final loop residual GPU {h[-1]:.3e} oracle {h_ref[-1]:.3e}")
    assert 0.25 < ratio < 4.0


def test_cg_vprec_jacobi_t52_matches_binary64_pcg(nb, ctx):
    import torch
    box = Box(2, 2, 2, 4, 0.05)
    mesh = nb.Mesh.from_box(ctx, box)
    P = oracle.Problem(box)
    b = P.to_local(rhs_global(box, 5))
    _, it, _, h_ref = P.pcg(b, tol=0.0, maxit=20, precond="jacobi", history=True)
    x = torch.zeros(box.n_local, dtype=torch.float64, device="cuda")
    h = mesh.cg_vprec(52, 20, torch.from_numpy(b).cuda(), x, pc=nb.NB_PC_JACOBI)
    np.testing.assert_allclose(h, h_ref, rtol=1e-9)


def test_vprec_arguments(nb, ctx):
    import torch
    box = Box(1, 1, 1, 3, 0.0)
    mesh = nb.Mesh.from_box(ctx, box)
    u = torch.zeros(box.n_local, dtype=torch.float64, device="cuda")
    for bad in (0, 53):
        with pytest.raises(nb.NbError):
            mesh.apply_vprec(bad, u, u.clone())


def test_cg_mca_statistics_match_oracle(nb, ctx):
    """Random rounding and full MCA at virtual precision t = 23, 10 runs on
    each side (different random streams): the mean log10 residual after 25
    iterations agrees within 0.25 decades, and every run stays within the
    same two decades."""
    import torch
    box = Box(2, 2, 2, 4, 0.05)
    mesh = nb.Mesh.from_box(ctx, box)
    P = oracle.Problem(box)
    b = P.to_local(rhs_global(box, 7))
    bt = torch.from_numpy(b).cuda()
    for mode in ("rr", "mca"):
        gpu = [np.log10(mesh.cg_mca(mode, 23, 100 + s, 25, bt, torch.zeros_like(bt))[-1])
               for s in range(10)]
        orc = [np.log10(P.cg_mca(b, 25, 23, mode, seed=200 + s)[1][-1]) for s in range(10)]
        print(f"{mode}: GPU mean {np.mean(gpu):.3f} spread {np.ptp(gpu):.3f}, "
              f"oracle mean {np.mean(orc):.3f} spread {np.ptp(orc):.3f}")
        assert abs(np.mean(gpu) - np.mean(orc)) < 0.25
        assert max(max(gpu), max(orc)) - min(min(gpu), min(orc)) < 2.0
    # a run is reproducible for its seed
    h1 = mesh.cg_mca("mca", 23, 5, 10, bt, torch.zeros_like(bt))
    h2 = mesh.cg_mca("mca", 23, 5, 10, bt, torch.zeros_like(bt))
    assert np.array_equal(h1, h2)
