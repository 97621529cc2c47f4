"""GPU parity: the CUDA path through the C ABI against the FP64 oracle,
element by element, on seeded inputs that span several blocks and ragged
tails, plus edge cases and determinism."""
import math

import numpy as np
import pytest

import oracle
from workloads import SMALL_FP64, Box, rhs_global

pytestmark = pytest.mark.gpu

BOXES = [
    Box(1, 1, 1, 1, 0.0),      # smallest: one element, N = 1
    Box(2, 2, 2, 7, 0.0),      # the plain FP64 workload
    Box(3, 2, 1, 4, 0.05),     # odd number of points per direction
    Box(5, 3, 2, 5, 0.05),     # E = 30: ragged tail of element groups
    Box(2, 3, 2, 9, 0.05),
    Box(1, 1, 3, 15, 0.05),    # highest supported order (16 points)
    Box(4, 4, 4, 11, 0.05),
]
IDS = [f"{b.nx}x{b.ny}x{b.nz}N{b.N}d{b.deform}" for b in BOXES]

# FP64 operator tolerance: both sides evaluate the same sums in FP64; the
# GPU fuses multiply-adds and orders the inner products differently, so the
# difference is a few ulps times the O(n) terms of each contraction.
TOL_AX64 = 1e-12
# FP32 operator: three chained contractions of n terms plus the 3x3 factor
# product; each output accumulates ~(6n + 9) roundings of unit 2^-24 relative
# to the largest term, bounded here by 64 n 2^-24 relative to max |w|.
def tol_ax32(n):
    return 64 * n * 2.0 ** -24


@pytest.fixture(scope="module")
def nb():
    import __graft_entry__ as g
    g.build()
    import paper_2405_11065_gb300 as nb
    return nb


@pytest.fixture(scope="module")
def ctx(nb):
    return nb.Context(0)


@pytest.fixture(scope="module", params=BOXES, ids=IDS)
def case(request, nb, ctx):
    box = request.param
    return box, nb.Mesh.from_box(ctx, box), oracle.Problem(box)


def _t(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def test_index_maps_bit_exact(case):
    box, mesh, P = case
    m = mesh.maps()
    np.testing.assert_array_equal(m["gid"].astype(np.int64), P.gid)
    np.testing.assert_array_equal(m["mult"], P.mult)
    np.testing.assert_array_equal(m["mask"], P.mask)
    off, loc = oracle.csr(P.gid, box.n_global)
    active = np.nonzero((P.mult > 1) | (P.mask == 0))[0]
    np.testing.assert_array_equal(m["gs_gid"].astype(np.int64), active)
    rows = [loc[off[g]:off[g + 1]] for g in active]
    ref_off = np.concatenate([[0], np.cumsum([len(r) for r in rows])])
    np.testing.assert_array_equal(m["gs_off"].astype(np.int64), ref_off)
    np.testing.assert_array_equal(m["gs_loc"].astype(np.int64), np.concatenate(rows))
    np.testing.assert_array_equal(m["gs_mask"], P.mask[active])


def test_geometry_and_jacobi(case):
    box, mesh, P = case
    G, dinv, c = mesh.geom()
    scale = np.abs(P.G).max()
    assert np.max(np.abs(G - P.G)) <= 1e-13 * scale
    np.testing.assert_array_equal(c, P.c)
    np.testing.assert_allclose(dinv, P.dinv, rtol=1e-12, atol=0)


def test_ax_fp64_local_and_assembled(case, nb):
    box, mesh, P = case
    import torch
    rng = np.random.default_rng(5)
    u = rng.uniform(-1, 1, box.n_local)
    w = torch.empty(box.n_local, dtype=torch.float64, device="cuda")
    mesh.ax(nb.NB_FP64, _t(u), w, assemble=False)
    ref = P.ax_local(u)
    err = np.max(np.abs(w.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert err <= TOL_AX64, err
    uc = P.to_local(rhs_global(box, 1))
    mesh.ax(nb.NB_FP64, _t(uc), w, assemble=True)
    ref = P.apply(uc)
    if not np.any(ref):  # every node is a Dirichlet node
        assert not torch.any(w)
        return
    err = np.max(np.abs(w.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert err <= TOL_AX64, err


def test_ax_fp32_error_stated(case, nb):
    box, mesh, P = case
    import torch
    rng = np.random.default_rng(6)
    u = rng.uniform(-1, 1, box.n_local).astype(np.float32)
    w = torch.empty(box.n_local, dtype=torch.float32, device="cuda")
    mesh.ax(nb.NB_FP32, _t(u), w)
    ref = P.ax_local(u.astype(np.float64))
    err = np.max(np.abs(w.cpu().numpy() - ref)) / np.max(np.abs(ref))
    print(f"FP32 ax max relative error vs FP64 oracle: {err:.3e} (n={box.n})")
    assert err <= tol_ax32(box.n), err


# Tensor-core operator: u and (wr, ws, wt) are rounded to 11 (FP16) or 8
# (BF16) significant bits; each output sums O(n) such terms with FP32
# accumulation, so the error relative to max |w| is bounded here by 16 units
# of the 16-bit format's rounding.
TOL_TC = {"tc_f16": 16 * 2.0 ** -11, "tc_bf16": 16 * 2.0 ** -8}


@pytest.mark.parametrize("prec", ["tc_f16", "tc_bf16"])
def test_ax_tensor_core_error_stated(case, nb, prec):
    box, mesh, P = case
    import torch
    rng = np.random.default_rng(16)
    u = rng.uniform(-1, 1, box.n_local).astype(np.float32) * 3e-3  # off-unit scale
    w = torch.empty(box.n_local, dtype=torch.float32, device="cuda")
    mesh.ax(nb.PREC_NAMES[prec], _t(u), w)
    ref = P.ax_local(u.astype(np.float64))
    err = np.max(np.abs(w.cpu().numpy() - ref)) / np.max(np.abs(ref))
    print(f"{prec} ax max relative error vs FP64 oracle: {err:.3e} (n={box.n})")
    assert err <= TOL_TC[prec], err


def test_dssum_bit_exact_fp64(case, nb):
    box, mesh, P = case
    rng = np.random.default_rng(7)
    v = rng.uniform(-1, 1, box.n_local)
    t = _t(v)
    mesh.dssum(nb.NB_FP64, t, masked=True)
    np.testing.assert_array_equal(t.cpu().numpy(), P.dssum(v, masked=True))
    t = _t(v)
    mesh.dssum(nb.NB_FP64, t, masked=False)
    np.testing.assert_array_equal(t.cpu().numpy(), P.dssum(v, masked=False))


def test_glsc3_and_maps(case, nb):
    box, mesh, P = case
    import torch
    rng = np.random.default_rng(8)
    a, b = rng.uniform(-1, 1, box.n_local), rng.uniform(-1, 1, box.n_local)
    got = mesh.glsc3(nb.NB_FP64, _t(a), _t(b))
    ref = oracle.glsc3(a, b, P.c)
    assert abs(got - ref) <= 1e-13 * np.sum(np.abs(a * b * P.c))
    ug = rhs_global(box, 2)
    uL = torch.empty(box.n_local, dtype=torch.float64, device="cuda")
    mesh.to_local(nb.NB_FP64, _t(ug), uL, masked=True)
    np.testing.assert_array_equal(uL.cpu().numpy(), P.to_local(ug))
    back = torch.empty(box.n_global, dtype=torch.float64, device="cuda")
    mesh.to_global(nb.NB_FP64, uL, back)
    np.testing.assert_array_equal(back.cpu().numpy(), ug * P.mask)


def test_fp64_pcg_matches_oracle(case, nb):
    box, mesh, P = case
    import torch
    b = P.to_local(rhs_global(box, 0))
    if not np.any(b):
        pytest.skip("no interior unknowns")
    xo, ito, relo, histo = P.pcg(b, tol=1e-12, maxit=5000, history=True)
    x = torch.zeros(box.n_local, dtype=torch.float64, device="cuda")
    out = mesh.solve(_t(b), x, nb.default_opts(prec=nb.NB_FP64, rtol=1e-12, maxiter=5000),
                     history_cap=5000)
    assert out["status"] == 0, out
    assert abs(out["iters"] - ito) <= 1, (out["iters"], ito)
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) <= 1e-10 * np.linalg.norm(xo)
    h = out["history"]
    k = min(len(h), len(histo), 20)
    np.testing.assert_allclose(h[:k], histo[:k], rtol=1e-8)
    assert P.true_relres(b, xg) < 1e-11


def test_small_fp64_workload_as_specified(nb, ctx):
    """The plain FP64 Jacobi-PCG workload: the 2x2x2 affine box, N = 7,
    right-hand side U[-1,1) per unique node from seed 0, 100 iterations, then
    continued to a relative residual of 1e-10.  The residual history of the
    100 iterations follows the oracle's, and the solve to 1e-10 takes the
    oracle's iteration count and reaches its solution."""
    import torch
    box = SMALL_FP64
    mesh = nb.Mesh.from_box(ctx, box)
    P = oracle.Problem(box)
    b = P.to_local(rhs_global(box, 0))
    _, it100, rel100, h100 = P.pcg(b, tol=1e-30, maxit=100, history=True)
    x = torch.zeros(box.n_local, dtype=torch.float64, device="cuda")
    out = mesh.solve(_t(b), x, nb.default_opts(prec=nb.NB_FP64, rtol=1e-30, maxiter=100),
                     history_cap=100)
    assert out["iters"] == 100 == it100
    h = np.asarray(out["history"])
    np.testing.assert_allclose(h[:60], h100[:60], rtol=1e-6)
    assert 0.5 < h[99] / h100[99] < 2.0, (h[99], h100[99])
    xo, ito, _, _ = P.pcg(b, tol=1e-10, maxit=1000)
    x.zero_()
    full = mesh.solve(_t(b), x, nb.default_opts(prec=nb.NB_FP64, rtol=1e-10))
    assert full["status"] == 0 and abs(full["iters"] - ito) <= 1, (full["iters"], ito)
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) <= 1e-10 * np.linalg.norm(xo)
    print(f"2x2x2 N=7 FP64 PCG: after 100 iterations {h[99]:.3e} (oracle {h100[99]:.3e}); "
          f"to 1e-10 in {full['iters']} iterations (oracle {ito})")


@pytest.mark.parametrize("prec", ["fp32"])
def test_mixed_refinement_reaches_fp64_accuracy(case, nb, prec):
    box, mesh, P = case
    import torch
    b = P.to_local(rhs_global(box, 0))
    if not np.any(b):
        pytest.skip("no interior unknowns")
    xo, _, _, _ = P.pcg(b, tol=1e-13, maxit=5000)
    x = torch.zeros(box.n_local, dtype=torch.float64, device="cuda")
    out = mesh.solve(_t(b), x, nb.default_opts(prec=nb.PREC_NAMES[prec], rtol=1e-10))
    assert out["status"] == 0, out
    assert out["rel_res"] < 1e-10
    xg = x.cpu().numpy()
    rel_oracle = P.true_relres(b, xg)
    assert rel_oracle < 1.01e-10, rel_oracle
    err = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    print(f"{prec}+refinement: {out['iters']} inner its, {out['outer_iters']} outer, "
          f"oracle residual {rel_oracle:.2e}, |x-x_oracle|/|x_oracle| {err:.2e}")
    assert err <= 1e-8


def test_identity_preconditioner_iterations(nb, ctx):
    box = Box(2, 2, 2, 7, 0.0)
    mesh = nb.Mesh.from_box(ctx, box)
    P = oracle.Problem(box)
    b = P.to_local(rhs_global(box, 0))
    _, ito, _, _ = P.pcg(b, tol=1e-10, maxit=1000, precond="none")
    import torch
    x = torch.zeros(box.n_local, dtype=torch.float64, device="cuda")
    out = mesh.solve(_t(b), x, nb.default_opts(prec=nb.NB_FP64, pc=nb.NB_PC_NONE, rtol=1e-10))
    assert abs(out["iters"] - ito) <= 1


def test_determinism_and_graph_equivalence(nb, ctx):
    import torch
    box = Box(3, 3, 2, 7, 0.05)
    mesh = nb.Mesh.from_box(ctx, box)
    P = oracle.Problem(box)
    b = _t(P.to_local(rhs_global(box, 4)))
    xs = []
    for use_graph in (1, 1, 0):
        for prec in (nb.NB_FP64, nb.NB_FP32):
            x = torch.zeros(box.n_local, dtype=torch.float64, device="cuda")
            mesh.solve(b, x, nb.default_opts(prec=prec, use_graph=use_graph))
            xs.append(x.cpu().numpy())
    # same precision, graph or not, repeated: bit-identical
    for k in (2, 4):
        np.testing.assert_array_equal(xs[0], xs[k])
        np.testing.assert_array_equal(xs[1], xs[k + 1])
    w1 = torch.empty_like(b)
    w2 = torch.empty_like(b)
    mesh.ax(nb.NB_FP64, b, w1, assemble=True)
    mesh.ax(nb.NB_FP64, b, w2, assemble=True)
    assert torch.equal(w1, w2)


def test_initial_guess_resume(nb, ctx):
    """A solve split in two (restart from the first half's iterate) reaches
    the same accuracy as one solve."""
    import torch
    box = Box(2, 2, 2, 7, 0.05)
    mesh = nb.Mesh.from_box(ctx, box)
    P = oracle.Problem(box)
    b = _t(P.to_local(rhs_global(box, 9)))
    x = torch.zeros_like(b)
    out1 = mesh.solve(b, x, nb.default_opts(prec=nb.NB_FP64, maxiter=20))
    assert out1["status"] == nb.NB_NOT_CONVERGED and out1["iters"] == 20
    out2 = mesh.solve(b, x, nb.default_opts(prec=nb.NB_FP64, use_x0=1))
    assert out2["status"] == 0 and out2["rel_res"] < 1e-10
    assert P.true_relres(b.cpu().numpy(), x.cpu().numpy()) < 1e-10


def test_host_entry_point(nb, ctx):
    box = Box(2, 2, 3, 5, 0.05)
    mesh = nb.Mesh.from_box(ctx, box)
    P = oracle.Problem(box)
    bg = rhs_global(box, 3)
    xg = np.zeros(box.n_global)
    out = mesh.solve_host(bg, xg, nb.default_opts(prec=nb.NB_FP32))
    assert out["status"] == 0
    b = P.to_local(bg)
    assert P.true_relres(b, P.to_local(xg)) < 1.01e-10


def test_failures_are_reported(nb, ctx):
    import torch
    box = Box(2, 2, 2, 5, 0.05)
    mesh = nb.Mesh.from_box(ctx, box)
    P = oracle.Problem(box)
    b = P.to_local(rhs_global(box, 0))
    bad = b.copy()
    bad[np.nonzero(bad)[0][3]] = np.nan
    x = torch.zeros(box.n_local, dtype=torch.float64, device="cuda")
    for prec in (nb.NB_FP64, nb.NB_FP32):
        with pytest.raises(nb.NbError) as ei:
            mesh.solve(_t(bad), x, nb.default_opts(prec=prec))
        assert ei.value.status == nb.NB_ERR_ARG
    out = mesh.solve(_t(b), x, nb.default_opts(prec=nb.NB_FP64, maxiter=1))
    assert out["status"] == nb.NB_NOT_CONVERGED and out["iters"] == 1
    out = mesh.solve(_t(b), x, nb.default_opts(prec=nb.NB_FP32, max_outer=1))
    assert out["status"] == nb.NB_NOT_CONVERGED
    with pytest.raises(nb.NbError) as ei:
        nb.Mesh(ctx, 1, 1, 1, 5, 3.0)
    assert ei.value.status == nb.NB_ERR_MESH
    with pytest.raises(nb.NbError):
        nb.Mesh(ctx, 1, 1, 1, 16, 0.0)
    with pytest.raises(nb.NbError):
        mesh.solve(_t(b), x, nb.default_opts(prec=nb.NB_FP32, pc=nb.NB_PC_LEARNED))
    # zero right-hand side: x = 0 exactly
    z = torch.zeros(box.n_local, dtype=torch.float64, device="cuda")
    x.fill_(1.0)
    for prec in (nb.NB_FP64, nb.NB_FP32):
        out = mesh.solve(z, x, nb.default_opts(prec=prec))
        assert out["status"] == 0 and float(x.abs().max()) == 0.0


# Odd element counts (ragged last wave of blocks) at even and odd n, through
# the plain operator and the mixed solve (fused CG step, folded update).
ODD_E_BOXES = [Box(3, 1, 1, 9, 0.05), Box(3, 3, 1, 5, 0.05), Box(1, 1, 1, 3, 0.0),
               Box(5, 1, 1, 3, 0.05), Box(3, 1, 1, 7, 0.05)]


@pytest.mark.parametrize("box", ODD_E_BOXES, ids=lambda b: f"{b.nx}x{b.ny}x{b.nz}N{b.N}")
def test_odd_element_counts(nb, ctx, box):
    import torch
    mesh = nb.Mesh.from_box(ctx, box)
    P = oracle.Problem(box)
    rng = np.random.default_rng(11)
    u = rng.uniform(-1, 1, box.n_local).astype(np.float32)
    w = torch.empty(box.n_local, dtype=torch.float32, device="cuda")
    mesh.ax(nb.NB_FP32, _t(u), w)
    ref = P.ax_local(u.astype(np.float64))
    err = np.max(np.abs(w.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert err <= tol_ax32(box.n), err
    # the fused CG step and the folded update inside the mixed solve
    b = P.to_local(rhs_global(box, 0))
    if not np.any(b):
        return
    xo, _, _, _ = P.pcg(b, tol=1e-13, maxit=5000)
    x = torch.zeros(box.n_local, dtype=torch.float64, device="cuda")
    out = mesh.solve(_t(b), x, nb.default_opts(prec=nb.NB_FP32, rtol=1e-10))
    assert out["status"] == 0, out
    xg = x.cpu().numpy()
    assert P.true_relres(b, xg) < 1.01e-10
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-8


def test_reliable_update_keeps_fp64_iteration_count(nb, ctx):
    """Refinement that keeps the search direction across the FP64 residual
    replacement (opts.restart = 0) needs about the FP64 PCG iteration count;
    restarting each inner solve (restart = 1) needs more.  Both reach the
    FP64 oracle's solution."""
    import torch
    box = Box(6, 5, 4, 7, 0.05)
    mesh = nb.Mesh.from_box(ctx, box)
    P = oracle.Problem(box)
    b = P.to_local(rhs_global(box, 2))
    xo, _, _, _ = P.pcg(b, tol=1e-13, maxit=5000)
    x = torch.zeros(box.n_local, dtype=torch.float64, device="cuda")
    f64 = mesh.solve(_t(b), x, nb.default_opts(prec=nb.NB_FP64, rtol=1e-10))
    its = {}
    for restart in (0, 1):
        x.zero_()
        out = mesh.solve(_t(b), x, nb.default_opts(prec=nb.NB_FP32, rtol=1e-10, restart=restart))
        assert out["status"] == 0, out
        xg = x.cpu().numpy()
        assert P.true_relres(b, xg) < 1.01e-10
        assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-8
        its[restart] = out["iters"]
    print(f"FP64 PCG {f64['iters']}, kept direction {its[0]}, restarted {its[1]}")
    assert its[0] <= 1.1 * f64["iters"]
    assert its[0] < its[1]
    with pytest.raises(nb.NbError):
        mesh.solve(_t(b), x, nb.default_opts(prec=nb.NB_FP32, restart=2))


def test_variant_change_after_a_solve_takes_effect(nb, ctx):
    """A solve captures its iteration in a CUDA graph; choosing another
    operator variant afterwards must re-capture it.  The variants round
    differently in FP32, so the solution bits tell which kernel ran: a solve
    after switching from variant 0 to the last variant must give the bits of
    a solve on a fresh mesh set to the last variant from the start."""
    import torch
    box = Box(3, 3, 2, 7, 0.05)
    P = oracle.Problem(box)
    b = _t(P.to_local(rhs_global(box, 6)))
    m1 = nb.Mesh.from_box(ctx, box)
    last = m1.ax_variants(nb.NB_FP32) - 1
    assert last >= 2
    x = torch.zeros_like(b)
    m1.set_ax_variant(nb.NB_FP32, 0)
    m1.solve(b, x, nb.default_opts(prec=nb.NB_FP32))
    x0 = x.clone()
    m1.set_ax_variant(nb.NB_FP32, last)
    x.zero_()
    m1.solve(b, x, nb.default_opts(prec=nb.NB_FP32))
    m2 = nb.Mesh.from_box(ctx, box)
    m2.set_ax_variant(nb.NB_FP32, last)
    y = torch.zeros_like(b)
    m2.solve(b, y, nb.default_opts(prec=nb.NB_FP32))
    assert torch.equal(x, y)
    assert not torch.equal(x0, y), "variants 0 and last give identical bits: no evidence"
    with pytest.raises(nb.NbError):
        m1.set_ax_variant(nb.NB_FP32, last + 1)


@pytest.mark.parametrize("box", [Box(3, 3, 2, 9, 0.05), Box(4, 3, 2, 7, 0.05), Box(2, 2, 3, 11, 0.05)],
                         ids=lambda b: f"{b.nx}x{b.ny}x{b.nz}N{b.N}")
def test_update_variants_are_bit_identical(nb, ctx, box):
    """The kernels of the FP32 update with the folded summation (element
    ranges, node pairs, bulk-copied element ranges) sum the copies of every
    node in the same order: the mixed solve gives the same bits with each,
    and reaches the oracle's solution."""
    import torch
    mesh = nb.Mesh.from_box(ctx, box)
    P = oracle.Problem(box)
    bl = P.to_local(rhs_global(box, 8))
    b = _t(bl)
    xs = []
    for v in (1, 2, 3, 0):
        mesh.set_update_variant(v)
        x = torch.zeros_like(b)
        out = mesh.solve(b, x, nb.default_opts(prec=nb.NB_FP32))
        assert out["status"] == 0, (v, out)
        xs.append(x)
    for x in xs[1:]:
        assert torch.equal(x, xs[0])
    xo, _, _, _ = P.pcg(bl, tol=1e-13, maxit=20000)
    xg = xs[0].cpu().numpy()
    assert P.true_relres(bl, xg) < 1.01e-10
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-8
    with pytest.raises(nb.NbError):
        mesh.set_update_variant(4)


@pytest.mark.parametrize("box", [Box(3, 3, 2, 9, 0.05), Box(4, 3, 2, 7, 0.05)],
                         ids=lambda b: f"{b.nx}x{b.ny}x{b.nz}N{b.N}")
@pytest.mark.parametrize("use_graph", [1, 0], ids=["graph", "host"])
@pytest.mark.parametrize("maxiter", [7, 8, 10000])
def test_deferred_x_steps_give_the_single_step_bits(nb, ctx, box, use_graph, maxiter):
    """Jacobi CG with the element-range update defers the x step over pairs of
    iterations (two direction buffers): its solution has the bits of the
    node-pair update, which steps x every iteration.  maxiter 7 stops the
    solve after the first iteration of a pair (the pending step is applied
    after the loop), 8 after the second; 10000 converges.  (The built-in rule
    defers only where the loop's vectors exceed L2; mode 1 forces it here.)"""
    import torch
    mesh = nb.Mesh.from_box(ctx, box)
    mesh.set_x_deferral(1)
    P = oracle.Problem(box)
    b = _t(P.to_local(rhs_global(box, 11)))
    res = {}
    for v in (1, 2):
        mesh.set_update_variant(v)
        x = torch.zeros_like(b)
        out = mesh.solve(b, x, nb.default_opts(prec=nb.NB_FP32, use_graph=use_graph,
                                               maxiter=maxiter))
        res[v] = (x, out)
    (x1, o1), (x2, o2) = res[1], res[2]
    assert o1["status"] == o2["status"], (o1, o2)
    assert (o1["status"] == 0) == (maxiter > 100), o1
    assert o1["iters"] == o2["iters"] and o1["outer_iters"] == o2["outer_iters"]
    assert torch.equal(x1, x2)
    # one step-completing launch after each inner solve of the deferred form
    assert 0 < o1["launches"] - o2["launches"] <= max(o1["outer_iters"], 1), (o1, o2)
    if maxiter > 100:
        assert P.true_relres(P.to_local(rhs_global(box, 11)), x1.cpu().numpy()) < 1.01e-10
    # mode 0 and the built-in rule (a mesh this small fits in L2) step x every
    # iteration: the same bits, no completing launch
    for mode in (0, -1):
        mesh.set_x_deferral(mode)
        mesh.set_update_variant(1)
        x = torch.zeros_like(b)
        o = mesh.solve(b, x, nb.default_opts(prec=nb.NB_FP32, use_graph=use_graph,
                                             maxiter=maxiter))
        assert torch.equal(x, x1) and o["launches"] == o2["launches"], (mode, o, o2)
    with pytest.raises(nb.NbError):
        mesh.set_x_deferral(2)


def test_x_deferral_rule_by_size(nb, ctx):
    """The built-in rule defers the x steps where the loop's six vectors (24 B
    per local node) exceed L2 -- an 8000-element N=9 mesh, 192 MB -- and not
    where they fit (a 2x2x2 mesh); either way the bits are those of x stepped
    every iteration."""
    import torch
    big = Box(20, 20, 20, 9, 0.05)
    mesh = nb.Mesh.from_box(ctx, big)
    b = torch.from_numpy(rhs_global(big, 3)).to("cuda")
    bl = torch.empty(big.n_local, dtype=torch.float64, device="cuda")
    mesh.to_local(nb.NB_FP64, b, bl, masked=True)
    res = {}
    for mode in (0, -1):
        mesh.set_x_deferral(mode)
        x = torch.zeros_like(bl)
        res[mode] = (x, mesh.solve(bl, x, nb.default_opts(prec=nb.NB_FP32)))
    (x0, o0), (xa, oa) = res[0], res[-1]
    assert o0["status"] == oa["status"] == 0 and o0["iters"] == oa["iters"]
    assert torch.equal(x0, xa)
    assert 0 < oa["launches"] - o0["launches"] <= oa["outer_iters"], (o0, oa)
    small = Box(2, 2, 2, 9, 0.05)
    m2 = nb.Mesh.from_box(ctx, small)
    b2 = _t(oracle.Problem(small).to_local(rhs_global(small, 3)))
    launches = []
    for mode in (0, -1):
        m2.set_x_deferral(mode)
        launches.append(m2.solve(b2, torch.zeros_like(b2), nb.default_opts(prec=nb.NB_FP32))["launches"])
    assert launches[0] == launches[1]


def test_mesh_outlives_its_context(nb):
    """A mesh keeps its context alive: destroying the context first (as a
    garbage collector may) leaves the mesh usable and its destruction safe."""
    import torch
    c = nb.Context(0)
    box = Box(2, 2, 2, 5, 0.05)
    m = nb.Mesh.from_box(c, box)
    c.close()
    P = oracle.Problem(box)
    b = _t(P.to_local(rhs_global(box, 1)))
    x = torch.zeros_like(b)
    out = m.solve(b, x, nb.default_opts(prec=nb.NB_FP64))
    assert out["status"] == 0
    m.close()


@pytest.mark.parametrize("prec", ["tc_bf16", "tc_f16"])
def test_tensor_core_refinement_reaches_the_oracle(nb, ctx, prec):
    """Refinement whose inner solves use the 16-bit tensor-core contractions
    (about 5e-3 / 5e-4 relative operator error) still reduces the FP64
    residual every step here and reaches the FP64 oracle's solution; the
    precision it finished in is reported."""
    import torch
    box = Box(8, 8, 8, 7, 0.05)
    mesh = nb.Mesh.from_box(ctx, box)
    P = oracle.Problem(box)
    b = P.to_local(rhs_global(box, 0))
    xo, _, _, _ = P.pcg(b, tol=1e-13, maxit=5000)
    x = torch.zeros(box.n_local, dtype=torch.float64, device="cuda")
    out = mesh.solve(_t(b), x, nb.default_opts(prec=nb.PREC_NAMES[prec], rtol=1e-10))
    print(f"{prec} inner solves: status {out['status']}, final precision {out['final_prec']}, "
          f"{out['iters']} iterations, {out['outer_iters']} refinement steps")
    assert out["status"] == nb.NB_OK, out
    xg = x.cpu().numpy()
    assert P.true_relres(b, xg) < 1.01e-10
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-8


@pytest.mark.parametrize("prec", ["fp32", "tc_bf16"])
def test_precision_adaptivity_reaches_fp64_inner_solves(nb, ctx, prec):
    """Asked for a residual below what FP64 resolves, the refinement stalls at
    the FP64 residual's rounding floor; each stall raises the inner precision
    one step (tensor-core -> FP32 -> FP64 PCG), and only when the FP64 inner
    solves stall too does the solve end as stagnated -- with the solution at
    the oracle's."""
    import torch
    box = Box(3, 3, 3, 5, 0.05)
    mesh = nb.Mesh.from_box(ctx, box)
    P = oracle.Problem(box)
    b = P.to_local(rhs_global(box, 1))
    xo, _, _, _ = P.pcg(b, tol=1e-14, maxit=5000)
    x = torch.zeros(box.n_local, dtype=torch.float64, device="cuda")
    out = mesh.solve(_t(b), x, nb.default_opts(prec=nb.PREC_NAMES[prec], rtol=1e-16,
                                               max_outer=80, maxiter=100000))
    print(f"{prec}, rtol 1e-16: status {out['status']}, final precision {out['final_prec']}, "
          f"rel_res {out['rel_res']:.2e}, {out['outer_iters']} refinement steps")
    assert out["status"] == nb.NB_STAGNATED, out
    assert out["final_prec"] == nb.NB_FP64
    assert out["rel_res"] < 1e-13
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-10
