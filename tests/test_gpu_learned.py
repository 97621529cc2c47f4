"""The learned per-element preconditioner: GPU gradients against the FP64
oracle's backward pass, the GPU training targets and the preconditioner
against the oracle, and flexible CG with the trained network against
Jacobi-PCG (the gain is measured and printed; written as JSON into the
directory NB_RESULTS_DIR names, if set)."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import mlp
from workloads import Box, HELDOUT_SEEDS, LEARNED_16CUBE_N7, TRAIN_SEEDS, rhs_global

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


def _cos(a, b):
    a, b = a.reshape(-1), b.reshape(-1)
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))


def test_gpu_gradients_match_oracle_backward(nb, ctx):
    import torch
    N, h, B = 3, 8, 96
    d = (N + 1) ** 3
    model = nb.Model(ctx, N, h, seed=1)
    p = mlp.init_params(d, h, seed=5)
    rng = np.random.default_rng(6)
    p["W"] = p["W"] * 3.0  # pre-activations of order one
    p["a"] = rng.uniform(-1.5, 1.5, h)
    # parameters exactly representable in BF16 so both sides use the same weights
    bf = lambda a: torch.from_numpy(np.asarray(a, np.float32)).bfloat16().float().numpy()
    p = {k: bf(v).astype(np.float64) for k, v in p.items()}
    model.set_params(p)
    X = bf(rng.uniform(-1, 1, (B, d))).astype(np.float64)
    T = rng.uniform(-1, 1, (B, d))
    loss, g = model.grad(torch.from_numpy(X.astype(np.float32)).cuda(),
                         torch.from_numpy(T.astype(np.float32)).cuda())
    ref = mlp.backward(p, X, T)
    lref = mlp.loss(p, X, T)
    assert abs(loss - lref) <= 1e-2 * lref
    for k in ("W", "a"):
        c = _cos(g[k].astype(np.float64), ref[k])
        rel = np.linalg.norm(g[k] - ref[k]) / np.linalg.norm(ref[k])
        print(f"grad {k}: cosine {c:.6f}, relative error {rel:.2e}")
        assert c > 0.999, (k, c)


def test_training_targets_match_oracle(nb, ctx):
    import torch
    box = Box(2, 2, 2, 5, 0.05)
    mesh = nb.Mesh.from_box(ctx, box)
    P = oracle.Problem(box)
    r = P.to_local(rhs_global(box, 4))
    elems = [0, 3, 7]
    X, T = nb.Model.targets(mesh, torch.from_numpy(r).cuda(), elems)
    Xo, To = mlp.interior_targets(P, r, elems)
    np.testing.assert_allclose(X.cpu().numpy(), Xo, atol=1e-7)
    err = np.max(np.abs(T.cpu().numpy() - To)) / np.max(np.abs(To))
    print(f"element-interior targets: max relative error vs dense solve {err:.2e}")
    assert err < 1e-5


def test_preconditioner_matches_oracle_forward(nb, ctx):
    import torch
    box = Box(2, 2, 2, 3, 0.05)
    mesh = nb.Mesh.from_box(ctx, box)
    P = oracle.Problem(box)
    model = nb.Model(ctx, box.N, 16, seed=2)
    params = {k: v.astype(np.float64) for k, v in model.params().items()}
    model.attach(mesh)
    r = P.to_local(rhs_global(box, 3))
    rt = torch.from_numpy(r.astype(np.float32)).cuda()
    z = torch.empty_like(rt)
    model.apply(mesh, rt, z)
    ref = mlp.precondition_interior(params, P, r.astype(np.float32).astype(np.float64))
    err = np.max(np.abs(z.cpu().numpy() - ref)) / np.max(np.abs(ref))
    print(f"learned preconditioner (BF16) max relative error vs FP64 oracle: {err:.2e}")
    assert err < 3e-2


def _bf16(a):
    """Round to BF16 (nearest even), as the kernels' __float2bfloat16_rn."""
    import torch
    return torch.from_numpy(np.asarray(a, np.float32)).bfloat16().double().numpy()


@pytest.mark.parametrize("nx,ny,nz,N,h", [
    (3, 2, 2, 7, 96),      # 12 elements: one per block
    (6, 5, 4, 5, 40),      # N = 5: padded K (224) and M (256); hidden width not a multiple of 16
    (16, 16, 16, 7, 96),   # the learned workload's mesh: 26-27 elements per block
    (18, 18, 16, 7, 96),   # 34-35 elements per block: a full tile and a ragged one
    (18, 18, 16, 5, 48),
])
def test_fused_step_matches_oracle(nb, ctx, nx, ny, nz, N, h):
    """The fused preconditioner step of the learned flexible CG (tensor-core
    products, the z pass and its two dot products) element by element against
    the FP64 oracle network, and against the same arithmetic with the
    kernel's two BF16 roundings (inputs X and hidden activations) emulated."""
    import torch
    box = Box(nx, ny, nz, N, 0.05)
    mesh = nb.Mesh.from_box(ctx, box)
    P = oracle.Problem(box)
    model = nb.Model(ctx, N, h, seed=3)
    p = mlp.init_params(box.n ** 3, h, seed=11)
    rng = np.random.default_rng(12)
    p["W"] = p["W"] * 2.0
    p["a"] = rng.uniform(0.5, 1.5, h)
    p = {k: _bf16(v) for k, v in p.items()}  # weights exact in BF16
    model.set_params(p)
    model.attach(mesh)
    r = P.to_local(rhs_global(box, 5)).astype(np.float32).astype(np.float64)
    wprev = rng.uniform(-1, 1, box.n_local).astype(np.float32).astype(np.float64)
    rt = torch.from_numpy(r.astype(np.float32)).cuda()
    wt = torch.from_numpy(wprev.astype(np.float32)).cuda()
    zt = torch.full_like(rt, float("nan"))
    zw, rz = model.step(mesh, rt, wt, zt)
    z = zt.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(z))
    # the FP64 oracle network
    ref = mlp.precondition_interior(p, P, r)
    err = np.max(np.abs(z - ref)) / np.max(np.abs(ref))
    # the same with X and a * gelu(H) rounded to BF16
    n3 = box.n ** 3
    R = r.reshape(-1, n3)
    nrm = np.linalg.norm(R, axis=1)
    X = _bf16(R / np.where(nrm > 0, nrm, 1.0)[:, None])
    Hs = _bf16(p["a"] * mlp.gelu(X @ p["W"]))
    corr = (Hs @ p["W"].T) * nrm[:, None] * mlp.interior_mask(N)[None, :]
    emu = P.dinv * r + corr.reshape(-1)
    err_emu = np.max(np.abs(z - emu)) / np.max(np.abs(emu))
    # the in-kernel dot products against FP64 sums of the kernel's own z
    zw_ref = float(np.dot(z, wprev))
    rz_ref = float(np.sum(P.c * r * z))
    dz = abs(zw - zw_ref) / np.sum(np.abs(z * wprev))
    dr = abs(rz - rz_ref) / abs(rz_ref)
    print(f"E={box.E} N={N} h={h}: z vs FP64 oracle {err:.2e}, vs BF16-emulated {err_emu:.2e}; "
          f"(z, w_prev) {dz:.1e}, (r, z) {dr:.1e}")
    assert err < 3e-2
    assert err_emu < 2e-3
    assert dz < 1e-6 and dr < 1e-6


def _rhs(nb, mesh, box, seed):
    import torch
    bg = torch.from_numpy(rhs_global(box, seed)).cuda()
    b = torch.empty(box.n_local, dtype=torch.float64, device="cuda")
    mesh.to_local(nb.NB_FP64, bg, b)
    return b


def _pipeline(nb, ctx, box, train_seeds, snaps, per_snap, epochs, hidden=48):
    """Pairs from the Jacobi-PCG iterates of the training seeds, then Adam
    (two thirds of the epochs at 1e-3, the rest at 3e-4)."""
    import torch
    mesh = nb.Mesh.from_box(ctx, box)
    model = nb.Model(ctx, box.N, hidden, seed=7)
    Xs, Ts = [], []
    for s in train_seeds:
        X, T = nb.Model.collect(mesh, _rhs(nb, mesh, box, s), snaps, per_snap, seed=s)
        Xs.append(X)
        Ts.append(T)
    X, T = torch.cat(Xs), torch.cat(Ts)
    model.train(X, T, epochs=2 * epochs // 3, batch=256, lr=1e-3)
    loss = model.train(X, T, epochs=epochs - 2 * epochs // 3, batch=256, lr=3e-4)
    model.attach(mesh)
    return mesh, model, loss, int(X.shape[0])


def _compare(nb, mesh, box, seeds):
    import torch
    res = []
    for s in seeds:
        b = _rhs(nb, mesh, box, s)
        x = torch.zeros_like(b)
        jac = mesh.solve(b, x, nb.default_opts(prec=nb.NB_FP32, pc=nb.NB_PC_JACOBI))
        xl = torch.zeros_like(b)
        mesh.solve(b, xl, nb.default_opts(prec=nb.NB_FP32, pc=nb.NB_PC_LEARNED))  # warm-up
        xl.zero_()
        lrn = mesh.solve(b, xl, nb.default_opts(prec=nb.NB_FP32, pc=nb.NB_PC_LEARNED))
        res.append((s, jac, lrn, b, xl))
    return res


def test_learned_fcg_small_mesh(nb, ctx):
    box = Box(4, 4, 4, 5, 0.05)
    mesh, model, loss, npairs = _pipeline(nb, ctx, box, TRAIN_SEEDS,
                                          [1, 2, 4, 8, 16, 32, 64, 100], 64, epochs=60)
    P = oracle.Problem(box)
    for s, jac, lrn, b, xl in _compare(nb, mesh, box, HELDOUT_SEEDS[:2]):
        print(f"seed {s}: Jacobi-PCG {jac['iters']} its {jac['seconds']*1e3:.2f} ms; "
              f"learned FCG {lrn['iters']} its {lrn['seconds']*1e3:.2f} ms status {lrn['status']}")
        assert lrn["status"] == nb.NB_OK
        assert lrn["rel_res"] < 1e-10
        assert P.true_relres(b.cpu().numpy(), xl.cpu().numpy()) < 1.01e-10
        assert lrn["iters"] < jac["iters"]  # the network's gain over Jacobi


def test_learned_preconditioner_workload(nb, ctx):
    """The learned-preconditioner workload: 16^3 deformed box, N = 7, about
    10,000 element pairs from Jacobi-PCG iterates on 8 training seeds, a
    network of 49,248 parameters, evaluated on held-out seeds against
    Jacobi-PCG (iterations and time)."""
    box = LEARNED_16CUBE_N7
    snaps = [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 800]  # across the ~900-iteration solve
    mesh, model, loss, npairs = _pipeline(nb, ctx, box, TRAIN_SEEDS, snaps, 120, epochs=60,
                                          hidden=96)
    assert npairs >= 10000
    out = []
    for s, jac, lrn, b, xl in _compare(nb, mesh, box, HELDOUT_SEEDS[:2]):
        out.append(dict(seed=s, jacobi_iters=jac["iters"], jacobi_ms=jac["seconds"] * 1e3,
                        learned_iters=lrn["iters"], learned_ms=lrn["seconds"] * 1e3,
                        learned_status=lrn["status"], learned_rel_res=lrn["rel_res"]))
        assert lrn["status"] == nb.NB_OK
        assert lrn["rel_res"] < 1e-10
        assert lrn["iters"] < jac["iters"]  # the network's gain over Jacobi
    summary = dict(pairs=npairs, params=model.nparam, final_train_loss=loss, results=out)
    print("learned workload:", json.dumps(summary))
    out_dir = os.environ.get("NB_RESULTS_DIR")
    if out_dir:
        os.makedirs(out_dir, exist_ok=True)
        with open(os.path.join(out_dir, "learned_workload.json"), "w") as f:
            json.dump(summary, f, indent=1)
