"""The slab-partitioned CG (paper_2405_11065_gb300.slab) on CPU with the
oracle's slab backend: several slabs in one process, and one slab per
process on two gloo ranks (the communication through torch.distributed) --
both against the oracle's PCG of the undivided box."""
import os
import socket

import numpy as np
import pytest

import oracle
from workloads import Box, rhs_global
from slab_oracle import OracleSlab


def _load_slab_module():
    """The driver module by path: its loop and communicators need no CUDA
    library (only its GpuSlab backend does), so this CPU test runs without
    importing the package, which loads the library."""
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location(
        "nb_slab_driver", os.path.join(root, "paper_2405_11065_gb300", "slab.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


S = _load_slab_module()


def _slabs(box, bounds):
    bg = rhs_global(box, 3)
    plane = (box.nx * box.N + 1) * (box.ny * box.N + 1)
    out = []
    for z0, z1 in bounds:
        s = OracleSlab(box, z0, z1)
        s.finish_diag(None, None) if not (s.lo or s.hi) else None
        out.append((s, bg[z0 * box.N * plane:(z1 * box.N + 1) * plane]))
    return out, bg


def _assemble(box, bounds, parts):
    plane = (box.nx * box.N + 1) * (box.ny * box.N + 1)
    xg = np.zeros(box.n_global)
    for (z0, z1), xs in zip(bounds, parts):
        xg[z0 * box.N * plane:(z1 * box.N + 1) * plane] = xs
    return xg


def test_slab_bounds():
    assert S.slab_bounds(7, 3) == [(0, 3), (3, 5), (5, 7)]
    assert S.slab_bounds(4, 1) == [(0, 4)]
    with pytest.raises(ValueError):
        S.slab_bounds(2, 3)


@pytest.mark.parametrize("nslabs", [2, 3])
def test_in_process_slabs_match_the_oracle(nslabs):
    box = Box(3, 4, 6, 4, 0.05)
    bounds = S.slab_bounds(box.nz, nslabs)
    pairs, bg = _slabs(box, bounds)
    slabs = [s for s, _ in pairs]
    comm = S.InProcessComm()
    S.setup_diagonal(slabs, comm)
    for s, bs in pairs:
        s.set_rhs(bs)
    it, rel, hist = S.slab_pcg(slabs, comm, tol=1e-10, maxit=2000)
    P = oracle.Problem(box)
    b = P.to_local(bg)
    xo, ito, relo, histo = P.pcg(b, tol=1e-10, maxit=2000, history=True)
    assert abs(it - ito) <= 1, (it, ito)
    k = min(len(hist), len(histo), 30)
    np.testing.assert_allclose(hist[:k], histo[:k], rtol=1e-9)
    xg = _assemble(box, bounds, [s.solution() for s in slabs])
    xL = P.to_local(xg)
    assert P.true_relres(b, xL) < 1.01e-10
    assert np.linalg.norm(xL - xo) <= 1e-9 * np.linalg.norm(xo)


def _rank(rank, world, port, box, bounds, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pairs, _ = _slabs(box, [bounds[rank]])
        s, bs = pairs[0]
        comm = S.TorchDistComm("cpu")
        S.setup_diagonal([s], comm)
        s.set_rhs(bs)
        it, rel, hist = S.slab_pcg([s], comm, tol=1e-10, maxit=2000)
        np.save(os.path.join(out_dir, f"x{rank}.npy"), s.solution())
        np.save(os.path.join(out_dir, f"h{rank}.npy"), np.array(hist))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_match_the_oracle(tmp_path, world):
    import torch.multiprocessing as mp
    box = Box(3, 3, 6, 4, 0.05)
    bounds = S.slab_bounds(box.nz, world)
    mp.start_processes(_rank, args=(world, _free_port(), box, bounds, str(tmp_path)),
                       nprocs=world, join=True, start_method="spawn")
    parts = [np.load(tmp_path / f"x{r}.npy") for r in range(world)]
    hists = [np.load(tmp_path / f"h{r}.npy") for r in range(world)]
    for h in hists[1:]:
        np.testing.assert_array_equal(h, hists[0])  # every rank saw the same sums
    P = oracle.Problem(box)
    b = P.to_local(rhs_global(box, 3))
    xo, ito, _, _ = P.pcg(b, tol=1e-10, maxit=2000)
    assert abs(len(hists[0]) - ito) <= 1
    xL = P.to_local(_assemble(box, bounds, parts))
    assert P.true_relres(b, xL) < 1.01e-10
    assert np.linalg.norm(xL - xo) <= 1e-9 * np.linalg.norm(xo)
