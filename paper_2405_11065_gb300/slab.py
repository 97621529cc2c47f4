"""Conjugate gradients on a box cut into z-slabs, one mesh per slab.

Nekbone runs its CG loop (Section 4.1, Table 1) on MPI ranks that each own a
block of elements: the direct-stiffness summation inside ``ax`` exchanges the
nodes shared between ranks, and each ``glsc3`` ends in a global sum (three
per iteration); Section 7.2 (Table 5) scales the code over ranks.  Here the
box of nx x ny x nz elements is cut along z; slab s holds the elements
z_s <= ez < z_(s+1) (``nb_setup_slab``) and shares one node plane with each
neighbouring slab.  Per iteration:

1. every slab forms p and w = A_L p (``nb_cg_step``); the slabs' p.w are summed;
2. every slab packs its sums of w on its interface planes (``nb_slab_face``),
   sums w over its own copies (``nb_dssum``), and adds the neighbours' planes
   (``nb_slab_face_add``): w is then the box's summed w on every slab;
3. every slab updates x and r (``nb_cg_update``); the slabs' (r, z) and
   (r, r) are summed, and beta and the stopping test follow.

The loop is written against two small interfaces, so that the same code runs
the slabs of one process (``InProcessComm``: several slabs on one GPU, or on
several GPUs of one node) and one slab per process (``TorchDistComm`` over
``torch.distributed``: NCCL between GPUs, gloo between CPU processes):

* a slab backend: ``lo`` / ``hi`` (interface below / above), ``diag_face``,
  ``finish_diag``, ``dots``, ``step``, ``face_w``, ``dssum_w``,
  ``face_add_w``, ``update`` -- ``GpuSlab`` calls the library;
* a communicator: ``allreduce(values)`` sums floats over all processes,
  ``exchange(slabs, lo_planes, hi_planes)`` returns, per local slab, the
  plane of the slab below (from its upper side) and of the slab above (from
  its lower side).

Every arithmetic step runs in the library's kernels; this module moves plane
vectors and scalars between slabs.
"""
from __future__ import annotations

import math
from typing import Sequence


def slab_bounds(nz: int, nslabs: int):
    """Element-layer bounds of nslabs z-slabs of nz layers, as even as
    possible (the lower slabs take the extra layers)."""
    if not 1 <= nslabs <= nz:
        raise ValueError("need 1 <= slabs <= nz")
    q, r = divmod(nz, nslabs)
    out, z = [], 0
    for s in range(nslabs):
        z1 = z + q + (1 if s < r else 0)
        out.append((z, z1))
        z = z1
    return out


class InProcessComm:
    """All slabs belong to this process: sums are already complete, and the
    neighbouring planes are handed over directly."""

    def allreduce(self, values: Sequence[float]):
        return list(values)

    def exchange(self, slabs, lo_planes, hi_planes):
        n = len(slabs)
        recv_lo = [hi_planes[i - 1] if i > 0 else None for i in range(n)]
        recv_hi = [lo_planes[i + 1] if i + 1 < n else None for i in range(n)]
        return recv_lo, recv_hi


class TorchDistComm:
    """Slabs spread over the ranks of a torch.distributed process group in
    rank order (each rank's slabs contiguous in z).  Sums are one all_reduce
    of a float64 tensor on ``device``; planes travel by isend / irecv between
    neighbouring ranks (NCCL: CUDA tensors; gloo: CPU tensors)."""

    def __init__(self, device="cpu", group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.device = device
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def allreduce(self, values: Sequence[float]):
        import torch
        t = torch.tensor(list(values), dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, group=self.group)
        return [float(v) for v in t.cpu()]

    def exchange(self, slabs, lo_planes, hi_planes):
        import torch
        n = len(slabs)
        recv_lo = [hi_planes[i - 1] if i > 0 else None for i in range(n)]
        recv_hi = [lo_planes[i + 1] if i + 1 < n else None for i in range(n)]
        ops = []
        if n and slabs[0].lo:  # the slab below lives on the previous rank
            buf = torch.empty_like(lo_planes[0])
            ops.append(self.dist.P2POp(self.dist.isend, lo_planes[0].contiguous(), self.rank - 1,
                                       self.group))
            ops.append(self.dist.P2POp(self.dist.irecv, buf, self.rank - 1, self.group))
            recv_lo[0] = buf
        if n and slabs[-1].hi:  # the slab above lives on the next rank
            buf = torch.empty_like(hi_planes[-1])
            ops.append(self.dist.P2POp(self.dist.isend, hi_planes[-1].contiguous(), self.rank + 1,
                                       self.group))
            ops.append(self.dist.P2POp(self.dist.irecv, buf, self.rank + 1, self.group))
            recv_hi[-1] = buf
        if ops:
            for req in self.dist.batch_isend_irecv(ops):
                req.wait()
        return recv_lo, recv_hi


def setup_diagonal(slabs, comm):
    """Complete every slab's Jacobi diagonal with its neighbours' parts."""
    lo = [s.diag_face(0) if s.lo else None for s in slabs]
    hi = [s.diag_face(1) if s.hi else None for s in slabs]
    recv_lo, recv_hi = comm.exchange(slabs, lo, hi)
    for s, a, b in zip(slabs, recv_lo, recv_hi):
        s.finish_diag(a, b)


def sum_w(slabs, comm):
    """w of every slab becomes the box's direct-stiffness sum of w (masked)."""
    lo = [s.face_w(0) if s.lo else None for s in slabs]
    hi = [s.face_w(1) if s.hi else None for s in slabs]
    for s in slabs:
        s.dssum_w()
    recv_lo, recv_hi = comm.exchange(slabs, lo, hi)
    for s, a, b in zip(slabs, recv_lo, recv_hi):
        if a is not None:
            s.face_add_w(0, a)
        if b is not None:
            s.face_add_w(1, b)


def slab_pcg(slabs, comm, tol: float = 1e-10, maxit: int = 10000):
    """Jacobi-PCG in the order of Table 1 over the slabs (each slab's r holds
    its part of the right-hand side, x and p are zero).  Returns (iterations,
    final relative residual sqrt(rtr) / |b|, residual history)."""
    rtz, rtr = comm.allreduce([sum(v) for v in zip(*(s.dots() for s in slabs))] or [0.0, 0.0])
    bn2 = rtr
    if not bn2 > 0.0:
        return 0, 0.0, []
    beta, hist, rel, it = 0.0, [], 1.0, 0
    for it in range(1, maxit + 1):
        pap = comm.allreduce([sum(s.step(beta) for s in slabs)])[0]
        if not pap > 0.0:
            raise FloatingPointError(f"p.Ap = {pap} at iteration {it}")
        alpha = rtz / pap
        sum_w(slabs, comm)
        rtz_new, rtr = comm.allreduce([sum(v) for v in zip(*(s.update(alpha) for s in slabs))])
        beta = rtz_new / rtz
        rtz = rtz_new
        rel = math.sqrt(rtr / bn2)
        hist.append(rel)
        if not math.isfinite(rel):
            raise FloatingPointError(f"non-finite residual at iteration {it}")
        if rel < tol:
            break
    return it, rel, hist


class GpuSlab:
    """One z-slab on the GPU: its mesh (``Mesh(..., slab=(z0, z1))``) and the
    CG vectors x, r, p, w as CUDA tensors of the precision's type."""

    def __init__(self, ctx, nx, ny, nz, z0, z1, N, deform=0.0, prec=None):
        import torch
        from . import NB_FP64, Mesh
        self.prec = NB_FP64 if prec is None else prec
        self.mesh = Mesh(ctx, nx, ny, nz, N, deform, slab=(z0, z1))
        self.box = (nx, ny, nz, N)
        self.z0, self.z1 = z0, z1
        self.lo, self.hi = z0 > 0, z1 < nz
        dt = torch.float64 if self.prec == NB_FP64 else torch.float32
        dev = torch.device("cuda", ctx.device)
        n = self.mesh.n_local
        self.x = torch.zeros(n, dtype=dt, device=dev)
        self.r = torch.zeros(n, dtype=dt, device=dev)
        self.p = torch.zeros(n, dtype=dt, device=dev)
        self.w = torch.zeros(n, dtype=dt, device=dev)
        np_ = self.mesh.plane_size()
        self.planes = [torch.zeros(np_, dtype=dt, device=dev) for _ in range(2)]
        self.dplanes = [torch.zeros(np_, dtype=torch.float64, device=dev) for _ in range(2)]

    def global_range(self):
        """[start, stop) of this slab's nodes in the box's G-vector."""
        nx, ny, _, N = self.box
        plane = (nx * N + 1) * (ny * N + 1)
        return self.z0 * N * plane, (self.z1 * N + 1) * plane

    def set_rhs(self, bg):
        """r = the slab's part of the box's right-hand side G-vector bg (CUDA
        tensor, float64), masked; x = p = 0."""
        from . import NB_FP64
        a, b = self.global_range()
        sub = bg[a:b].contiguous()
        if self.prec != NB_FP64:
            sub = sub.float()
        self.mesh.to_local(self.prec, sub, self.r, masked=True)
        self.x.zero_()
        self.p.zero_()

    def solution(self):
        """The slab's part of the solution as a G-vector of its nodes."""
        import torch
        a, b = self.global_range()
        out = torch.empty(b - a, dtype=self.x.dtype, device=self.x.device)
        self.mesh.to_global(self.prec, self.x, out)
        return out

    # --- the slab backend
    def diag_face(self, side):
        self.mesh.slab_diag_face(side, self.dplanes[side])
        return self.dplanes[side]

    def finish_diag(self, face_lo, face_hi):
        self.mesh.slab_finish_diag(face_lo, face_hi)

    def dots(self):
        return self.mesh.cg_dots(self.prec, self.r)

    def step(self, beta):
        return self.mesh.cg_step(self.prec, beta, self.r, self.p, self.w)

    def face_w(self, side):
        self.mesh.slab_face(self.prec, side, self.w, self.planes[side])
        return self.planes[side]

    def dssum_w(self):
        self.mesh.dssum(self.prec, self.w, masked=True)

    def face_add_w(self, side, plane):
        self.mesh.slab_face_add(self.prec, side, self.w, plane)

    def update(self, alpha):
        return self.mesh.cg_update(self.prec, alpha, self.x, self.r, self.p, self.w)
