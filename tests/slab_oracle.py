"""A z-slab of the box on the CPU, built from the FP64 oracle (test
infrastructure): the slab backend of ``paper_2405_11065_gb300.slab`` with
numpy arithmetic, so that the slab-partitioned CG loop and its
communication can run on CPU processes (gloo) and be compared with the
oracle's own single-domain PCG.

The slab holds the elements z0 <= ez < z1 of ``box`` with the box's
geometry (``oracle.geom`` of those elements); its numbering is that of an
nx x ny x (z1 - z0) box whose interface planes are free instead of
Dirichlet; its dot products weight each node by 1 / (the box's
multiplicity), so the slabs' partial sums add up to the box's glsc3."""
import numpy as np
import torch

import oracle
from workloads import Box


class OracleSlab:
    def __init__(self, box, z0, z1):
        self.N = N = box.N
        self.lo, self.hi = z0 > 0, z1 < box.nz
        sub = Box(box.nx, box.ny, z1 - z0, N, box.deform)
        self.nG = sub.n_global
        elems = np.array([ex + box.nx * (ey + box.ny * (ez + z0))
                          for ez in range(z1 - z0) for ey in range(box.ny) for ex in range(box.nx)],
                         dtype=np.int64)
        self.D = oracle.deriv(N)
        self.G = oracle.geom(box, elems)
        self.gid, mult, mask = oracle.numbering(sub)
        self.Gx, self.Gy = box.nx * N + 1, box.ny * N + 1
        self.plane = self.Gx * self.Gy
        Gz = (z1 - z0) * N + 1
        gx = np.arange(self.nG) % self.Gx
        gy = (np.arange(self.nG) // self.Gx) % self.Gy
        gz = np.arange(self.nG) // self.plane
        inner = (gx > 0) & (gx < self.Gx - 1) & (gy > 0) & (gy < self.Gy - 1)
        self.mask = mask.copy()
        shared = np.zeros(self.nG, dtype=bool)
        if self.lo:
            self.mask[(gz == 0) & inner] = 1
            shared |= gz == 0
        if self.hi:
            self.mask[(gz == Gz - 1) & inner] = 1
            shared |= gz == Gz - 1
        gmult = mult * np.where(shared, 2, 1)
        self.c = 1.0 / gmult[self.gid].astype(np.float64)
        self.m_l = self.mask[self.gid].astype(np.float64)
        dl = oracle.diag_local(N, self.D, self.G)
        self.diag_asm = oracle.dssum(self.gid, self.nG, dl, self.mask)
        self.dinv = None
        self.z_lo_off, self.z_hi_off = 0, (Gz - 1) * self.plane
        n = len(self.gid)
        self.x, self.r, self.p, self.w = (np.zeros(n) for _ in range(4))

    def _plane_nodes(self, side):
        off = self.z_lo_off if side == 0 else self.z_hi_off
        sel = np.nonzero((self.gid >= off) & (self.gid < off + self.plane))[0]
        return sel, self.gid[sel] - off

    def set_rhs(self, bg_slab):
        """r = the slab's part of the box's right-hand side (a G-vector of the
        slab's nodes), masked; x = p = 0."""
        self.r = np.asarray(bg_slab, dtype=np.float64)[self.gid] * self.m_l
        self.x[:] = 0.0
        self.p[:] = 0.0

    def solution(self):
        out = np.zeros(self.nG)
        out[self.gid[::-1]] = self.x[::-1]
        return out

    # --- the slab backend
    def diag_face(self, side):
        sel, pidx = self._plane_nodes(side)
        face = np.zeros(self.plane)
        face[pidx] = self.diag_asm[sel]
        return torch.from_numpy(face)

    def finish_diag(self, face_lo, face_hi):
        d = self.diag_asm.copy()
        for side, f in ((0, face_lo), (1, face_hi)):
            if f is not None:
                sel, pidx = self._plane_nodes(side)
                d[sel] += np.asarray(f)[pidx] * self.m_l[sel]
        self.dinv = np.where(self.m_l > 0, 1.0 / np.where(d != 0, d, 1.0), 0.0)

    def dots(self):
        return (oracle.glsc3(self.r, self.c, self.dinv * self.r),
                oracle.glsc3(self.r, self.c, self.r))

    def step(self, beta):
        self.p = beta * self.p + self.dinv * self.r
        self.w = oracle.ax_local(self.N, self.D, self.G, self.p)
        return float(np.sum(self.p * self.w))

    def face_w(self, side):
        sel, pidx = self._plane_nodes(side)
        face = np.zeros(self.plane)
        np.add.at(face, pidx, self.w[sel])
        return torch.from_numpy(face)

    def dssum_w(self):
        self.w = oracle.dssum(self.gid, self.nG, self.w, self.mask)

    def face_add_w(self, side, plane):
        sel, pidx = self._plane_nodes(side)
        self.w[sel] += np.asarray(plane)[pidx] * self.m_l[sel]

    def update(self, alpha):
        self.x = self.x + alpha * self.p
        self.r = self.r - alpha * self.w
        return self.dots()
