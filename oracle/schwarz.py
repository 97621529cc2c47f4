"""FP64 reference of the overlapping Schwarz preconditioner with fast
diagonalisation (the smoother of Nekbone's multigrid preconditioner, whose
routines the paper names in Section 4.1 -- h1mg_schwarz, h1mg_fdm,
h1mg_extrude, h1mg_do_fast, h1mg_tnsr3d_el -- without giving the algorithm).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

What it computes (the textbook one-level overlapping Schwarz method with
minimal overlap; Fischer, J. Comput. Phys. 133, 1997; Lynch, Rice and Thomas,
Numer. Math. 6, 1964 for the fast diagonalisation):

* subdomains: every element extended by one GLL node layer into each
  neighbour, i.e. the (n+2)^3 lattice points [ex N - 1, ex N + N + 1] x ... of
  the global GLL lattice; lattice points outside the domain or on its
  (Dirichlet) boundary carry no unknown;
* local operator: the separable approximation
  A_e = Bz (x) By (x) Ax + Bz (x) Ay (x) Bx + Az (x) By (x) Bx, with Ad and Bd the
  1D stiffness and (diagonal GLL) mass matrices assembled over the element
  and its two neighbours in direction d and restricted to the n+2 extended
  nodes, on the undeformed box (element length 1 / n_d) -- exact for an
  undeformed box;
* fast diagonalisation: Ad S = Bd S Lam (S^T Bd S = I), so
  A_e^-1 = (Sz (x) Sy (x) Sx) diag(1 / (lx + ly + lz)) (Sz (x) Sy (x) Sx)^T;
* additive combination: z = sum_e R_e^T A_e^-1 R_e r with R_e the restriction
  of the global vector to subdomain e (symmetric positive definite);
* two-level form (the coarse-grid level of the multigrid, textbook two-level
  additive Schwarz, e.g. Toselli and Widlund, Domain Decomposition Methods,
  2005, Ch. 3): z += R_0^T A_0^-1 R_0 r, with R_0^T the trilinear (Q1)
  interpolation from the interior element vertices to the GLL nodes and
  A_0 = R_0 A R_0^T the Galerkin coarse operator of the undeformed box --
  separable, Bz(x)By(x)Ax + Bz(x)Ay(x)Bx + Az(x)By(x)Bx with the 1D Galerkin
  stiffness / mass of the vertex hats (the Q1 matrices for N >= 2).

Pinned by ``tests/test_oracle_schwarz.py``: the fast diagonalisation against
a dense solve of the Kronecker operator, the single-element box (where the
preconditioner is the exact inverse and CG converges in one step),
symmetry, and the 1D operators against the element's GLL matrices; the
coarse level against the closed-form Q1 matrices, the Galerkin product of the
independently assembled fine operator, and exactness on the coarse space.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import deriv, gll


def gll_1d(N: int):
    """1D GLL stiffness and mass on [-1, 1]: K[i][j] = sum_q w_q D[q][i] D[q][j],
    M = diag(w)."""
    xi, w = gll(N)
    D = deriv(N, xi)
    K = (D.T * w) @ D
    return K, np.diag(w)


def fdm_1d(N: int, L: float, left: bool, right: bool):
    """Extended 1D operators for an element of length L with a neighbour of the
    same length on the left / right (flags), on the n+2 nodes
    [x_{-1}, x_0 .. x_N, x_{N+1}]; nodes without an unknown (outside the
    domain, or the domain's Dirichlet face) are decoupled as identity rows.
    Returns (S, lam, active): S^T B S = I, S^T A S = diag(lam)."""
    n = N + 1
    m = n + 2
    K, M = gll_1d(N)
    A = np.zeros((m, m))
    B = np.zeros((m, m))
    sk, sm = 2.0 / L, L / 2.0
    # the element: nodes 1..n of the extended grid
    A[1:n + 1, 1:n + 1] += sk * K
    B[1:n + 1, 1:n + 1] += sm * M
    if left:  # left neighbour's nodes N-1, N = extended nodes 0, 1
        A[0:2, 0:2] += sk * K[N - 1:N + 1, N - 1:N + 1]
        B[0:2, 0:2] += sm * M[N - 1:N + 1, N - 1:N + 1]
    if right:  # right neighbour's nodes 0, 1 = extended nodes n, n+1
        A[n:n + 2, n:n + 2] += sk * K[0:2, 0:2]
        B[n:n + 2, n:n + 2] += sm * M[0:2, 0:2]
    active = np.ones(m, dtype=bool)
    if not left:
        active[0] = False
        active[1] = False  # the domain's face: Dirichlet
    if not right:
        active[n + 1] = False
        active[n] = False
    A[~active, :] = 0.0
    A[:, ~active] = 0.0
    B[~active, :] = 0.0
    B[:, ~active] = 0.0
    idx = np.nonzero(~active)[0]
    A[idx, idx] = 1.0
    B[idx, idx] = 1.0
    lam, S = sla.eigh(A, B)
    return S, lam, active


def _element_fdm(N, box, ex, ey, ez):
    out = []
    for e_d, n_d in ((ex, box.nx), (ey, box.ny), (ez, box.nz)):
        out.append(fdm_1d(N, 1.0 / n_d, e_d > 0, e_d < n_d - 1))
    return out


def local_solve(fdm, rt: np.ndarray) -> np.ndarray:
    """A_e^-1 rt for an extended array rt[c][b][a] (a fastest) by fast
    diagonalisation; entries without an unknown stay zero."""
    (Sx, lx, ax), (Sy, ly, ay), (Sz, lz, az) = fdm
    act = az[:, None, None] & ay[None, :, None] & ax[None, None, :]
    r = np.where(act, rt, 0.0)
    t = np.einsum("ia,cbi->cba", Sx, r)      # apply Sx^T along a
    t = np.einsum("jb,cja->cba", Sy, t)
    t = np.einsum("kc,kba->cba", Sz, t)
    t = t / (lx[None, None, :] + ly[None, :, None] + lz[:, None, None])
    t = np.einsum("ai,cbi->cba", Sx, t)      # apply Sx along a
    t = np.einsum("bj,cja->cba", Sy, t)
    t = np.einsum("ck,kba->cba", Sz, t)
    return np.where(act, t, 0.0)


def coarse_1d(N: int, n_d: int):
    """The coarse space along one direction of n_d elements of length 1/n_d:
    R1[v][g] = the hat function of interior vertex v + 1 (v = 0..n_d-2) at
    global GLL node g (it is (1 + xi_i)/2 on element v, (1 - xi_i)/2 on element
    v + 1), and the Galerkin stiffness / mass R1 K R1^T, R1 M R1^T with K, M
    the 1D GLL stiffness / mass assembled over the n_d elements."""
    xi, _ = gll(N)
    K, M = gll_1d(N)
    L = 1.0 / n_d
    ng = n_d * N + 1
    Kf = np.zeros((ng, ng))
    Mf = np.zeros((ng, ng))
    for e in range(n_d):
        s = slice(e * N, e * N + N + 1)
        Kf[s, s] += (2.0 / L) * K
        Mf[s, s] += (L / 2.0) * M
    R1 = np.zeros((max(n_d - 1, 0), ng))
    for v in range(n_d - 1):
        for i in range(N + 1):
            R1[v, v * N + i] = (1.0 + xi[i]) / 2.0
            R1[v, (v + 1) * N + i] = (1.0 - xi[i]) / 2.0
    return R1, R1 @ Kf @ R1.T, R1 @ Mf @ R1.T


def coarse_parts(box):
    """(R1, Kc, Mc) per direction x, y, z."""
    return [coarse_1d(box.N, n_d) for n_d in (box.nx, box.ny, box.nz)]


def coarse_operator(box) -> np.ndarray:
    """A_0 = Bz(x)By(x)Ax + Bz(x)Ay(x)Bx + Az(x)By(x)Bx on the interior vertices
    ([vz][vy][vx], vx fastest), dense."""
    (_, Kx, Mx), (_, Ky, My), (_, Kz, Mz) = coarse_parts(box)
    return (np.kron(Mz, np.kron(My, Kx)) + np.kron(Mz, np.kron(Ky, Mx)) +
            np.kron(Kz, np.kron(My, Mx)))


def coarse_correction(P, r: np.ndarray) -> np.ndarray:
    """R_0^T A_0^-1 R_0 r for a continuous, masked L-vector r; the L-vector
    result (continuous, masked)."""
    box = P.box
    (Rx, _, _), (Ry, _, _), (Rz, _, _) = coarse_parts(box)
    if Rx.shape[0] == 0 or Ry.shape[0] == 0 or Rz.shape[0] == 0:
        return np.zeros_like(r)  # no interior vertex: no coarse space
    gx_n, gy_n, gz_n = box.nx * box.N + 1, box.ny * box.N + 1, box.nz * box.N + 1
    rg = P.to_global(r).reshape(gz_n, gy_n, gx_n)
    rc = np.einsum("cz,by,ax,zyx->cba", Rz, Ry, Rx, rg)
    zc = np.linalg.solve(coarse_operator(box), rc.reshape(-1)).reshape(rc.shape)
    zg = np.einsum("cz,by,ax,cba->zyx", Rz, Ry, Rx, zc)
    return P.to_local(zg.reshape(-1), masked=True)


def precondition(P, r: np.ndarray, coarse: bool = False) -> np.ndarray:
    """z = sum_e R_e^T A_e^-1 R_e r (+ R_0^T A_0^-1 R_0 r with ``coarse``) for a
    continuous, masked L-vector r (oracle.Problem P); returns the L-vector z
    (continuous, masked)."""
    box, N = P.box, P.N
    n = N + 1
    gx_n, gy_n, gz_n = box.nx * N + 1, box.ny * N + 1, box.nz * N + 1
    rg = P.to_global(r).reshape(gz_n, gy_n, gx_n)
    zg = np.zeros_like(rg)
    m = n + 2
    for ez in range(box.nz):
        for ey in range(box.ny):
            for ex in range(box.nx):
                fdm = _element_fdm(N, box, ex, ey, ez)
                x0, y0, z0 = ex * N - 1, ey * N - 1, ez * N - 1
                rt = np.zeros((m, m, m))
                xs = np.arange(x0, x0 + m)
                ys = np.arange(y0, y0 + m)
                zs = np.arange(z0, z0 + m)
                okx = (xs >= 0) & (xs < gx_n)
                oky = (ys >= 0) & (ys < gy_n)
                okz = (zs >= 0) & (zs < gz_n)
                sub = np.ix_(zs[okz], ys[oky], xs[okx])
                loc = np.ix_(np.nonzero(okz)[0], np.nonzero(oky)[0], np.nonzero(okx)[0])
                rt[loc] = rg[sub]
                zt = local_solve(fdm, rt)
                zg[sub] += zt[loc]
    z = P.to_local(zg.reshape(-1), masked=True)
    if coarse:
        z = z + coarse_correction(P, r)
    return z


def dense_local_operator(fdm) -> np.ndarray:
    """The separable extended-element operator as a dense matrix on the
    active extended nodes (for the pins)."""
    (Sx, lx, ax), (Sy, ly, ay), (Sz, lz, az) = fdm
    mats = []
    for S, lam in ((Sx, lx), (Sy, ly), (Sz, lz)):
        Binv = S @ S.T          # S S^T = B^-1
        B = np.linalg.inv(Binv)
        A = B @ S @ np.diag(lam) @ S.T @ B
        mats.append((A, B))
    (Ax, Bx), (Ay, By), (Az, Bz) = mats
    full = (np.kron(Bz, np.kron(By, Ax)) + np.kron(Bz, np.kron(Ay, Bx)) +
            np.kron(Az, np.kron(By, Bx)))
    act = (az[:, None, None] & ay[None, :, None] & ax[None, None, :]).reshape(-1)
    return full[np.ix_(act, act)], act


# --------------------------------------------------------------------------
# an intermediate p-level (a study of the multigrid's middle levels)
# --------------------------------------------------------------------------

def p_interpolation(N_c: int, N_f: int, n_el: int) -> np.ndarray:
    """Interpolation from the global GLL lattice of order N_c to that of order
    N_f along one direction of n_el elements: in each element the Lagrange
    basis of the N_c + 1 GLL points evaluated at the N_f + 1 GLL points
    (element end points shared, so continuous fields stay continuous).
    Shape (n_el N_f + 1, n_el N_c + 1)."""
    xc, _ = gll(N_c)
    xf, _ = gll(N_f)
    L = np.ones((N_f + 1, N_c + 1))
    for j in range(N_c + 1):
        for k in range(N_c + 1):
            if k != j:
                L[:, j] *= (xf - xc[k]) / (xc[j] - xc[k])
    J = np.zeros((n_el * N_f + 1, n_el * N_c + 1))
    for e in range(n_el):
        J[e * N_f:e * N_f + N_f + 1, e * N_c:e * N_c + N_c + 1] = L
    return J


def precondition_three_level(P, Pm, r: np.ndarray) -> np.ndarray:
    """Three-level additive form: the two-level preconditioner of P (order N)
    plus J S_m J^T r, S_m the one-level Schwarz preconditioner of the same
    box at the intermediate order N_m (oracle.Problem Pm), J the lattice
    interpolation from order N_m to N (p_interpolation per direction), the
    restricted residual masked on the coarse lattice's Dirichlet boundary."""
    box, bm = P.box, Pm.box
    gx, gy, gz = box.nx * box.N + 1, box.ny * box.N + 1, box.nz * box.N + 1
    Jx = p_interpolation(bm.N, box.N, box.nx)
    Jy = p_interpolation(bm.N, box.N, box.ny)
    Jz = p_interpolation(bm.N, box.N, box.nz)
    z = precondition(P, r, coarse=True)
    rg = P.to_global(r).reshape(gz, gy, gx)
    rm = np.einsum("zc,yb,xa,zyx->cba", Jz, Jy, Jx, rg)
    zm = precondition(Pm, Pm.to_local(rm.reshape(-1), masked=True), coarse=False)
    zmg = Pm.to_global(zm).reshape(rm.shape)
    zg = np.einsum("zc,yb,xa,cba->zyx", Jz, Jy, Jx, zmg)
    return z + P.to_local(zg.reshape(-1), masked=True)
