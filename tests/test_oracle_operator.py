"""Pins of the oracle's operator, gather-scatter, Jacobi diagonal and CG:
an independently assembled dense element matrix, the energy identity,
the null space, dense assembly with Cholesky and a direct solve, and a
manufactured solution with spectral convergence."""
import math

import numpy as np
import pytest

import oracle
from workloads import Box, rhs_global


def _grad_matrices(D):
    """Reference-direction derivative matrices on the n^3 tensor basis
    (index (k*n + j)*n + i): d/dr = I (x) I (x) D etc."""
    n = D.shape[0]
    I = np.eye(n)
    Dr = np.kron(I, np.kron(I, D))
    Ds = np.kron(I, np.kron(D, I))
    Dt = np.kron(D, np.kron(I, I))
    return Dr, Ds, Dt


def _dense_element_matrix(D, Ge):
    """A_e[p, p'] = sum_q sum_ab G_ab(q) d_a phi_p(q) d_b phi_p'(q)."""
    Dr, Ds, Dt = _grad_matrices(D)
    grads = [Dr, Ds, Dt]
    idx = {(0, 0): 0, (0, 1): 1, (0, 2): 2, (1, 1): 3, (1, 2): 4, (2, 2): 5}
    A = np.zeros((Dr.shape[0], Dr.shape[0]))
    for a in range(3):
        for b in range(3):
            g = Ge[idx[(min(a, b), max(a, b))]]
            A += grads[a].T @ (g[:, None] * grads[b])
    return A


@pytest.mark.parametrize("box", [Box(1, 1, 1, 3, 0.0), Box(2, 1, 1, 4, 0.05),
                                 Box(2, 2, 2, 5, 0.05)])
def test_ax_local_equals_dense_element_matrix(box):
    xi, _ = oracle.gll(box.N)
    D = oracle.deriv(box.N, xi)
    G = oracle.geom(box)
    rng = np.random.default_rng(1)
    u = rng.uniform(-1, 1, box.n_local)
    w = oracle.ax_local(box.N, D, G, u)
    n3 = box.n ** 3
    for e in range(box.E):
        A = _dense_element_matrix(D, G[e])
        ref = A @ u[e * n3:(e + 1) * n3]
        np.testing.assert_allclose(w[e * n3:(e + 1) * n3], ref,
                                   atol=1e-13 * np.abs(A).max() * np.abs(u).max() * n3 ** 0.5)
        # symmetric, and constants are in the null space
        np.testing.assert_allclose(A, A.T, atol=1e-13 * np.abs(A).max())
        assert np.max(np.abs(A @ np.ones(n3))) < 1e-12 * np.abs(A).max()
        # diagonal of the local operator
        dl = oracle.diag_local(box.N, D, G[e:e + 1])
        np.testing.assert_allclose(dl, np.diag(A), rtol=1e-13)


def test_energy_identity_affine():
    """u^T A_e u = integral over the element of |grad u|^2 for a polynomial u
    of degree <= N-1 per direction (GLL quadrature is exact there)."""
    box = Box(1, 1, 1, 5, 0.0)
    N = box.N
    xi, _ = oracle.gll(N)
    D = oracle.deriv(N, xi)
    G = oracle.geom(box)
    rng = np.random.default_rng(7)
    C = rng.uniform(-1, 1, (N, N, N))  # coefficients of x^a y^b z^c, a,b,c < N
    # element = unit cube [0,1]^3; reference r -> x = (1+r)/2
    X = (1 + xi) / 2
    # careful: einsum index order: C[a (x), b (y), c (z)]; node (k=z, j=y, i=x)
    u = np.einsum("abc,ia,jb,kc->kji", C, X[:, None] ** np.arange(N), X[:, None] ** np.arange(N),
                  X[:, None] ** np.arange(N)).reshape(-1)
    w = oracle.ax_local(N, D, G, u)
    energy = float(u @ w)

    # exact integral of |grad u|^2 over [0,1]^3 by polynomial algebra
    def integ(a, b, c):
        return 1.0 / ((a + 1) * (b + 1) * (c + 1))
    ex = 0.0
    idx = np.arange(N)
    for a1 in idx:
        for b1 in idx:
            for c1 in idx:
                for a2 in idx:
                    for b2 in idx:
                        for c2 in idx:
                            cc = C[a1, b1, c1] * C[a2, b2, c2]
                            t = 0.0
                            if a1 > 0 and a2 > 0:
                                t += a1 * a2 * integ(a1 + a2 - 2, b1 + b2, c1 + c2)
                            if b1 > 0 and b2 > 0:
                                t += b1 * b2 * integ(a1 + a2, b1 + b2 - 2, c1 + c2)
                            if c1 > 0 and c2 > 0:
                                t += c1 * c2 * integ(a1 + a2, b1 + b2, c1 + c2 - 2)
                            ex += cc * t
    assert abs(energy - ex) <= 1e-12 * abs(ex)


def _assembled_dense(P):
    """Dense assembled operator on the interior (unmasked) global nodes by
    applying the oracle operator to unit vectors."""
    box = P.box
    free = np.nonzero(P.mask)[0]
    A = np.zeros((len(free), len(free)))
    for col, g in enumerate(free):
        eg = np.zeros(box.n_global)
        eg[g] = 1.0
        wL = P.apply(P.to_local(eg))
        A[:, col] = P.to_global(wL)[free]
    return A, free


@pytest.mark.parametrize("box", [Box(1, 1, 1, 5, 0.0), Box(2, 1, 1, 4, 0.05),
                                 Box(2, 2, 2, 3, 0.05)])
def test_assembled_operator_spd_and_direct_solve(box):
    P = oracle.Problem(box)
    A, free = _assembled_dense(P)
    nrm = np.abs(A).max()
    np.testing.assert_allclose(A, A.T, atol=1e-13 * nrm)
    L = np.linalg.cholesky(A)  # raises unless SPD
    assert np.all(np.diag(L) > 0)
    # Jacobi diagonal equals the diagonal of the assembled matrix
    np.testing.assert_allclose(P.to_global(P.diag)[free], np.diag(A), rtol=1e-13)
    # direct solve vs PCG
    bg = rhs_global(box, 3)
    b = P.to_local(bg)
    x, it, rel, _ = P.pcg(b, tol=1e-14, maxit=2000)
    xd = np.linalg.solve(A, bg[free])
    xg = P.to_global(x)[free]
    assert np.linalg.norm(xg - xd) <= 1e-11 * np.linalg.norm(xd)
    # FCG with the (linear) Jacobi preconditioner reproduces the PCG iterates
    for k in (5, 12):
        xp, _, _, _ = P.pcg(b, tol=0.0, maxit=k)
        xf, _, _, _ = P.fcg(b, lambda r: P.dinv * r, tol=0.0, maxit=k)
        assert np.linalg.norm(xp - xf) <= 1e-12 * np.linalg.norm(xp)


@pytest.mark.parametrize("box", [Box(2, 2, 1, 5, 0.05), Box(2, 2, 2, 3, 0.05)])
def test_flexible_cg_with_a_nonlinear_preconditioner(box):
    """Flexible CG with one-vector truncation (Notay 2000), driven by a
    nonlinear preconditioner, keeps at every step what holds for any
    preconditioner: the new residual is orthogonal to the last direction
    (exact line search), consecutive directions are A-conjugate (the choice
    of beta), so the A-norm of the error never grows; and it converges to
    the dense direct solution.  The iterate after k steps comes from a run
    stopped there (the iteration is deterministic), the direction of step k
    is x_k - x_(k-1), and no quantity is taken from the routine's internals."""
    P = oracle.Problem(box)
    A, free = _assembled_dense(P)
    bg = rhs_global(box, 5)
    b = P.to_local(bg)
    xg = np.zeros(box.n_global)
    xg[free] = np.linalg.solve(A, bg[free])
    xstar = P.to_local(xg)

    def B(r):  # pointwise in a continuous, masked r: continuous and masked
        s = math.sqrt(P.glsc3(r, r) / max(len(free), 1)) or 1.0
        return P.dinv * (r + 0.5 * s * np.tanh(r / s))

    def inner_a(u, v):
        return P.glsc3(u, P.apply(v))

    K = 14
    X = [np.zeros_like(b)] + [P.fcg(b, B, tol=0.0, maxit=k)[0] for k in range(1, K + 1)]
    err = [inner_a(xstar - x, xstar - x) for x in X]
    for k in range(1, K + 1):
        d = X[k] - X[k - 1]
        r = b - P.apply(X[k])
        assert abs(P.glsc3(r, d)) <= 1e-8 * math.sqrt(P.glsc3(r, r) * P.glsc3(d, d)), k
        assert err[k] <= err[k - 1] * (1 + 1e-12), k
        if k >= 2:
            dp = X[k - 1] - X[k - 2]
            assert abs(inner_a(d, dp)) <= 1e-8 * math.sqrt(inner_a(d, d) * inner_a(dp, dp)), k
    assert err[K] < 1e-3 * err[0]
    # the preconditioner is not a linear one in disguise: the iterates leave PCG's
    xp, _, _, _ = P.pcg(b, tol=0.0, maxit=5)
    assert np.linalg.norm(X[5] - xp) > 1e-4 * np.linalg.norm(xp)
    x, _, rel, _ = P.fcg(b, B, tol=1e-12, maxit=500)
    assert rel < 1e-12
    assert np.linalg.norm(x - xstar) <= 1e-9 * np.linalg.norm(xstar)


def test_linear_function_annihilated_at_interior_nodes():
    box = Box(2, 2, 1, 4, 0.0)
    P = oracle.Problem(box)
    Gx, Gy, Gz = box.nx * box.N + 1, box.ny * box.N + 1, box.nz * box.N + 1
    # lattice coordinates of the global nodes on the affine mesh
    xi, _ = oracle.gll(box.N)
    def coord(m, G):
        out = []
        for g in range(G):
            e, i = divmod(g, box.N)
            if e == m:
                e, i = m - 1, box.N
            out.append((e + (1 + xi[i]) / 2) / m)
        return np.array(out)
    cx, cy, cz = coord(box.nx, Gx), coord(box.ny, Gy), coord(box.nz, Gz)
    ug = (0.3 + 1.7 * cx[None, None, :] - 0.4 * cy[None, :, None]
          + 2.2 * cz[:, None, None]).reshape(-1)
    w = P.dssum(P.ax_local(P.to_local(ug, masked=False)), masked=False)
    wg = P.to_global(w)
    interior = P.mask.astype(bool)
    assert np.max(np.abs(wg[interior])) < 1e-12 * np.max(np.abs(w))


def test_dssum_multiplicity_and_idempotence():
    box = Box(3, 2, 2, 3)
    P = oracle.Problem(box)
    ones = np.ones(box.n_local)
    np.testing.assert_array_equal(P.dssum(ones, masked=False), P.mult[P.gid].astype(float))
    rng = np.random.default_rng(0)
    v = rng.uniform(-1, 1, box.n_local)
    s = P.dssum(v, masked=False)
    np.testing.assert_allclose(P.dssum(P.c * s, masked=False), s, rtol=1e-14)
    # masked copies are zero, unmasked copies of one global node agree
    sm = P.dssum(v)
    assert np.all(sm[P.mask[P.gid] == 0] == 0)
    off, loc = oracle.csr(P.gid, box.n_global)
    for g in range(0, box.n_global, 7):
        row = loc[off[g]:off[g + 1]]
        assert np.all(sm[row] == sm[row[0]])
        if P.mask[g]:
            ref = 0.0
            for l in row:
                ref += v[l]
            assert sm[row[0]] == ref  # ascending-order sum, bit-exact


def test_pcg_error_decreases_in_energy_norm():
    box = Box(2, 2, 2, 4, 0.05)
    P = oracle.Problem(box)
    b = P.to_local(rhs_global(box, 11))
    xs, _, _, _ = P.pcg(b, tol=1e-15, maxit=3000)
    prev = math.inf
    for k in range(1, 40, 3):
        xk, _, _, _ = P.pcg(b, tol=0.0, maxit=k)
        e = xs - xk
        en = P.glsc3(e, P.apply(e))
        assert en < prev * (1 + 1e-12)
        prev = en


@pytest.mark.parametrize("precond", ["jacobi", "none"])
def test_pcg_reaches_tolerance(precond):
    box = Box(2, 2, 2, 7, 0.0)
    P = oracle.Problem(box)
    b = P.to_local(rhs_global(box, 0))
    x, it, rel, hist = P.pcg(b, tol=1e-10, maxit=1000, precond=precond, history=True)
    assert rel < 1e-10 and it < 1000
    assert abs(P.true_relres(b, x) - rel) < 1e-12


def test_manufactured_solution_spectral_convergence():
    """-lap u = f with u = sin(pi x) sin(pi y) sin(pi z), f = 3 pi^2 u; the
    weak right-hand side is the dssum of the mass-weighted f.  The nodal
    error decays spectrally in N on a deformed mesh."""
    errs = []
    for N in (3, 5, 7):
        box = Box(2, 2, 2, N, 0.05)
        P = oracle.Problem(box)
        xs = np.zeros((box.E, 3, box.n ** 3))
        for e in range(box.E):
            xs[e] = oracle.element_coords(box, e, P.xi)
        X, Y, Z = xs[:, 0].reshape(-1), xs[:, 1].reshape(-1), xs[:, 2].reshape(-1)
        u = np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)
        f = 3 * np.pi ** 2 * u
        _, mass = oracle.geom(box, with_mass=True)
        b = P.dssum(mass.reshape(-1) * f)
        x, it, rel, _ = P.pcg(b, tol=1e-13, maxit=5000)
        errs.append(np.max(np.abs(x - u * P.mask[P.gid])))
    assert errs[0] > 10 * errs[1] > 100 * errs[2]
    assert errs[2] < 1e-4
