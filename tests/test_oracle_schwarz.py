"""Pins of the Schwarz / fast-diagonalisation oracle: the 1D GLL matrices
against exact integrals, the extended 1D operator against a separately
assembled three-element chain, the fast diagonalisation against a dense solve
of the Kronecker operator, the single-element box (exact inverse), symmetry,
and the iteration count against Jacobi."""
import numpy as np
import pytest

import oracle
from oracle import schwarz
from workloads import Box, rhs_global


@pytest.mark.parametrize("N", [2, 4, 7])
def test_gll_1d_matrices(N):
    K, M = schwarz.gll_1d(N)
    xi, w = oracle.gll(N)
    np.testing.assert_allclose(K, K.T, atol=1e-13)
    assert np.abs(K @ np.ones(N + 1)).max() < 1e-12
    # (K x)_i = int phi_i' dx = phi_i(1) - phi_i(-1)
    ref = np.zeros(N + 1)
    ref[0], ref[-1] = -1.0, 1.0
    np.testing.assert_allclose(K @ xi, ref, atol=1e-12)
    # exact energy of x^2: int (2x)^2 = 8/3
    assert abs(xi ** 2 @ K @ xi ** 2 - 8.0 / 3.0) < 1e-12
    assert abs(np.trace(M) - 2.0) < 1e-14


def _chain(N, L, count):
    """1D stiffness and mass of `count` elements of length L, assembled."""
    K, M = schwarz.gll_1d(N)
    nn = count * N + 1
    A = np.zeros((nn, nn))
    B = np.zeros((nn, nn))
    for e in range(count):
        s = slice(e * N, e * N + N + 1)
        A[s, s] += (2.0 / L) * K
        B[s, s] += (L / 2.0) * M
    return A, B


@pytest.mark.parametrize("N", [3, 5])
def test_extended_1d_operator_is_the_chain_window(N):
    L = 0.25
    A3, B3 = _chain(N, L, 3)
    # interior element: window from the left neighbour's node N-1 to the right
    # neighbour's node 1, Dirichlet beyond (rows / columns outside dropped)
    lo, hi = N - 1, 2 * N + 1
    S, lam, act = schwarz.fdm_1d(N, L, True, True)
    assert act.all()
    A = A3[lo:hi + 1, lo:hi + 1]
    B = B3[lo:hi + 1, lo:hi + 1]
    # B S Lam S^T B = A and S^T B S = I reconstruct the window
    np.testing.assert_allclose(S.T @ B @ S, np.eye(N + 3), atol=1e-11)
    np.testing.assert_allclose(S.T @ A @ S, np.diag(lam), atol=1e-9 * np.abs(lam).max())
    # a boundary element (no left neighbour): its face node and the node
    # beyond carry no unknown
    S, lam, act = schwarz.fdm_1d(N, L, False, True)
    assert not act[0] and not act[1] and act[2:].all()


def _kron_operator(N, box, ex, ey, ez):
    """The separable operator built from the chain windows directly."""
    mats = []
    for e_d, n_d in ((ex, box.nx), (ey, box.ny), (ez, box.nz)):
        L = 1.0 / n_d
        A3, B3 = _chain(N, L, 3)
        A = A3[N - 1:2 * N + 2, N - 1:2 * N + 2].copy()
        B = B3[N - 1:2 * N + 2, N - 1:2 * N + 2].copy()
        act = np.ones(N + 3, dtype=bool)
        if e_d == 0:
            act[:2] = False
        if e_d == n_d - 1:
            act[-2:] = False
        mats.append((A, B, act))
    (Ax, Bx, ax), (Ay, By, ay), (Az, Bz, az) = mats
    full = (np.kron(Bz, np.kron(By, Ax)) + np.kron(Bz, np.kron(Ay, Bx)) +
            np.kron(Az, np.kron(By, Bx)))
    act = (az[:, None, None] & ay[None, :, None] & ax[None, None, :]).reshape(-1)
    return full[np.ix_(act, act)], act


@pytest.mark.parametrize("pos", [(1, 1, 1), (0, 1, 2), (2, 0, 0)])
def test_fast_diagonalisation_equals_dense_solve(pos):
    N = 3
    box = Box(3, 3, 3, N, 0.0)
    fdm = schwarz._element_fdm(N, box, *pos)
    Ad, act = _kron_operator(N, box, *pos)
    rng = np.random.default_rng(1)
    m = N + 3
    rt = rng.uniform(-1, 1, (m, m, m))
    z = schwarz.local_solve(fdm, rt)
    ref = np.linalg.solve(Ad, rt.reshape(-1)[act])
    np.testing.assert_allclose(z.reshape(-1)[act], ref, atol=1e-10 * np.abs(ref).max())
    assert np.all(z.reshape(-1)[~act] == 0)


def test_single_element_box_is_the_exact_inverse():
    """One undeformed element with Dirichlet faces: the subdomain is the
    domain and the separable operator is exact, so z = A^-1 r and CG with the
    preconditioner converges in one step."""
    box = Box(1, 1, 1, 5, 0.0)
    P = oracle.Problem(box)
    b = P.to_local(rhs_global(box, 0))
    z = schwarz.precondition(P, b)
    np.testing.assert_allclose(P.apply(z), b, atol=1e-11 * np.abs(b).max())
    x, it, rel, _ = P.fcg(b, lambda r: schwarz.precondition(P, r), tol=1e-10, maxit=10)
    assert it == 1 and rel < 1e-10


def test_preconditioner_is_symmetric_and_positive():
    box = Box(3, 2, 2, 4, 0.05)
    P = oracle.Problem(box)
    u = P.to_local(rhs_global(box, 1))
    v = P.to_local(rhs_global(box, 2))
    Mu = schwarz.precondition(P, u)
    Mv = schwarz.precondition(P, v)
    a, b = P.glsc3(v, Mu), P.glsc3(u, Mv)
    assert abs(a - b) <= 1e-12 * max(abs(a), abs(b))
    assert P.glsc3(u, Mu) > 0 and P.glsc3(v, Mv) > 0


def test_fewer_iterations_than_jacobi():
    box = Box(4, 4, 4, 5, 0.05)
    P = oracle.Problem(box)
    b = P.to_local(rhs_global(box, 3))
    _, it_j, _, _ = P.pcg(b, tol=1e-8, maxit=2000)
    _, it_s, rel, _ = P.fcg(b, lambda r: schwarz.precondition(P, r), tol=1e-8, maxit=2000)
    print(f"Jacobi {it_j} iterations, Schwarz {it_s}")
    assert rel < 1e-8
    assert it_s < 0.6 * it_j


# ---- the coarse level (two-level additive Schwarz) ----

@pytest.mark.parametrize("N", [2, 3, 7])
def test_coarse_1d_matrices_are_the_q1_matrices(N):
    """Galerkin products of the vertex hats with the GLL matrices: exact
    integration of linear functions for N >= 2, i.e. the Q1 stiffness
    (1/L) tridiag(-1, 2, -1) and consistent mass (L/6) tridiag(1, 4, 1)."""
    n_d = 5
    L = 1.0 / n_d
    R1, Kc, Mc = schwarz.coarse_1d(N, n_d)
    m = n_d - 1
    T = np.diag(np.full(m, 2.0)) - np.diag(np.ones(m - 1), 1) - np.diag(np.ones(m - 1), -1)
    S = np.diag(np.full(m, 4.0)) + np.diag(np.ones(m - 1), 1) + np.diag(np.ones(m - 1), -1)
    np.testing.assert_allclose(Kc, T / L, atol=1e-11)
    np.testing.assert_allclose(Mc, S * L / 6.0, atol=1e-13)
    # the hats sum to 1 away from the boundary elements and are 0 on the boundary
    assert R1[:, 0].max() == 0.0 and R1[:, -1].max() == 0.0
    np.testing.assert_allclose(R1.sum(axis=0)[N:-N], 1.0, atol=1e-14)


def _dense_global_operator(P):
    """The assembled, masked fine operator on global vectors, column by column
    through the oracle's apply (independent of the coarse code)."""
    ng = P.box.n_global
    A = np.zeros((ng, ng))
    for j in range(ng):
        e = np.zeros(ng)
        e[j] = 1.0
        A[:, j] = P.to_global(P.apply(P.to_local(e)))
    return A


def test_coarse_operator_is_the_galerkin_product():
    box = Box(3, 3, 2, 3, 0.0)
    P = oracle.Problem(box)
    A = _dense_global_operator(P)
    (Rx, _, _), (Ry, _, _), (Rz, _, _) = schwarz.coarse_parts(box)
    R0 = np.kron(Rz, np.kron(Ry, Rx))
    G = R0 @ A @ R0.T
    A0 = schwarz.coarse_operator(box)
    np.testing.assert_allclose(A0, G, atol=1e-11 * np.abs(G).max())


def test_coarse_correction_is_exact_on_the_coarse_space():
    """For v = R_0^T c on the undeformed box, R_0^T A_0^-1 R_0 A v = v."""
    box = Box(4, 3, 3, 4, 0.0)
    P = oracle.Problem(box)
    (Rx, _, _), (Ry, _, _), (Rz, _, _) = schwarz.coarse_parts(box)
    rng = np.random.default_rng(4)
    c = rng.uniform(-1, 1, (Rz.shape[0], Ry.shape[0], Rx.shape[0]))
    vg = np.einsum("cz,by,ax,cba->zyx", Rz, Ry, Rx, c).reshape(-1)
    v = P.to_local(vg)
    back = schwarz.coarse_correction(P, P.apply(v))
    np.testing.assert_allclose(back, v, atol=1e-11 * np.abs(v).max())


def test_two_level_is_symmetric_and_positive():
    box = Box(3, 3, 2, 4, 0.05)
    P = oracle.Problem(box)
    u = P.to_local(rhs_global(box, 1))
    v = P.to_local(rhs_global(box, 2))
    Mu = schwarz.precondition(P, u, coarse=True)
    Mv = schwarz.precondition(P, v, coarse=True)
    a, b = P.glsc3(v, Mu), P.glsc3(u, Mv)
    assert abs(a - b) <= 1e-12 * max(abs(a), abs(b))
    assert P.glsc3(u, Mu) > P.glsc3(u, schwarz.precondition(P, u)) > 0


def test_two_level_iterations_grow_little_with_the_element_count():
    """One level: iterations grow with the number of subdomains per direction;
    two levels: they stay nearly flat (and below one level)."""
    its = {}
    for k in (2, 6):
        box = Box(k, k, k, 3, 0.05)
        P = oracle.Problem(box)
        b = P.to_local(rhs_global(box, 3))
        for coarse in (False, True):
            _, it, rel, _ = P.fcg(b, lambda r: schwarz.precondition(P, r, coarse=coarse),
                                  tol=1e-8, maxit=2000)
            assert rel < 1e-8
            its[(k, coarse)] = it
    print(its)
    assert its[(6, True)] < its[(6, False)]
    assert its[(6, True)] - its[(2, True)] < its[(6, False)] - its[(2, False)]


@pytest.mark.parametrize("Nc,Nf", [(1, 5), (3, 7), (4, 9)])
def test_p_interpolation_is_exact_on_the_coarse_polynomials(Nc, Nf):
    """The lattice interpolation from order Nc to Nf reproduces, element by
    element, every polynomial of degree <= Nc (so it is the identity on the
    coarse space), has rows summing to one, and keeps the element end points."""
    n_el = 3
    J = schwarz.p_interpolation(Nc, Nf, n_el)
    assert J.shape == (n_el * Nf + 1, n_el * Nc + 1)
    xc, _ = oracle.gll(Nc)
    xf, _ = oracle.gll(Nf)
    # global coordinates of both lattices on [0, n_el]
    gc = np.concatenate([e + (xc[:-1] + 1) / 2 for e in range(n_el)] + [[n_el]])
    gf = np.concatenate([e + (xf[:-1] + 1) / 2 for e in range(n_el)] + [[n_el]])
    for e in range(n_el):  # a piecewise polynomial of degree Nc, different per element
        for k in range(Nc + 1):
            f = lambda x: (x - e) ** k
            sel_c = slice(e * Nc, e * Nc + Nc + 1)
            sel_f = slice(e * Nf, e * Nf + Nf + 1)
            np.testing.assert_allclose(J[sel_f, sel_c] @ f(gc[sel_c]), f(gf[sel_f]), atol=1e-12)
    np.testing.assert_allclose(J.sum(axis=1), 1.0, atol=1e-13)
    for e in range(n_el + 1):
        assert J[e * Nf, e * Nc] == pytest.approx(1.0, abs=1e-14)


def test_three_level_is_symmetric_and_adds_the_middle_level():
    """The three-level form is symmetric on continuous vectors, and with the
    intermediate order equal to the fine one (J the identity) it is the
    two-level form plus one more one-level Schwarz term."""
    box = Box(3, 2, 2, 4, 0.05)
    P = oracle.Problem(box)
    Pm = oracle.Problem(Box(3, 2, 2, 2, 0.05))
    rng = np.random.default_rng(4)
    r = P.to_local(rng.uniform(-1, 1, box.n_global))
    s = P.to_local(rng.uniform(-1, 1, box.n_global))
    zr = schwarz.precondition_three_level(P, Pm, r)
    zs = schwarz.precondition_three_level(P, Pm, s)
    a, b = P.to_global(s) @ P.to_global(zr), P.to_global(r) @ P.to_global(zs)
    assert abs(a - b) <= 1e-12 * abs(a)
    assert P.to_global(r) @ P.to_global(zr) > 0
    same = schwarz.precondition_three_level(P, P, r)
    expect = schwarz.precondition(P, r, coarse=True) + schwarz.precondition(P, r)
    np.testing.assert_allclose(same, expect, atol=1e-12 * np.max(np.abs(expect)))
