"""Pins of the oracle's box mesh: coordinates, geometric factors, numbering,
multiplicity, Dirichlet mask and CSR, against closed forms, the analytic
mapping and brute force."""
import itertools
import math

import numpy as np
import pytest

import oracle
from workloads import Box


@pytest.mark.parametrize("box", [Box(2, 2, 2, 3), Box(3, 1, 2, 4), Box(1, 1, 1, 7)])
def test_affine_geometric_factors_closed_form(box):
    """Affine box: J = hx hy hz / 8, G_rr = w w w J (2/hx)^2 etc., off-diagonals 0."""
    xi, w = oracle.gll(box.N)
    G, mass = oracle.geom(box, with_mass=True)
    n = box.n
    hx, hy, hz = 1 / box.nx, 1 / box.ny, 1 / box.nz
    J = hx * hy * hz / 8
    W3 = np.einsum("k,j,i->kji", w, w, w).reshape(-1)
    for e in range(box.E):
        np.testing.assert_allclose(G[e, 0], W3 * J * (2 / hx) ** 2, rtol=1e-12)
        np.testing.assert_allclose(G[e, 3], W3 * J * (2 / hy) ** 2, rtol=1e-12)
        np.testing.assert_allclose(G[e, 5], W3 * J * (2 / hz) ** 2, rtol=1e-12)
        for c in (1, 2, 4):
            assert np.max(np.abs(G[e, c])) < 1e-12 * np.max(G[e, 0])
        np.testing.assert_allclose(mass[e], W3 * J, rtol=1e-12)
    assert abs(mass.sum() - 1.0) < 1e-13


def _analytic_map(X, a):
    d = a * np.sin(np.pi * X[0]) * np.sin(np.pi * X[1]) * np.sin(np.pi * X[2])
    return X + d


def test_coordinates_closed_form_and_deformation():
    box = Box(2, 3, 2, 5, 0.05)
    xi, _ = oracle.gll(box.N)
    n = box.n
    a = 0.05 / 3
    for e in [0, 5, box.E - 1]:
        ex, ey, ez = e % box.nx, (e // box.nx) % box.ny, e // (box.nx * box.ny)
        X = oracle.element_coords(box, e, xi).reshape(3, n, n, n)  # [c][k][j][i]
        for (i, j, k) in [(0, 0, 0), (1, 2, 3), (n - 1, 0, n - 1)]:
            X0 = np.array([(ex + (1 + xi[i]) / 2) / box.nx, (ey + (1 + xi[j]) / 2) / box.ny,
                           (ez + (1 + xi[k]) / 2) / box.nz])
            np.testing.assert_allclose(X[:, k, j, i], _analytic_map(X0, a), atol=1e-15)


def test_deformed_jacobian_matches_analytic_map():
    """G from the interpolated map agrees with G from the exact derivative of
    the analytic map to interpolation accuracy (catches transposed indices)."""
    box = Box(2, 2, 2, 9, 0.05)
    xi, w = oracle.gll(box.N)
    n = box.n
    a = 0.05 / 2
    G = oracle.geom(box, elems=[3])[0]
    e = 3
    ex, ey, ez = e % 2, (e // 2) % 2, e // 4
    h = np.array([0.5, 0.5, 0.5])
    for (i, j, k) in [(0, 0, 0), (4, 5, 6), (9, 2, 7)]:
        X0 = np.array([(ex + (1 + xi[i]) / 2) / 2, (ey + (1 + xi[j]) / 2) / 2,
                       (ez + (1 + xi[k]) / 2) / 2])
        s = np.sin(np.pi * X0)
        c = np.cos(np.pi * X0)
        grad = a * np.pi * np.array([c[0] * s[1] * s[2], s[0] * c[1] * s[2], s[0] * s[1] * c[2]])
        dxdX = np.eye(3) + np.outer(np.ones(3), grad)
        M = dxdX * (h / 2)[None, :]          # dx/dr_a = dx/dX_a * h_a/2
        Minv = np.linalg.inv(M)
        J = np.linalg.det(M)
        Gex = w[i] * w[j] * w[k] * J * Minv @ Minv.T
        q = (k * n + j) * n + i
        got = G[:, q]
        ref = np.array([Gex[0, 0], Gex[0, 1], Gex[0, 2], Gex[1, 1], Gex[1, 2], Gex[2, 2]])
        np.testing.assert_allclose(got, ref, rtol=2e-4, atol=2e-4 * abs(ref[0]))


def test_deformed_geometry_spd_and_volume():
    box = Box(4, 4, 4, 7, 0.05)
    G, mass = oracle.geom(box, with_mass=True)
    M = np.stack([G[:, 0], G[:, 1], G[:, 2], G[:, 1], G[:, 3], G[:, 4],
                  G[:, 2], G[:, 4], G[:, 5]], axis=-1).reshape(-1, 3, 3)
    assert np.all(np.linalg.eigvalsh(M) > 0)
    assert abs(mass.sum() - 1.0) < 1e-6
    # off-diagonal factors are genuinely non-zero in the deformed case
    assert np.max(np.abs(G[:, 1])) > 1e-3 * np.max(G[:, 0])


def test_over_deformed_mesh_is_rejected():
    with pytest.raises(ValueError):
        oracle.geom(Box(1, 1, 1, 5, 2.0))


@pytest.mark.parametrize("box", [Box(2, 2, 2, 2), Box(3, 2, 1, 3), Box(1, 1, 1, 4)])
def test_numbering_brute_force(box):
    gid, mult, mask = oracle.numbering(box)
    n, N = box.n, box.N
    Gx, Gy, Gz = box.nx * N + 1, box.ny * N + 1, box.nz * N + 1
    # brute force: global node = rounded physical position on the lattice
    ref = np.zeros_like(gid)
    cnt = np.zeros(box.n_global, dtype=np.int64)
    l = 0
    for ez, ey, ex in itertools.product(range(box.nz), range(box.ny), range(box.nx)):
        for k, j, i in itertools.product(range(n), range(n), range(n)):
            g = (ex * N + i) + Gx * ((ey * N + j) + Gy * (ez * N + k))
            ref[l] = g
            cnt[g] += 1
            l += 1
    np.testing.assert_array_equal(gid, ref)
    np.testing.assert_array_equal(mult, cnt)
    assert set(np.unique(mult)) <= {1, 2, 4, 8}
    # every global node is owned by someone
    assert np.all(mult >= 1)
    # closed form of the multiplicity histogram: per direction, lattice
    # points on an interior element face count twice
    def per_dir(m):
        return np.array([1] * (m * N + 1)) + np.array(
            [1 if (g % N == 0 and 0 < g < m * N) else 0 for g in range(m * N + 1)])
    mx, my, mz = per_dir(box.nx), per_dir(box.ny), per_dir(box.nz)
    closed = np.einsum("k,j,i->kji", mz, my, mx).reshape(-1)
    np.testing.assert_array_equal(mult, closed)
    # sum of c = 1/mult over local nodes counts each global node once
    assert abs(np.sum(1.0 / mult[gid]) - box.n_global) < 1e-9
    # Dirichlet mask: zero exactly on the boundary of the lattice
    inner = (Gx - 2) * (Gy - 2) * (Gz - 2)
    assert int(mask.sum()) == inner


def test_csr_ascending_and_complete():
    box = Box(3, 2, 2, 3)
    gid, mult, _ = oracle.numbering(box)
    off, loc = oracle.csr(gid, box.n_global)
    np.testing.assert_array_equal(np.diff(off), mult)
    for g in range(box.n_global):
        row = loc[off[g]:off[g + 1]]
        assert np.all(np.diff(row) > 0)
        assert np.all(gid[row] == g)
    assert sorted(loc.tolist()) == list(range(box.n_local))
