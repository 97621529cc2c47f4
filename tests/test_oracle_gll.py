"""Pins of the oracle's GLL quadrature and derivative matrix against closed
forms, exact integration and an independently built Lagrange basis."""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gll_closed_forms.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        N, nodes, weights = (s.strip() for s in line.split("|"))
        ev = lambda s: [eval(t, {"sqrt": math.sqrt}) for t in s.split(",")]
        rows.append((int(N), np.array(ev(nodes)), np.array(ev(weights))))
    return rows


@pytest.mark.parametrize("N,xi_ref,w_ref", _golden())
def test_gll_closed_forms(N, xi_ref, w_ref):
    xi, w = oracle.gll(N)
    np.testing.assert_allclose(xi, xi_ref, rtol=0, atol=2e-16)
    np.testing.assert_allclose(w, w_ref, rtol=2e-15, atol=0)


@pytest.mark.parametrize("N", range(1, 17))
def test_gll_weights_sum_and_exactness(N):
    xi, w = oracle.gll(N)
    assert abs(w.sum() - 2.0) <= 1e-15 * N
    assert np.all(np.diff(xi) > 0)
    np.testing.assert_allclose(xi, -xi[::-1], atol=1e-16)
    # GLL with N+1 points integrates every polynomial of degree <= 2N-1 exactly
    for k in range(0, 2 * N):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, xi ** k) - exact) <= 5e-15, (N, k)
    # degree 2N is not exact: the rule gives sum_j w_j P_N(xi_j)^2 = 2/N
    # (from the weight formula) where the integral is 2/(2N+1)
    PN = np.polynomial.legendre.Legendre.basis(N)(xi)
    assert abs(np.dot(w, PN ** 2) - 2.0 / N) <= 1e-14 * N


@pytest.mark.parametrize("N", [2, 5, 7, 9, 15])
def test_gll_interior_nodes_are_zeros_of_dP(N):
    xi, _ = oracle.gll(N)
    dP = np.polynomial.legendre.Legendre.basis(N).deriv()
    assert np.max(np.abs(dP(xi[1:-1]))) < 1e-12 * N * N


@pytest.mark.parametrize("N", range(1, 16))
def test_derivative_exact_on_monomials(N):
    xi, _ = oracle.gll(N)
    D = oracle.deriv(N, xi)
    for k in range(0, N + 1):
        d = D @ xi ** k
        ref = k * xi ** (k - 1) if k > 0 else np.zeros_like(xi)
        assert np.max(np.abs(d - ref)) <= 1e-13 * N * N * max(1, k), (N, k)
    np.testing.assert_allclose(D.sum(axis=1), 0.0, atol=1e-12 * N * N)
    # centro-antisymmetry of the GLL derivative matrix
    np.testing.assert_allclose(D[::-1, ::-1], -D, atol=1e-13 * N * N)


@pytest.mark.parametrize("N", [1, 2, 4, 7, 9])
def test_derivative_against_lagrange_polynomials(N):
    """D[i,j] = l_j'(xi_i) with l_j built from its roots by numpy."""
    xi, _ = oracle.gll(N)
    D = oracle.deriv(N, xi)
    for j in range(N + 1):
        others = np.delete(xi, j)
        lj = np.poly1d(np.poly(others)) / np.prod(xi[j] - others)
        np.testing.assert_allclose(D[:, j], lj.deriv()(xi), atol=1e-11 * N * N)
