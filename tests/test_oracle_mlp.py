"""Pins of the network oracle: backward pass against central finite
differences of the loss, GELU against its closed form, the symmetric
Jacobian of the tied network against finite differences of the forward
pass, Adam against a hand-computed first step."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_gelu_closed_form_and_derivative():
    z = np.linspace(-4, 4, 81)
    ref = 0.5 * z * (1 + np.tanh(math.sqrt(2 / math.pi) * (z + 0.044715 * z ** 3)))
    np.testing.assert_allclose(mlp.gelu(z), ref, rtol=0, atol=0)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, rtol=1e-8, atol=1e-9)
    assert abs(mlp.gelu(np.array([0.0]))[0]) == 0.0
    assert abs(mlp.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15


@pytest.mark.parametrize("shape", [(8, 4, 5), (27, 6, 3)])
def test_backward_matches_finite_differences(shape):
    d, h, B = shape
    p = mlp.init_params(d, h, seed=3)
    rng = np.random.default_rng(4)
    p["W"] = p["W"] * 3.0  # pre-activations of order one: GELU far from linear
    p["a"] = rng.uniform(-1.5, 1.5, h)
    X = rng.uniform(-1, 1, (B, d))
    T = rng.uniform(-1, 1, (B, d))
    g = mlp.backward(p, X, T)
    eps = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp = mlp.loss(p, X, T)
            flat[idx] = old - eps
            lm = mlp.loss(p, X, T)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            got = g[k].reshape(-1)[idx]
            assert abs(got - fd) <= 1e-7 * max(1.0, abs(fd)) + 1e-10, (k, idx, got, fd)


def test_tied_network_jacobian_is_symmetric_and_zero_maps_to_zero():
    """y(x) = W (a * gelu(W^T x)): central differences of the forward pass
    give a symmetric Jacobian at random points, equal to
    W diag(a gelu'(W^T x)) W^T; an untied network fails the same check."""
    d, h = 12, 5
    rng = np.random.default_rng(7)
    p = {"W": rng.normal(size=(d, h)), "a": rng.uniform(-2, 2, h)}
    assert np.all(mlp.forward(p, np.zeros((1, d)))[0] == 0.0)
    eps = 1e-6
    for _ in range(3):
        x = rng.uniform(-1, 1, d)
        J = np.zeros((d, d))
        for q in range(d):
            e = np.zeros(d)
            e[q] = eps
            J[:, q] = (mlp.forward(p, (x + e)[None])[0][0] - mlp.forward(p, (x - e)[None])[0][0]) / (2 * eps)
        np.testing.assert_allclose(J, J.T, atol=1e-7 * np.abs(J).max())
        ref = p["W"] @ np.diag(p["a"] * mlp.gelu_grad(p["W"].T @ x)) @ p["W"].T
        np.testing.assert_allclose(J, ref, atol=1e-7 * np.abs(J).max())
    # the check has teeth: with separate output weights the Jacobian is not symmetric
    W2 = rng.normal(size=(h, d))
    x = rng.uniform(-1, 1, d)
    Ju = W2.T @ np.diag(mlp.gelu_grad(p["W"].T @ x)) @ p["W"].T
    assert np.abs(Ju - Ju.T).max() > 1e-2 * np.abs(Ju).max()


def test_adam_first_step_is_lr_times_sign():
    p = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -0.25, 0.0])}
    st = {}
    mlp.adam_step(p, g, st, lr=0.1)
    # first step: mhat = g, vhat = g^2 -> update = lr * g / (|g| + eps)
    np.testing.assert_allclose(p["w"], [1.0 - 0.1, -2.0 + 0.1, 3.0], atol=1e-9)


def test_training_reduces_loss_on_a_linear_map():
    """The tied network fits a symmetric linear map (the form its Jacobian has)."""
    rng = np.random.default_rng(0)
    d, h = 16, 16
    A = rng.normal(size=(d, d)) / 4
    A = 0.5 * (A + A.T)
    X = rng.normal(size=(256, d))
    T = X @ A
    p = mlp.init_params(d, h, seed=1)
    st = {}
    l0 = mlp.loss(p, X, T)
    for _ in range(1000):
        mlp.adam_step(p, mlp.backward(p, X, T), st, lr=3e-3)
    assert mlp.loss(p, X, T) < 0.5 * l0


def test_interior_targets_solve_the_interior_block():
    """The learned preconditioner's targets: the dense interior block equals
    the independently assembled element matrix restricted to the interior,
    and T + Dinv r solves it."""
    import oracle
    from test_oracle_operator import _dense_element_matrix
    from workloads import Box, rhs_global
    box = Box(2, 2, 1, 4, 0.05)
    P = oracle.Problem(box)
    mask = mlp.interior_mask(box.N)
    assert mask.sum() == (box.N - 1) ** 3
    for e in (0, 3):
        A = mlp.element_interior_block(P, e)
        ref = _dense_element_matrix(P.D, P.G[e])[np.ix_(mask, mask)]
        np.testing.assert_allclose(A, ref, atol=1e-13 * np.abs(ref).max())
    r = P.to_local(rhs_global(box, 5))
    X, T = mlp.interior_targets(P, r, [0, 3])
    n3 = box.n ** 3
    for t, e in enumerate((0, 3)):
        re = r[e * n3:(e + 1) * n3]
        nrm = np.linalg.norm(re)
        np.testing.assert_allclose(X[t], re / nrm, rtol=1e-15)
        A = mlp.element_interior_block(P, e)
        xi = T[t][mask] + P.dinv[e * n3:(e + 1) * n3][mask] * re[mask] / nrm
        np.testing.assert_allclose(A @ xi, re[mask] / nrm, atol=1e-12)
        assert np.all(T[t][~mask] == 0)
