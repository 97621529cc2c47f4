"""FP64 reference of the per-element network used as a learned preconditioner.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The network maps an element's residual, divided by its Euclidean norm, to a
correction of the same length d = (N+1)^3, which the preconditioner scales
back by that norm.  One hidden layer of width h whose output layer reuses the
input layer's weights (tied weights), with per-unit output gains a:

    Z = X W,  H = gelu(Z),  Y = (H * a) W^T          (W: d x h, a: h)

with the tanh form of GELU, gelu(z) = z/2 (1 + tanh(sqrt(2/pi)(z + 0.044715 z^3))).
Each row is y(x) = W (a * gelu(W^T x)), the gradient of the scalar potential
sum_j a_j G(w_j . x) with G' = gelu, so its Jacobian W diag(a gelu'(W^T x)) W^T
is symmetric at every input and y(0) = 0.  A preconditioner built from it is
therefore symmetric to first order, which the short-recurrence flexible CG
needs (an untied network with the same training error lost that property
and converged more slowly than plain Jacobi).
Training minimises the mean squared error L = sum((Y - T)^2) / (B d) over a
batch of B pairs with Adam (Kingma and Ba, 2015).  The backward pass below is
the chain rule written out; it is pinned against central finite differences
of ``loss`` by the tests.
"""
from __future__ import annotations

import math

import numpy as np

_C = math.sqrt(2.0 / math.pi)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(_C * (z + 0.044715 * z ** 3)))


def gelu_grad(z):
    u = _C * (z + 0.044715 * z ** 3)
    t = np.tanh(u)
    du = _C * (1.0 + 3 * 0.044715 * z ** 2)
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * du


def init_params(d: int, h: int, seed: int):
    """Deterministic initialisation: W uniform(-1, 1)/sqrt(d), gains a = 1."""
    rng = np.random.default_rng(seed)
    return {"W": rng.uniform(-1, 1, (d, h)) / math.sqrt(d), "a": np.ones(h)}


def forward(params, X):
    Z = X @ params["W"]
    H = gelu(Z)
    Y = (H * params["a"]) @ params["W"].T
    return Y, (X, Z, H)


def loss(params, X, T):
    Y, _ = forward(params, X)
    return float(np.sum((Y - T) ** 2) / Y.size)


def backward(params, X, T):
    """Gradients of ``loss`` with respect to W (both of its uses) and a."""
    Y, (X, Z, H) = forward(params, X)
    W, a = params["W"], params["a"]
    dY = 2.0 * (Y - T) / Y.size
    G = dY @ W                      # d loss / d (H * a)
    ga = np.sum(G * H, axis=0)
    dZ = G * a * gelu_grad(Z)
    gW = X.T @ dZ + dY.T @ (H * a)  # input use + output use of W
    return {"W": gW, "a": ga}


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update in place; ``state`` holds m, v and the step count t."""
    t = state.get("t", 0) + 1
    state["t"] = t
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[:] = b1 * m + (1 - b1) * grads[k]
        v[:] = b2 * v + (1 - b2) * grads[k] ** 2
        mhat = m / (1 - b1 ** t)
        vhat = v / (1 - b2 ** t)
        params[k] = params[k] - lr * mhat / (np.sqrt(vhat) + eps)
    return params


def precondition(params, r_elems: np.ndarray):
    """Element corrections |r_e| * MLP(r_e / |r_e|) (zero where r_e = 0)."""
    nrm = np.linalg.norm(r_elems, axis=1)
    safe = np.where(nrm > 0, nrm, 1.0)
    Y, _ = forward(params, r_elems / safe[:, None])
    return Y * nrm[:, None]


def interior_mask(N: int) -> np.ndarray:
    """True on the (N-1)^3 interior nodes of an element, index (k n + j) n + i."""
    n = N + 1
    q = np.arange(n ** 3)
    i, j, k = q % n, (q // n) % n, q // (n * n)
    return (i > 0) & (i < N) & (j > 0) & (j < N) & (k > 0) & (k < N)


def element_interior_block(P, e: int) -> np.ndarray:
    """Dense block of element e's operator on its interior nodes, built by
    applying the oracle's local operator to unit vectors."""
    n3 = P.box.n ** 3
    mask = interior_mask(P.N)
    cols = np.nonzero(mask)[0]
    Ge = P.G[e:e + 1]
    A = np.zeros((len(cols), len(cols)))
    for c, q in enumerate(cols):
        u = np.zeros(n3)
        u[q] = 1.0
        A[:, c] = ax_local_element(P, Ge, u)[cols]
    return A


def ax_local_element(P, Ge, u):
    from . import ax_local
    return ax_local(P.N, P.D, Ge, u)


def interior_targets(P, r: np.ndarray, elems):
    """The learned preconditioner's training pairs for residual r (L-vector):
    X = r_e/|r_e| and T = (A_ii^-1 r_i - Dinv r_i)/|r_e| on interior nodes,
    0 on the element's boundary nodes (dense direct solves)."""
    n3 = P.box.n ** 3
    mask = interior_mask(P.N)
    X = np.zeros((len(elems), n3))
    T = np.zeros((len(elems), n3))
    for t, e in enumerate(elems):
        re = r[e * n3:(e + 1) * n3]
        nrm = np.linalg.norm(re)
        if nrm == 0:
            continue
        A = element_interior_block(P, e)
        xi = np.linalg.solve(A, re[mask] / nrm)
        X[t] = re / nrm
        T[t, mask] = xi - P.dinv[e * n3:(e + 1) * n3][mask] * re[mask] / nrm
    return X, T


def precondition_interior(params, P, r: np.ndarray) -> np.ndarray:
    """z = Dinv r + M_int (|r_e| MLP(r_e/|r_e|)) for an L-vector r."""
    n3 = P.box.n ** 3
    corr = precondition(params, r.reshape(-1, n3))
    corr = corr * interior_mask(P.N)[None, :]
    return P.dinv * r + corr.reshape(-1)
