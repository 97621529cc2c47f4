"""Pins of the emulated-precision oracle (Section 2, the VPREC backend;
Section 4.2): rounding to t mantissa bits against IEEE binary32, binary16 and
bfloat16 conversions, its error bound, and the emulated CG loop against the
binary64 loop (t = 52) and against the same loop written in binary32 (t = 23);
the Monte Carlo Arithmetic perturbation against its distribution."""
import math

import numpy as np
import pytest

import oracle
from workloads import Box, rhs_global


def _samples(rng, lo_exp, hi_exp, count):
    mant = rng.uniform(1.0, 2.0, count)
    exps = rng.integers(lo_exp, hi_exp, count)
    sign = rng.choice([-1.0, 1.0], count)
    return sign * np.ldexp(mant, exps)


def test_t52_is_the_identity_and_rounding_is_idempotent():
    rng = np.random.default_rng(0)
    for x in _samples(rng, -300, 300, 2000):
        assert oracle.vround(x, 52) == x
        for t in (3, 10, 23, 40):
            y = oracle.vround(x, t)
            assert oracle.vround(y, t) == y


def test_t23_equals_binary32_rounding():
    rng = np.random.default_rng(1)
    xs = np.concatenate([_samples(rng, -120, 120, 5000), rng.uniform(-1, 1, 2000)])
    # ties: exactly halfway between two binary32 neighbours round to the even one
    ties = [1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, -(1.0 + 2.0 ** -24), 2.0 ** 20 * (1 + 2.0 ** -24)]
    for x in list(xs) + ties:
        assert oracle.vround(x, 23) == float(np.float32(x)), x
    assert oracle.vround(1.0 + 2.0 ** -24, 23) == 1.0
    assert oracle.vround(1.0 + 3 * 2.0 ** -24, 23) == 1.0 + 2.0 ** -22


def test_t10_equals_binary16_rounding():
    rng = np.random.default_rng(2)
    xs = _samples(rng, -14, 15, 5000)
    for x in xs:
        assert oracle.vround(x, 10) == float(np.float16(x)), x


def test_t7_equals_bfloat16_rounding():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    xs = _samples(rng, -100, 100, 3000)
    ref = torch.from_numpy(xs).to(torch.bfloat16).to(torch.float64).numpy()
    for x, y in zip(xs, ref):
        assert oracle.vround(x, 7) == y, x


def test_relative_error_bound():
    rng = np.random.default_rng(4)
    for x in _samples(rng, -200, 200, 3000):
        t = int(rng.integers(1, 52))
        assert abs(oracle.vround(x, t) - x) <= 2.0 ** -(t + 1) * abs(x)


def test_cg_t52_is_the_binary64_loop_bit_for_bit():
    box = Box(2, 2, 1, 4, 0.05)
    P = oracle.Problem(box)
    b = P.to_local(rhs_global(box, 0))
    x_ref, it, _, hist_ref = P.pcg(b, tol=0.0, maxit=25, precond="none", history=True)
    x, hist = P.cg_vprec(b, 25, 52)
    assert it == 25
    assert np.array_equal(hist, hist_ref)
    assert np.array_equal(x, x_ref)


def _cg_binary32(P, b, iters):
    """The oracle's CG loop written directly in binary32 (numpy float32
    element-wise operations; sums in the loop's sequential order)."""
    f = np.float32
    n = P.box.n
    D = P.D.astype(f)
    G = P.G.astype(f)
    c = P.c.astype(f)
    gid = P.gid
    mask = P.mask

    def glsc3(a, bb, cc):
        s = f(0.0)
        for l in range(a.size):
            s = f(s + f(f(a[l] * bb[l]) * cc[l]))
        return s

    def apply(u):
        E = P.box.E
        ue = u.reshape(E, n, n, n)  # [e][k][j][i]
        ur = np.zeros_like(ue)
        us = np.zeros_like(ue)
        ut = np.zeros_like(ue)
        for l in range(n):
            ur = ur + D[None, None, None, :, l] * ue[:, :, :, l][:, :, :, None]
            us = us + D[None, None, :, l, None] * ue[:, :, l, :][:, :, None, :]
            ut = ut + D[None, :, l, None, None] * ue[:, l, :, :][:, None, :, :]
        g = G.reshape(E, 6, n, n, n)
        wr = (g[:, 0] * ur + g[:, 1] * us) + g[:, 2] * ut
        ws = (g[:, 1] * ur + g[:, 3] * us) + g[:, 4] * ut
        wt = (g[:, 2] * ur + g[:, 4] * us) + g[:, 5] * ut
        s = np.zeros_like(ue)
        for l in range(n):
            s = s + D[None, None, None, l, :] * wr[:, :, :, l][:, :, :, None]
        for l in range(n):
            s = s + D[None, None, l, :, None] * ws[:, :, l, :][:, :, None, :]
        for l in range(n):
            s = s + D[None, l, :, None, None] * wt[:, l, :, :][:, None, :, :]
        w = s.reshape(-1)
        work = np.zeros(P.box.n_global, dtype=f)
        for l in range(w.size):
            work[gid[l]] = f(work[gid[l]] + w[l])
        return np.where(mask[gid] > 0, work[gid], f(0.0)).astype(f)

    bnorm = math.sqrt(P.glsc3(b.astype(np.float64), b.astype(np.float64)))
    x = np.zeros(b.size, dtype=f)
    r = b.astype(f).copy()
    p = np.zeros_like(r)
    rtz1 = f(1.0)
    hist = []
    for it in range(1, iters + 1):
        z = r.copy()
        rtz2 = rtz1
        rtz1 = glsc3(r, c, z)
        beta = f(0.0) if it == 1 else f(rtz1 / rtz2)
        p = (beta * p + z).astype(f)
        w = apply(p)
        pap = glsc3(w, c, p)
        alpha = f(rtz1 / pap)
        x = (x + alpha * p).astype(f)
        r = (r - alpha * w).astype(f)
        rtr = glsc3(r, c, r)
        hist.append(float(f(math.sqrt(float(rtr)) / bnorm)))
    return x, np.array(hist)


def test_cg_t23_matches_the_same_loop_in_binary32():
    """With binary32 data, rounding every binary64 result to 23 bits is
    binary32 arithmetic (products of two binary32 values are exact in
    binary64; a sum or quotient differs only if binary64 rounding lands on a
    binary32 tie).  The residual histories agree to 1e-6 relative."""
    box = Box(2, 1, 1, 3, 0.05)
    P = oracle.Problem(box)
    # binary32 data on both sides
    P._Df[:] = P._Df.astype(np.float32)
    P._Gf[:] = P._Gf.astype(np.float32)
    P.D[:] = P._Df.reshape(P.D.shape)
    P.G[:] = P._Gf.reshape(P.G.shape)
    b = P.to_local(rhs_global(box, 1)).astype(np.float32).astype(np.float64)
    iters = 12
    x, hist = P.cg_vprec(b, iters, 23)
    x32, hist32 = _cg_binary32(P, b, iters)
    np.testing.assert_allclose(hist, hist32, rtol=1e-6)
    np.testing.assert_allclose(x, x32.astype(np.float64), rtol=1e-5,
                               atol=1e-6 * np.abs(x).max())


def test_cg_residual_floor_falls_with_precision():
    """Fewer mantissa bits, higher stagnation level: after 60 iterations the
    loop's relative residual at t = 8 is above that at t = 23, which is above
    that at t = 52."""
    box = Box(2, 2, 2, 5, 0.05)
    P = oracle.Problem(box)
    b = P.to_local(rhs_global(box, 2))
    finals = {}
    for t in (8, 23, 52):
        x, hist = P.cg_vprec(b, 60, t)
        finals[t] = P.true_relres(b, x)
    assert finals[8] > finals[23] > finals[52]


def test_inexact_is_unbiased_and_bounded():
    """inexact(x) = x + 2^(e_x - t) xi, xi uniform on (-1/2, 1/2), e_x the
    exponent with 2^(e_x - 1) <= |x| < 2^e_x: every value within half a unit
    of 2^(e_x - t) of x, mean x, variance 2^(2(e_x - t)) / 12."""
    for x, t in ((1.5, 10), (-3.0e-5, 20), (7.0e8, 23)):
        e = math.frexp(x)[1]
        unit = 2.0 ** (e - t)
        state = 12345
        vals = []
        for _ in range(20000):
            v, state = oracle.inexact(x, t, state)
            vals.append(v)
        vals = np.array(vals)
        assert np.all(np.abs(vals - x) <= 0.5 * unit)
        assert abs(vals.mean() - x) <= 4 * unit / math.sqrt(12 * vals.size)
        assert abs(vals.var() / (unit ** 2 / 12) - 1.0) < 0.05
    assert oracle.inexact(0.0, 10, 1)[0] == 0.0


def test_mca_runs_are_reproducible_and_close_to_binary64_at_t52():
    box = Box(2, 2, 1, 4, 0.05)
    P = oracle.Problem(box)
    b = P.to_local(rhs_global(box, 6))
    _, h64 = P.cg_vprec(b, 20, 52)
    for mode in ("rr", "mca"):
        _, h1 = P.cg_mca(b, 20, 52, mode, seed=7)
        _, h2 = P.cg_mca(b, 20, 52, mode, seed=7)
        _, h3 = P.cg_mca(b, 20, 52, mode, seed=8)
        assert np.array_equal(h1, h2)
        assert not np.array_equal(h1, h3)
        np.testing.assert_allclose(h1, h64, rtol=1e-9)
