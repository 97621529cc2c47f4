"""The refinement reading on the CPU, with the oracle's parts: an inner
Jacobi-PCG whose operator and vector updates are rounded to binary32 (t = 23,
the oracle's VPREC rounding; dots in binary64), inside FP64 iterative
refinement.  Keeping the search direction across the FP64 residual
replacement (reliable update, residual replaced every 2 decades) needs about
the FP64 PCG iteration count; restarting every inner solve (each to 1e-4)
needs more.  Both reach the FP64 residual 1e-10."""
import math

import numpy as np

import oracle
from workloads import Box, rhs_global

T32 = 23


def _r32(v):
    """Round to binary32 (for these normal-range values, the oracle's t = 23
    rounding: pinned equal in test_oracle_vprec)."""
    return np.asarray(v, dtype=np.float64).astype(np.float32).astype(np.float64)


def _refined(P, b, reliable, rtol=1e-10, drop=1e-2, inner=1e-4, maxit=5000):
    """Total inner iterations and the final FP64 relative residual."""
    bn = math.sqrt(P.glsc3(b, b))
    x = np.zeros_like(b)
    p = np.zeros_like(b)
    rtz_prev, s_prev, have_dir = 0.0, 0.0, False
    total = 0
    for _ in range(40):
        r64 = b - P.apply(x)                       # FP64 residual
        rel = math.sqrt(P.glsc3(r64, r64)) / bn
        if rel < rtol or total >= maxit:
            return total, rel
        s = math.sqrt(P.glsc3(r64, r64))
        r = _r32(r64 / s)                          # scaled to unit norm, in FP32
        tau = min(0.5, max(drop if reliable else inner, 0.5 * rtol / rel))
        d = np.zeros_like(b)                       # this step's correction (FP32)
        z = _r32(P.dinv * r)
        rtz = P.glsc3(r, z)
        if reliable and have_dir:                  # resume: p in the old scale
            c = s_prev / s
            beta = rtz / (rtz_prev * c * c)
            p = _r32(z + beta * c * p)
        else:
            p = z.copy()
        it = 0
        while True:
            w = P.apply_vprec(p, T32)
            alpha = rtz / P.glsc3(w, p)
            d = _r32(d + alpha * p)
            r = _r32(r - alpha * w)
            it += 1
            if math.sqrt(P.glsc3(r, r)) < tau or it >= maxit:
                break
            z = _r32(P.dinv * r)
            rtz_new = P.glsc3(r, z)
            p = _r32(z + (rtz_new / rtz) * p)
            rtz = rtz_new
        total += it
        x = x + s * d                              # FP64 solution update
        rtz_prev, s_prev, have_dir = rtz, s, True
    return total, rel


def test_reliable_update_keeps_the_fp64_iteration_count():
    box = Box(4, 4, 3, 5, 0.05)
    P = oracle.Problem(box)
    b = P.to_local(rhs_global(box, 6))
    _, it64, _, _ = P.pcg(b, tol=1e-10, maxit=5000)
    it_rel, rel_rel = _refined(P, b, reliable=True)
    it_res, rel_res = _refined(P, b, reliable=False)
    print(f"FP64 PCG {it64}, reliable updates {it_rel}, restarted refinement {it_res}")
    assert rel_rel < 1e-10 and rel_res < 1e-10
    assert it_rel <= 1.05 * it64
    assert it_res > it_rel


def _refined_fcg(P, b, precond, reliable, rtol=1e-10, drop=1e-2, inner=1e-4, maxit=3000):
    """The same with flexible CG (one-vector truncation): p = z - ((z, A p_prev) /
    (p_prev, A p_prev)) p_prev, which does not depend on the scale of p_prev, so
    a resumed solve keeps p and A p unchanged across the residual replacement."""
    bn = math.sqrt(P.glsc3(b, b))
    x = np.zeros_like(b)
    p = w = None
    total = 0
    for _ in range(40):
        r64 = b - P.apply(x)
        rel = math.sqrt(P.glsc3(r64, r64)) / bn
        if rel < rtol or total >= maxit:
            return total, rel
        s = math.sqrt(P.glsc3(r64, r64))
        r = _r32(r64 / s)
        tau = min(0.5, max(drop if reliable else inner, 0.5 * rtol / rel))
        d = np.zeros_like(b)
        if not reliable:
            p = w = None
        it = 0
        while True:
            z = _r32(precond(r))
            if p is None:
                p = z
            else:
                p = _r32(z - (P.glsc3(z, w) / P.glsc3(p, w)) * p)
            w = P.apply_vprec(p, T32)
            alpha = P.glsc3(r, p) / P.glsc3(w, p)
            d = _r32(d + alpha * p)
            r = _r32(r - alpha * w)
            it += 1
            if math.sqrt(P.glsc3(r, r)) < tau or it >= maxit:
                break
        total += it
        x = x + s * d
    return total, rel


def test_reliable_update_in_flexible_cg_keeps_the_fp64_iteration_count():
    from oracle import schwarz
    box = Box(4, 3, 3, 5, 0.05)
    P = oracle.Problem(box)
    b = P.to_local(rhs_global(box, 7))
    M = lambda r: schwarz.precondition(P, r)
    _, it64, _, _ = P.fcg(b, M, tol=1e-10, maxit=2000)
    it_rel, rel_rel = _refined_fcg(P, b, M, reliable=True)
    it_res, rel_res = _refined_fcg(P, b, M, reliable=False)
    print(f"FP64 flexible CG {it64}, reliable updates {it_rel}, restarted refinement {it_res}")
    assert rel_rel < 1e-10 and rel_res < 1e-10
    assert it_rel <= 1.1 * it64
    assert it_res > it_rel
