"""FP64 CPU oracle of the spectral-element Poisson solve (test infrastructure).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the CUDA library and
its Python binding never do.  It shares no code with them; the only common
module is ``workloads`` (seeded inputs, no method arithmetic).

What it computes (the paper, Section 4.1 and Table 1, names the CG kernels
and their order but gives no discretisation formula, so each function follows
the textbook spectral-element definition, cited at its C implementation in
``nb_oracle.c``):

* GLL nodes/weights and the derivative matrix (``gll``, ``deriv``)
* coordinates of the deformed box and geometric factors (``geom``)
* global numbering, multiplicity, Dirichlet mask, CSR of copies
* the local operator ``ax`` and its diagonal, ``dssum`` + mask, ``glsc3``
* Jacobi-PCG in Table 1 order (``Problem.pcg``; ``Problem.pcg_par`` the same
  on all host cores) and flexible CG
  (``Problem.fcg``, Notay 2000) with a user-supplied preconditioner.
* emulated reduced precision (Section 2, the VPREC backend; Section 4.2):
  ``vround`` rounds a binary64 value to t mantissa bits, and
  ``Problem.apply_vprec`` / ``Problem.cg_vprec`` run the operator and the CG
  loop with every arithmetic operation so rounded; ``inexact`` and
  ``Problem.cg_mca`` do the same with Monte Carlo Arithmetic (the MCA
  backend's random-rounding and full modes).

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, exactness properties, an independently assembled dense
matrix with a direct solve, or brute force; none is "parity unpinned".  The
flexible CG is pinned by its reduction to PCG for a linear preconditioner
and, for a nonlinear one, by the properties every step keeps (residual
orthogonal to the last direction, consecutive directions A-conjugate, A-norm
error not growing) and its limit, the dense direct solution.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from .build import build_oracle

_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


class _Op(C.Structure):
    _fields_ = [("E", C.c_longlong), ("N", C.c_int), ("nL", C.c_longlong),
                ("nG", C.c_longlong), ("D", C.c_void_p), ("G", C.c_void_p),
                ("gid", C.c_void_p), ("mask", C.c_void_p), ("c", C.c_void_p),
                ("dinv", C.c_void_p), ("work", C.c_void_p)]


def lib():
    """Load (building if needed) the C oracle.  NBO_LIB, if set, names another
    build of it (the mutation test's planted copies)."""
    global _lib
    if _lib is None:
        L = C.CDLL(os.environ.get("NBO_LIB") or build_oracle())
        L.nbo_legendre.restype = C.c_double
        L.nbo_legendre.argtypes = [C.c_int, C.c_double]
        L.nbo_gll.restype = C.c_int
        L.nbo_gll.argtypes = [C.c_int, _dp, _dp]
        L.nbo_deriv.restype = None
        L.nbo_deriv.argtypes = [C.c_int, _dp, _dp]
        L.nbo_element_coords.restype = None
        L.nbo_element_coords.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                         _dp, C.c_longlong, _dp]
        L.nbo_geom.restype = C.c_longlong
        L.nbo_geom.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, _ip,
                               C.c_longlong, _dp, C.c_void_p]
        L.nbo_numbering.restype = None
        L.nbo_numbering.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _ip, _i32p, _u8p]
        L.nbo_csr.restype = None
        L.nbo_csr.argtypes = [C.c_longlong, C.c_longlong, _ip, _ip, _ip]
        L.nbo_ax_local.restype = None
        L.nbo_ax_local.argtypes = [C.c_longlong, C.c_int, _dp, _dp, _dp, _dp]
        L.nbo_diag_local.restype = None
        L.nbo_diag_local.argtypes = [C.c_longlong, C.c_int, _dp, _dp, _dp]
        L.nbo_dssum.restype = None
        L.nbo_dssum.argtypes = [C.c_longlong, C.c_longlong, _ip, C.c_void_p, _dp, _dp]
        L.nbo_glsc3.restype = C.c_double
        L.nbo_glsc3.argtypes = [_dp, _dp, _dp, C.c_longlong]
        L.nbo_apply.restype = None
        L.nbo_apply.argtypes = [C.POINTER(_Op), _dp, _dp]
        L.nbo_pcg.restype = C.c_int
        L.nbo_pcg.argtypes = [C.POINTER(_Op), _dp, _dp, C.c_int, C.c_double, C.c_int,
                              C.c_void_p, C.POINTER(C.c_double)]
        L.nbo_threads.restype = C.c_int
        L.nbo_threads.argtypes = [C.c_int]
        L.nbo_pcg_par.restype = C.c_int
        L.nbo_pcg_par.argtypes = [C.POINTER(_Op), _ip, _ip, _dp, _dp, C.c_int, C.c_double,
                                  C.c_int, C.c_void_p, C.POINTER(C.c_double)]
        L.nbo_vround.restype = C.c_double
        L.nbo_vround.argtypes = [C.c_double, C.c_int]
        L.nbo_apply_vprec.restype = None
        L.nbo_apply_vprec.argtypes = [C.POINTER(_Op), C.c_int, _dp, _dp]
        L.nbo_glsc3_vprec.restype = C.c_double
        L.nbo_glsc3_vprec.argtypes = [_dp, _dp, _dp, C.c_longlong, C.c_int]
        L.nbo_cg_vprec.restype = C.c_double
        L.nbo_cg_vprec.argtypes = [C.POINTER(_Op), _dp, _dp, C.c_int, C.c_int, C.c_int,
                                   C.c_void_p]
        L.nbo_cg_emu.restype = C.c_double
        L.nbo_cg_emu.argtypes = [C.POINTER(_Op), _dp, _dp, C.c_int, C.c_int, C.c_int,
                                 C.c_uint64, C.c_int, C.c_void_p]
        L.nbo_inexact.restype = C.c_double
        L.nbo_inexact.argtypes = [C.c_double, C.c_int, C.POINTER(C.c_uint64)]
        _lib = L
    return _lib


# --------------------------------------------------------------------------
# element-level building blocks
# --------------------------------------------------------------------------

def legendre(N: int, x: float) -> float:
    return lib().nbo_legendre(N, float(x))


def gll(N: int):
    """GLL nodes (ascending) and weights of order N."""
    xi = np.zeros(N + 1)
    w = np.zeros(N + 1)
    if lib().nbo_gll(N, xi, w) != 0:
        raise ValueError("N must be >= 1")
    return xi, w


def deriv(N: int, xi=None) -> np.ndarray:
    """D[i, j] = l_j'(xi_i) of the GLL Lagrange basis."""
    if xi is None:
        xi, _ = gll(N)
    D = np.zeros((N + 1) * (N + 1))
    lib().nbo_deriv(N, np.ascontiguousarray(xi, dtype=np.float64), D)
    return D.reshape(N + 1, N + 1)


def element_coords(box, e: int, xi=None) -> np.ndarray:
    """Nodal coordinates X[3][n^3] of element e of the (deformed) box."""
    if xi is None:
        xi, _ = gll(box.N)
    X = np.zeros(3 * box.n ** 3)
    lib().nbo_element_coords(box.nx, box.ny, box.nz, box.N, box.deform,
                             np.ascontiguousarray(xi), int(e), X)
    return X.reshape(3, box.n ** 3)


def geom(box, elems=None, with_mass: bool = False):
    """Geometric factors G[cnt, 6, n^3] (rr, rs, rt, ss, st, tt) of the listed
    elements (all by default); optionally the nodal mass w_i w_j w_k J."""
    if elems is None:
        elems = np.arange(box.E, dtype=np.int64)
    elems = np.ascontiguousarray(elems, dtype=np.int64)
    n3 = box.n ** 3
    G = np.zeros(len(elems) * 6 * n3)
    mass = np.zeros(len(elems) * n3) if with_mass else None
    bad = lib().nbo_geom(box.nx, box.ny, box.nz, box.N, box.deform, elems, len(elems), G,
                         mass.ctypes.data if with_mass else None)
    if bad != 0:
        raise ValueError(f"{bad} nodes with non-positive Jacobian")
    G = G.reshape(len(elems), 6, n3)
    return (G, mass.reshape(len(elems), n3)) if with_mass else G


def numbering(box):
    """gid (int64, per local node), mult (int32, per global node) and the
    Dirichlet mask (uint8, per global node)."""
    gid = np.zeros(box.n_local, dtype=np.int64)
    mult = np.zeros(box.n_global, dtype=np.int32)
    mask = np.zeros(box.n_global, dtype=np.uint8)
    lib().nbo_numbering(box.nx, box.ny, box.nz, box.N, gid, mult, mask)
    return gid, mult, mask


def csr(gid: np.ndarray, nG: int):
    """offsets[nG+1] and locals[nL]: copies of each global node, ascending."""
    offsets = np.zeros(nG + 1, dtype=np.int64)
    locals_ = np.zeros(len(gid), dtype=np.int64)
    lib().nbo_csr(len(gid), nG, np.ascontiguousarray(gid, dtype=np.int64), offsets, locals_)
    return offsets, locals_


def ax_local(N: int, D: np.ndarray, G: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Local operator A_L u on every element of u (G[cnt,6,n^3])."""
    n3 = (N + 1) ** 3
    G = np.ascontiguousarray(G, dtype=np.float64).reshape(-1)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    cnt = len(u) // n3
    w = np.zeros_like(u)
    lib().nbo_ax_local(cnt, N, np.ascontiguousarray(D, dtype=np.float64).reshape(-1), G, u, w)
    return w


def diag_local(N: int, D: np.ndarray, G: np.ndarray) -> np.ndarray:
    n3 = (N + 1) ** 3
    G = np.ascontiguousarray(G, dtype=np.float64).reshape(-1)
    cnt = len(G) // (6 * n3)
    d = np.zeros(cnt * n3)
    lib().nbo_diag_local(cnt, N, np.ascontiguousarray(D, dtype=np.float64).reshape(-1), G, d)
    return d


def dssum(gid: np.ndarray, nG: int, u: np.ndarray, mask=None) -> np.ndarray:
    """Direct-stiffness summation (sum over copies, ascending local index),
    then the Dirichlet mask if given."""
    out = np.array(u, dtype=np.float64, copy=True)
    work = np.zeros(nG)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    lib().nbo_dssum(len(out), nG, np.ascontiguousarray(gid, dtype=np.int64),
                    None if m is None else m.ctypes.data, out, work)
    return out


def threads(nt: int = 0) -> int:
    """Host threads of the oracle's parallel loops (nt > 0 sets the count);
    returns the count in force (1 without OpenMP)."""
    return lib().nbo_threads(int(nt))


def vround(x: float, t: int) -> float:
    """x rounded to t mantissa bits (round to nearest, ties to even)."""
    return lib().nbo_vround(float(x), int(t))


def inexact(x: float, t: int, state: int):
    """Monte Carlo Arithmetic perturbation of x at virtual precision t with
    the SplitMix64 state; returns (value, new state)."""
    st = C.c_uint64(state)
    v = lib().nbo_inexact(float(x), int(t), C.byref(st))
    return v, st.value


def glsc3(a, b, c) -> float:
    return lib().nbo_glsc3(np.ascontiguousarray(a, dtype=np.float64),
                           np.ascontiguousarray(b, dtype=np.float64),
                           np.ascontiguousarray(c, dtype=np.float64), len(a))


# --------------------------------------------------------------------------
# a whole problem
# --------------------------------------------------------------------------

class Problem:
    """Everything the oracle needs for one box: D, G, numbering, mask,
    c = 1/multiplicity and the Jacobi inverse diagonal."""

    def __init__(self, box):
        self.box = box
        self.N = box.N
        self.xi, self.w = gll(box.N)
        self.D = deriv(box.N, self.xi)
        self.G = geom(box)
        self.gid, self.mult, self.mask = numbering(box)
        self.c = 1.0 / self.mult[self.gid].astype(np.float64)
        dl = diag_local(box.N, self.D, self.G)
        diag = dssum(self.gid, box.n_global, dl)
        m_l = self.mask[self.gid].astype(np.float64)
        self.diag = diag
        self.dinv = np.where(m_l > 0, 1.0 / np.where(diag != 0, diag, 1.0), 0.0)
        self._work = np.zeros(box.n_global)
        self._Df = np.ascontiguousarray(self.D.reshape(-1))
        self._Gf = np.ascontiguousarray(self.G.reshape(-1))
        self._op = _Op(box.E, box.N, box.n_local, box.n_global,
                       self._Df.ctypes.data, self._Gf.ctypes.data, self.gid.ctypes.data,
                       self.mask.ctypes.data, self.c.ctypes.data, self.dinv.ctypes.data,
                       self._work.ctypes.data)

    # Q: global -> local (scatter to every copy), then the mask
    def to_local(self, ug: np.ndarray, masked: bool = True) -> np.ndarray:
        uL = np.asarray(ug, dtype=np.float64)[self.gid]
        if masked:
            uL = uL * self.mask[self.gid]
        return np.ascontiguousarray(uL)

    def to_global(self, uL: np.ndarray) -> np.ndarray:
        """Value of a continuous L-vector at each global node (first copy)."""
        out = np.zeros(self.box.n_global)
        out[self.gid[::-1]] = np.asarray(uL)[::-1]
        return out

    def apply(self, u: np.ndarray) -> np.ndarray:
        """Assembled, masked operator w = M Q Q^T A_L u."""
        u = np.ascontiguousarray(u, dtype=np.float64)
        w = np.zeros_like(u)
        lib().nbo_apply(C.byref(self._op), u, w)
        return w

    def ax_local(self, u):
        return ax_local(self.N, self.D, self.G, u)

    def dssum(self, u, masked=True):
        return dssum(self.gid, self.box.n_global, u, self.mask if masked else None)

    def glsc3(self, a, b):
        return glsc3(a, self.c, b)

    def pcg(self, b: np.ndarray, tol: float = 1e-10, maxit: int = 1000,
            precond: str = "jacobi", x0=None, history: bool = False):
        """Jacobi (or identity) PCG in Table 1 order.  Returns
        (x, iterations, final relative residual, history)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
        hist = np.zeros(max(maxit, 1))
        rel = C.c_double(0.0)
        it = lib().nbo_pcg(C.byref(self._op), b, x, maxit, tol,
                           1 if precond == "jacobi" else 0, hist.ctypes.data, C.byref(rel))
        return x, it, rel.value, (hist[:it].copy() if history else None)

    def pcg_par(self, b: np.ndarray, tol: float = 1e-10, maxit: int = 1000,
                precond: str = "jacobi", x0=None, history: bool = False):
        """``pcg`` on all host cores (``threads`` sets how many): the operator,
        the summation and the vector updates give ``pcg``'s bits; the dot
        products are summed in fixed chunks of 65536 terms, so the result does
        not depend on the thread count and differs from ``pcg`` by the
        rounding order of the dots only."""
        if getattr(self, "_csr", None) is None:
            self._csr = csr(self.gid, self.box.n_global)
        off, loc = self._csr
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
        hist = np.zeros(max(maxit, 1))
        rel = C.c_double(0.0)
        it = lib().nbo_pcg_par(C.byref(self._op), off, loc, b, x, maxit, tol,
                               1 if precond == "jacobi" else 0, hist.ctypes.data, C.byref(rel))
        return x, it, rel.value, (hist[:it].copy() if history else None)

    def fcg(self, b: np.ndarray, precond, tol: float = 1e-10, maxit: int = 1000,
            x0=None):
        """Flexible CG (Notay, SIAM J. Sci. Comput. 22, 2000) with one-vector
        truncation: z_k = B(r_k), p_k = z_k - (z_k^T A p_{k-1} /
        p_{k-1}^T A p_{k-1}) p_{k-1}.  ``precond`` maps an L-vector residual
        to an L-vector (continuous, masked).  Returns (x, iters, relres, hist)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
        r = b - self.apply(x)
        bnorm = math.sqrt(self.glsc3(b, b)) or 1.0
        p = np.zeros_like(b)
        w = np.zeros_like(b)
        pap_prev = None
        hist = []
        rel = math.sqrt(self.glsc3(r, r)) / bnorm
        it = 0
        for it in range(1, maxit + 1):
            z = precond(r)
            if pap_prev is None:
                p = z.copy()
            else:
                beta = -self.glsc3(z, w) / pap_prev
                p = z + beta * p
            w = self.apply(p)
            pap = self.glsc3(w, p)
            alpha = self.glsc3(r, p) / pap
            x = x + alpha * p
            r = r - alpha * w
            pap_prev = pap
            rel = math.sqrt(self.glsc3(r, r)) / bnorm
            hist.append(rel)
            if rel < tol:
                break
        return x, it, rel, np.array(hist)

    def apply_vprec(self, u: np.ndarray, t: int) -> np.ndarray:
        """Assembled operator with every +, -, *, / rounded to t bits."""
        u = np.ascontiguousarray(u, dtype=np.float64)
        w = np.zeros_like(u)
        lib().nbo_apply_vprec(C.byref(self._op), t, u, w)
        return w

    def cg_vprec(self, b: np.ndarray, iters: int, t: int, precond: str = "none"):
        """`iters` CG iterations (Table 1 order) with every arithmetic
        operation of the loop rounded to t mantissa bits.  Returns (x, hist)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        hist = np.zeros(max(iters, 1))
        lib().nbo_cg_vprec(C.byref(self._op), b, x, iters, t, 1 if precond == "jacobi" else 0,
                           hist.ctypes.data)
        return x, hist[:iters].copy()

    def cg_mca(self, b: np.ndarray, iters: int, t: int, mode: str, seed: int,
               precond: str = "none"):
        """`iters` CG iterations with Monte Carlo Arithmetic on every operation
        of the loop (mode "rr": results perturbed; "mca": operands and results),
        virtual precision t, SplitMix64 seed.  Returns (x, hist)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        hist = np.zeros(max(iters, 1))
        lib().nbo_cg_emu(C.byref(self._op), b, x, iters, {"rr": 1, "mca": 2}[mode], t, seed,
                         1 if precond == "jacobi" else 0, hist.ctypes.data)
        return x, hist[:iters].copy()

    def true_relres(self, b: np.ndarray, x: np.ndarray) -> float:
        r = b - self.apply(x)
        return math.sqrt(self.glsc3(r, r)) / (math.sqrt(self.glsc3(b, b)) or 1.0)


__all__ = ["lib", "legendre", "gll", "deriv", "element_coords", "geom", "numbering",
           "csr", "ax_local", "diag_local", "dssum", "glsc3", "threads", "vround", "inexact",
           "Problem"]
