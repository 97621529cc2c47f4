"""Python binding of the sm_103a spectral-element CG library.

Argument marshalling only: every step of the solve runs in the CUDA library
``_build/libnekbone_gb300.so`` (C ABI in ``include/nekbone_gb300.h``).  The
functions below carry the C names; ``Mesh`` bundles them for convenience.
Device vectors are ``torch`` CUDA tensors (PyTorch provides memory and
streams only).  If the library has not been built, importing this module
raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libnekbone_gb300.so")

NB_OK, NB_ERR_ARG, NB_ERR_CUDA, NB_ERR_OOM, NB_ERR_MESH, NB_ERR_STATE = 0, -1, -2, -3, -4, -5
NB_NOT_CONVERGED, NB_STAGNATED, NB_BREAKDOWN, NB_FELL_BACK = 1, 2, 3, 4
NB_FP64, NB_FP32, NB_TC_F16, NB_TC_BF16 = 0, 1, 2, 3
NB_PC_NONE, NB_PC_JACOBI, NB_PC_LEARNED, NB_PC_SCHWARZ, NB_PC_SCHWARZ2 = 0, 1, 2, 3, 4
STATUS_NAMES = {0: "ok", -1: "invalid argument", -2: "cuda error", -3: "out of memory",
                -4: "invalid mesh", -5: "bad state", 1: "not converged", 2: "stagnated",
                3: "breakdown", 4: "fell back"}
PREC_NAMES = {"fp64": NB_FP64, "fp32": NB_FP32, "tc_f16": NB_TC_F16, "tc_bf16": NB_TC_BF16}


class NbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class nb_opts(C.Structure):
    _fields_ = [("prec", C.c_int), ("pc", C.c_int), ("rtol", C.c_double), ("maxiter", C.c_int),
                ("inner_rtol", C.c_double), ("max_outer", C.c_int), ("use_graph", C.c_int),
                ("record_history", C.c_int), ("use_x0", C.c_int), ("restart", C.c_int)]


class nb_stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("outer_iters", C.c_int), ("rel_res", C.c_double),
                ("seconds", C.c_double), ("status", C.c_int), ("history_len", C.c_int),
                ("history_host", C.POINTER(C.c_double)), ("history_cap", C.c_int),
                ("launches", C.c_int64), ("final_prec", C.c_int)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"CUDA library not built ({LIB_PATH}); run `python -c 'import __graft_entry__ as g; "
            f"g.build()'` on a machine with nvcc")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
    sig = {
        "nb_version": (C.c_char_p, []),
        "nb_last_error": (C.c_char_p, []),
        "nb_create": (i32, [C.POINTER(vp), i32, vp]),
        "nb_set_stream": (i32, [vp, vp]),
        "nb_destroy": (i32, [vp]),
        "nb_setup_mesh": (i32, [vp, i32, i32, i32, i32, dbl, C.POINTER(vp)]),
        "nb_setup_gs": (i32, [vp]),
        "nb_mesh_destroy": (i32, [vp]),
        "nb_mesh_sizes": (i32, [vp, C.POINTER(i64)]),
        "nb_get_maps": (i32, [vp, vp, vp, vp, vp, vp, vp, vp]),
        "nb_get_geom": (i32, [vp, vp, vp, vp]),
        "nb_to_local": (i32, [vp, i32, vp, vp, i32]),
        "nb_to_global": (i32, [vp, i32, vp, vp]),
        "nb_ax": (i32, [vp, i32, i32, vp, vp]),
        "nb_dssum": (i32, [vp, i32, vp, i32]),
        "nb_glsc3": (i32, [vp, i32, vp, vp, C.POINTER(dbl)]),
        "nb_glsc3_noalloc": (i32, [vp, i32, vp, vp, C.POINTER(dbl)]),
        "nb_batch_create": (i32, [vp, i32, vp, vp, vp, vp, vp, C.POINTER(vp)]),
        "nb_batch_destroy": (i32, [vp]),
        "nb_batch_layout": (i32, [vp, vp, vp, vp]),
        "nb_batch_mesh": (vp, [vp, i32]),
        "nb_batch_to_local": (i32, [vp, vp, vp]),
        "nb_batch_solve": (i32, [vp, C.POINTER(nb_opts), vp, vp, vp, C.POINTER(nb_stats)]),
        "nb_batch_autotune": (i32, [vp, i32, vp, C.c_size_t]),
        "nb_model_create": (i32, [vp, i32, i32, C.c_uint64, C.POINTER(vp)]),
        "nb_model_destroy": (i32, [vp]),
        "nb_model_params": (i32, [vp, vp, vp, C.POINTER(i64)]),
        "nb_model_grad": (i32, [vp, vp, vp, i32, C.POINTER(dbl), vp]),
        "nb_model_train": (i32, [vp, vp, vp, i32, i32, i32, C.c_float, C.POINTER(dbl)]),
        "nb_learned_collect": (i32, [vp, vp, i32, vp, i32, C.c_uint64, i32, vp, vp,
                                     C.POINTER(i32)]),
        "nb_learned_targets": (i32, [vp, vp, vp, i32, vp, vp]),
        "nb_learned_attach": (i32, [vp, vp]),
        "nb_learned_apply": (i32, [vp, vp, vp]),
        "nb_learned_step": (i32, [vp, vp, vp, vp, C.POINTER(C.c_double),
                                  C.POINTER(C.c_double)]),
        "nb_default_opts": (None, [C.POINTER(nb_opts)]),
        "nb_solve": (i32, [vp, C.POINTER(nb_opts), vp, vp, C.POINTER(nb_stats)]),
        "nb_solve_host": (i32, [vp, C.POINTER(nb_opts), vp, vp, C.POINTER(nb_stats)]),
        "nb_time_ax": (i32, [vp, i32, i32, i32, i32, vp, C.c_size_t, C.POINTER(dbl)]),
        "nb_ax_variants": (i32, [vp, i32]),
        "nb_set_ax_variant": (i32, [vp, i32, i32]),
        "nb_set_update_variant": (i32, [vp, i32]),
        "nb_set_x_deferral": (i32, [vp, i32]),
        "nb_setup_slab": (i32, [vp, i32, i32, i32, i32, i32, i32, dbl, C.POINTER(vp)]),
        "nb_slab_face": (i32, [vp, i32, i32, vp, vp]),
        "nb_slab_face_add": (i32, [vp, i32, i32, vp, vp]),
        "nb_slab_diag_face": (i32, [vp, i32, vp]),
        "nb_slab_finish_diag": (i32, [vp, vp, vp]),
        "nb_cg_step": (i32, [vp, i32, dbl, vp, vp, vp, C.POINTER(dbl)]),
        "nb_cg_update": (i32, [vp, i32, dbl, vp, vp, vp, vp, C.POINTER(dbl)]),
        "nb_cg_dots": (i32, [vp, i32, vp, C.POINTER(dbl)]),
        "nb_ax_variant_name": (C.c_char_p, [vp, i32, i32]),
        "nb_ax_variant_in_use": (i32, [vp, i32]),
        "nb_autotune": (i32, [vp, i32, i32, vp, C.c_size_t, C.POINTER(i32), C.POINTER(dbl)]),
        "nb_apply_vprec": (i32, [vp, i32, vp, vp]),
        "nb_schwarz_apply": (i32, [vp, vp, vp]),
        "nb_schwarz2_apply": (i32, [vp, vp, vp]),
        "nb_cg_vprec": (i32, [vp, i32, i32, i32, vp, vp, vp, C.POINTER(dbl)]),
        "nb_cg_mca": (i32, [vp, i32, i32, C.c_uint64, i32, i32, vp, vp, vp, C.POINTER(dbl)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()

def check(status, allow_positive=True):
    if status < 0 or (status > 0 and not allow_positive):
        raise NbError(status, lib.nb_last_error().decode())
    return status


def nb_version() -> str:
    return lib.nb_version().decode()


def default_opts(**kw) -> nb_opts:
    o = nb_opts()
    lib.nb_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "prec" and isinstance(v, str):
            v = PREC_NAMES[v]
        setattr(o, k, v)
    return o


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return C.c_void_p(t.data_ptr())


class Context:
    """nb_create/nb_destroy.  With ``stream=None`` (or torch's legacy default
    stream) the library issues work on a stream of its own that is ordered
    with the legacy default stream, so tensors produced by ordinary torch
    calls are ready when the library reads them."""

    def __init__(self, device: int = 0, stream=None):
        handle = None
        if stream is not None and stream.cuda_stream:
            handle = C.c_void_p(stream.cuda_stream)
        self.stream = stream
        h = C.c_void_p()
        check(lib.nb_create(C.byref(h), device, handle))
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            lib.nb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    """A box mesh with its gather-scatter set up (nb_setup_mesh + nb_setup_gs)."""

    def __init__(self, ctx: Context, nx, ny, nz, N, deform=0.0, setup_gs=True, slab=None):
        """``slab=(z0, z1)``: the z-slab z0 <= ez < z1 of the box (nb_setup_slab)."""
        h = C.c_void_p()
        if slab is None:
            check(lib.nb_setup_mesh(ctx.h, nx, ny, nz, N, float(deform), C.byref(h)))
        else:
            check(lib.nb_setup_slab(ctx.h, nx, ny, nz, int(slab[0]), int(slab[1]), N,
                                    float(deform), C.byref(h)))
        self.slab = slab
        self.h = h
        self.ctx = ctx
        if setup_gs:
            check(lib.nb_setup_gs(self.h))
        s = (C.c_int64 * 9)()
        check(lib.nb_mesh_sizes(self.h, s))
        self.E, self.N, self.n_local, self.n_global, self.gs_rows, self.gs_copies = list(s)[:6]
        self.nx, self.ny, self.nz = list(s)[6:9]

    @classmethod
    def from_box(cls, ctx, box, **kw):
        return cls(ctx, box.nx, box.ny, box.nz, box.N, box.deform, **kw)

    def close(self):
        if self.h:
            lib.nb_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- inspection
    def maps(self):
        gid = np.zeros(self.n_local, np.int32)
        mult = np.zeros(self.n_global, np.int32)
        mask = np.zeros(self.n_global, np.uint8)
        rgid = np.zeros(max(self.gs_rows, 1), np.int32)
        roff = np.zeros(self.gs_rows + 1, np.int32)
        rloc = np.zeros(max(self.gs_copies, 1), np.int32)
        rmask = np.zeros(max(self.gs_rows, 1), np.uint8)
        check(lib.nb_get_maps(self.h, _ptr(gid), _ptr(mult), _ptr(mask), _ptr(rgid), _ptr(roff),
                              _ptr(rloc), _ptr(rmask)))
        return dict(gid=gid, mult=mult, mask=mask, gs_gid=rgid[:self.gs_rows], gs_off=roff,
                    gs_loc=rloc[:self.gs_copies], gs_mask=rmask[:self.gs_rows])

    def geom(self):
        G = np.zeros(6 * self.n_local)
        dinv = np.zeros(self.n_local)
        c = np.zeros(self.n_local)
        check(lib.nb_get_geom(self.h, _ptr(G), _ptr(dinv), _ptr(c)))
        return G.reshape(self.E, 6, -1), dinv, c

    # --- operations on torch CUDA tensors
    def _vec(self, t, prec, n=None):
        import torch
        n = self.n_local if n is None else n
        want = torch.float64 if prec == NB_FP64 else torch.float32
        if not (t.is_cuda and t.dtype == want and t.is_contiguous() and t.numel() == n):
            raise NbError(NB_ERR_ARG, f"expected contiguous CUDA {want} tensor of {n} values")
        return _ptr(t)

    def to_local(self, prec, ug, uL, masked=True):
        check(lib.nb_to_local(self.h, prec, self._vec(ug, prec, self.n_global),
                              self._vec(uL, prec), int(masked)))

    def to_global(self, prec, uL, ug):
        check(lib.nb_to_global(self.h, prec, self._vec(uL, prec), self._vec(ug, prec, self.n_global)))

    def ax(self, prec, u, w, assemble=False):
        check(lib.nb_ax(self.h, prec, int(assemble), self._vec(u, prec), self._vec(w, prec)))

    def dssum(self, prec, u, masked=True):
        check(lib.nb_dssum(self.h, prec, self._vec(u, prec), int(masked)))

    def glsc3(self, prec, a, b) -> float:
        out = C.c_double()
        check(lib.nb_glsc3(self.h, prec, self._vec(a, prec), self._vec(b, prec), C.byref(out)))
        return out.value

    def solve(self, b, x, opts: nb_opts | None = None, history_cap=0, raise_on_outcome=False):
        opts = opts or default_opts()
        st = nb_stats()
        hist = None
        if history_cap:
            hist = np.zeros(history_cap)
            st.history_host = hist.ctypes.data_as(C.POINTER(C.c_double))
            st.history_cap = history_cap
            opts.record_history = 1
        r = check(lib.nb_solve(self.h, C.byref(opts), self._vec(b, NB_FP64), self._vec(x, NB_FP64),
                               C.byref(st)), allow_positive=not raise_on_outcome)
        out = dict(status=r, iters=st.iters, outer_iters=st.outer_iters, rel_res=st.rel_res,
                   seconds=st.seconds, launches=st.launches, final_prec=st.final_prec)
        if hist is not None:
            out["history"] = hist[:st.history_len].copy()
        return out

    def solve_host(self, bg: np.ndarray, xg: np.ndarray, opts: nb_opts | None = None):
        """bg, xg: host float64 arrays of n_global values (pinned or pageable)."""
        opts = opts or default_opts()
        st = nb_stats()
        if hasattr(bg, "data_ptr"):
            pb, px = C.c_void_p(bg.data_ptr()), C.c_void_p(xg.data_ptr())
        else:
            assert bg.dtype == np.float64 and xg.dtype == np.float64
            pb, px = _ptr(bg), _ptr(xg)
        r = check(lib.nb_solve_host(self.h, C.byref(opts), pb, px, C.byref(st)))
        return dict(status=r, iters=st.iters, outer_iters=st.outer_iters, rel_res=st.rel_res,
                    seconds=st.seconds, launches=st.launches)

    # --- measurement
    def time_ax(self, prec, cg_step=True, variant=-1, reps=10, flush=None) -> float:
        """Mean milliseconds per operator launch (CUDA events, L2 flushed
        between launches by overwriting ``flush``, a CUDA byte tensor)."""
        ms = C.c_double()
        fp, fb = (_ptr(flush), flush.numel() * flush.element_size()) if flush is not None else (None, 0)
        check(lib.nb_time_ax(self.h, prec, int(cg_step), variant, reps, fp, fb, C.byref(ms)))
        return ms.value

    def schwarz_apply(self, r, z, coarse=False):
        """z = M r (FP32 L-vectors): one-level Schwarz, or with ``coarse`` the
        two-level form (nb_schwarz2_apply)."""
        f = lib.nb_schwarz2_apply if coarse else lib.nb_schwarz_apply
        check(f(self.h, self._vec(r, NB_FP32), self._vec(z, NB_FP32)))

    def apply_vprec(self, t, u, w):
        """w = A u with every operation rounded to t mantissa bits (FP64)."""
        check(lib.nb_apply_vprec(self.h, int(t), self._vec(u, NB_FP64), self._vec(w, NB_FP64)))

    def cg_vprec(self, t, iters, b, x, pc=None):
        """`iters` CG iterations from zero with every operation of the loop
        rounded to t mantissa bits; returns the loop's relative residuals."""
        hist = np.zeros(max(int(iters), 1))
        rel = C.c_double()
        check(lib.nb_cg_vprec(self.h, int(t), int(iters), NB_PC_NONE if pc is None else pc,
                              self._vec(b, NB_FP64), self._vec(x, NB_FP64), hist.ctypes.data,
                              C.byref(rel)))
        return hist[:int(iters)]

    def cg_mca(self, mode, t, seed, iters, b, x, pc=None):
        """Monte Carlo Arithmetic CG loop (mode "rr" or "mca", virtual
        precision t); returns the loop's relative residuals."""
        hist = np.zeros(max(int(iters), 1))
        rel = C.c_double()
        check(lib.nb_cg_mca(self.h, {"rr": 1, "mca": 2}[mode], int(t), int(seed), int(iters),
                            NB_PC_NONE if pc is None else pc, self._vec(b, NB_FP64),
                            self._vec(x, NB_FP64), hist.ctypes.data, C.byref(rel)))
        return hist[:int(iters)]

    def ax_variants(self, prec) -> int:
        return lib.nb_ax_variants(self.h, prec)

    # --- slabs and the split-phase CG (nb_slab_*, nb_cg_*)
    def plane_size(self) -> int:
        return (self.nx * self.N + 1) * (self.ny * self.N + 1)

    def slab_face(self, prec, side, u, face):
        check(lib.nb_slab_face(self.h, prec, int(side), self._vec(u, prec),
                               self._vec(face, prec, self.plane_size())))

    def slab_face_add(self, prec, side, u, face):
        check(lib.nb_slab_face_add(self.h, prec, int(side), self._vec(u, prec),
                                   self._vec(face, prec, self.plane_size())))

    def slab_diag_face(self, side, face):
        check(lib.nb_slab_diag_face(self.h, int(side), self._vec(face, NB_FP64, self.plane_size())))

    def slab_finish_diag(self, face_lo=None, face_hi=None):
        f = lambda t: None if t is None else self._vec(t, NB_FP64, self.plane_size())
        check(lib.nb_slab_finish_diag(self.h, f(face_lo), f(face_hi)))

    def cg_step(self, prec, beta, r, p, w) -> float:
        out = C.c_double()
        check(lib.nb_cg_step(self.h, prec, float(beta), self._vec(r, prec), self._vec(p, prec),
                             self._vec(w, prec), C.byref(out)))
        return out.value

    def cg_update(self, prec, alpha, x, r, p, w):
        out = (C.c_double * 2)()
        check(lib.nb_cg_update(self.h, prec, float(alpha), self._vec(x, prec), self._vec(r, prec),
                               self._vec(p, prec), self._vec(w, prec), out))
        return out[0], out[1]

    def cg_dots(self, prec, r):
        out = (C.c_double * 2)()
        check(lib.nb_cg_dots(self.h, prec, self._vec(r, prec), out))
        return out[0], out[1]

    def ax_variant_name(self, prec, variant=-1) -> str:
        """Kernel name of a variant (-1: the one in use)."""
        r = lib.nb_ax_variant_name(self.h, prec, int(variant))
        return r.decode() if r else ""

    def ax_variant_in_use(self, prec) -> int:
        return lib.nb_ax_variant_in_use(self.h, prec)

    def set_update_variant(self, variant=0):
        """Kernel of the FP32 update with the folded summation (0: built-in)."""
        check(lib.nb_set_update_variant(self.h, int(variant)))

    def set_x_deferral(self, mode=-1):
        """Deferred x steps of the FP32 Jacobi iteration: -1 by size (the
        built-in rule), 0 never, 1 wherever the kernels allow it."""
        check(lib.nb_set_x_deferral(self.h, int(mode)))

    def set_ax_variant(self, prec, variant=-1):
        """Use operator variant ``variant`` (-1: the default) from now on."""
        check(lib.nb_set_ax_variant(self.h, prec, int(variant)))

    def autotune(self, prec, reps=5, flush=None):
        v, ms = C.c_int(), C.c_double()
        fp, fb = (_ptr(flush), flush.numel() * flush.element_size()) if flush is not None else (None, 0)
        check(lib.nb_autotune(self.h, prec, reps, fp, fb, C.byref(v), C.byref(ms)))
        return v.value, ms.value


class Batch:
    """nb_batch_create/destroy/solve: independent problems of mixed size and
    order solved together.  ``boxes``: objects with nx, ny, nz, N, deform."""

    def __init__(self, ctx: Context, boxes):
        n = len(boxes)
        arr = lambda f, t: np.ascontiguousarray([f(b) for b in boxes], dtype=t)
        self._keep = [arr(lambda b: b.nx, np.int32), arr(lambda b: b.ny, np.int32),
                      arr(lambda b: b.nz, np.int32), arr(lambda b: b.N, np.int32),
                      arr(lambda b: b.deform, np.float64)]
        h = C.c_void_p()
        check(lib.nb_batch_create(ctx.h, n, *[_ptr(a) for a in self._keep], C.byref(h)))
        self.h = h
        self.ctx = ctx
        self.nprob = n
        self.l_off = np.zeros(n, np.int64)
        self.g_off = np.zeros(n, np.int64)
        tot = np.zeros(2, np.int64)
        check(lib.nb_batch_layout(self.h, _ptr(self.l_off), _ptr(self.g_off), _ptr(tot)))
        self.n_local, self.n_global = int(tot[0]), int(tot[1])

    def close(self):
        if self.h:
            lib.nb_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def to_local(self, ug, uL):
        check(lib.nb_batch_to_local(self.h, _ptr(ug), _ptr(uL)))

    def autotune(self, reps=3, flush=None):
        fp, fb = (_ptr(flush), flush.numel() * flush.element_size()) if flush is not None else (None, 0)
        check(lib.nb_batch_autotune(self.h, reps, fp, fb))

    def solve(self, b, x, opts: nb_opts | None = None):
        opts = opts or default_opts()
        st = (nb_stats * self.nprob)()
        tot = nb_stats()
        r = check(lib.nb_batch_solve(self.h, C.byref(opts), _ptr(b), _ptr(x), st, C.byref(tot)))
        per = [dict(status=s.status, iters=s.iters, outer_iters=s.outer_iters, rel_res=s.rel_res)
               for s in st]
        return dict(status=r, iters=tot.iters, outer_iters=tot.outer_iters, rel_res=tot.rel_res,
                    seconds=tot.seconds, launches=tot.launches, problems=per)


class Model:
    """The learned per-element preconditioner's network (nb_model_*)."""

    def __init__(self, ctx: Context, N: int, hidden: int = 48, seed: int = 0):
        h = C.c_void_p()
        check(lib.nb_model_create(ctx.h, N, hidden, seed, C.byref(h)))
        self.h, self.ctx, self.N, self.hidden = h, ctx, N, hidden
        self.d = (N + 1) ** 3
        n = C.c_int64()
        check(lib.nb_model_params(self.h, None, None, C.byref(n)))
        self.nparam = n.value

    def close(self):
        if self.h:
            lib.nb_model_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> dict:
        flat = np.zeros(self.nparam, np.float32)
        check(lib.nb_model_params(self.h, _ptr(flat), None, None))
        return self._split(flat)

    def set_params(self, p: dict):
        flat = np.ascontiguousarray(np.concatenate(
            [np.asarray(p[k], np.float32).reshape(-1) for k in ("W", "a")]))
        assert flat.size == self.nparam
        check(lib.nb_model_params(self.h, None, _ptr(flat), None))

    def _split(self, flat):
        d, h = self.d, self.hidden
        o = 0
        out = {}
        for k, shape in (("W", (d, h)), ("a", (h,))):
            size = int(np.prod(shape))
            out[k] = flat[o:o + size].reshape(shape)
            o += size
        return out

    def grad(self, X, T):
        loss = C.c_double()
        g = np.zeros(self.nparam, np.float32)
        check(lib.nb_model_grad(self.h, _ptr(X), _ptr(T), X.shape[0], C.byref(loss), _ptr(g)))
        return loss.value, self._split(g)

    def train(self, X, T, epochs=20, batch=256, lr=1e-3) -> float:
        loss = C.c_double()
        check(lib.nb_model_train(self.h, _ptr(X), _ptr(T), X.shape[0], epochs, batch, lr,
                                 C.byref(loss)))
        return loss.value

    @staticmethod
    def collect(mesh: "Mesh", b, snap_iters, per_snap, seed=0, use_learned=False):
        """Training pairs from the solver's own iterates of A x = b: Jacobi-PCG,
        or flexible CG with the attached network (see the C header)."""
        import torch
        its = np.ascontiguousarray(snap_iters, dtype=np.int32)
        cap = len(its) * per_snap
        d = (mesh.N + 1) ** 3
        X = torch.empty((cap, d), dtype=torch.float32, device=b.device)
        T = torch.empty((cap, d), dtype=torch.float32, device=b.device)
        cnt = C.c_int()
        check(lib.nb_learned_collect(mesh.h, _ptr(b), len(its), _ptr(its), per_snap, seed,
                                     int(use_learned), _ptr(X), _ptr(T), C.byref(cnt)))
        return X[:cnt.value], T[:cnt.value]

    @staticmethod
    def targets(mesh: "Mesh", r, elems):
        """X, T of nb_learned_targets for a residual L-vector (FP64 CUDA)."""
        import torch
        el = torch.as_tensor(np.ascontiguousarray(elems, dtype=np.int32)).to(r.device)
        d = (mesh.N + 1) ** 3
        X = torch.empty((len(el), d), dtype=torch.float32, device=r.device)
        T = torch.empty_like(X)
        check(lib.nb_learned_targets(mesh.h, _ptr(r), _ptr(el), len(el), _ptr(X), _ptr(T)))
        return X, T

    def attach(self, mesh: "Mesh"):
        check(lib.nb_learned_attach(mesh.h, self.h))
        mesh._model = self  # keep alive

    def apply(self, mesh: "Mesh", r, z):
        check(lib.nb_learned_apply(mesh.h, _ptr(r), _ptr(z)))

    def step(self, mesh: "Mesh", r, wprev, z):
        """The fused preconditioner step of the learned flexible CG: z = B(r)
        and the dots (z, w_prev) over every copy and (r, c, z); returns both."""
        zw, rz = C.c_double(), C.c_double()
        check(lib.nb_learned_step(mesh.h, _ptr(r), _ptr(wprev), _ptr(z), C.byref(zw),
                                  C.byref(rz)))
        return zw.value, rz.value


__all__ = ["lib", "LIB_PATH", "Batch", "Model", "NbError", "Context", "Mesh", "default_opts", "check",
           "nb_opts", "nb_stats", "nb_version", "PREC_NAMES",
           "NB_FP64", "NB_FP32", "NB_TC_F16", "NB_TC_BF16", "NB_PC_NONE", "NB_PC_JACOBI",
           "NB_PC_LEARNED", "NB_PC_SCHWARZ", "NB_PC_SCHWARZ2", "NB_OK", "NB_NOT_CONVERGED", "NB_STAGNATED", "NB_BREAKDOWN",
           "NB_FELL_BACK"]
