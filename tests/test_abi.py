"""Host-side checks of the C ABI: the library loads, exports every function
the header declares, and validates arguments without touching a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def _declared():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w \*]*?\b(nb_\w+)\s*\(", src, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def nb():
    import __graft_entry__ as g
    g.build()
    import paper_2405_11065_gb300 as nb
    return nb


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("nb_setup_mesh", "nb_setup_gs", "nb_ax", "nb_solve", "nb_dssum",
                     "nb_glsc3", "nb_solve_host"):
        assert required in names


def test_library_exports_every_declared_symbol(nb):
    lib = C.CDLL(nb.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_defaults(nb):
    assert "sm_103a" in nb.nb_version()
    o = nb.default_opts()
    assert o.prec == nb.NB_FP32 and o.pc == nb.NB_PC_JACOBI
    assert o.rtol == 1e-10 and o.use_graph == 1 and o.use_x0 == 0
    # refinement keeps the search direction by default (reliable updates);
    # the field is the last of the C struct, so this also checks the layout
    assert o.restart == 0 and o.inner_rtol == 1e-4 and o.max_outer == 30


def test_argument_validation_without_gpu(nb):
    lib = nb.lib
    h = C.c_void_p()
    # NULL output pointer and NULL context are rejected before any CUDA call
    assert lib.nb_create(None, 0, None) == nb.NB_ERR_ARG
    assert lib.nb_setup_mesh(None, 1, 1, 1, 3, 0.0, C.byref(h)) == nb.NB_ERR_ARG
    assert lib.nb_setup_gs(None) == nb.NB_ERR_ARG
    assert lib.nb_ax(None, 0, 0, None, None) == nb.NB_ERR_ARG
    assert lib.nb_solve(None, None, None, None, None) == nb.NB_ERR_ARG
    assert lib.nb_set_update_variant(None, 0) == nb.NB_ERR_ARG
    assert lib.nb_set_x_deferral(None, -1) == nb.NB_ERR_ARG
    assert b"invalid argument" in lib.nb_last_error()
    assert lib.nb_destroy(None) == nb.NB_OK
    assert lib.nb_mesh_destroy(None) == nb.NB_OK


def test_no_gpu_gives_an_error_not_a_crash(nb):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    st = nb.lib.nb_create(C.byref(h), 0, None)
    assert st in (nb.NB_ERR_CUDA, nb.NB_ERR_ARG)
