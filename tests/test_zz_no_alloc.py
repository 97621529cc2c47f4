"""The allocation-free glsc3 entry point (nb_glsc3_noalloc).

It exists for callers that cannot let the library allocate memory (a
framework's caching allocator that owns the device memory, a hard memory
budget, or a latency-critical loop that must not pay for cudaMalloc's
device synchronisation).  Its result must match nb_glsc3's, call after call,
although both calls reuse the same fixed device scratch.  This file is
collected last so that a failure here cannot hide another test's result.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from workloads import Box

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    import __graft_entry__ as g
    g.build()
    import paper_2405_11065_gb300 as nb
    return nb


@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
def test_noalloc_glsc3_matches_allocating_entry_point(nb, prec_name):
    import torch
    prec = nb.PREC_NAMES[prec_name]
    dtype = torch.float64 if prec == nb.NB_FP64 else torch.float32
    ctx = nb.Context(0)
    box = Box(4, 3, 2, 7, 0.05)  # 24 elements, 12,288 local nodes: several blocks
    mesh = nb.Mesh.from_box(ctx, box)
    c = mesh.geom()[2]
    rng = np.random.default_rng(42)
    for call in range(2):  # two calls in a row share the same scratch
        a = torch.from_numpy(rng.uniform(-1, 1, box.n_local)).to(dtype).cuda()
        b = torch.from_numpy(rng.uniform(-1, 1, box.n_local)).to(dtype).cuda()
        ref = mesh.glsc3(prec, a, b)
        got = C.c_double(np.nan)
        st = nb.lib.nb_glsc3_noalloc(mesh.h, prec, C.c_void_p(a.data_ptr()),
                                     C.c_void_p(b.data_ptr()), C.byref(got))
        assert st == nb.NB_OK, nb.lib.nb_last_error()
        a64, b64 = a.double().cpu().numpy(), b.double().cpu().numpy()
        scale = float(np.sum(np.abs(a64 * b64 * c)))
        assert abs(got.value - ref) <= 1e-13 * scale, (call, got.value, ref)
        # and the oracle's glsc3 of the same values: FP64 to summation order,
        # FP32 to the rounding of each product (2^-23 of its size)
        ora = oracle.glsc3(a64, b64, c)
        tol = 1e-13 if prec == nb.NB_FP64 else 2.0 ** -23
        assert abs(got.value - ora) <= tol * scale, (call, got.value, ora)
    # NULL output is rejected without touching the device
    st = nb.lib.nb_glsc3_noalloc(mesh.h, prec, C.c_void_p(a.data_ptr()),
                                 C.c_void_p(b.data_ptr()), None)
    assert st == nb.NB_ERR_ARG
