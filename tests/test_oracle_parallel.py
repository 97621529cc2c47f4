"""The oracle's parallel paths against its plain ones: the element loop and
the all-core PCG (the CPU baseline's all-core timing) give results that do
not depend on the thread count, and equal the single-threaded definitions --
bit for bit where the order of operations is the same, to the rounding order
of the dot products otherwise."""
import numpy as np
import pytest

import oracle
from workloads import Box, rhs_global


@pytest.fixture()
def restore_threads():
    n0 = oracle.threads()
    yield
    oracle.threads(n0)


def test_ax_local_does_not_depend_on_threads(restore_threads):
    box = Box(3, 2, 2, 6, 0.05)
    P = oracle.Problem(box)
    u = np.random.default_rng(3).uniform(-1, 1, box.n_local)
    oracle.threads(1)
    w1 = P.ax_local(u)
    for nt in (2, 5):
        oracle.threads(nt)
        assert np.array_equal(P.ax_local(u), w1)


def test_parallel_pcg_equals_pcg_within_one_chunk(restore_threads):
    # fewer local nodes than one dot-product chunk: the same sums in the same
    # order, so the parallel PCG reproduces pcg bit for bit
    box = Box(3, 3, 2, 5, 0.05)
    P = oracle.Problem(box)
    assert box.n_local < 65536
    b = P.to_local(rhs_global(box, 0))
    x1, it1, r1, h1 = P.pcg(b, tol=1e-10, maxit=500, history=True)
    oracle.threads(3)
    x2, it2, r2, h2 = P.pcg_par(b, tol=1e-10, maxit=500, history=True)
    assert it1 == it2
    assert np.array_equal(x1, x2) and np.array_equal(h1, h2)


def test_parallel_pcg_over_several_chunks(restore_threads):
    # 8 x 6 x 6 elements at N = 7: 147,456 local nodes, three chunks of the
    # dot products with a ragged last one
    box = Box(8, 6, 6, 7, 0.05)
    P = oracle.Problem(box)
    assert box.n_local > 2 * 65536
    b = P.to_local(rhs_global(box, 2))
    x1, it1, _, h1 = P.pcg(b, tol=1e-10, maxit=2000, history=True)
    runs = []
    for nt in (1, 2, 7):
        oracle.threads(nt)
        runs.append(P.pcg_par(b, tol=1e-10, maxit=2000, history=True))
    for x, it, rel, h in runs[1:]:
        assert it == runs[0][1]
        assert np.array_equal(x, runs[0][0]) and np.array_equal(h, runs[0][3])
    x2, it2, rel2, h2 = runs[0]
    assert abs(it2 - it1) <= 1
    assert rel2 < 1e-10
    # the rounding differences of the dots stay at the 1e-13 level for the
    # first hundred iterations (later the recurrence amplifies them, as for
    # any change of summation order); the solutions agree to 1e-12
    assert np.max(np.abs(h2[:100] - h1[:100]) / h1[:100]) < 1e-11
    assert np.max(np.abs(x2 - x1)) <= 1e-12 * np.max(np.abs(x1))
    assert P.true_relres(b, x2) < 2e-10
