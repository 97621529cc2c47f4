"""Mutation check of the oracle's pins: each plausible mistake below makes at
least one pin fail.  In the C oracle a mistake is one textual change in a
copy compiled into a temporary library (loaded through NBO_LIB in a child
process); in the Python parts (Schwarz, network, flexible CG) it is a changed
copy of one function patched in for the test.  The committed oracle is never
modified."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "nb_oracle.c")
PINS = [os.path.join(ROOT, "tests", f)
        for f in ("test_oracle_gll.py", "test_oracle_mesh.py", "test_oracle_operator.py",
                  "test_oracle_vprec.py")]

MUTANTS = {
    "transposed derivative matrix": ("D[i * n + j] = v;", "D[j * n + i] = v;"),
    "GLL weight with P_N to the first power": ("w[j] = 2.0 / (N * (N + 1.0) * pN * pN);",
                                               "w[j] = 2.0 / (N * (N + 1.0) * pN);"),
    "dropped G_rs term of the operator": ("wr[q] = grr * ur + grs * us + grt * ut;",
                                          "wr[q] = grr * ur + grt * ut;"),
    "cofactor sign of the inverse Jacobian": (
        "Minv[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) / det;",
        "Minv[0][1] = (M[0][1] * M[2][2] - M[0][2] * M[2][1]) / det;"),
    "dropped Dirichlet mask": ("u[l] = (mask && !mask[g]) ? 0.0 : work[g];", "u[l] = work[g];"),
    "inverted CG beta": ("double beta = (iter == 1) ? 0.0 : rtz1 / rtz2;",
                         "double beta = (iter == 1) ? 0.0 : rtz2 / rtz1;"),
    "factor 2 dropped in the Jacobi diagonal": (
        "s += 2.0 * D[i * n + i] * D[j * n + j] * Ge[1 * n3 + q];",
        "s += D[i * n + i] * D[j * n + j] * Ge[1 * n3 + q];"),
    "sign of the deformation along y": ("X[1 * n3 + q] = y0 + d;", "X[1 * n3 + q] = y0 - d;"),
    "VPREC ties rounded up instead of to even": (
        "if (rem > half || (rem == half && ((b >> drop) & 1))) b += (uint64_t)1 << drop;",
        "if (rem >= half) b += (uint64_t)1 << drop;"),
    "MCA perturbation one bit too wide": ("const double r = x + ldexp(emu_u01(&m) - 0.5, e - t);",
                                          "const double r = x + ldexp(emu_u01(&m) - 0.5, e - t + 1);"),
}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique: {old}"
    mut = tmp_path / "nb_oracle_mutant.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libnb_oracle_mutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                    "-shared", "-o", str(lib), str(mut), "-lm"], check=True)
    env = dict(os.environ, NBO_LIB=str(lib))
    out = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                          "-m", "not gpu", *PINS], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode != 0, f"no pin failed for: {name}\n{out.stdout[-2000:]}"
    assert "failed" in out.stdout


# ---- planted mistakes in the Python parts (Schwarz oracle) ----

def _schwarz_pins():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "pins_schwarz", os.path.join(ROOT, "tests", "test_oracle_schwarz.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_planted_mistakes_in_the_schwarz_oracle_fail_a_pin(monkeypatch):
    import numpy as np
    from oracle import schwarz
    pins = _schwarz_pins()
    good_coarse_1d, good_local_solve = schwarz.coarse_1d, schwarz.local_solve
    good_coarse_operator = schwarz.coarse_operator

    def mirrored_hats(N, n_d):  # hat of vertex v falling on element v instead of rising
        R1, _, _ = good_coarse_1d(N, n_d)
        xi, _ = schwarz.gll(N)
        R1 = np.zeros_like(R1)
        for v in range(n_d - 1):
            for i in range(N + 1):
                R1[v, v * N + i] = (1.0 - xi[i]) / 2.0
                R1[v, (v + 1) * N + i] = (1.0 + xi[i]) / 2.0
        K, M = schwarz.gll_1d(N)
        L = 1.0 / n_d
        ng = n_d * N + 1
        Kf, Mf = np.zeros((ng, ng)), np.zeros((ng, ng))
        for e in range(n_d):
            s = slice(e * N, e * N + N + 1)
            Kf[s, s] += (2.0 / L) * K
            Mf[s, s] += (L / 2.0) * M
        return R1, R1 @ Kf @ R1.T, R1 @ Mf @ R1.T

    monkeypatch.setattr(schwarz, "coarse_1d", mirrored_hats)
    with pytest.raises(AssertionError):
        pins.test_coarse_1d_matrices_are_the_q1_matrices(3)
    monkeypatch.setattr(schwarz, "coarse_1d", good_coarse_1d)

    def dropped_z_eigenvalue(fdm, rt):  # scaling by 1 / (lx + ly) only
        (Sx, lx, ax), (Sy, ly, ay), (Sz, lz, az) = fdm
        return good_local_solve(((Sx, lx, ax), (Sy, ly, ay), (Sz, 0.0 * lz, az)), rt)

    monkeypatch.setattr(schwarz, "local_solve", dropped_z_eigenvalue)
    with pytest.raises(AssertionError):
        pins.test_fast_diagonalisation_equals_dense_solve((1, 1, 1))
    monkeypatch.setattr(schwarz, "local_solve", good_local_solve)

    def mass_for_stiffness(box):  # Bz(x)By(x)Bx in the third term
        (_, Kx, Mx), (_, Ky, My), (_, Kz, Mz) = schwarz.coarse_parts(box)
        return (np.kron(Mz, np.kron(My, Kx)) + np.kron(Mz, np.kron(Ky, Mx)) +
                np.kron(Mz, np.kron(My, Mx)))

    monkeypatch.setattr(schwarz, "coarse_operator", mass_for_stiffness)
    with pytest.raises(AssertionError):
        pins.test_coarse_operator_is_the_galerkin_product()
    monkeypatch.setattr(schwarz, "coarse_operator", good_coarse_operator)


# ---- planted mistakes in the network oracle ----

def test_planted_mistakes_in_the_network_oracle_fail_a_pin(monkeypatch):
    import importlib.util
    import numpy as np
    from oracle import mlp
    spec = importlib.util.spec_from_file_location(
        "pins_mlp", os.path.join(ROOT, "tests", "test_oracle_mlp.py"))
    pins = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(pins)
    good_backward, good_grad = mlp.backward, mlp.gelu_grad

    def output_use_dropped(params, X, T):  # W's gradient only through its input use
        g = good_backward(params, X, T)
        Y, (X_, Z, H) = mlp.forward(params, X)
        dY = 2.0 * (Y - T) / Y.size
        g["W"] = g["W"] - dY.T @ (H * params["a"])
        return g

    monkeypatch.setattr(mlp, "backward", output_use_dropped)
    with pytest.raises(AssertionError):
        pins.test_backward_matches_finite_differences((8, 4, 5))
    monkeypatch.setattr(mlp, "backward", good_backward)

    def tanh_term_sign(z):  # 0.5 (1 - t) instead of 0.5 (1 + t)
        t = np.tanh(mlp._C * (z + 0.044715 * z ** 3))
        return good_grad(z) - t

    monkeypatch.setattr(mlp, "gelu_grad", tanh_term_sign)
    with pytest.raises(AssertionError):
        pins.test_backward_matches_finite_differences((8, 4, 5))


# ---- planted mistakes in the flexible CG ----

FCG_MUTANTS = {
    "wrong sign of the flexible-CG beta": ("beta = -self.glsc3(z, w) / pap_prev",
                                           "beta = self.glsc3(z, w) / pap_prev"),
    "flexible-CG beta dropped": ("p = z + beta * p", "p = z + 0.0 * beta * p"),
    "residual updated without alpha": ("r = r - alpha * w", "r = r - w"),
}


@pytest.mark.parametrize("name", sorted(FCG_MUTANTS))
def test_planted_mistakes_in_the_flexible_cg_fail_a_pin(name, monkeypatch):
    """One textual change in a copy of Problem.fcg (the committed oracle is
    untouched): the step-by-step pin of flexible CG under a nonlinear
    preconditioner fails, while the unchanged copy passes it."""
    import importlib.util
    import inspect
    import math
    import textwrap

    import numpy as np

    import oracle
    from workloads import Box
    spec = importlib.util.spec_from_file_location(
        "pins_operator", os.path.join(ROOT, "tests", "test_oracle_operator.py"))
    pins = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(pins)
    src = textwrap.dedent(inspect.getsource(oracle.Problem.fcg))
    old, new = FCG_MUTANTS[name]
    assert src.count(old) == 1
    box = Box(2, 2, 1, 5, 0.05)
    for text, fails in ((src, False), (src.replace(old, new), True)):
        ns = {"np": np, "math": math}
        exec(text, ns)
        monkeypatch.setattr(oracle.Problem, "fcg", ns["fcg"])
        if fails:
            with pytest.raises(AssertionError):
                pins.test_flexible_cg_with_a_nonlinear_preconditioner(box)
        else:
            pins.test_flexible_cg_with_a_nonlinear_preconditioner(box)
