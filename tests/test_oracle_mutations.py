"""The pins are sharp: plant a plausible mistake in a copy of the oracle and
check that at least one pin fails.

Each mutation is a one-line textual change of ``oracle/hz_oracle.c`` (a
dropped term, a wrong sign, a wrong index, a transposed operand), compiled
to a temporary library on the CPU.  The battery below is a subset of the
pins of test_oracle_pins.py, re-run against the mutant.
"""
import json
import os
import subprocess

import numpy as np
import pytest

import oracle
from oracle import brute
from synth import pencils as P
from conftest import rel_err

SRC = os.path.join(os.path.dirname(oracle.__file__), "hz_oracle.c")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tiny_pencils.json")

MUTATIONS = {
    "sigma_always_plus": ("double sigma = h >= 0.0 ? 1.0 : -1.0;", "double sigma = 1.0;"),
    "tan2theta_drops_x_term": ("double num = sigma * (2.0 * u - (h11 + h22) * x);",
                               "double num = sigma * (2.0 * u);"),
    "alpha1_phase_not_conjugated": ("zc uv = conj(e1) * h12;", "zc uv = e1 * h12;"),
    "column_update_transposed": ("xp[i] = a * Zp[0] + b * Zp[2];", "xp[i] = a * Zp[0] + b * Zp[1];"),
    "J_ignored_in_dot": ("s += (J && J[i] < 0) ? -t : t;", "s += t;"),
    "prescale_wrong_row": ("Zp[2] = dq * z21; Zp[3] = dq * z22;", "Zp[2] = dp * z21; Zp[3] = dp * z22;"),
    "sin_gamma_sign_dropped": ("double sing = sigma * 2.0 * v / hv;", "double sing = 2.0 * v / hv;"),
    "cos_psi_cos_phi_swapped": ("(t * sing * cos2t)) / (2.0 * cpsi);", "(t * sing * cos2t)) / (2.0 * cphi);"),
    "lambda_not_squared_norm": ("lambda[j] = hf / gg;", "lambda[j] = hf / sqrt(gg);"),
    "row_update_not_conjugated": ("A[a + j * k] = conj(Zp[0]) * x + conj(Zp[2]) * y;",
                                  "A[a + j * k] = Zp[0] * x + Zp[2] * y;"),
    "round_robin_off_by_one": ("q = (r - k + (N - 1)) % (N - 1); }", "q = (r - k + N) % (N - 1); }"),
    "t_not_sqrt_1_minus_x2": ("double t = sqrt((1.0 - x) * (1.0 + x));", "double t = sqrt(1.0 - x);"),
    "cos_gamma_signed": ("double cosg = fabs(h) / hv;", "double cosg = h / hv;"),
    "s_criterion_dropped": ("int crit_s = cabs(s12) >= tol;", "int crit_s = 0;"),
    "block_update_skips_last_slot": ("for (long l = 0; l < kk; ++l)", "for (long l = 0; l < kk - 1; ++l)"),
}


def build_mutant(tmp_path, name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old}"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=gnu11", str(path),
                    "-o", str(so), "-lm"], check=True)
    return oracle.load(str(so))


def battery(lib):
    """Raise AssertionError on the first violated pin."""
    rng = np.random.default_rng(1)
    # Section 6.1: the pivot transformation diagonalizes both pivots
    for _ in range(200):
        A = rng.standard_normal((6, 2)) + 1j * rng.standard_normal((6, 2))
        B = rng.standard_normal((7, 2)) + 1j * rng.standard_normal((7, 2))
        Jp = np.array([1, 1, 1, 1, -1, -1.0])
        H = A.conj().T @ (Jp[:, None] * A)
        S = B.conj().T @ B
        rc, Z, _ = oracle.pivot(H[0, 0].real, H[1, 1].real, H[0, 1], S[0, 0].real,
                                S[1, 1].real, S[0, 1], lib=lib)
        assert rc == 1
        assert np.allclose(Z.conj().T @ S @ Z, np.eye(2), atol=1e-12)
        H3 = Z.conj().T @ H @ Z
        assert abs(H3[0, 1]) < 1e-12 * np.abs(H3).max()
    # Section 6.3: the strategy
    t = oracle.rr_table(8, lib=lib)
    seen = {tuple(x) for x in t.reshape(-1, 2).tolist()}
    assert len(seen) == 28 and all(len(set(s.ravel())) == 8 for s in t)
    # brute-force eigenvalues of tiny integer pencils (eq. 3.2)
    for case in json.load(open(GOLDEN))["cases"]:
        F = np.array(case["F_re"]) + 1j * np.array(case["F_im"])
        G = np.array(case["G_re"]) + 1j * np.array(case["G_im"])
        J = np.array(case["J"])
        lam = np.array([float(x) for x in case["lam"]])
        for method, kw in (("pointwise", {}), ("blocked", dict(w=2))):
            out = _solve(lib, F, G, J, method, kw)
            assert out["status"] == 0
            assert rel_err(out["lam"], lam).max() < 1e-12
    # known eigenvalues by construction (eq. 3.1)
    F, J, G, lam = P.known_pencil(116, 24, 32, 16, 8, 4, cond_x=10.0, hyper=0.7, n_hyper=32)
    for method, kw in (("pointwise", {}), ("blocked", dict(w=4))):
        out = _solve(lib, F, G, J, method, kw)
        assert rel_err(out["lam"], lam).max() < 1e-12
    # H already diagonal, S not: only the S part of eq. 6.12 can start work
    n = 8
    rows = rng.permutation(12)[:n]
    F = np.zeros((12, n), dtype=np.complex128)
    F[rows, np.arange(n)] = rng.uniform(0.5, 2, n)
    J = np.where(np.arange(12) % 3 == 0, -1, 1)
    G = rng.standard_normal((10, n)) + 1j * rng.standard_normal((10, n))
    lam = brute.generalized_eigenvalues(F, G, J, dps=30)
    out = _solve(lib, F, G, J, "pointwise", {})
    assert rel_err(out["lam"], lam).max() < 1e-12
    # S-orthonormal eigenvectors
    Vg = G @ out["V"]
    assert np.allclose(Vg.conj().T @ Vg, np.eye(n), atol=1e-10)
    # already (J-)orthogonal columns: nothing transforms, lambda = J a^2 / b^2
    b = rng.uniform(0.5, 2, n)
    G = P.haar_columns(rng, 10, n) * b[None, :]
    out = _solve(lib, F, G, J, "pointwise", {})
    assert np.allclose(out["lam"], J[rows] * np.abs(F[rows, np.arange(n)]) ** 2 / b ** 2, rtol=1e-13)


def _solve(lib, F, G, J, method, kw):
    run = oracle.pointwise if method == "pointwise" else oracle.blocked
    out = run(F, G, J, lib=lib, **kw)
    lam, V, _, _ = oracle.finalize(out["F"], out["G"], out["Z"], J, lib=lib)
    out.update(lam=lam, V=V)
    return out


def test_battery_passes_on_the_real_oracle():
    battery(oracle.load())


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    lib = build_mutant(tmp_path, name)
    with pytest.raises((AssertionError, RuntimeError, ValueError, np.linalg.LinAlgError)):
        battery(lib)
