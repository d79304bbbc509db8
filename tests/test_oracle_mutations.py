"""The pins are sharp: plant a plausible mistake in a copy of the oracle and
check that at least one pin fails.

Each mutation is a one-line textual change of ``oracle/hz_oracle.c`` or
``oracle/phase24_oracle.c`` (a dropped term, a wrong sign, a wrong index, a
transposed operand), compiled to a temporary library on the CPU.  The
batteries below are subsets of the pins of test_oracle_pins.py and
test_oracle_phase24.py, re-run against the mutant.
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
SRC24 = os.path.join(os.path.dirname(oracle.__file__), "phase24_oracle.c")
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


MUTATIONS24 = {
    "jqr_tau_sign_flipped": ("const double tau = -1.0 / (h + rh * r1 * (double)J[k]);",
                             "const double tau = 1.0 / (h + rh * r1 * (double)J[k]);"),
    "jqr_no_row_pivoting": ("if (J[k] != sg) {                                     /* row pivoting */",
                            "if (0) {"),
    "jqr_jdot_not_conjugated": ("s += (double)J[i] * (conj(a[i]) * b[i]);",
                                "s += (double)J[i] * (a[i] * b[i]);"),
    "jqr_c1_phase_dropped": ("const zc c1 = rh * eid;", "const zc c1 = rh;"),
    "jqr_2x2_block_times_R_not_Rstar": ("f2[i] = x * conj(R21) + y * conj(R22);",
                                        "f2[i] = x * R21 + y * R22;"),
    "jqr_reflector_skips_last_row": ("for (long i = k; i < m; ++i) g[i] += t * s[i];",
                                     "for (long i = k; i < m - 1; ++i) g[i] += t * s[i];"),
    "jqr_column_swap_not_recorded": ("long t = perm[k]; perm[k] = perm[jmax]; perm[jmax] = t;",
                                     "long t = perm[k]; (void)t;"),
    "qr_beta_doubled": ("const double beta = 1.0 / (nrm * (nrm + ax));",
                        "const double beta = 2.0 / (nrm * (nrm + ax));"),
    "qr_v_not_conjugated": ("for (long i = k; i < p; ++i) d += conj(v[i]) * g[i];",
                            "for (long i = k; i < p; ++i) d += v[i] * g[i];"),
    "lu_column_exchange_not_undone": ("zc t = x[k]; x[k] = x[colp[k]]; x[colp[k]] = t;",
                                      "(void)0;"),
    "lu_multiplier_not_divided": ("for (long i = k + 1; i < n; ++i) A[i + lda * k] /= piv;",
                                  "for (long i = k + 1; i < n; ++i) A[i + lda * k] *= 1.0;"),
}


def build_mutant(tmp_path, name, table=None, src_path=SRC):
    old, new = (table or MUTATIONS)[name]
    src = open(src_path).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old}"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    other = SRC24 if src_path == SRC else SRC
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=gnu11", str(path), other,
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


def battery24(lib):
    """Phase 2 / Phase 4 pins (Sections 5 and 7); AssertionError on the first violated one."""
    rng = np.random.default_rng(3)

    def herm(F, J):
        return F.conj().T @ (np.asarray(J, dtype=np.float64)[:, None] * F)

    # J = I: the hyperbolic QR is the QR with column pivoting
    F = (rng.standard_normal((30, 12)) + 1j * rng.standard_normal((30, 12))) * \
        10.0 ** rng.uniform(-2, 2, 12)[None, :]
    out = oracle.jqr(F, np.ones(30, dtype=np.int8), lib=lib)
    assert out["status"] == 0
    Rn = np.linalg.qr(F[:, out["perm"]], mode="r")
    assert np.allclose(np.abs(np.diagonal(out["R"])), np.abs(np.diagonal(Rn)), rtol=1e-12)
    assert np.all(np.diff(np.abs(np.diagonal(out["R"]))) <= 1e-12 * np.abs(out["R"]).max())
    # QR of G against numpy
    G = rng.standard_normal((20, 9)) + 1j * rng.standard_normal((20, 9))
    R = oracle.qr(G, lib=lib)
    Rn = np.linalg.qr(G, mode="r")
    ph = np.diagonal(R) / np.diagonal(Rn)
    assert np.allclose(R, ph[:, None] * Rn, atol=1e-13 * np.abs(Rn).max())
    # the Hermitian form and the inertia on indefinite factors (with 2x2 pivots)
    n2 = 0
    for t in range(12):
        J = np.where(rng.random(20) < 0.5, -1, 1).astype(np.int8)
        F = rng.standard_normal((20, 12)) + 1j * rng.standard_normal((20, 12))
        out = oracle.jqr(F, J, lib=lib)
        assert out["status"] == 0
        H0 = herm(F[:, out["perm"]], J)
        assert np.max(np.abs(herm(out["R"], out["J"]) - H0)) <= 1e-13 * np.linalg.norm(F) ** 2
        assert np.all(np.tril(out["R"], -2) == 0)
        assert np.count_nonzero(out["J"] < 0) == np.count_nonzero(np.linalg.eigvalsh(herm(F, J)) < 0)
        n2 += out["n2x2"]
    assert n2 > 0
    # X = Z^{-1}
    Z = rng.standard_normal((15, 15)) + 1j * rng.standard_normal((15, 15))
    X = oracle.inverse(Z, lib=lib)
    assert np.max(np.abs(X - np.linalg.inv(Z))) <= 1e-10 * np.abs(X).max()


def test_battery_passes_on_the_real_oracle():
    battery(oracle.load())


def test_battery24_passes_on_the_real_oracle():
    battery24(oracle.load())


@pytest.mark.parametrize("name", sorted(MUTATIONS24))
def test_planted_phase24_mistake_is_caught(tmp_path, name):
    lib = build_mutant(tmp_path, name, MUTATIONS24, SRC24)
    with pytest.raises((AssertionError, RuntimeError, ValueError, np.linalg.LinAlgError)):
        battery24(lib)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    lib = build_mutant(tmp_path, name)
    with pytest.raises((AssertionError, RuntimeError, ValueError, np.linalg.LinAlgError)):
        battery(lib)
