"""Pins of the Phase 2 / Phase 4 oracle (arXiv 1907.08560, Sections 5 and 7).

Every check is a property the result must have, a special case that reduces
to a textbook or library routine, or an extended-precision brute force:

- the hyperbolic QR with J = +-I is the QR with column pivoting (the
  diagonal pivoting of Section 5.2 picks the column of largest norm, and the
  Bunch-Kaufman test never asks for a 2x2 pivot), so |diag R| and the column
  order match LAPACK's pivoted QR (scipy);
- the Householder QR of G matches numpy's R up to a unitary diagonal;
- F^* J F is preserved (the definition of the (J, I) URV factorization),
  the factor is block upper triangular with blocks of order 1 or 2, and the
  number of -1 signs left in J is the negative inertia of F^* J F
  (Sylvester's law);
- the generalized eigenvalues of the shortened pencil equal those of the
  tall pencil (50-digit brute force);
- X = Z^{-1} matches numpy's inverse; the GHSVD of a pencil with known
  eigenvalues has Sigma_F^2 + Sigma_G^2 = I, signed ratios equal to the
  eigenvalues, and X^* Sigma_G^2 X = G^* G, X^* J Sigma_F^2 X = F^* J F
  (eq. 3.1 and the derivation of eq. 3.2).
"""
import numpy as np
import pytest

import oracle
from oracle import brute
from synth import pencils as P

EPS = 2.0 ** -53


def cgauss(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


def hermitian_form(F, J):
    return F.conj().T @ (np.asarray(J, dtype=np.float64)[:, None] * F)


def check_urv_invariants(F, J, out, tol=1e-13):
    R, Js, perm = out["R"], out["J"], out["perm"]
    n = F.shape[1]
    assert sorted(perm.tolist()) == list(range(n))
    H0 = hermitian_form(F[:, perm], J)
    H1 = hermitian_form(R, Js)
    scale = np.linalg.norm(F) ** 2
    assert np.max(np.abs(H1 - H0)) <= tol * scale
    # block upper triangular, diagonal blocks of order 1 or 2, zeros below n
    assert np.all(np.tril(R, -2) == 0)
    assert np.all(out["full"][n:, :] == 0)
    sub = np.count_nonzero(np.diagonal(R, -1))
    assert sub <= out["n2x2"]
    k = 0
    while k < n - 1:                                  # no two adjacent 2x2 blocks overlap
        if R[k + 1, k] != 0:
            assert k + 2 >= n or R[k + 2, k + 1] == 0
            k += 2
        else:
            k += 1
    assert set(np.unique(Js).tolist()) <= {-1, 1}


@pytest.mark.parametrize("sign", [1, -1])
def test_jqr_with_definite_J_is_pivoted_qr(sign):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(11)
    F = cgauss(rng, 40, 25) * 10.0 ** rng.uniform(-2, 2, 25)[None, :]
    J = np.full(40, sign, dtype=np.int8)
    out = oracle.jqr(F, J)
    assert out["status"] == 0 and out["n2x2"] == 0
    _, Rs, piv = scipy_linalg.qr(F, mode="economic", pivoting=True)
    assert out["perm"].tolist() == piv.tolist()
    d = np.abs(np.diagonal(out["R"]))
    assert np.allclose(d, np.abs(np.diagonal(Rs)), rtol=1e-12)
    # with a definite J every reflector is unitary: R agrees with scipy's up to row phases
    ph = np.diagonal(out["R"]) / np.diagonal(Rs)
    assert np.allclose(np.abs(ph), 1.0, rtol=1e-12)
    assert np.allclose(out["R"], ph[:, None] * Rs, atol=1e-12 * np.abs(Rs).max())
    assert np.all(out["J"] == sign)


def test_householder_qr_matches_numpy():
    rng = np.random.default_rng(12)
    G = cgauss(rng, 50, 30) * 10.0 ** rng.uniform(-3, 3, 30)[None, :]
    R = oracle.qr(G)
    Rn = np.linalg.qr(G, mode="r")
    assert np.all(np.tril(R, -1) == 0)
    ph = np.diagonal(R) / np.diagonal(Rn)
    assert np.allclose(np.abs(ph), 1.0, rtol=1e-12)
    assert np.allclose(R, ph[:, None] * Rn, atol=1e-13 * np.abs(Rn).max())


@pytest.mark.parametrize("seed,m,n,m_minus", [(1, 30, 20, 8), (2, 45, 30, 20), (3, 21, 21, 7),
                                              (4, 64, 16, 60), (5, 33, 17, 16)])
def test_jqr_preserves_the_hermitian_form(seed, m, n, m_minus):
    F, J, _ = P.svd_pencil(7000 + seed, m, m + 4, n, m_minus, (1e-2, 1e2), (1e-2, 1e2),
                           permute_j=bool(seed % 2))
    out = oracle.jqr(F, J)
    assert out["status"] == 0
    check_urv_invariants(F, J, out)
    # Sylvester: the signs left in J are the inertia of F^* J F
    ev = np.linalg.eigvalsh(hermitian_form(F, J))
    assert np.count_nonzero(out["J"] < 0) == np.count_nonzero(ev < 0)
    # a J-unitary left factor keeps the sign multiset of the rows it used
    assert np.count_nonzero(out["J_full"] < 0) == np.count_nonzero(J < 0)


def test_forced_2x2_pivot():
    # both columns J-isotropic, their J-product nonzero: the diagonal test fails and
    # Section 5.2 has to take a 2x2 pivot
    J = np.array([1, 1, -1, -1], dtype=np.int8)
    F = np.zeros((4, 2), dtype=np.complex128)
    F[0, 0] = F[2, 0] = 1.0
    F[1, 1] = 1.0
    F[2, 1] = 1.0j
    out = oracle.jqr(F, J)
    assert out["status"] == 0 and out["n2x2"] == 1
    check_urv_invariants(F, J, out)
    assert sorted(out["J"].tolist()) == [-1, 1]          # inertia of [[0, -i], [i, 0]]


def test_2x2_pivots_on_random_indefinite_factors():
    rng = np.random.default_rng(13)
    seen = 0
    for t in range(20):
        m, n = 24, 16
        J = np.where(rng.random(m) < 0.5, -1, 1).astype(np.int8)
        F = cgauss(rng, m, n)
        out = oracle.jqr(F, J)
        assert out["status"] == 0
        check_urv_invariants(F, J, out)
        seen += out["n2x2"]
    assert seen > 0


def test_jqr_breakdown_and_zero_column():
    J = np.array([1, -1], dtype=np.int8)
    iso = np.array([[1.0], [1.0]], dtype=np.complex128)    # f^* J f = 0, f != 0
    assert oracle.jqr(iso, J)["status"] == -4
    out = oracle.jqr(np.zeros((3, 1), dtype=np.complex128), np.array([1, -1, 1], dtype=np.int8))
    assert out["status"] == 0 and np.all(out["R"] == 0)


@pytest.mark.parametrize("seed", [0, 1])
def test_shortened_pencil_has_the_same_eigenvalues(seed):
    F, J, G = P.svd_pencil(7100 + seed, 11, 13, 7, 4, (1e-2, 1e2), (1e-2, 1e2))
    u = oracle.urv(F, G, J)
    assert u["status"] == 0
    lam_tall = brute.generalized_eigenvalues(F, G, J, dps=50)
    lam_sq = brute.generalized_eigenvalues(u["F"], u["G"], u["J"], dps=50)
    assert np.max(np.abs(lam_sq - lam_tall) / np.abs(lam_tall)) < 1e-11
    # and the HZ iteration on the square pencil finds them
    out = oracle.solve(u["F"], u["G"], u["J"], method="blocked", w=2)
    assert out["status"] == 0
    assert np.max(np.abs(np.sort(out["lam"]) - lam_tall) / np.abs(lam_tall)) < 1e-11


def test_lu_complete_pivoting_and_inverse():
    rng = np.random.default_rng(14)
    Z = cgauss(rng, 30, 30) * 10.0 ** rng.uniform(-2, 2, 30)[None, :]
    LU, rowp, colp, rc = oracle.lu_complete(Z)
    assert rc == 0
    L = np.tril(LU, -1) + np.eye(30)
    U = np.triu(LU)
    assert np.max(np.abs(L)) <= 1.0 + 1e-15              # complete pivoting: |l_ij| <= 1
    assert abs(U[0, 0]) == np.abs(Z).max()               # the first pivot is the largest entry
    d = np.abs(np.diagonal(U))
    for k in range(30):                                   # each pivot dominates its row of U
        assert np.all(np.abs(U[k, k:]) <= d[k] * (1 + 1e-14))
    X = oracle.inverse(Z)
    Xn = np.linalg.inv(Z)
    assert np.max(np.abs(X - Xn)) <= 1e-10 * np.abs(Xn).max()
    # backward-stable solve of Z X = I: residual of order n eps |Z| |X|
    bound = 30 * EPS * np.max(np.abs(Z) @ np.abs(X))
    assert np.max(np.abs(Z @ X - np.eye(30))) < 10 * bound


def test_lu_singular():
    Z = np.ones((3, 3), dtype=np.complex128)
    assert oracle.lu_complete(Z)[3] == -5


def test_phase4_recovers_the_constructed_right_factor():
    # F = U_F E diag(a) X0, G = U_G diag(b) X0 (eq. 3.1) with known eigenvalues
    n = 10
    F, J, G, lam = P.known_pencil(7200, 16, 18, n, 6, 3, cond_x=20.0)
    out = oracle.solve(F, G, J, method="pointwise")
    assert out["status"] == 0
    g = oracle.ghsvd(F, G, J, out["F"], out["G"], out["Z"])
    assert g["err_F"] < 1e-13 and g["err_G"] < 1e-13
    assert np.allclose(g["sigma_f"] ** 2 + g["sigma_g"] ** 2, 1.0, rtol=1e-14)
    # signed squares of the generalized hyperbolic singular values are the eigenvalues
    Jsign = np.sign(out["lam"])
    assert np.allclose(np.sort(Jsign * (g["sigma_f"] / g["sigma_g"]) ** 2), lam, rtol=1e-12)
    # H = X^* Sigma_F^T J Sigma_F X and S = X^* Sigma_G^T Sigma_G X (the derivation of eq. 3.2)
    X = g["X"]
    SG2 = g["sigma_g"] ** 2
    SF2 = Jsign * g["sigma_f"] ** 2
    S = G.conj().T @ G
    H = hermitian_form(F, J)
    assert np.max(np.abs(X.conj().T @ (SG2[:, None] * X) - S)) < 1e-12 * np.abs(S).max()
    assert np.max(np.abs(X.conj().T @ (SF2[:, None] * X) - H)) < 1e-12 * np.abs(H).max()


def test_phase4_errors_small_after_phase2_and_phase3():
    F, J, G = P.svd_pencil(7300, 48, 64, 32, 8, (1e-3, 1e3), (1e-3, 1e3))
    u = oracle.urv(F, G, J)
    out = oracle.solve(u["F"], u["G"], u["J"], method="blocked", w=4)
    assert out["status"] == 0
    g = oracle.ghsvd(u["F"], u["G"], u["J"], out["F"], out["G"], out["Z"])
    # the paper reports 8e-14 .. 8e-13 (Section 7.1) on its datasets
    assert g["err_F"] < 1e-12 and g["err_G"] < 1e-12
