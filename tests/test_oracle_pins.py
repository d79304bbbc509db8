"""Pins of the FP64 CPU oracle to facts fixed by the paper and by mathematics.

Nothing here retypes the oracle's formulas: every check is a property the
result must have (eq. 3.1-3.2, Section 6.1 of arXiv 1907.08560), an exact
answer known by construction, or an extended-precision brute force.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import brute
from synth import pencils as P
from conftest import eig_tol, eig_tol_vec, rel_err

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tiny_pencils.json")


def random_pivot(rng, m=6, p=7, neg=2, scale_f=1.0, scale_g=1.0):
    A = (rng.standard_normal((m, 2)) + 1j * rng.standard_normal((m, 2))) * scale_f
    B = (rng.standard_normal((p, 2)) + 1j * rng.standard_normal((p, 2))) * scale_g
    A[:, 1] *= 10.0 ** rng.uniform(-3, 3)
    B[:, 1] *= 10.0 ** rng.uniform(-3, 3)
    J = np.ones(m)
    J[:neg] = -1
    H = A.conj().T @ (J[:, None] * A)
    S = B.conj().T @ B
    return H, S


def check_diagonalizes(H, S, Z, tol=2e-14):
    S3 = Z.conj().T @ S @ Z
    H3 = Z.conj().T @ H @ Z
    # Section 6.1.4: after the transformation the S pivot is the identity
    assert np.max(np.abs(S3 - np.eye(2))) <= tol * 10, S3
    # ... and the H pivot is diagonal relative to its diagonal
    scale = np.sqrt(abs(H3[0, 0].real * H3[1, 1].real)) + np.max(np.abs(H3)) * 1e-3
    assert abs(H3[0, 1]) <= tol * 50 * max(scale, np.max(np.abs(H3))), H3


# ---------------------------------------------------------------------------
# Section 6.1: the 2x2 transformation
# ---------------------------------------------------------------------------

def test_pivot_diagonalizes_random_pairs():
    rng = np.random.default_rng(1)
    for _ in range(4000):
        H, S = random_pivot(rng, neg=int(rng.integers(0, 4)))
        rc, Z, big = oracle.pivot(H[0, 0].real, H[1, 1].real, H[0, 1], S[0, 0].real,
                                  S[1, 1].real, S[0, 1])
        assert rc == 1 and big == 1
        check_diagonalizes(H, S, Z)


def test_pivot_invariants_over_1e5_random_pivots():
    # eq. 6.1-6.11 on 10^5 pivots of random factors (signatures with 0-3
    # negative rows, column scales over six decades): Z'^* S Z' = I and
    # Z'^* H Z' diagonal relative to its diagonal, checked all at once
    rng = np.random.default_rng(7)
    N = 100_000
    A = rng.standard_normal((N, 6, 2)) + 1j * rng.standard_normal((N, 6, 2))
    B = rng.standard_normal((N, 7, 2)) + 1j * rng.standard_normal((N, 7, 2))
    A[:, :, 1] *= (10.0 ** rng.uniform(-3, 3, N))[:, None]
    B[:, :, 1] *= (10.0 ** rng.uniform(-3, 3, N))[:, None]
    J = np.ones((N, 6))
    J[np.arange(6)[None, :] < rng.integers(0, 4, N)[:, None]] = -1.0
    H = np.einsum("nri,nr,nrj->nij", A.conj(), J, A)
    S = np.einsum("nri,nrj->nij", B.conj(), B)
    lib = oracle.load()
    Z = np.empty((N, 2, 2), dtype=np.complex128)
    for t in range(N):
        rc, Z[t], big = oracle.pivot(H[t, 0, 0].real, H[t, 1, 1].real, H[t, 0, 1], S[t, 0, 0].real,
                                     S[t, 1, 1].real, S[t, 0, 1], lib=lib)
        assert rc == 1 and big == 1, t
    S3 = np.einsum("nki,nkl,nlj->nij", Z.conj(), S, Z)
    H3 = np.einsum("nki,nkl,nlj->nij", Z.conj(), H, Z)
    assert np.max(np.abs(S3 - np.eye(2)[None])) <= 2e-13
    scale = np.maximum(np.sqrt(np.abs(H3[:, 0, 0].real * H3[:, 1, 1].real)) + 1e-3 * np.abs(H3).max(axis=(1, 2)),
                       np.abs(H3).max(axis=(1, 2)))
    assert np.all(np.abs(H3[:, 0, 1]) <= 1e-12 * scale)


def test_pivot_exceptional_case_already_diagonal():
    # Section 6.1.6: h_pq = s_pq = 0 gives no transformation
    rc, Z, big = oracle.pivot(2.0, -3.0, 0.0, 4.0, 5.0, 0.0)
    assert rc == 0 and big == 0


def test_pivot_x_zero_is_ordinary_jacobi_rotation():
    # Section 6.1.6: s_pq = 0 -> Z^ is a Jacobi rotation diagonalizing H^_0;
    # with s_pp = s_qq = 1 the transformation is unitary.
    rng = np.random.default_rng(2)
    for _ in range(200):
        hpp, hqq = rng.standard_normal(2) * 5
        hpq = complex(*rng.standard_normal(2))
        rc, Z, big = oracle.pivot(hpp, hqq, hpq, 1.0, 1.0, 0.0)
        assert rc == 1
        assert np.allclose(Z.conj().T @ Z, np.eye(2), atol=1e-14)
        H = np.array([[hpp, hpq], [np.conj(hpq), hqq]])
        D = Z.conj().T @ H @ Z
        assert abs(D[0, 1]) < 1e-13 * np.max(np.abs(H))
        # the eigenvalues of the 2x2 Hermitian matrix are on the diagonal
        assert np.allclose(np.sort(np.diag(D).real), np.linalg.eigvalsh(H), atol=1e-13 * np.max(np.abs(H)))


def test_pivot_h_v_zero_case_is_R1_D2():
    # Section 6.1.6: h = v = 0 (equal prescaled diagonals, arg h_pq = arg s_pq)
    # -> R1^ alone diagonalizes H^_0 as well; Z^ = R1^ D2^ must still make
    # S^ the identity and H^ diagonal.
    # (phases 1, -1, i, -i keep v exactly zero in floating point; with any
    # other phase v is a rounding error and the general formulas apply)
    rng = np.random.default_rng(3)
    for it in range(200):
        x = rng.uniform(0.05, 0.9)
        ph = [1.0, -1.0, 1j, -1j][it % 4]
        hd = rng.standard_normal() * 3
        r = rng.standard_normal() * 2
        H = np.array([[hd, r * ph], [np.conj(r * ph), hd]])
        S = np.array([[1.0, x * ph], [np.conj(x * ph), 1.0]])
        rc, Z, big = oracle.pivot(hd, hd, r * ph, 1.0, 1.0, x * ph)
        assert rc == 1 and big == 1
        check_diagonalizes(H, S, Z)
        # R1^ (phi_1 = -pi/4) has entries of equal modulus; D2^ scales columns
        col_ratio = np.abs(Z[:, 0]) / np.abs(Z[:, 1])
        assert np.allclose(np.abs(Z[0, 0]), np.abs(Z[1, 0]))
        assert np.allclose(col_ratio, np.sqrt((1 - x) / (1 + x)))


def test_pivot_near_exceptional_case_still_diagonalizes():
    # h = 0 with v a rounding error: the general branch must still work
    rng = np.random.default_rng(5)
    for _ in range(200):
        x = rng.uniform(0.05, 0.9)
        ph = np.exp(1j * rng.uniform(-np.pi, np.pi))
        hd, r = rng.standard_normal(2) * 3
        H = np.array([[hd, r * ph], [np.conj(r * ph), hd]])
        S = np.array([[1.0, x * ph], [np.conj(x * ph), 1.0]])
        rc, Z, big = oracle.pivot(hd, hd, r * ph, 1.0, 1.0, x * ph)
        assert rc == 1
        check_diagonalizes(H, S, Z)


def test_pivot_criterion_skips_converged_pairs():
    # eq. 6.12: an off-diagonal far below eps*sqrt(n) relative is not transformed
    rc, _, _ = oracle.pivot(1.0, 2.0, 1e-20, 1.0, 1.0, 1e-20, n=64)
    assert rc == 0
    rc, _, _ = oracle.pivot(1.0, 2.0, 1e-6, 1.0, 1.0, 0.0, n=64)
    assert rc == 1


def test_pivot_small_transformation_flag():
    # Section 6.1.7: a transformation with cos(phi) = cos(psi) = 1 is "small";
    # an off-diagonal of relative size ~1e-9 gives such a transformation.
    rc, Z, big = oracle.pivot(1.0, 3.0, 1e-9, 1.0, 1.0, 0.0, n=64)
    assert rc == 1 and big == 0
    assert Z[0, 0] == 1.0 and Z[1, 1] == 1.0
    rc, Z, big = oracle.pivot(1.0, 3.0, 1e-3, 1.0, 1.0, 0.0, n=64)
    assert rc == 1 and big == 1


def test_pivot_rank_deficient_is_an_error():
    rc, _, _ = oracle.pivot(1.0, 2.0, 0.5, 1.0, 1.0, 1.0)
    assert rc < 0
    rc, _, _ = oracle.pivot(1.0, 2.0, 0.5, 0.0, 1.0, 0.0)
    assert rc < 0


# ---------------------------------------------------------------------------
# Section 6.3: the strategy and Section 6.4.1: the partition
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("N", [2, 4, 6, 8, 16, 64])
def test_round_robin_is_a_parallel_cyclic_strategy(N):
    t = oracle.rr_table(N)
    seen = set()
    for step in t:
        idx = step.ravel().tolist()
        assert len(set(idx)) == N          # disjoint pairs within a step
        for a, b in step:
            assert 0 <= a < b < N
            seen.add((a, b))
    assert len(seen) == N * (N - 1) // 2   # every pair exactly once per sweep


@pytest.mark.parametrize("n,w", [(2048, 32), (64, 8), (65, 8), (1000, 32), (7, 2), (3, 1), (257, 16)])
def test_partition(n, w):
    off = oracle.partition(n, w)
    widths = np.diff(off)
    assert off[0] == 0 and off[-1] == n
    assert len(widths) % 2 == 0
    assert widths.max() - widths.min() <= 1 and widths.min() >= 1
    assert np.all(np.diff(widths) <= 0)    # non-increasing
    assert widths.max() <= max(w, (n + 1) // 2)


# ---------------------------------------------------------------------------
# Whole solver: brute force, closed forms, invariants
# ---------------------------------------------------------------------------

def _golden_cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
@pytest.mark.parametrize("method", ["pointwise", "blocked_w1", "blocked_w2"])
def test_golden_tiny_pencils(case, method):
    F = np.array(case["F_re"]) + 1j * np.array(case["F_im"])
    G = np.array(case["G_re"]) + 1j * np.array(case["G_im"])
    J = np.array(case["J"])
    lam = np.array([float(x) for x in case["lam"]])
    if method == "pointwise":
        out = oracle.solve(F, G, J)
    else:
        out = oracle.solve(F, G, J, method="blocked", w=int(method[-1]))
    assert out["status"] == 0
    assert rel_err(out["lam"], lam).max() < 1e-13


@pytest.mark.parametrize("seed,m,p,n,neg", [(20, 10, 12, 7, 3), (21, 14, 14, 12, 5),
                                            (22, 9, 11, 8, 0), (23, 16, 20, 11, 8)])
def test_brute_force_random_pencils(seed, m, p, n, neg):
    F, J, G = P.svd_pencil(seed, m, p, n, neg, (1e-2, 1e2), (1e-2, 1e2))
    lam = brute.generalized_eigenvalues(F, G, J, dps=40)
    for method, kw in (("pointwise", {}), ("blocked", dict(w=2)), ("blocked", dict(w=3)),
                       ("blocked", dict(w=2, inner_sweeps=30))):
        out = oracle.solve(F, G, J, method=method, **kw)
        assert out["status"] == 0, (method, kw)
        tol = eig_tol_vec(F, G, J, out["lam"], out["F"])
        assert np.all(rel_err(out["lam"], lam) < tol), (method, kw)
        # signs follow J: the number of negative eigenvalues is the negative
        # inertia of H (Sylvester), as counted by the brute force
        assert (out["lam"] < 0).sum() == (lam < 0).sum()


@pytest.mark.parametrize("n,neg_cols,hyper", [(16, 4, 0.0), (40, 10, 0.7), (64, 16, 0.3), (33, 0, 0.0)])
def test_known_eigenvalue_pencils(n, neg_cols, hyper):
    m, p = n + n // 2, 2 * n
    F, J, G, lam = P.known_pencil(100 + n, m, p, n, m // 3 if neg_cols else 0, neg_cols,
                                  cond_x=10.0, hyper=hyper, n_hyper=2 * n)
    for method, kw in (("pointwise", {}), ("blocked", dict(w=4)), ("blocked", dict(w=5))):
        out = oracle.solve(F, G, J, method=method, **kw)
        assert out["status"] == 0
        assert rel_err(out["lam"], lam).max() < 1e-12, (method, kw)


def test_gsvd_special_case_identity_signature():
    # J = I, G = I: the eigenvalues are the squared singular values of F
    rng = np.random.default_rng(7)
    F = rng.standard_normal((30, 20)) + 1j * rng.standard_normal((30, 20))
    G = np.eye(20, dtype=np.complex128)
    out = oracle.solve(F, G, None)
    s = np.linalg.svd(F, compute_uv=False)
    assert rel_err(out["lam"], s ** 2).max() < 1e-13
    # G = I with a signature: the eigenvalues of F^* J F (hyperbolic SVD)
    J = np.ones(30, dtype=np.int8)
    J[::3] = -1
    out = oracle.solve(F, G, J, method="blocked", w=3)
    ev = np.linalg.eigvalsh(F.conj().T @ (J[:, None] * F))
    assert rel_err(out["lam"], ev).max() < 1e-11


def test_n_equals_one():
    F = np.array([[1 + 2j], [3.0], [-1j]])
    G = np.array([[2.0], [1j]])
    J = np.array([1, -1, 1])
    out = oracle.solve(F, G, J)
    hf = abs(1 + 2j) ** 2 - 9 + 1
    assert out["sweeps"] == 0
    assert abs(out["lam"][0] - hf / 5.0) < 1e-15


def test_already_orthogonal_columns_take_one_sweep():
    # F = E diag(a) (columns on distinct rows), G with orthogonal columns:
    # every pivot is diagonal, nothing is transformed, lambda_j = J[r_j] a^2/b^2
    n, m, p = 10, 15, 12
    rng = np.random.default_rng(4)
    rows = rng.permutation(m)[:n]
    a = rng.uniform(0.5, 2, n)
    F = np.zeros((m, n), dtype=np.complex128)
    F[rows, np.arange(n)] = a * np.exp(1j * rng.uniform(0, 6, n))
    J = np.where(rng.uniform(size=m) < 0.4, -1, 1)
    b = rng.uniform(0.5, 2, n)
    G = P.haar_columns(rng, p, n) * b[None, :]
    for method, kw in (("pointwise", {}), ("blocked", dict(w=2))):
        out = oracle.solve(F, G, J, method=method, **kw)
        assert out["sweeps"] == 1 and out["counts"][0, 0] == 0
        assert np.allclose(out["lam"], J[rows] * a ** 2 / b ** 2, rtol=1e-14)


def test_single_pencil_64_against_brute_force_and_invariants():
    F, J, G = P.single_pencil_64()
    lam = brute.generalized_eigenvalues(F, G, J, dps=40)
    assert 1e-9 < eig_tol(F, G) < 5e-9        # cond(F_c) ~ cond(G_c) ~ 1e6
    for method, kw in (("pointwise", {}), ("blocked", dict(w=8)), ("blocked", dict(w=32))):
        out = oracle.solve(F, G, J, method=method, **kw)
        assert out["status"] == 0
        tol = eig_tol_vec(F, G, J, out["lam"], out["F"])
        assert np.all(rel_err(out["lam"], lam) < tol)
        Gp, Fp = out["G"], out["F"]
        n = Gp.shape[1]
        # converged columns: G' orthogonal, F' J-orthogonal (Section 6.1.7)
        gn = np.linalg.norm(Gp, axis=0)
        C = (Gp.conj().T @ Gp) / np.outer(gn, gn)
        assert np.max(np.abs(C - np.eye(n))) < 1e3 * n * oracle.EPS
        HF = Fp.conj().T @ (J[:, None] * Fp)
        d = np.sqrt(np.abs(np.diag(HF).real))
        off = np.abs(HF - np.diag(np.diag(HF))) / np.outer(d, d)
        assert off.max() < 1e4 * n * oracle.EPS
        # S-orthonormal eigenvectors: G V has orthonormal columns
        V = out["V"]
        GV = G @ V
        assert np.max(np.abs(GV.conj().T @ GV - np.eye(n))) < 1e-6
        # lambda signs follow f_j^* J f_j
        assert np.all(np.sign(out["lam"]) == np.sign(np.diag(HF).real))


def test_sweep_counters_end_with_no_big_transformation():
    F, J, G = P.single_pencil_64()
    for method, kw in (("pointwise", {}), ("blocked", dict(w=8))):
        out = oracle.solve(F, G, J, method=method, **kw)
        c = out["counts"]
        assert c[-1, 1] == 0 and np.all(c[:-1, 1] > 0)
        assert np.all(c[:, 1] <= c[:, 0])


def test_max_sweeps_reports_not_converged():
    F, J, G = P.single_pencil_64()
    out = oracle.solve(F, G, J, max_sweeps=2)
    assert out["status"] == 1 and out["sweeps"] == 2


def test_deterministic_across_thread_counts():
    F, J, G = P.single_pencil_64()
    a = oracle.blocked(F, G, J, w=8, nthreads=1)
    b = oracle.blocked(F, G, J, w=8, nthreads=4)
    assert np.array_equal(a["F"], b["F"]) and np.array_equal(a["Z"], b["Z"])
    c = oracle.pointwise(F, G, J, nthreads=1)
    d = oracle.pointwise(F, G, J, nthreads=3)
    assert np.array_equal(c["G"], d["G"])


def test_blocked_step_matches_block_pivot_update():
    # one outer step = block pivots, inner level, then X <- X Z^ per block pair
    F, J, G = P.single_pencil_64()
    w = 8
    Fs, Gs, Zs, na, nbig = oracle.blocked_step(F, G, J, w=w, r=3)
    off = oracle.partition(64, w)
    t = oracle.rr_table(len(off) - 1)[3]
    for k, (Pb, Qb) in enumerate(t):
        bp = oracle.block_pivot(F, G, J, w=w, r=3, k=k)
        cols = list(range(off[Pb], off[Pb + 1])) + list(range(off[Qb], off[Qb + 1]))
        Zh = bp["Z"]
        assert np.allclose(Fs[:, cols], F[:, cols] @ Zh, rtol=1e-12, atol=1e-12 * np.abs(F).max())
        # the block pivots are the Grams of eq. 6.1 on the pair's columns
        Fc, Gc = F[:, cols], G[:, cols]
        assert np.allclose(bp["H0"], Fc.conj().T @ (J[:, None] * Fc), rtol=1e-12,
                           atol=1e-12 * np.abs(bp["H0"]).max())
        assert np.allclose(bp["S0"], Gc.conj().T @ Gc, rtol=1e-12, atol=1e-12 * np.abs(bp["S0"]).max())
        # inner level result: Z^* S0 Z close to identity on the pivot pairs
        S3 = Zh.conj().T @ bp["S0"] @ Zh
        assert np.allclose(np.diag(S3).real, 1.0, atol=1e-8)


def test_rank_deficient_G_is_reported():
    # Section 6.4.2 stops on a rank-deficient pivot of S = G^* G; two equal
    # columns of G make S singular
    F, J, G = P.svd_pencil(31, 20, 20, 10, 4, (0.5, 2), (0.5, 2))
    ok = oracle.solve(F, G, J)
    assert ok["status"] == 0 and ok["kappa_est"] < 100
    Gr = G.copy()
    Gr[:, 3] = Gr[:, 7]
    for method, kw in (("pointwise", {}), ("blocked", dict(w=4))):
        assert oracle.solve(F, Gr, J, method=method, **kw)["status"] == -2
    # the estimate tracks cond(G): C1 has cond(G) = 1e6
    F, J, G = P.single_pencil_64()
    k = oracle.solve(F, G, J)["kappa_est"]
    assert 1e6 / 8 < k < 1e6 * 8
