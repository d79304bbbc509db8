"""Phase 2 (ghsvd_urv, opts.shorten) and Phase 4 (ghsvd_inverse, ghsvd_phase4,
ghsvd_decomposition_errors) on the GPU against the FP64 oracle
(arXiv 1907.08560, Sections 5 and 7)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from synth import pencils as P
from conftest import eig_tol_vec, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_08560_gb300 import build, ghsvd
    build.build()
    return ghsvd


def dev(gh, X):
    return gh.colmajor(torch.from_numpy(np.asarray(X))).cuda()


def herm(F, J):
    return F.conj().T @ (np.asarray(J, dtype=np.float64)[:, None] * F)


URV_CASES = [
    # (seed, m, p, n, m_minus, permute J)
    (1, 30, 40, 20, 8, False),
    (2, 45, 52, 30, 20, True),           # many 2x2 pivots likely
    (3, 21, 21, 21, 7, False),           # square input
    (4, 96, 128, 64, 16, False),         # the n = 64 workload's shape
    (5, 4500, 4300, 24, 900, True),      # columns longer than the register window (4096 rows)
    (6, 450, 600, 300, 75, False),       # several apply grids, ragged counts
    (7, 5, 6, 1, 2, False),              # n = 1
]


@pytest.mark.parametrize("case", URV_CASES, ids=[f"m{c[1]}n{c[3]}" for c in URV_CASES])
def test_urv_matches_oracle(gh, case):
    seed, m, p, n, m_minus, perm_j = case
    F, J, G = P.svd_pencil(8000 + seed, m, p, n, m_minus, (1e-2, 1e2), (1e-2, 1e2), permute_j=perm_j)
    Fs, Js, Gs, perm, n2 = gh.ghsvd_urv(dev(gh, F), torch.from_numpy(J).cuda(), dev(gh, G))
    ref = oracle.urv(F, G, J)
    assert ref["status"] == 0
    perm = perm.cpu().numpy()
    # the pivot decisions: FP64 on both sides, far from ties on these inputs
    assert perm.tolist() == ref["perm"].tolist()
    assert n2 == ref["n2x2"]
    assert Js.cpu().numpy().tolist() == ref["J"].tolist()
    R = Fs.cpu().numpy()
    RG = Gs.cpu().numpy()
    assert np.max(np.abs(R - ref["F"])) <= 1e-11 * np.abs(ref["F"]).max()
    assert np.max(np.abs(RG - ref["G"])) <= 1e-12 * np.abs(ref["G"]).max()
    # what defines the factorization: the Hermitian forms and the shapes
    H0 = herm(F[:, perm], J)
    assert np.max(np.abs(herm(R, Js.cpu().numpy()) - H0)) <= 1e-13 * np.linalg.norm(F) ** 2
    S0 = G[:, perm].conj().T @ G[:, perm]
    assert np.max(np.abs(RG.conj().T @ RG - S0)) <= 1e-13 * np.linalg.norm(G) ** 2
    assert np.all(np.tril(R, -2) == 0) and np.all(np.tril(RG, -1) == 0)


def test_urv_breakdown_is_reported(gh):
    F = np.array([[1.0], [1.0]], dtype=np.complex128)           # J-isotropic column
    J = np.array([1, -1], dtype=np.int8)
    G = np.array([[1.0], [0.5]], dtype=np.complex128)
    with pytest.raises(gh.GhsvdError) as ei:
        gh.ghsvd_urv(dev(gh, F), torch.from_numpy(J).cuda(), dev(gh, G))
    assert ei.value.status == gh.GHSVD_ERR_BREAKDOWN


@pytest.mark.parametrize("w,n", [(8, 64), (16, 77)])
def test_shortened_solve_matches_tall_oracle(gh, w, n):
    m, p = (3 * n) // 2, 2 * n
    F, J, G = P.svd_pencil(8100 + n, m, p, n, m // 6, (1e-3, 1e3), (1e-3, 1e3), permute_j=(n % 2 == 1))
    ref = oracle.solve(F, G, J, method="blocked", w=w)
    assert ref["status"] == 0
    tol = eig_tol_vec(F, G, J, ref["lam"], ref["F"])
    s = gh.Solver(0, block_width=w, shorten=1, sort_ascending=1)
    lam, V, sweeps, st = s.solve(dev(gh, F), dev(gh, G), torch.from_numpy(J).cuda())
    assert st == gh.GHSVD_OK
    lam = lam.cpu().numpy()
    # rel_err and eig_tol_vec both follow the ascending order of the eigenvalues
    assert np.all(rel_err(lam, ref["lam"]) < tol)
    # V refers to the caller's columns: G V orthonormal (Q_G is unitary) ...
    V = V.cpu().numpy()
    GV = G @ V
    assert np.max(np.abs(GV.conj().T @ GV - np.eye(n))) < 1e-8
    # ... and V^* H V = diag(lambda) where the iteration ran: on the square pencil
    # (Fs, Js) of Phase 2 (deterministic: the same factors as inside the solve).
    # Forming Fs V again errs by about eps |Fs| |V| (the hyperbolic Q_F need not
    # keep norms, and V is ill-conditioned), so that is the scale of the check.
    Fs, Js, _, perm, _ = gh.ghsvd_urv(dev(gh, F), torch.from_numpy(J).cuda(), dev(gh, G))
    Fs = Fs.cpu().numpy()
    Vs = V[perm.cpu().numpy(), :]
    FV = Fs @ Vs
    D = herm(FV, Js.cpu().numpy())
    nrm = np.linalg.norm(np.abs(Fs) @ np.abs(Vs), axis=0)
    assert np.all(np.abs(np.diag(D).real - lam) <= 1e-9 * nrm ** 2)
    off = np.abs(D - np.diag(np.diag(D)))
    assert np.all(off <= 1e-9 * np.outer(nrm, nrm))
    stt = s.stats()
    assert stt["ms_phase2"] > 0 and stt["n2x2"] >= 0


@pytest.mark.parametrize("n", [1, 7, 150])
def test_inverse_matches_oracle(gh, n):
    rng = np.random.default_rng(8200 + n)
    Z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * 10.0 ** rng.uniform(-2, 2, n)
    X = gh.ghsvd_inverse(dev(gh, Z)).cpu().numpy()
    Xo = oracle.inverse(Z)
    assert np.max(np.abs(X - Xo)) <= 1e-9 * np.abs(Xo).max()
    bound = 30 * 2.0 ** -53 * np.max(np.abs(Z) @ np.abs(X))
    assert np.max(np.abs(Z @ X - np.eye(n))) < 10 * n * bound


def test_inverse_singular(gh):
    Z = np.ones((5, 5), dtype=np.complex128)
    Z[:, 2] = 0.0
    with pytest.raises(gh.GhsvdError) as ei:
        gh.ghsvd_inverse(dev(gh, Z))
    assert ei.value.status == gh.GHSVD_ERR_RANK_DEFICIENT


@pytest.mark.parametrize("shorten", [0, 1])
def test_phase4_matches_oracle(gh, shorten):
    n = 64
    F, J, G = P.single_pencil_64()
    Fd, Gd, Jd = dev(gh, F), dev(gh, G), torch.from_numpy(J).cuda()
    if shorten:                                   # the GHSVD of the square pencil of Phase 2
        Fd, Jd, Gd, _, _ = gh.ghsvd_urv(Fd, Jd, Gd)
    s = gh.Solver(0, block_width=8)
    lam, _, _, st = s.solve(Fd, Gd, Jd, want_vectors=False)
    assert st == gh.GHSVD_OK
    m, p = Fd.shape[0], Gd.shape[0]
    Fp, Gp, Zp = s.factors(m, p, n)
    sf, sg, X = s.phase4(n)
    ref = oracle.ghsvd(Fd.cpu().numpy(), Gd.cpu().numpy(), Jd.cpu().numpy(), Fp.cpu().numpy(),
                       Gp.cpu().numpy(), Zp.cpu().numpy())
    assert np.max(np.abs(sf.cpu().numpy() - ref["sigma_f"]) / ref["sigma_f"]) < 1e-13
    assert np.max(np.abs(sg.cpu().numpy() - ref["sigma_g"]) / ref["sigma_g"]) < 1e-13
    Xn = X.cpu().numpy()
    assert np.max(np.abs(Xn - ref["X"])) <= 1e-9 * np.abs(ref["X"]).max()
    ef, eg = s.decomposition_errors(Fd, Gd, X)
    # eq. 7.1: both sides at the level the paper reports (1e-13 .. 1e-12)
    assert ef < 1e-12 and eg < 1e-12
    assert abs(ef - ref["err_F"]) < 1e-12 and abs(eg - ref["err_G"]) < 1e-12
