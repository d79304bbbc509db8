"""Batched solves (ghsvd_solve_batched) against the FP64 oracle, pencil by pencil."""
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


def small_batch():
    # uneven orders (odd ones bordered), ragged row counts, permuted J, one J = I
    specs = [(37, 0.3, True), (64, 0.2, False), (90, 0.25, True), (45, 0.0, False),
             (77, 0.2, True), (128, 0.2, False)]
    out = []
    for i, (n, frac, perm) in enumerate(specs):
        m, p = (3 * n) // 2 + i, 2 * n - i
        F, J, G = P.svd_pencil(4000 + i, m, p, n, int(round(frac * m)), (1e-2, 1e2), (1e-2, 1e2),
                               permute_j=perm)
        out.append((F, J, G))
    return out


@pytest.mark.parametrize("w", [8, 16])
def test_batched_matches_oracle_per_pencil(gh, w):
    batch = small_batch()
    s = gh.Solver(0, block_width=w)
    lams, Vs, sweeps, statuses, st = s.solve_batched(
        [dev(gh, F) for F, _, _ in batch], [dev(gh, G) for _, _, G in batch],
        [torch.from_numpy(J).cuda() for _, J, _ in batch])
    assert st == gh.GHSVD_OK and all(x == 0 for x in statuses)
    for (F, J, G), lam, V, sw in zip(batch, lams, Vs, sweeps):
        ref = oracle.solve(F, G, J, method="blocked", w=w)
        assert ref["status"] == 0
        tol = eig_tol_vec(F, G, J, ref["lam"], ref["F"])
        assert np.all(rel_err(lam.cpu().numpy(), ref["lam"]) < tol)
        assert abs(sw - ref["sweeps"]) <= 3
        GV = G @ V.cpu().numpy()
        assert np.max(np.abs(GV.conj().T @ GV - np.eye(F.shape[1]))) < 1e-8


def test_batched_equals_single_pencil_solves(gh):
    batch = small_batch()[:4]
    s = gh.Solver(0, block_width=16)
    lams, _, sweeps, statuses, st = s.solve_batched(
        [dev(gh, F) for F, _, _ in batch], [dev(gh, G) for _, _, G in batch],
        [torch.from_numpy(J).cuda() for _, J, _ in batch])
    # one graph launch; its while loop ran one tick per outer step until the
    # last pencil stopped (the control kernel ends the loop on the device):
    # max over the pencils of (steps per sweep) x (sweeps)
    stt = s.stats()
    assert stt["batch_graph_launches"] == 1
    steps = [len(oracle.partition(F.shape[1], 16)) - 2 for F, _, _ in batch]
    assert stt["batch_ticks"] == max(st_ * sw for st_, sw in zip(steps, sweeps))
    for (F, J, G), lam, sw in zip(batch, lams, sweeps):
        one = gh.Solver(0, block_width=16)
        l1, _, sw1, st1 = one.solve(dev(gh, F), dev(gh, G), torch.from_numpy(J).cuda())
        Fp, _, _ = one.factors(F.shape[0], G.shape[0], F.shape[1])
        tol = eig_tol_vec(F, G, J, l1.cpu().numpy(), Fp.cpu().numpy())
        assert np.all(rel_err(lam.cpu().numpy(), l1.cpu().numpy()) < tol)
        assert abs(sw - sw1) <= 2


def test_batched_autotuned_block_width(gh):
    batch = small_batch()
    s = gh.Solver(0, block_width=0)
    lams, _, _, statuses, st = s.solve_batched(
        [dev(gh, F) for F, _, _ in batch], [dev(gh, G) for _, _, G in batch],
        [torch.from_numpy(J).cuda() for _, J, _ in batch], want_vectors=False)
    assert st == gh.GHSVD_OK
    w = s.stats()["block_width"]
    assert w in (8, 16, 32)
    for (F, J, G), lam in zip(batch, lams):
        ref = oracle.solve(F, G, J, method="blocked", w=w)
        tol = eig_tol_vec(F, G, J, ref["lam"], ref["F"])
        assert np.all(rel_err(lam.cpu().numpy(), ref["lam"]) < tol)


def test_batched_failure_stays_in_its_pencil(gh):
    batch = small_batch()[:3]
    F1, J1, G1 = batch[1]
    G1 = G1.copy()
    G1[:, 5] = G1[:, 9]                 # rank-deficient G in pencil 1 only
    batch[1] = (F1, J1, G1)
    s = gh.Solver(0, block_width=8)
    lams, _, _, statuses, st = s.solve_batched(
        [dev(gh, F) for F, _, _ in batch], [dev(gh, G) for _, _, G in batch],
        [torch.from_numpy(J).cuda() for _, J, _ in batch], want_vectors=False)
    assert statuses[1] == gh.GHSVD_ERR_RANK_DEFICIENT
    assert statuses[0] == 0 and statuses[2] == 0
    assert st == gh.GHSVD_ERR_RANK_DEFICIENT
    for i in (0, 2):
        F, J, G = batch[i]
        ref = oracle.solve(F, G, J, method="blocked", w=8)
        tol = eig_tol_vec(F, G, J, ref["lam"], ref["F"])
        assert np.all(rel_err(lams[i].cpu().numpy(), ref["lam"]) < tol)


def test_batched_identity_signature_without_J(gh):
    Fs, Gs, lams_ref = [], [], []
    for i, n in enumerate((40, 66)):
        F, J, G, lam = P.known_pencil(300 + i, n + 20, n + 30, n, 0, 0, cond_x=10.0)
        Fs.append(F); Gs.append(G); lams_ref.append(lam)
    s = gh.Solver(0, block_width=8)
    lams, _, _, statuses, st = s.solve_batched([dev(gh, F) for F in Fs], [dev(gh, G) for G in Gs],
                                               None, want_vectors=False)
    assert st == gh.GHSVD_OK
    for lam, ref in zip(lams, lams_ref):
        assert rel_err(lam.cpu().numpy(), ref).max() < 1e-12


def test_batched_kpoint_pencils_match_oracle_golden(gh):
    # three of the 64 k-point pencils of the batched workload (n = 1511, 1147,
    # 1272; F 1.5n x n with 20 % negative signs, G 2n x n, cond(S) up to 6e9),
    # solved together with the autotuned block width, against the FP64
    # oracle's eigenvalues stored by tests/golden/make_fullsize.py
    from conftest import fullsize_golden, golden_ratio
    names = ("kpt56", "kpt11", "kpt23")
    goldens = [fullsize_golden(nm) for nm in names]
    pens = [P.batch_pencil(g["n"], g["cond_s"], g["seed"]) for g in goldens]
    s = gh.Solver(0, block_width=0, max_sweeps=80)
    lams, Vs, sweeps, statuses, st = s.solve_batched(
        [dev(gh, F) for F, _, _ in pens], [dev(gh, G) for _, _, G in pens],
        [torch.from_numpy(J).cuda() for _, J, _ in pens], want_vectors=False)
    s.close()
    assert st == gh.GHSVD_OK and all(x == 0 for x in statuses)
    for g, lam in zip(goldens, lams):
        assert golden_ratio(lam.cpu().numpy(), g) < 1.0, g["name"]


@pytest.mark.parametrize("w,param32", [(8, 0), (16, 0), (16, 1)])
def test_batched_mixed_schedule_matches_oracle_per_pencil(gh, w, param32):
    # every pencil runs its own complex64 rounds (Z'_low accumulated in
    # complex64, applied to the FP64 factors by one FP64 product per round)
    # and then FP64 sweeps to the stopping rule of Section 6.1.7
    batch = small_batch()
    s = gh.Solver(0, block_width=w, precision=gh.GHSVD_PRECISION_MIXED, mixed_param32=param32,
                  max_sweeps=80)
    lams, Vs, sweeps, statuses, st = s.solve_batched(
        [dev(gh, F) for F, _, _ in batch], [dev(gh, G) for _, _, G in batch],
        [torch.from_numpy(J).cuda() for _, J, _ in batch])
    assert st == gh.GHSVD_OK and all(x == 0 for x in statuses)
    stt = s.stats()
    assert stt["rounds_low"] >= len(batch)          # at least one round per pencil
    assert stt["sweeps_low"] >= len(batch)
    assert stt["batch_graph_launches"] == 1
    for (F, J, G), lam, V in zip(batch, lams, Vs):
        ref = oracle.solve(F, G, J, method="blocked", w=w)
        assert ref["status"] == 0
        tol = eig_tol_vec(F, G, J, ref["lam"], ref["F"])
        assert np.all(rel_err(lam.cpu().numpy(), ref["lam"]) < tol)
        GV = G @ V.cpu().numpy()
        assert np.max(np.abs(GV.conj().T @ GV - np.eye(F.shape[1]))) < 1e-8


def test_batched_mixed_with_starting_basis(gh):
    # a pencil given a starting Z' runs the mixed schedule from (F V0, G V0),
    # as a single solve does; the others from (F, G)
    batch = small_batch()[:3]
    n0 = batch[0][0].shape[1]
    rng = np.random.default_rng(77)
    V0h = np.eye(n0) + 0.05 * (rng.standard_normal((n0, n0)) + 1j * rng.standard_normal((n0, n0)))
    V0 = gh.colmajor(torch.from_numpy(V0h)).cuda()
    s = gh.Solver(0, block_width=8, precision=gh.GHSVD_PRECISION_MIXED, max_sweeps=60)
    lams, Vs, sweeps, statuses, st = s.solve_batched(
        [dev(gh, F) for F, _, _ in batch], [dev(gh, G) for _, _, G in batch],
        [torch.from_numpy(J).cuda() for _, J, _ in batch], V0s=[V0, None, None])
    assert st == gh.GHSVD_OK and all(x == 0 for x in statuses)
    assert s.stats()["rounds_low"] >= len(batch)
    for (F, J, G), lam, V in zip(batch, lams, Vs):
        ref = oracle.solve(F, G, J, method="blocked", w=8)
        tol = eig_tol_vec(F, G, J, ref["lam"], ref["F"])
        assert np.all(rel_err(lam.cpu().numpy(), ref["lam"]) < tol)
        GV = G @ V.cpu().numpy()
        assert np.max(np.abs(GV.conj().T @ GV - np.eye(F.shape[1]))) < 1e-8


def test_batched_mixed_failure_stays_in_its_pencil(gh):
    # a rank-deficient G in one pencil: its complex64 rounds pass over the
    # dependent pivots and its FP64 sweeps report it; the others converge
    batch = small_batch()[:3]
    F1, J1, G1 = batch[1]
    G1 = G1.copy()
    G1[:, 5] = G1[:, 9]
    batch[1] = (F1, J1, G1)
    s = gh.Solver(0, block_width=8, precision=gh.GHSVD_PRECISION_MIXED, max_sweeps=60)
    lams, _, _, statuses, st = s.solve_batched(
        [dev(gh, F) for F, _, _ in batch], [dev(gh, G) for _, _, G in batch],
        [torch.from_numpy(J).cuda() for _, J, _ in batch], want_vectors=False)
    assert statuses[1] == gh.GHSVD_ERR_RANK_DEFICIENT
    assert statuses[0] == 0 and statuses[2] == 0
    assert st == gh.GHSVD_ERR_RANK_DEFICIENT
    for i in (0, 2):
        F, J, G = batch[i]
        ref = oracle.solve(F, G, J, method="blocked", w=8)
        tol = eig_tol_vec(F, G, J, ref["lam"], ref["F"])
        assert np.all(rel_err(lams[i].cpu().numpy(), ref["lam"]) < tol)


def test_batched_mixed_sweep_limit(gh):
    # C_max counts the complex64 sweeps too: a limit below the schedule's
    # needs stops every pencil with NOT_CONVERGED and its sweep count at C_max
    batch = small_batch()[:2]
    s = gh.Solver(0, block_width=8, precision=gh.GHSVD_PRECISION_MIXED, max_sweeps=5)
    lams, _, sweeps, statuses, st = s.solve_batched(
        [dev(gh, F) for F, _, _ in batch], [dev(gh, G) for _, _, G in batch],
        [torch.from_numpy(J).cuda() for _, J, _ in batch], want_vectors=False)
    assert st == gh.GHSVD_ERR_NOT_CONVERGED
    assert all(x == gh.GHSVD_ERR_NOT_CONVERGED for x in statuses)
    assert all(sw == 5 for sw in sweeps)


def test_batched_mixed_kpoint_pencils_match_oracle_golden(gh):
    # the three k-point pencils of the golden test, mixed schedule
    from conftest import fullsize_golden, golden_ratio
    names = ("kpt56", "kpt11", "kpt23")
    goldens = [fullsize_golden(nm) for nm in names]
    pens = [P.batch_pencil(g["n"], g["cond_s"], g["seed"]) for g in goldens]
    s = gh.Solver(0, block_width=32, max_sweeps=80, precision=gh.GHSVD_PRECISION_MIXED)
    lams, _, sweeps, statuses, st = s.solve_batched(
        [dev(gh, F) for F, _, _ in pens], [dev(gh, G) for _, _, G in pens],
        [torch.from_numpy(J).cuda() for _, J, _ in pens], want_vectors=False)
    stt = s.stats()
    s.close()
    assert st == gh.GHSVD_OK and all(x == 0 for x in statuses)
    assert stt["sweeps_low"] >= 3
    for g, lam in zip(goldens, lams):
        assert golden_ratio(lam.cpu().numpy(), g) < 1.0, g["name"]


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_deterministic(gh, precision):
    batch = small_batch()[:4]
    outs = []
    for _ in range(2):
        s = gh.Solver(0, block_width=16, precision=precision, max_sweeps=60)
        lams, Vs, sweeps, statuses, st = s.solve_batched(
            [dev(gh, F) for F, _, _ in batch], [dev(gh, G) for _, _, G in batch],
            [torch.from_numpy(J).cuda() for _, J, _ in batch])
        assert st == gh.GHSVD_OK
        outs.append((lams, Vs, sweeps))
        s.close()
    (la, Va, sa), (lb, Vb, sb) = outs
    assert sa == sb
    for x, y in zip(la, lb):
        assert torch.equal(x, y)
    for x, y in zip(Va, Vb):
        assert torch.equal(x, y)
