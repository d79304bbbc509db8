"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerance for eigenvalues (FP64): per eigenvalue,
    1e-12 * max(1, (cond(F_c) + cond(G_c)) / 1e3) * a_j,
with F_c, G_c the column-scaled factors and a_j = ||f_j||^2 / |f_j^* J f_j|
the hyperbolic amplification of the oracle's converged column j (conftest).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from synth import pencils as P
from conftest import eig_tol, eig_tol_vec, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_08560_gb300 import build, ghsvd
    build.build()
    return ghsvd


def to_dev(gh, F, G, J):
    Fd = gh.colmajor(torch.from_numpy(np.asarray(F))).cuda()
    Gd = gh.colmajor(torch.from_numpy(np.asarray(G))).cuda()
    Jd = None if J is None else torch.from_numpy(np.asarray(J, dtype=np.int8)).cuda()
    return Fd, Gd, Jd


def gpu_solve(gh, F, G, J, **opts):
    s = gh.Solver(0, **opts)
    Fd, Gd, Jd = to_dev(gh, F, G, J)
    lam, V, sweeps, status = s.solve(Fd, Gd, Jd)
    torch.cuda.synchronize()
    m, n = F.shape
    p = G.shape[0]
    Fp, Gp, Zp = s.factors(m, p, n)
    out = dict(lam=lam.cpu().numpy(), V=V.cpu().numpy(), sweeps=sweeps, status=status,
               F=Fp.cpu().numpy(), G=Gp.cpu().numpy(), Z=Zp.cpu().numpy(), stats=s.stats())
    s.close()
    return out


def check_eigs(F, G, J, gpu, ref):
    tol = eig_tol_vec(F, G, J, ref["lam"], ref["F"])
    err = rel_err(gpu["lam"], ref["lam"])
    assert np.all(err < tol), (err.max(), tol.min(), np.argmax(err / tol))
    return err


@pytest.mark.parametrize("w", [4, 8, 16, 32])
def test_single_pencil_64_eigenvalues_match_oracle(gh, w):
    F, J, G = P.single_pencil_64()
    ref = oracle.solve(F, G, J, method="blocked", w=w)
    gpu = gpu_solve(gh, F, G, J, block_width=w)
    assert gpu["status"] == 0 and ref["status"] == 0
    check_eigs(F, G, J, gpu, ref)
    ref_pw = oracle.solve(F, G, J)
    check_eigs(F, G, J, gpu, ref_pw)


def _pencil(case):
    if case == "single64":
        return P.single_pencil_64()
    n = int(case[1:])
    return P.svd_pencil(900 + n, (3 * n) // 2 + 3, 2 * n + 5, n, n // 5, (1e-2, 1e2), (1e-3, 1e3),
                        permute_j=True)


# block pivots of 16 (one 16 x 16 tile of the Gram), 48 and 34 columns (three
# tiles, the last one ragged at 34) and 64 (four tiles)
@pytest.mark.parametrize("case,w", [("single64", 8), ("n96", 24), ("n100", 20), ("n128", 32)])
def test_one_sweep_factors_match_oracle_elementwise(gh, case, w):
    # the same block algorithm, same orderings: after one sweep the
    # transformed factors agree to rounding (relative to each column's norm)
    F, J, G = _pencil(case)
    ref = oracle.blocked(F, G, J, w=w, max_sweeps=1)
    gpu = gpu_solve(gh, F, G, J, block_width=w, max_sweeps=1)
    assert gpu["status"] == gh.GHSVD_ERR_NOT_CONVERGED
    assert gpu["stats"]["transforms"][0] == ref["counts"][0, 0]
    for X in ("F", "G", "Z"):
        a, b = gpu[X], ref[X]
        scale = np.linalg.norm(b, axis=0)[None, :]
        d = np.abs(a - b) / scale
        assert d.max() < 1e-11, (X, d.max())


@pytest.mark.parametrize("m,p,n,neg,w", [(70, 90, 65, 20, 8), (40, 41, 37, 10, 5),
                                         (130, 200, 100, 40, 7), (9, 8, 7, 3, 2),
                                         (150, 200, 96, 30, 24), (170, 230, 100, 33, 20)])
def test_ragged_and_odd_sizes(gh, m, p, n, neg, w):
    # odd n (bordering), uneven block widths, row counts not multiples of 64
    F, J, G = P.svd_pencil(500 + n, m, p, n, neg, (1e-2, 1e2), (1e-2, 1e2), permute_j=True)
    ref = oracle.solve(F, G, J, method="blocked", w=w)
    gpu = gpu_solve(gh, F, G, J, block_width=w)
    assert gpu["status"] == 0
    check_eigs(F, G, J, gpu, ref)


def test_positives_first_signature_without_J_array(gh):
    F, J, G = P.single_pencil_64()
    s = gh.Solver(0, block_width=16)
    Fd, Gd, _ = to_dev(gh, F, G, None)
    lam, _, _, st = s.solve(Fd, Gd, None, n_plus=int((J > 0).sum()))
    ref = oracle.solve(F, G, J, method="blocked", w=16)
    assert st == 0
    check_eigs(F, G, J, dict(lam=lam.cpu().numpy()), ref)


def test_known_eigenvalues_by_construction(gh):
    n = 256
    F, J, G, lam = P.known_pencil(77, 384, 512, n, 128, 40, cond_x=10.0, hyper=0.5, n_hyper=64)
    gpu = gpu_solve(gh, F, G, J, block_width=32)
    assert gpu["status"] == 0
    assert rel_err(gpu["lam"], lam).max() < 1e-12


def test_identity_signature_gsvd(gh):
    F, J, G, lam = P.known_pencil(78, 150, 200, 100, 0, 0, cond_x=10.0)
    gpu = gpu_solve(gh, F, G, None, block_width=16)
    assert gpu["status"] == 0 and np.all(gpu["lam"] > 0)
    assert rel_err(gpu["lam"], lam).max() < 1e-12


def test_full_block_inner_sweeps(gh):
    F, J, G = P.single_pencil_64()
    ref = oracle.solve(F, G, J, method="blocked", w=8, inner_sweeps=30)
    gpu = gpu_solve(gh, F, G, J, block_width=8, inner_sweeps=30)
    assert gpu["status"] == 0
    check_eigs(F, G, J, gpu, ref)


def test_outputs_satisfy_the_definition(gh):
    # V^* S V = I and V^* H V = diag(lambda), computed through the factors
    F, J, G = P.single_pencil_64()
    gpu = gpu_solve(gh, F, G, J, block_width=8)
    V = gpu["V"]
    GV = G @ V
    FV = F @ V
    n = V.shape[1]
    assert np.max(np.abs(GV.conj().T @ GV - np.eye(n))) < 1e-6
    HV = FV.conj().T @ (J[:, None] * FV)
    d = np.sqrt(np.abs(np.outer(gpu["lam"], gpu["lam"])))
    off = np.abs(HV - np.diag(np.diag(HV))) / np.maximum(d, 1e-300)
    assert off.max() < 1e-6
    assert np.all(np.sign(gpu["lam"]) == np.sign(np.diag(HV).real))


def test_sorted_output(gh):
    F, J, G = P.single_pencil_64()
    gpu = gpu_solve(gh, F, G, J, block_width=8, sort_ascending=1)
    assert np.all(np.diff(gpu["lam"]) >= 0)
    GV = G @ gpu["V"]
    assert np.max(np.abs(GV.conj().T @ GV - np.eye(64))) < 1e-6


@pytest.mark.parametrize("opts", [dict(block_width=8), dict(block_width=32, precision=1, max_sweeps=60),
                                  dict(block_width=32, precision=1, mixed_tc=0, max_sweeps=60)])
def test_deterministic(gh, opts):
    # the same inputs give the same bits: FP64 sweeps, and the mixed schedule
    # with its complex64 Grams and updates on the tensor cores or the CUDA
    # cores (every reduction has a fixed order)
    F, J, G = P.single_pencil_64()
    a = gpu_solve(gh, F, G, J, **opts)
    b = gpu_solve(gh, F, G, J, **opts)
    assert a["status"] == 0 and a["sweeps"] == b["sweeps"]
    assert np.array_equal(a["lam"], b["lam"]) and np.array_equal(a["V"], b["V"])


def test_host_entry_point_matches_device(gh):
    F, J, G = P.single_pencil_64()
    s = gh.Solver(0, block_width=8)
    lam_h, V_h, sw_h, st_h = s.solve_host(F, G, J)
    a = gpu_solve(gh, F, G, J, block_width=8)
    assert st_h == 0 and sw_h == a["sweeps"]
    assert np.array_equal(lam_h, a["lam"]) and np.array_equal(V_h, a["V"])


def test_small_orders(gh):
    for n in (1, 2, 3):
        F, J, G = P.svd_pencil(900 + n, n + 2, n + 1, n, 1, (0.5, 2), (0.5, 2))
        ref = oracle.solve(F, G, J)
        gpu = gpu_solve(gh, F, G, J, block_width=1)
        assert gpu["status"] == 0
        assert rel_err(gpu["lam"], ref["lam"]).max() < 1e-13


def test_warm_start_from_converged_vectors(gh):
    F, J, G = P.single_pencil_64()
    a = gpu_solve(gh, F, G, J, block_width=8)
    s = gh.Solver(0, block_width=8)
    Fd, Gd, Jd = to_dev(gh, F, G, J)
    V0 = gh.colmajor(torch.from_numpy(a["V"])).cuda()
    lam, V, sweeps, st = s.solve(Fd, Gd, Jd, V0=V0)
    assert st == 0 and sweeps <= 2
    ref = oracle.solve(F, G, J, method="blocked", w=8)
    check_eigs(F, G, J, dict(lam=lam.cpu().numpy()), ref)
    # a random nonsingular start converges to the same eigenvalues
    rng = np.random.default_rng(5)
    R = np.eye(64) + 0.3 * (rng.standard_normal((64, 64)) + 1j * rng.standard_normal((64, 64))) / 8
    lam2, _, _, st2 = s.solve(Fd, Gd, Jd, V0=gh.colmajor(torch.from_numpy(R)).cuda())
    assert st2 == 0
    check_eigs(F, G, J, dict(lam=lam2.cpu().numpy()), ref)


def test_error_statuses(gh):
    s = gh.Solver(0, block_width=8)
    F, J, G = P.svd_pencil(31, 20, 20, 10, 4, (0.5, 2), (0.5, 2))
    # rank-deficient G: two equal columns
    Gr = G.copy()
    Gr[:, 3] = Gr[:, 7]
    Fd, Gd, Jd = to_dev(gh, F, Gr, J)
    with pytest.raises(gh.GhsvdError) as e:
        s.solve(Fd, Gd, Jd)
    assert e.value.status == gh.GHSVD_ERR_RANK_DEFICIENT
    # non-finite input
    Fn = F.copy()
    Fn[2, 2] = np.nan
    Fd, Gd, Jd = to_dev(gh, Fn, G, J)
    with pytest.raises(gh.GhsvdError) as e:
        s.solve(Fd, Gd, Jd)
    assert e.value.status == gh.GHSVD_ERR_NONFINITE
    # a J entry that is not +-1
    Jb = J.copy()
    Jb[0] = 0
    Fd, Gd, Jd = to_dev(gh, F, G, Jb)
    with pytest.raises(gh.GhsvdError) as e:
        s.solve(Fd, Gd, Jd)
    assert e.value.status == gh.GHSVD_ERR_INVALID_ARG
    # m < n
    Fd, Gd, Jd = to_dev(gh, F[:8], G, J[:8])
    with pytest.raises(gh.GhsvdError) as e:
        s.solve(Fd, Gd, Jd)
    assert e.value.status == gh.GHSVD_ERR_INVALID_ARG
    # the handle still works after the errors
    Fd, Gd, Jd = to_dev(gh, F, G, J)
    lam, _, _, st = s.solve(Fd, Gd, Jd)
    assert st == 0


def test_not_converged_status_still_writes_outputs(gh):
    F, J, G = P.single_pencil_64()
    gpu = gpu_solve(gh, F, G, J, block_width=8, max_sweeps=3)
    assert gpu["status"] == gh.GHSVD_ERR_NOT_CONVERGED and gpu["sweeps"] == 3
    assert np.all(np.isfinite(gpu["lam"]))


def test_mixed_precision_schedule(gh):
    F, J, G = P.single_pencil_64()
    ref = oracle.solve(F, G, J, method="blocked", w=8)
    # at n = 64 the complex64 rounds and the FP64 sweeps that follow take
    # 27-32 sweeps (FP64 alone: 21), near the default C_max of 30: the limit
    # is raised
    gpu = gpu_solve(gh, F, G, J, block_width=8, precision=gh.GHSVD_PRECISION_MIXED, max_sweeps=40)
    assert gpu["status"] == 0
    assert gpu["stats"]["sweeps_low"] >= 1
    check_eigs(F, G, J, gpu, ref)


@pytest.mark.parametrize("precision,param32,tc", [(0, 0, 0), (1, 0, 0), (1, 1, 0), (1, 0, 1),
                                                   (1, 1, 1)])
def test_lapw_shaped_pencil_256_matches_oracle(gh, precision, param32, tc):
    # the benchmark's pencil family at n = 256 (F 384 x 256 with 64 negative
    # signs, G 512 x 256, cond(S) = 1e10), FP64 and mixed schedules (the
    # complex64 sweeps with FP64 or FP32 2x2 parameters, their Grams and
    # updates on the CUDA cores or on the tensor cores)
    F, J, G = P.lapw_pencil(256)
    ref = oracle.solve(F, G, J, method="blocked", w=32)
    assert ref["status"] == 0
    gpu = gpu_solve(gh, F, G, J, block_width=32, precision=precision, max_sweeps=80,
                    mixed_param32=param32, mixed_tc=tc)
    assert gpu["status"] == 0
    if precision:
        assert gpu["stats"]["sweeps_low"] > 0
    assert gpu["stats"]["sweeps_tc"] == (gpu["stats"]["sweeps_low"] if tc else 0)
    check_eigs(F, G, J, gpu, ref)
