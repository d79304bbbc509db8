"""The block update on the bf16 tensor cores with FP64 accuracy
(GHSVD_UPDATE_SPLIT_BF16) against the FP64 update and the FP64 oracle."""
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


def solve(gh, F, J, G, **opts):
    s = gh.Solver(0, **opts)
    lam, V, sw, st = s.solve(dev(gh, F), dev(gh, G), torch.from_numpy(J).cuda())
    m, p, n = F.shape[0], G.shape[0], F.shape[1]
    Fp, Gp, Zp = s.factors(m, p, n)
    out = dict(lam=lam.cpu().numpy(), V=V.cpu().numpy(), sweeps=sw, status=st,
               F=Fp.cpu().numpy(), G=Gp.cpu().numpy(), Z=Zp.cpu().numpy(), stats=s.stats())
    s.close()
    return out


def test_one_sweep_matches_the_fp64_update(gh):
    # the same sweep with the two engines: the factors agree column by column
    # to the level of FP64 rounding (the transformations are computed from the
    # factors, so differences propagate, but stay at a few ulps over a sweep)
    F, J, G = P.lapw_pencil(256)
    a = solve(gh, F, J, G, block_width=16, max_sweeps=1)
    b = solve(gh, F, J, G, block_width=16, max_sweeps=1, update_engine=gh.GHSVD_UPDATE_SPLIT_BF16)
    for X, Y in ((a["F"], b["F"]), (a["G"], b["G"]), (a["Z"], b["Z"])):
        d = np.linalg.norm(X - Y, axis=0) / np.linalg.norm(X, axis=0)
        assert d.max() < 1e-11, d.max()


@pytest.mark.parametrize("name,w", [("single64", 8), ("lapw256", 16), ("lapw512", 32)])
def test_split_update_solve_matches_oracle(gh, name, w):
    if name == "single64":
        F, J, G = P.single_pencil_64()
    else:
        F, J, G = P.lapw_pencil(int(name[4:]))
    ref = oracle.solve(F, G, J, method="blocked", w=w)
    assert ref["status"] == 0
    tol = eig_tol_vec(F, G, J, ref["lam"], ref["F"])
    out = solve(gh, F, J, G, block_width=w, max_sweeps=80, update_engine=gh.GHSVD_UPDATE_SPLIT_BF16)
    assert out["status"] == gh.GHSVD_OK
    order = np.argsort(ref["lam"])
    assert np.all(rel_err(out["lam"], ref["lam"]) < tol[order])
    assert abs(out["sweeps"] - ref["sweeps"]) <= 3
    GV = G @ out["V"]
    assert np.max(np.abs(GV.conj().T @ GV - np.eye(F.shape[1]))) < 1e-8


def test_split_update_with_ragged_blocks_and_permuted_J(gh):
    # odd order (bordering), widths wb and wb - 1, permuted signs
    n = 77
    F, J, G = P.svd_pencil(9100, 120, 160, n, 30, (1e-3, 1e3), (1e-3, 1e3), permute_j=True)
    ref = oracle.solve(F, G, J, method="blocked", w=16)
    tol = eig_tol_vec(F, G, J, ref["lam"], ref["F"])
    out = solve(gh, F, J, G, block_width=16, max_sweeps=80, update_engine=gh.GHSVD_UPDATE_SPLIT_BF16)
    assert out["status"] == gh.GHSVD_OK
    order = np.argsort(ref["lam"])
    assert np.all(rel_err(out["lam"], ref["lam"]) < tol[order])
