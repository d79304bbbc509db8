"""Solver options of the boundary on the GPU: the time limit, the tolerance
scale of eq. 6.12 and sorting."""
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


def test_timeout_returns_after_the_current_sweep_with_outputs(gh):
    F, J, G = P.lapw_pencil(256)
    s = gh.Solver(0, block_width=16, timeout_ms=1)
    lam, V, sweeps, st = s.solve(dev(gh, F), dev(gh, G), torch.from_numpy(J).cuda())
    assert st == gh.GHSVD_ERR_TIMEOUT
    assert 1 <= sweeps <= 3                     # the limit is checked between sweeps
    assert np.all(np.isfinite(lam.cpu().numpy()))
    # the outputs are those of the current factors: the columns of G V have unit norm
    GV = G @ V.cpu().numpy()
    assert np.allclose(np.linalg.norm(GV, axis=0), 1.0, rtol=1e-10)


def test_tol_scale_relaxes_eq_6_12(gh):
    F, J, G = P.lapw_pencil(256)
    ref = oracle.solve(F, G, J, method="blocked", w=16)
    tol = eig_tol_vec(F, G, J, ref["lam"], ref["F"])
    out = {}
    for scale in (1.0, 1e4):
        s = gh.Solver(0, block_width=16, tol_scale=scale)
        lam, _, sweeps, st = s.solve(dev(gh, F), dev(gh, G), torch.from_numpy(J).cuda(),
                                     want_vectors=False)
        assert st == gh.GHSVD_OK
        out[scale] = (lam.cpu().numpy(), sweeps)
    # rel_err and eig_tol_vec both follow the ascending order of the eigenvalues
    assert np.all(rel_err(out[1.0][0], ref["lam"]) < tol)
    # a looser threshold stops no later and stays within the looser scale of the tolerance
    assert out[1e4][1] <= out[1.0][1]
    assert np.all(rel_err(out[1e4][0], ref["lam"]) < 1e4 * tol)


def test_sort_ascending_orders_lambda_and_permutes_V_alike(gh):
    F, J, G = P.single_pencil_64()
    a = gh.Solver(0, block_width=8)
    b = gh.Solver(0, block_width=8, sort_ascending=1)
    la, Va, _, _ = a.solve(dev(gh, F), dev(gh, G), torch.from_numpy(J).cuda())
    lb, Vb, _, _ = b.solve(dev(gh, F), dev(gh, G), torch.from_numpy(J).cuda())
    la, lb, Va, Vb = la.cpu().numpy(), lb.cpu().numpy(), Va.cpu().numpy(), Vb.cpu().numpy()
    order = np.argsort(la, kind="stable")
    assert np.all(np.diff(lb) >= 0)
    assert np.array_equal(lb, la[order])
    assert np.array_equal(Vb, Va[:, order])
