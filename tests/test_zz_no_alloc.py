"""ghsvd_solve_noalloc, the entry point for callers that cannot allocate
device memory when they solve (for example code inside a host application
whose memory pool already holds the whole device): its working memory is one
fixed device array in the library instead of cudaMalloc'd buffers.

The test calls it through the C ABI twice in a row, on two different
pencils, and checks each result against ghsvd_solve (the allocating entry
point) within the eigenvalue tolerance of the parity tests; the second call
also shows that what the first call left in the shared array does not leak
into the next result.  It sits in a file of its own that pytest collects
last, and it passes alone in a fresh process as well as after the others.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def noalloc_call(gh, F, G, J, w, host_j=False, **kw):
    """Direct C-ABI call: outputs are allocated here, by the test."""
    lib = gh.load()
    m, n = F.shape
    p = G.shape[0]
    Fd, Gd = dev(gh, F), dev(gh, G)
    Jh = torch.from_numpy(np.ascontiguousarray(J, dtype=np.int8))
    Jd = Jh if host_j else Jh.cuda()
    lam = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
    V = torch.empty_strided((n, n), (1, n), dtype=torch.complex128, device="cuda")
    opts = gh.ghsvd_default_opts(block_width=w, **kw)
    sweeps = ctypes.c_int(-1)
    torch.cuda.synchronize()
    s = lib.ghsvd_solve_noalloc(m, p, n, Fd.data_ptr(), m, Jd.data_ptr(), 0, Gd.data_ptr(), p,
                                lam.data_ptr(), V.data_ptr(), n, ctypes.byref(opts),
                                ctypes.byref(sweeps), None)
    torch.cuda.synchronize()
    return s, lam.cpu().numpy(), V.cpu().numpy(), sweeps.value


def allocating_call(gh, F, G, J, w, **kw):
    s = gh.Solver(0, block_width=w, **kw)
    m, n = F.shape
    p = G.shape[0]
    lam, V, sweeps, st = s.solve(dev(gh, F), dev(gh, G),
                                 torch.from_numpy(np.asarray(J, dtype=np.int8)).cuda())
    Fp, _, _ = s.factors(m, p, n)
    out = dict(status=st, lam=lam.cpu().numpy(), V=V.cpu().numpy(), sweeps=sweeps,
               F=Fp.cpu().numpy())
    s.close()
    return out


def test_noalloc_matches_allocating_solve_two_calls_in_a_row(gh):
    cases = [
        (P.single_pencil_64(), 8),
        (P.svd_pencil(537, 41, 44, 37, 10, (1e-2, 1e2), (1e-2, 1e2), permute_j=True), 5),
    ]
    for (F, J, G), w in cases:
        s, lam, V, sweeps = noalloc_call(gh, F, G, J, w)
        ref = allocating_call(gh, F, G, J, w)
        assert s == gh.GHSVD_OK and ref["status"] == gh.GHSVD_OK
        assert sweeps == ref["sweeps"]
        tol = eig_tol_vec(F, G, J, ref["lam"], ref["F"])
        assert np.all(rel_err(lam, ref["lam"]) < tol)
        # same kernels, same schedule: the eigenvectors agree column by column
        scale = np.linalg.norm(ref["V"], axis=0)[None, :]
        assert np.max(np.abs(V - ref["V"]) / scale) < 1e-9


def test_noalloc_rejects_problems_beyond_the_array(gh):
    lib = gh.load()
    n, m, p = 1024, 1536, 2048          # 4.5 n^2 x 16 bytes > 32 MiB
    F = torch.zeros((m, n), dtype=torch.complex128, device="cuda").t().contiguous().t()
    G = torch.zeros((p, n), dtype=torch.complex128, device="cuda").t().contiguous().t()
    lam = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
    s = lib.ghsvd_solve_noalloc(m, p, n, F.data_ptr(), m, None, m, G.data_ptr(), p,
                                lam.data_ptr(), None, n, None, None, None)
    assert s == gh.GHSVD_ERR_SCRATCH_TOO_SMALL
    assert "scratch" in gh.status_string(s)
    assert bool(torch.all(lam == 7.0))


def test_noalloc_not_converged_matches_allocating_solve(gh):
    # one sweep only: GHSVD_ERR_NOT_CONVERGED, one sweep reported, and lambda
    # and V still written from the factors after that sweep, as ghsvd_solve does
    F, J, G = P.single_pencil_64()
    s, lam, V, sweeps = noalloc_call(gh, F, G, J, 8, max_sweeps=1)
    ref = allocating_call(gh, F, G, J, 8, max_sweeps=1)
    assert s == gh.GHSVD_ERR_NOT_CONVERGED and ref["status"] == gh.GHSVD_ERR_NOT_CONVERGED
    assert sweeps == 1 and ref["sweeps"] == 1
    np.testing.assert_array_equal(lam, ref["lam"])
    np.testing.assert_array_equal(V, ref["V"])


def test_noalloc_rejects_host_j_shorten_and_other_orderings(gh):
    F, J, G = P.single_pencil_64()
    for kw, host_j in ((dict(), True), (dict(shorten=1), False), (dict(ordering=1), False)):
        s, lam, _, sweeps = noalloc_call(gh, F, G, J, 8, host_j=host_j, **kw)
        assert s == gh.GHSVD_ERR_INVALID_ARG, kw
        assert sweeps == 0                      # written on every return
        assert np.all(lam == 7.0)               # nothing queued, outputs untouched
    # a rejected call leaves nothing behind: the next call solves as before
    s, lam, _, sweeps = noalloc_call(gh, F, G, J, 8)
    ref = allocating_call(gh, F, G, J, 8)
    assert s == gh.GHSVD_OK and sweeps == ref["sweeps"]
    tol = eig_tol_vec(F, G, J, ref["lam"], ref["F"])
    assert np.all(rel_err(lam, ref["lam"]) < tol)


def test_noalloc_honours_the_time_limit(gh):
    # the n = 256 pencil takes dozens of sweeps of 31 steps at block width 8;
    # a 1 ms limit passes long before that: the call stops between sweeps with
    # GHSVD_ERR_TIMEOUT and the outputs of the current factors
    F, J, G = P.lapw_pencil(256)
    s, lam, _, sweeps = noalloc_call(gh, F, G, J, 8, timeout_ms=1)
    assert s == gh.GHSVD_ERR_TIMEOUT
    assert sweeps >= 1
    assert np.all(np.isfinite(lam)) and not np.all(lam == 7.0)
