"""Checks at the benchmark's full size: the n = 2048 LAPW-shaped pencil
(F 3072 x 2048 with 512 negative signs, G 4096 x 2048, cond(S) = 1e10) in the
benchmark's configuration (block width 32, C_max 80).

The eigenvalues of every solve (FP64, mixed precision with FP64 or FP32 2x2
parameters, Phase 2 first) are compared element by element with the FP64
oracle's, stored in tests/golden/fullsize_oracle.json by
tests/golden/make_fullsize.py (a whole blocked oracle solve on the CPU), within
the per-eigenvalue tolerance 1e-12 * max(1, (cond(F_c) + cond(G_c)) / 1e3) * a_j
(eq. 3.2; a_j the hyperbolic amplification of the oracle's converged column j).
Beside that, properties that hold at any size: the definition of the outputs
(eq. 3.2: V^* S V = I, V^* H V diagonal, computed through the factors, never
through S) and Sylvester's inertia."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import pencils as P
from conftest import fullsize_golden, golden_ratio

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fp64():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_08560_gb300 import build, ghsvd
    build.build()
    F, J, G = P.lapw_pencil(2048)
    Fd = ghsvd.colmajor(torch.from_numpy(F)).cuda()
    Gd = ghsvd.colmajor(torch.from_numpy(G)).cuda()
    Jd = torch.from_numpy(J).cuda()
    s = ghsvd.Solver(0, block_width=32, max_sweeps=80)
    lam, V, sweeps, st = s.solve(Fd, Gd, Jd)
    torch.cuda.synchronize()
    Fp, _, _ = s.factors(F.shape[0], G.shape[0], F.shape[1])
    F1 = Fp.cpu().numpy()
    s.close()
    # hyperbolic amplification of each converged column (reading 12)
    amp = (np.einsum("ij,ij->j", F1.conj(), F1).real /
           np.abs(np.einsum("ij,i,ij->j", F1.conj(), J.astype(np.float64), F1).real))
    return dict(gh=ghsvd, F=Fd, G=Gd, J=Jd, lam=lam, V=V, sweeps=sweeps, status=st, amp=amp)


def test_fullsize_fp64_solve_converges(fp64):
    assert fp64["status"] == 0 and 1 <= fp64["sweeps"] <= 80


def test_fullsize_outputs_satisfy_the_definition(fp64):
    F, G, V, lam = fp64["F"], fp64["G"], fp64["V"], fp64["lam"]
    n = V.shape[1]
    GV = G @ V
    e = (GV.conj().T @ GV - torch.eye(n, dtype=GV.dtype, device=GV.device)).abs().max().item()
    assert e < 1e-9, e                                            # V^* S V = I (measured 1.3e-10)
    FV = F @ V
    Jd = fp64["J"].to(torch.float64)
    HV = FV.conj().T @ (Jd[:, None] * FV)                          # V^* H V
    dg = torch.diagonal(HV).real
    scale = torch.sqrt(torch.outer(dg.abs(), dg.abs()))
    off = ((HV - torch.diag(torch.diagonal(HV))).abs() / scale).max().item()
    assert off < 1e-6, off                                        # measured 1.2e-7
    assert torch.equal(torch.sign(lam), torch.sign(dg))
    r = ((dg - lam).abs() / lam.abs()).max().item()               # lambda_j = v_j^* H v_j
    assert r < 5e-7, r                                            # measured 5.8e-8


def test_fullsize_inertia(fp64):
    # Sylvester: with S > 0 the pencil has the inertia of H = F^* J F
    F, Jd = fp64["F"], fp64["J"].to(torch.float64)
    H = F.conj().T @ (Jd[:, None] * F)
    ev = torch.linalg.eigvalsh(H)
    assert int((ev < 0).sum()) == int((fp64["lam"] < 0).sum())


def test_fullsize_fp64_matches_oracle(fp64):
    g = fullsize_golden("lapw2048")
    assert golden_ratio(fp64["lam"].cpu().numpy(), g) < 1.0


@pytest.mark.parametrize("kind", ["mixed", "mixed_param32", "mixed_cuda_cores", "shortened"])
def test_fullsize_variants_match_oracle_and_fp64(fp64, kind):
    gh = fp64["gh"]
    opts = dict(block_width=32, max_sweeps=80)
    if kind.startswith("mixed"):
        opts.update(precision=gh.GHSVD_PRECISION_MIXED, mixed_max_sweeps=60,
                    mixed_param32=int(kind == "mixed_param32"),
                    mixed_tc=int(kind != "mixed_cuda_cores"))
    else:
        opts.update(shorten=1)
    s = gh.Solver(0, **opts)
    lam, _, _, st = s.solve(fp64["F"], fp64["G"], fp64["J"], want_vectors=False)
    torch.cuda.synchronize()
    s.close()
    assert st == 0
    ref = fp64["lam"].cpu().numpy()
    order = np.argsort(ref)
    tol = 1e-12 * max(1.0, (1e6 + 1e5) / 1e3) * fp64["amp"][order]
    err = np.abs(np.sort(lam.cpu().numpy()) - ref[order]) / np.abs(ref[order])
    assert np.all(err < tol), (err / tol).max()
    assert golden_ratio(lam.cpu().numpy(), fullsize_golden("lapw2048")) < 1.0
