"""The tensor-core (tcgen05, 3xTF32) Gram and block update of the complex64
sweeps, through the C ABI (ghsvd_tc_block_ops), against FP64 references
computed from their definitions (Section 6.4.2 eq. 6.1: the block pivot
X^* J X; Section 6.4.3: the block update X Z).

Bound: each real product is formed from TF32 parts (hi*hi + hi*lo + lo*hi,
about 2^-21 relative) and accumulated in FP32, so an entry is within a small
multiple of 2^-21 * sum_k |x_k| |y_k| of the exact value (plus FP32
accumulation); the tests allow 8e-6 of that sum (2^-17)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_08560_gb300 import build, ghsvd
    build.build()
    return ghsvd


def random_block(rng, rows, scales=True):
    X = (rng.standard_normal((rows, 64)) + 1j * rng.standard_normal((rows, 64)))
    if scales:                      # columns over six decades, as in a pencil's factors
        X *= 10.0 ** rng.uniform(-3, 3, size=64)[None, :]
    return X.astype(np.complex64)


def to_dev(gh, X):
    """Column-major complex64 CUDA tensor (the library's colmajor() would
    widen to complex128)."""
    return torch.from_numpy(np.ascontiguousarray(np.asarray(X, dtype=np.complex64).T)).cuda().t()


@pytest.mark.parametrize("rows,with_j", [(64, True), (1088, True), (1088, False), (4096, True)])
def test_tc_gram_and_update_match_fp64(gh, rows, with_j):
    rng = np.random.default_rng(rows + 7 * with_j)
    X = random_block(rng, rows)
    J = np.where(rng.random(rows) < 0.2, -1, 1).astype(np.int8) if with_j else None
    Z = (rng.standard_normal((64, 64)) + 1j * rng.standard_normal((64, 64))).astype(np.complex64)
    ident = [3, 40, 63]                          # columns e_j: must stay bit for bit
    for j in ident:
        Z[:, j] = 0
        Z[j, j] = 1
    Xd = to_dev(gh, X)
    Zd = to_dev(gh, Z)
    Jd = None if J is None else torch.from_numpy(J).cuda()
    gram = gh.ghsvd_tc_block_ops(Xd, Jd, Zd).cpu().numpy()
    Y = Xd.cpu().numpy()

    X64 = X.astype(np.complex128)
    Jf = np.ones(rows) if J is None else J.astype(np.float64)
    ref = X64.conj().T @ (Jf[:, None] * X64)
    A = np.abs(X64)
    bound = A.T @ A                               # sum_k |x_ki| |x_kj|
    err = np.abs(gram.astype(np.complex128) - ref)
    assert np.max(err / bound) < 8e-6, np.max(err / bound)

    refY = X64 @ Z.astype(np.complex128)
    boundY = A @ np.abs(Z.astype(np.complex128))
    errY = np.abs(Y.astype(np.complex128) - refY)
    assert np.max(errY / np.maximum(boundY, 1e-300)) < 8e-6, np.max(errY / boundY)
    for j in ident:
        np.testing.assert_array_equal(Y[:, j], X[:, j])


def test_tc_rejects_bad_sizes(gh):
    X = torch.zeros((64, 100), dtype=torch.complex64, device="cuda").t()
    Z = torch.eye(64, dtype=torch.complex64, device="cuda")
    with pytest.raises(gh.GhsvdError) as e:
        gh.ghsvd_tc_block_ops(X, None, Z)
    assert e.value.status == gh.GHSVD_ERR_INVALID_ARG
