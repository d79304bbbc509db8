"""The three block-update routes of the FP64 sweeps (ghsvd_fp64_block_update)
against an extended-precision product: the FP64 product X Z, and the delta
form X + X (Z - I) with the product in FP32 (every entry of Z - I at most
2^-29) or in double-float arithmetic (at most 2^-11), each within its stated
error bound (include/ghsvd.h, the delta_update option)."""
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


def cplx(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def run(gh, X, Z, route):
    Xd = gh.colmajor(torch.from_numpy(X)).cuda()
    Zd = gh.colmajor(torch.from_numpy(Z)).cuda()
    gh.ghsvd_fp64_block_update(Xd, Zd, route)
    return Xd.cpu().numpy()


@pytest.mark.parametrize("route,emax", [(0, 2.0 ** -29), (1, 2.0 ** -11), (2, 0.5)])
def test_fp64_block_update_route_within_its_bound(gh, route, emax):
    rng = np.random.default_rng(1907 + route)
    rows = 256
    # columns of very different norms, as the stacked factors hold
    X = cplx(rng, (rows, 64)) * 10.0 ** rng.uniform(-3, 3, 64)
    E = emax * (rng.uniform(-1, 1, (64, 64)) + 1j * rng.uniform(-1, 1, (64, 64)))
    E[:, 7] = 0.0                         # an untouched column: Z e_7 = e_7
    Z = np.eye(64) + E
    out = run(gh, X, Z, route)
    # reference in extended precision (80-bit or quad long double)
    Xl, El = X.astype(np.clongdouble), E.astype(np.clongdouble)
    ref = Xl + Xl @ El
    err = np.abs(out.astype(np.clongdouble) - ref).astype(np.float64)
    ax, ae = np.abs(X), np.abs(E)
    sxe = ax @ ae                          # sum_l |x_il| |e_lj|
    aref = np.abs(ref).astype(np.float64)
    u = 2.0 ** -53
    if route == 0:
        bound = 68 * 2.0 ** -24 * sxe + 2 * u * aref
    elif route == 1:
        bound = 2.0 ** -40 * sxe + 2 * u * aref
    else:
        bound = 2 * 64 * u * (ax @ np.abs(Z)) + 2 * u * aref
    assert np.all(err <= bound), float(np.max(err / bound))
    if route in (0, 1):
        # the delta forms leave an untouched column exactly as it was
        assert np.array_equal(out[:, 7], X[:, 7])


def test_fp64_block_update_rejects_bad_arguments(gh):
    X = gh.colmajor(torch.zeros((100, 64), dtype=torch.complex128)).cuda()     # rows not a multiple of 64
    Z = gh.colmajor(torch.eye(64, dtype=torch.complex128)).cuda()
    with pytest.raises(gh.GhsvdError):
        gh.ghsvd_fp64_block_update(X, Z, 1)
    X = gh.colmajor(torch.zeros((128, 64), dtype=torch.complex128)).cuda()
    with pytest.raises(gh.GhsvdError):
        gh.ghsvd_fp64_block_update(X, Z, 3)
