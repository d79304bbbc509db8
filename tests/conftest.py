import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


def rel_err(a, b):
    """Element-wise relative error of sorted eigenvalue vectors."""
    a = np.sort(np.asarray(a, dtype=np.float64))
    b = np.sort(np.asarray(b, dtype=np.float64))
    return np.abs(a - b) / np.maximum(np.abs(b), np.finfo(float).tiny)


def cond_cols(X):
    """2-norm condition number of X with its columns scaled to unit norm."""
    X = np.asarray(X)
    Xc = X / np.linalg.norm(X, axis=0)[None, :]
    s = np.linalg.svd(Xc, compute_uv=False)
    return s[0] / s[-1]


def eig_tol(F, G):
    """Relative eigenvalue tolerance for FP64 results on the pencil (F, G):
    1e-12 * max(1, (cond(F_c) + cond(G_c)) / 1e3), F_c, G_c column-scaled."""
    return 1e-12 * max(1.0, (cond_cols(F) + cond_cols(G)) / 1e3)


def hyperbolic_amp(Fp, J):
    """a_j = ||f_j||^2 / |f_j^* J f_j| >= 1 for converged columns f_j of F'.

    The cancellation between the +1 and the -1 rows in the J-norm of the
    eigenvector's column magnifies the relative error of lambda_j by a_j
    (a_j = 1 when J = I or the column lives on rows of one sign)."""
    Fp = np.asarray(Fp)
    if J is None:
        return np.ones(Fp.shape[1])
    Jf = np.asarray(J, dtype=np.float64)
    hf = np.einsum("ij,i,ij->j", Fp.conj(), Jf, Fp).real
    fn = np.einsum("ij,ij->j", Fp.conj(), Fp).real
    return fn / np.maximum(np.abs(hf), np.finfo(float).tiny)


def eig_tol_vec(F, G, J, ref_lam, ref_F):
    """Per-eigenvalue FP64 tolerance, ordered like np.sort(ref_lam):
    1e-12 * max(1, (cond(F_c) + cond(G_c)) / 1e3) * a_j, with a_j the
    hyperbolic amplification of the reference's converged column j."""
    amp = hyperbolic_amp(ref_F, J)
    order = np.argsort(np.asarray(ref_lam))
    return eig_tol(F, G) * amp[order]


def fullsize_golden(name):
    """A case of tests/golden/fullsize_oracle.json (written by
    tests/golden/make_fullsize.py from the FP64 oracle alone): the oracle's
    eigenvalues sorted ascending, and the per-eigenvalue FP64 tolerance
    1e-12 * max(1, (cond(F_c) + cond(G_c)) / 1e3) * a_j in the same order."""
    import json
    path = os.path.join(ROOT, "tests", "golden", "fullsize_oracle.json")
    with open(path) as f:
        cases = {c["name"]: c for c in json.load(f)["cases"]}
    c = dict(cases[name])
    c["lam"] = np.array([float(x) for x in c["lam"]])
    c["amp"] = np.array([float(x) for x in c["amp"]])
    c["tol"] = 1e-12 * max(1.0, (c["cond_F_c"] + c["cond_G_c"]) / 1e3) * c["amp"]
    return c


def golden_ratio(lam, golden):
    """max_j |lam_j - lam_j^oracle| / (|lam_j^oracle| tol_j), both sorted ascending."""
    ref = golden["lam"]
    err = np.abs(np.sort(np.asarray(lam, dtype=np.float64)) - ref) / np.abs(ref)
    return float(np.max(err / golden["tol"]))
