"""FP64 CPU oracle for the implicit one-sided Hari-Zimmermann GHSVD.

TEST INFRASTRUCTURE ONLY: the independent checker of the CUDA path.  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It shares no code with the GPU library.

The arithmetic lives in ``hz_oracle.c`` (plain C, ``double complex``), which
follows arXiv 1907.08560 Section 6 step by step, and ``phase24_oracle.c``
(Phase 2 of Section 5 and Phase 4 of Section 7); this module only compiles
them and marshals numpy arrays (column-major complex128) to them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hz_oracle.c")
_SRC24 = os.path.join(_HERE, "phase24_oracle.c")
_LIB = os.path.join(_HERE, "libhz_oracle.so")

_lib = None


def build(force: bool = False, out: str | None = None, defines: tuple[str, ...] = ()) -> str:
    """Compile the oracle sources with gcc (-O2, OpenMP) into a shared library."""
    out = out or _LIB
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC24))
    if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=gnu11",
           "-fno-fast-math", "-ffp-contract=off", *[f"-D{d}" for d in defines],
           _SRC, _SRC24, "-o", out, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def _bind(lib):
    c_long, c_int, c_double, vp = ctypes.c_long, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    lib.hzo_pointwise.restype = c_int
    lib.hzo_pointwise.argtypes = [c_long, c_long, c_long, vp, c_long, vp, vp, c_long, vp,
                                  c_long, c_int, c_int, c_int, ctypes.POINTER(c_long), vp]
    lib.hzo_blocked.restype = c_int
    lib.hzo_blocked.argtypes = [c_long, c_long, c_long, vp, c_long, vp, vp, c_long, vp, c_long,
                                c_long, c_int, c_int, c_int, c_int, ctypes.POINTER(c_long), vp]
    lib.hzo_blocked_step.restype = c_long
    lib.hzo_blocked_step.argtypes = [c_long, c_long, c_long, vp, c_long, vp, vp, c_long, vp,
                                     c_long, c_long, c_int, c_long, c_int, c_int,
                                     ctypes.POINTER(c_long)]
    lib.hzo_block_pivot.restype = c_long
    lib.hzo_block_pivot.argtypes = [c_long, c_long, c_long, vp, c_long, vp, vp, c_long, c_long,
                                    c_int, c_long, c_long, c_int, vp, vp, vp, vp, vp,
                                    ctypes.POINTER(c_long), ctypes.POINTER(c_long)]
    lib.hzo_finalize.restype = c_int
    lib.hzo_finalize.argtypes = [c_long, c_long, c_long, vp, c_long, vp, vp, c_long, vp, c_long,
                                 vp, vp, c_long, vp, vp]
    lib.hzo_partition.restype = c_long
    lib.hzo_partition.argtypes = [c_long, c_long, vp, c_long]
    lib.hzo_rr_table.restype = None
    lib.hzo_rr_table.argtypes = [c_long, vp]
    lib.hzo_max_threads.restype = c_int
    lib.hzo_rank_check.restype = c_int
    lib.hzo_rank_check.argtypes = [c_long, c_long, vp, c_long, vp, c_long, ctypes.POINTER(c_double)]
    lib.hzo_pivot2.restype = c_int
    lib.hzo_pivot2.argtypes = [vp, c_double, c_int, vp, ctypes.POINTER(c_int)]
    lib.p24_jqr.restype = c_int
    lib.p24_jqr.argtypes = [c_long, c_long, vp, c_long, vp, vp, ctypes.POINTER(c_long)]
    lib.p24_qr.restype = c_int
    lib.p24_qr.argtypes = [c_long, c_long, vp, c_long]
    lib.p24_lu_complete.restype = c_int
    lib.p24_lu_complete.argtypes = [c_long, vp, c_long, vp, vp]
    lib.p24_inverse.restype = c_int
    lib.p24_inverse.argtypes = [c_long, vp, c_long, vp, vp, vp, c_long]
    return lib


def load(path: str | None = None):
    """Load (building if needed) the oracle library; ``path`` loads a variant."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _fortran(a, dtype=np.complex128):
    return np.array(a, dtype=dtype, order="F", copy=True)


def _signs(J, m):
    if J is None:
        return None
    J = np.ascontiguousarray(np.asarray(J), dtype=np.int8)
    if J.shape != (m,) or not np.all(np.abs(J) == 1):
        raise ValueError("J must hold m entries equal to +1 or -1")
    return J


EPS = 2.0 ** -53


def pivot(hpp, hqq, hpq, spp, sqq, spq, n=2, crit_mode=0, lib=None):
    """The 2x2 transformation Z' of Section 6.1 (eq. 6.1-6.12).

    Returns ``(rc, Zp, big)``: rc 1 = transform, 0 = none, <0 = error; Zp is
    the 2x2 complex matrix D0^ Z^.
    """
    lib = lib or load()
    hpq = complex(hpq)
    spq = complex(spq)
    inp = np.array([hpp, hqq, hpq.real, hpq.imag, spp, sqq, spq.real, spq.imag], dtype=np.float64)
    Z = np.zeros(4, dtype=np.complex128)
    big = ctypes.c_int(0)
    rc = lib.hzo_pivot2(_ptr(inp), EPS * np.sqrt(n), crit_mode, _ptr(Z), ctypes.byref(big))
    return rc, Z.reshape(2, 2), big.value


def pointwise(F, G, J=None, Z0=None, max_sweeps=30, crit_mode=0, nthreads=0, lib=None):
    """Algorithm 1 (Section 6.1.8).  Returns dict(F, G, Z, status, sweeps, counts)."""
    lib = lib or load()
    F = _fortran(F); G = _fortran(G)
    m, n = F.shape
    p = G.shape[0]
    Jv = _signs(J, m)
    Z = _fortran(np.eye(n) if Z0 is None else Z0)
    sweeps = ctypes.c_long(0)
    counts = np.zeros(2 * max(max_sweeps, 1), dtype=np.int64)
    rc = lib.hzo_pointwise(m, p, n, _ptr(F), m, _ptr(Jv), _ptr(G), p, _ptr(Z), n, max_sweeps,
                           crit_mode, nthreads, ctypes.byref(sweeps), _ptr(counts))
    s = sweeps.value
    return dict(F=F, G=G, Z=Z, status=rc, sweeps=s, counts=counts[: 2 * s].reshape(-1, 2))


def blocked(F, G, J=None, w=32, inner_sweeps=1, Z0=None, max_sweeps=30, crit_mode=0,
            nthreads=0, lib=None):
    """The Level-2 block algorithm of Section 6.4 (BO: inner_sweeps=1)."""
    lib = lib or load()
    F = _fortran(F); G = _fortran(G)
    m, n = F.shape
    p = G.shape[0]
    Jv = _signs(J, m)
    Z = _fortran(np.eye(n) if Z0 is None else Z0)
    sweeps = ctypes.c_long(0)
    counts = np.zeros(2 * max(max_sweeps, 1), dtype=np.int64)
    rc = lib.hzo_blocked(m, p, n, _ptr(F), m, _ptr(Jv), _ptr(G), p, _ptr(Z), n, w, inner_sweeps,
                         max_sweeps, crit_mode, nthreads, ctypes.byref(sweeps), _ptr(counts))
    s = sweeps.value
    return dict(F=F, G=G, Z=Z, status=rc, sweeps=s, counts=counts[: 2 * s].reshape(-1, 2))


def blocked_step(F, G, J=None, Z=None, w=32, r=0, inner_sweeps=1, crit_mode=0, lib=None):
    """One outer step r of the block algorithm; returns (F, G, Z, n_all, n_big)."""
    lib = lib or load()
    F = _fortran(F); G = _fortran(G)
    m, n = F.shape
    p = G.shape[0]
    Jv = _signs(J, m)
    Z = _fortran(np.eye(n) if Z is None else Z)
    nbig = ctypes.c_long(0)
    na = lib.hzo_blocked_step(m, p, n, _ptr(F), m, _ptr(Jv), _ptr(G), p, _ptr(Z), n, w,
                              inner_sweeps, r, crit_mode, 0, ctypes.byref(nbig))
    if na < 0:
        raise RuntimeError(f"hzo_blocked_step failed: {na}")
    return F, G, Z, na, nbig.value


def time_blocked_steps(F, G, J=None, w=32, target_s=10.0, nthreads=0, max_steps=10**9,
                       lib=None):
    """Run consecutive outer steps r = 0, 1, ... of the first block sweep in
    place on copies of (F, G, I) until target_s seconds (at least one step,
    at most max_steps); returns (mean seconds per step, steps run)."""
    import time
    lib = lib or load()
    F = _fortran(F); G = _fortran(G)
    m, n = F.shape
    p = G.shape[0]
    Jv = _signs(J, m)
    Z = _fortran(np.eye(n))
    nsteps_sweep = len(partition(n, w, lib=lib)) - 2
    nbig = ctypes.c_long(0)
    t0 = time.perf_counter()
    steps = 0
    while True:
        r = steps % nsteps_sweep
        na = lib.hzo_blocked_step(m, p, n, _ptr(F), m, _ptr(Jv), _ptr(G), p, _ptr(Z), n, w, 1, r,
                                  0, nthreads, ctypes.byref(nbig))
        if na < 0:
            raise RuntimeError(f"hzo_blocked_step failed: {na}")
        steps += 1
        el = time.perf_counter() - t0
        if steps >= max_steps or el >= target_s:
            break
    return el / steps, steps


def block_pivot(F, G, J=None, w=32, r=0, k=0, inner_sweeps=1, crit_mode=0, lib=None):
    """Block pivots (H0, S0) of pair k in step r, and after the inner level (H, S, Zhat)."""
    lib = lib or load()
    F = _fortran(F); G = _fortran(G)
    m, n = F.shape
    p = G.shape[0]
    Jv = _signs(J, m)
    off = np.zeros(n + 2, dtype=np.int64)
    nb = lib.hzo_partition(n, w, _ptr(off), n + 1)
    kk = 2 * int(off[1] - off[0])
    bufs = [np.zeros((kk, kk), dtype=np.complex128, order="F") for _ in range(5)]
    n_all = ctypes.c_long(0)
    nbig = ctypes.c_long(0)
    rc = lib.hzo_block_pivot(m, p, n, _ptr(F), m, _ptr(Jv), _ptr(G), p, w, inner_sweeps, r, k,
                             crit_mode, *[_ptr(b) for b in bufs], ctypes.byref(n_all),
                             ctypes.byref(nbig))
    if rc < 0:
        raise RuntimeError(f"hzo_block_pivot failed: {rc}")
    H, S, Zh, H0, S0 = bufs
    return dict(H0=H0, S0=S0, H=H, S=S, Z=Zh, n_all=n_all.value, n_big=nbig.value, nb=nb)


def finalize(F, G, Z, J=None, lib=None):
    """Outputs of Section 6.1.7 / eq. 3.2: (lambda, V, Sigma_F', Sigma_G')."""
    lib = lib or load()
    F = _fortran(F); G = _fortran(G); Z = _fortran(Z)
    m, n = F.shape
    p = G.shape[0]
    Jv = _signs(J, m)
    lam = np.zeros(n)
    V = np.zeros((n, n), dtype=np.complex128, order="F")
    sf = np.zeros(n)
    sg = np.zeros(n)
    rc = lib.hzo_finalize(m, p, n, _ptr(F), m, _ptr(Jv), _ptr(G), p, _ptr(Z), n, _ptr(lam),
                          _ptr(V), n, _ptr(sf), _ptr(sg))
    if rc != 0:
        raise RuntimeError(f"hzo_finalize failed: {rc}")
    return lam, V, sf, sg


def rank_check(G, V, lib=None):
    """(status, kappa_est): status -2 if G is numerically rank deficient."""
    lib = lib or load()
    G = _fortran(G); V = _fortran(V)
    k = ctypes.c_double(0.0)
    rc = lib.hzo_rank_check(G.shape[0], G.shape[1], _ptr(G), G.shape[0], _ptr(V), V.shape[0],
                            ctypes.byref(k))
    return rc, k.value


def solve(F, G, J=None, method="pointwise", lib=None, **kw):
    """Run the oracle, finalize and check the rank of G.

    Returns a dict with lam (unsorted), V, the transformed factors and the
    status (0 converged, 1 max_sweeps reached, <0 error)."""
    if method == "pointwise":
        out = pointwise(F, G, J, lib=lib, **kw)
    else:
        out = blocked(F, G, J, lib=lib, **kw)
    if out["status"] < 0:
        return out
    lam, V, sf, sg = finalize(out["F"], out["G"], out["Z"], J, lib=lib)
    rc, kappa = rank_check(G, V, lib=lib)
    if rc < 0:
        out["status"] = rc
    out.update(lam=lam, V=V, sigma_f=sf, sigma_g=sg, kappa_est=kappa)
    return out


def partition(n, w, lib=None):
    lib = lib or load()
    off = np.zeros(n + 2, dtype=np.int64)
    nb = lib.hzo_partition(n, w, _ptr(off), n + 1)
    return off[: nb + 1].copy() if nb > 0 else None


def rr_table(N, lib=None):
    lib = lib or load()
    t = np.zeros((N - 1, N // 2, 2), dtype=np.int64)
    lib.hzo_rr_table(N, _ptr(t))
    return t


def max_threads(lib=None):
    return (lib or load()).hzo_max_threads()


# --------------------------------------------------------------------------
# Phase 2 (Section 5) and Phase 4 (Section 7).
# --------------------------------------------------------------------------

def jqr(F, J=None, lib=None):
    """The hyperbolic QR of Section 5 (p24_jqr).

    Returns dict(R = the n x n block upper triangular factor, J = its
    signature (n entries), perm (F~[:, perm] = F~ P2), n2x2, status, and the
    whole transformed m x n factor ``full`` with its row-permuted ``J_full``)."""
    lib = lib or load()
    F = _fortran(F)
    m, n = F.shape
    Jv = np.ones(m, dtype=np.int8) if J is None else _signs(J, m).copy()
    perm = np.zeros(n, dtype=np.int64)
    n2 = ctypes.c_long(0)
    rc = lib.p24_jqr(m, n, _ptr(F), m, _ptr(Jv), _ptr(perm), ctypes.byref(n2))
    return dict(R=np.asfortranarray(F[:n, :]), J=Jv[:n].copy(), perm=perm, n2x2=n2.value,
                status=rc, full=F, J_full=Jv)


def qr(G, lib=None):
    """Householder QR of G (p24_qr): the n x n upper triangular R with G^*G = R^*R."""
    lib = lib or load()
    G = _fortran(G)
    p, n = G.shape
    rc = lib.p24_qr(p, n, _ptr(G), p)
    if rc != 0:
        raise RuntimeError(f"p24_qr failed: {rc}")
    return np.asfortranarray(G[:n, :])


def urv(F, G, J=None, lib=None):
    """Phase 2: the square pencil (R_F, J', R_G) of the tall (F~, J~, G~):
    R_F from the JQR of F~, R_G from the QR of G~ P2 (Section 5).
    Returns dict(F, J, G, perm, n2x2, status)."""
    out = jqr(F, J, lib=lib)
    if out["status"] != 0:
        return dict(status=out["status"])
    Gp = np.asarray(G)[:, out["perm"]]
    return dict(F=out["R"], J=out["J"], G=qr(Gp, lib=lib), perm=out["perm"],
                n2x2=out["n2x2"], status=0)


def lu_complete(A, lib=None):
    """P A Q = L U by complete pivoting (p24_lu_complete); returns (LU, rowp, colp, status)."""
    lib = lib or load()
    A = _fortran(A)
    n = A.shape[0]
    rowp = np.zeros(n, dtype=np.int64)
    colp = np.zeros(n, dtype=np.int64)
    rc = lib.p24_lu_complete(n, _ptr(A), n, _ptr(rowp), _ptr(colp))
    return A, rowp, colp, rc


def inverse(Z, lib=None):
    """X = Z^{-1} by complete pivoting and Z X = I (Section 7)."""
    lib = lib or load()
    LU, rowp, colp, rc = lu_complete(Z, lib=lib)
    if rc != 0:
        raise RuntimeError(f"p24_lu_complete failed: {rc}")
    n = LU.shape[0]
    X = np.zeros((n, n), dtype=np.complex128, order="F")
    rc = lib.p24_inverse(n, _ptr(LU), n, _ptr(rowp), _ptr(colp), _ptr(X), n)
    if rc != 0:
        raise RuntimeError(f"p24_inverse failed: {rc}")
    return X


def ghsvd(F, G, J, Fp, Gp, Zp, lib=None):
    """Phase 4 and the errors of eq. 7.1 for converged factors F' = F Z',
    G' = G Z' (Section 6.1.7 outputs, Section 7):
    Sigma_F' = |f'_j^* J f'_j|^{1/2}, Sigma_G' = ||g'_j||,
    Sigma = (Sigma_F'^2 + Sigma_G'^2)^{1/2}, Z = Z' Sigma^{-1}, X = Z^{-1},
    U = F' Sigma_F'^{-1}, V = G' Sigma_G'^{-1}, Sigma_F = Sigma_F' / Sigma,
    Sigma_G = Sigma_G' / Sigma, and
    err_F = ||F - U Sigma_F X||_F / ||F||_F, err_G = ||G - V Sigma_G X||_F / ||G||_F."""
    F = np.asarray(F); G = np.asarray(G)
    Fp = np.asarray(Fp); Gp = np.asarray(Gp); Zp = np.asarray(Zp)
    m = F.shape[0]
    Jd = np.ones(m) if J is None else np.asarray(J, dtype=np.float64)
    sfp = np.sqrt(np.abs(np.einsum("ij,i,ij->j", Fp.conj(), Jd, Fp).real))
    sgp = np.sqrt(np.einsum("ij,ij->j", Gp.conj(), Gp).real)
    sig = np.sqrt(sfp ** 2 + sgp ** 2)
    Z = Zp / sig[None, :]
    X = inverse(Z, lib=lib)
    U = Fp / sfp[None, :]
    V = Gp / sgp[None, :]
    SF, SG = sfp / sig, sgp / sig
    errF = np.linalg.norm(F - (U * SF[None, :]) @ X) / np.linalg.norm(F)
    errG = np.linalg.norm(G - (V * SG[None, :]) @ X) / np.linalg.norm(G)
    return dict(X=X, Z=Z, U=U, V=V, sigma_f=SF, sigma_g=SG, sigma=sig, err_F=errF, err_G=errG)
