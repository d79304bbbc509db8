"""Extended-precision brute force for small pencils (test infrastructure only).

Forms H = F^* J F and S = G^* G in multi-precision arithmetic (mpmath),
factors S = L L^* by Cholesky, and takes the Hermitian eigenvalues of
L^{-1} H L^{-*}: the textbook reduction of the definite pencil (H, S)
(arXiv 1907.08560, Section 3, eq. 3.2).  Forming S squares cond(G), which
ruins this route in FP64 (the failure mode of the formed-H, S solver the
paper compares against, Section 6.5.4); at 50 significant digits it does
not matter for cond(G) up to ~1e10.
"""
from __future__ import annotations

import numpy as np


def generalized_eigenvalues(F, G, J=None, dps: int = 50) -> np.ndarray:
    """Eigenvalues of (F^* J F, G^* G), ascending, as float64."""
    import mpmath as mp

    F = np.asarray(F)
    G = np.asarray(G)
    m, n = F.shape
    p = G.shape[0]
    Jv = np.ones(m) if J is None else np.asarray(J, dtype=np.float64)
    with mp.workdps(dps):
        Fm = mp.matrix(m, n)
        Gm = mp.matrix(p, n)
        for i in range(m):
            for j in range(n):
                Fm[i, j] = mp.mpc(float(F[i, j].real), float(F[i, j].imag))
        for i in range(p):
            for j in range(n):
                Gm[i, j] = mp.mpc(float(G[i, j].real), float(G[i, j].imag))
        JF = mp.matrix(m, n)
        for i in range(m):
            for j in range(n):
                JF[i, j] = Fm[i, j] * int(Jv[i])
        H = Fm.transpose_conj() * JF
        S = Gm.transpose_conj() * Gm
        L = mp.cholesky(S)
        Li = mp.inverse(L)
        C = Li * H * Li.transpose_conj()
        for i in range(n):           # exact Hermitian symmetry
            C[i, i] = mp.re(C[i, i])
            for j in range(i + 1, n):
                C[j, i] = mp.conj(C[i, j])
        ev = mp.eighe(C, eigvals_only=True)
        lam = np.array(sorted(float(mp.re(x)) for x in ev))
    return lam
