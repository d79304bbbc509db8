"""Seeded synthetic pencils (F, J, G) for tests and benchmarks.

This module draws random inputs only: it holds none of the Hari-Zimmermann
arithmetic, and both the CUDA path and the CPU oracle consume what it makes.

Layout: every matrix is a complex128 numpy array in column-major (Fortran)
order, the layout of the library's C ABI.  ``J`` is an int8 vector of +-1.

The pencils stand in for the LAPW datasets of arXiv 1907.08560 (Table in
Section 3.2), which are not available: tall factors with ``m`` and ``p``
between 1.5 and 2 times ``n``, a signature with both signs (positives first,
as the Hermitian indefinite factorization of Section 4 arranges them) and
ill-conditioned ``G``.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1907085600


def rng_for(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(int(seed)))


def haar_columns(rng: np.random.Generator, m: int, n: int) -> np.ndarray:
    """m x n matrix with orthonormal columns, Haar distributed.

    QR of a complex Gaussian matrix, with the phases of R's diagonal moved
    into Q (Mezzadri, "How to generate random matrices from the classical
    compact groups", Notices AMS 54, 2007).
    """
    if n > m:
        raise ValueError("need n <= m")
    Z = (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))) / np.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R)
    ph = d / np.abs(d)
    return np.asfortranarray(Q * ph[None, :])


def log_uniform(rng: np.random.Generator, n: int, lo: float, hi: float) -> np.ndarray:
    """n values log-uniform on [lo, hi] with both endpoints present (n >= 2)."""
    if n == 1:
        return np.array([np.sqrt(lo * hi)])
    e = rng.uniform(np.log10(lo), np.log10(hi), size=n)
    e[0], e[1] = np.log10(lo), np.log10(hi)
    rng.shuffle(e)
    return 10.0 ** e


def signature(m: int, m_minus: int, permute: np.random.Generator | None = None) -> np.ndarray:
    """J = diag(+1 x (m - m_minus), -1 x m_minus), positives first unless permuted."""
    J = np.ones(m, dtype=np.int8)
    J[m - m_minus:] = -1
    if permute is not None:
        J = J[permute.permutation(m)]
    return J


def svd_factor(rng: np.random.Generator, rows: int, n: int, sigma: np.ndarray) -> np.ndarray:
    """U diag(sigma) W^* with Haar U (rows x n, orthonormal columns) and Haar W (n x n)."""
    U = haar_columns(rng, rows, n)
    W = haar_columns(rng, n, n)
    return np.asfortranarray((U * sigma[None, :]) @ W.conj().T)


def svd_pencil(seed: int, m: int, p: int, n: int, m_minus: int,
               sf=(1e-3, 1e3), sg=(1e-3, 1e3), permute_j: bool = False):
    """F = U_F diag(s_F) W_F^*, G = U_G diag(s_G) W_G^*, log-uniform singular values."""
    rng = rng_for(seed)
    s_f = log_uniform(rng, n, *sf)
    s_g = log_uniform(rng, n, *sg)
    F = svd_factor(rng, m, n, s_f)
    G = svd_factor(rng, p, n, s_g)
    J = signature(m, m_minus, rng if permute_j else None)
    return F, J, G


def known_pencil(seed: int, m: int, p: int, n: int, m_minus: int, n_minus: int,
                 cond_x: float = 10.0, a_range=(0.1, 10.0), b_range=(0.1, 10.0),
                 hyper: float = 0.0, n_hyper: int = 0):
    """A pencil whose generalized eigenvalues are known by construction (eq. 3.1).

    F = U_F E diag(a) X and G = U_G diag(b) X, where
      - J = diag(+1 x (m - m_minus), -1 x m_minus);
      - U_F is J-unitary: block-diagonal Haar unitaries on the +1 and the -1
        rows, times ``n_hyper`` hyperbolic rotations of angle up to ``hyper``
        between a +1 row and a -1 row (U_F^* J U_F = J);
      - E (m x n) puts column j of diag(a) X on its own row r_j, with
        ``n_minus`` of those rows among the -1 rows;
      - U_G (p x n) has Haar orthonormal columns;
      - X (n x n) = W1 diag(x) W2^* with cond(X) = cond_x.
    Then H = F^* J F = X^* diag(J[r_j] a_j^2) X and S = G^* G = X^* diag(b_j^2) X,
    so the eigenvalues of (H, S) are lambda_j = J[r_j] a_j^2 / b_j^2.
    Returns (F, J, G, lam) with lam sorted ascending.
    """
    if not (0 <= n_minus <= min(m_minus, n)) or n - n_minus > m - m_minus:
        raise ValueError("cannot place the columns on rows of the requested signs")
    rng = rng_for(seed)
    m_plus = m - m_minus
    J = signature(m, m_minus)
    UF = np.zeros((m, m), dtype=np.complex128)
    UF[:m_plus, :m_plus] = haar_columns(rng, m_plus, m_plus) if m_plus else 0
    if m_minus:
        UF[m_plus:, m_plus:] = haar_columns(rng, m_minus, m_minus)
    for _ in range(n_hyper if m_plus and m_minus else 0):
        i = rng.integers(0, m_plus)
        j = m_plus + rng.integers(0, m_minus)
        t = rng.uniform(-hyper, hyper)
        c, s = np.cosh(t), np.sinh(t)
        ri, rj = UF[i].copy(), UF[j].copy()
        UF[i], UF[j] = c * ri + s * rj, s * ri + c * rj
    rows_minus = m_plus + rng.choice(m_minus, size=n_minus, replace=False) if n_minus else []
    rows_plus = rng.choice(m_plus, size=n - n_minus, replace=False)
    rows = np.concatenate([np.asarray(rows_minus, dtype=np.int64), rows_plus.astype(np.int64)])
    rng.shuffle(rows)
    a = log_uniform(rng, n, *a_range)
    b = log_uniform(rng, n, *b_range)
    xs = log_uniform(rng, n, 1.0, cond_x) if n > 1 else np.ones(1)
    X = (haar_columns(rng, n, n) * xs[None, :]) @ haar_columns(rng, n, n).conj().T
    EA = np.zeros((m, n), dtype=np.complex128)
    EA[rows, np.arange(n)] = a
    F = np.asfortranarray(UF @ (EA @ X))
    G = np.asfortranarray((haar_columns(rng, p, n) * b[None, :]) @ X)
    lam = np.sort(J[rows].astype(np.float64) * a * a / (b * b))
    return F, J, G, lam


# --------------------------------------------------------------------------
# The workloads (shapes and distributions of the LAPW-like pencils).
# --------------------------------------------------------------------------

def single_pencil_64(seed: int = SEED_BASE + 1):
    """n = 64: F 96 x 64 with J = diag(+1 x 80, -1 x 16), G 128 x 64,
    singular values log-uniform on [1e-3, 1e3] (cond(F) = cond(G) = 1e6)."""
    return svd_pencil(seed, 96, 128, 64, 16, (1e-3, 1e3), (1e-3, 1e3))


def lapw_pencil(n: int = 2048, seed: int = SEED_BASE + 2):
    """n x n pencil shaped like an LAPW one: F 1.5n x n with J holding 2560 +1
    and 512 -1 entries at n = 2048 (1/6 negative), G 2n x n.  Singular values
    log-uniform: F on [1e-3, 1e3], G on [10^-2.5, 10^2.5] (cond(S) = 1e10)."""
    m, p = (3 * n) // 2, 2 * n
    return svd_pencil(seed, m, p, n, m // 6, (1e-3, 1e3), (10 ** -2.5, 10 ** 2.5))


def batch_shapes(count: int = 64, lo: int = 256, hi: int = 1536, seed: int = SEED_BASE + 4):
    """Orders n uniform in [lo, hi] and cond(S) log-uniform in [1e4, 1e10]."""
    rng = rng_for(seed)
    ns = rng.integers(lo, hi + 1, size=count)
    conds = 10.0 ** rng.uniform(4, 10, size=count)
    return [(int(n), float(c)) for n, c in zip(ns, conds)]


def batch_pencil(n: int, cond_s: float, seed: int):
    """One k-point pencil: F 1.5n x n with round(0.2 m) -1 signs, G 2n x n with
    log-uniform singular values giving cond(G^* G) = cond_s."""
    m, p = (3 * n) // 2, 2 * n
    g = np.sqrt(np.sqrt(cond_s))
    return svd_pencil(seed, m, p, n, int(round(0.2 * m)), (1e-3, 1e3), (1.0 / g, g))


def pencil_family(n: int = 256, seed: int = SEED_BASE + 5, eps: float = 0.05, k: int = 4,
                  sf=(1e-3, 1e3), sg=(10 ** -2.5, 10 ** 2.5)):
    """An affine family F(t) = F0 + sum_i t_i F_i, G(t) = G0 + sum_i t_i G_i.

    (F0, J, G0) is LAPW-shaped (F 1.5n x n with 1/6 negative signs, G 2n x n)
    with singular values log-uniform on sf and sg (default: those of the
    n = 2048 benchmark pencil, cond(S) = 1e10).  The k perturbations are
    relative, of size eps:
    F_i = eps F0 E_i and G_i = eps G0 E'_i with E_i, E'_i complex Gaussian
    n x n matrices scaled by 1/sqrt(2n) (spectral norm about sqrt(2)).
    Returns (F0, J, G0, [F_i], [G_i])."""
    m, p = (3 * n) // 2, 2 * n
    F0, J, G0 = svd_pencil(seed, m, p, n, m // 6, sf, sg)
    rng = rng_for(seed + 1)
    Fs, Gs = [], []
    for _ in range(k):
        E = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0 * n)
        Fs.append(np.asfortranarray(eps * (F0 @ E)))
        E = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0 * n)
        Gs.append(np.asfortranarray(eps * (G0 @ E)))
    return F0, J, G0, Fs, Gs


def family_parameters(count: int, k: int = 4, seed: int = SEED_BASE + 6) -> np.ndarray:
    """count parameter vectors t uniform in [-1, 1]^k."""
    return rng_for(seed).uniform(-1.0, 1.0, size=(count, k))
