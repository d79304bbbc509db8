"""Writes tests/golden/tiny_pencils.json: small pencils with integer complex
entries (exact in binary) and their generalized eigenvalues, computed at 60
significant digits by the extended-precision brute force of oracle.brute
(Cholesky of S = G^* G, Hermitian eigenvalues of L^{-1} H L^{-*}; the
definition of eq. 3.2 of arXiv 1907.08560).  Calls nothing but oracle/.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle import brute  # noqa: E402

CASES = [  # (name, m, p, n, number of -1 signs, seed of the integer entries)
    ("n2_hyperbolic", 3, 2, 2, 1, 11),
    ("n3_odd_bordered", 4, 3, 3, 1, 12),
    ("n4_two_negative", 5, 6, 4, 2, 13),
    ("n5_gsvd_J_identity", 6, 7, 5, 0, 14),
    ("n6_tall", 9, 8, 6, 3, 15),
]


def integer_matrix(rng, r, c):
    return rng.integers(-3, 4, size=(r, c)) + 1j * rng.integers(-3, 4, size=(r, c))


def main():
    out = []
    for name, m, p, n, mneg, seed in CASES:
        rng = np.random.default_rng(seed)
        while True:
            F = integer_matrix(rng, m, n)
            G = integer_matrix(rng, p, n)
            if np.linalg.matrix_rank(G) == n and np.linalg.matrix_rank(F) == n:
                break
        J = np.ones(m, dtype=int)
        if mneg:
            J[rng.choice(m, size=mneg, replace=False)] = -1
        lam = brute.generalized_eigenvalues(F, G, J, dps=60)
        out.append(dict(name=name, m=m, p=p, n=n,
                        F_re=F.real.astype(int).tolist(), F_im=F.imag.astype(int).tolist(),
                        G_re=G.real.astype(int).tolist(), G_im=G.imag.astype(int).tolist(),
                        J=J.tolist(), lam=[repr(float(x)) for x in lam]))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_pencils.json")
    with open(path, "w") as f:
        json.dump(dict(source="oracle.brute at 60 digits; eq. 3.2 of arXiv 1907.08560",
                       cases=out), f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
