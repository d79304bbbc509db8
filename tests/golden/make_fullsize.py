"""Writes tests/golden/fullsize_oracle.json: the FP64 oracle's generalized
eigenvalues of the full-size seeded pencils, for the GPU parity tests at the
benchmark's own sizes.

Cases:
  lapw2048   the n = 2048 LAPW-shaped pencil (F 3072 x 2048 with 512 negative
             signs, G 4096 x 2048, cond(S) = 1e10; synth.pencils.lapw_pencil)
  kpt56, kpt11, kpt23
             three of the 64 k-point pencils (n uniform in [256, 1536],
             F 1.5n x n with round(0.2 m) negative signs, G 2n x n, cond(S)
             log-uniform in [1e4, 1e10]; synth.pencils.batch_shapes /
             batch_pencil with the seeds the batched benchmark uses): the
             largest odd one (n = 1511, cond(S) 4.6e9), an odd one at
             n = 1147 (cond(S) 6.3e9) and an even one at n = 1272.

Each is solved by the blocked oracle of Section 6.4 (oracle.solve,
method="blocked": block width 32, BO inner level, round-robin orderings,
C_max = 80 since the n = 2048 pencil needs more than the paper's 30 sweeps),
then finalized by Section 6.1.7 (lambda_j = f_j^* J f_j / g_j^* g_j).  Stored
per case: the eigenvalues sorted ascending, the hyperbolic amplification
a_j = ||f_j||^2 / |f_j^* J f_j| of each converged column of F' (same order),
the condition numbers of the column-scaled F and G (numpy SVD, the
definition), the sweep count, the status and the wall time with the thread
count and host that produced it.  Calls only oracle/ (and synth/ for the
inputs); nothing here comes from the CUDA path.

Run from the repository root:
    python tests/golden/make_fullsize.py [--only NAME ...] [--out PATH]
"""
import argparse
import json
import os
import platform
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
from synth import pencils  # noqa: E402

BATCH_SEED0 = pencils.SEED_BASE + 4000   # seed of k-point pencil i is BATCH_SEED0 + i
KPOINTS = (56, 11, 23)


def cases():
    out = [("lapw2048", lambda: pencils.lapw_pencil(2048, pencils.SEED_BASE + 2),
            dict(generator="lapw_pencil", n=2048, seed=pencils.SEED_BASE + 2))]
    shapes = pencils.batch_shapes(64, lo=256, hi=1536)
    for i in KPOINTS:
        n, c = shapes[i]
        out.append((f"kpt{i}", (lambda n=n, c=c, i=i: pencils.batch_pencil(n, c, BATCH_SEED0 + i)),
                    dict(generator="batch_pencil", n=n, cond_s=c, seed=BATCH_SEED0 + i,
                         batch_index=i)))
    return out


def cond_cols(X):
    Xc = X / np.linalg.norm(X, axis=0)[None, :]
    s = np.linalg.svd(Xc, compute_uv=False)
    return float(s[0] / s[-1])


def host():
    model = platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    model += " " + line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return model


def run(name, make, meta, w=32, max_sweeps=80):
    F, J, G = make()
    lib = oracle.load()
    threads = oracle.max_threads(lib=lib)
    t0 = time.perf_counter()
    out = oracle.solve(F, G, J, method="blocked", w=w, max_sweeps=max_sweeps, lib=lib)
    wall = time.perf_counter() - t0
    if out["status"] != 0:
        raise RuntimeError(f"{name}: oracle status {out['status']} after {out['sweeps']} sweeps")
    lam = out["lam"]
    Fp = out["F"]
    Jf = J.astype(np.float64)
    amp = (np.einsum("ij,ij->j", Fp.conj(), Fp).real /
           np.abs(np.einsum("ij,i,ij->j", Fp.conj(), Jf, Fp).real))
    order = np.argsort(lam)
    rec = dict(name=name, **meta, m=int(F.shape[0]), p=int(G.shape[0]), w=w,
               max_sweeps=max_sweeps, sweeps=int(out["sweeps"]), status=int(out["status"]),
               wall_s=round(wall, 2), threads=int(threads), host=host(),
               kappa_est=float(out["kappa_est"]),
               cond_F_c=cond_cols(F), cond_G_c=cond_cols(G),
               lam=[repr(float(x)) for x in lam[order]],
               amp=[repr(float(x)) for x in amp[order]])
    print(f"{name}: n={meta['n']} sweeps={rec['sweeps']} wall={wall:.1f}s threads={threads}",
          flush=True)
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", nargs="*", default=None)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                  "fullsize_oracle.json"))
    args = ap.parse_args()
    recs = {}
    if os.path.exists(args.out):
        with open(args.out) as f:
            recs = {r["name"]: r for r in json.load(f)["cases"]}
    for name, make, meta in cases():
        if args.only is not None and name not in args.only:
            continue
        recs[name] = run(name, make, meta)
        with open(args.out, "w") as f:
            json.dump(dict(source="oracle.solve(method='blocked'), FP64 CPU oracle of "
                                  "arXiv 1907.08560 Section 6.4 / 6.1.7",
                           cases=list(recs.values())), f, indent=0)
    print("wrote", args.out)


if __name__ == "__main__":
    main()
