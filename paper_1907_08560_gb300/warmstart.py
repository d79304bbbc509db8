"""Learned warm start for a family of pencils F(t), G(t) (parameters t).

The solver's own eigenvectors V(t) (sorted by eigenvalue, column phases
aligned with V(t0) of the family's centre) are the training targets of an MLP
t -> V(t) - V(t0) (the library's FP32 MLP kernels).  For a new t the
predicted V0 = V(t0) + MLP(t) is made S-orthonormal for G(t)
(ghsvd_s_orthonormalize) and the HZ sweeps start from it
(ghsvd_solve_batched with V0, or ghsvd_solve_from); V0 = I stays available
as the cold start.  Every numerical step runs in libghsvd's kernels; this
module only moves tensors between them.
"""
from __future__ import annotations

import numpy as np

from . import ghsvd


class Family:
    """F(t) = F0 + sum t_i F_i, G(t) = G0 + sum t_i G_i, on the device."""

    def __init__(self, F0, J, G0, Fs, Gs, device="cuda"):
        import torch
        self.F0 = ghsvd.colmajor(torch.from_numpy(F0)).to(device)
        self.G0 = ghsvd.colmajor(torch.from_numpy(G0)).to(device)
        self.Fs = [ghsvd.colmajor(torch.from_numpy(F)).to(device) for F in Fs]
        self.Gs = [ghsvd.colmajor(torch.from_numpy(G)).to(device) for G in Gs]
        self.J = torch.from_numpy(np.asarray(J, dtype=np.int8)).to(device)
        self.m, self.n = F0.shape
        self.p = G0.shape[0]

    def at(self, t):
        """Column-major (F(t), G(t)) for one parameter vector t (input synthesis)."""
        F = self.F0.clone()
        G = self.G0.clone()
        for ti, Fi, Gi in zip(t, self.Fs, self.Gs):
            F.add_(Fi, alpha=float(ti))
            G.add_(Gi, alpha=float(ti))
        return F, G


def solve_many(solver, fam, ts, V0s=None, chunk=256, times=None):
    """Batched solves of the family at the parameter vectors ts; returns
    (lambdas, Vs, sweeps, statuses, seconds).  `times` (a dict) receives the
    seconds spent applying the starting bases (ghsvd_stats.ms_v0)."""
    import time

    import torch
    lams, Vs, sweeps, statuses = [], [], [], []
    v0_ms = 0.0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for a in range(0, len(ts), chunk):
        pairs = [fam.at(t) for t in ts[a:a + chunk]]
        V0 = None if V0s is None else V0s[a:a + chunk]
        l, V, sw, st, _ = solver.solve_batched([F for F, _ in pairs], [G for _, G in pairs],
                                               [fam.J] * len(pairs), V0s=V0)
        v0_ms += solver.stats()["ms_v0"] if V0 is not None else 0.0
        lams += l
        Vs += V
        sweeps += sw
        statuses += st
    torch.cuda.synchronize()
    if times is not None:
        times["v0_apply_s"] = times.get("v0_apply_s", 0.0) + v0_ms / 1e3
    return lams, Vs, sweeps, statuses, time.perf_counter() - t0


def canonical_targets(Vs, Vref):
    """Phase-align every V (sorted by eigenvalue) to Vref; return the
    normalized training targets vec(V - Vref) / scale (count x 2 n^2 FP32)
    and the scale (ghsvd_align_phases, ghsvd_v0_targets)."""
    for V in Vs:
        ghsvd.ghsvd_align_phases(Vref, V)
    return ghsvd.ghsvd_v0_targets(Vref, Vs)


def predict_v0(net, fam, Vref, ts, scale, times=None):
    """V0(t) = Vref + scale * MLP(t) (ghsvd_mlp_forward, ghsvd_v0_compose),
    made S-orthonormal for G(t) (ghsvd_s_orthonormalize).  `times` (a dict)
    receives the seconds of the prediction and of the S-orthonormalization."""
    import time

    import torch
    X = torch.as_tensor(np.asarray(ts), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Y = net.forward(X)
    out = ghsvd.ghsvd_v0_compose(Y, scale, Vref)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    Gs = [fam.at(t)[1] for t in ts]                 # input synthesis of G(t)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    ghsvd.ghsvd_s_orthonormalize(Gs, out)
    torch.cuda.synchronize()
    if times is not None:
        times["predict_s"] = times.get("predict_s", 0.0) + (t1 - t0)
        times["s_orthonormalize_s"] = times.get("s_orthonormalize_s", 0.0) + (time.perf_counter() - t2)
    return out


def reference_v0(fam, Vref, ts):
    """The non-learned warm start: V(t0) made S-orthonormal for G(t)."""
    out = [ghsvd.colmajor(Vref.clone()) for _ in ts]
    ghsvd.ghsvd_s_orthonormalize([fam.at(t)[1] for t in ts], out)
    return out
