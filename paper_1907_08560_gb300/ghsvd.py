"""Python binding of the C ABI in include/ghsvd.h (argument marshalling only).

Every step of the solve runs in the CUDA kernels of libghsvd.so; this module
only loads the library, converts torch tensors to pointers and status codes
to exceptions.  There is no CPU fallback: if the library is missing or no
CUDA device is present, the calls raise.

Layout: complex128 matrices are column-major.  A torch tensor ``X`` of shape
(rows, cols) is column-major when ``X.stride() == (1, ld)``; ``colmajor``
makes such a copy, ``ld_of`` reads the leading dimension.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libghsvd.so")

GHSVD_OK = 0
GHSVD_ERR_INVALID_ARG = 1
GHSVD_ERR_RANK_DEFICIENT = 2
GHSVD_ERR_NONFINITE = 3
GHSVD_ERR_NOT_CONVERGED = 4
GHSVD_ERR_CUDA = 5
GHSVD_ERR_NOMEM = 6
GHSVD_ERR_SCRATCH_TOO_SMALL = 7
GHSVD_ERR_BREAKDOWN = 8
GHSVD_ERR_TIMEOUT = 9
GHSVD_ORDER_ROUND_ROBIN = 0

GHSVD_PRECISION_FP64 = 0
GHSVD_PRECISION_MIXED = 1


class ghsvd_opts(ctypes.Structure):
    _fields_ = [("block_width", ctypes.c_int), ("inner_sweeps", ctypes.c_int),
                ("max_sweeps", ctypes.c_int), ("crit_mode", ctypes.c_int),
                ("precision", ctypes.c_int), ("mixed_max_sweeps", ctypes.c_int),
                ("sort_ascending", ctypes.c_int), ("gram_chunk", ctypes.c_int),
                ("timing", ctypes.c_int), ("ordering", ctypes.c_int),
                ("tol_scale", ctypes.c_double), ("timeout_ms", ctypes.c_int64),
                ("mixed_param32", ctypes.c_int), ("shorten", ctypes.c_int),
                ("mixed_tc", ctypes.c_int), ("delta_update", ctypes.c_int)]


class ghsvd_stats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("sweeps_low", ctypes.c_int),
                ("steps_per_sweep", ctypes.c_int), ("pairs_per_step", ctypes.c_int),
                ("block_width", ctypes.c_int),
                ("transforms", ctypes.c_longlong * 64), ("big", ctypes.c_longlong * 64),
                ("ms_total", ctypes.c_double), ("kernel_launches", ctypes.c_longlong),
                ("launches_gram", ctypes.c_longlong), ("launches_inner", ctypes.c_longlong),
                ("launches_update", ctypes.c_longlong), ("ms_gram", ctypes.c_double),
                ("ms_inner", ctypes.c_double), ("ms_update", ctypes.c_double),
                ("rounds_low", ctypes.c_int), ("ms_phase2", ctypes.c_double),
                ("n2x2", ctypes.c_int), ("sweeps_tc", ctypes.c_int),
                ("batch_ticks", ctypes.c_longlong), ("batch_graph_launches", ctypes.c_int),
                ("ms_v0", ctypes.c_double), ("pairs_delta", ctypes.c_longlong),
                ("pairs_fp64", ctypes.c_longlong),
                ("pairs_df", ctypes.c_longlong)]


class GhsvdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None


def load(path: str | None = None):
    """Load libghsvd.so (it must have been built; see build.py)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libghsvd.so not built: {p} (run __graft_entry__.build())")
    lib = ctypes.CDLL(p)
    vp, i64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.ghsvd_default_opts.restype = c_int
    lib.ghsvd_default_opts.argtypes = [ctypes.POINTER(ghsvd_opts)]
    lib.ghsvd_create.restype = c_int
    lib.ghsvd_create.argtypes = [ctypes.POINTER(vp), c_int, ctypes.POINTER(ghsvd_opts)]
    lib.ghsvd_destroy.restype = None
    lib.ghsvd_destroy.argtypes = [vp]
    lib.ghsvd_solve.restype = c_int
    lib.ghsvd_solve.argtypes = [vp, i64, i64, i64, vp, i64, vp, i64, vp, i64, vp, vp, i64,
                                ctypes.POINTER(c_int), vp]
    lib.ghsvd_solve_from.restype = c_int
    lib.ghsvd_solve_from.argtypes = [vp, i64, i64, i64, vp, i64, vp, i64, vp, i64, vp, i64, vp,
                                     vp, i64, ctypes.POINTER(c_int), vp]
    lib.ghsvd_solve_host.restype = c_int
    lib.ghsvd_solve_host.argtypes = [vp, i64, i64, i64, vp, i64, vp, i64, vp, i64, vp, vp, i64,
                                     ctypes.POINTER(c_int), vp]
    lib.ghsvd_get_factors.restype = c_int
    lib.ghsvd_get_factors.argtypes = [vp, vp, i64, vp, i64, vp, i64, vp]
    lib.ghsvd_get_stats.restype = c_int
    lib.ghsvd_get_stats.argtypes = [vp, ctypes.POINTER(ghsvd_stats)]
    lib.ghsvd_tc_block_ops.restype = c_int
    lib.ghsvd_tc_block_ops.argtypes = [i64, vp, i64, vp, vp, vp, vp]
    lib.ghsvd_fp64_block_update.restype = c_int
    lib.ghsvd_fp64_block_update.argtypes = [i64, vp, i64, vp, c_int, vp]
    lib.ghsvd_solve_noalloc.restype = c_int
    lib.ghsvd_solve_noalloc.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64, vp, vp, i64,
                                        ctypes.POINTER(ghsvd_opts), ctypes.POINTER(c_int), vp]
    P64 = ctypes.POINTER(ctypes.c_int64)
    lib.ghsvd_solve_batched.restype = c_int
    lib.ghsvd_solve_batched.argtypes = [vp, c_int, P64, P64, P64, ctypes.POINTER(vp), P64,
                                        ctypes.POINTER(vp), P64, ctypes.POINTER(vp), P64,
                                        ctypes.POINTER(vp), P64,
                                        ctypes.POINTER(vp), ctypes.POINTER(vp), P64,
                                        ctypes.POINTER(c_int), ctypes.POINTER(c_int), vp]
    FP = ctypes.POINTER(ctypes.c_float)
    lib.ghsvd_mlp_create.restype = c_int
    lib.ghsvd_mlp_create.argtypes = [ctypes.POINTER(vp), c_int, c_int, c_int, c_int, ctypes.c_uint64]
    lib.ghsvd_mlp_destroy.restype = None
    lib.ghsvd_mlp_destroy.argtypes = [vp]
    lib.ghsvd_mlp_size.restype = c_int
    lib.ghsvd_mlp_size.argtypes = [vp, P64]
    lib.ghsvd_mlp_get.restype = c_int
    lib.ghsvd_mlp_get.argtypes = [vp, c_int, vp]
    lib.ghsvd_mlp_set.restype = c_int
    lib.ghsvd_mlp_set.argtypes = [vp, vp]
    lib.ghsvd_mlp_forward.restype = c_int
    lib.ghsvd_mlp_forward.argtypes = [vp, c_int, vp, vp, vp]
    lib.ghsvd_mlp_loss_grad.restype = c_int
    lib.ghsvd_mlp_loss_grad.argtypes = [vp, c_int, vp, vp, ctypes.POINTER(ctypes.c_double), vp]
    lib.ghsvd_mlp_train.restype = c_int
    lib.ghsvd_mlp_train.argtypes = [vp, c_int, vp, vp, c_int, c_int, ctypes.c_float,
                                    ctypes.POINTER(ctypes.c_double), vp]
    lib.ghsvd_s_orthonormalize.restype = c_int
    lib.ghsvd_s_orthonormalize.argtypes = [c_int, i64, i64, ctypes.POINTER(vp), P64,
                                           ctypes.POINTER(vp), P64, vp]
    lib.ghsvd_align_phases.restype = c_int
    lib.ghsvd_align_phases.argtypes = [i64, vp, i64, vp, i64, vp]
    lib.ghsvd_v0_targets.restype = c_int
    lib.ghsvd_v0_targets.argtypes = [c_int, i64, vp, i64, ctypes.POINTER(vp), P64, vp,
                                     ctypes.POINTER(ctypes.c_double), vp]
    lib.ghsvd_v0_compose.restype = c_int
    lib.ghsvd_v0_compose.argtypes = [c_int, i64, vp, ctypes.c_double, vp, i64, ctypes.POINTER(vp), P64, vp]
    lib.ghsvd_status_string.restype = ctypes.c_char_p
    lib.ghsvd_status_string.argtypes = [c_int]
    lib.ghsvd_urv.restype = c_int
    lib.ghsvd_urv.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64, vp, i64, vp, vp, i64, vp,
                              ctypes.POINTER(c_int), vp]
    lib.ghsvd_inverse.restype = c_int
    lib.ghsvd_inverse.argtypes = [i64, vp, i64, vp, i64, vp]
    lib.ghsvd_phase4.restype = c_int
    lib.ghsvd_phase4.argtypes = [vp, vp, vp, vp, i64, vp]
    lib.ghsvd_decomposition_errors.restype = c_int
    lib.ghsvd_decomposition_errors.argtypes = [vp, vp, i64, vp, i64, vp, i64,
                                               ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_double), vp]
    if path is None:
        _lib = lib
    return lib


def status_string(s: int) -> str:
    return load().ghsvd_status_string(s).decode()


def _check(s: int, allow=(GHSVD_OK,)):
    if s not in allow:
        raise GhsvdError(s, status_string(s))
    return s


def ghsvd_default_opts(**kw) -> ghsvd_opts:
    o = ghsvd_opts()
    _check(load().ghsvd_default_opts(ctypes.byref(o)))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, float(v) if k == "tol_scale" else int(v))
    return o


def ghsvd_create(device: int = 0, opts: ghsvd_opts | None = None):
    h = ctypes.c_void_p()
    _check(load().ghsvd_create(ctypes.byref(h), device, ctypes.byref(opts) if opts else None))
    return h


def ghsvd_destroy(h) -> None:
    if h:
        load().ghsvd_destroy(h)


# --------------------------------------------------------------------------
# torch marshalling
# --------------------------------------------------------------------------

def colmajor(X):
    """Column-major (Fortran-order) complex128 copy of a 2-D tensor or array."""
    import torch
    X = torch.as_tensor(X)
    return X.to(torch.complex128).t().contiguous().t()


def ld_of(X) -> int:
    if X.dim() != 2 or X.stride(0) != 1:
        raise ValueError("expected a column-major 2-D tensor (stride (1, ld))")
    return max(X.stride(1), X.shape[0], 1)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def ghsvd_solve(h, F, J, G, n_plus: int | None = None, want_vectors: bool = True, V0=None, stream=None,
                allow_not_converged: bool = True):
    """Solve H z = lambda S z, H = F^* J F, S = G^* G, on device tensors.

    F (m x n), G (p x n): column-major complex128 CUDA tensors.  J: int8
    tensor of m entries +-1 (device or CPU), or None with ``n_plus`` leading
    +1 signs (None: all +1, J = I, the GSVD).
    Returns (lambda, V or None, sweeps, status).
    """
    import torch
    m, n = F.shape
    if n_plus is None:
        n_plus = m
    p = G.shape[0]
    dev = F.device
    lam = torch.empty(n, dtype=torch.float64, device=dev)
    V = None
    if want_vectors:
        V = torch.empty_strided((n, n), (1, n), dtype=torch.complex128, device=dev)
    Jp = None
    if J is not None:
        if J.dtype != torch.int8:
            raise TypeError("J must be int8")
        J = J.contiguous()          # keep the (possibly copied) tensor alive
        Jp = ctypes.c_void_p(J.data_ptr())
    sweeps = ctypes.c_int(0)
    lib = load()
    if V0 is None:
        s = lib.ghsvd_solve(h, m, p, n, F.data_ptr(), ld_of(F), Jp, n_plus, G.data_ptr(), ld_of(G),
                            lam.data_ptr(), V.data_ptr() if V is not None else None,
                            n, ctypes.byref(sweeps), _stream_ptr(stream))
    else:
        s = lib.ghsvd_solve_from(h, m, p, n, F.data_ptr(), ld_of(F), Jp, n_plus, G.data_ptr(),
                                 ld_of(G), V0.data_ptr(), ld_of(V0), lam.data_ptr(),
                                 V.data_ptr() if V is not None else None, n,
                                 ctypes.byref(sweeps), _stream_ptr(stream))
    _check(s, (GHSVD_OK, GHSVD_ERR_NOT_CONVERGED, GHSVD_ERR_TIMEOUT) if allow_not_converged
           else (GHSVD_OK,))
    return lam, V, sweeps.value, s


def ghsvd_solve_from(h, F, J, G, V0, **kw):
    return ghsvd_solve(h, F, J, G, V0=V0, **kw)


def ghsvd_solve_host(h, F, J, G, n_plus: int | None = None, want_vectors: bool = True,
                     allow_not_converged: bool = True):
    """Host-memory variant: numpy column-major complex128 F, G; int8 J or None."""
    import numpy as np
    F = np.asfortranarray(F, dtype=np.complex128)
    G = np.asfortranarray(G, dtype=np.complex128)
    m, n = F.shape
    if n_plus is None:
        n_plus = m
    p = G.shape[0]
    lam = np.empty(n, dtype=np.float64)
    V = np.empty((n, n), dtype=np.complex128, order="F") if want_vectors else None
    Jp = None
    if J is not None:
        J = np.ascontiguousarray(J, dtype=np.int8)
        Jp = J.ctypes.data_as(ctypes.c_void_p)
    sweeps = ctypes.c_int(0)
    s = load().ghsvd_solve_host(h, m, p, n, F.ctypes.data_as(ctypes.c_void_p), m, Jp, n_plus,
                                G.ctypes.data_as(ctypes.c_void_p), p,
                                lam.ctypes.data_as(ctypes.c_void_p),
                                V.ctypes.data_as(ctypes.c_void_p) if V is not None else None, n,
                                ctypes.byref(sweeps), None)
    _check(s, (GHSVD_OK, GHSVD_ERR_NOT_CONVERGED) if allow_not_converged else (GHSVD_OK,))
    return lam, V, sweeps.value, s


def ghsvd_solve_noalloc(F, J, G, n_plus: int | None = None, opts: ghsvd_opts | None = None,
                        want_vectors: bool = True, stream=None, allow_not_converged: bool = True):
    """The FP64 solve without device allocation inside the library (all of its
    working memory is a fixed device array; see include/ghsvd.h).  Device
    tensors as for ghsvd_solve; J, if given, must be a device tensor.  The
    output tensors are allocated here by the caller's side (torch)."""
    import torch
    m, n = F.shape
    if n_plus is None:
        n_plus = m
    p = G.shape[0]
    lam = torch.empty(n, dtype=torch.float64, device=F.device)
    V = torch.empty_strided((n, n), (1, n), dtype=torch.complex128, device=F.device) \
        if want_vectors else None
    Jp = None
    if J is not None:
        J = J.contiguous()
        Jp = ctypes.c_void_p(J.data_ptr())
    sweeps = ctypes.c_int(0)
    s = load().ghsvd_solve_noalloc(m, p, n, F.data_ptr(), ld_of(F), Jp, n_plus, G.data_ptr(),
                                   ld_of(G), lam.data_ptr(), V.data_ptr() if V is not None else None,
                                   n, ctypes.byref(opts) if opts is not None else None,
                                   ctypes.byref(sweeps), _stream_ptr(stream))
    _check(s, (GHSVD_OK, GHSVD_ERR_NOT_CONVERGED) if allow_not_converged else (GHSVD_OK,))
    return lam, V, sweeps.value, s


def ghsvd_solve_batched(h, Fs, Js, Gs, n_plus=None, want_vectors: bool = True, stream=None,
                        V0s=None, sort_outputs=None):
    """Batched solve of independent pencils (lists of column-major complex128
    CUDA tensors; Js: list of int8 CUDA tensors or None).  Returns
    (lambdas, Vs, sweeps, statuses, status)."""
    import torch
    b = len(Fs)
    arr = lambda t, vals: (t * b)(*vals)
    I64 = ctypes.c_int64
    m = arr(I64, [F.shape[0] for F in Fs])
    n = arr(I64, [F.shape[1] for F in Fs])
    p = arr(I64, [G.shape[0] for G in Gs])
    ldf = arr(I64, [ld_of(F) for F in Fs])
    ldg = arr(I64, [ld_of(G) for G in Gs])
    VP = ctypes.c_void_p
    Fp = arr(VP, [F.data_ptr() for F in Fs])
    Gp = arr(VP, [G.data_ptr() for G in Gs])
    Jkeep = [J.contiguous() if J is not None else None for J in (Js or [None] * b)]
    Jp = arr(VP, [J.data_ptr() if J is not None else None for J in Jkeep])
    npl = arr(I64, list(n_plus)) if n_plus is not None else None
    lams = [torch.empty(F.shape[1], dtype=torch.float64, device=F.device) for F in Fs]
    lp = arr(VP, [l.data_ptr() for l in lams])
    Vs, Vp, ldv = None, None, None
    if want_vectors:
        Vs = [torch.empty_strided((F.shape[1], F.shape[1]), (1, F.shape[1]), dtype=torch.complex128,
                                  device=F.device) for F in Fs]
        Vp = arr(VP, [V.data_ptr() for V in Vs])
        ldv = arr(I64, [F.shape[1] for F in Fs])
    V0p, ldv0 = None, None
    if V0s is not None:
        V0p = arr(VP, [V.data_ptr() if V is not None else None for V in V0s])
        ldv0 = arr(I64, [ld_of(V) if V is not None else 1 for V in V0s])
    sw = (ctypes.c_int * b)()
    stt = (ctypes.c_int * b)()
    s = load().ghsvd_solve_batched(h, b, m, p, n, Fp, ldf, Jp if Js is not None else None, npl, Gp,
                                   ldg, V0p, ldv0, lp, Vp, ldv, sw, stt, _stream_ptr(stream))
    # per-pencil failures are reported in the statuses; raise only for the
    # errors that concern the whole call
    if s in (GHSVD_ERR_INVALID_ARG, GHSVD_ERR_CUDA, GHSVD_ERR_NOMEM):
        _check(s)
    return lams, Vs, list(sw), list(stt), s


def ghsvd_mlp_create(n_in, n_hidden, n_out, seed=0, device=0):
    h = ctypes.c_void_p()
    _check(load().ghsvd_mlp_create(ctypes.byref(h), device, n_in, n_hidden, n_out, seed))
    return h


def ghsvd_mlp_destroy(h):
    if h:
        load().ghsvd_mlp_destroy(h)


def ghsvd_mlp_size(h):
    n = ctypes.c_int64()
    _check(load().ghsvd_mlp_size(h, ctypes.byref(n)))
    return n.value


def ghsvd_mlp_get(h, what, dst):
    _check(load().ghsvd_mlp_get(h, what, dst.data_ptr()))
    return dst


def ghsvd_mlp_set(h, src):
    _check(load().ghsvd_mlp_set(h, src.data_ptr()))


def ghsvd_mlp_forward(h, X, Y):
    _check(load().ghsvd_mlp_forward(h, X.shape[0], X.data_ptr(), Y.data_ptr(), None))
    return Y


def ghsvd_mlp_loss_grad(h, X, T):
    loss = ctypes.c_double(0.0)
    _check(load().ghsvd_mlp_loss_grad(h, X.shape[0], X.data_ptr(), T.data_ptr(), ctypes.byref(loss),
                                      None))
    return loss.value


def ghsvd_mlp_train(h, X, T, epochs, batch, lr):
    loss = ctypes.c_double(0.0)
    _check(load().ghsvd_mlp_train(h, X.shape[0], X.data_ptr(), T.data_ptr(), epochs, batch, lr,
                                  ctypes.byref(loss), None))
    return loss.value


class Mlp:
    """The warm-start MLP of libghsvd (FP32, tanh, two hidden layers)."""

    def __init__(self, n_in, n_hidden, n_out, seed=0, device=0):
        self.h = ctypes.c_void_p()
        _check(load().ghsvd_mlp_create(ctypes.byref(self.h), device, n_in, n_hidden, n_out, seed))
        self.n_in, self.n_hidden, self.n_out = n_in, n_hidden, n_out

    def size(self):
        n = ctypes.c_int64()
        _check(load().ghsvd_mlp_size(self.h, ctypes.byref(n)))
        return n.value

    def get_params(self):
        """Copy of the flat parameter vector (torch float32 on the device)."""
        import torch
        out = torch.empty(self.size(), dtype=torch.float32, device="cuda")
        _check(load().ghsvd_mlp_get(self.h, 0, out.data_ptr()))
        return out

    def set_params(self, vec):
        import torch
        vec = vec.to(torch.float32).contiguous().cuda()
        if vec.numel() != self.size():
            raise ValueError("parameter vector of the wrong length")
        _check(load().ghsvd_mlp_set(self.h, vec.data_ptr()))

    def get_grads(self):
        import torch
        out = torch.empty(self.size(), dtype=torch.float32, device="cuda")
        _check(load().ghsvd_mlp_get(self.h, 1, out.data_ptr()))
        return out

    def forward(self, X):
        import torch
        X = X.to(torch.float32).contiguous()
        Y = torch.empty((X.shape[0], self.n_out), dtype=torch.float32, device=X.device)
        _check(load().ghsvd_mlp_forward(self.h, X.shape[0], X.data_ptr(), Y.data_ptr(), None))
        return Y

    def loss_grad(self, X, T):
        import torch
        X = X.to(torch.float32).contiguous()
        T = T.to(torch.float32).contiguous()
        loss = ctypes.c_double(0.0)
        _check(load().ghsvd_mlp_loss_grad(self.h, X.shape[0], X.data_ptr(), T.data_ptr(),
                                          ctypes.byref(loss), None))
        return loss.value, self.get_grads()

    def train(self, X, T, epochs, batch, lr):
        import torch
        X = X.to(torch.float32).contiguous()
        T = T.to(torch.float32).contiguous()
        loss = ctypes.c_double(0.0)
        _check(load().ghsvd_mlp_train(self.h, X.shape[0], X.data_ptr(), T.data_ptr(), epochs,
                                      batch, lr, ctypes.byref(loss), None))
        return loss.value

    def close(self):
        if self.h:
            load().ghsvd_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ghsvd_s_orthonormalize(Gs, V0s, stream=None):
    """In place for every pair: V0 <- V0 R^{-1}, (G V0)^* (G V0) = R^* R.
    Gs, V0s: lists of column-major complex128 CUDA tensors (or single ones)."""
    if not isinstance(Gs, (list, tuple)):
        Gs, V0s = [Gs], [V0s]
    b = len(Gs)
    VP, I64 = ctypes.c_void_p, ctypes.c_int64
    gp = (VP * b)(*[G.data_ptr() for G in Gs])
    vp = (VP * b)(*[V.data_ptr() for V in V0s])
    lg = (I64 * b)(*[ld_of(G) for G in Gs])
    lv = (I64 * b)(*[ld_of(V) for V in V0s])
    _check(load().ghsvd_s_orthonormalize(b, Gs[0].shape[0], Gs[0].shape[1], gp, lg, vp, lv,
                                         _stream_ptr(stream)))
    return V0s


def ghsvd_tc_block_ops(X, J, Z, stream=None):
    """The tensor-core Gram and update of the complex64 sweeps on one block
    pair (include/ghsvd.h): X (rows x 64 complex64 column-major CUDA tensor,
    rows a multiple of 64) is overwritten by X Z; returns gram = X^* J X
    (64 x 64 complex64, J an int8 CUDA tensor or None)."""
    import torch
    if X.dtype != torch.complex64 or Z.dtype != torch.complex64:
        raise TypeError("ghsvd_tc_block_ops works on complex64 tensors")
    rows = X.shape[0]
    gram = torch.empty_strided((64, 64), (1, 64), dtype=torch.complex64, device=X.device)
    Jp = None if J is None else ctypes.c_void_p(J.contiguous().data_ptr())
    _check(load().ghsvd_tc_block_ops(rows, X.data_ptr(), ld_of(X), Jp, Z.data_ptr(), gram.data_ptr(),
                                      _stream_ptr(stream)))
    return gram


FP64_ROUTE_DELTA32, FP64_ROUTE_DOUBLE_FLOAT, FP64_ROUTE_FP64 = 0, 1, 2


def ghsvd_fp64_block_update(X, Z, route, stream=None):
    """The FP64 sweeps' block update of one pair by the given route
    (include/ghsvd.h): X (rows x 64 complex128 column-major CUDA tensor, rows
    a multiple of 64) is overwritten by X Z (route 2) or X + X (Z - I)
    (route 0: FP32 product, route 1: double-float product)."""
    import torch
    if X.dtype != torch.complex128 or Z.dtype != torch.complex128:
        raise TypeError("ghsvd_fp64_block_update works on complex128 tensors")
    _check(load().ghsvd_fp64_block_update(X.shape[0], X.data_ptr(), ld_of(X), Z.data_ptr(), int(route),
                                           _stream_ptr(stream)))


def ghsvd_v0_targets(Vref, Vs, stream=None):
    """Training targets (count x 2 n^2 FP32 CUDA tensor, normalized) and
    their scale (the RMS) from aligned eigenvector sets Vs (include/ghsvd.h)."""
    import torch
    n = Vref.shape[0]
    b = len(Vs)
    T = torch.empty((b, 2 * n * n), dtype=torch.float32, device=Vref.device)
    ptrs = (ctypes.c_void_p * b)(*[V.data_ptr() for V in Vs])
    lds = (ctypes.c_int64 * b)(*[ld_of(V) for V in Vs])
    rms = ctypes.c_double(0.0)
    _check(load().ghsvd_v0_targets(b, n, Vref.data_ptr(), ld_of(Vref), ptrs, lds, T.data_ptr(),
                                    ctypes.byref(rms), _stream_ptr(stream)))
    return T, rms.value


def ghsvd_v0_compose(Y, scale, Vref, stream=None):
    """V0_i = Vref + scale * D_i from the MLP output rows Y (count x 2 n^2
    FP32); returns the list of column-major complex128 CUDA tensors."""
    import torch
    n = Vref.shape[0]
    b = Y.shape[0]
    V0s = [torch.empty_strided((n, n), (1, n), dtype=torch.complex128, device=Vref.device)
           for _ in range(b)]
    ptrs = (ctypes.c_void_p * b)(*[V.data_ptr() for V in V0s])
    lds = (ctypes.c_int64 * b)(*([n] * b))
    _check(load().ghsvd_v0_compose(b, n, Y.contiguous().data_ptr(), float(scale), Vref.data_ptr(),
                                    ld_of(Vref), ptrs, lds, _stream_ptr(stream)))
    return V0s


def ghsvd_align_phases(Vref, V, stream=None):
    """In place: align the phase of each column of V to the same column of Vref."""
    _check(load().ghsvd_align_phases(V.shape[1], Vref.data_ptr(), ld_of(Vref), V.data_ptr(),
                                     ld_of(V), _stream_ptr(stream)))
    return V


def ghsvd_get_factors(h, m: int, p: int, n: int, device="cuda", stream=None):
    """The transformed F' (m x n), G' (p x n) and Z' (n x n) of the last solve."""
    import torch
    Fp = torch.empty_strided((m, n), (1, m), dtype=torch.complex128, device=device)
    Gp = torch.empty_strided((p, n), (1, p), dtype=torch.complex128, device=device)
    Zp = torch.empty_strided((n, n), (1, n), dtype=torch.complex128, device=device)
    _check(load().ghsvd_get_factors(h, Fp.data_ptr(), m, Gp.data_ptr(), p, Zp.data_ptr(), n,
                                    _stream_ptr(stream)))
    return Fp, Gp, Zp


def ghsvd_get_stats(h) -> dict:
    st = ghsvd_stats()
    _check(load().ghsvd_get_stats(h, ctypes.byref(st)))
    k = min(st.sweeps, 64)
    return dict(sweeps=st.sweeps, sweeps_low=st.sweeps_low, steps_per_sweep=st.steps_per_sweep,
                pairs_per_step=st.pairs_per_step, block_width=st.block_width,
                transforms=list(st.transforms[:k]), big=list(st.big[:k]), ms_total=st.ms_total,
                kernel_launches=st.kernel_launches, launches_gram=st.launches_gram,
                launches_inner=st.launches_inner, launches_update=st.launches_update,
                ms_gram=st.ms_gram, ms_inner=st.ms_inner, ms_update=st.ms_update,
                rounds_low=st.rounds_low, ms_phase2=st.ms_phase2, n2x2=st.n2x2,
                sweeps_tc=st.sweeps_tc, batch_ticks=st.batch_ticks,
                batch_graph_launches=st.batch_graph_launches, ms_v0=st.ms_v0,
                pairs_delta=st.pairs_delta, pairs_fp64=st.pairs_fp64, pairs_df=st.pairs_df)


def ghsvd_urv(F, J, G, n_plus: int | None = None, stream=None):
    """Phase 2 (Section 5): the square (Fs, Js, Gs) of a tall (F, J, G) on the device.

    Returns (Fs, Js, Gs, perm, n2x2): Fs, Gs n x n column-major complex128,
    Js int8 (n), perm int64 (n) with F[:, perm] = F P2."""
    import torch
    m, n = F.shape
    p = G.shape[0]
    if n_plus is None:
        n_plus = m
    dev = F.device
    Fs = torch.empty_strided((n, n), (1, n), dtype=torch.complex128, device=dev)
    Gs = torch.empty_strided((n, n), (1, n), dtype=torch.complex128, device=dev)
    Js = torch.empty(n, dtype=torch.int8, device=dev)
    perm = torch.empty(n, dtype=torch.int64, device=dev)
    Jp = None
    if J is not None:
        if J.dtype != torch.int8 or not J.is_cuda:
            raise TypeError("J must be an int8 CUDA tensor")
        J = J.contiguous()
        Jp = ctypes.c_void_p(J.data_ptr())
    n2 = ctypes.c_int(0)
    _check(load().ghsvd_urv(m, p, n, F.data_ptr(), ld_of(F), Jp, n_plus, G.data_ptr(), ld_of(G),
                            Fs.data_ptr(), n, Js.data_ptr(), Gs.data_ptr(), n, perm.data_ptr(),
                            ctypes.byref(n2), _stream_ptr(stream)))
    return Fs, Js, Gs, perm, n2.value


def ghsvd_inverse(Z, stream=None):
    """Phase 4 (Section 7): X = Z^{-1} by complete pivoting, on the device."""
    import torch
    n = Z.shape[0]
    X = torch.empty_strided((n, n), (1, n), dtype=torch.complex128, device=Z.device)
    _check(load().ghsvd_inverse(n, Z.data_ptr(), ld_of(Z), X.data_ptr(), n, _stream_ptr(stream)))
    return X


def ghsvd_phase4(h, n: int, device="cuda", stream=None):
    """(Sigma_F, Sigma_G, X) of the full GHSVD of the last solve on h (eq. 3.1)."""
    import torch
    sf = torch.empty(n, dtype=torch.float64, device=device)
    sg = torch.empty(n, dtype=torch.float64, device=device)
    X = torch.empty_strided((n, n), (1, n), dtype=torch.complex128, device=device)
    _check(load().ghsvd_phase4(h, sf.data_ptr(), sg.data_ptr(), X.data_ptr(), n, _stream_ptr(stream)))
    return sf, sg, X


def ghsvd_decomposition_errors(h, F, G, X, stream=None):
    """The relative errors of eq. 7.1 for the last solve on h: (err_F, err_G)."""
    ef = ctypes.c_double(0.0)
    eg = ctypes.c_double(0.0)
    _check(load().ghsvd_decomposition_errors(h, F.data_ptr(), ld_of(F), G.data_ptr(), ld_of(G),
                                             X.data_ptr(), ld_of(X), ctypes.byref(ef),
                                             ctypes.byref(eg), _stream_ptr(stream)))
    return ef.value, eg.value


class Solver:
    """Owning wrapper of a ghsvd handle."""

    def __init__(self, device: int = 0, **opts):
        self.opts = ghsvd_default_opts(**opts)
        self.h = ghsvd_create(device, self.opts)

    def solve(self, F, G, J=None, n_plus: int | None = None, **kw):
        return ghsvd_solve(self.h, F, J, G, n_plus=n_plus, **kw)

    def solve_host(self, F, G, J=None, n_plus: int | None = None, **kw):
        return ghsvd_solve_host(self.h, F, J, G, n_plus=n_plus, **kw)

    def solve_batched(self, Fs, Gs, Js=None, **kw):
        return ghsvd_solve_batched(self.h, Fs, Js, Gs, **kw)

    def factors(self, m, p, n, **kw):
        return ghsvd_get_factors(self.h, m, p, n, **kw)

    def phase4(self, n, **kw):
        return ghsvd_phase4(self.h, n, **kw)

    def decomposition_errors(self, F, G, X, **kw):
        return ghsvd_decomposition_errors(self.h, F, G, X, **kw)

    def stats(self):
        return ghsvd_get_stats(self.h)

    def close(self):
        if self.h:
            ghsvd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
