"""ctypes binding of the tps C ABI (include/tps.h): argument marshalling only.

Every computation runs inside libtps.so (hand-written CUDA for sm_103a).  PyTorch
supplies device memory (tensors' ``data_ptr()``) and streams; nothing else.
Importing this module raises if the compiled library is missing: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtps.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"tps CUDA library not found at {LIB_PATH}; build it with "
        "`python -m paper_2111_02534_gb300.build` (nvcc, sm_103a)")
_lib = C.CDLL(LIB_PATH)

OK = 0
ERR_INVALID_ARG = -1
ERR_NOT_CONFIGURED = -2
ERR_CUDA = -3
ERR_NOMEM = -4
ERR_SINGULAR = -5
ERR_NOT_CONVERGED = -6
ERR_TIMEOUT = -7
GAUSS, LORENTZ3 = 0, 1
ANY, X_EVEN, X_ODD = 0, 1, 2
F64 = 0
F32 = 1
F64_TC = 2
TF32_TC = 3     # preconditioner on the tensor cores in TF32 (1D)
RR_MIXED, RR_JACOBI64 = 0, 1   # Rayleigh-Ritz eigensolver (solver option rr_method)


class SolverOpts(C.Structure):
    _fields_ = [("m_min", C.c_int), ("m_max", C.c_int), ("inner_steps", C.c_int),
                ("max_outer", C.c_int), ("use_prec", C.c_int), ("prec_shift", C.c_double),
                ("seed", C.c_ulonglong), ("inner_tol", C.c_double), ("timing", C.c_int),
                ("guard", C.c_int), ("smooth_start", C.c_int), ("prec_dtype", C.c_int),
                ("h_dtype", C.c_int), ("switch_tol", C.c_double), ("refine_block", C.c_int),
                ("refine_inner_steps", C.c_int), ("refine_inner_dtype", C.c_int),
                ("h64_dtype", C.c_int), ("rr_method", C.c_int),
                ("rr_refine_max", C.c_int),
                ("correction_dtype", C.c_int),
                ("update_dtype", C.c_int), ("graph", C.c_int), ("gram_dtype", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("outer_iters", C.c_int), ("h_applies", C.c_int), ("prec_applies", C.c_int),
                ("inner_steps", C.c_int), ("restarts", C.c_int), ("n_converged", C.c_int),
                ("hnorm_est", C.c_double), ("time_ms", C.c_double), ("h_ms", C.c_double),
                ("prec_ms", C.c_double), ("h_flops", C.c_double), ("prec_flops", C.c_double),
                ("h_launches", C.c_longlong), ("prec_launches", C.c_longlong),
                ("kernel_launches", C.c_longlong), ("h32_ms", C.c_double),
                ("h32_flops", C.c_double), ("h32_launches", C.c_longlong),
                ("gram_ms", C.c_double), ("gram_flops", C.c_double), ("gram_bytes", C.c_double),
                ("gram_launches", C.c_longlong), ("upd_ms", C.c_double),
                ("upd_flops", C.c_double), ("upd_bytes", C.c_double),
                ("upd_launches", C.c_longlong), ("jacobi_calls", C.c_int),
                ("jacobi_sweeps", C.c_int), ("jacobi_rounds", C.c_int),
                ("gs_orthogonalisations", C.c_int), ("gs_second_passes", C.c_int),
                ("rr_mixed_calls", C.c_int), ("rr_fp32_solves", C.c_int),
                ("rr_refine_iters", C.c_int), ("rr_groups_rotated", C.c_int),
                ("rr_fallbacks", C.c_int), ("rr_ms", C.c_double), ("rr_launches", C.c_longlong),
                ("rr_timed", C.c_longlong), ("graph_build_ms", C.c_double),
                ("graph_run_ms", C.c_double),
                ("resid", C.c_double * 64)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "resid"}
        d["resid"] = list(self.resid[: self.n_converged])
        return d


_vp, _dp, _ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
_ll = C.c_longlong
_sig = {
    "tps_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int]),
    "tps_destroy": (C.c_int, [_vp]),
    "tps_last_error": (C.c_char_p, [_vp]),
    "tps_status_string": (C.c_char_p, [C.c_int]),
    "tps_device_status": (C.c_int, [_vp]),
    "tps_selftest_wait_timeout": (C.c_int, [C.c_int, C.c_double]),
    "tps_set_masses": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double]),
    "tps_set_alpha": (C.c_int, [_vp, C.c_double]),
    "tps_set_grid": (C.c_int, [_vp, _ip, _dp]),
    "tps_set_grid_chebyshev": (C.c_int, [_vp, _ip, _dp]),
    "tps_set_potential": (C.c_int, [_vp, _vp, C.c_int]),
    "tps_set_pair_potential": (C.c_int, [_vp, C.c_int, C.c_double, C.c_double]),
    "tps_two_body_v0": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_double, C.c_int,
                                  C.c_double, C.c_int, C.c_double, _dp]),
    "tps_chebyshev_grid": (C.c_int, [C.c_int, C.c_double, _dp, _dp, _dp, _dp, _dp]),
    "tps_get_info": (C.c_int, [_vp, C.POINTER(_ll), _dp]),
    "tps_set_autotune": (C.c_int, [C.c_int]),
    "tps_apply_h": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_double, C.c_int, _vp]),
    "tps_apply_prec": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_double, C.c_int, _vp]),
    "tps_default_opts": (None, [C.POINTER(SolverOpts)]),
    "tps_solve": (C.c_int, [_vp, C.c_int, C.c_int, C.c_double, C.c_int, _vp, C.c_int,
                            C.POINTER(SolverOpts), _dp, _vp, C.POINTER(Stats), _vp]),
    "tps_gram": (C.c_int, [_vp, _vp, _ll, C.c_int, _vp, _ll, C.c_int, _ll, _vp, C.c_int, _vp]),
    "tps_gram_tc": (C.c_int, [_vp, _vp, _ll, C.c_int, _vp, _ll, C.c_int, _ll, _vp, C.c_int, _vp]),
    "tps_block_update": (C.c_int, [_vp, _vp, _ll, C.c_int, _vp, C.c_int, C.c_int, C.c_double,
                                   _vp, _ll, _ll, _vp]),
    "tps_block_update_tc": (C.c_int, [_vp, _vp, _ll, C.c_int, _vp, C.c_int, C.c_int, C.c_double,
                                      _vp, _ll, _ll, _vp]),
    "tps_orthonormalize": (C.c_int, [_vp, _vp, _ll, C.c_int, _vp, _ll, C.c_int, _ll, _ip, _vp]),
    "tps_small_eigh": (C.c_int, [_vp, _vp, C.c_int, C.c_int, _vp, _vp, C.c_int, _vp]),
    "tps_correction": (C.c_int, [_vp, _vp, C.c_int, _vp, _vp, C.c_int, C.c_int, C.c_int,
                                 C.c_double, _vp, _vp]),
    "tps_gram_noalloc": (C.c_int, [_vp, _ll, C.c_int, _vp, _ll, C.c_int, _ll, _vp, C.c_int, _vp]),
    "tps_solve_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_int), C.c_int,
                                  C.c_double, C.c_int, C.POINTER(SolverOpts), _dp, C.c_int,
                                  C.POINTER(C.c_void_p), C.POINTER(Stats), C.POINTER(C.c_int),
                                  C.c_int]),
    "tps_ws_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int, C.c_int,
                                C.c_int, C.c_ulonglong]),
    "tps_ws_destroy": (C.c_int, [_vp]),
    "tps_ws_last_error": (C.c_char_p, [_vp]),
    "tps_ws_info": (C.c_int, [_vp, C.POINTER(_ll), C.POINTER(C.c_int)]),
    "tps_ws_get_params": (C.c_int, [_vp, _vp, _ll]),
    "tps_ws_set_params": (C.c_int, [_vp, _vp, _ll]),
    "tps_ws_features": (C.c_int, [C.c_int, _dp, _dp, _dp, _ip, C.POINTER(C.c_float)]),
    "tps_ws_forward": (C.c_int, [_vp, _vp, C.c_int, C.c_int, _vp, _vp]),
    "tps_ws_loss_grad": (C.c_int, [_vp, _vp, _vp, C.c_int, _dp, _vp, _vp]),
    "tps_ws_adam_step": (C.c_int, [_vp, C.c_float, C.c_float, C.c_float, C.c_float, _vp]),
    "tps_ws_project": (C.c_int, [_vp, _vp, _vp, C.c_int, _vp, _vp]),
    "tps_ws_predict": (C.c_int, [_vp, _vp, _vp, C.c_int, _vp, _vp]),
    "tps_ws_solve": (C.c_int, [_vp, _vp, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int,
                               C.c_double, C.c_int, C.POINTER(SolverOpts), _dp, _vp,
                               C.POINTER(Stats), _ip, _vp]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_sig)


class TpsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_lib.tps_status_string(status).decode()} ({status}): {msg}")
        self.status = status


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def default_opts() -> SolverOpts:
    o = SolverOpts()
    _lib.tps_default_opts(C.byref(o))
    return o


def gram_noalloc(A, p, B, q, nrows, G, ldg=None, stream=None):
    """G = A^T B through the allocation-free entry point (no context needed)."""
    st = _lib.tps_gram_noalloc(_ptr(A), nrows, p, _ptr(B), nrows, q, nrows, _ptr(G), ldg or p,
                               _stream(stream))
    if st != OK:
        raise TpsError(st, "tps_gram_noalloc")


def solve_batch(contexts, ks, parity, tol, block, evecs, opts=None, nstreams=8):
    """Solve independent problems concurrently (tps_solve_batch).  contexts: list of
    Context; ks: pairs per instance; evecs: list of float64 CUDA tensors [k_i, N_i].
    Returns (list of eigenvalue arrays, list of Stats, list of statuses)."""
    n = len(contexts)
    kstride = max(ks) if n else 1
    ctx_arr = (C.c_void_p * n)(*[c._h for c in contexts])
    k_arr = (C.c_int * n)(*ks)
    ev = (C.c_double * (n * kstride))()
    vec_arr = (C.c_void_p * n)(*[e.data_ptr() for e in evecs])
    stats = (Stats * n)()
    status = (C.c_int * n)()
    st = _lib.tps_solve_batch(ctx_arr, n, k_arr, parity, tol, block,
                              C.byref(opts) if opts is not None else None, ev, kstride, vec_arr,
                              stats, status, nstreams)
    if st != OK and st != ERR_NOT_CONVERGED:
        raise TpsError(st, "tps_solve_batch")
    lam = [np.array(ev[i * kstride: i * kstride + ks[i]]) for i in range(n)]
    return lam, list(stats), list(status)


def two_body_v0(dim, mu_hl, hbar, E0, shape, sigma, n, L) -> float:
    out = C.c_double()
    st = _lib.tps_two_body_v0(dim, mu_hl, hbar, E0, shape, sigma, n, L, C.byref(out))
    if st != OK:
        raise TpsError(st, "tps_two_body_v0")
    return out.value


def chebyshev_grid(n, L, factors=False):
    """tps_chebyshev_grid: (y [n], D2 [n, n]) of the paper's mapped Chebyshev grid, plus
    (lam [n], S [n, n], Sinv [n, n]) with D2 = S diag(lam) S^-1 when factors is true."""
    y = np.empty(n)
    D2 = np.empty((n, n))
    f = [np.empty(n), np.empty((n, n)), np.empty((n, n))] if factors else [None] * 3
    ptr = lambda a: a.ctypes.data_as(_dp) if a is not None else None
    st = _lib.tps_chebyshev_grid(n, L, ptr(y), ptr(D2), *[ptr(a) for a in f])
    if st != OK:
        raise TpsError(st, "tps_chebyshev_grid")
    return (y, D2, *f) if factors else (y, D2)


class Context:
    """Owns one tps_ctx.  Tensors passed in must be contiguous float64 CUDA tensors."""

    def __init__(self, dim: int, device: int = 0):
        h = C.c_void_p()
        st = _lib.tps_create(C.byref(h), dim, device)
        if st != OK:
            raise TpsError(st, "tps_create")
        self._h = h
        self.dim = dim
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            _lib.tps_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _check(self, st, what):
        if st != OK:
            raise TpsError(st, f"{what}: {_lib.tps_last_error(self._h).decode()}")

    # ---- problem definition -------------------------------------------------
    def set_masses(self, M, m, hbar=1.0):
        self._check(_lib.tps_set_masses(self._h, M, m, hbar), "set_masses")

    def set_alpha(self, alpha):
        self._check(_lib.tps_set_alpha(self._h, alpha), "set_alpha")

    def set_grid(self, n, L):
        na = (C.c_int * len(n))(*n)
        La = (C.c_double * len(L))(*L)
        self._check(_lib.tps_set_grid(self._h, na, La), "set_grid")

    def set_grid_chebyshev(self, n, L):
        """The paper's mapped Chebyshev grid (1D): n[k] roots, map parameters L[k]."""
        na = (C.c_int * len(n))(*n)
        La = (C.c_double * len(L))(*L)
        self._check(_lib.tps_set_grid_chebyshev(self._h, na, La), "set_grid_chebyshev")

    def set_potential(self, V):
        """V: float64 tensor of N entries (host or device) or a numpy array (host)."""
        if isinstance(V, np.ndarray):
            V = np.ascontiguousarray(V, dtype=np.float64)
            self._check(_lib.tps_set_potential(self._h, V.ctypes.data_as(C.c_void_p), 0),
                        "set_potential")
        else:
            self._check(_lib.tps_set_potential(self._h, _ptr(V), 1 if V.is_cuda else 0),
                        "set_potential")

    def set_pair_potential(self, shape, v0, sigma):
        self._check(_lib.tps_set_pair_potential(self._h, shape, v0, sigma), "set_pair_potential")

    def info(self):
        N = C.c_longlong()
        h = C.c_double()
        self._check(_lib.tps_get_info(self._h, C.byref(N), C.byref(h)), "get_info")
        return N.value, h.value

    def device_status(self):
        """Synchronise; raise TpsError(TIMEOUT) if a tensor-core kernel gave up a wait."""
        self._check(_lib.tps_device_status(self._h), "device_status")

    # ---- operator applications -------------------------------------------------
    def apply_h(self, psi, out, theta=0.0, stream=None, dtype=F64):
        nvec = psi.numel() // self.info()[0]
        self._check(_lib.tps_apply_h(self._h, _ptr(psi), _ptr(out), nvec, theta, dtype,
                                     _stream(stream)), "apply_h")

    def apply_prec(self, r, out, theta, stream=None, dtype=F64):
        nvec = r.numel() // self.info()[0]
        self._check(_lib.tps_apply_prec(self._h, _ptr(r), _ptr(out), nvec, theta, dtype,
                                        _stream(stream)), "apply_prec")

    # ---- solver -----------------------------------------------------------------
    def solve(self, k, parity, tol, block, evecs, x0=None, opts=None, stream=None,
              allow_not_converged=False):
        """Returns (evals numpy [k], Stats); eigenvectors written into ``evecs`` [k, N]."""
        ev = (C.c_double * k)()
        stats = Stats()
        n_x0 = 0 if x0 is None else x0.numel() // self.info()[0]
        st = _lib.tps_solve(self._h, k, parity, tol, block, _ptr(x0), n_x0,
                            C.byref(opts) if opts is not None else None, ev, _ptr(evecs),
                            C.byref(stats), _stream(stream))
        if st != OK and not (allow_not_converged and st == ERR_NOT_CONVERGED):
            self._check(st, "solve")
        return np.array(ev[: stats.n_converged]), stats

    # ---- building blocks ----------------------------------------------------------
    def gram(self, A, p, B, q, nrows, G, ldg=None, lda=None, ldb=None, stream=None, dtype=F64):
        """G = A^T B; dtype F64 (FMA pipe) or F64_TC (digit-split tensor-core products)."""
        fn = _lib.tps_gram_tc if dtype == F64_TC else _lib.tps_gram
        self._check(fn(self._h, _ptr(A), lda or nrows, p, _ptr(B), ldb or nrows, q, nrows,
                       _ptr(G), ldg or p, _stream(stream)), "gram")

    def block_update(self, A, p, Y, q, beta, Cm, nrows, ldy=None, stream=None, dtype=F64):
        """C = beta C + A Y; dtype F64 (FMA pipe) or F64_TC (digit-split tensor-core products)."""
        fn = _lib.tps_block_update_tc if dtype == F64_TC else _lib.tps_block_update
        self._check(fn(self._h, _ptr(A), nrows, p, _ptr(Y), ldy or p, q, beta, _ptr(Cm), nrows,
                       nrows, _stream(stream)), "block_update")

    def orthonormalize(self, Q, nq, T, b, nrows, stream=None):
        rank = C.c_int()
        self._check(_lib.tps_orthonormalize(self._h, _ptr(Q), nrows, nq, _ptr(T), nrows, b, nrows,
                                            C.byref(rank), _stream(stream)), "orthonormalize")
        return rank.value

    def small_eigh(self, G, m, theta, Y, stream=None):
        self._check(_lib.tps_small_eigh(self._h, _ptr(G), m, m, _ptr(theta), _ptr(Y), m,
                                        _stream(stream)), "small_eigh")

    def correction(self, Qt, nq, R, theta, nsys, steps, use_prec, shift, T, stream=None):
        self._check(_lib.tps_correction(self._h, _ptr(Qt), nq, _ptr(R), _ptr(theta), nsys, steps,
                                        use_prec, shift if use_prec else math.nan, _ptr(T),
                                        _stream(stream)), "correction")


class WarmStart:
    """Learned warm-start model (tps_ws_*): an MLP from (M/m, v0, sigma, state index) to a
    rank-R separable start vector, trained on the GPU by the library's own kernels."""

    def __init__(self, px=32, py=32, rank=16, hidden=256, seed=1, device=0):
        h = C.c_void_p()
        st = _lib.tps_ws_create(C.byref(h), device, px, py, rank, hidden, seed)
        if st != OK:
            raise TpsError(st, "tps_ws_create")
        self._h, self.px, self.py, self.rank, self.hidden = h, px, py, rank, hidden
        n, d = C.c_longlong(), C.c_int()
        _lib.tps_ws_info(self._h, C.byref(n), C.byref(d))
        self.nparam, self.out_dim = n.value, d.value

    def close(self):
        if getattr(self, "_h", None):
            _lib.tps_ws_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _check(self, st, what):
        if st != OK:
            raise TpsError(st, f"{what}: {_lib.tps_ws_last_error(self._h).decode()}")

    def get_params(self):
        a = np.empty(self.nparam, dtype=np.float32)
        self._check(_lib.tps_ws_get_params(self._h, a.ctypes.data_as(C.c_void_p), self.nparam),
                    "get_params")
        return a

    def set_params(self, a):
        a = np.ascontiguousarray(a, dtype=np.float32)
        self._check(_lib.tps_ws_set_params(self._h, a.ctypes.data_as(C.c_void_p), a.size),
                    "set_params")

    @staticmethod
    def features(mass_ratio, v0, sigma, state):
        mr, vv, sg = (np.ascontiguousarray(np.atleast_1d(a), dtype=np.float64)
                      for a in (mass_ratio, v0, sigma))
        stt = np.ascontiguousarray(np.atleast_1d(state), dtype=np.int32)
        n = stt.size
        out = np.empty((n, 4), dtype=np.float32)
        st = _lib.tps_ws_features(n, mr.ctypes.data_as(_dp), vv.ctypes.data_as(_dp),
                                  sg.ctypes.data_as(_dp), stt.ctypes.data_as(_ip),
                                  out.ctypes.data_as(C.POINTER(C.c_float)))
        if st != OK:
            raise TpsError(st, "tps_ws_features")
        return out

    def forward(self, X, bf16=False, stream=None):
        import torch
        out = torch.empty(X.shape[0], self.out_dim, dtype=torch.float32, device=X.device)
        self._check(_lib.tps_ws_forward(self._h, _ptr(X), X.shape[0], 1 if bf16 else 0,
                                        _ptr(out), _stream(stream)), "forward")
        return out

    def loss_grad(self, X, T, want_grad=False, stream=None):
        loss = C.c_double()
        g = np.empty(self.nparam, dtype=np.float32) if want_grad else None
        self._check(_lib.tps_ws_loss_grad(self._h, _ptr(X), _ptr(T), X.shape[0], C.byref(loss),
                                          g.ctypes.data_as(C.c_void_p) if want_grad else None,
                                          _stream(stream)), "loss_grad")
        return loss.value, g

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        self._check(_lib.tps_ws_adam_step(self._h, lr, beta1, beta2, eps, _stream(stream)),
                    "adam_step")

    def project(self, ctx, evecs, stream=None):
        import torch
        k = evecs.shape[0]
        T = torch.empty(k, self.px, self.py, dtype=torch.float32, device=evecs.device)
        self._check(_lib.tps_ws_project(self._h, ctx._h, _ptr(evecs), k, _ptr(T),
                                        _stream(stream)), "project")
        return T

    def predict(self, ctx, X, stream=None):
        import torch
        k = X.shape[0]
        out = torch.empty(k, ctx.info()[0], dtype=torch.float64, device=X.device)
        self._check(_lib.tps_ws_predict(self._h, ctx._h, _ptr(X), k, _ptr(out), _stream(stream)),
                    "predict")
        return out


def solve_warm(model, ctx, mass_ratio, v0, sigma, k, parity, tol, block, evecs, opts=None,
               stream=None):
    """tps_ws_solve: solve from the model's predicted start (model None: cold start).
    Returns (eigenvalues, Stats, used_warm)."""
    ev = (C.c_double * k)()
    stats = Stats()
    used = C.c_int()
    st = _lib.tps_ws_solve(model._h if model is not None else None, ctx._h, mass_ratio, v0,
                           sigma, k, parity, tol, block,
                           C.byref(opts) if opts is not None else None, ev, _ptr(evecs),
                           C.byref(stats), C.byref(used), _stream(stream))
    if st != OK:
        raise TpsError(st, f"tps_ws_solve: {_lib.tps_last_error(ctx._h).decode()}")
    return np.array(ev[:k]), stats, bool(used.value)
