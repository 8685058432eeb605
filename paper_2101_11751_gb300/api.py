"""ctypes binding of libfkski.so with the C ABI's names (argument marshalling only).

Every computation runs in the CUDA library; this module converts torch tensors to device
pointers, fills the C structs and raises on non-zero status codes.  ``load()`` raises if the
library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfkski.so")

OK = 0
E_INVALID_ARG, E_OUT_OF_GRID, E_NONFINITE, E_NOT_CONVERGED = -1, -2, -3, -4
E_BREAKDOWN, E_TIMEOUT, E_OOM, E_CUDA, E_UNSUPPORTED, E_IO = -5, -6, -7, -8, -9, -10
F32, F64, F32X2 = 0, 1, 2
RBF, MATERN52 = 0, 1
X0_ZERO, X0_Y_OVER_S2 = 0, 1
MIXED, DOUBLE, FP32 = 0, 1, 2


class FkskiError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib.fkski_strerror(code).decode() if _lib is not None else str(code)
        if _lib is not None and code in (E_CUDA, E_OOM):
            msg += " [" + _lib.fkski_last_error_detail().decode() + "]"
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


class CGrid(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("M", ctypes.c_int64 * 3), ("lo", ctypes.c_double * 3),
                ("h", ctypes.c_double * 3)]


class CKernel(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("lengthscale", ctypes.c_double * 3),
                ("outputscale", ctypes.c_double), ("noise_var", ctypes.c_double)]


class COpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("maxiter", ctypes.c_int), ("x0_mode", ctypes.c_int),
                ("precision", ctypes.c_int), ("check_every", ctypes.c_int), ("n_probes", ctypes.c_int),
                ("probe_seed", ctypes.c_uint64), ("iterate_budget_bytes", ctypes.c_size_t),
                ("keep_sort", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("keep_points", ctypes.c_int), ("reserved", ctypes.c_int * 5)]


class CInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("t_ms", ctypes.c_double * 8), ("iters_rhs", ctypes.c_int * 65)]


_lib = None
P = ctypes.c_void_p
PI64 = ctypes.POINTER(ctypes.c_int64)
PD = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "fkski_default_opts": (None, [ctypes.POINTER(COpts)]),
    "fkski_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "fkski_last_error_detail": (ctypes.c_char_p, []),
    "fkski_kernel_launches": (ctypes.c_longlong, []),
    "fkski_precompute": (ctypes.c_int, [ctypes.POINTER(CGrid), P, P, P, ctypes.c_int64, ctypes.c_int,
                                        ctypes.POINTER(COpts), ctypes.POINTER(P), P]),
    "fkski_stats_info": (ctypes.c_int, [P, ctypes.POINTER(CGrid), PI64, PI64, PI64,
                                        ctypes.POINTER(ctypes.c_int), PD, ctypes.POINTER(ctypes.c_int)]),
    "fkski_stats_export": (ctypes.c_int, [P, P, P, P, P, P]),
    "fkski_stats_export_sort": (ctypes.c_int, [P, P, P, P, P]),
    "fkski_stats_save": (ctypes.c_int, [P, ctypes.c_char_p, P]),
    "fkski_stats_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(P), P]),
    "fkski_destroy": (None, [P]),
    "fkski_kg_mvm": (ctypes.c_int, [ctypes.POINTER(CGrid), ctypes.POINTER(CKernel), ctypes.c_int, P, P,
                                    ctypes.c_int, ctypes.c_int, P]),
    "fkski_tuning_table": (ctypes.c_size_t, [ctypes.c_char_p, ctypes.c_size_t]),
    "fkski_trim_memory": (ctypes.c_int, []),
    "fkski_kg_mvm_noalloc": (ctypes.c_int, [ctypes.POINTER(CGrid), ctypes.POINTER(CKernel), ctypes.c_int, P, P,
                                            ctypes.c_int, ctypes.c_int, P]),
    "fkski_band_mvm": (ctypes.c_int, [P, P, P, ctypes.c_int, ctypes.c_int, P]),
    "fkski_solve": (ctypes.c_int, [P, ctypes.POINTER(CKernel), ctypes.POINTER(COpts), P, P,
                                   ctypes.POINTER(CInfo), P]),
    "fkski_predict": (ctypes.c_int, [P, P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int64, P, P]),
    "fkski_logdet_lanczos": (ctypes.c_int, [P, ctypes.POINTER(CKernel), ctypes.c_int, PD, PD, ctypes.POINTER(CInfo), P]),
    "fkski_ski_solve": (ctypes.c_int, [P, ctypes.POINTER(CKernel), ctypes.POINTER(COpts), P, P,
                                       ctypes.POINTER(CInfo), P]),
    "fkski_posterior_cov": (ctypes.c_int, [P, ctypes.POINTER(CKernel), ctypes.POINTER(COpts), P, ctypes.c_int,
                                           ctypes.c_int64, P, ctypes.POINTER(CInfo), P]),
    "fkski_posterior_cov_lowrank": (ctypes.c_int, [P, ctypes.POINTER(CKernel), ctypes.POINTER(COpts), ctypes.c_int, P,
                                                   ctypes.c_int, ctypes.c_int64, P, ctypes.POINTER(CInfo), P]),
    "fkski_precompute_batched": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(CGrid), P, P,
                                                ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.POINTER(COpts),
                                                P, P]),
    "fkski_solve_batched": (ctypes.c_int, [ctypes.c_int, P, ctypes.POINTER(CKernel), ctypes.POINTER(COpts), P, P,
                                           ctypes.POINTER(CInfo), P]),
    "fkski_predict_batched": (ctypes.c_int, [ctypes.c_int, P, P, ctypes.c_int, P, ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_int64), P, ctypes.POINTER(ctypes.c_int), P]),
    "fkski_loglik_forward": (ctypes.c_int, [P, ctypes.POINTER(CKernel), ctypes.POINTER(COpts), PD,
                                            ctypes.POINTER(CInfo), P]),
    "fkski_loglik_backward": (ctypes.c_int, [P, ctypes.POINTER(CKernel), ctypes.POINTER(COpts), PD,
                                             ctypes.POINTER(CInfo), P]),
    "fkski_grad": (ctypes.c_int, [P, ctypes.POINTER(CKernel), ctypes.POINTER(COpts), PD, PD,
                                  ctypes.POINTER(CInfo), P]),
}


def load(path: Optional[str] = None):
    """Load libfkski.so (raises if absent: the CUDA library is the only implementation)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libfkski.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(code: int, where: str):
    if code != OK:
        raise FkskiError(code, where)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor], allow_pinned: bool = False):
    if t is None:
        return None
    if not t.is_cuda and not (allow_pinned and t.is_pinned()):
        raise ValueError("expected a CUDA tensor" + (" or a pinned host tensor" if allow_pinned else ""))
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float64:
        return F64
    raise TypeError(t.dtype)


def c_grid(grid) -> CGrid:
    g = CGrid()
    g.d = grid.d
    for k in range(3):
        g.M[k] = int(grid.M[k]) if k < grid.d else 1
        g.lo[k] = float(grid.lo[k]) if k < grid.d else 0.0
        g.h[k] = float(grid.h[k]) if k < grid.d else 1.0
    return g


def c_kernel(kernel) -> CKernel:
    k = CKernel()
    k.type = int(kernel.type)
    for i in range(3):
        k.lengthscale[i] = float(kernel.lengthscale[i]) if i < len(kernel.lengthscale) else 1.0
    k.outputscale = float(kernel.outputscale)
    k.noise_var = float(kernel.noise_var)
    return k


def opts(**kw) -> COpts:
    o = COpts()
    load().fkski_default_opts(ctypes.byref(o))
    for key, val in kw.items():
        setattr(o, key, val)
    return o


class Stats:
    """Owner of an fkski_stats handle (released by fkski_destroy)."""

    def __init__(self, handle: ctypes.c_void_p, grid, n_points: int):
        self.handle = handle
        self.grid = grid
        self.n = n_points

    def info(self):
        g = CGrid()
        n, m, nc = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        npb, dt = ctypes.c_int(), ctypes.c_int()
        yty = ctypes.c_double()
        _check(load().fkski_stats_info(self.handle, ctypes.byref(g), ctypes.byref(n), ctypes.byref(m),
                                       ctypes.byref(nc), ctypes.byref(npb), ctypes.byref(yty),
                                       ctypes.byref(dt)), "fkski_stats_info")
        return dict(n=n.value, m=m.value, ncells=nc.value, n_probes=npb.value, yty=yty.value,
                    dtype=dt.value)

    def close(self):
        if self.handle is not None and _lib is not None:
            _lib.fkski_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def precompute(X: torch.Tensor, y: torch.Tensor, grid, Z: Optional[torch.Tensor] = None, n_probes: int = 0,
               probe_seed: int = 0, keep_sort: bool = False, keep_points: bool = False, stream=None) -> Stats:
    """fkski_precompute: X (d, n) and y (n) of one dtype, CUDA tensors or pinned host tensors (read
    once by the key kernel over the host link); Z optional (T, n)."""
    load()
    if Z is not None:
        n_probes = Z.shape[0]
    o = opts(n_probes=n_probes, probe_seed=probe_seed, keep_sort=int(keep_sort), keep_points=int(keep_points))
    h = ctypes.c_void_p()
    g = c_grid(grid)
    code = _lib.fkski_precompute(ctypes.byref(g), _ptr(X, True), _ptr(y, True), _ptr(Z, True), X.shape[1], _dtype_code(X),
                                 ctypes.byref(o), ctypes.byref(h), _stream(stream))
    _check(code, "fkski_precompute")
    return Stats(h, grid, X.shape[1])


def stats_export(st: Stats, want_band: bool = True):
    import numpy as np
    inf = st.info()
    nb = 7 ** st.grid.d
    band = np.zeros((nb, inf["m"])) if want_band else None
    wty = np.zeros(inf["m"])
    wtz = np.zeros((inf["n_probes"], inf["m"]))
    ztz = np.zeros(max(inf["n_probes"], 1))
    vp = lambda a: ctypes.c_void_p(a.ctypes.data) if a is not None else None  # noqa: E731
    _check(load().fkski_stats_export(st.handle, vp(band), vp(wty), vp(wtz) if inf["n_probes"] else None,
                                     vp(ztz), _stream(None)), "fkski_stats_export")
    return dict(band=band, wty=wty, wtz=wtz, ztz=ztz[:inf["n_probes"]], yty=inf["yty"])


def stats_export_sort(st: Stats):
    import numpy as np
    inf = st.info()
    keys = np.zeros(inf["n"], np.uint32)
    perm = np.zeros(inf["n"], np.int64)
    off = np.zeros(inf["ncells"] + 1, np.int64)
    vp = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    _check(load().fkski_stats_export_sort(st.handle, vp(keys), vp(perm), vp(off), _stream(None)),
           "fkski_stats_export_sort")
    return dict(keys=keys, perm=perm, offsets=off)


def stats_save(st: Stats, path: str):
    _check(load().fkski_stats_save(st.handle, path.encode(), _stream(None)), "fkski_stats_save")


def stats_load(path: str, grid) -> Stats:
    h = ctypes.c_void_p()
    _check(load().fkski_stats_load(path.encode(), ctypes.byref(h), _stream(None)), "fkski_stats_load")
    st = Stats(h, grid, 0)
    st.n = st.info()["n"]
    return st


def kg_mvm(grid, kernel, V: torch.Tensor, param: int = -1, stream=None, double_float: bool = False) -> torch.Tensor:
    """fkski_kg_mvm: K_G V (or dK_G/dtheta V) for V of shape (R, m) or (m,).  With double_float,
    V is an FP32 tensor of shape (..., m, 2) holding (hi, lo) pairs (FKSKI_F32X2)."""
    load()
    out = torch.empty_like(V)
    if double_float:
        if V.dtype != torch.float32 or V.shape[-1] != 2:
            raise ValueError("double-float vectors are float32 tensors of shape (..., m, 2)")
        R, code = (1 if V.dim() == 2 else V.shape[0]), F32X2
    else:
        R, code = (1 if V.dim() == 1 else V.shape[0]), _dtype_code(V)
    g, k = c_grid(grid), c_kernel(kernel)
    _check(_lib.fkski_kg_mvm(ctypes.byref(g), ctypes.byref(k), param, _ptr(V), _ptr(out), R, code,
                             _stream(stream)), "fkski_kg_mvm")
    return out


NOALLOC_SCRATCH_BYTES = 16 << 20


def kg_mvm_noalloc(grid, kernel, V: torch.Tensor, out: torch.Tensor, param: int = -1, stream=None) -> torch.Tensor:
    """fkski_kg_mvm_noalloc: out = K_G V without any device allocation inside the call (RBF only).

    The caller provides `out` (same shape and dtype as V); the library works in one fixed
    per-device scratch array, so calls on one device must not overlap."""
    load()
    if out.shape != V.shape or out.dtype != V.dtype or not out.is_contiguous():
        raise ValueError("out must be a contiguous tensor of V's shape and dtype")
    R = 1 if V.dim() == 1 else V.shape[0]
    g, k = c_grid(grid), c_kernel(kernel)
    rc = _lib.fkski_kg_mvm_noalloc(ctypes.byref(g), ctypes.byref(k), param, _ptr(V), _ptr(out), R,
                                   _dtype_code(V), _stream(stream))
    if rc == E_UNSUPPORTED:
        raise FkskiError(rc, "fkski_kg_mvm_noalloc: needs an RBF kernel, M_k <= 2048 and, for d > 1, "
                             f"nrhs*m*{V.element_size()} bytes within {NOALLOC_SCRATCH_BYTES} - 96 KiB")
    _check(rc, "fkski_kg_mvm_noalloc")
    return out


def tuning_table() -> str:
    """The K_G pass configurations chosen by the autotuner so far (fkski_tuning_table)."""
    load()
    n = _lib.fkski_tuning_table(None, 0)
    buf = ctypes.create_string_buffer(n)
    _lib.fkski_tuning_table(buf, n)
    return buf.value.decode()


def band_mvm(st: Stats, X: torch.Tensor, stream=None, double_float: bool = False) -> torch.Tensor:
    """fkski_band_mvm: (W^T W) X for X of shape (R, m) or (m,).  With double_float, X is an FP32
    tensor of shape (..., m, 2) holding (hi, lo) pairs (FKSKI_F32X2, the MIXED solver's vectors)."""
    load()
    out = torch.empty_like(X)
    if double_float:
        if X.dtype != torch.float32 or X.shape[-1] != 2:
            raise ValueError("double-float vectors are float32 tensors of shape (..., m, 2)")
        R = 1 if X.dim() == 2 else X.shape[0]
        code = F32X2
    else:
        R = 1 if X.dim() == 1 else X.shape[0]
        code = _dtype_code(X)
    _check(_lib.fkski_band_mvm(st.handle, _ptr(X), _ptr(out), R, code, _stream(stream)), "fkski_band_mvm")
    return out


def solve(st: Stats, kernel, rtol: float = 1e-6, maxiter: int = 1000, x0_mode: int = X0_Y_OVER_S2,
          precision: int = MIXED, check_every: int = 16, stream=None, allow_not_converged: bool = False):
    """fkski_solve: returns (a = W^T z, v = K_G W^T z, info dict)."""
    load()
    m = st.info()["m"]
    dt = torch.float64 if precision == DOUBLE else torch.float32
    a = torch.empty(m, dtype=dt, device="cuda")
    v = torch.empty(m, dtype=dt, device="cuda")
    o = opts(rtol=rtol, maxiter=maxiter, x0_mode=x0_mode, precision=precision, check_every=check_every)
    inf = CInfo()
    k = c_kernel(kernel)
    code = _lib.fkski_solve(st.handle, ctypes.byref(k), ctypes.byref(o), _ptr(a), _ptr(v), ctypes.byref(inf),
                            _stream(stream))
    if not (allow_not_converged and code == E_NOT_CONVERGED):
        _check(code, "fkski_solve")
    return a, v, dict(iters=inf.iters, rel_residual=inf.rel_residual, status=code)


def predict(st: Stats, v: torch.Tensor, Xstar: torch.Tensor, stream=None) -> torch.Tensor:
    load()
    mu = torch.empty(Xstar.shape[1], dtype=v.dtype, device="cuda")
    _check(_lib.fkski_predict(st.handle, _ptr(v), _dtype_code(v), _ptr(Xstar), _dtype_code(Xstar),
                              Xstar.shape[1], _ptr(mu), _stream(stream)), "fkski_predict")
    return mu


def logdet_lanczos(st: Stats, kernel, k: int, stream=None):
    """fkski_logdet_lanczos: SLQ log-determinant with k EFLA steps per probe; (estimate, terms)."""
    load()
    import numpy as np
    npb = st.info()["n_probes"]
    L = ctypes.c_double()
    terms = np.zeros(max(npb, 1))
    inf = CInfo()
    k_ = c_kernel(kernel)
    _check(_lib.fkski_logdet_lanczos(st.handle, ctypes.byref(k_), k, ctypes.byref(L),
                                     terms.ctypes.data_as(PD), ctypes.byref(inf), _stream(stream)),
           "fkski_logdet_lanczos")
    return L.value, terms[:npb], dict(steps=inf.iters)


def ski_solve(st: Stats, kernel, rtol: float = 1e-6, maxiter: int = 1000, check_every: int = 16, stream=None,
              allow_not_converged: bool = False, precision: int = MIXED):
    """fkski_ski_solve: plain SKI n-space CG (Alg. 1); needs precompute(..., keep_points=True).
    Outputs are FP64 for FP64 points or precision DOUBLE, else FP32."""
    load()
    inf_ = st.info()
    dt = torch.float64 if (inf_["dtype"] == F64 or precision == DOUBLE) else torch.float32
    a = torch.empty(inf_["m"], dtype=dt, device="cuda")
    v = torch.empty(inf_["m"], dtype=dt, device="cuda")
    o = opts(rtol=rtol, maxiter=maxiter, check_every=check_every, precision=precision)
    inf = CInfo()
    k = c_kernel(kernel)
    code = _lib.fkski_ski_solve(st.handle, ctypes.byref(k), ctypes.byref(o), _ptr(a), _ptr(v), ctypes.byref(inf),
                                _stream(stream))
    if not (allow_not_converged and code == E_NOT_CONVERGED):
        _check(code, "fkski_ski_solve")
    return a, v, dict(iters=inf.iters, rel_residual=inf.rel_residual, status=code)


def posterior_cov(st: Stats, kernel, Xstar: torch.Tensor, rtol: float = 1e-6, maxiter: int = 1000,
                  precision: int = MIXED, check_every: int = 16, stream=None, allow_not_converged: bool = False):
    """fkski_posterior_cov: (nstar, nstar) FP64 posterior covariance at the test points."""
    load()
    ns = Xstar.shape[1]
    cov = torch.empty(ns, ns, dtype=torch.float64, device="cuda")
    o = opts(rtol=rtol, maxiter=maxiter, precision=precision, check_every=check_every)
    inf = CInfo()
    k = c_kernel(kernel)
    code = _lib.fkski_posterior_cov(st.handle, ctypes.byref(k), ctypes.byref(o), _ptr(Xstar), _dtype_code(Xstar), ns,
                                    _ptr(cov), ctypes.byref(inf), _stream(stream))
    if not (allow_not_converged and code == E_NOT_CONVERGED):
        _check(code, "fkski_posterior_cov")
    return cov, dict(iters=inf.iters, rel_residual=inf.rel_residual, status=code)


def posterior_cov_lowrank(st: Stats, kernel, Xstar: torch.Tensor, k: int, stream=None):
    """fkski_posterior_cov_lowrank: rank-k (EFLA) approximation of the posterior covariance."""
    load()
    ns = Xstar.shape[1]
    cov = torch.empty(ns, ns, dtype=torch.float64, device="cuda")
    o = opts()
    inf = CInfo()
    kk = c_kernel(kernel)
    _check(_lib.fkski_posterior_cov_lowrank(st.handle, ctypes.byref(kk), ctypes.byref(o), k, _ptr(Xstar),
                                            _dtype_code(Xstar), ns, _ptr(cov), ctypes.byref(inf), _stream(stream)),
           "fkski_posterior_cov_lowrank")
    return cov, dict(steps=inf.iters)


def precompute_batched(Xs: Sequence[torch.Tensor], ys: Sequence[torch.Tensor], grids, stream=None):
    """fkski_precompute_batched: one statistics object per problem (X_p (d_p, n_p), y_p (n_p))."""
    load()
    P = len(Xs)
    G = (CGrid * P)(*[c_grid(g) for g in grids])
    Xp = (ctypes.c_void_p * P)(*[X.data_ptr() for X in Xs])
    yp = (ctypes.c_void_p * P)(*[y.data_ptr() for y in ys])
    n = (ctypes.c_int64 * P)(*[X.shape[1] for X in Xs])
    out = (ctypes.c_void_p * P)()
    o = opts()
    _check(_lib.fkski_precompute_batched(P, G, Xp, yp, n, _dtype_code(Xs[0]), ctypes.byref(o), out, _stream(stream)),
           "fkski_precompute_batched")
    return [Stats(ctypes.c_void_p(out[p]), grids[p], Xs[p].shape[1]) for p in range(P)]


def solve_batched(sts: Sequence[Stats], kernels, rtol: float = 1e-6, maxiter: int = 1000,
                  x0_mode: int = X0_Y_OVER_S2, precision: int = MIXED, check_every: int = 16, stream=None,
                  allow_not_converged: bool = False):
    """fkski_solve_batched: returns lists a_p, v_p and per-problem info dicts."""
    load()
    P = len(sts)
    dt = torch.float64 if precision == DOUBLE else torch.float32
    ms = [st.info()["m"] for st in sts]
    a = [torch.empty(m, dtype=dt, device="cuda") for m in ms]
    v = [torch.empty(m, dtype=dt, device="cuda") for m in ms]
    H = (ctypes.c_void_p * P)(*[st.handle.value for st in sts])
    K = (CKernel * P)(*[c_kernel(k) for k in kernels])
    A = (ctypes.c_void_p * P)(*[t.data_ptr() for t in a])
    V = (ctypes.c_void_p * P)(*[t.data_ptr() for t in v])
    inf = (CInfo * P)()
    o = opts(rtol=rtol, maxiter=maxiter, x0_mode=x0_mode, precision=precision, check_every=check_every)
    code = _lib.fkski_solve_batched(P, H, K, ctypes.byref(o), A, V, inf, _stream(stream))
    if not (allow_not_converged and code == E_NOT_CONVERGED):
        _check(code, "fkski_solve_batched")
    infos = [dict(iters=inf[p].iters, rel_residual=inf[p].rel_residual, status=inf[p].status) for p in range(P)]
    return a, v, infos


def predict_batched(sts: Sequence[Stats], vs: Sequence[torch.Tensor], Xstars: Sequence[torch.Tensor], stream=None):
    """fkski_predict_batched: mu_p = w_{x*}^T v_p for every problem (one launch per distinct d)."""
    load()
    P = len(sts)
    mus = [torch.empty(X.shape[1], dtype=vs[0].dtype, device="cuda") for X in Xstars]
    H = (ctypes.c_void_p * P)(*[st.handle.value for st in sts])
    Vp = (ctypes.c_void_p * P)(*[t.data_ptr() for t in vs])
    Xp = (ctypes.c_void_p * P)(*[t.data_ptr() for t in Xstars])
    n = (ctypes.c_int64 * P)(*[X.shape[1] for X in Xstars])
    M = (ctypes.c_void_p * P)(*[t.data_ptr() for t in mus])
    status = (ctypes.c_int * P)()
    _check(_lib.fkski_predict_batched(P, H, Vp, _dtype_code(vs[0]), Xp, _dtype_code(Xstars[0]), n, M, status,
                                      _stream(stream)), "fkski_predict_batched")
    return mus


def _grad_opts(rtol, maxiter, precision, budget, check_every):
    return opts(rtol=rtol, maxiter=maxiter, precision=precision, iterate_budget_bytes=budget,
                check_every=check_every)


def loglik_forward(st: Stats, kernel, rtol=1e-4, maxiter=1000, precision=MIXED, budget=1 << 30,
                   check_every=16, stream=None, allow_not_converged: bool = False):
    """fkski_loglik_forward: (L, info).  Raises FkskiError when a solve stops at maxiter unless
    allow_not_converged is set (then info['status'] is E_NOT_CONVERGED and L is approximate)."""
    load()
    L = ctypes.c_double()
    inf = CInfo()
    o = _grad_opts(rtol, maxiter, precision, budget, check_every)
    k = c_kernel(kernel)
    code = _lib.fkski_loglik_forward(st.handle, ctypes.byref(k), ctypes.byref(o), ctypes.byref(L),
                                     ctypes.byref(inf), _stream(stream))
    if not (allow_not_converged and code == E_NOT_CONVERGED):
        _check(code, "fkski_loglik_forward")
    return L.value, dict(iters=list(inf.iters_rhs[: 1 + st.info()["n_probes"]]), status=code,
                         rel_residual=inf.rel_residual)


def loglik_backward(st: Stats, kernel, rtol=1e-4, maxiter=1000, precision=MIXED, budget=1 << 30,
                    check_every=16, stream=None):
    load()
    d = st.grid.d
    g = (ctypes.c_double * (d + 2))()
    o = _grad_opts(rtol, maxiter, precision, budget, check_every)
    k = c_kernel(kernel)
    _check(_lib.fkski_loglik_backward(st.handle, ctypes.byref(k), ctypes.byref(o), g, None, _stream(stream)),
           "fkski_loglik_backward")
    return list(g)


def grad(st: Stats, kernel, rtol=1e-4, maxiter=1000, precision=MIXED, check_every=16, stream=None,
         allow_not_converged: bool = False):
    """fkski_grad: (L, gradient, info).  Raises FkskiError when a solve stops at maxiter unless
    allow_not_converged is set."""
    load()
    d = st.grid.d
    L = ctypes.c_double()
    g = (ctypes.c_double * (d + 2))()
    inf = CInfo()
    o = _grad_opts(rtol, maxiter, precision, 1 << 62, check_every)
    k = c_kernel(kernel)
    code = _lib.fkski_grad(st.handle, ctypes.byref(k), ctypes.byref(o), ctypes.byref(L), g, ctypes.byref(inf),
                           _stream(stream))
    if not (allow_not_converged and code == E_NOT_CONVERGED):
        _check(code, "fkski_grad")
    return L.value, list(g), dict(iters=list(inf.iters_rhs[: 1 + st.info()["n_probes"]]), status=code,
                                  rel_residual=inf.rel_residual)


class LogMarginalLikelihood(torch.autograd.Function):
    """L(theta) with theta = (l_1..l_d, s, sigma^2) as a float64 tensor.

    forward runs fkski_loglik_forward (solves + SLQ); backward runs fkski_loglik_backward
    (derivative-Toeplitz MVMs and Hutchinson traces), reusing the forward's solutions when they
    fit the iterate budget and recomputing them otherwise.  A solve that stops at maxiter raises
    FkskiError (E_NOT_CONVERGED) in forward or backward, so an unconverged L or gradient never
    reaches the optimiser silently."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, st: Stats, ktype: int, rtol: float, maxiter: int, precision: int,
                budget: int):
        d = st.grid.d
        th = [float(v) for v in theta.detach().cpu().tolist()]
        from .synth import Kernel
        kern = Kernel(ktype, tuple(th[:d]), th[d], th[d + 1])
        L, _ = loglik_forward(st, kern, rtol=rtol, maxiter=maxiter, precision=precision, budget=budget)
        ctx.st, ctx.kern = st, kern
        ctx.cfg = (rtol, maxiter, precision, budget)
        return theta.new_tensor(L)

    @staticmethod
    def backward(ctx, gout):
        rtol, maxiter, precision, budget = ctx.cfg
        g = loglik_backward(ctx.st, ctx.kern, rtol=rtol, maxiter=maxiter, precision=precision, budget=budget)
        gt = torch.tensor(g, dtype=torch.float64, device=gout.device) * gout
        return gt, None, None, None, None, None, None


def log_marginal_likelihood(theta: torch.Tensor, st: Stats, ktype: int = RBF, rtol: float = 1e-4,
                            maxiter: int = 1000, precision: int = MIXED, budget: int = 1 << 30):
    return LogMarginalLikelihood.apply(theta, st, ktype, rtol, maxiter, precision, budget)
