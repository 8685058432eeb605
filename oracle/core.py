"""fkski oracle, numpy/scipy part -- TEST INFRASTRUCTURE ONLY (see package docstring).

Every function is a plain FP64 restatement of a definition in the paper (section / equation /
algorithm cited in its docstring), with library primitives (dense LU/Cholesky, eigh, sparse
matrix products, FFT) as steps.  No blocking, fusion or reordering beyond the cited definition.

Parity pins (tests/test_oracle_pins.py) -- every function below is pinned:
  keys / Keys weights     worked values of Keys' kernel, partition of unity, exact quadratics,
                          exact rational floor for cell indices
  precompute              brute-force dense W, Claim 2 sparsity, symmetry, PSD, 1^T W^T W 1 = n
  kg_*                    dense kernel matrix from grid points; Toeplitz symmetry; FFT vs direct
  cg                      dense solve; Prop. 1 (factorized recurrences give the same iterates)
  ski_* / gsgp_*          Theorem 1 (mean, covariance), Claim 7 (log-det), Fact 2 log-likelihood
  slq_logdet              exact log-det when probes are unit vectors and Lanczos runs to the end
  grad_*                  central finite differences of the exact dense log-likelihood
"""
from __future__ import annotations

import math
from typing import Dict, Optional, Tuple

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .lib import get, or_grid, ptr

RBF = 0
MATERN52 = 1
OR_OK, OR_E_INVALID, OR_E_OUT_OF_GRID, OR_E_NONFINITE, OR_E_OOM = 0, 1, 2, 3, 4


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle status {code}")
        self.code = code


def _check(st: int):
    if st != OR_OK:
        raise OracleError(st)


def _xdtype(X: np.ndarray) -> int:
    if X.dtype == np.float32:
        return 0
    if X.dtype == np.float64:
        return 1
    raise TypeError(X.dtype)


# ------------------------------------------------------------------ interpolation (Sec. 3, Def. 2)

def keys_u(s: float) -> float:
    """Keys' cubic convolution kernel with a = -1/2 (reference [keys1981cubic])."""
    return get().or_keys_u(float(s))


def keys_weights(t: float) -> np.ndarray:
    """Weights on the 4 nodes c-1..c+2 for local coordinate t in [0, 1]."""
    w = np.zeros(4)
    get().or_keys_weights(float(t), ptr(w))
    return w


def cell_key_f32(x: float, lo: float, h: float, M: int):
    """(status, cell, t32, t64) for one FP32 coordinate (exact float sequence; see C source)."""
    import ctypes
    c = ctypes.c_int64()
    t32 = ctypes.c_float()
    t64 = ctypes.c_double()
    st = get().or_cell_key_f32(ctypes.c_float(x), lo, h, M, ctypes.byref(c), ctypes.byref(t32),
                               ctypes.byref(t64))
    return st, c.value, t32.value, t64.value


def keys(grid, X: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Linear cell key (C order over cells c_k - 1) and FP32 local coordinates per point."""
    X = np.ascontiguousarray(X)
    n = X.shape[1]
    k = np.zeros(n, dtype=np.uint32)
    t = np.zeros((grid.d, n), dtype=np.float32)
    g = or_grid(grid)
    _check(get().or_keys(g, ptr(X), _xdtype(X), n, ptr(k), ptr(t)))
    return k, t


def cell_sort(grid, X: np.ndarray, y: np.ndarray) -> Dict[str, np.ndarray]:
    """The precompute's cell sort alone (Sec. 3.1 reading: stable by cell key, ties by input
    index): keys, perm and segment offsets, O(n)."""
    X = np.ascontiguousarray(X)
    y = np.ascontiguousarray(y, dtype=X.dtype)
    n = X.shape[1]
    out = dict(keys=np.zeros(n, np.uint32), perm=np.zeros(n, np.int64),
               offsets=np.zeros(grid.ncells + 1, np.int64))
    _check(get().or_precompute(or_grid(grid), ptr(X), _xdtype(X), ptr(y), n, 0, 0, ptr(out["keys"]),
                               ptr(out["perm"]), ptr(out["offsets"]), None, None, None, None))
    return out


def rademacher(seed: int, j: int, n: int) -> np.ndarray:
    """Probe j: z(i) = +-1 from SplitMix64 at counter j*2^40 + i + 1."""
    out = np.zeros(n)
    get().or_rademacher_fill(seed, j, n, ptr(out))
    return out


def precompute(grid, X: np.ndarray, y: np.ndarray, nprobe: int = 0, seed: int = 0,
               want_band: bool = True) -> Dict[str, np.ndarray]:
    """Sufficient statistics of Sec. 3.1 by explicit per-point sums, plus the stable cell sort.

    Returns keys, perm, offsets, band (7^d x m, band[o, j] = (W^T W)[j, j + delta(o)]), wty, yty
    and wtz (nprobe x m)."""
    X = np.ascontiguousarray(X)
    y = np.ascontiguousarray(y, dtype=X.dtype)
    n = X.shape[1]
    m = grid.m
    nb = 7 ** grid.d
    out = dict(keys=np.zeros(n, np.uint32), perm=np.zeros(n, np.int64),
               offsets=np.zeros(grid.ncells + 1, np.int64),
               band=np.zeros((nb, m)) if want_band else None, wty=np.zeros(m),
               yty=np.zeros(1), wtz=np.zeros((max(nprobe, 0), m)))
    g = or_grid(grid)
    st = get().or_precompute(g, ptr(X), _xdtype(X), ptr(y), n, nprobe, seed, ptr(out["keys"]),
                             ptr(out["perm"]), ptr(out["offsets"]), ptr(out["band"]),
                             ptr(out["wty"]), ptr(out["yty"]),
                             ptr(out["wtz"]) if nprobe > 0 else None)
    _check(st)
    out["yty"] = float(out["yty"][0])
    return out


def w_csr(grid, X: np.ndarray) -> sp.csr_matrix:
    """Explicit interpolation matrix W (n x m), row i = w_{x_i} (Sec. 2.2, 4^d nonzeros)."""
    X = np.ascontiguousarray(X)
    n = X.shape[1]
    nnz = 4 ** grid.d
    cols = np.zeros((n, nnz), np.int64)
    vals = np.zeros((n, nnz))
    _check(get().or_w_rows(or_grid(grid), ptr(X), _xdtype(X), n, ptr(cols), ptr(vals)))
    indptr = np.arange(0, n * nnz + 1, nnz, dtype=np.int64)
    return sp.csr_matrix((vals.ravel(), cols.ravel(), indptr), shape=(n, grid.m))


def predict(grid, v: np.ndarray, Xs: np.ndarray) -> np.ndarray:
    """mu(x*) = w_{x*}^T v (Def. 1 / Fact 2 mean with v = K_G W^T z_tilde)."""
    Xs = np.ascontiguousarray(Xs)
    v = np.ascontiguousarray(v, dtype=np.float64)
    mu = np.zeros(Xs.shape[1])
    _check(get().or_predict(or_grid(grid), ptr(v), ptr(Xs), _xdtype(Xs), Xs.shape[1], ptr(mu)))
    return mu


def band_to_dense(grid, band: np.ndarray) -> np.ndarray:
    """Dense m x m matrix from 7^d diagonals (inverse of the band layout)."""
    m = grid.m
    d = grid.d
    Mv = np.asarray(grid.M)
    A = np.zeros((m, m))
    idx = np.stack(np.unravel_index(np.arange(m), tuple(Mv)), axis=1)
    for o in range(7 ** d):
        delta = np.array(np.unravel_index(o, (7,) * d)) - 3
        nb = idx + delta[None, :]
        ok = np.all((nb >= 0) & (nb < Mv[None, :]), axis=1)
        j = np.nonzero(ok)[0]
        jj = np.ravel_multi_index(tuple(nb[ok].T), tuple(Mv))
        A[j, jj] = band[o, j]
    return A


def band_matvec(grid, band: np.ndarray, x: np.ndarray) -> np.ndarray:
    """u = (W^T W) x from the 7^d diagonals (Claim 2: O(m 7^d))."""
    d = grid.d
    Mv = tuple(grid.M)
    X = x.reshape(Mv + x.shape[1:])
    U = np.zeros_like(X, dtype=np.float64)
    B = band.reshape((7 ** d,) + Mv)
    for o in range(7 ** d):
        delta = np.array(np.unravel_index(o, (7,) * d)) - 3
        src = []
        dst = []
        for k in range(d):
            lo_ = max(0, -delta[k])
            hi_ = min(Mv[k], Mv[k] - delta[k])
            dst.append(slice(lo_, hi_))
            src.append(slice(lo_ + delta[k], hi_ + delta[k]))
        bb = B[(o,) + tuple(dst)]
        if x.ndim > 1:
            bb = bb[..., None]
        U[tuple(dst)] += bb * X[tuple(src)]
    return U.reshape(x.shape)


# ------------------------------------------------------------------ kernels and K_G (Sec. 2.2)

def grid_points(grid) -> np.ndarray:
    axes = [grid.lo[k] + grid.h[k] * np.arange(grid.M[k]) for k in range(grid.d)]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([a.ravel() for a in mesh], axis=1)


def kernel_value(kernel, diff: np.ndarray) -> np.ndarray:
    """k(x, x') for stationary kernels as a function of x - x' (last axis = d).

    RBF ARD in a scale kernel: s * exp(-1/2 sum_k (diff_k / l_k)^2)  (App. C.1: squared
    exponential wrapped in a scale kernel).  Matern-5/2 on r = ||diff / l||:
    s * (1 + sqrt5 r + 5/3 r^2) exp(-sqrt5 r)."""
    ell = np.asarray(kernel.lengthscale, dtype=np.float64)
    q = np.sum((diff / ell) ** 2, axis=-1)
    if kernel.type == RBF:
        return kernel.outputscale * np.exp(-0.5 * q)
    r = np.sqrt(q)
    return kernel.outputscale * (1 + math.sqrt(5) * r + 5.0 / 3.0 * r * r) * np.exp(-math.sqrt(5) * r)


def kernel_dvalue(kernel, diff: np.ndarray, param) -> np.ndarray:
    """Derivative of kernel_value w.r.t. ('ell', k) or 'scale'."""
    ell = np.asarray(kernel.lengthscale, dtype=np.float64)
    if param == "scale":
        return kernel_value(kernel, diff) / kernel.outputscale
    k = param[1]
    q = np.sum((diff / ell) ** 2, axis=-1)
    dk2 = diff[..., k] ** 2 / ell[k] ** 3
    if kernel.type == RBF:
        return kernel.outputscale * np.exp(-0.5 * q) * dk2
    r = np.sqrt(q)
    return kernel.outputscale * (5.0 / 3.0) * (1 + math.sqrt(5) * r) * np.exp(-math.sqrt(5) * r) * dk2


def kg_dense(grid, kernel, param=None) -> np.ndarray:
    """K_G = [k(g_i, g_j)] on the grid points (or its derivative), dense m x m."""
    P = grid_points(grid)
    diff = P[:, None, :] - P[None, :, :]
    return kernel_value(kernel, diff) if param is None else kernel_dvalue(kernel, diff, param)


def toeplitz_factor(grid, kernel, k: int, param=None) -> np.ndarray:
    """RBF factor along axis k: T_k[i, j] = exp(-1/2 ((i - j) h_k / l_k)^2) (or d/dl_k)."""
    ell = kernel.lengthscale[k]
    off = (np.arange(grid.M[k])[:, None] - np.arange(grid.M[k])[None, :]) * grid.h[k]
    T = np.exp(-0.5 * (off / ell) ** 2)
    if param is not None and param != "scale" and param[1] == k:
        T = T * off ** 2 / ell ** 3
    return T


def _mode_product(T: np.ndarray, V: np.ndarray, k: int, Mv) -> np.ndarray:
    R = V.shape[1]
    X = V.reshape(tuple(Mv) + (R,))
    X = np.moveaxis(np.tensordot(T, X, axes=([1], [k])), 0, k)
    return X.reshape(-1, R)


def _bttb_first_columns(grid, kernel, param):
    """Kernel on all grid offsets delta in (-M_k, M_k)^d, embedded circulantly (Lee 1986)."""
    d = grid.d
    L = [2 * grid.M[k] for k in range(d)]
    offs = []
    for k in range(d):
        i = np.arange(L[k])
        o = np.where(i < grid.M[k], i, i - L[k]).astype(np.float64)
        o[i == grid.M[k]] = 0.0  # unused slot between the two halves
        offs.append(o * grid.h[k])
    mesh = np.meshgrid(*offs, indexing="ij")
    diff = np.stack(mesh, axis=-1)
    c = kernel_value(kernel, diff) if param is None else kernel_dvalue(kernel, diff, param)
    # zero the slot that does not correspond to any |delta| < M
    for k in range(d):
        sl = [slice(None)] * d
        sl[k] = grid.M[k]
        c[tuple(sl)] = 0.0
    return c


def kg_matvec(grid, kernel, V: np.ndarray, param=None, method: str = "auto") -> np.ndarray:
    """K_G V (or dK_G/dtheta V).  V is m or m x R.

    RBF: K_G = s T_1 (x) ... (x) T_d exactly (the ARD squared exponential factorises over axes),
    applied by dense mode products.  Matern-5/2: multilevel Toeplitz (Sec. 2.2); method 'dense'
    builds K_G from grid points, 'fft' applies the circulant embedding with numpy's FFT."""
    squeeze = V.ndim == 1
    V2 = V.reshape(grid.m, -1).astype(np.float64)
    Mv = grid.M
    if kernel.type == RBF and method in ("auto", "kron"):
        out = V2
        for k in range(grid.d):
            out = _mode_product(toeplitz_factor(grid, kernel, k, param), out, k, Mv)
        scale = 1.0 if param == "scale" else kernel.outputscale
        out = scale * out
    else:
        if method == "auto":
            method = "dense" if grid.m <= 4096 else "fft"
        if method == "dense":
            out = kg_dense(grid, kernel, param) @ V2
        else:
            c = _bttb_first_columns(grid, kernel, param)
            lam = np.real(np.fft.fftn(c))
            R = V2.shape[1]
            out = np.zeros_like(V2)
            for r in range(R):
                X = np.zeros(c.shape)
                X[tuple(slice(0, mk) for mk in Mv)] = V2[:, r].reshape(Mv)
                Y = np.real(np.fft.ifftn(lam * np.fft.fftn(X)))
                out[:, r] = Y[tuple(slice(0, mk) for mk in Mv)].ravel()
    return out.ravel() if squeeze else out


# ------------------------------------------------------------------ solvers (Sec. 4)

def cg(matvec, b: np.ndarray, x0: Optional[np.ndarray], eps: float, maxiter: int):
    """Alg. 1 (conjugate gradient) as printed: exit once r^T r <= eps.

    Returns x, number of alpha steps taken, the alphas and the betas (for Lanczos/SLQ)."""
    x = np.zeros_like(b) if x0 is None else x0.astype(np.float64).copy()
    r = b - matvec(x) if x0 is not None else b.astype(np.float64).copy()
    p = r.copy()
    rr = float(r @ r)
    alphas, betas = [], []
    if rr <= eps:
        return x, 0, alphas, betas
    it = 0
    for _ in range(maxiter):
        Ap = matvec(p)
        alpha = rr / float(p @ Ap)
        x = x + alpha * p
        r = r - alpha * Ap
        alphas.append(alpha)
        it += 1
        rr_new = float(r @ r)
        if rr_new <= eps:
            break
        beta = rr_new / rr
        betas.append(beta)
        p = r + beta * p
        rr = rr_new
    return x, it, alphas, betas


def ski_operator(grid, kernel, W: sp.csr_matrix):
    """v -> (W K_G W^T + sigma^2 I) v, the SKI system of Def. 1.  Where kg_matvec would apply
    K_G as a dense matrix (non-separable kernel, m <= 4096) that matrix is formed once here
    instead of on every product."""
    s2 = kernel.noise_var
    if kernel.type != RBF and grid.m <= 4096:
        K = kg_dense(grid, kernel)

        def mv(v):
            return W @ (K @ (W.T @ v)) + s2 * v
        return mv

    def mv(v):
        return W @ kg_matvec(grid, kernel, W.T @ v) + s2 * v
    return mv


def nspace_mean(grid, kernel, X, y, rtol: float, x0_mode: int = 0, maxiter: int = 10000):
    """Posterior mean by CG in n-space (Alg. 1 on Def. 1's system).

    x0_mode 0: x0 = 0; x0_mode 1: x0 = y / sigma^2 (the start that puts r0 in span(W)).
    Stops when ||r_k||_2 <= rtol ||y||_2.  Returns a = W^T z_tilde, v = K_G a, iteration count."""
    W = w_csr(grid, X)
    y = np.asarray(y, dtype=np.float64)
    mv = ski_operator(grid, kernel, W)
    x0 = None if x0_mode == 0 else y / kernel.noise_var
    z, it, _, _ = cg(mv, y, x0, (rtol ** 2) * float(y @ y), maxiter)
    a = W.T @ z
    return a, kg_matvec(grid, kernel, a), it, z


def nspace_cov(grid, kernel, X, Xs, rtol: float, maxiter: int = 10000):
    """SKI posterior covariance at test points Xs (Def. 1 / Theorem 1) by n-space CG (Alg. 1),
    one solve per test point from x0 = 0:
        cov[:, j] = W_s K w_j - W_s K W^T A^{-1} (W K w_j),  A = W K W^T + sigma^2 I,
    each solve stopped at ||r|| <= rtol ||W K w_j||.  Returns (cov, max iterations)."""
    W = w_csr(grid, X)
    Ws = w_csr(grid, Xs)
    mv = ski_operator(grid, kernel, W)
    ns = Ws.shape[0]
    cov = np.zeros((ns, ns))
    itmax = 0
    for j in range(ns):
        kw = kg_matvec(grid, kernel, Ws[j].toarray().ravel())
        b = W @ kw
        z, it, _, _ = cg(mv, b, None, (rtol ** 2) * float(b @ b), maxiter)
        itmax = max(itmax, it)
        c = kw - kg_matvec(grid, kernel, W.T @ z)
        cov[:, j] = Ws @ c
    return cov, itmax


def lanczos(mv, b: np.ndarray, k: int, breakdown: float = 1e-10):
    """Lanczos tridiagonalisation with full reorthogonalisation (Alg. 6, with its garbled
    updates read as q_{i+1} - alpha_i q_i and T_{i+1,i} = T_{i,i+1}), started at b / ||b||.
    Stops early when beta_{i+1} <= breakdown * ||A q_i|| (invariant Krylov space).
    Returns Q (n x k') and T (k' x k')."""
    n = len(b)
    Q = np.zeros((n, k))
    T = np.zeros((k, k))
    q = b / np.linalg.norm(b)
    q_prev = np.zeros(n)
    beta = 0.0
    kk = k
    for i in range(k):
        Q[:, i] = q
        w = mv(q)
        aq = np.linalg.norm(w)
        w = w - beta * q_prev
        alpha = float(q @ w)
        T[i, i] = alpha
        if i == k - 1:
            break
        w = w - alpha * q
        w = w - Q[:, :i + 1] @ (Q[:, :i + 1].T @ w)
        beta = float(np.linalg.norm(w))
        if beta <= breakdown * aq:
            kk = i + 1
            break
        T[i, i + 1] = T[i + 1, i] = beta
        q_prev, q = q, w / beta
    return Q[:, :kk], T[:kk, :kk]


def lowrank_cov(grid, kernel, X, y, Xs, k: int):
    """Rank-k posterior covariance at test points from k Lanczos steps on A = W K W^T + sigma^2 I
    started at y (the predictive-covariance approximation the paper uses, ref. [ConstantTimePD]):
        A^{-1} ~ Q T^{-1} Q^T,   cov ~ W_s K W_s^T - (Q^T W K W_s^T)^T T^{-1} (Q^T W K W_s^T).
    Returns (cov, T)."""
    W = w_csr(grid, X)
    Ws = w_csr(grid, Xs)
    mv = ski_operator(grid, kernel, W)
    Q, T = lanczos(mv, np.asarray(y, dtype=np.float64), k)
    KWs = kg_matvec(grid, kernel, Ws.T.toarray())  # m x ns
    Ks = W @ KWs                                     # n x ns
    prior = Ws @ KWs
    G = Q.T @ Ks
    return prior - G.T @ np.linalg.solve(T, G), T


def dense_system(grid, kernel, X):
    W = w_csr(grid, X).toarray()
    K = kg_dense(grid, kernel)
    A = W @ K @ W.T + kernel.noise_var * np.eye(W.shape[0])
    return W, K, A


def ski_inference_dense(grid, kernel, X, y, Xs):
    """Def. 1 (SKI) mean, covariance at test points and log-likelihood, by dense algebra."""
    W, K, A = dense_system(grid, kernel, X)
    Ws = w_csr(grid, Xs).toarray()
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    cf = sla.cho_factor(A)
    zt = sla.cho_solve(cf, y)
    mean = Ws @ K @ W.T @ zt
    kt = W @ K @ Ws.T
    cov = Ws @ K @ Ws.T - kt.T @ sla.cho_solve(cf, kt)
    logdet = 2.0 * np.sum(np.log(np.diag(cf[0])))
    ll = -0.5 * (logdet + y @ zt + n * math.log(2 * math.pi))
    return dict(mean=mean, cov=cov, ll=ll, logdet=logdet, ztilde=zt)


def gsgp_inference_dense(grid, kernel, X, y, Xs):
    """Fact 2 (GSGP) mean, covariance and log-likelihood in m-space, by dense algebra."""
    W = w_csr(grid, X).toarray()
    K = kg_dense(grid, kernel)
    Ws = w_csr(grid, Xs).toarray()
    y = np.asarray(y, dtype=np.float64)
    n, m = W.shape
    s2 = kernel.noise_var
    B = K @ (W.T @ W) + s2 * np.eye(m)
    zbar = np.linalg.solve(B, K @ (W.T @ y))
    Cbar = s2 * np.linalg.solve(B, K)
    sign, logdetB = np.linalg.slogdet(B)
    c = n * math.log(2 * math.pi) + (n - m) * math.log(s2)
    ll = -0.5 * (logdetB + y @ (y - W @ zbar) / s2 + c)
    return dict(mean=Ws @ zbar, cov=Ws @ Cbar @ Ws.T, ll=ll, logdetB=logdetB, zbar=zbar)


# ------------------------------------------------------------------ log-likelihood and gradient

def lanczos_from_cg(alphas, betas) -> np.ndarray:
    """Tridiagonal Lanczos matrix from CG coefficients (standard CG-Lanczos relation):
    T[0,0] = 1/a_0, T[i,i] = 1/a_i + b_{i-1}/a_{i-1}, T[i,i+1] = sqrt(b_i)/a_i."""
    k = len(alphas)
    T = np.zeros((k, k))
    for i in range(k):
        T[i, i] = 1.0 / alphas[i] + (betas[i - 1] / alphas[i - 1] if i > 0 else 0.0)
        if i + 1 < k:
            T[i, i + 1] = T[i + 1, i] = math.sqrt(betas[i]) / alphas[i]
    return T


def quad_e1(T: np.ndarray, f) -> float:
    """e_1^T f(T) e_1 through the eigendecomposition of T."""
    lam, V = np.linalg.eigh(T)
    return float(np.sum(V[0, :] ** 2 * f(lam)))


def slq_logdet(mv, Z: np.ndarray, rtol: float, maxiter: int = 10000):
    """Stochastic Lanczos quadrature (refs [ScalableLD], [ubaru2017fast]): logdet A ~
    mean_j ||z_j||^2 e_1^T log(T_j) e_1 with T_j from CG on A x = z_j (x0 = 0).
    Returns the estimate, the solutions x_j and the iteration counts."""
    ests, xs, its = [], [], []
    for j in range(Z.shape[0]):
        z = Z[j]
        zz = float(z @ z)
        x, it, al, be = cg(mv, z, None, (rtol ** 2) * zz, maxiter)
        ests.append(zz * quad_e1(lanczos_from_cg(al, be), np.log))
        xs.append(x)
        its.append(it)
    return float(np.mean(ests)), np.array(xs), its


def slq_logdet_lanczos(mv, Z: np.ndarray, k: int):
    """Stochastic Lanczos quadrature with k steps of Lanczos with full reorthogonalisation
    (Alg. 6) per probe, the route the paper's factorized Lanczos (FLA / EFLA, App. B) serves:
    logdet A ~ mean_j ||z_j||^2 e_1^T log(T_j) e_1.  Returns the estimate and the per-probe terms."""
    terms = []
    for j in range(Z.shape[0]):
        z = np.asarray(Z[j], dtype=np.float64)
        _, T = lanczos(mv, z, k)
        terms.append(float(z @ z) * quad_e1(T, np.log))
    return float(np.mean(terms)), np.array(terms)


def theta_names(kernel):
    return [("ell", k) for k in range(len(kernel.lengthscale))] + ["scale", "noise"]


def loglik_exact(grid, kernel, X, y) -> float:
    _, _, A = dense_system(grid, kernel, X)
    y = np.asarray(y, dtype=np.float64)
    cf = sla.cho_factor(A)
    return float(-0.5 * (2 * np.sum(np.log(np.diag(cf[0]))) + y @ sla.cho_solve(cf, y)
                         + len(y) * math.log(2 * math.pi)))


def grad_exact(grid, kernel, X, y) -> np.ndarray:
    """dL/dtheta for theta = (l_1..l_d, s, sigma^2), exact dense traces:
    dL/dtheta = 1/2 a^T dK a - 1/2 tr(A^{-1} W dK W^T); dL/dsigma^2 = 1/2 z^T z - 1/2 tr(A^{-1})."""
    W, K, A = dense_system(grid, kernel, X)
    y = np.asarray(y, dtype=np.float64)
    Ainv = np.linalg.inv(A)
    z = Ainv @ y
    a = W.T @ z
    g = []
    for th in theta_names(kernel):
        if th == "noise":
            g.append(0.5 * z @ z - 0.5 * np.trace(Ainv))
        else:
            dK = kg_dense(grid, kernel, th)
            g.append(0.5 * a @ dK @ a - 0.5 * np.trace(Ainv @ W @ dK @ W.T))
    return np.array(g)


def grad_fd(grid, kernel, X, y, h: float = 1e-5) -> np.ndarray:
    """Central finite differences of the exact log-likelihood (relative step h)."""
    import copy
    g = []
    for th in theta_names(kernel):
        vals = []
        for sgn in (+1, -1):
            kk = copy.deepcopy(kernel)
            if th == "noise":
                step = h * kk.noise_var
                kk.noise_var = kk.noise_var + sgn * step
            elif th == "scale":
                step = h * kk.outputscale
                kk.outputscale = kk.outputscale + sgn * step
            else:
                ls = list(kk.lengthscale)
                step = h * ls[th[1]]
                ls[th[1]] += sgn * step
                kk.lengthscale = tuple(ls)
            vals.append(loglik_exact(grid, kk, X, y))
        g.append((vals[0] - vals[1]) / (2 * step))
    return np.array(g)


def loglik_grad_stochastic(grid, kernel, X, y, Z: np.ndarray, rtol: float, maxiter: int = 10000):
    """Same-probe stochastic log-likelihood and gradient in n-space.

    logdet by SLQ over probes Z (P x n); traces by Hutchinson with the same probes:
      tr(A^{-1} W dK W^T) ~ mean_j (W^T x_j)^T dK (W^T z_j),  tr(A^{-1}) ~ mean_j z_j^T x_j,
    with x_j = A^{-1} z_j from Alg. 1 (x0 = 0).  The mean solve z_tilde = A^{-1} y uses the same
    CG and tolerance."""
    W = w_csr(grid, X)
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    mv = ski_operator(grid, kernel, W)
    zt, it_y, _, _ = cg(mv, y, None, (rtol ** 2) * float(y @ y), maxiter)
    logdet, xs, its = slq_logdet(mv, Z, rtol, maxiter)
    L = -0.5 * (logdet + y @ zt + n * math.log(2 * math.pi))
    a = W.T @ zt
    WtZ = (W.T @ Z.T)            # m x P
    WtX = (W.T @ xs.T)           # m x P
    g = []
    for th in theta_names(kernel):
        if th == "noise":
            tr = np.mean(np.sum(Z * xs, axis=1))
            g.append(0.5 * zt @ zt - 0.5 * tr)
        else:
            dKa = kg_matvec(grid, kernel, a, th)
            dKz = kg_matvec(grid, kernel, WtZ, th)
            tr = np.mean(np.sum(WtX * dKz, axis=0))
            g.append(0.5 * a @ dKa - 0.5 * tr)
    return dict(L=float(L), grad=np.array(g), logdet=logdet, quad=float(y @ zt), iters=its,
                iters_y=it_y, a=a, v=kg_matvec(grid, kernel, a))
