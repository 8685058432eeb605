"""Pins for the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks an oracle function against something other than itself: hand-evaluated
closed forms (tests/golden), exact rational arithmetic, brute-force dense constructions,
the paper's identities (Theorem 1, Claims 2/6/7, Fact 2, Prop. 1) and finite differences.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2101_11751_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ----------------------------------------------------------------- interpolation weights

def test_keys_kernel_golden(oracle_mod):
    from oracle import core
    for s, u in _load("keys_kernel.txt"):
        assert core.keys_u(float(s)) == pytest.approx(float(u), abs=1e-15)


def test_keys_weights_golden(oracle_mod):
    from oracle import core
    for row in _load("keys_weights.txt"):
        t = float(row[0])
        w = core.keys_weights(t)
        np.testing.assert_allclose(w, [float(v) for v in row[1:]], atol=1e-15)


@pytest.mark.parametrize("t", np.linspace(0.0, 1.0, 23))
def test_keys_weights_invariants(oracle_mod, t):
    """Partition of unity; linear and quadratic functions reproduced exactly; cubic not."""
    from oracle import core
    w = core.keys_weights(t)
    nodes = np.arange(4) - 1.0
    assert w.sum() == pytest.approx(1.0, abs=1e-14)
    assert (w * nodes).sum() == pytest.approx(t, abs=1e-14)
    assert (w * nodes ** 2).sum() == pytest.approx(t * t, abs=1e-14)
    cubic_err = (w * nodes ** 3).sum() - t ** 3
    if 0.05 < t < 0.95 and abs(t - 0.5) > 0.05:   # the error vanishes at t=0, 1/2, 1 by symmetry
        assert abs(cubic_err) > 1e-4


def test_keys_continuity_across_cells(oracle_mod):
    """t = 1 in cell c equals t = 0 in cell c+1: the basis functions are continuous (Fig. 1)."""
    from oracle import core
    np.testing.assert_allclose(core.keys_weights(1.0)[1:], core.keys_weights(0.0)[:3], atol=1e-15)


# ----------------------------------------------------------------- cell keys

def test_cell_key_exact_floor(oracle_mod):
    """The float-pair cell index equals floor((x - lo)/h) computed in exact rationals."""
    from oracle import core
    rng = np.random.default_rng(5)
    cases = 0
    for trial in range(40):
        M = int(rng.integers(8, 600))
        h = float(rng.uniform(1e-3, 3.0))
        lo = float(rng.uniform(-50, 50))
        xs = (lo + h * rng.uniform(1.0, M - 2.0, 200)).astype(np.float32)
        for x in xs:
            s_exact = (Fraction(float(x)) - Fraction(lo)) / Fraction(h)
            if not (1 <= s_exact <= M - 2):
                continue
            fl = math.floor(s_exact)
            if abs(s_exact - round(s_exact)) < Fraction(1, 10 ** 9):
                continue
            st, c, t32, t64 = core.cell_key_f32(float(x), lo, h, M)
            assert st == 0
            assert c == min(max(fl, 1), M - 3)
            t_exact = float(s_exact - c)
            assert abs(t32 - t_exact) <= 2.0 ** -22
            cases += 1
    assert cases > 7000


def test_cell_key_boundaries(oracle_mod):
    """Exactly representable grid: s = 1 and s = M-2 are inside, just outside is rejected."""
    from oracle import core
    M, lo, h = 10, 0.0, 0.25
    st, c, t32, _ = core.cell_key_f32(0.25, lo, h, M)          # s = 1
    assert (st, c, t32) == (0, 1, 0.0)
    st, c, t32, _ = core.cell_key_f32(2.0, lo, h, M)           # s = 8 = M - 2
    assert (st, c, t32) == (0, M - 3, 1.0)
    st, *_ = core.cell_key_f32(float(np.nextafter(np.float32(0.25), np.float32(0))), lo, h, M)
    assert st == core.OR_E_OUT_OF_GRID
    st, *_ = core.cell_key_f32(float(np.nextafter(np.float32(2.0), np.float32(3))), lo, h, M)
    assert st == core.OR_E_OUT_OF_GRID
    st, *_ = core.cell_key_f32(float("nan"), lo, h, M)
    assert st == core.OR_E_NONFINITE


# ----------------------------------------------------------------- W, W^T W, W^T y (Sec. 3.1)

def _dense_W_bruteforce(grid, X):
    """W[i, j] = prod_k u((x_ik - g_jk) / h_k) straight from Keys' kernel on node distances."""
    from oracle import core
    P = core.grid_points(grid)
    Xd = X.astype(np.float64).T
    W = np.ones((Xd.shape[0], P.shape[0]))
    u = np.vectorize(core.keys_u)
    for k in range(grid.d):
        W *= u((Xd[:, None, k] - P[None, :, k]) / grid.h[k])
    return W


def _tiny(d, n=60, seed=0, dtype=np.float64):
    rng = np.random.default_rng(seed)
    M = {1: (13,), 2: (7, 9), 3: (6, 5, 7)}[d]
    grid = synth.grid_for_box([0.0] * d, [1.0] * d, M)
    X = rng.uniform(0, 1, size=(d, n)).astype(dtype)
    y = rng.normal(size=n).astype(dtype)
    return grid, X, y


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_precompute_bruteforce(oracle_mod, d, dtype):
    from oracle import core
    grid, X, y = _tiny(d, dtype=dtype)
    st = core.precompute(grid, X, y, nprobe=2, seed=3)
    W = _dense_W_bruteforce(grid, X)
    np.testing.assert_allclose(core.w_csr(grid, X).toarray(), W, atol=1e-6 if dtype == np.float32 else 1e-12)
    WtW = core.band_to_dense(grid, st["band"])
    atol = 1e-5 if dtype == np.float32 else 1e-11
    np.testing.assert_allclose(WtW, W.T @ W, atol=atol)
    np.testing.assert_allclose(st["wty"], W.T @ y.astype(np.float64), atol=atol)
    assert st["yty"] == pytest.approx(float(y.astype(np.float64) @ y.astype(np.float64)), rel=1e-12)
    for p in range(2):
        z = core.rademacher(3, p, X.shape[1])
        np.testing.assert_allclose(st["wtz"][p], W.T @ z, atol=atol)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_band_structure_claim2(oracle_mod, d):
    """Claim 2: at most 7^d nonzeros per row (offsets within +-3); symmetric; PSD;
    rows of W sum to one so 1^T W^T W 1 = n and 1^T W^T y = sum(y); trace = sum_i ||w_i||^2."""
    from oracle import core
    grid, X, y = _tiny(d, n=400, seed=1)
    st = core.precompute(grid, X, y)
    A = core.band_to_dense(grid, st["band"])
    assert np.count_nonzero(np.abs(A) > 0, axis=1).max() <= 7 ** d
    np.testing.assert_allclose(A, A.T, atol=1e-13)
    assert np.linalg.eigvalsh(A).min() > -1e-10
    assert A.sum() == pytest.approx(X.shape[1], rel=1e-12)
    assert st["wty"].sum() == pytest.approx(y.sum(), rel=1e-10, abs=1e-10)
    W = core.w_csr(grid, X)
    assert np.trace(A) == pytest.approx(float(W.multiply(W).sum()), rel=1e-12)
    # every entry of the dense W^T W outside the band is zero
    full = (W.T @ W).toarray()
    np.testing.assert_allclose(full, A, atol=1e-12)


def test_stable_sort_and_offsets(oracle_mod):
    from oracle import core
    grid, X, y = _tiny(2, n=3000, seed=2, dtype=np.float32)
    st = core.precompute(grid, X, y, want_band=False)
    k = st["keys"]
    perm = st["perm"]
    assert sorted(perm.tolist()) == list(range(len(k)))
    ks = k[perm]
    assert np.all(np.diff(ks.astype(np.int64)) >= 0)
    same = np.diff(ks.astype(np.int64)) == 0
    assert np.all(np.diff(perm)[same] > 0)
    off = st["offsets"]
    np.testing.assert_array_equal(off, np.searchsorted(ks, np.arange(grid.ncells + 1), side="left"))


def test_rademacher_splitmix_golden(oracle_mod):
    from oracle import core
    rows = _load("splitmix64.txt")
    for kstr, hexv in rows:
        k = int(kstr)
        expect = -1.0 if (int(hexv, 16) >> 63) else 1.0
        assert core.rademacher(0, 0, k)[k - 1] == expect
    z = core.rademacher(11, 3, 100000)
    assert set(np.unique(z)) == {-1.0, 1.0}
    assert abs(z.mean()) < 0.02


# ----------------------------------------------------------------- K_G (Sec. 2.2)

def test_kernel_values_golden(oracle_mod):
    """The kernel conventions by number: the RBF's 1/2 inside the exponent, the scale factor,
    ARD per-axis lengthscales, the Matern-5/2 polynomial, and the lengthscale derivative
    (tests/golden/kernel_values.txt, closed forms evaluated independently)."""
    from oracle import core
    for kind, s, ell, off, val, *_ in _load("kernel_values.txt"):
        ell_v = tuple(float(v) for v in ell.split(","))
        diff = np.array([[float(v) for v in off.split(",")]])
        ktype = synth.MATERN52 if kind == "matern52" else synth.RBF
        kern = synth.Kernel(ktype, ell_v, float(s), 1.0)
        if kind == "d_l0":
            got = core.kernel_dvalue(kern, diff, ("ell", 0))[0]
        else:
            got = core.kernel_value(kern, diff)[0]
        assert got == pytest.approx(float(val), rel=1e-14), (kind, s, ell, off)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_kg_kronecker_equals_dense(oracle_mod, d):
    from oracle import core
    grid, _, _ = _tiny(d)
    kern = synth.Kernel(synth.RBF, (0.2, 0.3, 0.25)[:d], 1.7, 0.1)
    rng = np.random.default_rng(0)
    V = rng.normal(size=(grid.m, 3))
    K = core.kg_dense(grid, kern)
    np.testing.assert_allclose(K, K.T, atol=0)
    np.testing.assert_allclose(core.kg_matvec(grid, kern, V), K @ V, rtol=1e-12, atol=1e-12)
    for th in [("ell", k) for k in range(d)] + ["scale"]:
        np.testing.assert_allclose(core.kg_matvec(grid, kern, V, th), core.kg_dense(grid, kern, th) @ V,
                                   rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("d", [1, 2])
def test_kg_matern_fft_equals_dense(oracle_mod, d):
    from oracle import core
    grid, _, _ = _tiny(d)
    kern = synth.Kernel(synth.MATERN52, (0.2, 0.35)[:d], 1.3, 0.1)
    rng = np.random.default_rng(1)
    V = rng.normal(size=(grid.m, 2))
    np.testing.assert_allclose(core.kg_matvec(grid, kern, V, method="fft"), core.kg_dense(grid, kern) @ V,
                               rtol=1e-11, atol=1e-11)
    for th in [("ell", 0), "scale"]:
        np.testing.assert_allclose(core.kg_matvec(grid, kern, V, th, method="fft"),
                                   core.kg_dense(grid, kern, th) @ V, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("ktype", [0, 1])
def test_kernel_derivative_fd(oracle_mod, ktype):
    from oracle import core
    import copy
    kern = synth.Kernel(ktype, (0.3, 0.2), 1.5, 0.1)
    diff = np.random.default_rng(3).normal(scale=0.3, size=(50, 2))
    for k in range(2):
        e = 1e-6
        kp, km = copy.deepcopy(kern), copy.deepcopy(kern)
        kp.lengthscale = tuple(v + (e if i == k else 0) for i, v in enumerate(kern.lengthscale))
        km.lengthscale = tuple(v - (e if i == k else 0) for i, v in enumerate(kern.lengthscale))
        fd = (core.kernel_value(kp, diff) - core.kernel_value(km, diff)) / (2 * e)
        np.testing.assert_allclose(core.kernel_dvalue(kern, diff, ("ell", k)), fd, rtol=1e-6, atol=1e-9)
    # Matern-5/2 closed form at r = 1: s (1 + sqrt5 + 5/3) e^{-sqrt5}
    if ktype == 1:
        k1 = synth.Kernel(1, (1.0,), 2.0, 0.1)
        assert core.kernel_value(k1, np.array([[1.0]]))[0] == pytest.approx(
            2.0 * (1 + math.sqrt(5) + 5 / 3) * math.exp(-math.sqrt(5)), rel=1e-15)


# ----------------------------------------------------------------- CG and the paper's identities

def test_cg_matches_dense_solve(oracle_mod):
    from oracle import core
    rng = np.random.default_rng(4)
    B = rng.normal(size=(40, 40))
    A = B @ B.T + 0.5 * np.eye(40)
    b = rng.normal(size=40)
    x, it, al, be = core.cg(lambda v: A @ v, b, None, 1e-28 * (b @ b), 500)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-10)
    assert it <= 80


@pytest.mark.parametrize("d,ktype", [(1, 0), (2, 0), (2, 1), (3, 0)])
def test_theorem1_ski_equals_gsgp(oracle_mod, d, ktype):
    """Theorem 1 / Claims 6-7 / Fact 2: m-space GSGP mean, covariance and log-likelihood equal
    the n-space SKI expressions of Def. 1."""
    from oracle import core
    grid, X, y = _tiny(d, n=90, seed=7)
    kern = synth.Kernel(ktype, (0.3, 0.25, 0.35)[:d], 1.2, 0.05)
    Xs = np.random.default_rng(8).uniform(0, 1, size=(d, 17))
    a = core.ski_inference_dense(grid, kern, X, y, Xs)
    b = core.gsgp_inference_dense(grid, kern, X, y, Xs)
    np.testing.assert_allclose(a["mean"], b["mean"], rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(a["cov"], b["cov"], rtol=1e-8, atol=1e-10)
    assert a["ll"] == pytest.approx(b["ll"], rel=1e-10)
    n, m = X.shape[1], grid.m
    assert a["logdet"] == pytest.approx(b["logdetB"] + (n - m) * math.log(kern.noise_var), rel=1e-10)


@pytest.mark.parametrize("d", [1, 2])
def test_nspace_cov_matches_dense(oracle_mod, d):
    """The CG covariance oracle equals the dense Def. 1 covariance (pinned to Fact 2 by Theorem 1
    above) at a tight tolerance, is symmetric, and has a non-negative diagonal no larger than the
    prior variance w^T K w."""
    from oracle import core
    grid, X, y = _tiny(d, n=80, seed=9)
    kern = synth.Kernel(synth.RBF, (0.3, 0.25)[:d], 1.1, 0.04)
    Xs = np.random.default_rng(10).uniform(0, 1, size=(d, 9))
    cov, _ = core.nspace_cov(grid, kern, X, Xs, rtol=1e-13)
    ref = core.ski_inference_dense(grid, kern, X, y, Xs)["cov"]
    np.testing.assert_allclose(cov, ref, rtol=1e-7, atol=1e-9 * np.abs(ref).max())
    np.testing.assert_allclose(cov, cov.T, rtol=1e-7, atol=1e-9 * np.abs(ref).max())
    Ws = core.w_csr(grid, Xs).toarray()
    prior = np.einsum("ij,ij->i", Ws, (core.kg_dense(grid, kern) @ Ws.T).T)
    assert np.all(np.diag(cov) >= -1e-12) and np.all(np.diag(cov) <= prior + 1e-12)


def test_lanczos_lowrank_cov_exact_at_full_rank(oracle_mod):
    """Lanczos with full reorthogonalisation: Q orthonormal, T symmetric tridiagonal and
    Q^T A Q = T; run until the Krylov space of y is invariant (it then contains span(W), as A
    acts as sigma^2 on the complement), the low-rank covariance equals the exact one."""
    from oracle import core
    grid, X, y = _tiny(2, n=70, seed=12)
    kern = synth.Kernel(synth.RBF, (0.3, 0.35), 1.0, 0.05)
    W = core.w_csr(grid, X)
    mv = core.ski_operator(grid, kern, W)
    Q, T = core.lanczos(mv, y.astype(np.float64), 12)
    np.testing.assert_allclose(Q.T @ Q, np.eye(Q.shape[1]), atol=1e-10)
    AQ = np.stack([mv(Q[:, i]) for i in range(Q.shape[1])], axis=1)
    np.testing.assert_allclose(Q.T @ AQ, T, atol=1e-9 * np.abs(T).max())
    assert np.all(np.abs(np.triu(T, 2)) == 0) and np.allclose(T, T.T)
    Xs = np.random.default_rng(13).uniform(0, 1, size=(2, 11))
    cov, Tf = core.lowrank_cov(grid, kern, X, y, Xs, k=X.shape[1])
    assert Tf.shape[0] <= grid.m + 1  # invariant Krylov space reached
    ref = core.ski_inference_dense(grid, kern, X, y, Xs)["cov"]
    np.testing.assert_allclose(cov, ref, rtol=1e-6, atol=1e-8 * np.abs(ref).max())
    # few steps: a partial correction, between the prior and the exact covariance on the diagonal
    cov5, _ = core.lowrank_cov(grid, kern, X, y, Xs, k=5)
    prior = np.diag(core.w_csr(grid, Xs).toarray() @ core.kg_dense(grid, kern) @ core.w_csr(grid, Xs).toarray().T)
    assert np.all(np.diag(cov5) <= prior + 1e-12) and np.all(np.diag(cov5) >= np.diag(ref) - 1e-9)


def test_slq_lanczos_unit_probes_exact(oracle_mod):
    """SLQ by Lanczos with full reorthogonalisation: probes sqrt(n) e_i run to an invariant
    Krylov space give the exact log-determinant (Gauss quadrature is exact there); a few Rademacher
    probes land near it."""
    from oracle import core
    grid, X, y = _tiny(2, n=50, seed=14)
    kern = synth.Kernel(synth.RBF, (0.3, 0.3), 1.0, 0.1)
    W = core.w_csr(grid, X)
    mv = core.ski_operator(grid, kern, W)
    n = X.shape[1]
    exact = core.ski_inference_dense(grid, kern, X, y, X[:, :2])["logdet"]
    est, terms = core.slq_logdet_lanczos(mv, math.sqrt(n) * np.eye(n), k=n)
    assert est == pytest.approx(exact, rel=1e-9)
    Z = np.stack([core.rademacher(3, p, n) for p in range(64)])
    est64, _ = core.slq_logdet_lanczos(mv, Z, k=30)
    assert est64 == pytest.approx(exact, rel=0.05)


def test_nspace_cg_mean_matches_dense(oracle_mod):
    from oracle import core
    grid, X, y = _tiny(2, n=150, seed=9)
    kern = synth.Kernel(0, (0.3, 0.25), 1.0, 0.05)
    Xs = np.random.default_rng(1).uniform(0, 1, size=(2, 11))
    ref = core.ski_inference_dense(grid, kern, X, y, Xs)
    for mode in (0, 1):
        a, v, it, _ = core.nspace_mean(grid, kern, X, y, rtol=1e-12, x0_mode=mode)
        np.testing.assert_allclose(core.predict(grid, v, Xs), ref["mean"], rtol=1e-8, atol=1e-9)


def _efcg_simplified(grid, kern, band, wty, eps, maxiter):
    """Alg. 5 (simplified EFCG) written from its invariants, for the Prop. 1 pin."""
    from oracle import core
    s2 = kern.noise_var

    def B(x):
        u = core.band_matvec(grid, band, x)
        return core.kg_matvec(grid, kern, u) + s2 * x, u
    r = -core.kg_matvec(grid, kern, wty) / s2
    xd = np.zeros_like(r)
    v, u = B(r)
    z, s = v.copy(), u.copy()
    gam = u @ r
    it = 0
    for _ in range(maxiter):
        alpha = gam / (s @ z)
        xd = xd + alpha * s
        r = r - alpha * z
        it += 1
        v, u = B(r)
        gnew = u @ r
        if gnew <= eps:
            break
        beta = gnew / gam
        s = u + beta * s
        z = v + beta * z
        gam = gnew
    return xd + wty / s2, it


def test_prop1_factorized_cg_equals_cg(oracle_mod):
    """Prop. 1: the factorized recurrences (Alg. 5 with x0 = y/sigma^2) give the same W^T x as
    n-space CG (Alg. 1) from the same start, and iteration counts that differ only by rounding."""
    from oracle import core
    grid, X, y = _tiny(2, n=300, seed=10)
    kern = synth.Kernel(0, (0.3, 0.25), 1.0, 0.02)
    st = core.precompute(grid, X, y)
    eps = (1e-9 ** 2) * st["yty"]
    a_f, it_f = _efcg_simplified(grid, kern, st["band"], st["wty"], eps, 2000)
    a_n, v_n, it_n, _ = core.nspace_mean(grid, kern, X, y, rtol=1e-9, x0_mode=1)
    assert np.linalg.norm(a_f - a_n) <= 1e-7 * np.linalg.norm(a_n)
    # App. C.2 (Fig. 5): counts are "close", differing only through finite precision
    assert abs(it_f - it_n) <= max(3, 0.05 * it_n)


# ----------------------------------------------------------------- log-likelihood and gradient

def test_slq_unit_probes_exact(oracle_mod):
    """With the scaled unit vectors sqrt(n) e_i as probes (so that E[z z^T] = I holds for a
    uniformly drawn probe) and Lanczos run to convergence, SLQ equals the exact log-det."""
    from oracle import core
    grid, X, y = _tiny(1, n=40, seed=11)
    kern = synth.Kernel(0, (0.2,), 1.0, 0.1)
    W, K, A = core.dense_system(grid, kern, X)
    est, _, _ = core.slq_logdet(lambda v: A @ v, math.sqrt(40) * np.eye(40), rtol=1e-13)
    assert est == pytest.approx(np.linalg.slogdet(A)[1], rel=1e-9)


@pytest.mark.parametrize("ktype", [0, 1])
def test_grad_exact_matches_fd(oracle_mod, ktype):
    from oracle import core
    grid, X, y = _tiny(2, n=70, seed=12)
    kern = synth.Kernel(ktype, (0.3, 0.25), 1.3, 0.05)
    np.testing.assert_allclose(core.grad_exact(grid, kern, X, y), core.grad_fd(grid, kern, X, y),
                               rtol=1e-6, atol=1e-7)


def test_stochastic_with_unit_probes_is_exact(oracle_mod):
    from oracle import core
    grid, X, y = _tiny(2, n=50, seed=13)
    kern = synth.Kernel(0, (0.3, 0.25), 1.3, 0.05)
    res = core.loglik_grad_stochastic(grid, kern, X, y, math.sqrt(50) * np.eye(50), rtol=1e-13)
    assert res["L"] == pytest.approx(core.loglik_exact(grid, kern, X, y), rel=1e-9)
    np.testing.assert_allclose(res["grad"], core.grad_exact(grid, kern, X, y), rtol=1e-7, atol=1e-9)
