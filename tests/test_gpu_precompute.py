"""GPU precompute (keys, stable cell sort, W^T W band, W^T y, probes) against the CPU oracle.

Bars: keys, permutation and segment offsets bit-exact; band and W^T y within 1e-6 relative
(Frobenius over the whole array, and max-abs relative to the largest entry); y^T y 1e-6."""
import numpy as np
import pytest
import torch

from gpu_helpers import max_rel, problem, rel_fro

pytestmark = pytest.mark.gpu

CASES = [
    # d, M, n, dtype, clustered
    (1, (3000,), 30000, np.float32, False),     # > 1 tile along the only axis (D=1 cap 2048 cells)
    (1, (1000,), 10000, np.float64, False),     # the sine workload's grid, FP64
    (2, (40, 37), 50000, np.float32, True),
    (2, (9, 600), 20000, np.float32, False),    # last axis longer than a D=2 tile
    (2, (33, 21), 7777, np.float64, False),
    (3, (12, 10, 11), 20001, np.float32, False),
    (3, (6, 5, 130), 20000, np.float32, False), # last axis longer than a D=3 tile (halo recompute)
    (3, (8, 9, 7), 5000, np.float64, True),
]


def _tt(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("d,M,n,dtype,clustered", CASES)
def test_precompute_matches_oracle(fk, oracle_mod, d, M, n, dtype, clustered):
    from oracle import core
    grid, X, y = problem(d, M, n, seed=n % 97, dtype=dtype, clustered=clustered)
    st = fk.precompute(_tt(X), _tt(y), grid, n_probes=3, probe_seed=7, keep_sort=True)
    ex = fk.stats_export(st)
    srt = fk.stats_export_sort(st)
    ref = core.precompute(grid, X, y, nprobe=3, seed=7)
    np.testing.assert_array_equal(srt["keys"], ref["keys"])
    np.testing.assert_array_equal(srt["perm"], ref["perm"])
    np.testing.assert_array_equal(srt["offsets"], ref["offsets"])
    assert rel_fro(ex["band"], ref["band"]) <= 1e-6
    assert max_rel(ex["band"], ref["band"]) <= 1e-6
    assert rel_fro(ex["wty"], ref["wty"]) <= 1e-6
    assert max_rel(ex["wty"], ref["wty"]) <= 1e-6
    assert rel_fro(ex["wtz"], ref["wtz"]) <= 1e-6
    assert ex["yty"] == pytest.approx(ref["yty"], rel=1e-6)
    np.testing.assert_allclose(ex["ztz"], [n] * 3)


def test_skewed_cell_fp32(fk, oracle_mod):
    """One cell holding 2e5 FP32 points (it spans many tiles and all warps of the per-cell
    moment reduction, and its FP32 partial sums run over the most terms) next to sparse cells:
    keys, permutation and offsets bit-exact, band and W^T y within 1e-6 of the FP64 oracle."""
    from oracle import core
    from paper_2101_11751_gb300 import synth
    rng = np.random.default_rng(17)
    grid = synth.grid_for_box([0.0] * 3, [1.0] * 3, (10, 9, 8))
    # dense cell: cell indices (3, 2, 1) -> the box [lo + (c+1) h, lo + (c+2) h) per axis
    c = np.array([3, 2, 1])
    lo = np.array(grid.lo) + (c + 1) * np.array(grid.h)
    dense = lo[:, None] + rng.uniform(0.02, 0.98, size=(3, 200000)) * np.array(grid.h)[:, None]
    sparse = rng.uniform(0.0, 1.0, size=(3, 30000))
    X = np.ascontiguousarray(np.concatenate([dense, sparse], axis=1)[:, rng.permutation(230000)].astype(np.float32))
    y = (np.sin(3 * X[0]) + X[1] * X[2] + 0.1 * rng.normal(size=X.shape[1])).astype(np.float32)
    st = fk.precompute(_tt(X), _tt(y), grid, keep_sort=True)
    ex = fk.stats_export(st)
    srt = fk.stats_export_sort(st)
    ref = core.precompute(grid, X, y)
    assert np.max(np.diff(ref["offsets"])) >= 199000
    np.testing.assert_array_equal(srt["keys"], ref["keys"])
    np.testing.assert_array_equal(srt["perm"], ref["perm"])
    np.testing.assert_array_equal(srt["offsets"], ref["offsets"])
    eb, ew = rel_fro(ex["band"], ref["band"]), rel_fro(ex["wty"], ref["wty"])
    print(f"skewed cell: band rel {eb:.2e} max {max_rel(ex['band'], ref['band']):.2e}, W^T y rel {ew:.2e}")
    assert eb <= 1e-6 and max_rel(ex["band"], ref["band"]) <= 1e-6
    assert ew <= 1e-6 and max_rel(ex["wty"], ref["wty"]) <= 1e-6


def test_sort_three_radix_passes(fk, oracle_mod):
    """More than 2^20 cells: three 7-bit digit passes; keys/permutation/offsets bit-exact."""
    from oracle import core
    grid, X, y = problem(3, (110, 105, 100), 200000, seed=3)
    st = fk.precompute(_tt(X), _tt(y), grid, keep_sort=True)
    srt = fk.stats_export_sort(st)
    ref = core.precompute(grid, X, y, want_band=False)
    assert grid.ncells > (1 << 20)
    np.testing.assert_array_equal(srt["keys"], ref["keys"])
    np.testing.assert_array_equal(srt["perm"], ref["perm"])
    np.testing.assert_array_equal(srt["offsets"], ref["offsets"])


def test_single_point_and_boundaries(fk, oracle_mod):
    """n = 1, and points exactly on s = 1 and s = M-2 of an exactly representable grid."""
    from oracle import core
    from paper_2101_11751_gb300 import synth
    grid = synth.Grid(d=2, M=(10, 12), lo=(0.0, 0.0), h=(0.25, 0.5))
    X = np.array([[0.25, 2.0, 1.0, 0.6], [0.5, 5.0, 2.75, 3.3]], dtype=np.float32)
    y = np.array([1.0, -2.0, 0.5, 3.0], dtype=np.float32)
    for k in (1, 4):
        st = fk.precompute(_tt(X[:, :k]), _tt(y[:k]), grid, keep_sort=True)
        ex = fk.stats_export(st)
        ref = core.precompute(grid, X[:, :k], y[:k])
        np.testing.assert_allclose(ex["band"], ref["band"], atol=1e-6)
        np.testing.assert_allclose(ex["wty"], ref["wty"], atol=1e-6)
        srt = fk.stats_export_sort(st)
        np.testing.assert_array_equal(srt["keys"], ref["keys"])


def test_point_errors(fk):
    from paper_2101_11751_gb300 import synth
    grid = synth.Grid(d=1, M=(10,), lo=(0.0,), h=(0.25,))
    y = _tt(np.ones(3, np.float32))
    with pytest.raises(fk.FkskiError) as e:
        fk.precompute(_tt(np.array([[0.3, 0.1, 1.0]], np.float32)), y, grid)
    assert e.value.code == fk.E_OUT_OF_GRID
    with pytest.raises(fk.FkskiError) as e:
        fk.precompute(_tt(np.array([[0.3, float("nan"), 1.0]], np.float32)), y, grid)
    assert e.value.code == fk.E_NONFINITE
    with pytest.raises(fk.FkskiError) as e:
        fk.precompute(_tt(np.array([[0.3, 0.5, 1.0]], np.float32)), _tt(np.array([1, np.inf, 0], np.float32)), grid)
    assert e.value.code == fk.E_NONFINITE
    bad = synth.Grid(d=1, M=(3,), lo=(0.0,), h=(0.25,))
    with pytest.raises(fk.FkskiError) as e:
        fk.precompute(_tt(np.array([[0.3]], np.float32)), _tt(np.ones(1, np.float32)), bad)
    assert e.value.code == fk.E_INVALID_ARG


def test_user_probes(fk, oracle_mod):
    """Caller-supplied probes Z give W^T Z and Z Z^T diagonals."""
    from oracle import core
    grid, X, y = problem(2, (20, 18), 9000, seed=5)
    Z = np.random.default_rng(1).normal(size=(5, 9000)).astype(np.float32)
    st = fk.precompute(_tt(X), _tt(y), grid, Z=_tt(Z))
    ex = fk.stats_export(st, want_band=False)
    W = core.w_csr(grid, X)
    ref = (W.T @ Z.astype(np.float64).T).T
    assert rel_fro(ex["wtz"], ref) <= 1e-6
    np.testing.assert_allclose(ex["ztz"], np.sum(Z.astype(np.float64) ** 2, axis=1), rtol=1e-6)


def test_deterministic(fk):
    grid, X, y = problem(3, (10, 11, 9), 30000, seed=9)
    st1 = fk.precompute(_tt(X), _tt(y), grid, n_probes=2)
    st2 = fk.precompute(_tt(X), _tt(y), grid, n_probes=2)
    a, b = fk.stats_export(st1), fk.stats_export(st2)
    for k in ("band", "wty", "wtz"):
        np.testing.assert_array_equal(a[k], b[k])


def test_save_load_roundtrip(fk, tmp_path):
    grid, X, y = problem(2, (16, 15), 4000, seed=2)
    st = fk.precompute(_tt(X), _tt(y), grid, n_probes=2)
    p = str(tmp_path / "stats.bin")
    fk.stats_save(st, p)
    st2 = fk.stats_load(p, grid)
    a, b = fk.stats_export(st), fk.stats_export(st2)
    for k in ("band", "wty", "wtz"):
        np.testing.assert_array_equal(a[k], b[k])
    assert st2.info()["n"] == 4000


def test_band_mvm_matches_oracle(fk, oracle_mod):
    from oracle import core
    grid, X, y = problem(3, (9, 8, 10), 6000, seed=4)
    st = fk.precompute(_tt(X), _tt(y), grid)
    ref = core.precompute(grid, X, y)
    V = np.random.default_rng(0).normal(size=(3, grid.m)).astype(np.float32)
    U = fk.band_mvm(st, _tt(V)).cpu().numpy()
    Uref = core.band_matvec(grid, ref["band"], V.astype(np.float64).T).T
    assert rel_fro(U, Uref) <= 2e-6


@pytest.mark.parametrize("d,M", [(1, (400,)), (2, (36, 44)), (3, (12, 10, 16)), (3, (9, 8, 10))])
@pytest.mark.parametrize("R", [1, 2, 5, 9])
def test_band_mvm_paths(fk, oracle_mod, d, M, R):
    """Banded W^T W products on every kernel path: the symmetric half-band form (one FP32 rhs,
    M_last a multiple of 4), the vectorised full-band form (several rhs, groups of <= 8), the
    generic form (M_last not a multiple of 4) and FP64 vectors."""
    from oracle import core
    grid, X, y = problem(d, M, 20000, seed=7)
    st = fk.precompute(_tt(X), _tt(y), grid)
    ref = core.precompute(grid, X, y)
    V = np.random.default_rng(R).normal(size=(R, grid.m))
    Uref = core.band_matvec(grid, ref["band"], V.T).T
    U32 = fk.band_mvm(st, _tt(V.astype(np.float32))).cpu().numpy()
    assert rel_fro(U32, Uref) <= 2e-6
    U64 = fk.band_mvm(st, _tt(V)).cpu().numpy()
    assert rel_fro(U64, Uref) <= 2e-6  # FP32 band values (statistics of FP32 inputs)
    # one rhs alone (half band when eligible) equals the same rhs inside the batch
    u0 = fk.band_mvm(st, _tt(V[:1].astype(np.float32))).cpu().numpy()
    assert rel_fro(u0, U32[:1]) <= 1e-6


@pytest.mark.parametrize("d,M,R", [(1, (400,), 1), (2, (36, 44), 1), (3, (12, 10, 16), 1), (3, (9, 8, 10), 1),
                                   (3, (48, 44, 40), 1), (3, (12, 10, 16), 3)])
def test_band_mvm_double_float(fk, oracle_mod, d, M, R):
    """The MIXED solver's band product: double-float (hi, lo) vectors against the stored FP32 band,
    on the half-band path (one rhs, M_last a multiple of 4; the many-tile grid included), the
    generic path and several rhs.  Each entry is held to the double-float accumulation bound,
    |u - (W^T W) x| <= 2^-40 sum_j |b_ij x_j| + 2^-47 |u|, against the exact product of the band
    values the GPU holds (exported, FP32 values) with the exact values hi + lo it was given."""
    from oracle import core
    grid, X, y = problem(d, M, 20000, seed=13)
    st = fk.precompute(_tt(X), _tt(y), grid)
    band = fk.stats_export(st)["band"]
    v = np.random.default_rng(R + d).normal(size=(R, grid.m))
    hi = v.astype(np.float32)
    lo = (v - hi.astype(np.float64)).astype(np.float32)
    xdf = np.stack([hi, lo], axis=-1)
    x = hi.astype(np.float64) + lo.astype(np.float64)
    out = fk.band_mvm(st, _tt(xdf if R > 1 else xdf[0]), double_float=True).cpu().numpy().reshape(R, grid.m, 2)
    u = out[..., 0].astype(np.float64) + out[..., 1].astype(np.float64)
    uref = core.band_matvec(grid, band, x.T).T
    scale = core.band_matvec(grid, np.abs(band), np.abs(x).T).T
    err = np.abs(u - uref)
    assert np.all(err <= 2.0 ** -40 * scale + 2.0 ** -47 * np.abs(uref)), float(np.max(err / np.maximum(scale, 1e-300)))
    # normalised pairs: hi = fl(hi + lo)
    np.testing.assert_array_equal(out[..., 0], (out[..., 0] + out[..., 1]).astype(np.float32))


def test_band_mvm_half_many_tiles(fk, oracle_mod):
    """The symmetric half-band product on a grid with more row tiles than SMs, so that each
    persistent CTA walks several tiles and the mirrored windows (up to ~10 tiles back) cross tile
    and CTA boundaries; one FP32 rhs, compared with the oracle's band product."""
    from oracle import core
    grid, X, y = problem(3, (48, 44, 40), 20000, seed=11)
    st = fk.precompute(_tt(X), _tt(y), grid)
    ref = core.precompute(grid, X, y)
    v = np.random.default_rng(5).normal(size=(1, grid.m))
    uref = core.band_matvec(grid, ref["band"], v.T).T
    u = fk.band_mvm(st, _tt(v.astype(np.float32))).cpu().numpy()
    assert rel_fro(u, uref) <= 2e-6
    # repeated launches give identical bits (fixed summation order)
    u2 = fk.band_mvm(st, _tt(v.astype(np.float32))).cpu().numpy()
    np.testing.assert_array_equal(u, u2)


def test_pinned_host_inputs(fk, oracle_mod):
    """X and y in page-locked host memory, read in place by the key kernel, give the same
    statistics as device copies, bit for bit.  Pageable host memory is rejected by the binding;
    the library rejects memory the CUDA runtime reports without a device mapping before any
    device work (a platform that maps pageable memory must then give the same statistics)."""
    import ctypes
    grid, X, y = problem(3, (12, 10, 16), 30000, seed=13)
    st_d = fk.precompute(_tt(X), _tt(y), grid, keep_sort=True)
    Xh, yh = torch.from_numpy(X).pin_memory(), torch.from_numpy(y).pin_memory()
    st_h = fk.precompute(Xh, yh, grid, keep_sort=True)
    a, b = fk.stats_export(st_d), fk.stats_export(st_h)
    for k in ("band", "wty"):
        np.testing.assert_array_equal(a[k], b[k])
    assert a["yty"] == b["yty"]
    np.testing.assert_array_equal(fk.stats_export_sort(st_d)["perm"], fk.stats_export_sort(st_h)["perm"])
    with pytest.raises(ValueError):
        fk.precompute(torch.from_numpy(X), torch.from_numpy(y), grid)
    h = ctypes.c_void_p()
    code = fk.load().fkski_precompute(ctypes.byref(fk.c_grid(grid)), ctypes.c_void_p(X.ctypes.data),
                                      ctypes.c_void_p(y.ctypes.data), None, X.shape[1], fk.F32,
                                      ctypes.byref(fk.opts()), ctypes.byref(h), None)
    if code == fk.OK:
        st_p = fk.Stats(h, grid, X.shape[1])
        np.testing.assert_array_equal(fk.stats_export(st_p)["band"], a["band"])
    else:
        assert code == fk.E_INVALID_ARG and not h.value
