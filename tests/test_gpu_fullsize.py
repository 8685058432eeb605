"""Parity at the full sizes of the benchmarked workloads (the sizes and launch shapes bench.py
times), on outputs the oracle can compute one by one, and through properties that hold at any size.

- Band / W^T y / W^T z rows at sampled grid nodes: the oracle's precompute over exactly the points
  whose cells touch those nodes (a node's row only depends on them) must equal the GPU's full-size
  rows (1e-6 relative, as the small-size tests).
- Posterior mean: every solve must converge (status OK) to its tolerance rtol, ||r|| <= rtol ||y||
  for the n-space residual r; by the identity (K W^T W + s^2 I) K W^T z = K W^T (y - r) (Claim 6),
  the m-space residual ||(K B + s^2 I) v - K W^T y|| = ||K W^T r|| must then be at most
  ||K||_2 ||W||_2 rtol ||y||, checked with the oracle's K_G and the GPU band (whose rows were checked
  above) -- a bound that uses the target tolerance, not the solver's own report.
- The sine workload (n = 1e4) is small enough for the oracle's full n-space CG.
- The serving batch: every problem of the 64 equals its single-problem solve; the smallest ones
  also match the oracle's n-space CG."""
import numpy as np
import pytest
import torch

from gpu_helpers import rel_fro
from paper_2101_11751_gb300 import synth

pytestmark = pytest.mark.gpu


def _tt(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _digits(keys, grid):
    nc = [int(grid.M[k]) - 3 for k in range(grid.d)]
    out = np.empty((grid.d, keys.size), np.int64)
    r = keys.astype(np.int64)
    for k in range(grid.d - 1, -1, -1):
        out[k] = r % nc[k]
        r //= nc[k]
    return out


def _check_sampled_rows(fk, st, X, y, grid, keys, n_nodes, seed, nprobe=0, probe_seed=0, nodes=None):
    """Oracle rows at sampled nodes (or the given d x k node array) from the points of the cells
    around them."""
    from oracle import core
    rng = np.random.default_rng(seed)
    d = grid.d
    M = [int(grid.M[k]) for k in range(d)]
    if nodes is None:
        nodes = np.stack([rng.integers(0, M[k], n_nodes) for k in range(d)])
    n_nodes = nodes.shape[1]
    dig = _digits(keys, grid)
    sel = np.zeros(keys.size, bool)
    for j in range(n_nodes):
        inside = np.ones(keys.size, bool)
        for k in range(d):
            inside &= (dig[k] >= nodes[k, j] - 3) & (dig[k] <= nodes[k, j])
        sel |= inside
    idx = np.nonzero(sel)[0]
    Xs, ys = np.ascontiguousarray(X[:, idx]), np.ascontiguousarray(y[idx])
    ref = core.precompute(grid, Xs, ys, nprobe=0)
    ex = fk.stats_export(st)
    flat = np.ravel_multi_index(tuple(nodes), tuple(M))
    gb, rb = ex["band"][:, flat], ref["band"][:, flat]
    eb, em = rel_fro(gb, rb), float(np.max(np.abs(gb - rb)) / np.max(np.abs(rb)))
    ew = rel_fro(ex["wty"][flat], ref["wty"][flat])
    print(f"rows at {n_nodes} nodes ({idx.size} points): band rel {eb:.2e} max {em:.2e}, W^T y rel {ew:.2e}")
    assert eb <= 1e-6 and em <= 1e-6
    assert ew <= 1e-6
    if nprobe:
        # W^T z over the same points: the probe signs depend on the global point index
        Z = np.stack([core.rademacher(probe_seed, p, X.shape[1])[idx] for p in range(nprobe)])
        W = core.w_csr(grid, Xs)
        wtz = (W.T @ Z.T).T
        assert rel_fro(ex["wtz"][:nprobe][:, flat], wtz[:, flat]) <= 1e-6
    return ex


def _check_mean_residual(fk, ex, grid, kern, v, rel_res, yty):
    """||(K B + s^2 I) v - K W^T y|| <= ||K|| ||W|| ||r||  (||r|| <= rel_res ||y||)."""
    from oracle import core
    v = v.double().cpu().numpy()
    Bv = core.band_matvec(grid, ex["band"], v)
    lhs = core.kg_matvec(grid, kern, Bv) + kern.noise_var * v - core.kg_matvec(grid, kern, ex["wty"])
    # ||K||_2 <= max row sum of |K| (symmetric); ||W||_2^2 = ||W^T W||_2 <= max row sum of the band
    ones = np.ones(grid.m)
    kmax = float(np.max(np.abs(core.kg_matvec(grid, kern, ones))))
    wmax = float(np.sqrt(np.max(np.abs(ex["band"]).sum(axis=0))))
    bound = kmax * wmax * rel_res * np.sqrt(yty)
    assert np.linalg.norm(lhs) <= 1.05 * bound + 1e-12 * np.linalg.norm(core.kg_matvec(grid, kern, ex["wty"])), \
        (np.linalg.norm(lhs), bound)


def test_sine_full(fk, oracle_mod):
    """c1: n = 1e4 FP64, M = 1000, rtol 1e-10 -- full precompute and mean against the oracle."""
    from oracle import core
    pr = synth.sine_1d()
    st = fk.precompute(_tt(pr.X), _tt(pr.y), pr.grid, keep_sort=True)
    ex = fk.stats_export(st)
    ref = core.precompute(pr.grid, pr.X, pr.y)
    assert rel_fro(ex["band"], ref["band"]) <= 1e-6 and rel_fro(ex["wty"], ref["wty"]) <= 1e-6
    srt = fk.stats_export_sort(st)
    np.testing.assert_array_equal(srt["perm"], ref["perm"])
    a, v, info = fk.solve(st, pr.kernel, rtol=pr.rtol, maxiter=20000, precision=fk.DOUBLE)
    _, v_ref, it_ref, _ = core.nspace_mean(pr.grid, pr.kernel, pr.X, pr.y, rtol=pr.rtol, x0_mode=1)
    assert rel_fro(v.cpu().numpy(), v_ref) <= 1e-4
    assert abs(info["iters"] - it_ref) <= max(3, 0.05 * it_ref)
    mu = fk.predict(st, v, _tt(pr.Xstar)).cpu().numpy()
    assert rel_fro(mu, core.predict(pr.grid, v_ref, pr.Xstar)) <= 1e-4


def test_gmm_full(fk, oracle_mod):
    """c2: n = 1e6 clustered 2-D, grid 128^2, Matern-5/2, rtol 1e-6."""
    pr = synth.gmm_2d()
    st = fk.precompute(_tt(pr.X), _tt(pr.y), pr.grid, keep_sort=True)
    keys = fk.stats_export_sort(st)["keys"]
    ex = _check_sampled_rows(fk, st, pr.X, pr.y, pr.grid, keys, 24, seed=1)
    a, v, info = fk.solve(st, pr.kernel, rtol=pr.rtol, maxiter=20000)
    assert info["status"] == fk.OK and info["rel_residual"] <= pr.rtol
    _check_mean_residual(fk, ex, pr.grid, pr.kernel, v, pr.rtol, ex["yty"])


def test_grf_full(fk, oracle_mod):
    """c3: n = 1e7 uniform 3-D, grid 64^3, 16 probes."""
    pr = synth.grf_3d()
    st = fk.precompute(_tt(pr.X), _tt(pr.y), pr.grid, n_probes=pr.n_probes, probe_seed=pr.probe_seed,
                       keep_sort=True)
    keys = fk.stats_export_sort(st)["keys"]
    ex = _check_sampled_rows(fk, st, pr.X, pr.y, pr.grid, keys, 12, seed=2, nprobe=2, probe_seed=pr.probe_seed)
    a, v, info = fk.solve(st, pr.kernel, rtol=1e-4, maxiter=20000)
    assert info["status"] == fk.OK and info["rel_residual"] <= 1e-4
    _check_mean_residual(fk, ex, pr.grid, pr.kernel, v, 1e-4, ex["yty"])


def test_radar_full(fk, oracle_mod):
    """c4: n = 119,548,800 radar points, grid 128 x 128 x 32, rtol 1e-5 (the benchmarked step)."""
    from oracle import core
    pr = synth.radar_3d(device="cuda")
    st = fk.precompute(_tt(pr.X), _tt(pr.y), pr.grid, keep_sort=True)
    srt = fk.stats_export_sort(st)
    keys = srt["keys"]
    # the whole cell sort, bit-exact: keys, stable permutation, segment offsets
    ref = core.cell_sort(pr.grid, pr.X, pr.y)
    np.testing.assert_array_equal(keys, ref["keys"])
    np.testing.assert_array_equal(srt["offsets"], ref["offsets"])
    np.testing.assert_array_equal(srt["perm"], ref["perm"])
    del ref
    ex = _check_sampled_rows(fk, st, pr.X, pr.y, pr.grid, keys, 16, seed=3)
    # rows at the two nodes next to the densest cell (about 2.3e5 points in that cell, 2.4e6 and
    # 2.8e6 in the cells around each node): the longest segments of the per-cell reduction
    nc = [int(pr.grid.M[k]) - 3 for k in range(3)]
    dense = np.array(np.unravel_index(int(np.argmax(np.diff(srt["offsets"]))), nc))
    _check_sampled_rows(fk, st, pr.X, pr.y, pr.grid, keys, 0, seed=0,
                        nodes=np.stack([dense + 1, np.minimum(dense + 2, np.array(nc) + 2)], axis=1))
    a, v, info = fk.solve(st, pr.kernel, rtol=pr.rtol, maxiter=60000, check_every=16)
    assert info["status"] == fk.OK and info["rel_residual"] <= pr.rtol
    _check_mean_residual(fk, ex, pr.grid, pr.kernel, v, pr.rtol, ex["yty"])


def test_batch_full(fk, oracle_mod):
    """c5: 64 uneven problems under one graph; each equals its single-problem solve, and the
    smallest match the oracle's n-space CG."""
    from oracle import core
    probs = synth.batch_2d()
    sts = fk.precompute_batched([_tt(p.X) for p in probs], [_tt(p.y) for p in probs], [p.grid for p in probs])
    a_b, v_b, info_b = fk.solve_batched(sts, [p.kernel for p in probs], rtol=1e-4, maxiter=20000)
    assert all(i["status"] == fk.OK for i in info_b)
    mus = fk.predict_batched(sts, v_b, [_tt(p.Xstar) for p in probs])
    for i, p in enumerate(probs):
        a, v, info = fk.solve(sts[i], p.kernel, rtol=1e-4, maxiter=20000)
        assert info_b[i]["iters"] == info["iters"]
        assert rel_fro(v_b[i].double().cpu().numpy(), v.double().cpu().numpy()) <= 1e-6
    # the smallest problems against the oracle: both sides solved to rtol 1e-8 (two CG runs stopped at
    # a loose rtol may differ by about that rtol, so parity is checked at a tight one)
    small = sorted(range(len(probs)), key=lambda i: probs[i].X.shape[1])[:3]
    _, v_t, info_t = fk.solve_batched([sts[i] for i in small], [probs[i].kernel for i in small], rtol=1e-8,
                                      maxiter=20000)
    mus_t = fk.predict_batched([sts[i] for i in small], v_t, [_tt(probs[i].Xstar) for i in small])
    for k, i in enumerate(small):
        p = probs[i]
        _, v_ref, _, _ = core.nspace_mean(p.grid, p.kernel, p.X.astype(np.float64), p.y.astype(np.float64),
                                          rtol=1e-8, x0_mode=1)
        assert rel_fro(v_t[k].double().cpu().numpy(), v_ref) <= 1e-4
        mu_ref = core.predict(p.grid, v_ref, p.Xstar[:, :2000].astype(np.float64))
        assert rel_fro(mus_t[k][:2000].double().cpu().numpy(), mu_ref) <= 1e-4
