"""Measured error of every output against the FP64 oracle, per precision mode (run with -s to see
the table).  One 3-D problem with FP32 points (uniform, 1.5e5 points on a 20 x 18 x 16 grid, RBF
ARD, 4 probes): cell keys and permutation, band, W^T y, the posterior mean v on the grid and
mu at test points (rtol 1e-8), log-likelihood L and gradient (same probes, rtol 1e-6).  The
asserts are the parity bars: keys exact, statistics 1e-6, mean 1e-4, L and gradient 1e-4 (the
FP32 mode's gradient is not asserted: its probe solves stall at its attainable accuracy)."""
import numpy as np
import pytest
import torch

from gpu_helpers import max_rel, problem, rel_fro
from paper_2101_11751_gb300 import synth

pytestmark = pytest.mark.gpu


def _tt(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_precision_report(fk, oracle_mod):
    from oracle import core
    d, M, n, T, seed = 3, (16, 15, 14), 60000, 4, 7
    grid, X, y = problem(d, M, n, seed=91, dtype=np.float32)
    kern = synth.Kernel(synth.RBF, (0.25, 0.2, 0.3), 1.0, 0.05)
    st = fk.precompute(_tt(X), _tt(y), grid, n_probes=T, probe_seed=seed, keep_sort=True)
    ex = fk.stats_export(st)
    srt = fk.stats_export_sort(st)
    ref = core.precompute(grid, X, y, nprobe=T, seed=seed)
    rows = []
    keys_ok = np.array_equal(srt["keys"], ref["keys"]) and np.array_equal(srt["perm"], ref["perm"])
    rows.append(("keys, permutation, offsets", "exact" if keys_ok else "DIFFER"))
    rows.append(("band W^T W (rel Frobenius / max)", f"{rel_fro(ex['band'], ref['band']):.2e} / "
                                                      f"{max_rel(ex['band'], ref['band']):.2e}"))
    rows.append(("W^T y", f"{rel_fro(ex['wty'], ref['wty']):.2e}"))
    rows.append(("W^T z (probes)", f"{rel_fro(ex['wtz'], ref['wtz']):.2e}"))
    assert keys_ok
    assert rel_fro(ex["band"], ref["band"]) <= 1e-6 and rel_fro(ex["wty"], ref["wty"]) <= 1e-6
    _, v_ref, it_ref, _ = core.nspace_mean(grid, kern, X, y, rtol=1e-8, x0_mode=1)
    Xs = np.random.default_rng(5).uniform(0, 1, size=(d, 2000)).astype(np.float32)
    mu_ref = core.predict(grid, v_ref, Xs)
    Z = np.stack([core.rademacher(seed, p, n) for p in range(T)])
    gref = core.loglik_grad_stochastic(grid, kern, X, y, Z, rtol=1e-6)
    names = {fk.MIXED: "MIXED", fk.DOUBLE: "DOUBLE", fk.FP32: "FP32"}
    for prec in (fk.MIXED, fk.DOUBLE, fk.FP32):
        a, v, info = fk.solve(st, kern, rtol=1e-8, maxiter=20000, precision=prec, allow_not_converged=True)
        ev = rel_fro(v.double().cpu().numpy(), v_ref)
        mu = fk.predict(st, v, _tt(Xs)).double().cpu().numpy()
        emu = rel_fro(mu, mu_ref)
        rows.append((f"{names[prec]}: mean v (iters {info['iters']}, oracle {it_ref}, status {info['status']})",
                     f"{ev:.2e}"))
        rows.append((f"{names[prec]}: mu(x*)", f"{emu:.2e}"))
        if prec != fk.FP32:
            assert ev <= 1e-4 and emu <= 1e-4
        L, g, ginfo = fk.grad(st, kern, rtol=1e-6, maxiter=20000, precision=prec, allow_not_converged=True)
        eL = abs(L - gref["L"]) / abs(gref["L"])
        eg = float(np.max(np.abs(np.array(g) - gref["grad"])) / np.max(np.abs(gref["grad"])))
        rows.append((f"{names[prec]}: L / gradient (max rel to largest)", f"{eL:.2e} / {eg:.2e}"))
        if prec != fk.FP32:
            assert eL <= 1e-4 and eg <= 1e-4
    print("\nprecision report (3-D, n = 6e4 FP32 points, m = 3360):")
    for k, v in rows:
        print(f"  {k:58s} {v}")
