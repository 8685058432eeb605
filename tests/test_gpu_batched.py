"""Batches of independent, uneven problems (fkski_*_batched) against the single-problem calls and
the oracle.

Per problem a batch runs the same kernels in the same order as the single-problem call, so the
bar against it is equality of iterations and outputs to 1e-6 relative (FP32 values); one small
problem is also checked against the oracle's n-space mean (1e-4, as for fkski_solve)."""
import numpy as np
import pytest
import torch

from gpu_helpers import rel_fro
from paper_2101_11751_gb300 import synth

pytestmark = pytest.mark.gpu


def _tt(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _batch(P=6, n_hi=2e5, n_test=5000):
    return synth.batch_2d(n_problems=P, seed=1000, n_lo=1e4, n_hi=n_hi, n_test=n_test, sides=(32, 64))


@pytest.mark.parametrize("x0_mode", [1, 0])
def test_batched_equals_single(fk, x0_mode):
    probs = _batch()
    Xs = [_tt(p.X) for p in probs]
    ys = [_tt(p.y) for p in probs]
    sts = fk.precompute_batched(Xs, ys, [p.grid for p in probs])
    kernels = [p.kernel for p in probs]
    a_b, v_b, info_b = fk.solve_batched(sts, kernels, rtol=1e-4, maxiter=3000, x0_mode=x0_mode)
    mus = fk.predict_batched(sts, v_b, [_tt(p.Xstar) for p in probs])
    for i, p in enumerate(probs):
        st = fk.precompute(Xs[i], ys[i], p.grid)
        a, v, info = fk.solve(st, p.kernel, rtol=1e-4, maxiter=3000, x0_mode=x0_mode)
        assert info_b[i]["iters"] == info["iters"], (i, info_b[i], info)
        assert rel_fro(v_b[i].double().cpu().numpy(), v.double().cpu().numpy()) <= 1e-6
        assert rel_fro(a_b[i].double().cpu().numpy(), a.double().cpu().numpy()) <= 1e-6
        mu = fk.predict(st, v, _tt(p.Xstar))
        assert rel_fro(mus[i].double().cpu().numpy(), mu.double().cpu().numpy()) <= 1e-6


def test_batched_against_oracle(fk, oracle_mod):
    from oracle import core
    probs = synth.batch_2d(n_problems=3, seed=2000, n_lo=3000, n_hi=8000, n_test=2000, sides=(32,))
    sts = fk.precompute_batched([_tt(p.X) for p in probs], [_tt(p.y) for p in probs], [p.grid for p in probs])
    _, v_b, _ = fk.solve_batched(sts, [p.kernel for p in probs], rtol=1e-6, maxiter=6000)
    mus = fk.predict_batched(sts, v_b, [_tt(p.Xstar) for p in probs])
    for i, p in enumerate(probs):
        _, v_ref, _, _ = core.nspace_mean(p.grid, p.kernel, p.X.astype(np.float64), p.y.astype(np.float64),
                                          rtol=1e-6, x0_mode=1)
        assert rel_fro(v_b[i].double().cpu().numpy(), v_ref) <= 1e-4
        mu_ref = core.predict(p.grid, v_ref, p.Xstar.astype(np.float64))
        assert rel_fro(mus[i].double().cpu().numpy(), mu_ref) <= 1e-4


def test_batched_errors(fk):
    probs = _batch(P=2, n_hi=2e4, n_test=10)
    sts = fk.precompute_batched([_tt(p.X) for p in probs], [_tt(p.y) for p in probs], [p.grid for p in probs])
    with pytest.raises(fk.FkskiError) as e:
        fk.solve_batched([sts[0], sts[0]], [probs[0].kernel] * 2)
    assert e.value.code == fk.E_INVALID_ARG
    bad = np.array([[0.5, 3.0], [0.5, 0.5]], np.float32)  # second point off the grid
    with pytest.raises(fk.FkskiError) as e:
        fk.predict_batched(sts, [torch.ones(st.info()["m"], device="cuda") for st in sts],
                           [_tt(bad), _tt(probs[1].Xstar)])
    assert e.value.code == fk.E_OUT_OF_GRID
