"""GPU posterior covariance at test points (fkski_posterior_cov) against the oracle.

The covariance is the prior w_i^T K w_j minus a correction of nearly the same size wherever the
data pin the function down: on these problems the posterior variance is 1e2-1e4 times smaller than
the prior, so a CG solve stopped at relative residual rtol leaves errors near rtol x that ratio x
cond(A) in the result (both for the oracle's n-space CG and for the factorized solve; measured
8e-5 at rtol 1e-8 on the 1-D case).  Bars therefore use tight tolerances: FP64 at rtol 1e-12
against the dense Def. 1 covariance, 1e-6 relative Frobenius (and symmetric to 1e-6); MIXED
(double-float arithmetic on the FP32 statistics of FP32 points) at rtol 1e-10 on a problem with a
variance ratio near 1e2, 1e-4; the FP32 mode (FP32 operators, ~1e-7 relative error each) at rtol
1e-6, 1e-2."""
import numpy as np
import pytest
import torch

from gpu_helpers import problem, rel_fro
from paper_2101_11751_gb300 import synth

pytestmark = pytest.mark.gpu


def _tt(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("d,M,n,kern", [
    (1, (120,), 3000, synth.Kernel(synth.RBF, (0.05,), 1.0, 0.01)),
    (2, (20, 21), 4000, synth.Kernel(synth.MATERN52, (0.15, 0.2), 1.2, 0.03)),
    (3, (10, 9, 12), 6000, synth.Kernel(synth.RBF, (0.25, 0.3, 0.2), 1.0, 0.05)),
])
def test_cov_fp64_matches_dense(fk, oracle_mod, d, M, n, kern):
    from oracle import core
    grid, X, y = problem(d, M, n, seed=31, dtype=np.float64)
    Xs = np.random.default_rng(5).uniform(0.02, 0.98, size=(d, 45))  # two blocks of 32, ragged
    st = fk.precompute(_tt(X), _tt(y), grid)
    cov, info = fk.posterior_cov(st, kern, _tt(Xs), rtol=1e-12, maxiter=20000, precision=fk.DOUBLE)
    cov = cov.cpu().numpy()
    dense = core.ski_inference_dense(grid, kern, X, y, Xs)["cov"]
    assert rel_fro(cov, dense) <= 1e-6, rel_fro(cov, dense)
    assert rel_fro(cov, cov.T) <= 1e-6
    ref, _ = core.nspace_cov(grid, kern, X, Xs, rtol=1e-12)
    assert rel_fro(cov, ref) <= 1e-6


def test_cov_mixed(fk, oracle_mod):
    from oracle import core
    grid, X, y = problem(2, (24, 28), 1500, seed=32)
    kern = synth.Kernel(synth.RBF, (0.15, 0.2), 1.0, 0.1)
    Xs = np.random.default_rng(6).uniform(0.02, 0.98, size=(2, 40)).astype(np.float32)
    st = fk.precompute(_tt(X), _tt(y), grid)
    dense = core.ski_inference_dense(grid, kern, X.astype(np.float64), y.astype(np.float64), Xs.astype(np.float64))
    cov, _ = fk.posterior_cov(st, kern, _tt(Xs), rtol=1e-10, maxiter=6000)
    cov = cov.cpu().numpy()
    assert rel_fro(cov, dense["cov"]) <= 1e-4, rel_fro(cov, dense["cov"])
    cov32, _ = fk.posterior_cov(st, kern, _tt(Xs), rtol=1e-6, maxiter=6000, precision=fk.FP32)
    assert rel_fro(cov32.cpu().numpy(), dense["cov"]) <= 1e-2


def test_cov_out_of_grid(fk):
    grid, X, y = problem(2, (16, 16), 2000, seed=1)
    st = fk.precompute(_tt(X), _tt(y), grid)
    Xs = np.array([[0.5, 0.3], [0.5, 5.0]], np.float32)
    with pytest.raises(fk.FkskiError) as e:
        fk.posterior_cov(st, synth.Kernel(synth.RBF, (0.2, 0.2), 1.0, 0.05), _tt(Xs))
    assert e.value.code == fk.E_OUT_OF_GRID


@pytest.mark.parametrize("d,M,n,kern,k", [
    (1, (60,), 2000, synth.Kernel(synth.RBF, (0.08,), 1.0, 0.02), 25),
    (2, (16, 18), 3000, synth.Kernel(synth.RBF, (0.2, 0.25), 1.0, 0.05), 40),
])
def test_lowrank_cov_matches_oracle_lanczos(fk, oracle_mod, d, M, n, kern, k):
    """EFLA vs the oracle's plain n-space Lanczos with full reorthogonalisation (same k, same
    start y): the rank-k covariance agrees to 1e-6 (FP64 on both sides)."""
    from oracle import core
    grid, X, y = problem(d, M, n, seed=41, dtype=np.float64)
    Xs = np.random.default_rng(6).uniform(0.02, 0.98, size=(d, 37))
    st = fk.precompute(_tt(X), _tt(y), grid)
    cov, info = fk.posterior_cov_lowrank(st, kern, _tt(Xs), k)
    ref, T = core.lowrank_cov(grid, kern, X, y, Xs, k)
    assert info["steps"] == T.shape[0]
    assert rel_fro(cov.cpu().numpy(), ref) <= 1e-6, rel_fro(cov.cpu().numpy(), ref)
    # cached factor: a second call with other test points reuses it
    Xs2 = np.random.default_rng(7).uniform(0.02, 0.98, size=(d, 5))
    cov2, _ = fk.posterior_cov_lowrank(st, kern, _tt(Xs2), k)
    ref2, _ = core.lowrank_cov(grid, kern, X, y, Xs2, k)
    assert rel_fro(cov2.cpu().numpy(), ref2) <= 1e-6


def test_lowrank_cov_full_rank_is_exact(fk, oracle_mod):
    """With k past the Krylov dimension (m + 1) the Lanczos factor is exact: the rank-k
    covariance equals the exact covariance."""
    from oracle import core
    grid, X, y = problem(2, (8, 9), 600, seed=42, dtype=np.float64)
    kern = synth.Kernel(synth.RBF, (0.3, 0.3), 1.0, 0.05)
    Xs = np.random.default_rng(8).uniform(0.05, 0.95, size=(2, 12))
    st = fk.precompute(_tt(X), _tt(y), grid)
    cov, info = fk.posterior_cov_lowrank(st, kern, _tt(Xs), grid.m + 10)
    assert info["steps"] <= grid.m + 1
    dense = core.ski_inference_dense(grid, kern, X, y, Xs)["cov"]
    assert rel_fro(cov.cpu().numpy(), dense) <= 1e-6
