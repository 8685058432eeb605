"""GPU log-likelihood and gradient (SLQ + Hutchinson, adjoint via factorized CG).

Bars: against the oracle's same-probe stochastic value and gradient (n-space CG, same probes,
same tolerance) within 1e-4 relative in both precisions; with sqrt(n)-scaled unit-vector probes (exact traces) the
gradient matches central finite differences of the exact dense log-likelihood within 1e-3."""
import math

import numpy as np
import pytest
import torch

from gpu_helpers import problem
from paper_2101_11751_gb300 import synth

pytestmark = pytest.mark.gpu


def _tt(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("d,M,n,kern,prec", [
    (2, (24, 22), 6000, synth.Kernel(synth.RBF, (0.15, 0.2), 1.0, 0.02), 1),
    (2, (24, 22), 6000, synth.Kernel(synth.RBF, (0.15, 0.2), 1.0, 0.02), 0),
    (2, (20, 21), 5000, synth.Kernel(synth.MATERN52, (0.15, 0.2), 1.2, 0.03), 1),
    (3, (10, 9, 11), 8000, synth.Kernel(synth.RBF, (0.25, 0.3, 0.2), 1.0, 0.05), 1),
    (3, (10, 9, 11), 8000, synth.Kernel(synth.RBF, (0.25, 0.3, 0.2), 1.0, 0.05), 0),
])
def test_grad_matches_same_probe_oracle(fk, oracle_mod, d, M, n, kern, prec):
    from oracle import core
    dtype = np.float64 if prec == 1 else np.float32
    grid, X, y = problem(d, M, n, seed=21, dtype=dtype)
    T, seed = 8, 5
    st = fk.precompute(_tt(X), _tt(y), grid, n_probes=T, probe_seed=seed)
    rtol = 1e-8 if prec == 1 else 1e-5
    L, g, info = fk.grad(st, kern, rtol=rtol, maxiter=4000, precision=prec)
    Z = np.stack([core.rademacher(seed, p, n) for p in range(T)])
    ref = core.loglik_grad_stochastic(grid, kern, X, y, Z, rtol=rtol)
    tol = 1e-4
    assert L == pytest.approx(ref["L"], rel=tol)
    np.testing.assert_allclose(g, ref["grad"], rtol=tol, atol=tol * np.max(np.abs(ref["grad"])))


def test_grad_not_converged_raises(fk):
    """A solve stopped at maxiter reaches the caller as an error, also through autograd."""
    grid, X, y = problem(2, (16, 15), 3000, seed=4)
    st = fk.precompute(_tt(X), _tt(y), grid, n_probes=2, probe_seed=1)
    kern = synth.Kernel(synth.RBF, (0.2, 0.25), 1.0, 0.02)
    with pytest.raises(fk.FkskiError) as e:
        fk.grad(st, kern, rtol=1e-12, maxiter=3)
    assert e.value.code == fk.E_NOT_CONVERGED
    L, g, info = fk.grad(st, kern, rtol=1e-12, maxiter=3, allow_not_converged=True)
    assert info["status"] == fk.E_NOT_CONVERGED and np.isfinite(L)
    theta = torch.tensor([0.2, 0.25, 1.0, 0.02], dtype=torch.float64, requires_grad=True)
    with pytest.raises(fk.FkskiError):
        fk.log_marginal_likelihood(theta, st, rtol=1e-12, maxiter=3)


def test_grad_exact_traces_vs_fd(fk, oracle_mod):
    """Probes sqrt(n) e_i make the traces exact: the gradient is then the exact one."""
    from oracle import core
    grid, X, y = problem(2, (9, 8), 40, seed=2, dtype=np.float64)
    kern = synth.Kernel(synth.RBF, (0.3, 0.25), 1.3, 0.05)
    n = X.shape[1]
    Z = math.sqrt(n) * np.eye(n)
    st = fk.precompute(_tt(X), _tt(y), grid, Z=_tt(Z))
    L, g, _ = fk.grad(st, kern, rtol=1e-12, maxiter=500, precision=1)
    fd = core.grad_fd(grid, kern, X, y)
    np.testing.assert_allclose(g, fd, rtol=1e-3, atol=1e-3 * np.max(np.abs(fd)))
    assert L == pytest.approx(core.loglik_exact(grid, kern, X, y), rel=1e-6)


def test_autograd_function_and_budget_recompute(fk, oracle_mod):
    grid, X, y = problem(2, (16, 15), 3000, seed=4)
    st = fk.precompute(_tt(X), _tt(y), grid, n_probes=4, probe_seed=1)
    theta = torch.tensor([0.2, 0.25, 1.0, 0.02], dtype=torch.float64, requires_grad=True)
    L1 = fk.log_marginal_likelihood(theta, st, rtol=1e-4)
    L1.backward()
    g1 = theta.grad.clone()
    theta.grad = None
    L2 = fk.log_marginal_likelihood(theta, st, rtol=1e-4, budget=0)  # solutions not kept
    L2.backward()
    assert L1.item() == L2.item()
    torch.testing.assert_close(theta.grad, g1, rtol=0, atol=0)
    kern = synth.Kernel(synth.RBF, (0.2, 0.25), 1.0, 0.02)
    Lg, gg, _ = fk.grad(st, kern, rtol=1e-4)
    assert Lg == L1.item()
    np.testing.assert_array_equal(np.array(gg), g1.numpy())


@pytest.mark.parametrize("d,M,n,kern", [
    (2, (20, 22), 4000, synth.Kernel(synth.RBF, (0.15, 0.2), 1.0, 0.05)),
    (3, (9, 10, 8), 5000, synth.Kernel(synth.RBF, (0.25, 0.3, 0.2), 1.0, 0.05)),
])
def test_logdet_lanczos_matches_oracle(fk, oracle_mod, d, M, n, kern):
    """EFLA-based SLQ vs the oracle's n-space Lanczos (full reorthogonalisation, same probes, same
    k): the same Krylov spaces, so the per-probe quadratures agree to 1e-8 (FP64 both sides)."""
    from oracle import core
    grid, X, y = problem(d, M, n, seed=61, dtype=np.float64)
    T, seed, k = 4, 9, 40
    st = fk.precompute(_tt(X), _tt(y), grid, n_probes=T, probe_seed=seed)
    L, terms, info = fk.logdet_lanczos(st, kern, k)
    Z = np.stack([core.rademacher(seed, p, n) for p in range(T)])
    mv = core.ski_operator(grid, kern, core.w_csr(grid, X))
    ref, rterms = core.slq_logdet_lanczos(mv, Z, k)
    np.testing.assert_allclose(terms, rterms, rtol=1e-8)
    assert L == pytest.approx(ref, rel=1e-8)


def test_logdet_lanczos_exact_with_unit_probes(fk, oracle_mod):
    from oracle import core
    grid, X, y = problem(2, (8, 9), 40, seed=3, dtype=np.float64)
    kern = synth.Kernel(synth.RBF, (0.3, 0.25), 1.3, 0.05)
    n = X.shape[1]
    st = fk.precompute(_tt(X), _tt(y), grid, Z=_tt(math.sqrt(n) * np.eye(n)))
    L, _, _ = fk.logdet_lanczos(st, kern, n + 5)
    exact = core.ski_inference_dense(grid, kern, X, y, X[:, :2])["logdet"]
    assert L == pytest.approx(exact, rel=1e-8)
