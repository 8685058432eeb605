"""GPU K_G MVM (circulant-embedding FFT) against the oracle's dense/Kronecker definitions.

FP32 bar: relative Frobenius 2e-6 (an FFT of length L accumulates ~log2(L) roundings of 2^-24
relative to the largest spectral values); FP64 bar: 1e-12; double-float vectors (the MIXED
solver's K_G): 1e-11 (the same roundings at ~2^-46, plus the spectra rounded once from FP64)."""
import numpy as np
import pytest
import torch

from gpu_helpers import rel_fro
from paper_2101_11751_gb300 import synth

pytestmark = pytest.mark.gpu

GRIDS = [((7,), (0.2,)), ((1000,), (0.05,)), ((128, 128), (0.04, 0.06)), ((33, 20), (0.3, 0.1)),
         ((12, 10, 11), (0.2, 0.3, 0.25)), ((64, 64, 64), (0.1, 0.1, 0.1)), ((5, 130, 6), (0.3, 0.05, 0.4)),
         ((4, 9), (0.5, 0.3)), ((300,), (0.02,))]  # L = 8 and 32; L = 1024 (shared-memory transform)


@pytest.mark.parametrize("M,ell", GRIDS)
@pytest.mark.parametrize("ktype", [synth.RBF, synth.MATERN52])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_kg_mvm(fk, oracle_mod, M, ell, ktype, dtype, nrhs):
    from oracle import core
    d = len(M)
    if ktype == synth.MATERN52 and np.prod(M) > 20000:
        pytest.skip("oracle Matern reference via FFT is exercised on the smaller grids")
    grid = synth.grid_for_box([0.0] * d, [1.0] * d, M)
    kern = synth.Kernel(ktype, ell, 1.7, 0.1)
    V = np.random.default_rng(len(M) + nrhs).normal(size=(nrhs, grid.m)).astype(dtype)
    tol = 2e-6 if dtype == np.float32 else 1e-12
    for param in [None] + [("ell", k) for k in range(d)] + ["scale"]:
        p = -1 if param is None else (d if param == "scale" else param[1])
        out = fk.kg_mvm(grid, kern, torch.from_numpy(V).cuda(), param=p).cpu().numpy()
        ref = core.kg_matvec(grid, kern, V.astype(np.float64).T, param).T
        assert rel_fro(out, ref) <= tol, (param, rel_fro(out, ref))


@pytest.mark.parametrize("M,ell", [((1000,), (0.05,)), ((128, 128), (0.04, 0.06)), ((33, 20), (0.3, 0.1)),
                                   ((12, 10, 11), (0.2, 0.3, 0.25)), ((128, 128, 32), (0.05, 0.05, 0.02)),
                                   ((5, 130, 6), (0.3, 0.05, 0.4)), ((300,), (0.02,))])
@pytest.mark.parametrize("ktype", [synth.RBF, synth.MATERN52])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_kg_mvm_double_float(fk, oracle_mod, M, ell, ktype, nrhs):
    """K_G on double-float vectors (hi, lo FP32 pairs), every transform path the MIXED solver
    uses (register lines, shared-memory radix-4 lines, the Matern multilevel embedding), against
    the oracle applied in FP64 to the exact values hi + lo."""
    from oracle import core
    d = len(M)
    if ktype == synth.MATERN52 and np.prod(M) > 20000:
        pytest.skip("oracle Matern reference via FFT is exercised on the smaller grids")
    grid = synth.grid_for_box([0.0] * d, [1.0] * d, M)
    kern = synth.Kernel(ktype, ell, 1.7, 0.1)
    V = np.random.default_rng(len(M) + 7 * nrhs).normal(size=(nrhs, grid.m))
    hi = V.astype(np.float32)
    lo = (V - hi.astype(np.float64)).astype(np.float32)
    x = hi.astype(np.float64) + lo.astype(np.float64)
    xdf = torch.from_numpy(np.ascontiguousarray(np.stack([hi, lo], axis=-1))).cuda()
    for param in [None, ("ell", 0), "scale"]:
        p = -1 if param is None else (d if param == "scale" else param[1])
        out = fk.kg_mvm(grid, kern, xdf if nrhs > 1 else xdf[0], param=p, double_float=True).cpu().numpy()
        out = out.reshape(nrhs, grid.m, 2)
        got = out[..., 0].astype(np.float64) + out[..., 1].astype(np.float64)
        ref = core.kg_matvec(grid, kern, x.T, param).T
        assert rel_fro(got, ref) <= 1e-11, (param, rel_fro(got, ref))
