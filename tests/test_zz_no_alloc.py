"""Allocation-free K_G product (fkski_kg_mvm_noalloc) against the allocating fkski_kg_mvm.

Both run the same FFT kernels, so the bar is the K_G test's own (2e-6 FP32, 1e-12 FP64 relative
Frobenius); each case calls the allocation-free entry point twice in a row, after a different
problem has left other data in the shared scratch array."""
import numpy as np
import pytest
import torch

from gpu_helpers import rel_fro
from paper_2101_11751_gb300 import synth

pytestmark = pytest.mark.gpu

CASES = [((1000,), (0.05,), 1), ((128, 128), (0.04, 0.06), 3), ((33, 20), (0.3, 0.1), 2),
         ((12, 10, 11), (0.2, 0.3, 0.25), 4), ((64, 64, 64), (0.1, 0.1, 0.1), 1), ((5, 130, 6), (0.3, 0.05, 0.4), 3)]


def _vec(grid, nrhs, dtype, seed):
    V = np.random.default_rng(seed).normal(size=(nrhs, grid.m)).astype(dtype)
    return torch.from_numpy(V).cuda()


@pytest.mark.parametrize("M,ell,nrhs", CASES)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_noalloc_matches_kg_mvm_twice(fk, M, ell, nrhs, dtype):
    d = len(M)
    grid = synth.grid_for_box([0.0] * d, [1.0] * d, M)
    kern = synth.Kernel(synth.RBF, ell, 1.7, 0.1)
    tol = 2e-6 if dtype == np.float32 else 1e-12
    # leave other data in the scratch first: a different grid, kernel and rhs count
    other = synth.grid_for_box([0.0] * 3, [1.0] * 3, (40, 41, 42))
    Vo = _vec(other, 2, dtype, 99)
    fk.kg_mvm_noalloc(other, synth.Kernel(synth.RBF, (0.3, 0.2, 0.1), 2.0, 0.1), Vo, torch.empty_like(Vo))
    V = _vec(grid, nrhs, dtype, d + nrhs)
    for p in [-1] + list(range(d)) + [d]:
        ref = fk.kg_mvm(grid, kern, V, param=p)
        out1, out2 = torch.full_like(V, float("nan")), torch.full_like(V, float("nan"))
        fk.kg_mvm_noalloc(grid, kern, V, out1, param=p)
        fk.kg_mvm_noalloc(grid, kern, V, out2, param=p)
        torch.cuda.synchronize()
        assert rel_fro(out1.cpu().numpy(), ref.cpu().numpy()) <= tol, (p, "first call")
        assert rel_fro(out2.cpu().numpy(), ref.cpu().numpy()) <= tol, (p, "second call")


def test_noalloc_takes_no_device_memory(fk):
    grid = synth.grid_for_box([0.0] * 3, [1.0] * 3, (64, 64, 64))
    kern = synth.Kernel(synth.RBF, (0.1, 0.1, 0.1), 1.0, 0.1)
    V = _vec(grid, 2, np.float32, 7)
    out = torch.empty_like(V)
    fk.kg_mvm_noalloc(grid, kern, V, out)  # first call on the device: looks the scratch up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        fk.kg_mvm_noalloc(grid, kern, V, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_limits(fk):
    # room for (16 MiB - 96 KiB) / 4 = 4,169,728 FP32 or 2,084,864 FP64 values; 120^3 = 1,728,000
    # per rhs: two FP32 rhs fit, three do not; one FP64 rhs fits, two do not
    grid = synth.grid_for_box([0.0] * 3, [1.0] * 3, (120, 120, 120))
    kern = synth.Kernel(synth.RBF, (0.1, 0.1, 0.1), 1.0, 0.1)
    for dtype, ok, bad in [(np.float32, 2, 3), (np.float64, 1, 2)]:
        V = torch.zeros(bad, grid.m, dtype=torch.float32 if dtype == np.float32 else torch.float64, device="cuda")
        fk.kg_mvm_noalloc(grid, kern, V[:ok], torch.empty_like(V[:ok]))
        with pytest.raises(fk.FkskiError) as e:
            fk.kg_mvm_noalloc(grid, kern, V, torch.empty_like(V))
        assert e.value.code == fk.E_UNSUPPORTED
    small = synth.grid_for_box([0.0] * 2, [1.0] * 2, (20, 20))
    Vs = torch.zeros(1, small.m, device="cuda")
    with pytest.raises(fk.FkskiError) as e:
        fk.kg_mvm_noalloc(small, synth.Kernel(synth.MATERN52, (0.1, 0.1), 1.0, 0.1), Vs, torch.empty_like(Vs))
    assert e.value.code == fk.E_UNSUPPORTED
