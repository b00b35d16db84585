"""gp_kernel_mvm_noalloc: the kernel-matrix product for callers that cannot allocate
device memory (real-time loops with a fixed memory budget, frameworks that own the
allocator and hand the library only its inputs and outputs).  Its scratch is a static
device array in the library, reused by every call.

Checked through the C ABI against gp_kernel_mvm (which uses a caller workspace) on
two calls in a row, the second smaller than the first so that contents left in the
shared array by the first call cannot leak into the second; the bound is the kernel
product's parity tolerance (2e-5 normwise in FP32, 1e-11 in FP64), and against the
FP64 oracle's product at the same tolerance.  Sizes beyond the array are rejected
before anything runs.  Collected last on purpose.
"""
import numpy as np
import pytest
import torch

from oracle import kernels
from paper_2107_00243_gb300 import gp, workloads

pytestmark = pytest.mark.gpu

TOL = {gp.FP32: 2e-5, gp.FP64: 1e-11}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2107_00243_gb300 import build
    build.build()
    gp.load()


def _rel(a, b):
    return (a - b).abs().max().item() / b.abs().max().item()


@pytest.mark.parametrize("prec", [gp.FP32, gp.FP64])
def test_noalloc_matches_kernel_mvm_on_two_calls(prec):
    cases = [(3000, 16, 33, gp.RBF, 1), (517, 3, 7, gp.MATERN52, 2)]
    for n, d, t, kind, seed in cases:
        p = workloads.random_problem(n, d, kind=kind, ard=True, seed=seed)
        prob = gp.Problem(p.X, p.theta, kind, True, prec)
        V = torch.from_numpy(np.random.default_rng(seed).standard_normal((n, t)))
        ref = gp.gp_kernel_mvm(prob, V)
        got = gp.gp_kernel_mvm_noalloc(prob, V)
        torch.cuda.synchronize()
        assert got.shape == (n, t)
        assert _rel(got, ref) <= TOL[prec], _rel(got, ref)
        exact = torch.from_numpy(
            kernels.KernelOperator(kind, p.X, p.theta, True).matvec(V.numpy()))
        assert _rel(got.cpu().double(), exact) <= TOL[prec], _rel(got.cpu().double(), exact)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    n, d = 140000, 32                     # 140000 * 32 * 4 bytes > 16 MiB
    X = torch.zeros((n, d), dtype=torch.float32, device="cuda")
    theta = np.concatenate([np.ones(d), [1.0, 0.1]])
    prob = gp.Problem(X, theta, gp.RBF, True, gp.FP32)
    V = torch.zeros((n, 1), dtype=torch.float32)
    with pytest.raises(gp.GPError) as e:
        gp.gp_kernel_mvm_noalloc(prob, V)
    assert e.value.status == -1 and "scratch" in str(e.value)
