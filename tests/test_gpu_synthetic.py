"""The bias / variance mechanism of the synthetic study (Tab. S1) on the GPU estimator,
at a size the oracle handles in seconds (n = 1,500, d = 1, FP64, l = 16 probes, six probe
seeds).

With no preconditioner (k = 0) the estimates scatter over seeds; they must stay within
the statistical bound of the exact values (dense Cholesky, FP64 oracle): 4 standard
errors of the seed mean.  With a rank-32 pivoted-Cholesky preconditioner the RBF and
rational quadratic kernels at d = 1 are numerically low-rank (lengthscale 0.2), so
P_hat = K_hat to rounding: every seed's estimate equals the exact value to 1e-8, and
the variance over seeds falls by at least 10^4 (the FP64 oracle measures 10^12 - 10^23
on the same problems).
"""
import numpy as np
import pytest
import torch

from oracle import exact, kernels
from paper_2107_00243_gb300 import gp, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2107_00243_gb300 import build
    build.build()
    gp.load()


@pytest.mark.parametrize("kind", [kernels.RBF, kernels.RATQUAD])
def test_preconditioning_removes_bias_and_variance(kind):
    p = workloads.synthetic_study(kind, 1, n=1500)
    ex = exact.exact_mll_and_grad(p.kind, p.X, p.y, p.theta, p.ard)
    ref = np.array([ex["mll"]] + list(ex["grad"]))
    prob = gp.Problem(p.X, p.theta, p.kind, p.ard, gp.FP64)
    vals = {}
    for k in (0, 32):
        v = []
        for sd in range(6):
            o = gp.opts(cg_tol=1e-10, max_iter=1500, seed=sd)
            st, out, iout = gp.gp_mll_and_grad(prob, p.y, k, 16, o)
            r = gp.unpack(out, iout, prob.p, 16, k)
            assert st >= 0 and r["status"] >= 0
            v.append([r["mll"]] + list(r["grad"]))
        vals[k] = np.array(v)
    mean0, se0 = vals[0].mean(0), vals[0].std(0, ddof=1) / np.sqrt(6)
    print("k=0 relative bias", np.abs(mean0 - ref) / np.abs(ref),
          "k=32:", np.abs(vals[32].mean(0) - ref) / np.abs(ref))
    assert np.all(np.abs(mean0 - ref) <= 4 * se0 + 1e-9 * np.abs(ref))
    assert np.all(np.abs(vals[32] - ref) <= 1e-8 * np.abs(ref))
    ratio = vals[0].var(0, ddof=1) / np.maximum(vals[32].var(0, ddof=1), 1e-300)
    print("variance ratio k=0 / k=32:", ratio)
    assert np.all(ratio >= 1e4)
