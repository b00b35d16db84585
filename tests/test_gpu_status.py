"""Statuses of the C ABI on conditions a caller can cause, through real GPU calls.

Every failure here is made on the host side of the call: a CG cap that is too small,
hyperparameters that are not finite or not positive, a preconditioner factor with a
non-finite column.  None of them faults, traps or hangs the GPU; each returns normally
with a status:
  GP_WARN_NOT_CONVERGED  a CG column reached max_iter above the tolerance; every
                         result is still written (and finite)
  GP_ERR_INVALID_ARG     theta has an entry that is NaN, infinite or <= 0 (checked on
                         the device, read back before anything else runs)
  GP_ERR_NOT_SPD         the Woodbury core sigma^2 I + L^T L has no Cholesky factor
The first device error wins: the NaNs that a failed core spreads into CG do not
replace GP_ERR_NOT_SPD by GP_ERR_NUMERIC.
"""
import numpy as np
import pytest
import torch

from paper_2107_00243_gb300 import gp, workloads

pytestmark = pytest.mark.gpu

GP_WARN_NOT_CONVERGED, GP_ERR_INVALID_ARG, GP_ERR_NOT_SPD = 1, -1, -3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2107_00243_gb300 import build
    build.build()
    gp.load()


@pytest.mark.parametrize("prec", [gp.FP64, gp.FP32, gp.BF16])
def test_iteration_cap_warns_and_writes_results(prec):
    p = workloads.random_problem(700, 3, seed=31, s2=0.01, k=10, n_probes=4, tol=1e-8,
                                 max_iter=2)
    prob = gp.Problem(p.X, p.theta, p.kind, p.ard, prec)
    o = gp.opts(cg_tol=p.tol, max_iter=p.max_iter, seed=1, flags=gp.OPT_FAST_ONLY)
    st, out, iout = gp.gp_mll_and_grad(prob, p.y, p.k, p.n_probes, o)
    r = gp.unpack(out, iout, prob.p, p.n_probes, p.k)
    assert st == GP_WARN_NOT_CONVERGED and r["status"] == GP_WARN_NOT_CONVERGED
    assert np.all(r["iters"] == 2)
    assert np.all(np.isfinite(out.cpu().numpy()))
    # the same problem with room to converge: no warning
    o2 = gp.opts(cg_tol=1e-4, max_iter=700, seed=1, flags=gp.OPT_FAST_ONLY)
    st2, out2, iout2 = gp.gp_mll_and_grad(prob, p.y, p.k, p.n_probes, o2)
    assert st2 == 0 and int(iout2[0]) == 0


def test_iteration_cap_in_mbcg():
    p = workloads.random_problem(500, 2, seed=32, s2=0.01)
    prob = gp.Problem(p.X, p.theta, p.kind, p.ard, gp.FP64)
    B = np.random.default_rng(0).standard_normal((p.n, 3))
    res = gp.gp_mbcg(prob, None, torch.from_numpy(B), gp.opts(cg_tol=1e-10, max_iter=3))
    assert res["status"] == GP_WARN_NOT_CONVERGED
    assert np.all(res["iters"].cpu().numpy() == 3)
    assert np.all(np.isfinite(res["X"].cpu().numpy()))


@pytest.mark.parametrize("bad", ["nan_lengthscale", "zero_noise", "negative_scale",
                                 "inf_noise"])
@pytest.mark.parametrize("prec", [gp.FP64, gp.BF16])
def test_invalid_theta_rejected(bad, prec):
    p = workloads.random_problem(300, 2, seed=33, k=5, n_probes=3, tol=1e-6, max_iter=300)
    th = p.theta.copy()
    if bad == "nan_lengthscale":
        th[0] = np.nan
    elif bad == "zero_noise":
        th[-1] = 0.0
    elif bad == "negative_scale":
        th[-2] = -1.0
    else:
        th[-1] = np.inf
    prob = gp.Problem(p.X, th, p.kind, p.ard, prec)
    o = gp.opts(cg_tol=p.tol, max_iter=p.max_iter, seed=0)
    iout = torch.zeros(2 + p.n_probes + 1 + p.k, dtype=torch.int32, device="cuda")
    l0 = gp.launch_count()
    with pytest.raises(gp.GPError) as ei:
        gp.gp_mll_and_grad(prob, p.y, p.k, p.n_probes, o, iout=iout)
    assert ei.value.status == GP_ERR_INVALID_ARG
    assert "theta" in str(ei.value)
    assert int(iout[0]) == GP_ERR_INVALID_ARG
    assert gp.launch_count() - l0 <= 2        # the check itself, nothing after it
    # and the same problem with valid hyperparameters runs
    prob.set_theta(p.theta)
    st, out, iout = gp.gp_mll_and_grad(prob, p.y, p.k, p.n_probes, o)
    assert st == 0


@pytest.mark.parametrize("prec", [gp.FP64, gp.FP32])
def test_non_spd_woodbury_core(prec):
    """A preconditioner factor with a NaN column: the core's Cholesky fails and the
    call reports GP_ERR_NOT_SPD (not the later CG breakdown the NaNs cause)."""
    p = workloads.random_problem(400, 2, seed=34, s2=0.05)
    prob = gp.Problem(p.X, p.theta, p.kind, p.ard, prec)
    L = np.random.default_rng(1).standard_normal((p.n, 6)) * 0.1
    L[:, 3] = np.nan
    B = np.random.default_rng(2).standard_normal((p.n, 2))
    with pytest.raises(gp.GPError) as ei:
        gp.gp_mbcg(prob, torch.from_numpy(L), torch.from_numpy(B),
                   gp.opts(cg_tol=1e-6, max_iter=50))
    assert ei.value.status == GP_ERR_NOT_SPD, ei.value.status
