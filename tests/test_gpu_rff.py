"""The estimator with the Fourier feature preconditioners of Tab. 2 against the FP64
oracle through the C ABI: random features ("RFF"; gp_mll_and_grad_rff) and quadrature
features of the RBF kernel ("QFF"; gp_mll_and_grad_qff).

Matched runs: the same feature draws (eps, g), the same probe signs (one seed, one
counter-based generator on both sides) and the oracle's per-column CG iteration counts
forced on the GPU.  Bounds as for the partial Cholesky preconditioner: FP64 5e-9 on the
results and 1e-7 on gradient entries (relative to 1/2 (|quad_p| + |trace_p|)) with CG to
1e-8; FP32 1e-4 with CG to 1e-5; the mixed precision 5e-3.
"""
import numpy as np
import pytest
import torch

from oracle import estimator, kernels
from paper_2107_00243_gb300 import gp, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2107_00243_gb300 import build
    build.build()
    gp.load()


CASES = {
    "rbf_ard_d3": (kernels.RBF, True, 3, 800, 40),
    "matern32_ard_d4": (kernels.MATERN32, True, 4, 900, 50),
    "matern52_ard_d3": (kernels.MATERN52, True, 3, 700, 32),
    "ratquad_iso_d2": (kernels.RATQUAD, False, 2, 640, 24),
}
TOL = {gp.FP64: (1e-8, (5e-9, 1e-7)), gp.FP32: (1e-5, (1e-4, 1e-4)),
       gp.BF16: (1e-3, (5e-3, 5e-3))}


def _errors(r, ref):
    e = {k: abs(r[k] - ref[k]) / abs(ref[k]) for k in ("mll", "quad", "logdet", "logdetP")}
    scale = 0.5 * (np.abs(ref["quad_p"]) + np.abs(ref["trace_p"]))
    e["grad"] = float(np.max(np.abs(r["grad"] - ref["grad"]) / scale))
    e["trP"] = float(np.max(np.abs(r["trP_p"] - ref["trP_p"]) / scale))
    e["probeP"] = float(np.max(np.abs(r["probeP_p"] - ref["probeP_p"]) / scale))
    return e


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("prec", [gp.FP64, gp.FP32, gp.BF16])
def test_rff_estimator_vs_oracle(name, prec):
    kind, ard, d, n, m = CASES[name]
    p = workloads.random_problem(n, d, kind=kind, ard=ard, seed=41, s2=0.05, k=2 * m,
                                 n_probes=6, tol=TOL[prec][0], max_iter=600)
    eps, g = workloads.rff_draws(m, d, gp.rff_gamma_shape(kind), seed=3)
    ref = estimator.mll_and_grad(p.kind, p.X, p.y, p.theta, p.ard, 2 * m, p.n_probes, p.tol,
                                 p.max_iter, seed=5, rff=(eps, g))
    prob = gp.Problem(p.X, p.theta, p.kind, p.ard, prec)
    o = gp.opts(cg_tol=p.tol, max_iter=p.max_iter, seed=5)
    st, out, iout = gp.gp_mll_and_grad_rff(prob, p.y, m, p.n_probes, o, eps, g,
                                           iters_override=ref["iters"])
    r = gp.unpack(out, iout, prob.p, p.n_probes, 2 * m)
    assert st >= 0 and r["status"] == 0 and r["rank"] == 2 * m
    assert np.all(r["piv"] == -1)
    np.testing.assert_array_equal(r["iters"], ref["iters"])
    e = _errors(r, ref)
    print(name, prec, {k: f"{v:.1e}" for k, v in e.items()})
    tv, tg = TOL[prec][1]
    assert all(e[k] <= tv for k in ("mll", "quad", "logdet", "logdetP")), e
    assert e["grad"] <= tg and e["trP"] <= 3 * tg and e["probeP"] <= 3 * tg, e


def test_rff_rejects_bad_arguments():
    p = workloads.random_problem(100, 2, kind=kernels.MATERN32, seed=2, k=10, n_probes=2)
    prob = gp.Problem(p.X, p.theta, p.kind, p.ard, gp.FP64)
    o = gp.opts()
    eps, g = workloads.rff_draws(8, 2, 1.5)
    with pytest.raises(gp.GPError):            # Matern needs g
        gp.gp_mll_and_grad_rff(prob, p.y, 8, 2, o, eps, None)
    with pytest.raises(gp.GPError):            # 2m > n
        gp.gp_mll_and_grad_rff(prob, p.y, 51, 2, o, np.zeros((51, 2)), np.ones(51))


QFF_CASES = {"ard_d1": (True, 1, 16), "ard_d2": (True, 2, 8), "iso_d3": (False, 3, 4)}


@pytest.mark.parametrize("name", sorted(QFF_CASES))
@pytest.mark.parametrize("prec", [gp.FP64, gp.FP32, gp.BF16])
def test_qff_estimator_vs_oracle(name, prec):
    """Quadrature features make P_hat nearly K_hat (CG needs 1-5 iterations), which sets
    how the two lower precisions are compared:
    * the MLL is a small difference here (|MLL| ~ 1 % of y^T u and log det), so it is
      compared on the scale 1/2 (|y^T u| + |log det|) of its components;
    * FP32: the Woodbury apply sigma^-2 (r - Phi C^-1 Phi^T r) cancels to rounding of
      eps_32 kappa, kappa = lambda_max(K_hat) / sigma^2 (~1e4 here, eps_32 kappa ~ 8e-4),
      in every term that uses P^-1 z; the bounds are max(1e-4, 2 eps_32 kappa) on the
      results and 4 eps_32 kappa on gradient entries;
    * mixed precision runs the precise split mode (k(r) / s to 22 bits), which is the
      mode for problems this well preconditioned: fast mode's 11-bit k(r) moved a
      gradient entry by 5.8e-3 (d = 2)."""
    ard, d, mbar = QFF_CASES[name]
    k = mbar ** d
    p = workloads.random_problem(700, d, kind=kernels.RBF, ard=ard, seed=43, s2=0.05, k=k,
                                 n_probes=6, tol=TOL[prec][0], max_iter=600)
    ref = estimator.mll_and_grad(p.kind, p.X, p.y, p.theta, p.ard, k, p.n_probes, p.tol,
                                 p.max_iter, seed=7, qff=mbar)
    prob = gp.Problem(p.X, p.theta, p.kind, p.ard, prec)
    o = gp.opts(cg_tol=p.tol, max_iter=p.max_iter, seed=7,
                flags=gp.OPT_SPLIT_P if prec == gp.BF16 else 0)
    st, out, iout = gp.gp_mll_and_grad_qff(prob, p.y, mbar, p.n_probes, o,
                                           iters_override=ref["iters"])
    r = gp.unpack(out, iout, prob.p, p.n_probes, k)
    assert st >= 0 and r["status"] == 0 and r["rank"] == k
    np.testing.assert_array_equal(r["iters"], ref["iters"])
    e = _errors(r, ref)
    e["mll"] = abs(r["mll"] - ref["mll"]) / (0.5 * (abs(ref["quad"]) + abs(ref["logdet"])))
    print(name, prec, {kk: f"{v:.1e}" for kk, v in e.items()})
    tv, tg = TOL[prec][1]
    if prec == gp.FP32:
        K_hat = kernels.khat_dense(p.kind, p.X, p.theta, p.ard)
        kappa = np.linalg.eigvalsh(K_hat)[-1] / p.theta[-1]
        tv, tg = max(tv, 2 * 2.0 ** -24 * kappa), max(tg, 4 * 2.0 ** -24 * kappa)
    assert all(e[kk] <= tv for kk in ("mll", "quad", "logdet", "logdetP")), e
    assert e["grad"] <= tg and e["trP"] <= 3 * tg and e["probeP"] <= 3 * tg, e


def test_qff_rejects_other_kernels_and_odd_rules():
    p = workloads.random_problem(100, 2, kind=kernels.MATERN32, seed=2, k=16, n_probes=2)
    prob = gp.Problem(p.X, p.theta, p.kind, p.ard, gp.FP64)
    with pytest.raises(gp.GPError):
        gp.gp_mll_and_grad_qff(prob, p.y, 4, 2, gp.opts())
    p = workloads.random_problem(100, 2, kind=kernels.RBF, seed=2, k=16, n_probes=2)
    prob = gp.Problem(p.X, p.theta, p.kind, p.ard, gp.FP64)
    with pytest.raises(gp.GPError):
        gp.gp_mll_and_grad_qff(prob, p.y, 5, 2, gp.opts())
