"""The estimator with the random Fourier feature preconditioner (Tab. 2 "RFF";
gp_mll_and_grad_rff) against the FP64 oracle through the C ABI.

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
