"""autograd.Function around the estimator (the differentiated FP32 workload).

* With a full-rank preconditioner (k = n) the estimator is exact, so the
  hand-written backward must equal a central finite difference of the forward at
  step 1e-3 (relative, in log-space), up to O(h^2) and CG tolerance.
* On the Matern-5/2 ARD workload (d = 8; a subsample) the quadratic-term part of
  the gradient is checked against finite differences of -1/2 y^T K^-1 y, and the
  full gradient against the exact FP64 gradient within the statistical bound.
* An Adam step moves log(theta) along the estimated gradient.
"""
import numpy as np
import pytest
import torch

from oracle import exact
from paper_2107_00243_gb300 import autograd, gp, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2107_00243_gb300 import build
    build.build()
    gp.load()


def test_backward_matches_fd_full_rank():
    # short lengthscales keep K well conditioned, so the rank-n factor is complete
    p = workloads.random_problem(150, 3, kind=gp.MATERN52, ard=True, seed=31, s2=0.05,
                                 lo=0.15, hi=0.25)
    prob = gp.Problem(p.X, p.theta, p.kind, p.ard, gp.FP64)
    o = gp.opts(cg_tol=1e-12, max_iter=400, seed=1)
    phi = torch.log(torch.tensor(p.theta)).requires_grad_(True)
    val = autograd.mll(torch.exp(phi), prob, p.y, p.n, 4, o)
    val.backward()
    g = phi.grad.numpy()
    h = 1e-3
    for q in range(len(p.theta)):
        e = np.zeros_like(p.theta)
        e[q] = h
        fp = autograd.mll(torch.exp(torch.tensor(np.log(p.theta) + e)), prob, p.y, p.n, 4, o)
        fm = autograd.mll(torch.exp(torch.tensor(np.log(p.theta) - e)), prob, p.y, p.n, 4, o)
        fd = float(fp - fm) / (2 * h)
        assert abs(fd - g[q]) <= 1e-5 * max(1.0, abs(fd)), (q, fd, g[q])


def test_matern52_gradient_within_statistical_bound_fp32():
    p = workloads.subsample(workloads.c2_matern52_ard(n=20000), 1500)
    ex = exact.exact_mll_and_grad(p.kind, p.X, p.y, p.theta, p.ard)
    prob = gp.Problem(p.X, p.theta, p.kind, p.ard, gp.FP32)
    o = gp.opts(cg_tol=1e-4, max_iter=1000, seed=3)
    grads = []
    for seed in range(8):
        o.seed = seed
        theta = torch.tensor(p.theta, requires_grad=True)
        val = autograd.mll(theta, prob, p.y, p.k, p.n_probes, o)
        val.backward()
        grads.append(theta.grad.numpy().copy())
    grads = np.array(grads)
    mean = grads.mean(axis=0)
    se = grads.std(axis=0, ddof=1) / np.sqrt(len(grads))
    scale = 0.5 * (np.abs(ex["quad_p"]) + np.abs(ex["trace_p"]))
    # 4 standard errors plus a CG-tolerance term
    assert np.all(np.abs(mean - ex["grad"]) <= 4 * se + 2e-3 * scale), (mean, ex["grad"], se)


def test_adam_step_increases_mll():
    p = workloads.random_problem(800, 2, kind=gp.MATERN32, ard=True, seed=33, s2=0.2,
                                 lo=0.2, hi=0.3)
    prob = gp.Problem(p.X, p.theta, p.kind, p.ard, gp.FP32)
    o = gp.opts(cg_tol=1e-3, max_iter=400, seed=0)
    theta0 = np.array([1.0, 1.0, 1.0, 0.5])
    _, hist = autograd.adam_fit(prob, p.y, theta0, 20, 8, o, steps=6, lr=0.1)
    vals = [h[0] for h in hist]
    assert vals[-1] > vals[0]
