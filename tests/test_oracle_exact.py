"""Pins for oracle/exact.py.

* The exact MLL equals scipy's multivariate-normal log-density of y under
  N(0, K_hat) (eq. likelihood is that log-density).
* n = 1 reduces to a scalar Gaussian log-density, written out by hand.
* The analytic gradient (eq. derivative_likelihood) equals a central finite
  difference of the exact MLL.
"""
import numpy as np
import pytest
from scipy.stats import multivariate_normal, norm

from oracle import exact, kernels
from paper_2107_00243_gb300 import workloads


@pytest.mark.parametrize("kind", kernels.KINDS)
def test_mll_is_gaussian_logpdf(kind):
    p = workloads.random_problem(60, 3, kind=kind, seed=4)
    ex = exact.exact_mll_and_grad(kind, p.X, p.y, p.theta, p.ard)
    Kh = kernels.khat_dense(kind, p.X, p.theta, p.ard)
    ref = multivariate_normal(mean=np.zeros(60), cov=Kh).logpdf(p.y)
    assert abs(ex["mll"] - ref) < 1e-9 * abs(ref)


def test_single_point_by_hand():
    X = np.array([[0.25, 0.5]])
    y = np.array([0.7])
    theta = np.array([0.3, 1.4, 0.2])          # isotropic: l, s, sigma^2
    ex = exact.exact_mll_and_grad(kernels.RBF, X, y, theta, False)
    var = 1.4 + 0.2
    assert abs(ex["mll"] - norm(0.0, np.sqrt(var)).logpdf(0.7)) < 1e-14
    # d/ds and d/dsigma^2 of log N(y; 0, s + sigma^2): (y^2/var^2 - 1/var) / 2
    g = 0.5 * (0.49 / var ** 2 - 1.0 / var)
    np.testing.assert_allclose(ex["grad"], [0.0, g, g], atol=1e-14)


@pytest.mark.parametrize("kind", kernels.KINDS)
@pytest.mark.parametrize("ard", [True, False])
def test_gradient_matches_finite_differences(kind, ard):
    p = workloads.random_problem(50, 2, kind=kind, ard=ard, seed=5)
    ex = exact.exact_mll_and_grad(kind, p.X, p.y, p.theta, ard)
    for q in range(len(p.theta)):
        h = 1e-5 * p.theta[q]
        tp, tm = p.theta.copy(), p.theta.copy()
        tp[q] += h
        tm[q] -= h
        fd = (exact.exact_mll_and_grad(kind, p.X, p.y, tp, ard)["mll"]
              - exact.exact_mll_and_grad(kind, p.X, p.y, tm, ard)["mll"]) / (2 * h)
        assert abs(ex["grad"][q] - fd) <= 1e-7 * max(1.0, abs(fd)), (q, ex["grad"][q], fd)
