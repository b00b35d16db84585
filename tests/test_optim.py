"""L-BFGS with a strong Wolfe line search (paper_2107_00243_gb300/optim.py), on the CPU.

* The line search returns steps meeting both Wolfe conditions on 1-D functions with a
  known minimiser.
* L-BFGS reaches the minimiser of Rosenbrock's function (2-D and 10-D) and of a convex
  quadratic with known solution.
* On the exact GP negative log-marginal likelihood of a small problem (the FP64 oracle,
  in log-hyperparameter space) it reaches the same optimum as scipy's L-BFGS-B.
* Validation-based early stopping returns the best-validated iterate.
* lbfgs_fit's plumbing (log-space chain rule, status handling) is checked with the
  estimator call replaced by the exact oracle, so no GPU is needed.
"""
import math

import numpy as np
import pytest

from paper_2107_00243_gb300 import optim


def _rosen(x):
    f = np.sum(100.0 * (x[1:] - x[:-1] ** 2) ** 2 + (1.0 - x[:-1]) ** 2)
    g = np.zeros_like(x)
    g[:-1] += -400.0 * x[:-1] * (x[1:] - x[:-1] ** 2) - 2.0 * (1.0 - x[:-1])
    g[1:] += 200.0 * (x[1:] - x[:-1] ** 2)
    return f, g


@pytest.mark.parametrize("c2", [0.9, 0.1])
def test_wolfe_search_conditions(c2):
    # phi(a) = (a - 3)^2 + 0.3 sin(2 a): descent at 0, minimiser near 3
    def phi(a):
        return (a - 3.0) ** 2 + 0.3 * math.sin(2 * a), 2 * (a - 3.0) + 0.6 * math.cos(2 * a), a
    f0, g0, _ = phi(0.0)
    c1 = 1e-4
    for a1 in (0.01, 1.0, 50.0):
        a, fa, pay, evals, ok = optim._wolfe_search(phi, f0, g0, a1, c1, c2, 30)
        assert ok and pay == a
        assert fa <= f0 + c1 * a * g0                       # sufficient decrease
        assert abs(phi(a)[1]) <= -c2 * g0                   # strong curvature


def test_cubic_interpolation_exact_on_cubics():
    # f(x) = (x - 1)^3 / 3 - (x - 1)  has its local minimiser at x = 2
    f = lambda x: (x - 1) ** 3 / 3 - (x - 1)
    g = lambda x: (x - 1) ** 2 - 1
    assert abs(optim._cubic_min(1.5, f(1.5), g(1.5), 3.0, f(3.0), g(3.0)) - 2.0) < 1e-12


@pytest.mark.parametrize("n", [2, 10])
def test_rosenbrock(n):
    x0 = np.full(n, -1.2)
    x0[1::2] = 1.0
    res = optim.lbfgs_minimize(_rosen, x0, max_iter=500, gtol=1e-8, ftol=0.0)
    assert res["reason"] == "gtol", res["reason"]
    assert np.allclose(res["x"], 1.0, atol=1e-6)
    fh = np.array(res["history"]["f"])
    assert np.all(np.diff(fh) <= 1e-11 * np.maximum(np.abs(fh[:-1]), 1.0))   # descent


def test_quadratic():
    rng = np.random.default_rng(0)
    Q = rng.standard_normal((20, 20))
    A = Q @ Q.T + 0.5 * np.eye(20)
    b = rng.standard_normal(20)
    fun = lambda x: (0.5 * x @ A @ x - b @ x, A @ x - b)
    res = optim.lbfgs_minimize(fun, np.zeros(20), m=20, max_iter=200, gtol=1e-10, ftol=0.0)
    assert res["reason"] == "gtol"
    assert np.allclose(res["x"], np.linalg.solve(A, b), atol=1e-8)


def _exact_problem():
    from oracle import exact
    rng = np.random.default_rng(3)
    n, d = 60, 2
    X = rng.uniform(0, 1, (n, d))
    y = np.sin(4 * X[:, 0]) + 0.5 * X[:, 1] + 0.1 * rng.standard_normal(n)

    def negmll_log(phi):
        th = np.exp(phi)
        r = exact.exact_mll_and_grad(0, X, y, th, True)     # RBF, ARD
        return -r["mll"], -th * r["grad"]
    return X, y, negmll_log


def test_exact_gp_optimum_matches_scipy():
    scipy_opt = pytest.importorskip("scipy.optimize")
    _, _, fun = _exact_problem()
    phi0 = np.log(np.array([0.5, 0.5, 1.0, 0.1]))           # l1, l2, s, sigma^2
    res = optim.lbfgs_minimize(fun, phi0, max_iter=200, gtol=1e-7, ftol=0.0)
    ref = scipy_opt.minimize(fun, phi0, jac=True, method="L-BFGS-B",
                             options={"gtol": 1e-9, "ftol": 1e-15, "maxiter": 500})
    assert res["reason"] == "gtol", res["reason"]
    assert abs(res["f"] - ref.fun) <= 1e-8 * abs(ref.fun)
    assert np.allclose(res["x"], ref.x, atol=1e-4)


def test_early_stopping_returns_best_validated_iterate():
    _, _, fun = _exact_problem()
    phi0 = np.log(np.array([0.5, 0.5, 1.0, 0.1]))
    target = np.log(np.array([0.45, 0.5, 1.0, 0.08]))
    val = lambda phi: float(np.sum((phi - target) ** 2))     # prefers an early iterate
    res = optim.lbfgs_minimize(fun, phi0, max_iter=200, gtol=1e-9, ftol=0.0,
                               validation=val, patience=2)
    hv = res["history"]["val"]
    assert res["reason"] == "early_stop"
    assert val(res["x"]) == min(hv)
    assert len(hv) >= 3 and hv[-1] > min(hv)


def test_lbfgs_fit_plumbing_with_exact_objective(monkeypatch):
    """lbfgs_fit with the estimator call replaced by the exact oracle: the log-space
    gradient it hands to the optimiser is -theta * dMLL/dtheta, and it finds the same
    optimum as optimising the exact objective directly."""
    torch = pytest.importorskip("torch")
    from oracle import exact
    from paper_2107_00243_gb300 import gp
    X, y, fun = _exact_problem()

    class FakeProblem:
        p = 4

        def __init__(self):
            self.theta = np.array([0.5, 0.5, 1.0, 0.1])

        def set_theta(self, th):
            self.theta = np.array(th, dtype=np.float64)

    prob = FakeProblem()

    def fake_call(problem, yy, k, n_probes, o, workspace=None):
        r = exact.exact_mll_and_grad(0, X, y, problem.theta, True)
        return 0, r, None

    def fake_unpack(out, iout, p, n_probes, k):
        return {"mll": out["mll"], "grad": out["grad"], "status": 0}

    monkeypatch.setattr(gp, "gp_mll_and_grad", fake_call)
    monkeypatch.setattr(gp, "unpack", fake_unpack)
    monkeypatch.setattr(gp, "Workspace", lambda: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    theta, res = optim.lbfgs_fit(prob, y, prob.theta.copy(), 0, 0, None, max_iter=200,
                                 gtol=1e-7)
    direct = optim.lbfgs_minimize(fun, np.log(np.array([0.5, 0.5, 1.0, 0.1])),
                                  max_iter=200, gtol=1e-7)
    assert np.allclose(theta, np.exp(direct["x"]), rtol=1e-10)
    assert np.allclose(prob.theta, theta)
    assert res["f"] == pytest.approx(direct["f"], rel=1e-14)


def test_failed_start_is_not_reported_converged():
    """An objective that cannot be evaluated at x0 (inf, zero gradient) ends the run
    with reason 'eval_failed', not 'gtol'."""
    res = optim.lbfgs_minimize(lambda x: (math.inf, np.zeros_like(x)), np.zeros(3))
    assert res["reason"] == "eval_failed"
    assert res["nit"] == 0 and res["nfev"] == 1


def test_lbfgs_fit_failed_evaluation_at_start(monkeypatch):
    """lbfgs_fit on an estimator that reports a device-side error at theta0."""
    torch = pytest.importorskip("torch")
    from paper_2107_00243_gb300 import gp

    class FakeProblem:
        p = 3

        def set_theta(self, th):
            self.theta = np.array(th)

    monkeypatch.setattr(gp, "gp_mll_and_grad", lambda *a, **kw: (0, None, None))
    monkeypatch.setattr(gp, "unpack", lambda *a: {"mll": 1.0, "grad": np.ones(3),
                                                  "status": -3})
    monkeypatch.setattr(gp, "Workspace", lambda: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    _, res = optim.lbfgs_fit(FakeProblem(), None, np.ones(3), 0, 0, None)
    assert res["reason"] == "eval_failed"
