"""L-BFGS with a strong Wolfe (Armijo + curvature) line search and validation-based
early stopping: the hyperparameter optimiser of the paper's experiments (Sec. 5),
driving the CUDA estimator.

The optimiser is host logic on a handful of scalars per step; every objective value
and gradient comes from one call of gp_mll_and_grad.  The algorithm is written from
Nocedal & Wright, *Numerical Optimization* (2nd ed.):
  * search direction by the two-loop recursion over the last m (s, y) pairs, with the
    initial inverse Hessian gamma I, gamma = s^T y / y^T y of the newest pair;
  * pairs whose curvature s^T y is not positive (relative to |s| |y|) are skipped, so
    the implied inverse Hessian stays positive definite;
  * step length by bracketing and zooming until the sufficient-decrease (Armijo, c1)
    and strong curvature (c2) conditions hold; zoom steps interpolate with the
    minimiser of the cubic through both bracket ends, safeguarded to the bracket's
    inner 80%, else bisect.  Once f changes by less than its own rounding, the
    decrease test is replaced by the approximate Wolfe condition of Hager & Zhang
    (SIAM J. Optim. 16, 2005): phi'(a) <= (2 c1 - 1) phi'(0) with phi(a) <= phi(0)
    + eps |phi(0)|, which judges the step by its derivative alone.
Early stopping: with a validation function, the iterate with the best validation loss
is returned once `patience` iterations pass without improving it.

The estimator is stochastic through its probes; lbfgs_fit keeps one probe seed for the
whole run, so the objective is a fixed function of theta.  Its gradient is the paper's
estimator of dL/dtheta, which equals the derivative of that function only in
expectation (and exactly when the preconditioner has full rank).  A line search that
fails to meet the Wolfe conditions therefore ends the run with the best point seen,
rather than raising.
"""
import math

import numpy as np


def _cubic_min(a, fa, ga, b, fb, gb):
    """Minimiser of the cubic interpolating (a, fa, ga) and (b, fb, gb), or None."""
    d1 = ga + gb - 3.0 * (fa - fb) / (a - b)
    rad = d1 * d1 - ga * gb
    if rad < 0.0:
        return None
    d2 = math.copysign(math.sqrt(rad), b - a)
    den = gb - ga + 2.0 * d2
    if den == 0.0:
        return None
    return b - (b - a) * (gb + d2 - d1) / den


def _wolfe_search(phi, f0, g0, alpha1, c1, c2, max_evals, alpha_max=1e10, eps_f=1e-11):
    """Strong Wolfe step along a descent direction.  phi(alpha) -> (f, dphi, payload).
    Returns (alpha, f, payload, evals, ok)."""
    tol_f = eps_f * max(abs(f0), 1.0)        # below this, differences of f are rounding

    def decrease(a, fa, ga):
        if fa <= f0 + c1 * a * g0:
            return True
        return fa <= f0 + tol_f and ga <= (2.0 * c1 - 1.0) * g0

    evals = 0
    a_prev, f_prev, g_prev = 0.0, f0, g0
    alpha = alpha1
    best = (0.0, f0, None)

    def zoom(lo, flo, glo, hi, fhi, ghi):
        nonlocal evals, best
        while evals < max_evals:
            a = _cubic_min(lo, flo, glo, hi, fhi, ghi)
            left, right = min(lo, hi), max(lo, hi)
            margin = 0.1 * (right - left)
            if a is None or not (left + margin <= a <= right - margin):
                a = 0.5 * (lo + hi)
            fa, ga, pay = phi(a)
            evals += 1
            if fa < best[1]:
                best = (a, fa, pay)
            if not decrease(a, fa, ga) or fa > flo + tol_f:
                hi, fhi, ghi = a, fa, ga
            else:
                if abs(ga) <= -c2 * g0:
                    return a, fa, pay, True
                if ga * (hi - lo) >= 0.0:
                    hi, fhi, ghi = lo, flo, glo
                lo, flo, glo = a, fa, ga
        return best[0], best[1], best[2], False

    while evals < max_evals:
        f, g, pay = phi(alpha)
        evals += 1
        if f < best[1]:
            best = (alpha, f, pay)
        if not decrease(alpha, f, g) or (evals > 1 and f > f_prev + tol_f):
            a, fa, pa, ok = zoom(a_prev, f_prev, g_prev, alpha, f, g)
            return a, fa, pa, evals, ok
        if abs(g) <= -c2 * g0:
            return alpha, f, pay, evals, True
        if g >= 0.0:
            a, fa, pa, ok = zoom(alpha, f, g, a_prev, f_prev, g_prev)
            return a, fa, pa, evals, ok
        a_prev, f_prev, g_prev = alpha, f, g
        alpha = min(2.0 * alpha, alpha_max)
    return best[0], best[1], best[2], evals, False


def lbfgs_minimize(fun, x0, m=10, max_iter=100, gtol=1e-5, ftol=1e-10, c1=1e-4, c2=0.9,
                   max_ls=20, validation=None, patience=3, callback=None):
    """Minimise fun over x (1-D float64 array).  fun(x) -> (f, g).

    Returns at once with reason "eval_failed" when f or g is not finite at x0.
    Otherwise stops when max|g| <= gtol, when the relative decrease of f in an iteration is below
    ftol (ftol = 0: never), after max_iter iterations, when a line search fails, or (with validation(x)
    -> loss) after `patience` iterations without a new best validation loss; then the
    best-validated iterate is returned.  Returns a dict with x, f, g, nit, nfev, reason
    and history (f per iteration, and the validation loss when given).
    """
    x = np.array(x0, dtype=np.float64)
    f, g = fun(x)
    f = float(f)
    g = np.asarray(g, dtype=np.float64)
    nfev = 1
    S, Y = [], []
    hist = {"f": [f], "val": []}
    best_val, best_x, best_fg, since = math.inf, x.copy(), (f, g.copy()), 0
    if validation is not None:
        best_val = float(validation(x))
        hist["val"].append(best_val)
    reason = "max_iter"
    nit = 0
    if not (math.isfinite(f) and np.all(np.isfinite(g))):
        # the objective cannot be evaluated at the start: nothing to optimise
        return {"x": x, "f": f, "g": g, "nit": 0, "nfev": nfev, "reason": "eval_failed",
                "history": hist}
    for nit in range(1, max_iter + 1):
        if np.max(np.abs(g)) <= gtol:
            reason = "gtol"
            nit -= 1
            break
        # two-loop recursion: d = -H g
        q = g.copy()
        alphas = []
        for s, y in zip(reversed(S), reversed(Y)):
            a = (s @ q) / (y @ s)
            alphas.append(a)
            q -= a * y
        if S:
            q *= (S[-1] @ Y[-1]) / (Y[-1] @ Y[-1])
        else:
            q /= max(1.0, np.linalg.norm(g))          # first step of length <= 1
        for (s, y), a in zip(zip(S, Y), reversed(alphas)):
            b = (y @ q) / (y @ s)
            q += (a - b) * s
        d = -q
        gd = float(g @ d)
        if not gd < 0.0:                               # not a descent direction: reset
            S.clear()
            Y.clear()
            d = -g / max(1.0, np.linalg.norm(g))
            gd = float(g @ d)

        def phi(alpha):
            fx, gx = fun(x + alpha * d)
            gx = np.asarray(gx, dtype=np.float64)
            return float(fx), float(gx @ d), gx

        alpha, f_new, g_new, evals, ok = _wolfe_search(phi, f, gd, 1.0, c1, c2, max_ls)
        nfev += evals
        if g_new is None or alpha == 0.0:
            reason = "line_search"
            break
        s = alpha * d
        x_new = x + s
        y = g_new - g
        if s @ y > 1e-12 * np.linalg.norm(s) * np.linalg.norm(y):
            S.append(s)
            Y.append(y)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
        decrease = f - f_new
        x, f, g = x_new, f_new, g_new
        hist["f"].append(f)
        if callback is not None:
            callback(nit, x, f, g)
        if validation is not None:
            v = float(validation(x))
            hist["val"].append(v)
            if v < best_val:
                best_val, best_x, best_fg, since = v, x.copy(), (f, g.copy()), 0
            else:
                since += 1
                if since >= patience:
                    reason = "early_stop"
                    break
        if not ok:
            reason = "line_search"
            break
        if ftol > 0.0 and decrease <= ftol * max(1.0, abs(f)):
            reason = "ftol"
            break
    if validation is not None:
        x, (f, g) = best_x, best_fg
    return {"x": x, "f": f, "g": g, "nit": nit, "nfev": nfev, "reason": reason,
            "history": hist}


def lbfgs_fit(problem, y, theta0, k, n_probes, opts, max_iter=50, validation=None,
              patience=3, gtol=1e-4, m=10, callback=None):
    """Maximise the estimated MLL over log(theta) with lbfgs_minimize.

    problem: a gp.Problem (its theta is overwritten); y: targets; theta0: raw
    (l_1..l_D, s, sigma^2); opts: gp.opts, whose probe seed stays fixed for the run.
    validation(theta) -> loss (e.g. a held-out error) enables early stopping.  Returns
    (theta, result) with result as lbfgs_minimize's, for the objective -MLL in log space.
    In GP_BF16 precision with the default flags an evaluation may switch to split mode
    at some theta (a jump of the objective of up to ~5e-3 relative); GP_OPT_SPLIT_P or
    GP_OPT_FAST_ONLY in opts.flags keeps the objective one smooth function.
    """
    import torch

    from . import gp

    ws = gp.Workspace()

    def fun(phi):
        theta = np.exp(phi)
        problem.set_theta(theta)
        st, out, iout = gp.gp_mll_and_grad(problem, y, k, n_probes, opts, workspace=ws)
        r = gp.unpack(out, iout, problem.p, n_probes, k)
        # warnings (> 0: CG capped, rank-deficient preconditioner) still give results
        if st < 0 or r["status"] < 0 or not np.isfinite(r["mll"]):
            return math.inf, np.zeros_like(phi)
        # d(-mll)/d(log theta) = -theta * dmll/dtheta
        return -float(r["mll"]), -theta * np.asarray(r["grad"], dtype=np.float64)

    val = None if validation is None else (lambda phi: validation(np.exp(phi)))
    res = lbfgs_minimize(fun, np.log(np.asarray(theta0, dtype=np.float64)), m=m,
                         max_iter=max_iter, gtol=gtol, validation=val, patience=patience,
                         callback=callback)
    theta = np.exp(res["x"])
    problem.set_theta(theta)
    torch.cuda.synchronize()
    return theta, res
