"""Preconditioned conjugate gradients on many right-hand sides, FP64 (test infrastructure only).

Sec. 2.2 "Conjugate Gradient Method" / "Preconditioning" and the footnote to Sec. 4.4:
all probe vectors and y are solved in one CG call with several right-hand sides.
Each column is an independent preconditioned CG (Hestenes & Stiefel 1952) that
needs only products with K_hat and solves with P_hat:

    x_0 = 0, r_0 = b, z_0 = P^-1 r_0, p_0 = z_0, rho_0 = r_0^T z_0
    for j = 0, 1, ...:
        q = K_hat p_j;  alpha_j = rho_j / (p_j^T q)
        x += alpha_j p_j;  r -= alpha_j q
        every R-th iteration (R = recompute_every > 0): r = b - K_hat x
        stop the column if ||r||_2 <= tol ||b||_2, or j + 1 == max_iter
            (with a per-column iteration override: stop exactly when j + 1 == cap)
        z = P^-1 r;  rho_{j+1} = r^T z;  beta_j = rho_{j+1} / rho_j
        p_{j+1} = z + beta_j p_j

A column with b = 0 (or an override of 0) takes no step.  The step lengths alpha_j
and corrections beta_j are kept for the Lanczos tridiagonal (Sec. S1.2, citing
Saad 2003 Sec. 6.7.3); so are rho_0 = b^T P^-1 b and z_0 = P^-1 b, which the
estimator needs.  The stopping rule and norm are not stated in the paper; this is
the unpreconditioned relative 2-norm residual.
"""
import numpy as np


def mbcg(matvec, precond, B, tol, max_iter, recompute_every=0, iters_override=None):
    B = np.asarray(B, np.float64)
    n, t = B.shape
    X = np.zeros((n, t))
    R = B.copy()
    Z = precond(R)
    P = Z.copy()
    rho = np.sum(R * Z, axis=0)
    z0 = Z.copy()
    rho0 = rho.copy()
    bnorm = np.linalg.norm(B, axis=0)
    if iters_override is not None:
        caps = np.minimum(np.asarray(iters_override, dtype=np.int64), max_iter)
        active = caps > 0
    else:
        caps = np.full(t, max_iter, dtype=np.int64)
        active = bnorm > 0
    alpha = np.zeros((t, max_iter))
    beta = np.zeros((t, max_iter))
    iters = np.zeros(t, dtype=np.int64)
    for j in range(max_iter):
        if not active.any():
            break
        act = np.flatnonzero(active)
        Q = matvec(P[:, act])
        a = rho[act] / np.sum(P[:, act] * Q, axis=0)
        alpha[act, j] = a
        X[:, act] += a * P[:, act]
        R[:, act] -= a * Q
        if recompute_every > 0 and (j + 1) % recompute_every == 0:
            R[:, act] = B[:, act] - matvec(X[:, act])
        if iters_override is not None:
            stop = (j + 1) >= caps[act]
        else:
            stop = (np.linalg.norm(R[:, act], axis=0) <= tol * bnorm[act]) | (j + 1 >= max_iter)
        iters[act[stop]] = j + 1
        active[act[stop]] = False
        cont = act[~stop]
        if cont.size == 0:
            continue
        Zc = precond(R[:, cont])
        rho_new = np.sum(R[:, cont] * Zc, axis=0)
        b = rho_new / rho[cont]
        beta[cont, j] = b
        P[:, cont] = Zc + b * P[:, cont]
        rho[cont] = rho_new
    return {
        "X": X, "alpha": alpha, "beta": beta, "iters": iters,
        "rho0": rho0, "z0": z0, "bnorm": bnorm, "R": R,
    }
