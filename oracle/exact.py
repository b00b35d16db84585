"""Exact log-marginal likelihood and gradient by dense Cholesky, FP64 (test infrastructure only).

Sec. 2.1, eq. (likelihood):
    L(theta) = -1/2 ( y^T K_hat^-1 y + log det K_hat + n log 2 pi )
Sec. 2.1, eq. (derivative_likelihood):
    dL/dtheta_p = 1/2 y^T K_hat^-1 dK_hat_p K_hat^-1 y - 1/2 tr(K_hat^-1 dK_hat_p)

This is the quantity the stochastic estimator (``estimator.py``) approximates.
Feasible for n up to a few thousand.
"""
import numpy as np

from . import kernels


def exact_mll_and_grad(kind, X, y, theta, ard):
    X = np.asarray(X, np.float64)
    y = np.asarray(y, np.float64)
    n = X.shape[0]
    Khat = kernels.khat_dense(kind, X, theta, ard)
    G = np.linalg.cholesky(Khat)                     # K_hat = G G^T
    u = np.linalg.solve(G.T, np.linalg.solve(G, y))  # u = K_hat^-1 y
    logdet = 2.0 * np.sum(np.log(np.diag(G)))
    quad = float(y @ u)
    mll = -0.5 * (quad + logdet + n * np.log(2.0 * np.pi))
    Ginv = np.linalg.solve(G, np.eye(n))
    Kinv = Ginv.T @ Ginv
    grads, quad_p, trace_p = [], [], []
    for dK in kernels.dkhat_dense(kind, X, theta, ard):
        qp = 0.5 * float(u @ dK @ u)
        tp = float(np.sum(Kinv * dK))                # tr(K^-1 dK) for symmetric dK
        quad_p.append(qp)
        trace_p.append(tp)
        grads.append(qp - 0.5 * tp)
    return {
        "mll": float(mll),
        "grad": np.array(grads),
        "quad": quad,
        "logdet": float(logdet),
        "quad_p": np.array(quad_p),
        "trace_p": np.array(trace_p),
        "u": u,
    }
