"""Lanczos tridiagonal from CG coefficients and Lanczos quadrature, FP64 (test infrastructure only).

Sec. S1.2 "Lanczos Algorithm": the tridiagonal T can be formed from the CG step
lengths alpha_j and corrections beta_j (Saad 2003, Sec. 6.7.3).  For m CG steps:

    T[j, j]     = 1/alpha_j + beta_{j-1}/alpha_{j-1}     (second term absent at j = 0)
    T[j, j + 1] = sqrt(beta_j) / alpha_j                 (j = 0 .. m-2)

m nodes are used; a beta of a step that did not finish is not used.

Alg. 1 steps 6-8 (Lanczos quadrature, Golub & Meurant 2009 Ch. 7): with
T = W diag(lambda) W^T, weights omega_j = (e_1^T w_j)^2 and
    e_1^T log(T) e_1 = sum_j omega_j log(lambda_j).
Preconditioned CG from b is Lanczos on P^-1/2 K_hat P^-1/2 from the unit vector
P^-1/2 b / sqrt(rho_0), rho_0 = b^T P^-1 b, so
    (P^-1/2 b)^T log(P^-1/2 K_hat P^-1/2) (P^-1/2 b) ~= rho_0 * e_1^T log(T) e_1.
The eigendecomposition of the small dense T is a library call.
"""
import numpy as np


def tridiag_from_cg(alpha, beta, m):
    alpha = np.asarray(alpha, np.float64)
    beta = np.asarray(beta, np.float64)
    diag = np.zeros(m)
    off = np.zeros(max(m - 1, 0))
    for j in range(m):
        diag[j] = 1.0 / alpha[j]
        if j > 0:
            diag[j] += beta[j - 1] / alpha[j - 1]
        if j < m - 1:
            off[j] = np.sqrt(beta[j]) / alpha[j]
    return diag, off


def dense_tridiag(diag, off):
    T = np.diag(diag)
    if len(off):
        T += np.diag(off, 1) + np.diag(off, -1)
    return T


def quadrature(diag, off, f=np.log):
    """e_1^T f(T) e_1 = sum_j (e_1^T w_j)^2 f(lambda_j)."""
    if len(diag) == 0:
        return 0.0
    lam, W = np.linalg.eigh(dense_tridiag(diag, off))
    return float(np.sum(W[0, :] ** 2 * f(lam)))
