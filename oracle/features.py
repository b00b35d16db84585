"""Random Fourier feature preconditioner, FP64 (test infrastructure only).

Tab. 2 of the paper lists random Fourier features (RFF; Prop. "RFF approximation
quality", after Rahimi and Recht 2007) as a diagonal-plus-low-rank preconditioner
P_hat = sigma^2 I + Phi Phi^T whose error decays like k^-1/2 with high probability.
The features are not printed; this is the standard paired form.  By Bochner's theorem a
stationary kernel is k(x - y) = s E_w[cos(w . (x - y))] with w drawn from its spectral
density, and cos(a - b) = cos a cos b + sin a sin b, so with m frequencies w_j

    Phi[a, j] = sqrt(s / m) cos(w_j . x_a),   Phi[a, m + j] = sqrt(s / m) sin(w_j . x_a)

(k = 2m features) gives E[Phi Phi^T] = K.  The spectral densities, written as scale
mixtures of the Gaussian N(0, diag(l)^-2) with w_j = rho_j eps_j / l (elementwise),
eps_j ~ N(0, I_d):
    RBF                        rho = 1
    Matern-nu (nu = 3/2, 5/2)  rho = sqrt(nu / g_j), g_j ~ Gamma(nu, 1)
                               (a multivariate t with 2 nu degrees of freedom)
    rational quadratic, alpha = 1   rho = sqrt(g_j), g_j ~ Gamma(1, 1)
                               (1 / (1 + r^2 / 2) = E_g[exp(-g r^2 / 2)])
The random draws (eps, g) are inputs, so the oracle and the CUDA path see the same
frequencies.  The paper fixes no origin for x: shifting every x by c turns each
(cos, sin) pair by the angle u_j . c, which leaves Phi Phi^T (so P_hat) unchanged but
changes the probes Phi eps_1.  The features are taken at x~ = (x - mean x) / l, the
inputs' own mean as the origin (the CUDA path centres its inputs the same way).

The gradient's preconditioner terms need dP_hat/dtheta at frozen draws (the analogue
of the partial Cholesky's frozen pivots):
    dPhi/dl_i: with u_j = rho_j eps_j and x~ = (x - mean x) / l, arg = u_j . x~ and
               d arg / d l_i = -u_ji x~_i / l_i, so d cos = sin u_ji x~_i / l_i and
               d sin = -cos u_ji x~_i / l_i (an isotropic l sums over i: -arg / l);
    dPhi/ds  = Phi / (2 s);
    dP_hat   = dPhi Phi^T + Phi dPhi^T (noise: the identity).
"""
import numpy as np

from . import kernels


def gamma_shape(kind):
    """Shape of the Gamma draws g_j the kernel's spectral density needs (None: RBF)."""
    return {kernels.RBF: None, kernels.MATERN32: 1.5, kernels.MATERN52: 2.5,
            kernels.RATQUAD: 1.0}[kind]


def frequencies(kind, eps, g):
    """u_j = rho_j eps_j: the frequencies in units of 1 / l (m x d)."""
    eps = np.asarray(eps, np.float64)
    if kind == kernels.RBF:
        rho = np.ones(eps.shape[0])
    elif kind == kernels.RATQUAD:
        rho = np.sqrt(np.asarray(g, np.float64))
    else:
        rho = np.sqrt(gamma_shape(kind) / np.asarray(g, np.float64))
    return rho[:, None] * eps


def hermite_grid(mbar, d):
    """Quadrature Fourier features (Tab. 2 "QFF", Prop. "QFF approximation quality",
    after Mutny and Krause 2018) for the RBF kernel: E_w[cos(w . D)] with w ~ N(0, I_d)
    by the tensor-product Gauss-Hermite rule of mbar nodes per dimension (numpy's
    hermgauss, weight exp(-t^2)): w = sqrt(2) t, weight prod_i w_i / sqrt(pi).  The rule
    is symmetric, and w and -w give the same cos(w . D), so each pair is kept once with
    twice the weight (mbar even: no zero node).  Returns (U, weights): mbar^d / 2
    frequencies in units of 1 / l and their weights, which sum to 1."""
    if mbar % 2:
        raise ValueError("mbar must be even")
    t, w = np.polynomial.hermite.hermgauss(mbar)
    grids = np.meshgrid(*([np.sqrt(2.0) * t] * d), indexing="ij")
    U = np.stack([g.reshape(-1) for g in grids], axis=1)
    W = np.ones(U.shape[0])
    for wi in np.meshgrid(*([w / np.sqrt(np.pi)] * d), indexing="ij"):
        W = W * wi.reshape(-1)
    # keep the half with a positive first nonzero coordinate (none is zero: mbar even)
    keep = U[:, 0] > 0
    return U[keep], 2.0 * W[keep]


class RandomFourier:
    """Phi (n x 2m) and its derivatives for the hyperparameters theta (the order of
    ``kernels.kernel_grad_blocks`` followed by the noise).  With ``eps, g`` the random
    features above (weights 1/m); with ``U, weights`` given instead, any weighted
    frequency set (the quadrature features of ``hermite_grid``)."""

    def __init__(self, kind, X, theta, ard, eps=None, g=None, U=None, weights=None):
        self.X = np.asarray(X, np.float64)
        self.n, self.d = self.X.shape
        self.ard = ard
        self.ls, self.s, self.s2 = kernels.unpack(theta, self.d, ard)
        self.p = kernels.n_hyper(self.d, ard)
        if U is None:
            self.U = frequencies(kind, eps, g)                  # m x d
            weights = np.full(self.U.shape[0], 1.0 / self.U.shape[0])
        else:
            self.U = np.asarray(U, np.float64)
        self.m = self.U.shape[0]
        # x~ = (x - mean x) / l: the origin of the features is the input mean (any fixed
        # shift rotates each cos / sin pair and leaves Phi Phi^T unchanged)
        self.Xs = (self.X - self.X.mean(axis=0)) / self.ls
        arg = self.Xs @ self.U.T                                # n x m
        self.amp = np.sqrt(self.s * np.asarray(weights, np.float64))[None, :]
        self.cos, self.sin = np.cos(arg), np.sin(arg)
        self.arg = arg
        self.Phi = np.hstack([self.amp * self.cos, self.amp * self.sin])

    def dphi(self, q):
        """dPhi / dtheta_q (n x 2m) for q < p - 1."""
        nls = kernels.n_lengthscales(self.d, self.ard)
        if q == nls:                                            # output scale
            return self.Phi / (2.0 * self.s)
        if self.ard:
            # d arg / d l_q = -u_jq x~_q / l_q
            darg = -(self.Xs[:, q][:, None] * self.U[:, q][None, :]) / self.ls[q]
        else:
            darg = -self.arg / self.ls[0]
        return np.hstack([-self.amp * self.sin * darg, self.amp * self.cos * darg])

    def apply(self, q, V):
        """dP_hat / dtheta_q @ V."""
        V = np.asarray(V, np.float64)
        if q == self.p - 1:
            return V.copy()
        dP = self.dphi(q)
        return dP @ (self.Phi.T @ V) + self.Phi @ (dP.T @ V)

    def diag(self, q):
        if q == self.p - 1:
            return np.ones(self.n)
        return 2.0 * np.sum(self.dphi(q) * self.Phi, axis=1)

    def dense(self, q):
        return self.apply(q, np.eye(self.n))
