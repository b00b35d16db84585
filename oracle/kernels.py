"""Kernel functions and hyperparameter derivatives, FP64 (test infrastructure only).

Sec. 5 "Experimental Setup" of the paper: RBF and Matern(3/2) kernels with an output
scale, one lengthscale per input dimension (ARD) and a noise variance sigma^2; the
kernel matrix with noise is K_hat = K + sigma^2 I (Sec. 2.1).  The paper does not
print the kernel formulas.  The forms used here are the textbook ones
(Rasmussen & Williams 2006, eqs. 4.9 and 4.17), with the output scale ``s`` equal
to k(x, x) (the paper writes o^2 = k(0) in Prop. "Cholesky approximation quality"):

    r^2      = sum_j ((x_j - x'_j) / l_j)^2
    RBF      k = s exp(-r^2 / 2)
    Matern32 k = s (1 + sqrt(3) r) exp(-sqrt(3) r)
    Matern52 k = s (1 + sqrt(5) r + 5 r^2 / 3) exp(-sqrt(5) r)
    RatQuad  k = s (1 + r^2 / (2 alpha))^-alpha with alpha = 1, i.e. s / (1 + r^2 / 2)
             (Rasmussen & Williams 2006, eq. 4.19; the paper's RatQuad kernel, Tab. S1,
             does not state alpha: it is read as 1 and held fixed, not a hyperparameter)

Hyperparameters are theta = (l_1..l_D, s, sigma^2) with D = d (ARD) or 1
(isotropic).  Derivatives are taken with respect to these raw values.

Derivative with respect to a lengthscale: d r^2 / d l_j = -2 (dx_j)^2 / l_j^3, so
d k / d l_j = -2 (dk/d r^2) (dx_j)^2 / l_j^3.  ``neg2_dk_dr2`` below is the factor
-2 dk/dr^2, written per kernel from the closed forms above:

    RBF      -2 dk/dr^2 = s exp(-r^2/2)
    Matern32 -2 dk/dr^2 = 3 s exp(-sqrt(3) r)
    Matern52 -2 dk/dr^2 = (5/3) s (1 + sqrt(5) r) exp(-sqrt(5) r)
    RatQuad  -2 dk/dr^2 = s (1 + r^2/2)^-2

(For Matern: dk/dr = -s a^2 r exp(-a r) with a = sqrt(3), resp.
-s (a^2/3) r (1 + a r) exp(-a r) with a = sqrt(5); dividing by dr^2/dr = 2 r gives
the factors above, which stay finite at r = 0.)
"""
import numpy as np

RBF = 0
MATERN32 = 3
MATERN52 = 5
RATQUAD = 7
KINDS = (RBF, MATERN32, MATERN52, RATQUAD)


def n_lengthscales(d, ard):
    return d if ard else 1


def n_hyper(d, ard):
    """Number of hyperparameters p = #lengthscales + outputscale + noise."""
    return n_lengthscales(d, ard) + 2


def unpack(theta, d, ard):
    theta = np.asarray(theta, dtype=np.float64)
    D = n_lengthscales(d, ard)
    assert theta.shape == (D + 2,), (theta.shape, D)
    lengthscales = np.broadcast_to(theta[:D], (d,)).copy()
    return lengthscales, float(theta[D]), float(theta[D + 1])


def k_of_r2(kind, r2, s):
    """Kernel value as a function of the scaled squared distance r^2."""
    r2 = np.maximum(r2, 0.0)
    if kind == RBF:
        return s * np.exp(-0.5 * r2)
    if kind == RATQUAD:
        return s / (1.0 + 0.5 * r2)
    r = np.sqrt(r2)
    if kind == MATERN32:
        a = np.sqrt(3.0)
        return s * (1.0 + a * r) * np.exp(-a * r)
    if kind == MATERN52:
        a = np.sqrt(5.0)
        return s * (1.0 + a * r + (5.0 / 3.0) * r2) * np.exp(-a * r)
    raise ValueError(kind)


def neg2_dk_dr2(kind, r2, s):
    """-2 dk/dr^2: the common factor of every lengthscale derivative."""
    r2 = np.maximum(r2, 0.0)
    if kind == RBF:
        return s * np.exp(-0.5 * r2)
    if kind == RATQUAD:
        return s / (1.0 + 0.5 * r2) ** 2
    r = np.sqrt(r2)
    if kind == MATERN32:
        a = np.sqrt(3.0)
        return 3.0 * s * np.exp(-a * r)
    if kind == MATERN52:
        a = np.sqrt(5.0)
        return (5.0 / 3.0) * s * (1.0 + a * r) * np.exp(-a * r)
    raise ValueError(kind)


def scaled_r2(Xa, Xb, lengthscales):
    """r^2 between every row of Xa and every row of Xb, straight from differences."""
    Xa = np.asarray(Xa, np.float64)
    Xb = np.asarray(Xb, np.float64)
    r2 = np.zeros((Xa.shape[0], Xb.shape[0]))
    for j in range(Xa.shape[1]):
        diff = (Xa[:, j][:, None] - Xb[:, j][None, :]) / lengthscales[j]
        r2 += diff * diff
    return r2


def kernel_block(kind, Xa, Xb, theta, ard):
    """Noise-free kernel block K[a, b] = k(x_a, x_b)."""
    d = np.asarray(Xa).shape[1]
    ls, s, _ = unpack(theta, d, ard)
    return k_of_r2(kind, scaled_r2(Xa, Xb, ls), s)


def kernel_grad_blocks(kind, Xa, Xb, theta, ard):
    """d K / d theta_p on a block, for every hyperparameter except the noise.

    Returns a list: one block per lengthscale, then the output-scale block.
    (The noise derivative of K_hat is the identity; callers add it where the
    block touches the diagonal.)
    """
    Xa = np.asarray(Xa, np.float64)
    Xb = np.asarray(Xb, np.float64)
    d = Xa.shape[1]
    ls, s, _ = unpack(theta, d, ard)
    r2 = scaled_r2(Xa, Xb, ls)
    g = neg2_dk_dr2(kind, r2, s)
    blocks = []
    if ard:
        for j in range(d):
            dx2 = (Xa[:, j][:, None] - Xb[:, j][None, :]) ** 2
            blocks.append(g * dx2 / ls[j] ** 3)
    else:
        # isotropic: sum_j (dx_j)^2 / l^3 = r^2 / l
        blocks.append(g * r2 / ls[0])
    blocks.append(k_of_r2(kind, r2, s) / s)
    return blocks


def khat_dense(kind, X, theta, ard):
    d = np.asarray(X).shape[1]
    _, _, s2 = unpack(theta, d, ard)
    K = kernel_block(kind, X, X, theta, ard)
    return K + s2 * np.eye(K.shape[0])


def dkhat_dense(kind, X, theta, ard):
    """All p derivative matrices d K_hat / d theta_p (noise last: the identity)."""
    blocks = kernel_grad_blocks(kind, X, X, theta, ard)
    blocks.append(np.eye(np.asarray(X).shape[0]))
    return blocks


class KernelOperator:
    """Matrix-free v -> K_hat v and v -> dK_hat/dtheta_p v (Sec. 2.2: CG only needs
    products with K_hat).  Rows are formed in blocks only to bound memory; each
    block is the plain definition above."""

    def __init__(self, kind, X, theta, ard, block_entries=1 << 24):
        self.kind = kind
        self.X = np.asarray(X, np.float64)
        self.theta = np.asarray(theta, np.float64)
        self.ard = ard
        self.n, self.d = self.X.shape
        self.ls, self.s, self.s2 = unpack(self.theta, self.d, ard)
        self.p = n_hyper(self.d, ard)
        self.rows = max(1, min(self.n, block_entries // max(1, self.n)))
        self._dense = None
        if self.n <= 2048:
            self._dense = khat_dense(kind, self.X, self.theta, ard)

    def _blocks(self):
        for a0 in range(0, self.n, self.rows):
            yield a0, min(self.n, a0 + self.rows)

    def matvec(self, V):
        V = np.asarray(V, np.float64)
        if self._dense is not None:
            return self._dense @ V
        out = np.empty_like(V)
        for a0, a1 in self._blocks():
            Kb = kernel_block(self.kind, self.X[a0:a1], self.X, self.theta, self.ard)
            out[a0:a1] = Kb @ V
        return out + self.s2 * V

    def grad_matvec(self, V):
        """[dK_hat/dtheta_p @ V for p in range(p)] (noise block = V itself)."""
        V = np.asarray(V, np.float64)
        outs = [np.empty_like(V) for _ in range(self.p - 1)]
        for a0, a1 in self._blocks():
            blocks = kernel_grad_blocks(self.kind, self.X[a0:a1], self.X, self.theta, self.ard)
            for q, B in enumerate(blocks):
                outs[q][a0:a1] = B @ V
        outs.append(V.copy())
        return outs

    def column(self, j):
        """Noise-free kernel column K[:, j]."""
        return kernel_block(self.kind, self.X, self.X[j:j + 1], self.theta, self.ard)[:, 0]

    def diag(self):
        """Noise-free kernel diagonal k(x_i, x_i)."""
        return k_of_r2(self.kind, np.zeros(self.n), self.s)

    def grad_columns(self, idx):
        """d K[:, idx] / d theta_p for lengthscales and output scale: list of N x len(idx)."""
        return kernel_grad_blocks(self.kind, self.X, self.X[idx], self.theta, self.ard)
