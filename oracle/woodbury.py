"""Diagonal-plus-low-rank preconditioner P_hat = sigma^2 I + L L^T, FP64 (test infrastructure only).

Sec. 2.2 "Preconditioning": solves with P_hat in O(n k^2) by the matrix inversion
lemma; Alg. 1 step 3 needs log det P_hat; Alg. 2 step 3 needs tr(P_hat^-1 dP_hat).

    core      C = sigma^2 I_k + L^T L
    solve     P_hat^-1 V = sigma^-2 (V - L C^-1 L^T V)           (matrix inversion lemma)
    logdet    log det P_hat = (n - k) log sigma^2 + log det C    (determinant lemma)
    trace     tr(P_hat^-1 dP) = sigma^-2 sum_i dP_ii
                                - sigma^-2 1^T ((L C^-1) o (dP L)) 1      (eq. preconditioner_trace)

The last formula ends in "... ) 1" in the paper, which is a vector; the trace is the
sum of all entries of the Hadamard product, i.e. 1^T (A o B) 1 = tr(A^T B).

dP_hat / dtheta (the paper leaves it open).  Pivots are held fixed.  With the
pivots fixed, the rank-k pivoted Cholesky equals the Nystrom approximation
L L^T = C W^-1 C^T, C = K[:, piv], W = K[piv, piv], so by the product rule

    d(L L^T) = dC W^-1 C^T + C W^-1 dC^T - C W^-1 dW W^-1 C^T,  dW = dC[piv, :]

and dP_hat/dsigma^2 = I.  Here these are applied to vectors directly from C and W.
"""
import numpy as np

from . import kernels


def core(L, s2):
    k = L.shape[1]
    return s2 * np.eye(k) + L.T @ L


def solve(L, s2, V):
    V = np.asarray(V, np.float64)
    C = core(L, s2)
    return (V - L @ np.linalg.solve(C, L.T @ V)) / s2


def logdet(L, s2):
    n, k = L.shape
    sign, ld = np.linalg.slogdet(core(L, s2))
    assert sign > 0
    return (n - k) * np.log(s2) + ld


def dense(L, s2):
    return s2 * np.eye(L.shape[0]) + L @ L.T


class NystromDerivative:
    """dP_hat/dtheta_p at frozen pivots, applied matrix-free (p in the order of
    ``kernels.kernel_grad_blocks`` followed by the noise)."""

    def __init__(self, op, piv):
        self.op = op
        self.piv = np.asarray(piv, dtype=np.int64)
        self.n = op.n
        self.p = op.p
        if len(self.piv) == 0:
            self.C = np.zeros((self.n, 0))
            self.W = np.zeros((0, 0))
            self.dC = [np.zeros((self.n, 0)) for _ in range(self.p - 1)]
        else:
            self.C = kernels.kernel_block(op.kind, op.X, op.X[self.piv], op.theta, op.ard)
            self.W = self.C[self.piv, :]
            self.dC = op.grad_columns(self.piv)
        self.dW = [dc[self.piv, :] for dc in self.dC]

    def _Winv(self, M):
        if self.W.shape[0] == 0:
            return M
        return np.linalg.solve(self.W, M)

    def apply(self, q, V):
        V = np.asarray(V, np.float64)
        if q == self.p - 1:                       # noise: dP/dsigma^2 = I
            return V.copy()
        C, dC, dW = self.C, self.dC[q], self.dW[q]
        WiCtV = self._Winv(C.T @ V)
        return (dC @ WiCtV + C @ self._Winv(dC.T @ V)
                - C @ self._Winv(dW @ WiCtV))

    def diag(self, q):
        if q == self.p - 1:
            return np.ones(self.n)
        C, dC, dW = self.C, self.dC[q], self.dW[q]
        WiCt = self._Winv(C.T)                    # k x n
        term1 = np.sum(dC * WiCt.T, axis=1)       # (dC W^-1 C^T)_ii
        term3 = np.sum((C @ self._Winv(dW)) * WiCt.T, axis=1)
        return 2.0 * term1 - term3

    def dense(self, q):
        return self.apply(q, np.eye(self.n))


def precond_trace(L, s2, dP_apply, dP_diag):
    """tr(P_hat^-1 dP_hat) by eq. (preconditioner_trace), read as a full sum."""
    if L.shape[1] == 0:
        return float(np.sum(dP_diag)) / s2
    C = core(L, s2)
    LCinv = np.linalg.solve(C, L.T).T              # L C^-1 (C symmetric)
    dPL = dP_apply(L)
    return float(np.sum(dP_diag)) / s2 - float(np.sum(LCinv * dPL)) / s2


def nystrom_dense(op, piv, s2):
    """P_hat = sigma^2 I + C W^-1 C^T rebuilt from the kernel at frozen pivots."""
    piv = np.asarray(piv, dtype=np.int64)
    C = kernels.kernel_block(op.kind, op.X, op.X[piv], op.theta, op.ard)
    W = C[piv, :]
    return s2 * np.eye(op.n) + C @ np.linalg.solve(W, C.T)
