"""Greedy partial pivoted Cholesky, FP64 (test infrastructure only).

The paper uses a "partial Cholesky" preconditioner P_hat = sigma^2 I + L_k L_k^T
(Sec. 2.2 "Preconditioning"; Prop. "Cholesky approximation quality", which cites
Harbrecht et al. 2012 for the greedy pivoted algorithm and its trace-error rate).
The algorithm itself is not printed.  This is the textbook greedy form:

    d_i = k(x_i, x_i)                                  (noise-free diagonal)
    for m = 0 .. k-1:
        stop if sum_i d_i <= tol * tr(K)                (residual-trace tolerance)
        pi_m = argmax over not-yet-chosen i of d_i     (lowest index on exact ties)
        stop if d_{pi_m} <= floor * max_i K_ii          (rank deficient)
        L[:, m] = (K[:, pi_m] - L[:, :m] L[pi_m, :m]^T) / sqrt(d_{pi_m})
        L[pi_j, m] = 0 for the earlier pivots j < m;  L[pi_m, m] = sqrt(d_{pi_m})
        d_i = max(d_i - L[i, m]^2, 0);  d_{pi_m} = 0

The preconditioner approximates K without noise, so P_hat = sigma^2 I + L L^T.
The zero entries of L at earlier pivots hold exactly in exact arithmetic (the
residual at a chosen pivot is zero); they are set explicitly.

The paper does not say when a numerically rank-deficient K stops the factor.  With
floor = 0 (the default) only a residual that is exactly zero or negative stops it.
A caller that forms L in a precision with unit roundoff u passes floor = n u, the
default rank rule of LAPACK's pivoted Cholesky (xPSTRF): below it the residual is
rounding error of the earlier columns.
"""
import numpy as np


def pivoted_cholesky(op, k, tol=0.0, piv_override=None, floor=0.0):
    """Rank-k greedy pivoted Cholesky of the noise-free kernel matrix.

    ``op`` is an ``oracle.kernels.KernelOperator``.  Returns (L [n x rank],
    piv [rank], rank, residual_traces [rank + 1]).
    """
    n = op.n
    k = int(min(k, n))
    d = op.diag().astype(np.float64).copy()
    trace0 = float(np.sum(d))
    dmin = float(floor) * float(np.max(d)) if n > 0 else 0.0
    L = np.zeros((n, k))
    chosen = np.zeros(n, dtype=bool)
    piv = []
    traces = [trace0]
    rank = 0
    for m in range(k):
        if np.sum(d) <= tol * trace0:
            break
        if piv_override is not None:
            pm = int(piv_override[m])
        else:
            cand = np.where(chosen, -np.inf, d)
            pm = int(np.argmax(cand))            # numpy returns the first maximum
        dm = d[pm]
        if not dm > 0.0 or dm <= dmin:
            break
        root = np.sqrt(dm)
        col = op.column(pm) - L[:, :m] @ L[pm, :m]
        col = col / root
        col[chosen] = 0.0
        col[pm] = root
        L[:, m] = col
        d = np.maximum(d - col * col, 0.0)
        d[pm] = 0.0
        chosen[pm] = True
        piv.append(pm)
        rank = m + 1
        traces.append(float(np.sum(d)))
    return L[:, :rank].copy(), np.array(piv, dtype=np.int64), rank, np.array(traces)
