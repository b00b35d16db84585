"""Pins for oracle/woodbury.py.

* P^-1 V and log det P against a dense solve / dense slogdet of sigma^2 I + L L^T.
* dP/dtheta at frozen pivots (applied and its diagonal) against a central finite
  difference of the dense Nystrom preconditioner rebuilt at theta +- h.
* tr(P^-1 dP) by eq. (preconditioner_trace) against the dense trace of
  P^-1 (finite-difference dP).
* For the output scale, dP/ds = L L^T / s exactly (pivots are scale invariant).
"""
import numpy as np
import pytest

from oracle import kernels, pivchol, woodbury


def _setup(kind, ard, k=7, n=50, seed=0):
    rng = np.random.default_rng(seed)
    d = 2
    X = rng.uniform(size=(n, d))
    D = d if ard else 1
    theta = np.concatenate([rng.uniform(0.4, 0.9, D), [1.1, 0.03]])
    op = kernels.KernelOperator(kind, X, theta, ard)
    L, piv, rank, _ = pivchol.pivoted_cholesky(op, k)
    return op, L, piv


@pytest.mark.parametrize("k", [0, 3, 9])
def test_solve_and_logdet_match_dense(k):
    op, L, piv = _setup(kernels.RBF, True, k=k)
    P = woodbury.dense(L, op.s2)
    V = np.random.default_rng(1).standard_normal((op.n, 4))
    np.testing.assert_allclose(woodbury.solve(L, op.s2, V), np.linalg.solve(P, V),
                               rtol=1e-10, atol=1e-10)
    sign, ld = np.linalg.slogdet(P)
    assert abs(woodbury.logdet(L, op.s2) - ld) < 1e-10 * abs(ld)


def _fd_dP(op, piv, q, h_rel=1e-6):
    theta = op.theta
    if q == op.p - 1:
        return np.eye(op.n)
    h = h_rel * theta[q]
    mats = []
    for sgn in (+1, -1):
        t = theta.copy()
        t[q] += sgn * h
        o = kernels.KernelOperator(op.kind, op.X, t, op.ard)
        mats.append(woodbury.nystrom_dense(o, piv, op.s2))
    return (mats[0] - mats[1]) / (2 * h)


@pytest.mark.parametrize("kind", kernels.KINDS)
@pytest.mark.parametrize("ard", [True, False])
def test_nystrom_derivative_matches_fd(kind, ard):
    op, L, piv = _setup(kind, ard)
    nd = woodbury.NystromDerivative(op, piv)
    for q in range(op.p):
        fd = _fd_dP(op, piv, q)
        got = nd.dense(q)
        scale = np.abs(fd).max()
        np.testing.assert_allclose(got, fd, atol=2e-6 * scale)
        np.testing.assert_allclose(nd.diag(q), np.diag(fd), atol=2e-6 * scale)


def test_outputscale_derivative_is_LLt_over_s():
    op, L, piv = _setup(kernels.MATERN32, True)
    nd = woodbury.NystromDerivative(op, piv)
    q = op.p - 2
    np.testing.assert_allclose(nd.dense(q), L @ L.T / op.s, atol=1e-10)


@pytest.mark.parametrize("kind", kernels.KINDS)
def test_precond_trace_matches_dense(kind):
    op, L, piv = _setup(kind, True, k=6)
    nd = woodbury.NystromDerivative(op, piv)
    P = woodbury.dense(L, op.s2)
    for q in range(op.p):
        fd = _fd_dP(op, piv, q)
        ref = np.trace(np.linalg.solve(P, fd))
        got = woodbury.precond_trace(L, op.s2, lambda V: nd.apply(q, V), nd.diag(q))
        assert abs(got - ref) <= 1e-5 * max(1.0, abs(ref)), (q, got, ref)


def test_precond_trace_rank_zero():
    op, L, piv = _setup(kernels.RBF, True, k=0)
    nd = woodbury.NystromDerivative(op, piv)
    q = op.p - 1
    assert abs(woodbury.precond_trace(L, op.s2, lambda V: nd.apply(q, V), nd.diag(q))
               - op.n / op.s2) < 1e-9
