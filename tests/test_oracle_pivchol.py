"""Pins for oracle/pivchol.py.

* Full rank (k = n): L L^T = K, and L[piv] is the Cholesky factor of the
  symmetrically permuted K (numpy's Cholesky).
* Any rank: L L^T equals the Nystrom approximation K[:, piv] K[piv, piv]^-1 K[piv, :]
  (Schur-complement identity).
* Greedy rule by brute force: each pivot maximises the diagonal of the dense
  Schur complement K - L_m L_m^T (lowest index on ties).
* The residual trace tr(K - L L^T) is non-increasing and, for a 1-D RBF kernel,
  decays roughly exponentially in k (Prop. "Cholesky approximation quality").
"""
import numpy as np
import pytest

from oracle import kernels, pivchol
from paper_2107_00243_gb300 import workloads


def _op(n, d, kind=kernels.RBF, seed=0, ls=0.5):
    rng = np.random.default_rng(seed)
    X = rng.uniform(size=(n, d))
    theta = np.concatenate([np.full(d, ls), [1.2, 0.01]])
    return kernels.KernelOperator(kind, X, theta, True)


@pytest.mark.parametrize("kind", kernels.KINDS)
def test_full_rank_is_cholesky_of_permuted_K(kind):
    op = _op(25, 2, kind, ls=0.3)
    K = kernels.kernel_block(kind, op.X, op.X, op.theta, True)
    L, piv, rank, _ = pivchol.pivoted_cholesky(op, 25)
    if rank < 25:
        pytest.skip("numerically rank deficient")
    np.testing.assert_allclose(L @ L.T, K, atol=1e-10)
    G = np.linalg.cholesky(K[np.ix_(piv, piv)])
    np.testing.assert_allclose(L[piv], G, atol=1e-8)


@pytest.mark.parametrize("k", [1, 5, 12])
def test_low_rank_equals_nystrom(k):
    op = _op(60, 3, kernels.MATERN32, seed=1)
    K = kernels.kernel_block(op.kind, op.X, op.X, op.theta, True)
    L, piv, rank, _ = pivchol.pivoted_cholesky(op, k)
    C = K[:, piv]
    W = K[np.ix_(piv, piv)]
    np.testing.assert_allclose(L @ L.T, C @ np.linalg.solve(W, C.T), atol=1e-10)


def test_greedy_rule_brute_force():
    op = _op(40, 2, kernels.MATERN52, seed=2)
    K = kernels.kernel_block(op.kind, op.X, op.X, op.theta, True)
    L, piv, rank, _ = pivchol.pivoted_cholesky(op, 15)
    chosen = []
    for m in range(rank):
        S = K - L[:, :m] @ L[:, :m].T
        dS = np.diag(S).copy()
        dS[chosen] = -np.inf
        best = dS.max()
        # the pick must attain the maximum up to rounding, lowest index among equals
        assert dS[piv[m]] >= best - 1e-12
        ties = np.flatnonzero(dS >= best - 1e-12)
        assert piv[m] == ties[0] or abs(dS[ties[0]] - dS[piv[m]]) <= 1e-12
        chosen.append(piv[m])
    assert piv[0] == 0        # all diagonals equal s at step 0: lowest index


def test_residual_trace_monotone_and_exponential_in_1d():
    op = _op(400, 1, kernels.RBF, seed=3, ls=0.3)
    K = kernels.kernel_block(op.kind, op.X, op.X, op.theta, True)
    L, piv, rank, traces = pivchol.pivoted_cholesky(op, 20)
    assert np.all(np.diff(traces) <= 1e-12)
    np.testing.assert_allclose(traces[-1], np.trace(K - L @ L.T), atol=1e-9)
    # exponential decay: the log-trace falls at least linearly between k=4 and k=16
    assert traces[16] < traces[4] * 1e-6


def test_tolerance_stops_early():
    op = _op(300, 1, kernels.RBF, seed=4, ls=0.3)
    L, piv, rank, traces = pivchol.pivoted_cholesky(op, 100, tol=1e-6)
    assert rank < 100
    assert traces[-1] <= 1e-6 * traces[0]
    assert traces[-2] > 1e-6 * traces[0]


def test_zero_rank_and_override():
    op = _op(30, 2)
    L, piv, rank, _ = pivchol.pivoted_cholesky(op, 0)
    assert rank == 0 and L.shape == (30, 0)
    L1, piv1, r1, _ = pivchol.pivoted_cholesky(op, 6)
    L2, piv2, r2, _ = pivchol.pivoted_cholesky(op, 6, piv_override=piv1)
    np.testing.assert_array_equal(piv1, piv2)
    np.testing.assert_allclose(L1, L2)


@pytest.mark.parametrize("kind", [kernels.RBF, kernels.MATERN32, kernels.RATQUAD])
@pytest.mark.parametrize("u", [2.0 ** -53, 2.0 ** -24])
def test_rank_floor_stops_at_exact_rank(kind, u):
    """r distinct points, each repeated: K has rank exactly r for these strictly
    positive definite kernels.  After r pivots every residual is rounding error, so
    with floor = n u the factor stops at rank r; the rank-r factor reproduces K."""
    r, rep = 9, 7
    rng = np.random.default_rng(4)
    Xd = rng.uniform(size=(r, 2))
    X = np.repeat(Xd, rep, axis=0)[rng.permutation(r * rep)]
    theta = np.array([0.4, 0.7, 1.3, 0.01])
    op = kernels.KernelOperator(kind, X, theta, True)
    n = r * rep
    L, piv, rank, _ = pivchol.pivoted_cholesky(op, 30, floor=n * u)
    assert rank == r
    assert len(set(map(tuple, X[piv]))) == r          # one pivot per distinct point
    K = kernels.kernel_block(kind, X, X, theta, True)
    np.testing.assert_allclose(L @ L.T, K, atol=1e-10)


def test_rank_floor_zero_is_the_textbook_rule():
    """floor = 0 keeps the plain rule (stop only at a residual <= 0): the same factor
    as before the option existed, and a positive floor below every pivot residual
    changes nothing."""
    op = _op(80, 3, kernels.MATERN52, seed=6)
    L0, piv0, r0, t0 = pivchol.pivoted_cholesky(op, 20)
    L1, piv1, r1, t1 = pivchol.pivoted_cholesky(op, 20, floor=0.0)
    d = np.diag(L0[piv0]) ** 2
    L2, piv2, r2, _ = pivchol.pivoted_cholesky(op, 20, floor=0.5 * d.min() / op.diag().max())
    assert r0 == r1 == r2 == 20
    np.testing.assert_array_equal(piv0, piv1)
    np.testing.assert_array_equal(piv0, piv2)
    np.testing.assert_array_equal(L0, L2)
