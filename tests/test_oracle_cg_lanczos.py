"""Pins for oracle/mbcg.py and oracle/lanczos.py.

* Preconditioned CG at a tight tolerance matches a dense solve for every column.
* Gauss quadrature exactness: after m steps, rho0 e1^T T^j e1 equals
  b^T (P^-1 K_hat)^j P^-1 b for every j <= 2m - 1 (no square roots involved, so
  this checks T's formula independently of any matrix function).
* At convergence, rho0 e1^T log(T) e1 equals (P^-1/2 b)^T log(A) (P^-1/2 b) with
  A = P^-1/2 K_hat P^-1/2, evaluated from dense eigendecompositions.
* Unpreconditioned case (k = 0): the T built from CG coefficients equals the T of a
  plain Lanczos three-term recurrence (written out below) started at b / ||b||.
* Per-column iteration overrides run exactly the requested number of steps.
"""
import numpy as np
import pytest

from oracle import kernels, lanczos, mbcg, pivchol, woodbury


def _system(n=40, k=5, seed=0, kind=kernels.MATERN52, s2=0.05):
    rng = np.random.default_rng(seed)
    X = rng.uniform(size=(n, 2))
    theta = np.array([0.5, 0.3, 1.0, s2])
    op = kernels.KernelOperator(kind, X, theta, True)
    L, piv, rank, _ = pivchol.pivoted_cholesky(op, k)
    Kh = kernels.khat_dense(kind, X, theta, True)
    P = woodbury.dense(L, s2)
    B = rng.standard_normal((n, 3))
    return op, L, Kh, P, B


def _sym_fn(M, f):
    lam, V = np.linalg.eigh(M)
    return (V * f(lam)) @ V.T


def test_cg_matches_dense_solve():
    op, L, Kh, P, B = _system()
    res = mbcg.mbcg(Kh.__matmul__, lambda V: woodbury.solve(L, op.s2, V), B, 1e-13, 200)
    np.testing.assert_allclose(res["X"], np.linalg.solve(Kh, B), rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(res["z0"], np.linalg.solve(P, B), rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(res["rho0"], np.sum(B * np.linalg.solve(P, B), axis=0))


def test_gauss_quadrature_exactness():
    op, L, Kh, P, B = _system(n=60, k=4, seed=1)
    m = 5
    res = mbcg.mbcg(Kh.__matmul__, lambda V: woodbury.solve(L, op.s2, V), B, 0.0, 50,
                    iters_override=[m, m, m])
    assert list(res["iters"]) == [m, m, m]
    PinvK = np.linalg.solve(P, Kh)
    for c in range(3):
        diag, off = lanczos.tridiag_from_cg(res["alpha"][c], res["beta"][c], m)
        T = lanczos.dense_tridiag(diag, off)
        b = B[:, c]
        v = np.linalg.solve(P, b)
        for j in range(2 * m):
            lhs = res["rho0"][c] * np.linalg.matrix_power(T, j)[0, 0]
            rhs = b @ np.linalg.matrix_power(PinvK, j) @ v
            assert abs(lhs - rhs) <= 1e-8 * abs(rhs), (c, j, lhs, rhs)


def test_log_quadrature_exact_at_convergence():
    op, L, Kh, P, B = _system(n=30, k=3, seed=2)
    res = mbcg.mbcg(Kh.__matmul__, lambda V: woodbury.solve(L, op.s2, V), B, 1e-14, 200)
    Ph = _sym_fn(P, lambda x: x ** -0.5)
    A = Ph @ Kh @ Ph
    logA = _sym_fn(A, np.log)
    for c in range(3):
        m = int(res["iters"][c])
        diag, off = lanczos.tridiag_from_cg(res["alpha"][c], res["beta"][c], m)
        got = res["rho0"][c] * lanczos.quadrature(diag, off)
        w = Ph @ B[:, c]
        ref = w @ logA @ w
        assert abs(got - ref) <= 1e-8 * max(1.0, abs(ref)), (c, got, ref)


def _plain_lanczos(A, q1, m):
    """Textbook Lanczos three-term recurrence (no reorthogonalisation)."""
    n = len(q1)
    alphas, betas = [], []
    q_prev = np.zeros(n)
    q = q1 / np.linalg.norm(q1)
    b_prev = 0.0
    for j in range(m):
        w = A @ q - b_prev * q_prev
        a = q @ w
        w = w - a * q
        alphas.append(a)
        if j < m - 1:
            b = np.linalg.norm(w)
            betas.append(b)
            q_prev, q, b_prev = q, w / b, b
    return np.array(alphas), np.array(betas)


def test_cg_tridiagonal_equals_plain_lanczos_without_preconditioner():
    op, L, Kh, P, B = _system(n=50, k=0, seed=3)
    m = 6
    res = mbcg.mbcg(Kh.__matmul__, lambda V: woodbury.solve(L, op.s2, V), B[:, :1], 0.0, 50,
                    iters_override=[m])
    diag, off = lanczos.tridiag_from_cg(res["alpha"][0], res["beta"][0], m)
    # P = sigma^2 I: preconditioned CG is Lanczos on K_hat / sigma^2
    a, b = _plain_lanczos(Kh / op.s2, B[:, 0], m)
    np.testing.assert_allclose(diag, a, rtol=1e-9)
    np.testing.assert_allclose(off, b, rtol=1e-9)


def test_iteration_override_and_zero_column():
    op, L, Kh, P, B = _system(seed=4)
    B[:, 1] = 0.0
    res = mbcg.mbcg(Kh.__matmul__, lambda V: woodbury.solve(L, op.s2, V), B, 1e-10, 100)
    assert res["iters"][1] == 0
    np.testing.assert_array_equal(res["X"][:, 1], 0.0)
    res2 = mbcg.mbcg(Kh.__matmul__, lambda V: woodbury.solve(L, op.s2, V), B, 1e-10, 100,
                     iters_override=[3, 0, 7])
    assert list(res2["iters"]) == [3, 0, 7]


def test_residual_recompute_keeps_solution():
    op, L, Kh, P, B = _system(seed=5)
    pre = lambda V: woodbury.solve(L, op.s2, V)
    a = mbcg.mbcg(Kh.__matmul__, pre, B, 1e-12, 200)
    b = mbcg.mbcg(Kh.__matmul__, pre, B, 1e-12, 200, recompute_every=3)
    np.testing.assert_allclose(a["X"], b["X"], rtol=1e-8, atol=1e-10)
