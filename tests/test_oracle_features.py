"""Pins for oracle/features.py (random Fourier feature preconditioner, Tab. 2).

* Bochner: with many frequencies, Phi Phi^T reproduces K for every kernel, each entry
  within 6 standard errors of the Monte Carlo mean.  A wrong spectral density (the other
  Matern order, a Gamma shape off by a factor of two) misses by several times that.
* The derivative at frozen draws against central finite differences of Phi(theta).
* eq. preconditioner_trace with features against the dense tr(P_hat^-1 dP_hat).
* The estimator stays unbiased with this P_hat: exact enumeration of all sign
  patterns (n = 4, k = 4) gives E[stochastic log-det] = log det K_hat - log det P_hat
  and E[trace estimate] = tr(K_hat^-1 dK_hat_p).
* The rate of Prop. "RFF approximation quality": the Frobenius error of P_hat falls
  like k^-1/2 (16x the features, about 4x smaller).
* Quadrature Fourier features (RBF): the folded Gauss-Hermite tensor rule has the
  moments of N(0, I_d); Phi Phi^T converges to K exponentially in the nodes per
  dimension (Prop. "QFF approximation quality"); finite differences; unbiasedness by
  enumeration as above.
"""
import itertools

import numpy as np
import pytest

from oracle import estimator, features, kernels, woodbury


def _draws(m, d, kind, seed):
    rng = np.random.default_rng(seed)
    eps = rng.standard_normal((m, d))
    shape = features.gamma_shape(kind)
    g = rng.gamma(shape, 1.0, m) if shape is not None else np.ones(m)
    return eps, g


def _points(n, d, seed=0):
    return np.random.default_rng(seed).uniform(size=(n, d))


@pytest.mark.parametrize("kind", kernels.KINDS)
def test_features_reproduce_the_kernel(kind):
    X = _points(10, 2, 1)
    theta = np.array([0.4, 0.7, 1.3, 0.01])
    K = kernels.kernel_block(kind, X, X, theta, True)
    acc, m_tot = np.zeros_like(K), 0
    for c in range(8):                     # 8 x 50,000 frequencies
        eps, g = _draws(50_000, 2, kind, 100 + c)
        f = features.RandomFourier(kind, X, theta, True, eps, g)
        acc += f.Phi @ f.Phi.T * f.m
        m_tot += f.m
    est = acc / m_tot
    se = 1.3 / np.sqrt(m_tot)              # each term s cos(.) has variance <= s^2
    assert np.max(np.abs(est - K)) <= 6 * se
    if kind in (kernels.MATERN32, kernels.MATERN52):
        other = kernels.MATERN52 if kind == kernels.MATERN32 else kernels.MATERN32
        K_other = kernels.kernel_block(other, X, X, theta, True)
        assert np.max(np.abs(est - K_other)) > 3 * 6 * se


@pytest.mark.parametrize("kind", kernels.KINDS)
@pytest.mark.parametrize("ard", [True, False])
def test_derivative_against_finite_differences(kind, ard):
    X = _points(15, 3, 2)
    theta = np.array([0.5, 0.8, 1.1, 1.4, 0.02]) if ard else np.array([0.6, 1.4, 0.02])
    eps, g = _draws(40, 3, kind, 7)
    f = features.RandomFourier(kind, X, theta, ard, eps, g)
    for q in range(f.p - 1):
        h = 1e-6 * theta[q]
        tp, tm = theta.copy(), theta.copy()
        tp[q] += h
        tm[q] -= h
        fd = (features.RandomFourier(kind, X, tp, ard, eps, g).Phi
              - features.RandomFourier(kind, X, tm, ard, eps, g).Phi) / (2 * h)
        np.testing.assert_allclose(f.dphi(q), fd, rtol=1e-6, atol=1e-8)
        np.testing.assert_allclose(f.diag(q), np.diag(f.dense(q)), rtol=1e-12, atol=1e-14)


def test_preconditioner_trace_with_features():
    X = _points(30, 2, 3)
    theta = np.array([0.3, 0.5, 1.2, 0.05])
    eps, g = _draws(12, 2, kernels.MATERN52, 4)
    f = features.RandomFourier(kernels.MATERN52, X, theta, True, eps, g)
    P = 0.05 * np.eye(30) + f.Phi @ f.Phi.T
    Pinv = np.linalg.inv(P)
    for q in range(f.p):
        dense = float(np.trace(Pinv @ f.dense(q)))
        got = woodbury.precond_trace(f.Phi, 0.05, lambda V, q=q: f.apply(q, V), f.diag(q))
        assert abs(got - dense) <= 1e-9 * max(1.0, abs(dense))


@pytest.mark.parametrize("kind", [kernels.RBF, kernels.RATQUAD])
def test_estimator_unbiased_with_features(kind):
    n, m = 4, 2                             # k = 4 features: 2^(4 + 4) sign patterns
    X = _points(n, 2, 5)
    y = np.array([0.3, -1.1, 0.7, 0.2])
    theta = np.array([0.6, 0.9, 1.1, 0.3])
    rff = _draws(m, 2, kind, 6)
    f = features.RandomFourier(kind, X, theta, True, *rff)
    Kh = kernels.khat_dense(kind, X, theta, True)
    P = theta[-1] * np.eye(n) + f.Phi @ f.Phi.T
    dK = kernels.dkhat_dense(kind, X, theta, True)
    acc_s, acc_t, cnt = 0.0, 0.0, 0
    for bits in itertools.product([-1.0, 1.0], repeat=2 * m + n):
        e1 = np.array(bits[:2 * m])[:, None]
        e2 = np.array(bits[2 * m:])[:, None]
        out = estimator.mll_and_grad(kind, X, y, theta, True, 0, 1, 1e-15, 60, eps=(e1, e2),
                                     rff=rff)
        acc_s = acc_s + out["stoch"]
        acc_t = acc_t + out["trace_p"] - out["trP_p"]
        cnt += 1
    want_s = np.linalg.slogdet(Kh)[1] - np.linalg.slogdet(P)[1]
    Khi, Pi = np.linalg.inv(Kh), np.linalg.inv(P)
    want_t = np.array([np.trace(Khi @ dK[q]) - np.trace(Pi @ f.dense(q))
                       for q in range(f.p)])
    assert abs(acc_s / cnt - want_s) <= 1e-10 * max(1.0, abs(want_s))
    np.testing.assert_allclose(acc_t / cnt, want_t, rtol=1e-9, atol=1e-10)


def test_error_falls_like_inverse_square_root_of_k():
    X = _points(60, 2, 8)
    theta = np.array([0.3, 0.3, 1.0, 0.01])
    K = kernels.kernel_block(kernels.RBF, X, X, theta, True)

    def mean_err(m):
        errs = []
        for r in range(40):
            f = features.RandomFourier(kernels.RBF, X, theta, True,
                                       *_draws(m, 2, kernels.RBF, 1000 + 97 * m + r))
            errs.append(np.linalg.norm(K - f.Phi @ f.Phi.T))
        return float(np.mean(errs))

    ratio = mean_err(16) / mean_err(256)    # k = 32 vs 512 features
    assert 3.0 <= ratio <= 5.3, ratio


# ---- quadrature Fourier features (Tab. 2 "QFF", RBF kernel) ---------------------------

@pytest.mark.parametrize("d", [1, 2, 3])
def test_hermite_grid_moments(d):
    """The folded tensor rule integrates against N(0, I_d): weights sum to 1, E[w_i^2] = 1,
    E[w_i^4] = 3, E[w_i^2 w_j^2] = 1 (i != j), and it is exact for cos(w . D) up to the
    rule's degree (checked through the moments that cos's Taylor terms need)."""
    U, W = features.hermite_grid(6, d)
    assert U.shape == (6 ** d // 2, d) and np.all(W > 0)
    assert abs(W.sum() - 1.0) < 1e-14
    for i in range(d):
        assert abs(np.sum(W * U[:, i] ** 2) - 1.0) < 1e-13
        assert abs(np.sum(W * U[:, i] ** 4) - 3.0) < 1e-12
        for j in range(i + 1, d):
            assert abs(np.sum(W * U[:, i] ** 2 * U[:, j] ** 2) - 1.0) < 1e-13


@pytest.mark.parametrize("d,mbars,last", [(1, (4, 8, 16, 32), 1e-12), (2, (4, 8, 16), 1e-8)])
def test_quadrature_features_converge_to_the_kernel(d, mbars, last):
    """Prop. "QFF approximation quality": the error of Phi Phi^T falls exponentially in
    the nodes per dimension."""
    X = _points(25, d, 9)
    theta = np.concatenate([np.full(d, 0.35), [1.1, 0.01]])
    K = kernels.kernel_block(kernels.RBF, X, X, theta, True)
    errs = []
    for mb in mbars:
        f = features.RandomFourier(kernels.RBF, X, theta, True,
                                   *(None, None), *features.hermite_grid(mb, d))
        errs.append(np.max(np.abs(f.Phi @ f.Phi.T - K)))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < last, errs


@pytest.mark.parametrize("ard", [True, False])
def test_quadrature_feature_derivative(ard):
    X = _points(12, 2, 10)
    theta = np.array([0.4, 0.6, 1.2, 0.02]) if ard else np.array([0.5, 1.2, 0.02])
    U, W = features.hermite_grid(6, 2)
    f = features.RandomFourier(kernels.RBF, X, theta, ard, U=U, weights=W)
    for q in range(f.p - 1):
        h = 1e-6 * theta[q]
        tp, tm = theta.copy(), theta.copy()
        tp[q] += h
        tm[q] -= h
        fd = (features.RandomFourier(kernels.RBF, X, tp, ard, U=U, weights=W).Phi
              - features.RandomFourier(kernels.RBF, X, tm, ard, U=U, weights=W).Phi) / (2 * h)
        np.testing.assert_allclose(f.dphi(q), fd, rtol=1e-6, atol=1e-8)


def test_estimator_unbiased_with_quadrature_features():
    n = 4                                   # mbar = 4 in 1-D: k = 4 features
    X = _points(n, 1, 11)
    y = np.array([0.5, -0.2, 1.1, -0.7])
    theta = np.array([0.5, 1.1, 0.2])
    U, W = features.hermite_grid(4, 1)
    f = features.RandomFourier(kernels.RBF, X, theta, True, U=U, weights=W)
    Kh = kernels.khat_dense(kernels.RBF, X, theta, True)
    P = theta[-1] * np.eye(n) + f.Phi @ f.Phi.T
    dK = kernels.dkhat_dense(kernels.RBF, X, theta, True)
    acc_s, acc_t, cnt = 0.0, 0.0, 0
    for bits in itertools.product([-1.0, 1.0], repeat=4 + n):
        e1 = np.array(bits[:4])[:, None]
        e2 = np.array(bits[4:])[:, None]
        out = estimator.mll_and_grad(kernels.RBF, X, y, theta, True, 0, 1, 1e-15, 60,
                                     eps=(e1, e2), qff=4)
        acc_s = acc_s + out["stoch"]
        acc_t = acc_t + out["trace_p"] - out["trP_p"]
        cnt += 1
    want_s = np.linalg.slogdet(Kh)[1] - np.linalg.slogdet(P)[1]
    Khi, Pi = np.linalg.inv(Kh), np.linalg.inv(P)
    want_t = np.array([np.trace(Khi @ dK[q]) - np.trace(Pi @ f.dense(q)) for q in range(f.p)])
    assert abs(acc_s / cnt - want_s) <= 1e-10 * max(1.0, abs(want_s))
    np.testing.assert_allclose(acc_t / cnt, want_t, rtol=1e-9, atol=1e-10)
