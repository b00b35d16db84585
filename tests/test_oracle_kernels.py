"""Pins for oracle/kernels.py against facts outside the oracle.

* Matern(3/2) and Matern(5/2) equal the general Matern form with the modified
  Bessel function K_nu (Rasmussen & Williams 2006, eq. 4.14), evaluated by scipy.
* RBF is the nu -> infinity limit of Matern, and an ARD RBF factorises over
  dimensions.
* The rational quadratic kernel is a scale mixture of RBF kernels:
  (1 + r^2/(2 alpha))^-alpha = int_0^inf exp(-tau r^2 / 2) Gamma(tau; alpha, rate alpha) dtau
  (Rasmussen & Williams 2006, eq. 4.20), evaluated by numerical quadrature over the
  oracle's own RBF; it also approaches the RBF as alpha grows (checked on the general form).
* Every derivative equals a central finite difference of the kernel value.
"""
import numpy as np
import pytest
from scipy import integrate
from scipy.special import gammaln, kve

from oracle import kernels


def matern_bessel(nu, r, s):
    r = np.asarray(r, np.float64)
    x = np.sqrt(2.0 * nu) * r
    out = np.full_like(r, s)
    nz = x > 0
    xs = x[nz]
    # log of s 2^(1-nu)/Gamma(nu) x^nu K_nu(x), with K_nu(x) = kve(nu, x) e^-x
    logv = (np.log(s) + (1.0 - nu) * np.log(2.0) - gammaln(nu) + nu * np.log(xs)
            + np.log(kve(nu, xs)) - xs)
    out[nz] = np.exp(logv)
    return out


@pytest.mark.parametrize("kind,nu", [(kernels.MATERN32, 1.5), (kernels.MATERN52, 2.5)])
def test_matern_matches_bessel_form(kind, nu):
    r = np.linspace(0.0, 6.0, 61)
    s = 1.7
    np.testing.assert_allclose(kernels.k_of_r2(kind, r * r, s), matern_bessel(nu, r, s),
                               rtol=1e-12, atol=1e-14)


def test_rbf_is_matern_limit():
    r = np.linspace(0.8, 3.0, 23)
    mid = matern_bessel(10.0, r, 1.0)
    far = matern_bessel(40.0, r, 1.0)
    rbf = kernels.k_of_r2(kernels.RBF, r * r, 1.0)
    assert np.all(np.isfinite(far))
    # the Matern family approaches the RBF as nu grows
    assert np.abs(rbf - far).max() < 0.3 * np.abs(rbf - mid).max()
    np.testing.assert_allclose(rbf, far, atol=1e-2)


def test_rbf_ard_factorises_over_dimensions():
    rng = np.random.default_rng(0)
    Xa, Xb = rng.uniform(size=(5, 3)), rng.uniform(size=(4, 3))
    ls = np.array([0.3, 0.7, 1.1])
    theta = np.concatenate([ls, [2.0, 0.1]])
    K = kernels.kernel_block(kernels.RBF, Xa, Xb, theta, True)
    prod = np.full((5, 4), 2.0)
    for j in range(3):
        Kj = kernels.kernel_block(kernels.RBF, Xa[:, j:j + 1], Xb[:, j:j + 1],
                                  np.array([ls[j], 1.0, 0.1]), False)
        prod *= Kj
    np.testing.assert_allclose(K, prod, rtol=1e-13)


@pytest.mark.parametrize("kind", kernels.KINDS)
@pytest.mark.parametrize("ard", [True, False])
def test_derivatives_match_finite_differences(kind, ard):
    rng = np.random.default_rng(1)
    d = 3
    Xa, Xb = rng.uniform(size=(6, d)), rng.uniform(size=(5, d))
    Xb[0] = Xa[0]                          # include r = 0
    D = d if ard else 1
    theta = np.concatenate([rng.uniform(0.4, 1.2, D), [1.3, 0.05]])
    blocks = kernels.kernel_grad_blocks(kind, Xa, Xb, theta, ard)
    assert len(blocks) == D + 1
    for q in range(D + 1):
        h = 1e-6 * theta[q]
        tp, tm = theta.copy(), theta.copy()
        tp[q] += h
        tm[q] -= h
        fd = (kernels.kernel_block(kind, Xa, Xb, tp, ard)
              - kernels.kernel_block(kind, Xa, Xb, tm, ard)) / (2 * h)
        np.testing.assert_allclose(blocks[q], fd, rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("kind", kernels.KINDS)
def test_kernel_matrix_is_psd_with_diag_s(kind):
    rng = np.random.default_rng(2)
    X = rng.uniform(size=(40, 2))
    theta = np.array([0.5, 0.8, 1.5, 0.0])
    K = kernels.kernel_block(kind, X, X, theta, True)
    assert np.allclose(np.diag(K), 1.5)
    assert np.linalg.eigvalsh(K).min() > -1e-10


def test_operator_matches_dense():
    rng = np.random.default_rng(3)
    X = rng.uniform(size=(300, 2))
    theta = np.array([0.4, 0.6, 1.0, 0.02])
    V = rng.standard_normal((300, 3))
    op = kernels.KernelOperator(kernels.MATERN52, X, theta, True, block_entries=300 * 37)
    op._dense = None                        # force the blocked path
    Kh = kernels.khat_dense(kernels.MATERN52, X, theta, True)
    np.testing.assert_allclose(op.matvec(V), Kh @ V, rtol=1e-12, atol=1e-12)
    dK = kernels.dkhat_dense(kernels.MATERN52, X, theta, True)
    for got, ref in zip(op.grad_matvec(V), dK):
        np.testing.assert_allclose(got, ref @ V, rtol=1e-12, atol=1e-12)


def test_ratquad_is_gamma_mixture_of_rbf():
    alpha = 1.0
    s_out = 1.4
    for r in (0.0, 0.3, 1.0, 2.5, 6.0):
        def integrand(tau):
            gamma_pdf = np.exp(alpha * np.log(alpha) - gammaln(alpha)
                               + (alpha - 1.0) * np.log(tau) - alpha * tau)
            return float(kernels.k_of_r2(kernels.RBF, tau * r * r, s_out)) * gamma_pdf
        val, err = integrate.quad(integrand, 0.0, np.inf, epsabs=1e-14, epsrel=1e-12)
        got = float(kernels.k_of_r2(kernels.RATQUAD, np.array(r * r), s_out))
        assert abs(got - val) <= 1e-10 * s_out, (r, got, val)


def test_ratquad_general_alpha_tends_to_rbf():
    """The alpha = 1 member used here belongs to the family (1 + r^2/(2 alpha))^-alpha,
    which tends to exp(-r^2/2) as alpha grows."""
    r2 = np.linspace(0.0, 9.0, 19)
    fam = lambda a: (1.0 + r2 / (2.0 * a)) ** (-a)
    np.testing.assert_allclose(fam(1.0), kernels.k_of_r2(kernels.RATQUAD, r2, 1.0), rtol=1e-15)
    rbf = kernels.k_of_r2(kernels.RBF, r2, 1.0)
    assert np.abs(fam(1e6) - rbf).max() < 1e-4 < np.abs(fam(1.0) - rbf).max()
