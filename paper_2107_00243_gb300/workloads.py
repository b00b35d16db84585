"""Seeded synthetic GP-regression workloads.

This module only draws inputs: data X, targets y and hyperparameters theta.  It
holds none of the estimator's arithmetic, so both the CUDA path and the CPU
oracle can be fed from it.

The paper measures on UCI datasets (Sec. 5, Tab. 1: Elevators, Bike, Kin40k,
Protein, KEGGdir, 3DRoad), which are not available here.  The workloads below are
synthetic stand-ins with comparable (n, d) and kernel choice:

  c1_small_rbf     n=1,000   d=3   U[0,1]^3, y = sin(2 pi x1) + cos(2 pi x2) x3 + N(0, 0.1^2);
                   RBF isotropic l=0.3, s=1, sigma^2=0.01; k=20, l=10, tol 1e-6, 200 its, FP64
  c2_matern52_ard  n=20,000  d=8   N(0, I); y = a Matern-5/2 GP draw via 2,048 random
                   Fourier features + N(0, 0.05^2); ARD l_j ~ U[0.5, 2], s=1,
                   sigma^2 = 0.05^2; k=100, l=50, tol 1e-3, FP32
  c3_rbf_ard_1e5   n=100,000 d=16  U[0,1]^16; y = sum of 16 random sinusoids + N(0, 0.1^2);
                   RBF ARD l_j ~ U[0.2, 1], s=1, sigma^2=0.01; k=200, l=32, tol 1e-2,
                   recompute every 25, BF16 tiles (and the same in FP32)
  c4_matern32_5e5  n=500,000 d=10  mixture of 20 Gaussians (means U[-2,2]^10, sd 0.3);
                   y = random cubic polynomial (all 286 monomials) + N(0, 0.1^2);
                   Matern-3/2 ARD, l=1, s=1, sigma^2=0.1; k=500, l=16, tol 1e-2, TF32
  c5_batched       64 problems, n_b log-uniform in [2,000, 50,000], d_b in {4, 8, 12},
                   U[0,1]^d; y = sinusoid sum + noise; RBF isotropic l ~ U[0.1, 1],
                   sigma^2 ~ U[1e-3, 1e-1], s=1; k=50, l=16, tol 1e-2, BF16

Every draw comes from ``numpy.random.default_rng(seed)``.  ``n`` may be overridden
to make a smaller problem of the same shape and distribution.
"""
from dataclasses import dataclass, field
import math

import numpy as np

RBF, MATERN32, MATERN52, RATQUAD = 0, 3, 5, 7
FP64, FP32, TF32, BF16 = 0, 1, 2, 3


@dataclass
class Problem:
    name: str
    X: np.ndarray            # n x d float64
    y: np.ndarray            # n float64
    theta: np.ndarray        # [l_1..l_D, s, sigma^2] float64
    kind: int
    ard: bool
    k: int                   # preconditioner rank
    n_probes: int            # l
    tol: float
    max_iter: int
    precision: int
    recompute_every: int = 0
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.X.shape[0]

    @property
    def d(self):
        return self.X.shape[1]


def _sinusoid_targets(rng, X, n_terms, noise_sd):
    n, d = X.shape
    a = rng.standard_normal(n_terms) / 4.0
    omega = rng.standard_normal((n_terms, d))
    phi = rng.uniform(0.0, 2.0 * np.pi, n_terms)
    f = np.sin(2.0 * np.pi * (X @ omega.T) + phi) @ a
    return f + noise_sd * rng.standard_normal(n)


def c1_small_rbf(n=1000, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, (n, 3))
    y = (np.sin(2 * np.pi * X[:, 0]) + np.cos(2 * np.pi * X[:, 1]) * X[:, 2]
         + 0.1 * rng.standard_normal(n))
    theta = np.array([0.3, 1.0, 0.01])
    return Problem("c1_small_rbf", X, y, theta, RBF, False, k=20, n_probes=10,
                   tol=1e-6, max_iter=200, precision=FP64, seed=seed)


def c2_matern52_ard(n=20000, seed=0, n_features=2048):
    rng = np.random.default_rng(seed)
    d = 8
    X = rng.standard_normal((n, d))
    ls = rng.uniform(0.5, 2.0, d)
    # Matern-5/2 spectral density: multivariate t with 2 nu = 5 degrees of freedom.
    z = rng.standard_normal((n_features, d))
    u = rng.chisquare(5.0, n_features)
    omega = z / np.sqrt(u / 5.0)[:, None] / ls[None, :]
    b = rng.uniform(0.0, 2.0 * np.pi, n_features)
    w = rng.standard_normal(n_features)
    f = np.sqrt(2.0 / n_features) * (np.cos(X @ omega.T + b) @ w)
    y = f + 0.05 * rng.standard_normal(n)
    theta = np.concatenate([ls, [1.0, 0.05 ** 2]])
    return Problem("c2_matern52_ard", X, y, theta, MATERN52, True, k=100, n_probes=50,
                   tol=1e-3, max_iter=1000, precision=FP32, seed=seed)


def c3_rbf_ard_1e5(n=100000, seed=0, precision=BF16):
    rng = np.random.default_rng(seed)
    d = 16
    X = rng.uniform(0.0, 1.0, (n, d))
    y = _sinusoid_targets(rng, X, 16, 0.1)
    ls = rng.uniform(0.2, 1.0, d)
    theta = np.concatenate([ls, [1.0, 0.01]])
    return Problem("c3_rbf_ard_1e5", X, y, theta, RBF, True, k=200, n_probes=32,
                   tol=1e-2, max_iter=1000, precision=precision, recompute_every=25,
                   seed=seed)


def c4_matern32_5e5(n=500000, seed=0):
    rng = np.random.default_rng(seed)
    d, n_comp = 10, 20
    means = rng.uniform(-2.0, 2.0, (n_comp, d))
    comp = rng.integers(0, n_comp, n)
    X = means[comp] + 0.3 * rng.standard_normal((n, d))
    # all monomials of degree <= 3 in 10 variables: C(13, 3) = 286
    monos = [()]
    for i in range(d):
        monos.append((i,))
    for i in range(d):
        for j in range(i, d):
            monos.append((i, j))
    for i in range(d):
        for j in range(i, d):
            for m in range(j, d):
                monos.append((i, j, m))
    assert len(monos) == 286
    coef = rng.standard_normal(len(monos)) / math.sqrt(len(monos))
    f = np.zeros(n)
    for c, mono in zip(coef, monos):
        term = np.ones(n)
        for i in mono:
            term = term * X[:, i]
        f += c * term
    y = f + 0.1 * rng.standard_normal(n)
    theta = np.concatenate([np.ones(d), [1.0, 0.1]])
    return Problem("c4_matern32_5e5", X, y, theta, MATERN32, True, k=500, n_probes=16,
                   tol=1e-2, max_iter=1000, precision=TF32, seed=seed,
                   extra={"adam_steps": 20, "lr": 0.05})


def c5_batched(n_problems=64, seed=0, n_lo=2000, n_hi=50000):
    rng = np.random.default_rng(seed)
    probs = []
    for b in range(n_problems):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        d = int(rng.choice([4, 8, 12]))
        X = rng.uniform(0.0, 1.0, (n, d))
        s2 = float(rng.uniform(1e-3, 1e-1))
        ls = float(rng.uniform(0.1, 1.0))
        y = _sinusoid_targets(rng, X, 16, math.sqrt(s2))
        theta = np.array([ls, 1.0, s2])
        probs.append(Problem(f"c5_batched[{b}]", X, y, theta, RBF, False, k=50,
                             n_probes=16, tol=1e-2, max_iter=1000, precision=BF16,
                             seed=seed + b))
    return probs


def synthetic_study(kind, d, n=10000, seed=0):
    """The synthetic data of the bias / variance study (Tab. S1): n points uniform on
    [0, 1]^d, targets sum_j sin(2 pi x_j) / sqrt(d) plus N(0, sigma^2) noise with
    sigma^2 = 1e-2 (the paper's value).  The paper prints no lengthscale or output
    scale; an isotropic lengthscale of 0.2 and s = 1 are used."""
    rng = np.random.default_rng(seed + 101 * d + kind)
    X = rng.uniform(0.0, 1.0, (n, d))
    y = np.sin(2.0 * np.pi * X).sum(1) / math.sqrt(d) + 0.1 * rng.standard_normal(n)
    theta = np.array([0.2, 1.0, 1e-2])
    return Problem(f"synthetic_study[kind={kind},d={d}]", X, y, theta, kind, False, k=128,
                   n_probes=128, tol=1e-10, max_iter=2000, precision=FP64, seed=seed)


def rff_draws(m, d, shape, seed=0):
    """Seeded draws for a random Fourier feature preconditioner: eps (m, d) standard
    normal and g (m,) from Gamma(shape, 1), or None when shape is None."""
    rng = np.random.default_rng(10_000 + seed)
    eps = rng.standard_normal((m, d))
    g = rng.gamma(shape, 1.0, m) if shape is not None else None
    return eps, g


def subsample(prob, n, seed=1):
    """A smaller problem drawn from the same workload (rows chosen at random)."""
    if n >= prob.n:
        return prob
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(prob.n, n, replace=False))
    return Problem(prob.name + f"[sub{n}]", prob.X[idx].copy(), prob.y[idx].copy(),
                   prob.theta.copy(), prob.kind, prob.ard, prob.k, prob.n_probes,
                   prob.tol, prob.max_iter, prob.precision, prob.recompute_every,
                   prob.seed, dict(prob.extra))


def random_problem(n, d, kind=RBF, ard=True, seed=0, lo=0.3, hi=1.0, s=1.0, s2=0.05,
                   k=8, n_probes=4, tol=1e-8, max_iter=None, precision=FP64):
    """Small generic problem for unit tests."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, (n, d))
    y = _sinusoid_targets(rng, X, 4, math.sqrt(s2))
    D = d if ard else 1
    ls = rng.uniform(lo, hi, D)
    theta = np.concatenate([ls, [s, s2]])
    return Problem(f"random[{n}x{d}]", X, y, theta, kind, ard, k, n_probes, tol,
                   max_iter if max_iter is not None else n, precision, seed=seed)
