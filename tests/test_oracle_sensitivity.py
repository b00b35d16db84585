"""How much the FP64 oracle's own estimator moves under rounding-sized changes of its
kernel products.  These measurements set the FP64 parity bounds of the GPU tests.

Two FP64 implementations of the same estimator differ in the summation order of every
kernel-matrix product.  The model of that difference used here adds
2^-53 (|K_hat| |V|)_ic N(0, 1) to each output entry of each product; the operator
itself is unchanged.  The pivots and the per-column iteration counts are frozen
(matched runs), exactly as in the GPU parity tests.

What the measurement shows (small RBF workload, d = 3):
* At its own CG tolerance of 1e-6, y^T u moves by up to ~6e-8 relative.  Finite-precision
  CG stopped at a loose tolerance amplifies rounding in its iterates.  The log-det term
  moves by only ~1e-14: the Lanczos quadrature is insensitive.  No FP64 bound below
  ~1e-7 can hold on the MLL at this tolerance, whatever the implementation.
* With CG run to 1e-10, the same perturbations move the MLL by ~3e-12 and gradient
  entries by ~1e-10.  Tight FP64 parity is therefore checked at tight tolerances.
"""
import numpy as np

from oracle import estimator, kernels
from paper_2107_00243_gb300 import workloads


def _spread(p, tol, draws):
    ref = estimator.mll_and_grad(p.kind, p.X, p.y, p.theta, p.ard, p.k, p.n_probes, tol,
                                 p.max_iter, seed=p.seed)
    K = kernels.kernel_block(p.kind, p.X, p.X, p.theta, p.ard)
    s2 = p.theta[-1]
    scale = 0.5 * (np.abs(ref["quad_p"]) + np.abs(ref["trace_p"]))
    worst = {"mll": 0.0, "quad": 0.0, "logdet": 0.0, "grad": 0.0}
    orig = kernels.KernelOperator.matvec
    try:
        for v in range(draws):
            rng = np.random.default_rng(100 + v)

            def noisy(self, V, _o=orig, rng=rng):
                V = np.asarray(V, np.float64)
                W = _o(self, V)
                bound = np.abs(K) @ np.abs(V) + s2 * np.abs(V)
                return W + 2.0 ** -53 * bound * rng.standard_normal(W.shape)

            kernels.KernelOperator.matvec = noisy
            r = estimator.mll_and_grad(p.kind, p.X, p.y, p.theta, p.ard, p.k, p.n_probes,
                                       tol, p.max_iter, seed=p.seed,
                                       piv_override=ref["piv"], iters_override=ref["iters"])
            kernels.KernelOperator.matvec = orig
            for key in ("mll", "quad", "logdet"):
                worst[key] = max(worst[key], abs(r[key] - ref[key]) / abs(ref[key]))
            worst["grad"] = max(worst["grad"],
                                float(np.max(np.abs(r["grad"] - ref["grad"]) / scale)))
    finally:
        kernels.KernelOperator.matvec = orig
    return worst


def test_loose_tolerance_quadratic_term_is_rounding_sensitive():
    w = _spread(workloads.c1_small_rbf(n=300), 1e-6, draws=6)
    print("tol 1e-6:", {k: f"{v:.2e}" for k, v in w.items()})
    assert w["quad"] > 1e-8          # a 1e-8 FP64 bound at this tolerance cannot hold
    assert w["mll"] < 3e-7 and w["grad"] < 1e-5
    assert w["logdet"] < 1e-12


def test_tight_tolerance_results_are_stable():
    w = _spread(workloads.c1_small_rbf(n=300), 1e-10, draws=6)
    print("tol 1e-10:", {k: f"{v:.2e}" for k, v in w.items()})
    assert w["mll"] < 5e-11 and w["quad"] < 5e-11
    assert w["grad"] < 3e-9
    assert w["logdet"] < 1e-13
