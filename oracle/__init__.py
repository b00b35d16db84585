"""FP64 CPU oracle for the preconditioned GP log-marginal-likelihood estimator.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` use it.  It shares no code, constants or
helpers with the CUDA library in ``paper_2107_00243_gb300/csrc``.

Everything here is plain numpy in float64, written for a reader checking it
against the paper (Wenger et al., "Preconditioning for Scalable Gaussian Process
Hyperparameter Optimization", ICML 2022) by eye.  Library primitives (a matmul,
a dense Cholesky, a symmetric eigensolver) stand in for single steps only.

Modules
-------
kernels    kernel functions k(r) and their hyperparameter derivatives (Sec. 5 setup)
exact      exact MLL and gradient by dense Cholesky (eqs. likelihood / derivative_likelihood)
pivchol    greedy partial pivoted Cholesky (Prop. "Cholesky approximation quality")
woodbury   P = sigma^2 I + L L^T: solve (matrix inversion lemma), log-det (determinant
           lemma), dP/dtheta at frozen pivots, tr(P^-1 dP) (eq. preconditioner_trace)
probes     counter-based Rademacher signs from SplitMix64
mbcg       preconditioned CG with many right-hand sides and Lanczos coefficients
lanczos    tridiagonal T from CG coefficients and Lanczos quadrature of log
estimator  Alg. 1 (LogMargLikelihood) and Alg. 2 (Derivative) with the paper's
           variance reduction
"""
