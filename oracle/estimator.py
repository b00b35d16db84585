"""The paper's preconditioned estimator of the GP log-marginal likelihood and its gradient,
FP64 (test infrastructure only).

Alg. 1 (LogMargLikelihood) and Alg. 2 (Derivative), run as one CG call over
B = [y, z_1 .. z_l] as the footnote to Sec. 4.4 suggests.

Forward (Alg. 1; Thm. 2):
    u        = CG(K_hat, y, P_hat)                      ~ K_hat^-1 y
    tau_P    = log det P_hat                            (determinant lemma)
    gamma_i  = rho0_i * e_1^T log(T_i) e_1              ~ z_i'^T log(P^-1/2 K_hat P^-1/2) z_i'
    tau_log  = tau_P + (1/l) sum_i gamma_i              ~ log det K_hat   (eq. logdet-decomposition)
    mll      = -1/2 (y^T u + tau_log + n log 2 pi)

Backward (Alg. 2; eq. logdet-decomposition_deriv; Thm. 3):
    quad_p   = 1/2 u^T dK_hat_p u
    probeK_p = (1/l) sum_i (K_hat^-1 z_i)^T dK_hat_p (P^-1 z_i)
    probeP_p = (1/l) sum_i (P^-1 z_i)^T dP_hat_p (P^-1 z_i)
    trP_p    = tr(P_hat^-1 dP_hat_p)                    (eq. preconditioner_trace)
    trace_p  = trP_p + probeK_p - probeP_p              ~ tr(K_hat^-1 dK_hat_p)
    grad_p   = quad_p - 1/2 trace_p

Readings of the paper used here (the paper is silent or ambiguous on these):
* Probes have covariance P_hat (z_i = L eps1_i + sigma eps2_i, see probes.py), the
  quadrature is scaled by rho0_i = z_i^T P^-1 z_i and averaged with 1/l.  Both
  stochastic terms are then unbiased: E[P^-1/2 z z^T P^-1/2] = I and
  E[P^-1 z z^T] = I.  ``literal=True`` runs Alg. 1/2 as printed instead
  (normalised Rademacher z, gamma_i = e_1^T log(T_i) e_1, n/l scaling).
* Alg. 2 solves K_hat^-1 (dK_hat z_i) per hyperparameter; by symmetry
  z^T K^-1 dK w = (K^-1 z)^T dK w, so the probe solves of the forward pass are reused.
* dK_hat uses the noise too (dK_hat/dsigma^2 = I).
* ``rank_floor`` stops the pivoted Cholesky at a residual of rank_floor * max K_ii
  (pivchol.py); a comparison with a factor formed in precision u passes n u.
* ``rff = (eps, g)`` replaces the partial Cholesky factor by random Fourier features
  (Tab. 2; features.py), k = 2m columns, with dP_hat at frozen draws; ``qff = mbar``
  by the quadrature Fourier features of the RBF kernel (mbar^d columns).
* dP_hat is taken at frozen pivots (woodbury.NystromDerivative).
"""
import numpy as np

from . import features, kernels, lanczos, mbcg, pivchol, probes, woodbury


def mll_and_grad(kind, X, y, theta, ard, k, n_probes, tol, max_iter, seed=0,
                 recompute_every=0, pivchol_tol=0.0, piv_override=None,
                 iters_override=None, eps=None, literal=False, with_grad=True, rank_floor=0.0,
                 rff=None, qff=None):
    X = np.asarray(X, np.float64)
    y = np.asarray(y, np.float64)
    n = X.shape[0]
    op = kernels.KernelOperator(kind, X, theta, ard)
    s2 = op.s2

    if rff is None and qff is None:
        L, piv, rank, _ = pivchol.pivoted_cholesky(op, k, pivchol_tol, piv_override, rank_floor)
        dprec = None
    else:
        # random Fourier features from the draws (eps, g), or the quadrature features of
        # qff = mbar nodes per dimension (features.py): k = 2m columns
        if rff is not None:
            dprec = features.RandomFourier(kind, X, theta, ard, *rff)
        else:
            if kind != kernels.RBF:
                raise ValueError("quadrature Fourier features are defined for the RBF kernel")
            U, w = features.hermite_grid(qff, X.shape[1])
            dprec = features.RandomFourier(kind, X, theta, ard, U=U, weights=w)
        L, piv, rank = dprec.Phi, np.zeros(0, np.int64), dprec.Phi.shape[1]
        k = rank
    logdetP = woodbury.logdet(L, s2)

    if eps is None:
        eps1, eps2 = probes.eps_pair(seed, k, n, n_probes)
    else:
        eps1, eps2 = eps
    Z = probes.probes(L, s2, eps1, eps2, literal=literal)
    B = np.column_stack([y, Z])

    cg = mbcg.mbcg(op.matvec, lambda V: woodbury.solve(L, s2, V), B, tol, max_iter,
                   recompute_every, iters_override)
    u = cg["X"][:, 0]
    quad = float(y @ u)

    gamma = np.zeros(n_probes)
    for i in range(n_probes):
        c = i + 1
        m = int(cg["iters"][c])
        diag, off = lanczos.tridiag_from_cg(cg["alpha"][c], cg["beta"][c], m)
        q = lanczos.quadrature(diag, off)
        gamma[i] = q if literal else cg["rho0"][c] * q
    stoch = (n / n_probes if literal else 1.0 / n_probes) * float(np.sum(gamma))
    logdet = logdetP + stoch
    mll = -0.5 * (quad + logdet + n * np.log(2.0 * np.pi))

    out = {
        "mll": float(mll), "quad": quad, "logdetP": float(logdetP), "stoch": stoch,
        "logdet": float(logdet), "gamma": gamma, "piv": piv, "rank": rank,
        "iters": cg["iters"], "rho0": cg["rho0"], "L": L, "Z": Z, "cg": cg,
    }
    if not with_grad:
        return out

    p = op.p
    dKu = op.grad_matvec(u[:, None])
    quad_p = np.array([0.5 * float(u @ dKu[q][:, 0]) for q in range(p)])

    Xp = cg["X"][:, 1:]                  # ~ K_hat^-1 z_i
    Wp = cg["z0"][:, 1:]                 # = P_hat^-1 z_i
    nd = woodbury.NystromDerivative(op, piv) if dprec is None else dprec
    probeK = np.zeros(p)
    probeP = np.zeros(p)
    trP = np.zeros(p)
    if literal:
        dKz = op.grad_matvec(Z)
        for q in range(p):
            probeK[q] = (n / n_probes) * float(np.sum(Xp * dKz[q]))
            probeP[q] = (n / n_probes) * float(np.sum(Wp * nd.apply(q, Z)))
    else:
        dKW = op.grad_matvec(Wp)
        for q in range(p):
            probeK[q] = float(np.sum(Xp * dKW[q])) / n_probes
            probeP[q] = float(np.sum(Wp * nd.apply(q, Wp))) / n_probes
    for q in range(p):
        trP[q] = woodbury.precond_trace(L, s2, lambda V, q=q: nd.apply(q, V), nd.diag(q))
    trace_p = trP + probeK - probeP
    grad = quad_p - 0.5 * trace_p
    out.update({
        "grad": grad, "quad_p": quad_p, "probeK_p": probeK, "probeP_p": probeP,
        "trP_p": trP, "trace_p": trace_p,
    })
    return out
