"""torch.autograd.Function around gp_mll_and_grad, and an Adam loop on log-hyperparameters.

The forward pass evaluates Alg. 1 and Alg. 2 together in one call of the CUDA
library; the gradient it returns is the paper's estimator of dL/dtheta
(eq. derivative_likelihood with the variance-reduced trace estimate), so the
backward pass only scales it by the incoming gradient.  It is not the derivative
of the stochastic forward value: the two agree in expectation, and exactly when
the preconditioner has full rank (P_hat = K_hat).

Hyperparameters are raw (l_1..l_D, s, sigma^2); optimising log(theta) goes through
torch's chain rule for exp.
"""
import math

import torch

from . import gp


class MarginalLogLikelihood(torch.autograd.Function):
    """mll = MarginalLogLikelihood.apply(theta, problem, y, k, n_probes, opts)."""

    @staticmethod
    def forward(ctx, theta, problem, y, k, n_probes, opts, workspace=None):
        problem.set_theta(theta.detach().to(torch.float64))
        st, out, iout = gp.gp_mll_and_grad(problem, y, k, n_probes, opts, workspace=workspace)
        dev_status = int(iout[gp.IOUT_STATUS].item())
        if st < 0 or dev_status < 0:
            code = st if st < 0 else dev_status
            raise RuntimeError(f"gp_mll_and_grad failed: {gp.status_string(code)}")
        if not bool(torch.isfinite(out[gp.OUT_MLL]).item()):
            raise RuntimeError("gp_mll_and_grad returned a non-finite MLL")
        p = problem.p
        grad = out[gp.OUT_HEAD:gp.OUT_HEAD + p].to(theta.device, theta.dtype)
        ctx.save_for_backward(grad)
        ctx.info = (st, iout)
        return out[gp.OUT_MLL].to(theta.device, theta.dtype)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None, None, None, None, None, None


def mll(theta, problem, y, k, n_probes, opts, workspace=None):
    return MarginalLogLikelihood.apply(theta, problem, y, k, n_probes, opts, workspace)


def adam_fit(problem, y, theta0, k, n_probes, opts, steps=20, lr=0.05, betas=(0.9, 0.999),
             eps=1e-8, seed0=0, callback=None):
    """Maximise the estimated MLL with Adam on log(theta) (Kingma & Ba 2015).

    Each step draws fresh probes (seed0 + step).  Returns (theta, history) where
    history holds (mll, theta) per step.  The update is a handful of scalar
    operations on the host; the evaluation is the CUDA estimator.
    """
    phi = torch.log(torch.as_tensor(theta0, dtype=torch.float64)).clone()
    m = torch.zeros_like(phi)
    v = torch.zeros_like(phi)
    ws = gp.Workspace()
    history = []
    for step in range(steps):
        o = gp.opts_with(opts, seed=seed0 + step)   # every other option as the caller set it
        x = phi.clone().requires_grad_(True)
        val = mll(torch.exp(x), problem, y, k, n_probes, o, ws)
        (-val).backward()
        g = x.grad.detach()
        m = betas[0] * m + (1 - betas[0]) * g
        v = betas[1] * v + (1 - betas[1]) * g * g
        mh = m / (1 - betas[0] ** (step + 1))
        vh = v / (1 - betas[1] ** (step + 1))
        phi = phi - lr * mh / (torch.sqrt(vh) + eps)
        history.append((float(val.detach()), torch.exp(phi).tolist()))
        if callback is not None:
            callback(step, history[-1])
    return torch.exp(phi), history
