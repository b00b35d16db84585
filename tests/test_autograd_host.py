"""Host logic of the autograd wrapper and the Adam loop (no GPU: the estimator call
is replaced by a fake that records what it was given)."""
import numpy as np
import pytest
import torch

from paper_2107_00243_gb300 import autograd, gp


class _FakeProblem:
    p = 3

    def __init__(self):
        self.theta = torch.tensor([0.5, 1.0, 0.1], dtype=torch.float64)

    def set_theta(self, th):
        self.theta = torch.as_tensor(th, dtype=torch.float64).clone()


def _fake_call(seen, status=0, dev_status=0, mll=-1.0):
    def call(problem, y, k, n_probes, o, workspace=None):
        seen.append(gp.opts_with(o))
        out = torch.zeros(gp.OUT_HEAD + 4 * problem.p + n_probes, dtype=torch.float64)
        out[gp.OUT_MLL] = mll
        th = problem.theta
        out[gp.OUT_HEAD:gp.OUT_HEAD + problem.p] = -(th - 0.3)     # a concave toy objective
        iout = torch.zeros(gp.IOUT_ITERS + n_probes + 1 + k, dtype=torch.int32)
        iout[gp.IOUT_STATUS] = dev_status
        return status, out, iout
    return call


def test_opts_with_copies_every_field():
    o = gp.opts(cg_tol=1e-3, max_iter=77, recompute_every=5, seed=9, pivchol_tol=1e-7,
                check_every=3, flags=gp.OPT_SPLIT_P | gp.OPT_FAST_ONLY)
    o2 = gp.opts_with(o, seed=42)
    for name, _ in o._fields_:
        want = 42 if name == "seed" else getattr(o, name)
        assert getattr(o2, name) == want, name
    with pytest.raises(KeyError):
        gp.opts_with(o, no_such_field=1)


def test_adam_fit_keeps_caller_flags(monkeypatch):
    """Every Adam step evaluates with the caller's options (flags included); only the
    probe seed changes from step to step."""
    seen = []
    monkeypatch.setattr(gp, "gp_mll_and_grad", _fake_call(seen))
    monkeypatch.setattr(gp, "Workspace", lambda: None)
    o = gp.opts(cg_tol=1e-2, max_iter=50, recompute_every=25, seed=0,
                flags=gp.OPT_SPLIT_P)
    theta, hist = autograd.adam_fit(_FakeProblem(), None, [0.5, 1.0, 0.1], 0, 2, o, steps=4,
                                    seed0=100)
    assert len(seen) == 4 and len(hist) == 4
    for step, s in enumerate(seen):
        assert s.flags == gp.OPT_SPLIT_P
        assert s.seed == 100 + step
        assert (s.cg_tol, s.max_iter, s.recompute_every) == (1e-2, 50, 25)


@pytest.mark.parametrize("status,dev_status,mll", [(-1, 0, -1.0), (0, -3, -1.0),
                                                   (0, -6, -1.0), (0, 0, float("nan"))])
def test_forward_raises_on_failed_evaluation(monkeypatch, status, dev_status, mll):
    monkeypatch.setattr(gp, "gp_mll_and_grad", _fake_call([], status, dev_status, mll))
    monkeypatch.setattr(gp, "status_string", lambda c: f"status {c}")
    theta = torch.tensor([0.5, 1.0, 0.1], dtype=torch.float64, requires_grad=True)
    with pytest.raises(RuntimeError):
        autograd.mll(theta, _FakeProblem(), None, 0, 2, gp.opts())


def test_forward_accepts_warnings(monkeypatch):
    """A positive status (e.g. not converged) still returns the estimate."""
    monkeypatch.setattr(gp, "gp_mll_and_grad", _fake_call([], 1, 1, -2.5))
    theta = torch.tensor([0.5, 1.0, 0.1], dtype=torch.float64, requires_grad=True)
    v = autograd.mll(theta, _FakeProblem(), None, 0, 2, gp.opts())
    assert float(v) == -2.5
    v.backward()
    np.testing.assert_allclose(theta.grad.numpy(), -(theta.detach().numpy() - 0.3))
