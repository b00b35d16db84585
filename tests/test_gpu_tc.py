"""The mixed-precision tensor-core (tcgen05) kernel product and estimator against
the FP64 oracle, through the C ABI.

Bounds come from the arithmetic:
* exponent tile S = -c r^2 / 2 (c = log2 e for RBF, 1 for Matern): each operand is
  split into BF16 hi + lo (16 significant bits) and the lo.lo product is dropped, so
  |S - S_ref| stays below ~2^-15 of the largest augmented term; with |terms| <= ~60
  here the test allows 5e-3 absolute.
* W = K V: P = k(S)/s is rounded to FP16 (relative error <= 2^-11), V is carried as
  FP16 hi + lo of a power-of-two scaled column (~2^-22), FP32 accumulation, so
  |W_i - W_ref_i| <= (2^-11 + small) (|K| |V|)_i; the test allows 2^-10 (|K||V|)_i.
* estimator results in mixed precision: the mixed-precision bound of 5e-3 relative per
  result (values; gradient entries against 1/2(|quad_p| + |trace_p|)).
"""
import numpy as np
import pytest
import torch

from oracle import estimator, kernels
from paper_2107_00243_gb300 import gp, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2107_00243_gb300 import build
    build.build()
    gp.load()


def _problem(n, d, kind, ard, seed=0, lo=0.3, hi=1.0, s=1.0, s2=0.05):
    return workloads.random_problem(n, d, kind=kind, ard=ard, seed=seed, lo=lo, hi=hi, s=s, s2=s2)


@pytest.mark.parametrize("kind", kernels.KINDS)
@pytest.mark.parametrize("d", [3, 16])
def test_exponent_tile(kind, d):
    n, t = 300, 7
    p = _problem(n, d, kind, True, seed=d, s=1.7)
    prob = gp.Problem(p.X, p.theta, kind, True, gp.BF16)
    V = torch.randn(n, t, dtype=torch.float64)
    W, S = gp.gp_tc_exponent_tile(prob, V)
    S = S.cpu().numpy().astype(np.float64)
    ls = p.theta[:d]
    r2 = kernels.scaled_r2(p.X[:128], p.X[:128], ls)
    if kind == kernels.RBF:
        ref = -0.5 * r2 / np.log(2.0)
    else:
        ref = -0.5 * r2
    err = np.abs(S - ref).max()
    assert err <= 5e-3, err


SHAPES = [(300, 3, 7), (1000, 16, 33), (129, 1, 1), (517, 8, 17), (256, 12, 64)]


@pytest.mark.parametrize("kind", kernels.KINDS)
@pytest.mark.parametrize("ard", [True, False])
@pytest.mark.parametrize("shape", SHAPES)
def test_kernel_mvm_bf16(kind, ard, shape):
    n, d, t = shape
    p = _problem(n, d, kind, ard, seed=n + t)
    V = np.random.default_rng(7).standard_normal((n, t))
    op = kernels.KernelOperator(kind, p.X, p.theta, ard)
    ref = op.matvec(V)
    K = kernels.kernel_block(kind, p.X, p.X, p.theta, ard)
    bound = 2.0 ** -10 * (np.abs(K) @ np.abs(V)) + 1e-6
    prob = gp.Problem(p.X, p.theta, kind, ard, gp.BF16)
    got = gp.gp_kernel_mvm(prob, torch.from_numpy(V)).cpu().numpy()
    excess = (np.abs(got - ref) / bound).max()
    assert excess <= 1.0, excess


def test_kernel_mvm_bf16_full_size_sampled_rows():
    """n=1e5, d=16, t=33: 64 sampled rows against the oracle, row by row."""
    p = workloads.c3_rbf_ard_1e5(precision=gp.BF16)
    V = np.random.default_rng(5).standard_normal((p.n, 33))
    prob = gp.Problem(p.X, p.theta, p.kind, p.ard, gp.BF16)
    got = gp.gp_kernel_mvm(prob, torch.from_numpy(V)).cpu().numpy()
    rows = np.random.default_rng(6).choice(p.n, 64, replace=False)
    Kr = kernels.kernel_block(p.kind, p.X[rows], p.X, p.theta, p.ard)
    ref = Kr @ V + p.theta[-1] * V[rows]
    bound = 2.0 ** -10 * (np.abs(Kr) @ np.abs(V)) + 1e-6
    assert (np.abs(got[rows] - ref) / bound).max() <= 1.0


def _compare(r, ref, tol):
    errs = {
        "mll": abs(r["mll"] - ref["mll"]) / abs(ref["mll"]),
        "quad": abs(r["quad"] - ref["quad"]) / abs(ref["quad"]),
        "logdet": abs(r["logdet"] - ref["logdet"]) / abs(ref["logdet"]),
    }
    scale = 0.5 * (np.abs(ref["quad_p"]) + np.abs(ref["trace_p"]))
    g = np.abs(r["grad"] - ref["grad"]) / scale
    errs["grad_max"] = float(g.max())
    print("mixed-precision per-result relative errors:",
          {k: f"{v:.2e}" for k, v in errs.items()}, "grad:", np.array2string(g, precision=2))
    assert all(v <= tol for v in errs.values()), errs


@pytest.mark.parametrize("n", [3000])
def test_estimator_bf16_matched(n):
    """RBF ARD d=16 (the n=1e5 workload's shape: k=200, l=32, tol 1e-2, recompute 25)
    on a subsample, BF16 tiles, same probes, pivots and iteration counts."""
    p = workloads.subsample(workloads.c3_rbf_ard_1e5(n=20000, precision=gp.BF16), n)
    ref = estimator.mll_and_grad(p.kind, p.X, p.y, p.theta, p.ard, p.k, p.n_probes, p.tol,
                                 p.max_iter, seed=p.seed, recompute_every=p.recompute_every)
    prob = gp.Problem(p.X, p.theta, p.kind, p.ard, gp.BF16)
    o = gp.opts(cg_tol=p.tol, max_iter=p.max_iter, recompute_every=p.recompute_every,
                seed=p.seed)
    st, out, iout = gp.gp_mll_and_grad(prob, p.y, p.k, p.n_probes, o, piv_override=ref["piv"],
                                       iters_override=ref["iters"])
    r = gp.unpack(out, iout, prob.p, p.n_probes, p.k)
    assert st >= 0 and r["status"] == 0
    _compare(r, ref, 5e-3)


def test_estimator_bf16_full_size():
    """The whole estimator at n=1e5 in mixed precision: finite, full rank, every
    column stopped by the tolerance; MLL within 5e-3 of the FP32 form's."""
    p = workloads.c3_rbf_ard_1e5(precision=gp.BF16)
    o = gp.opts(cg_tol=p.tol, max_iter=p.max_iter, recompute_every=p.recompute_every, seed=0)
    res = {}
    for prec in (gp.BF16, gp.FP32):
        prob = gp.Problem(p.X, p.theta, p.kind, p.ard, prec)
        st, out, iout = gp.gp_mll_and_grad(prob, p.y, p.k, p.n_probes, o)
        r = gp.unpack(out, iout, prob.p, p.n_probes, p.k)
        assert st == 0 and r["rank"] == p.k
        assert np.all(np.isfinite(out.cpu().numpy()))
        assert np.all(r["iters"] < p.max_iter)
        res[prec] = r
    a, b = res[gp.BF16], res[gp.FP32]
    assert abs(a["mll"] - b["mll"]) <= 5e-3 * abs(b["mll"])


def test_autotune_records_config_and_keeps_product():
    """The tuner times its candidates, records the fastest for this shape, and the
    product stays within the same bound under the tuned configuration."""
    n, d, t = 3000, 8, 17
    p = _problem(n, d, kernels.RBF, True, seed=13)
    prob = gp.Problem(p.X, p.theta, p.kind, True, gp.BF16)
    V = np.random.default_rng(2).standard_normal((n, t))
    W, best = gp.gp_autotune(prob, torch.from_numpy(V))
    assert best["candidates"] >= 3 and best["chunks"] >= 1
    cfg = gp.gp_tc_config(prob, t)
    assert cfg["tuned"]
    assert (cfg["chunks"], cfg["b_ring"], cfg["v_ring"]) == (best["chunks"], best["b_ring"],
                                                            best["v_ring"])
    op = kernels.KernelOperator(p.kind, p.X, p.theta, True)
    K = kernels.kernel_block(p.kind, p.X, p.X, p.theta, True)
    ref = op.matvec(V)
    bound = 2.0 ** -10 * (np.abs(K) @ np.abs(V)) + 1e-6
    for got in (W.cpu().numpy(), gp.gp_kernel_mvm(prob, torch.from_numpy(V)).cpu().numpy()):
        assert (np.abs(got - ref) / bound).max() <= 1.0
