"""The tensor-core gradient contraction (Alg. 2's O(n^2) pass) and the mixed-precision
estimator on every kernel and mode the product ships, against the FP64 oracle, through
the C ABI.

Matched runs: the oracle's probes, pivots and per-column iteration counts are forced
on the GPU.  Each problem is evaluated twice in mixed precision, with the contraction
on the tensor cores (the default) and on CUDA cores in FP32 (GP_OPT_SIMT_GRAD).  CG
is identical in both (the contraction runs after it), so:
* the two MLLs agree bit for bit, and the difference of their contraction outputs
  isolates the tensor-core contraction's own arithmetic.  It evaluates k(r) from the
  product's exponent tile (BF16 hi / lo operands, |dS| ~ 2e-5 on these inputs), where
  the CUDA-core form uses FP32 differences; then FP16 hi / lo M operands with
  power-of-two column scales, H as FP16 hi + lo, FP16 hi / lo coordinates, FP32
  accumulation and an FP64 row combination.  A CPU emulation of every one of those rounding steps puts the
  gradient entries within 5.7e-4 of the exact contraction, relative to
  1/2 (|quad_p| + |trace_p|) (the output-scale entry of the isotropic Matern-3/2
  problem; 4.8e-4 of it from the exponent tile alone), and within 1.2e-4 without the
  exponent's error; the test allows 2e-3;
* every estimator result, and each gradient entry against 1/2 (|quad_p| + |trace_p|),
  is within the mixed-precision bound of 5e-3 of the oracle.
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


def _oracle(p):
    return estimator.mll_and_grad(p.kind, p.X, p.y, p.theta, p.ard, p.k, p.n_probes, p.tol,
                                  p.max_iter, seed=p.seed, recompute_every=p.recompute_every)


def _gpu(p, ref, flags=0):
    prob = gp.Problem(p.X, p.theta, p.kind, p.ard, gp.BF16)
    o = gp.opts(cg_tol=p.tol, max_iter=p.max_iter, recompute_every=p.recompute_every,
                seed=p.seed, flags=flags)
    st, out, iout = gp.gp_mll_and_grad(prob, p.y, p.k, p.n_probes, o, piv_override=ref["piv"],
                                       iters_override=ref["iters"])
    r = gp.unpack(out, iout, prob.p, p.n_probes, p.k)
    assert st >= 0 and r["status"] == 0, (st, r["status"])
    return r


def _errors(r, ref):
    scale = 0.5 * (np.abs(ref["quad_p"]) + np.abs(ref["trace_p"]))
    gk_ref = ref["quad_p"] - 0.5 * ref["probeK_p"]
    e = {k: abs(r[k] - ref[k]) / abs(ref[k]) for k in ("mll", "quad", "logdet")}
    e["grad"] = float(np.max(np.abs(r["grad"] - ref["grad"]) / scale))
    e["gK"] = float(np.max(np.abs(r["gK"] - gk_ref) / scale))
    return e, scale


PROBLEMS = {
    # the n = 1e5 RBF ARD workload's shape (d = 16, t = 33, k = 200, tol 1e-2)
    "rbf_ard_d16": lambda: workloads.subsample(
        workloads.c3_rbf_ard_1e5(n=20000, precision=gp.BF16), 2000),
    # the n = 5e5 Matern-3/2 ARD workload's shape (Gaussian-mixture inputs, d = 10, t = 17)
    "matern32_ard_d10": lambda: _with(workloads.subsample(workloads.c4_matern32_5e5(n=20000),
                                                          2000), k=100),
    # the n = 5e5 Matern-3/2 workload's own settings (k = 500, l = 16, tol 1e-2)
    "matern32_ard_c4_k500": lambda: workloads.subsample(workloads.c4_matern32_5e5(n=20000),
                                                        2000),
    # the Matern-5/2 ARD workload's shape (d = 8, t = 51, tol 1e-3)
    "matern52_ard_d8": lambda: _with(workloads.subsample(workloads.c2_matern52_ard(n=20000),
                                                         1500), n_probes=24),
    # isotropic lengthscales, ragged tails (n not a multiple of 128)
    "matern32_iso_d4": lambda: workloads.random_problem(1111, 4, kind=kernels.MATERN32,
                                                        ard=False, seed=3, s2=0.01, k=20,
                                                        n_probes=8, tol=1e-3, max_iter=500),
    # the rational quadratic kernel of the synthetic study (alpha = 1), ARD, d = 3
    "ratquad_ard_d3": lambda: workloads.random_problem(1500, 3, kind=kernels.RATQUAD,
                                                       ard=True, seed=9, s2=0.02, k=20,
                                                       n_probes=8, tol=1e-3, max_iter=500),
    "rbf_iso_d3": lambda: workloads.random_problem(777, 3, kind=kernels.RBF, ard=False,
                                                   seed=5, s2=0.05, k=12, n_probes=6,
                                                   tol=1e-4, max_iter=400),
    # one dimension; the widest supported input (d = 31, 128 coordinate columns)
    "matern52_ard_d1": lambda: workloads.random_problem(600, 1, kind=kernels.MATERN52,
                                                        ard=True, seed=7, s2=0.05, k=10,
                                                        n_probes=5, tol=1e-4, max_iter=400),
    "rbf_ard_d31": lambda: workloads.random_problem(900, 31, kind=kernels.RBF, ard=True,
                                                    seed=8, lo=1.0, hi=2.0, s2=0.05, k=10,
                                                    n_probes=4, tol=1e-4, max_iter=400),
    # a very smooth kernel (31 lengthscales in [2, 4]): fast mode's FP16 k(r)/s moves its
    # gradient entries by ~3e-2, which split mode removes (test_split_mode_vs_oracle)
    "rbf_ard_d31_smooth": lambda: workloads.random_problem(900, 31, kind=kernels.RBF,
                                                           ard=True, seed=8, lo=2.0, hi=4.0,
                                                           s2=0.05, k=10, n_probes=4,
                                                           tol=1e-4, max_iter=400),
}
FAST_MODE = sorted(k for k in PROBLEMS if not k.endswith("_smooth"))


def _with(p, **kw):
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("name", FAST_MODE)
def test_contraction_and_estimator_vs_oracle(name):
    p = PROBLEMS[name]()
    ref = _oracle(p)
    r_tc = _gpu(p, ref)
    r_simt = _gpu(p, ref, flags=gp.OPT_SIMT_GRAD)
    e_tc, scale = _errors(r_tc, ref)
    e_simt, _ = _errors(r_simt, ref)
    # identical CG: the contraction is the only difference
    assert r_tc["mll"] == r_simt["mll"]
    d_con = np.abs(r_tc["gK"] - r_simt["gK"]) / scale
    fmt = {"float_kind": lambda v: f"{v:.1e}"}
    print(name, "TC vs FP32 contraction:", np.array2string(d_con, formatter=fmt))
    print(name, "vs oracle (TC):", {k: f"{v:.1e}" for k, v in e_tc.items()},
          "(FP32 contraction):", {k: f"{v:.1e}" for k, v in e_simt.items()})
    g = np.abs(r_tc["grad"] - ref["grad"]) / scale
    print(name, "gradient entries vs oracle:", np.array2string(g, formatter=fmt))
    assert d_con.max() <= 2e-3, d_con
    assert all(v <= 5e-3 for v in e_tc.values()), e_tc


@pytest.mark.parametrize("name", ["rbf_ard_d16", "matern32_iso_d4", "rbf_ard_d31_smooth"])
def test_split_mode_vs_oracle(name):
    """GP_OPT_SPLIT_P (k(r)/s as FP16 hi + lo in the product) against the oracle."""
    p = PROBLEMS[name]()
    ref = _oracle(p)
    r = _gpu(p, ref, flags=gp.OPT_SPLIT_P)
    e, _ = _errors(r, ref)
    print(name, "split mode vs oracle:", {k: f"{v:.1e}" for k, v in e.items()})
    assert all(v <= 5e-3 for v in e.values()), e


def test_contraction_full_size_tc_vs_fp32():
    """n = 1e5, d = 16, t = 33: the tensor-core contraction against the FP32 CUDA-core
    one on the same CG solutions (identical MLL), and the phase timer of each.  No
    oracle at this size: entries are compared against |gK| + (|probeP| + |trP|) / 2 of
    the FP32 contraction's evaluation, a stand-in for 1/2 (|quad_p| + |trace_p|)."""
    p = workloads.c3_rbf_ard_1e5(precision=gp.BF16)
    prob = gp.Problem(p.X, p.theta, p.kind, p.ard, gp.BF16)
    res = {}
    gp.mvm_timing(True)
    try:
        for flags in (0, gp.OPT_SIMT_GRAD):
            gp.phase_timing_read(1)
            o = gp.opts(cg_tol=p.tol, max_iter=p.max_iter, recompute_every=p.recompute_every,
                        seed=0, flags=flags | gp.OPT_FAST_ONLY)
            st, out, iout = gp.gp_mll_and_grad(prob, p.y, p.k, p.n_probes, o)
            r = gp.unpack(out, iout, prob.p, p.n_probes, p.k)
            assert st == 0 and r["status"] == 0
            ms, cnt = gp.phase_timing_read(1)
            assert cnt == 1
            res[flags] = (r, ms)
    finally:
        gp.mvm_timing(False)
    (a, ms_tc), (b, ms_simt) = res[0], res[gp.OPT_SIMT_GRAD]
    assert a["mll"] == b["mll"]
    scale = np.abs(b["gK"]) + 0.5 * (np.abs(b["probeP_p"]) + np.abs(b["trP_p"]))
    d = np.abs(a["gK"] - b["gK"]) / scale
    print(f"contraction at n=1e5: tensor cores {ms_tc:.2f} ms, FP32 CUDA cores {ms_simt:.2f} ms;"
          f" max difference {d.max():.1e} of scale")
    assert d.max() <= 2e-3, d
