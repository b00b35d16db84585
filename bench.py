#!/usr/bin/env python
"""Seconds per MLL + gradient evaluation of the preconditioned GP estimator.

Workload (synthetic stand-in for the paper's UCI regressions, Sec. 5): n = 100,000
points uniform on [0,1]^16, targets a sum of 16 random sinusoids plus noise, RBF
ARD kernel with lengthscales in [0.2, 1], s = 1, sigma^2 = 0.01; pivoted-Cholesky
preconditioner of rank k = 200, l = 32 probes, CG tolerance 1e-2, true residual
every 25 steps.  One step = one call of gp_mll_and_grad (Alg. 1 + Alg. 2: pivoted
Cholesky, Woodbury core, probes, mBCG, Lanczos quadrature, gradient contraction,
preconditioner terms) on inputs resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision bf16|tf32|fp32]

Prints one JSON line (rank 0).  Under torchrun each rank evaluates its own replica
(the estimator does not shard; the metric is whole-job seconds per evaluation).
``--impl reference`` times the FP64 CPU oracle on a bounded sample instead.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "s per MLL+grad eval at N=1e5 (mixed vs FP32 GPU); kernel-MVM TFLOP/s vs peak"
WORKLOAD = "rbf_ard_n100000_d16_k200_l32_tol1e-2"
SM_COUNT, FP32_LANES = 152, 128


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


def _traffic_from_profiles(kernel_tag):
    """Per-launch DRAM bytes of a kernel from an ncu capture (profiles/dram_traffic.txt:
    tag, bytes, source file, sha256[:16] of that file when the counters were taken).
    None when there is no entry or the source has changed since."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 4 and parts[0] == kernel_tag:
                src = os.path.join(ROOT, parts[2])
                if not os.path.exists(src):
                    return None
                with open(src, "rb") as g:
                    if hashlib.sha256(g.read()).hexdigest()[:16] != parts[3]:
                        return None
                try:
                    return float(parts[1])
                except ValueError:
                    return None
    return None


def _unit_peak(key):
    """A measured unit throughput from profiles/unit_peaks_gb300.txt (key, value), or
    None when the file or the key is missing."""
    path = os.path.join(ROOT, "profiles", "unit_peaks_gb300.txt")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 2 and parts[0] == key:
                try:
                    return float(parts[1])
                except ValueError:
                    return None
    return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = max(smax, float(r[2]))
                for name, v in zip(names, r[5:9]):
                    if v.strip() == "Active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0, None
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", "0"))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return rank, ws, local, dist


def _max_over_ranks(value, dist):
    if dist is None:
        return value
    import torch
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(dist):
    if dist is not None:
        dist.barrier()


# CG iterations (max over the 33 columns) this workload needs at tol 1e-2, measured
# with the FP32 GPU form; used only to scale the oracle's timing in the reference arm.
WORKLOAD_MAX_ITERS = 323
SUBSAMPLE_N = 2000


def _cpu_info():
    """CPU model, logical cores and the threads the oracle's BLAS uses."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.TimeoutExpired):
        pass
    try:
        from threadpoolctl import threadpool_info
        threads = max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except Exception:
        threads = os.cpu_count() or 1
    return {"cpu_model": model, "nproc": os.cpu_count(), "threads": threads}


def products_per_eval(max_iters, recompute_every=25, n_hyper=18):
    """Kernel-product equivalents of one oracle evaluation: one per CG iteration, one
    per residual recompute, and two derivative passes over all p - 1 kernel
    derivatives for the gradient (K_hat^-1 y and the probe solves)."""
    return max_iters + math.ceil(max_iters / recompute_every) + 2 * (n_hyper - 1)


def oracle_subsample_seconds(n_sub=SUBSAMPLE_N):
    """The FP64 oracle estimator (MLL and gradient, Alg. 1 + Alg. 2) end to end on an
    n_sub-point subsample of the n = 1e5 workload (same d, kernel, k, l, tol): seconds
    and the largest CG iteration count."""
    from oracle import estimator
    from paper_2107_00243_gb300 import workloads
    p = workloads.subsample(workloads.c3_rbf_ard_1e5(n=20000), n_sub)
    t0 = time.perf_counter()
    r = estimator.mll_and_grad(p.kind, p.X, p.y, p.theta, p.ard, p.k, p.n_probes, p.tol,
                               p.max_iter, seed=p.seed, recompute_every=p.recompute_every)
    return time.perf_counter() - t0, int(max(r["iters"]))


def extrapolate(t_sub, m_sub, m_full, n_full=100000, n_sub=SUBSAMPLE_N, n_hyper=18):
    """Scale a subsample's time to the full workload: (n / n_sub)^2 per kernel product,
    times the ratio of product-equivalents per evaluation at the two sizes."""
    return (t_sub * (n_full / n_sub) ** 2 * products_per_eval(m_full, 25, n_hyper)
            / products_per_eval(m_sub, 25, n_hyper))


def oracle_small_configs():
    """Oracle timings beside the bench line (about 10 s of host work in all):
    * timed, not scaled: the oracle estimator and the exact dense-Cholesky MLL and
      gradient on the small RBF workload (n = 1,000, d = 3) and on a 1,500-point
      subsample of the Matern-5/2 ARD workload (d = 8, k = 100, l = 50, tol 1e-3);
    * one kernel product K_hat V of the n = 1e5 RBF workload (t = 33) and of the n = 5e5
      Matern-3/2 workload (t = 17), timed on 200 and 50 rows (the oracle's own kernel
      blocks times V) and scaled by the row count to the full product (labelled)."""
    import numpy as np
    from oracle import estimator, exact, kernels
    from paper_2107_00243_gb300 import workloads
    out = {}
    for name, p in (("small_rbf_n1000", workloads.c1_small_rbf()),
                    ("matern52_ard_subsample_n1500",
                     workloads.subsample(workloads.c2_matern52_ard(), 1500))):
        t0 = time.perf_counter()
        estimator.mll_and_grad(p.kind, p.X, p.y, p.theta, p.ard, p.k, p.n_probes, p.tol,
                               p.max_iter, seed=p.seed)
        t1 = time.perf_counter()
        exact.exact_mll_and_grad(p.kind, p.X, p.y, p.theta, p.ard)
        t2 = time.perf_counter()
        out[f"{name}_estimator_s"] = t1 - t0
        out[f"{name}_exact_s"] = t2 - t1
    for name, p, t, rows in (("rbf_ard_n1e5", workloads.c3_rbf_ard_1e5(), 33, 200),
                             ("matern32_ard_n5e5", workloads.c4_matern32_5e5(), 17, 50)):
        V = np.random.default_rng(0).standard_normal((p.n, t))
        t0 = time.perf_counter()
        kernels.kernel_block(p.kind, p.X[:rows], p.X, p.theta, p.ard) @ V
        dt = time.perf_counter() - t0
        out[f"{name}_product_{rows}_rows_s"] = dt
        out[f"{name}_product_s_extrapolated"] = dt * p.n / rows
    return out


def run_reference(args, rank, ws, dist):
    if rank != 0:
        _barrier(dist)
        return
    sample_times, m_sub = [], 0
    for i in range(args.warmup + args.steps):
        t_sub, m_sub = oracle_subsample_seconds()
        if i >= args.warmup:
            sample_times.append(t_sub)
    t_mean = statistics.mean(sample_times)
    value = extrapolate(t_mean, m_sub, WORKLOAD_MAX_ITERS)
    info = _cpu_info()
    sample = (f"extrapolated: each of the {args.steps} timed steps ran the FP64 oracle "
              f"estimator (MLL + gradient) end to end on a {SUBSAMPLE_N}-point subsample of "
              f"the n=1e5 workload ({t_mean:.2f} s mean, {m_sub} CG iterations); the value "
              f"scales that by (1e5/{SUBSAMPLE_N})^2 and by the product-equivalents per "
              f"evaluation ({WORKLOAD_MAX_ITERS} CG iterations at n=1e5)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "fp64-cpu-oracle"},
            "extrapolated": True, "steps_run": len(sample_times),
            "sample_s_per_step": sample_times,
            "cpu_baseline": {"value": value, "unit": "s", "cores": info["threads"],
                             "kind": "oracle", "sample": sample, **info},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    _barrier(dist)


def run_peaks():
    """Throughput peaks the HBM-copy and BF16-GEMM measurements do not cover: FP32 FMA,
    MUFU ex2 (FP32 and FP16x2), FP64 FMA (the library's microbenchmarks), and TF32 GEMM
    (cuBLAS through torch.matmul, 8192^3, best of 5)."""
    import torch
    from paper_2107_00243_gb300 import build, gp
    build.build()
    gp.load()
    res = gp.measure_peaks()
    n = 8192
    a = torch.randn(n, n, device="cuda")
    b = torch.randn(n, n, device="cuda")
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        torch.matmul(a, b)
        best = 1e30
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    res["tf32_gemm_flops"] = 2.0 * n ** 3 / best
    dev = torch.cuda.get_device_properties(0)
    res["device"] = dev.name
    res["sms"] = dev.multi_processor_count
    print(json.dumps({k: (float(f"{v:.4g}") if isinstance(v, float) else v)
                      for k, v in res.items()}))


def run_case(args):
    """Time one building block on a smaller instance of the workload (same d, kernel,
    hyperparameters; n points drawn the same way).  Used for profiling captures."""
    import torch
    from paper_2107_00243_gb300 import build, gp, workloads
    build.build()
    gp.load()
    prec = {"bf16": gp.BF16, "tf32": gp.TF32, "fp32": gp.FP32}[args.precision]
    p = workloads.c3_rbf_ard_1e5(n=args.n or 100000, precision=prec)
    prob = gp.Problem(p.X, p.theta, p.kind, p.ard, prec)
    t = p.n_probes + 1
    gen = torch.Generator(device="cuda").manual_seed(0)
    V = torch.randn(p.n, t, device="cuda", generator=gen)
    times = []
    if args.case == "grad":
        # the estimator with CG capped at 4 iterations: one gradient contraction per call
        o = gp.opts(cg_tol=p.tol, max_iter=4, recompute_every=p.recompute_every, seed=0,
                    flags=gp.OPT_FAST_ONLY)
        gp.mvm_timing(True)
        for _ in range(args.reps):
            gp.phase_timing_read(1)
            gp.gp_mll_and_grad(prob, p.y, p.k, p.n_probes, o)
            torch.cuda.synchronize()
            times.append(gp.phase_timing_read(1)[0])
        gp.mvm_timing(False)
    elif args.case == "kmvm":
        for _ in range(args.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            gp.gp_kernel_mvm(prob, V)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    else:
        # 20 CG iterations (the tolerance is out of reach, so every column runs them all);
        # phase 0 times the products, phase 2 the rest of each iteration
        L, piv, rank = gp.gp_pivchol(prob, p.k)
        its = 20
        o = gp.opts(cg_tol=1e-12, max_iter=its, recompute_every=0, seed=0)
        gp.mvm_timing(True)
        side = []
        for _ in range(args.reps):
            gp.phase_timing_read(0)
            gp.phase_timing_read(2)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            gp.gp_mbcg(prob, L, V, o)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            prod_ms, prod_n = gp.phase_timing_read(0)
            side_ms, side_n = gp.phase_timing_read(2)
            side.append({"products_ms": prod_ms, "products": prod_n, "cg_side_ms": side_ms,
                         "iterations": side_n // 2,
                         # the whole call less its products, per iteration (includes the
                         # set-up and the first preconditioner solve)
                         "call_less_products_ms_per_iteration": (times[-1] - prod_ms) / its})
        gp.mvm_timing(False)
        per = [x["cg_side_ms"] / max(x["iterations"], 1) for x in side[1:] or side]
        best = min(per) if min(per) > 0 else float("nan")
        esz = 4 if prec != gp.FP64 else 8
        # algorithmic bytes of one iteration's CG side: L streamed twice, and the n x t
        # vectors: P, Q (alpha); X, P, Q, R read and X, R written (update); R (L^T R);
        # R read, Z written (z); P, Z read and P written (direction)
        traffic = (2 * p.n * p.k + 14 * p.n * t) * esz
        fmas = 2 * p.n * p.k * t
        print(json.dumps({"case": "cg_side", "n": p.n, "k": p.k, "t": t,
                          "precision": args.precision, "ms_per_iteration": best,
                          "ms_per_iteration_all": per, "algorithmic_bytes": traffic,
                          "achieved_gbs": traffic / (best * 1e-3) / 1e9,
                          "fma_per_iteration": fmas,
                          "achieved_fp32_tflops": 2 * fmas / (best * 1e-3) / 1e12,
                          "calls": side}), flush=True)
    print(json.dumps({"case": args.case, "n": p.n, "t": t, "precision": args.precision,
                      "ms": times}), flush=True)


def run_batched(args):
    """The batched workload: 64 independent RBF problems (n log-uniform in [2000,
    50000], d in {4, 8, 12}, own lengthscale and noise; k = 50, l = 16, CG tol 1e-2,
    BF16 tiles with the automatic split choice), one gp_mll_and_grad_batched call per
    step (a cached CUDA graph after the first).  Launch configurations are autotuned
    per shape first.  Reference point: the same 64 evaluations as eager single calls
    one after another."""
    import numpy as np
    import torch
    from paper_2107_00243_gb300 import build, gp, workloads
    build.build()
    gp.load()
    ps = workloads.c5_batched(64, seed=0)
    probs = [gp.Problem(p.X, p.theta, p.kind, p.ard, gp.BF16) for p in ps]
    k, nl = ps[0].k, ps[0].n_probes
    o = gp.opts(cg_tol=ps[0].tol, max_iter=ps[0].max_iter, recompute_every=25, seed=0,
                flags=gp.OPT_AUTO_SPLIT)
    tuned = {}
    t0 = time.perf_counter()
    for pr in probs:                                   # one tuning run per shape key
        key = (pr.d, int(math.ceil(math.log2(max(pr.n / 128.0, 1.0)))))
        if key not in tuned:
            V = torch.randn(pr.n, nl + 1, device="cuda")
            _, best = gp.gp_autotune(pr, V)
            tuned[key] = best
    tune_s = time.perf_counter() - t0
    b = gp.Batch(probs, [p.y for p in ps], k, nl, o)
    t0 = time.perf_counter()
    b.run()                                            # records and instantiates the graph
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t0
    for _ in range(max(args.warmup - 1, 0)):
        b.run()
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.run()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    res = b.results()
    # the same evaluations as eager single calls, one after another
    seq = 0.0
    ws = gp.Workspace()
    for i, (pr, y) in enumerate(zip(probs, b.ys)):
        oi = gp.opts(cg_tol=o.cg_tol, max_iter=o.max_iter, recompute_every=25, seed=i,
                     flags=gp.OPT_AUTO_SPLIT)
        gp.gp_mll_and_grad(pr, y, k, nl, oi, workspace=ws)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        gp.gp_mll_and_grad(pr, y, k, nl, oi, workspace=ws)
        e1.record()
        torch.cuda.synchronize()
        seq += e0.elapsed_time(e1) / 1e3
    value = statistics.median(times)
    line = {"case": "batched", "metric": "s per batched MLL+grad step (64 problems)",
            "value": value, "unit": "s", "higher_is_better": False, "steps": args.steps,
            "warmup": args.warmup, "problems_per_s": 64.0 / value,
            "sequential_single_calls_s": seq, "speedup_vs_sequential": seq / value,
            "first_call_s_incl_capture": first_s, "autotune_s": tune_s,
            "tuned_shapes": {f"d{d}_b{b_}": v for (d, b_), v in tuned.items()},
            "n_range": [min(p.n for p in ps), max(p.n for p in ps)],
            "statuses": sorted(set(r["status"] for r in res)),
            "iters_max": int(max(int(r["iters"].max()) for r in res)),
            "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "rbf_batched64_n2e3-5e4_k50_l16_tol1e-2"}}
    print(json.dumps(line), flush=True)


def run_c4(args):
    """The large Matern-3/2 workload (n = 500,000 points of a 20-component Gaussian
    mixture in d = 10, cubic-polynomial targets; Matern-3/2 ARD, k = 500, l = 16, CG
    tol 1e-2): 20 Adam steps (lr 0.05) on log-hyperparameters through the autograd
    wrapper of gp_mll_and_grad.  Tiles: the BF16 hi / lo exponent GEMM and FP16 k(r)/s
    of the mixed path stand in for TF32 tiles (FP16 carries TF32's 10 explicit mantissa
    bits at twice the tensor rate).  Prints per-step seconds and the MLL trajectory."""
    import torch
    from paper_2107_00243_gb300 import autograd, build, gp, workloads
    build.build()
    gp.load()
    p = workloads.c4_matern32_5e5(n=args.n or 500000)
    steps, lr = p.extra["adam_steps"], p.extra["lr"]
    prob = gp.Problem(p.X, p.theta, p.kind, p.ard, gp.BF16)
    # at this size FP16 k(r)/s perturbs K by up to 2^-11 lambda_max(K) ~ 6, far above
    # sigma^2 = 0.1, so fast mode cannot run: the device-side Gershgorin rule picks split
    # mode (FP16 hi + lo k(r)/s and the three-part exponent operands) before CG
    o = gp.opts(cg_tol=p.tol, max_iter=p.max_iter, recompute_every=25, seed=0,
                flags=gp.OPT_AUTO_SPLIT)
    y = torch.as_tensor(p.y).to(device="cuda", dtype=prob.dtype)
    marks = [time.perf_counter()]

    def cb(step, rec):
        torch.cuda.synchronize()
        marks.append(time.perf_counter())
        print(json.dumps({"step": step, "s": marks[-1] - marks[-2], "mll": rec[0],
                          "theta": rec[1]}), flush=True)

    theta, hist = autograd.adam_fit(prob, y, p.theta, p.k, p.n_probes, o, steps=steps, lr=lr,
                                    callback=cb)
    step_s = [b - a for a, b in zip(marks[:-1], marks[1:])]
    # one more evaluation at the final hyperparameters, for its iterations and status
    prob.set_theta(theta.numpy())
    st, out, iout = gp.gp_mll_and_grad(prob, y, p.k, p.n_probes, gp.opts_with(o, seed=steps))
    r = gp.unpack(out, iout, prob.p, p.n_probes, p.k)
    line = {"case": "c4", "config": {"workload": f"matern32_ard_n{p.n}_d10_k500_l16_tol1e-2",
                                     "adam_steps": steps, "lr": lr,
                                     "tiles": "bf16 hi/lo exponent, fp16 k(r)/s (for tf32)"},
            "s_per_step": step_s, "mean_s_per_step": statistics.mean(step_s),
            "total_s": sum(step_s), "mll": [h[0] for h in hist],
            "theta0": p.theta.tolist(), "theta_final": [float(x) for x in theta],
            "final": {"status": r["status"], "mll": r["mll"], "rank": r["rank"],
                      "iters_max": int(r["iters"].max()), "iters_min": int(r["iters"].min())},
            "dtype": "bf16", "data": "synthetic"}
    print(json.dumps(line), flush=True)


def run_synthetic(args):
    """The bias / variance study of the paper's synthetic experiment (Tab. S1): n = 10,000
    points, d in {1, 2, 3}, RBF, Matern-3/2 and rational quadratic kernels, l = 128
    probes, 25 probe seeds, with no preconditioner (k = 0) and with a rank-128 pivoted
    Cholesky preconditioner.  Relative bias |mean - exact| / |exact| and relative
    variance var / exact^2 of the MLL estimate and of each gradient entry (lengthscale,
    output scale, noise) against the exact values of
    tests/golden/synthetic_study_exact.json (dense Cholesky, FP64 oracle).  k = 0 runs
    in FP32 (CG tol 1e-5: its errors are 1e-5 and larger), k = 128 in FP64 (CG tol 1e-10).
    Where K is numerically low-rank (d = 1, and d = 2 for the smooth kernels) the factor
    stops below 128 at the FP64 rounding floor of its residual; the rank column shows it.
    Prints one JSON line per (kernel, d, k) and a markdown table."""
    import numpy as np
    import torch
    from paper_2107_00243_gb300 import build, gp, workloads
    build.build()
    gp.load()
    with open(os.path.join(ROOT, "tests", "golden", "synthetic_study_exact.json")) as f:
        exact = json.load(f)["problems"]
    names = {workloads.RBF: "RBF", workloads.MATERN32: "Matern32", workloads.RATQUAD: "RatQuad"}
    seeds = args.reps if args.reps and args.reps > 3 else 25
    rows = []
    only = None
    if args.rows:
        only = {tuple(int(v) for v in r.split(":")) for r in args.rows.split(",")}
    for kind in (workloads.MATERN32, workloads.RBF, workloads.RATQUAD):
        for d in (1, 2, 3):
            if only is not None and (kind, d) not in only:
                continue
            p = workloads.synthetic_study(kind, d)
            ex = exact[f"{kind}_{d}"]
            ref = np.array([ex["mll"]] + ex["grad"])
            for k, prec, tol in ((0, gp.FP32, 1e-5), (128, gp.FP64, 1e-10)):
                prob = gp.Problem(p.X, p.theta, p.kind, p.ard, prec)
                ws = gp.Workspace()
                vals, its, ranks, t0 = [], [], [], time.perf_counter()
                for sd in range(seeds):
                    o = gp.opts(cg_tol=tol, max_iter=1000, recompute_every=50, seed=sd)
                    st, out, iout = gp.gp_mll_and_grad(prob, p.y, k, p.n_probes, o, workspace=ws)
                    r = gp.unpack(out, iout, prob.p, p.n_probes, k)
                    vals.append([r["mll"]] + list(r["grad"]))
                    its.append(int(r["iters"].max()))
                    ranks.append(r["rank"])
                vals = np.array(vals)
                bias = np.abs(vals.mean(0) - ref) / np.abs(ref)
                var = vals.var(0, ddof=1) / ref ** 2
                row = {"kernel": names[kind], "d": d, "k": k, "n_probes": p.n_probes,
                       "precision": "fp64" if prec == gp.FP64 else "fp32", "seeds": seeds,
                       "bias": {"mll": bias[0], "lengthscale": bias[1], "outputscale": bias[2],
                                "noise": bias[3]},
                       "var": {"mll": var[0], "lengthscale": var[1], "outputscale": var[2],
                               "noise": var[3]},
                       "rank": max(ranks), "cg_iters_max": max(its),
                       "s": time.perf_counter() - t0}
                rows.append(row)
                print(json.dumps(row), flush=True)
    print("| kernel | d | k (rank) | MLL bias | MLL var | d/ds bias | d/ds var | d/dl bias "
          "| d/dl var | d/dsigma2 bias | d/dsigma2 var | CG its |")
    print("|---|---|---|---|---|---|---|---|---|---|---|---|")
    for r in rows:
        b, v = r["bias"], r["var"]
        print(f"| {r['kernel']} | {r['d']} | {r['k']} ({r['rank']}) | {b['mll']:.0e} | "
              f"{v['mll']:.0e} | "
              f"{b['outputscale']:.0e} | {v['outputscale']:.0e} | {b['lengthscale']:.0e} | "
              f"{v['lengthscale']:.0e} | {b['noise']:.0e} | {v['noise']:.0e} | "
              f"{r['cg_iters_max']} |")


def run_decay(args):
    """The residual-decay experiment (Fig. 2; rates of Tab. 2): as the rank k of the partial
    Cholesky preconditioner (or the number of random Fourier features, mean over four
    draws, or of quadrature Fourier features for the RBF kernel) grows, log det P_hat_k -> log det K_hat and tr(P_hat_k^-1 dP_hat_k) ->
    tr(K_hat^-1 dK_hat) for every hyperparameter, at the rate at which P_hat_k -> K_hat
    (the residual trace tr(K - L L^T) / tr K).  Four n = 1,000 problems of the synthetic
    study's generator (RBF and Matern-3/2, d = 1 and 3), FP64; the exact values are
    tests/golden/residual_decay_exact.json (dense Cholesky, FP64 oracle).  Prints one
    JSON line per (problem, k) and a markdown table."""
    import torch
    from paper_2107_00243_gb300 import build, gp, workloads
    build.build()
    gp.load()
    with open(os.path.join(ROOT, "tests", "golden", "residual_decay_exact.json")) as f:
        gold = json.load(f)
    names = {workloads.RBF: "RBF", workloads.MATERN32: "Matern32"}
    ks = [0, 1, 2, 4, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256]
    rows = []
    for key, ex in gold["problems"].items():
        kind, d = (int(v) for v in key.split("_"))
        p = workloads.synthetic_study(kind, d, n=gold["n"])
        prob = gp.Problem(p.X, p.theta, p.kind, p.ard, gp.FP64)
        o = gp.opts(cg_tol=1e-10, max_iter=1, seed=0)      # CG is not needed here
        trK = p.n * p.theta[-2]                            # noise-free tr K
        for k in ks:
            st, out, iout = gp.gp_mll_and_grad(prob, p.y, k, 1, o)
            r = gp.unpack(out, iout, prob.p, 1, k)
            res = 1.0
            if k > 0:
                L, _, _ = gp.gp_pivchol(prob, k)
                res = max(trK - float((L.double() ** 2).sum()), 0.0) / trK
            e_ld = abs(r["logdetP"] - ex["logdet"]) / abs(ex["logdet"])
            tp = [float(v) for v in ex["trace_p"]]
            e_tr = [abs(float(a) - b) / abs(b) for a, b in zip(r["trP_p"], tp)]
            row = {"kernel": names[kind], "d": d, "n": p.n, "preconditioner": "cholesky",
                   "k": k, "rank": r["rank"], "residual_trace": res, "logdet_rel_err": e_ld,
                   "trace_rel_err": {"lengthscale": e_tr[0], "outputscale": e_tr[1],
                                     "noise": e_tr[2]}}
            rows.append(row)
            print(json.dumps(row), flush=True)
        # random Fourier features (Tab. 2: error ~ k^-1/2), the mean over four draws
        for k in (16, 64, 256, 1000):
            m = k // 2
            acc = [0.0, 0.0, 0.0, 0.0]
            for draw in range(4):
                eps, g = workloads.rff_draws(m, d, gp.rff_gamma_shape(kind), seed=draw)
                st, out, iout = gp.gp_mll_and_grad_rff(prob, p.y, m, 1, o, eps, g)
                r = gp.unpack(out, iout, prob.p, 1, k)
                acc[0] += abs(r["logdetP"] - ex["logdet"]) / abs(ex["logdet"]) / 4
                for q in range(3):
                    acc[1 + q] += abs(float(r["trP_p"][q]) - float(ex["trace_p"][q])) / abs(
                        float(ex["trace_p"][q])) / 4
            row = {"kernel": names[kind], "d": d, "n": p.n, "preconditioner": "rff", "k": k,
                   "rank": k, "residual_trace": float("nan"), "logdet_rel_err": acc[0],
                   "trace_rel_err": {"lengthscale": acc[1], "outputscale": acc[2],
                                     "noise": acc[3]}, "draws": 4}
            rows.append(row)
            print(json.dumps(row), flush=True)
        # quadrature Fourier features (RBF only; Tab. 2: error ~ exp(-b k^(1/d)))
        if kind != workloads.RBF:
            continue
        for mbar in ((4, 8, 16, 32) if d == 1 else (2, 4, 6, 8)):
            k = mbar ** d
            st, out, iout = gp.gp_mll_and_grad_qff(prob, p.y, mbar, 1, o)
            r = gp.unpack(out, iout, prob.p, 1, k)
            e_tr = [abs(float(a) - float(b)) / abs(float(b))
                    for a, b in zip(r["trP_p"], ex["trace_p"])]
            row = {"kernel": names[kind], "d": d, "n": p.n, "preconditioner": "qff", "k": k,
                   "rank": r["rank"], "residual_trace": float("nan"),
                   "logdet_rel_err": abs(r["logdetP"] - ex["logdet"]) / abs(ex["logdet"]),
                   "trace_rel_err": {"lengthscale": e_tr[0], "outputscale": e_tr[1],
                                     "noise": e_tr[2]}, "nodes_per_dim": mbar}
            rows.append(row)
            print(json.dumps(row), flush=True)
    print("| kernel | d | preconditioner | k (rank) | tr(K - LL^T) / tr K | log det rel. err | "
          "tr d/dl rel. err | tr d/ds rel. err | tr d/dsigma2 rel. err |")
    print("|---|---|---|---|---|---|---|---|---|")
    for r in rows:
        t = r["trace_rel_err"]
        print(f"| {r['kernel']} | {r['d']} | {r['preconditioner']} | {r['k']} ({r['rank']}) | "
              f"{r['residual_trace']:.1e} | {r['logdet_rel_err']:.1e} | {t['lengthscale']:.1e} | "
              f"{t['outputscale']:.1e} | {t['noise']:.1e} |")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["bf16", "tf32", "fp32"], default="bf16")
    ap.add_argument("--fp32-steps", type=int, default=1,
                    help="timed steps of the plain FP32 form when --precision is mixed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rows", default="",
                    help="synthetic: only these kernel:d problems, e.g. 7:2,7:3")
    ap.add_argument("--case", choices=["estimator", "kmvm", "mbcg", "grad", "batched", "peaks",
                                       "c4", "synthetic", "decay"],
                    default="estimator",
                    help="kmvm / mbcg / grad: time only the kernel product, a short CG call "
                         "or the gradient contraction on an instance of the workload (for "
                         "profiling)")
    ap.add_argument("--n", type=int, default=None, help="instance size for --case")
    ap.add_argument("--reps", type=int, default=3, help="calls for --case")
    args = ap.parse_args()
    if args.case == "batched":
        run_batched(args)
        return
    if args.case == "peaks":
        run_peaks()
        return
    if args.case == "c4":
        run_c4(args)
        return
    if args.case == "decay":
        run_decay(args)
        return
    if args.case == "synthetic":
        run_synthetic(args)
        return
    if args.case != "estimator":
        run_case(args)
        return
    rank, ws, local, dist = _dist()
    if args.impl == "reference":
        run_reference(args, rank, ws, dist)
        return
    args.warmup = max(args.warmup, 3)

    import numpy as np
    import torch
    from paper_2107_00243_gb300 import build, gp, workloads
    build.build()
    gp.load()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    prec = {"bf16": gp.BF16, "tf32": gp.TF32, "fp32": gp.FP32}[args.precision]

    p = workloads.c3_rbf_ard_1e5(precision=prec)
    o = gp.opts(cg_tol=p.tol, max_iter=p.max_iter, recompute_every=p.recompute_every,
                seed=p.seed)
    t = p.n_probes + 1

    def setup(precision):
        prob = gp.Problem(p.X, p.theta, p.kind, p.ard, precision, device=dev)
        wsp = gp.Workspace()
        out = torch.empty(gp.out_len(prob.p, p.n_probes), dtype=torch.float64, device=dev)
        iout = torch.empty(2 + t + p.k, dtype=torch.int32, device=dev)
        y = torch.as_tensor(p.y).to(device=dev, dtype=prob.dtype)
        return prob, wsp, out, iout, y

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2

    def timed_steps(prob, wsp, out, iout, y, steps, measure_mvm=False):
        stream = torch.cuda.current_stream()
        total = 0.0
        gp.mvm_timing(measure_mvm)
        gp.mvm_timing_read()
        l0 = gp.launch_count()
        for _ in range(steps):
            flush.fill_(1)                                     # L2 flush between steps
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            gp.gp_mll_and_grad(prob, y, p.k, p.n_probes, o, workspace=wsp, out=out, iout=iout)
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1) / 1e3
        launches = gp.launch_count() - l0
        mvm_ms, mvm_n = gp.mvm_timing_read()
        con = gp.phase_timing_read(1)
        gp.mvm_timing(False)
        return total, launches, mvm_ms, mvm_n, con

    prob, wsp, out, iout, y = setup(prec)
    for _ in range(args.warmup):
        gp.gp_mll_and_grad(prob, y, p.k, p.n_probes, o, workspace=wsp, out=out, iout=iout)
    torch.cuda.synchronize()
    res = gp.unpack(out, iout, prob.p, p.n_probes, p.k)

    sampler = ClockSampler(local)
    _barrier(dist)
    torch.cuda.synchronize()
    sampler.start()
    total, launches, mvm_ms, mvm_n, (con_ms, con_n) = timed_steps(
        prob, wsp, out, iout, y, args.steps, measure_mvm=True)
    clocks = sampler.stop()
    torch.cuda.synchronize()
    _barrier(dist)
    total = _max_over_ranks(total, dist)
    value = total / (args.steps * ws)

    # the plain FP32 form of the same evaluation (speedup denominator of the mixed path)
    fp32_value = None
    fp32_mll = None
    if prec != gp.FP32 and args.fp32_steps > 0:
        prob32, wsp32, out32, iout32, y32 = setup(gp.FP32)
        # one warm-up evaluation: the plain FP32 form runs for tens of seconds
        gp.gp_mll_and_grad(prob32, y32, p.k, p.n_probes, o, workspace=wsp32, out=out32,
                           iout=iout32)
        tot32, _, _, _, _ = timed_steps(prob32, wsp32, out32, iout32, y32, args.fp32_steps)
        fp32_value = _max_over_ranks(tot32, dist) / (args.fp32_steps * ws)
        fp32_mll = gp.unpack(out32, iout32, prob32.p, p.n_probes, p.k)["mll"]
        del wsp32, out32, iout32

    # end to end: host (pinned) inputs -> device -> estimator -> host outputs
    Xh = torch.as_tensor(p.X).to(prob.dtype).pin_memory()
    yh = torch.as_tensor(p.y).to(prob.dtype).pin_memory()
    th = torch.as_tensor(p.theta).to(torch.float64).pin_memory()
    outh = torch.empty(out.numel(), dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    stream = torch.cuda.current_stream()
    e2e_total = 0.0
    for _ in range(e2e_steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        prob.X.copy_(Xh, non_blocking=True)
        y.copy_(yh, non_blocking=True)
        prob.theta.copy_(th, non_blocking=True)
        gp.gp_mll_and_grad(prob, y, p.k, p.n_probes, o, workspace=wsp, out=out, iout=iout)
        outh.copy_(out, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_total += e0.elapsed_time(e1) / 1e3
    e2e_total = _max_over_ranks(e2e_total, dist)
    e2e_value = e2e_total / (e2e_steps * ws)
    h2d = Xh.numel() * Xh.element_size() + yh.numel() * yh.element_size() + th.numel() * 8
    d2h = outh.numel() * 8

    if rank != 0:
        return

    # roofline of the dominant kernel: the kernel-matrix product (algorithmic FLOPs
    # 2 n^2 (d + t) per product; d = 16, t = 33)
    peaks, peak_src = _peaks()
    flops_per = 2.0 * p.n * p.n * (p.d + t)
    avg_mvm_s = (mvm_ms / 1e3) / max(mvm_n, 1)
    achieved = flops_per / avg_mvm_s / 1e12 if mvm_n else None
    if prec == gp.FP32:
        bound = "alu"
        peak = SM_COUNT * FP32_LANES * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        peak_note = ("FP32 FFMA: 152 SMs x 128 lanes x 2 FLOP x max SM clock "
                     f"({peaks.get('sm_max_mhz', 2070.0):.0f} MHz, {peak_src})")
    else:
        bound = "tensor"
        bf = peaks.get("bf16_tflops_sustained", 1700.0)
        peak = bf if prec == gp.BF16 else bf / 2.0
        peak_note = (f"bf16 dense sustained, {peak_src}" if prec == gp.BF16 else
                     f"tf32 = bf16 sustained ({peak_src}) x 1/2 (nominal ratio)")
    kernel_tag = {gp.FP32: "kmvm_simt_fp32", gp.BF16: "kmvm_tc_bf16",
                  gp.TF32: "kmvm_tc_tf32"}[prec]
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": _traffic_from_profiles(kernel_tag), "kernel": kernel_tag,
            "peak_source": peak_note, "algorithmic_flops_per_product": flops_per,
            "products_timed": mvm_n, "avg_product_ms": avg_mvm_s * 1e3}
    # the product's other roofline: one exponential per kernel entry (n^2 per product)
    # against the measured MUFU ex2 rate
    ex2_peak = _unit_peak("ex2_f32_per_s")
    if avg_mvm_s and ex2_peak:
        ex2_rate = float(p.n) ** 2 / avg_mvm_s
        roof["exp"] = {"achieved": ex2_rate, "peak": ex2_peak, "unit": "exp/s",
                       "frac": ex2_rate / ex2_peak,
                       "peak_source": "ex2.approx.f32, measured (profiles/unit_peaks_gb300.txt)"}

    # the gradient contraction (Alg. 2's O(n^2) pass): algorithmic FLOPs per kernel
    # entry 2 d (distance) + 2 t (m_ab) + 2 (2 d + 1) ([1, x, x^2] contraction); the
    # tensor-core form executes 2 kx + 2 tm + 4 nr per entry (hi / lo operands, padding)
    contraction = None
    if con_n:
        con_s = (con_ms / 1e3) / con_n
        cflops = float(p.n) ** 2 * (2 * p.d + 2 * t + 2 * (2 * p.d + 1))
        con_ach = cflops / con_s / 1e12
        kx = 64 if 3 * (p.d + 2) <= 64 else 128
        tm = (3 * t + 15) // 16 * 16
        nr = (4 + 4 * p.d + 15) // 16 * 16
        executed = 2 * kx + 2 * tm + 4 * nr
        bf = peaks.get("bf16_tflops_sustained", 1700.0)
        contraction = {
            "kernel": "grad_tc_kernel" if prec == gp.BF16 else "contract_kernel",
            "ms_per_eval": con_s * 1e3, "evals_timed": con_n,
            "bound": "tensor" if prec == gp.BF16 else "alu",
            "achieved": con_ach, "unit": "TFLOP/s",
            "peak": bf if prec == gp.BF16 else roof["peak"],
            "frac": con_ach / (bf if prec == gp.BF16 else roof["peak"]),
            "algorithmic_flops_per_entry": 2 * p.d + 2 * t + 2 * (2 * p.d + 1),
            "executed_tensor_flops_per_entry": executed if prec == gp.BF16 else None,
            "peak_source": peak_note if prec == gp.BF16 else roof["peak_source"]}

    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        t_sub, m_sub = oracle_subsample_seconds()
        m_full = int(max(res["iters"]))
        small = oracle_small_configs()
        info = _cpu_info()
        cpu = {"value": extrapolate(t_sub, m_sub, m_full, p.n, SUBSAMPLE_N, prob.p),
               "unit": "s", "cores": info["threads"], "kind": "oracle", "extrapolated": True,
               "sample": (f"FP64 oracle estimator (MLL + gradient) end to end on a "
                          f"{SUBSAMPLE_N}-point subsample of the same workload ({t_sub:.2f} s, "
                          f"{m_sub} CG iterations), scaled by (1e5/{SUBSAMPLE_N})^2 and by the "
                          f"product-equivalents per evaluation ({m_full} CG iterations in this "
                          "run, residual recomputes, 2 x (p-1) derivative passes). Also timed "
                          "('timed'): the oracle estimator and the exact MLL + gradient on the "
                          "small RBF workload and a 1,500-point Matern-5/2 subsample, and row "
                          "samples of one kernel product at n = 1e5 and n = 5e5 scaled to the "
                          "whole product"),
               "timed": {"subsample_estimator_s": t_sub, "subsample_n": SUBSAMPLE_N, **small},
               **info}

    dtype = {gp.FP32: "f32", gp.BF16: "bf16", gp.TF32: "tf32"}[prec]
    line = {
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": value * 1e3 * ws, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": args.precision, "n": p.n, "d": p.d,
                   "k": p.k, "n_probes": p.n_probes, "cg_tol": p.tol,
                   "recompute_every": p.recompute_every, "l2": "flushed between steps",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "fp32_form_s_per_eval": fp32_value,
        "speedup_vs_fp32_form": (fp32_value / value) if fp32_value else None,
        "fp32_form_mll": fp32_mll,
        "iters": res["iters"].tolist(), "mll": res["mll"], "status": res["status"],
        "roofline": roof, "contraction": contraction, "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "gpu_launches_per_step": launches / max(args.steps, 1),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
