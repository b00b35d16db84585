"""Writes synthetic_study_exact.json: the exact log-marginal likelihood and gradient
(dense Cholesky, FP64, the oracle only) of the nine problems of the bias / variance
study (paper_2107_00243_gb300.workloads.synthetic_study: RBF, Matern-3/2 and rational
quadratic kernels, d = 1, 2, 3, n = 10,000).  The study compares the estimator's mean
and spread over probe seeds against these values.

    python tests/golden/make_synthetic_study_exact.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact, kernels  # noqa: E402
from paper_2107_00243_gb300 import workloads  # noqa: E402


def main():
    out = {}
    for kind in (kernels.RBF, kernels.MATERN32, kernels.RATQUAD):
        for d in (1, 2, 3):
            p = workloads.synthetic_study(kind, d)
            t0 = time.time()
            r = exact.exact_mll_and_grad(p.kind, p.X, p.y, p.theta, p.ard)
            out[f"{kind}_{d}"] = {"mll": r["mll"], "grad": r["grad"].tolist(),
                                  "quad_p": r["quad_p"].tolist(),
                                  "trace_p": r["trace_p"].tolist(),
                                  "quad": r["quad"], "logdet": r["logdet"]}
            print(f"kind {kind} d {d}: mll {r['mll']:.6f} ({time.time() - t0:.0f} s)", flush=True)
    with open(os.path.join(HERE, "synthetic_study_exact.json"), "w") as f:
        json.dump({"source": "oracle.exact.exact_mll_and_grad (dense Cholesky, FP64)",
                   "problems": out}, f, indent=1)


if __name__ == "__main__":
    main()
