"""Writes residual_decay_exact.json: log det K_hat and tr(K_hat^-1 dK_hat/dtheta_p) (dense
Cholesky, FP64, the oracle only) of the four n = 1,000 problems of the residual-decay
experiment (Fig. 2: f(P_hat_k) -> f(K_hat) as the partial Cholesky rank k grows), drawn
by paper_2107_00243_gb300.workloads.synthetic_study: RBF and Matern-3/2 kernels, d = 1
and 3.  The experiment compares log det P_hat_k and tr(P_hat_k^-1 dP_hat_k) with them.

    python tests/golden/make_residual_decay_exact.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact, kernels  # noqa: E402
from paper_2107_00243_gb300 import workloads  # noqa: E402

N = 1000
PROBLEMS = [(kernels.RBF, 1), (kernels.RBF, 3), (kernels.MATERN32, 1), (kernels.MATERN32, 3)]


def main():
    out = {}
    for kind, d in PROBLEMS:
        p = workloads.synthetic_study(kind, d, n=N)
        r = exact.exact_mll_and_grad(p.kind, p.X, p.y, p.theta, p.ard)
        out[f"{kind}_{d}"] = {"logdet": r["logdet"], "trace_p": r["trace_p"].tolist(),
                              "trace_K": float(N * (p.theta[-2] + p.theta[-1]))}
        print(f"kind {kind} d {d}: logdet {r['logdet']:.6f}", flush=True)
    with open(os.path.join(HERE, "residual_decay_exact.json"), "w") as f:
        json.dump({"source": "oracle.exact.exact_mll_and_grad (dense Cholesky, FP64)",
                   "n": N, "problems": out}, f, indent=1)


if __name__ == "__main__":
    main()
