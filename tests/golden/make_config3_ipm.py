"""Writes config3_sub20000_ipm.json: the optimum of the SVM dual on a fixed 20,000-point subsample
of workload 3, computed by the oracle alone (dense FP64 kernel matrix, Algorithm 1 with dense
LU Newton solves, Sec. 2).

Workload 3 is n = 1e5, d = 12 (8 Gaussian + 4 binary features), four consecutive 3-D windows,
sigma = 1, C = 10, tanh teacher with 5 % flips. A dense Newton matrix at n = 1e5 would take
80 GB, so the oracle solves the stated subsample: rows subsample_rows(1e5, 20000, SEED_BASE + 300)
of the full workload (features scaled on the full set, labels as drawn there). The reference is
run to a relative duality gap of 1e-9, well below the 1e-6 bar the device solver is held to.

Run from the repository root:  python -m tests.golden.make_config3_ipm
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import ipm as oi          # noqa: E402
from oracle import kernel as ok       # noqa: E402
from synth import SEED_BASE, config3, subsample_rows  # noqa: E402

N_FULL = 100_000
N_SUB = 20_000
SUB_SEED = SEED_BASE + 300
TOL = 1e-9
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config3_sub20000_ipm.json")


def subsample():
    """The stated subsample: (X, y, windows, sigma, C, idx)."""
    cfg = config3(n=N_FULL)
    idx = subsample_rows(N_FULL, N_SUB, SUB_SEED)
    return cfg["X"][idx], cfg["y"][idx], cfg["windows"], cfg["sigma"], cfg["C"], idx


def main():
    X, y, W, sigma, C, idx = subsample()
    t0 = time.time()
    K = ok.anova_kernel_matrix(X, W, sigma)
    print("kernel matrix %.1f s" % (time.time() - t0), flush=True)
    t1 = [time.time()]

    def record(alpha, lam):
        now = time.time()
        print("  iteration %.1f s  sum(alpha) %.10g" % (now - t1[0], alpha.sum()), flush=True)
        t1[0] = now

    ref = oi.ipm_dense(K, y, C, tol=TOL, max_iter=300, record=record)
    alpha, b = ref["alpha"], ref["b"]
    D = oi.dual_objective(K, y, alpha)
    P = oi.primal_objective(K, y, alpha, b, C)
    out = {
        "_source": "written by tests/golden/make_config3_ipm.py from oracle/ only: Algorithm 1 "
                   "(arXiv 2312.00538, Sec. 2) with dense FP64 Newton solves on a fixed subsample of "
                   "workload 3",
        "n_full": N_FULL, "n_sub": N_SUB, "subsample_seed": SUB_SEED,
        "idx_sum": int(idx.sum()), "y_sum": float(y.sum()),
        "C": C, "sigma": sigma, "tol": TOL,
        "iterations": ref["iterations"], "reason": ref["reason"],
        "dual": D, "primal": P, "rel_gap": (P - D) / max(1.0, abs(P)),
        "y_dot_alpha": float(y @ alpha), "b": b,
        "n_free": int(np.sum((alpha > 1e-6 * C) & (alpha < C * (1 - 1e-6)))),
        "n_at_C": int(np.sum(alpha >= C * (1 - 1e-6))),
        "seconds": time.time() - t0,
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
