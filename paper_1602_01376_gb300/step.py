"""Warm-up and measured factor + solve steps of one workload through the public API,
for profilers (ncu launch lists skip the first step's launches and capture the next).

    python -m paper_1602_01376_gb300.step C4 [--N 524288] [--steps 2] [--opts '{"knn_prune": 0}']

Prints one JSON line per step: the library's kernel launches in the step (plus one
torch copy of the right-hand sides), its CUDA-event time and the phase times of
iaskit_stats.  The chosen (mixed) form, refinement to 1e-10.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main() -> int:
    import numpy as np
    import torch

    import paper_1602_01376_gb300 as ia
    from workloads import make_points, make_rhs, workload

    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("--N", type=int, default=None)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--opts", default="{}", help="JSON object of iaskit options")
    ap.add_argument("--profile", action="store_true", help="per-class CUDA-event times")
    a = ap.parse_args()
    w = workload(a.workload, N=a.N)
    ia.load()
    ia.iaskit_set_stream(None)
    X = torch.from_numpy(make_points(w)).cuda()
    U0 = torch.from_numpy(np.ascontiguousarray(make_rhs(w).T)).cuda()
    U = torch.empty_like(U0)
    ia.iaskit_set_option("precision", 1)
    ia.iaskit_set_option("refine", 400)
    opts = json.loads(a.opts)
    for k, v in opts.items():
        ia.iaskit_set_option(k, v)
    for k in range(a.steps):
        if a.profile:
            ia.iaskit_set_option("profile", 1)
        l0 = ia.iaskit_stats()["launches"]
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        try:
            ia.iaskit_factor_device(X, w.h, w.lam, w.m, w.s_max, w.tol)
            U.copy_(U0)
            ia.iaskit_solve_device(U)
            err = None
        except ia.IaskitError as e:
            err = str(e)
        ev1.record()
        torch.cuda.synchronize()
        st = ia.iaskit_stats()
        out = {"step": k, "workload": a.workload, "N": w.N, "opts": opts, "launches": st["launches"] - l0,
               "step_ms": ev0.elapsed_time(ev1), "ms": st["ms"], "refine_history": st["refine_history"],
               "refine_iters": st["refine_iters"], "mean_rank_per_height": st["mean_rank_per_height"],
               "knn_pairs_scanned_frac": st["knn_pairs_scanned"] / max(st["knn_pairs_all"], 1.0),
               "error": err}
        if a.profile:
            out["kernels"] = {kk: round(v["ms"], 3) for kk, v in st["kernels"].items() if v["ms"] > 0}
            ia.iaskit_set_option("profile", 0)
        print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
