"""A fixed workload run a few times, as a target for a profiler.

    python -m paper_1006_2269_gb300.profile_case [--workload clusters-1m] [--evals 3]
        [--p 20] [--mode mixed|fp64] [--lists plain|parents|exchange|parents+exchange]
        [--m2l auto|simt|tensor] [--steps]

Builds the tree and the lists of the workload once, then runs `--evals` evaluations (with
`--steps`, whole steps: tree, lists and evaluation), synchronises and prints one line.  The
launch order is the library's own, so a profiler's `-s/-c` counts select the same kernels on
every run.

Workloads: ``clusters-1m`` -- 2^20 points in Gaussian clusters (the mixed clustered workload),
8 levels, theta = 1/2; ``uniform-1m`` -- 2^20 uniform points in the unit square, 8 levels.
"""
from __future__ import annotations

import argparse

import numpy as np
import torch

from . import build, fmm
from . import workloads as W


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_1006_2269_gb300.profile_case")
    ap.add_argument("--workload", default="clusters-1m", choices=["clusters-1m", "uniform-1m"])
    ap.add_argument("--evals", type=int, default=3)
    ap.add_argument("--p", type=int, default=20)
    ap.add_argument("--mode", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--lists", default="plain", choices=["plain", "parents", "exchange", "parents+exchange"])
    ap.add_argument("--m2l", default="auto", choices=["auto", "simt", "tensor"])
    ap.add_argument("--steps", action="store_true", help="time whole steps, not evaluations only")
    a = ap.parse_args(argv)
    build.build()
    fmm.load_library()
    dev = torch.device("cuda", 0)
    if a.workload == "clusters-1m":
        c, L, theta = W.mixed_1m_cloud(), W.MIXED_1M.levels, W.MIXED_1M.theta
    else:
        c, L, theta = W.uniform(1 << 20, W.SEED_BASE + 7), 8, 0.5
    x, y, q = (torch.as_tensor(np.ascontiguousarray(v), device=dev) for v in (c.x, c.y, c.q))
    f = fmm.FMM(x, y, L, theta, parents="parents" in a.lists, exchange="exchange" in a.lists)
    try:
        fmm.fmm_set_m2l_kernel(f.tree, {"auto": fmm.FMM_M2L_AUTO, "simt": fmm.FMM_M2L_SIMT,
                                        "tensor": fmm.FMM_M2L_TENSOR}[a.m2l])
        mode = fmm.FMM_MODE_MIXED if a.mode == "mixed" else fmm.FMM_MODE_FP64
        phi = torch.empty(c.x.shape[0], dtype=torch.float64, device=dev)
        for _ in range(a.evals):
            if a.steps:
                fmm.fmm_build_tree(f.tree, x, y)
                fmm.fmm_interaction_lists(f.tree, f.lists, theta)
            fmm.fmm_evaluate(f.tree, f.lists, q, a.p, mode, phi)
        torch.cuda.synchronize()
        fmm.fmm_sync_status(f.tree, f.lists)
        nweak, nstrong = fmm.fmm_lists_sync(f.lists)
        print(f"{a.workload}: {a.evals} {'steps' if a.steps else 'evaluations'}, p = {a.p}, {a.mode}, "
              f"lists {a.lists} ({nweak} weak, {nstrong} strong entries), phi[0] = {float(phi[0]):.6e}")
    finally:
        f.close()


if __name__ == "__main__":
    main()
