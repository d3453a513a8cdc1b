"""The paper's experiments rerun with this library on one GPU.

``errors``  -- the first experiment (Section 5, Fig. 5.1): the relative error of the complex field
               G(z_i, z_j) = -m_j / (z_i - z_j) as a function of the expansion order p, for
               theta in {1/4, 1/2, sqrt(1/2)}, a million unit-total-mass sources in the unit disc
               distributed (i) uniformly and (ii) with radial density ~ 1/r, the error measured on
               a random sample of M = 1000 points against direct summation.  The paper plots the
               curves without numbers; this command prints them.  Both paths are reported: the
               binary64 path shows the method's truncation error, the mixed path adds its
               binary32 rounding.
``timing``  -- the third experiment's shape (Section 5, Fig. 5.3): time against N for uniform,
               normal and "layer" distributions at p = 20, theta = 1/2, about 20 points per leaf.
``adaptivity`` -- the second experiment (Section 5, Fig. 5.2): the speedup of the adaptive mesh
               over the uniform-grid mesh (``fmm_build_tree_uniform``, on the unit square the
               points are drawn into and on their bounding square) on 200,000 points from the
               normal and "layer" distributions as sigma shrinks, p = 20, theta = 1/2, the same
               levels, lists and kernels on every mesh; each run is checked against the direct
               sum on 1000 sampled targets.

    python -m paper_1006_2269_gb300.experiments errors [--n 1000000] [--out FILE]
    python -m paper_1006_2269_gb300.experiments timing [--out FILE]
    python -m paper_1006_2269_gb300.experiments adaptivity [--n 200000] [--out FILE]

Every number is computed by the library's kernels (the tree, lists, expansions, and the binary64
direct kernels that measure the error); this module only drives them.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np
import torch

from . import fmm
from . import workloads as W

THETAS = (0.25, 0.5, math.sqrt(0.5))


def _t(a, dev, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), device=dev, dtype=dtype)


def field_errors(n: int, dev, ps=range(2, 31, 2), levels: int | None = None, samples: int = 1000, seed: int = 0):
    """{distribution: {theta: {"fp64": [err per p], "mixed": [...]}}} and the p values."""
    L = levels if levels is not None else max(1, int(round(math.log(n / 20.0) / math.log(4.0))))
    out = {}
    for name, make in (("uniform", W.disc_uniform), ("density 1/r", W.disc_inv_r)):
        c = make(n, W.SEED_BASE + 20 + seed)
        x, y, q = _t(c.x, dev), _t(c.y, dev), _t(c.q, dev)
        tg = _t(W.sample_targets(n, samples, W.SEED_BASE + 120 + seed), dev, torch.int64)
        rr = torch.empty(samples, dtype=torch.float64, device=dev)
        ri = torch.empty(samples, dtype=torch.float64, device=dev)
        fmm.fmm_direct_field(x, y, q, tg, rr, ri)
        ref = torch.complex(rr, ri)
        scale = float(ref.abs().max().item())
        per = {}
        for theta in THETAS:
            f = fmm.FMM(x, y, L, theta)
            try:
                res = {"fp64": [], "mixed": []}
                for p in ps:
                    for mode in ("fp64", "mixed"):
                        F = f.evaluate_field(q, p, mode)
                        res[mode].append(float((F[tg] - ref).abs().max().item()) / scale)
                per[f"{theta:.4f}"] = res
            finally:
                f.close()
        out[name] = per
    return {"n": n, "levels": L, "samples": samples, "p": list(ps), "errors": out}


def timing(dev, ns=(200_000, 1_000_000, 5_000_000), p: int = 20, theta: float = 0.5, reps: int = 5):
    """Milliseconds per complete step (tree, lists, potentials: fmm_step; mixed and binary64
    paths) for the distributions of the paper's robustness experiments."""
    kinds = {
        "uniform": lambda n, s: W.uniform(n, s),
        "normal sigma 0.1": lambda n, s: W.normal_sq(n, s, 0.1),
        "layer sigma 0.01": lambda n, s: W.layer(n, s, 0.01),
    }
    rows = []
    for name, make in kinds.items():
        for n in ns:
            c = make(n, W.SEED_BASE + 30)
            x, y, q = _t(c.x, dev), _t(c.y, dev), _t(c.q, dev)
            L = max(1, int(round(math.log(n / 20.0) / math.log(4.0))))
            f = fmm.FMM(x, y, L, theta)
            phi = torch.empty(n, dtype=torch.float64, device=dev)
            try:
                row = {"distribution": name, "n": n, "levels": L}
                for mode in (fmm.FMM_MODE_MIXED, fmm.FMM_MODE_FP64):
                    def step():  # tree, lists and evaluation (two streams, plain launches)
                        fmm.fmm_step(f.tree, f.lists, x, y, theta, q, p, mode, phi)
                    step()
                    torch.cuda.synchronize()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record()
                    for _ in range(reps):
                        step()
                    b.record()
                    torch.cuda.synchronize()
                    row["ms_mixed" if mode == fmm.FMM_MODE_MIXED else "ms_fp64"] = a.elapsed_time(b) / reps
                fmm.fmm_sync_status(f.tree, f.lists)
                rows.append(row)
            finally:
                f.close()
    return {"p": p, "theta": theta, "rows": rows}


SIGMAS = (1.0, 0.3, 0.1, 0.03, 0.01, 0.003, 0.001)


def _step_ms(f, x, y, q, theta, p, phi, reps):
    """Milliseconds per whole step (mesh, lists, binary32 evaluation), CUDA events."""
    def step():
        if f.mesh == "uniform":
            fmm.fmm_build_tree_uniform(f.tree, x, y, f.root)
        else:
            fmm.fmm_build_tree(f.tree, x, y)
        fmm.fmm_interaction_lists(f.tree, f.lists, theta)
        fmm.fmm_evaluate(f.tree, f.lists, q, p, fmm.FMM_MODE_MIXED, phi)

    step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        step()
    b.record()
    torch.cuda.synchronize()
    fmm.fmm_sync_status(f.tree, f.lists)
    return a.elapsed_time(b) / reps


def adaptivity(dev, n: int = 200_000, sigmas=SIGMAS, p: int = 20, theta: float = 0.5, reps: int = 5,
               samples: int = 1000):
    """Adaptive against uniform-grid mesh, same method otherwise (Section 5, second experiment)."""
    L = max(1, int(round(math.log(n / 20.0) / math.log(4.0))))
    rows = []
    for name, make in (("normal", W.normal_sq), ("layer", W.layer)):
        for k, sigma in enumerate(sigmas):
            c = make(n, W.SEED_BASE + 40 + k, sigma)
            x, y, q = _t(c.x, dev), _t(c.y, dev), _t(c.q, dev)
            tg = _t(W.sample_targets(n, samples, W.SEED_BASE + 140 + k), dev, torch.int64)
            ref = torch.empty(samples, dtype=torch.float64, device=dev)
            fmm.fmm_direct(x, y, q, tg, ref)
            scale = float(ref.abs().max().item())
            row = {"distribution": name, "sigma": sigma, "n": n, "levels": L}
            # the uniform mesh on the unit square every point was drawn into (the comparison of
            # the experiment) and on the points' bounding square
            for key, mesh, root in (("adaptive", "adaptive", None), ("unit", "uniform", (0.0, 0.0, 1.0)),
                                    ("bbox", "uniform", None)):
                f = fmm.FMM(x, y, L, theta, mesh=mesh, root=root)
                phi = torch.empty(n, dtype=torch.float64, device=dev)
                try:
                    row[f"ms_{key}"] = _step_ms(f, x, y, q, theta, p, phi, reps)
                    row[f"err_{key}"] = float((phi[tg] - ref).abs().max().item()) / scale
                    lb = f.export_tree()[2]
                    row[f"maxleaf_{key}"] = int((lb[1:] - lb[:-1]).max().item())
                finally:
                    f.close()
            row["speedup_unit"] = row["ms_unit"] / row["ms_adaptive"]
            row["speedup_bbox"] = row["ms_bbox"] / row["ms_adaptive"]
            rows.append(row)
    return {"p": p, "theta": theta, "rows": rows}


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_1006_2269_gb300.experiments")
    sub = ap.add_subparsers(dest="cmd", required=True)
    e = sub.add_parser("errors")
    e.add_argument("--n", type=int, default=1_000_000)
    e.add_argument("--out", default=None)
    t = sub.add_parser("timing")
    t.add_argument("--out", default=None)
    ad = sub.add_parser("adaptivity")
    ad.add_argument("--n", type=int, default=200_000)
    ad.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    from . import build
    build.build()
    fmm.load_library()
    dev = torch.device("cuda", 0)
    if a.cmd == "errors":
        res = field_errors(a.n, dev)
    elif a.cmd == "adaptivity":
        res = adaptivity(dev, a.n)
    else:
        res = timing(dev)
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(res, fh, indent=1)
    if a.cmd == "errors":
        print(f"N = {res['n']}, levels = {res['levels']}, M = {res['samples']} sampled targets")
        for dist, per in res["errors"].items():
            print(f"\n{dist}: relative error of the field (max over the sample / max |F|)")
            print("p      " + "  ".join(f"th={k} fp64   mixed" for k in per))
            for i, p in enumerate(res["p"]):
                print(f"{p:<6d} " + "  ".join(f"{v['fp64'][i]:.2e} {v['mixed'][i]:.2e}" for v in per.values()))
    elif a.cmd == "adaptivity":
        print(f"p = {res['p']}, theta = {res['theta']}: whole steps (mesh, lists, mixed evaluation)")
        print("uniform mesh on the unit square (unit) and on the bounding square (bbox)")
        print("distribution sigma    adaptive ms  unit ms  speedup  bbox ms  speedup  max leaf (adaptive / unit / bbox)"
              "  error (adaptive / unit / bbox)")
        for r in res["rows"]:
            print(f"{r['distribution']:<12} {r['sigma']:<8g} {r['ms_adaptive']:>10.3f} {r['ms_unit']:>8.3f} "
                  f"{r['speedup_unit']:>8.2f} {r['ms_bbox']:>8.3f} {r['speedup_bbox']:>8.2f}  "
                  f"{r['maxleaf_adaptive']:>5d} / {r['maxleaf_unit']:>6d} / {r['maxleaf_bbox']:<6d}"
                  f"            {r['err_adaptive']:.1e} / {r['err_unit']:.1e} / {r['err_bbox']:.1e}")
    else:
        for r in res["rows"]:
            print(r)


if __name__ == "__main__":
    main()
