"""Learned (levels, p) selector: pick the parameters that meet a tolerance fastest.

The paper chooses the parameters by rule: p ~ log TOL / log theta from the error estimate of
Section 3, and about 20 points per leaf (end of Section 4).  This module keeps that rule as the
fallback (:func:`fallback_params`) and adds a network that learns the choice from runs of the
method itself:

1. :func:`run_table` runs the method on one point set for a grid of (levels, p), timing each run
   (tree, lists, evaluation; CUDA events) and measuring its error against the direct sum on
   sampled targets (the library's binary64 direct kernel).
2. :func:`label` turns a table and a tolerance into a class: the fastest run whose error meets
   the tolerance.
3. :class:`Selector` computes the 64 features of a point set (a probe tree, the library's
   feature kernel), trains the 64-128-128-225 network with the library's forward, backward and
   Adam kernels, and selects with the library's masked arg-max.

All arithmetic runs in the CUDA library; this module only orchestrates (which runs to make,
mini-batch order, bookkeeping).  Mode: the mixed mode throughout; the library runs tolerances
below 1e-7 in its split precision (binary64 expansions, float-float near field).

Command line (trains on synthetic point sets and writes the weights next to this file):

    python -m paper_1006_2269_gb300.selector train [--instances 300] [--out PATH]
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np
import torch

from . import fmm
from . import workloads as W

LMIN, LMAX, PMIN, PMAX, NP = (fmm.FMM_SEL_LMIN, fmm.FMM_SEL_LMAX, fmm.FMM_SEL_PMIN, fmm.FMM_SEL_PMAX,
                              fmm.FMM_SEL_NP)
NCLASS = fmm.FMM_MLP_OUT
THETA = 0.5
MIXED_FLOOR = 1e-7  # tolerances below it take the split precision (binary64 expansions)
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_weights")


def class_of(levels: int, p: int) -> int:
    return (levels - LMIN) * NP + (p - PMIN)


def params_of(c: int):
    return LMIN + c // NP, PMIN + c % NP


def max_levels(n: int) -> int:
    L = 0
    while 4 ** (L + 1) <= n:
        L += 1
    return L


def fallback_params(n: int, tol: float, theta: float = THETA, leaf: float = 20.0):
    """The plain rule: the smallest p with theta^(p+1) / (1 - theta)^2 <= tol (Section 3's
    estimate with unit constant) and about `leaf` points per leaf (end of Section 4)."""
    p = math.ceil(math.log(tol * (1.0 - theta) ** 2) / math.log(theta)) - 1
    p = min(PMAX, max(PMIN, p))
    L = int(round(math.log(n / leaf) / math.log(4.0)))
    L = min(LMAX, max(LMIN, L), max_levels(n))
    return L, p


PROBE_LMAX = 7  # deepest probe tree (N >= 4^8 * 16 = 1,048,576 points would go one level deeper)


def probe_levels(n: int) -> int:
    """Levels of the tree the features are read from: about 16 points per leaf, at most
    PROBE_LMAX.  The training sets (N <= 1e6) never reach an eighth level, so a larger set's
    features stay in the range the network was trained on (an eighth level's occupancy block,
    zero in every training sample, turned the choice for 2^20 points into nonsense)."""
    return max(1, min(PROBE_LMAX, int(math.floor(math.log(max(n / 16.0, 1.0)) / math.log(4.0)))))


def _t(a, dev, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), device=dev, dtype=dtype)


# ---- method runs ----------------------------------------------------------------------------

class Instance:
    """One point set on the device, with its direct-sum reference at sampled targets."""

    def __init__(self, cloud, dev, n_check: int = 256, seed: int = 0):
        self.cloud = cloud
        self.n = cloud.x.shape[0]
        self.x, self.y, self.q = (_t(a, dev) for a in (cloud.x, cloud.y, cloud.q))
        self.tg = _t(W.sample_targets(self.n, min(n_check, self.n), seed), dev, torch.int64)
        self.ref = torch.empty(self.tg.numel(), dtype=torch.float64, device=dev)
        fmm.fmm_direct(self.x, self.y, self.q, self.tg, self.ref)
        self.scale = float(self.ref.abs().max().item())
        self.dev = dev

    def error(self, phi) -> float:
        return float((phi[self.tg] - self.ref).abs().max().item()) / self.scale


def _events():
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_table(inst: Instance, levels, ps, tol: float, reps: int = 2):
    """[(levels, p, ms, err)] for every combination; ms = tree + lists + evaluation (best of
    `reps` after one warm-up), err = max-norm relative error at the sampled targets."""
    out = []
    stream = torch.cuda.current_stream()
    phi = torch.empty(inst.n, dtype=torch.float64, device=inst.dev)
    for L in levels:
        f = fmm.FMM(inst.x, inst.y, L, THETA)
        try:
            a, b = _events()
            t_struct = float("inf")
            for _ in range(reps + 1):
                a.record(stream)
                fmm.fmm_build_tree(f.tree, inst.x, inst.y)
                fmm.fmm_interaction_lists(f.tree, f.lists, THETA)
                b.record(stream)
                torch.cuda.synchronize()
                t_struct = min(t_struct, a.elapsed_time(b))
            for p in ps:
                t_eval = float("inf")
                for r in range(reps + 1):
                    a.record(stream)
                    fmm.fmm_evaluate(f.tree, f.lists, inst.q, p, fmm.FMM_MODE_MIXED, phi, tol)
                    b.record(stream)
                    torch.cuda.synchronize()
                    if r:
                        t_eval = min(t_eval, a.elapsed_time(b))
                fmm.fmm_sync_status(f.tree, f.lists)
                out.append((L, p, t_struct + t_eval, inst.error(phi)))
        finally:
            f.close()
    return out


LABEL_MARGIN = 0.5  # a label must meet margin * tol: neighbouring point sets then still meet tol


def label(table, tol: float, margin: float = 1.0) -> int:
    """Class of the fastest run whose error is at most margin * tol (the most accurate run if
    none is)."""
    ok = [r for r in table if r[3] <= margin * tol]
    best = min(ok, key=lambda r: r[2]) if ok else min(table, key=lambda r: r[3])
    return class_of(best[0], best[1])


def centre_level(n: int) -> int:
    """round(log4(N / 32)), halves rounded up, from the bit length of N: floor((b - 4) / 2) with
    b = floor(log2 N) (the rule fmm_select_params applies on the device)."""
    return (int(n).bit_length() - 1 - 4) // 2


def candidate_levels(n: int):
    """Level counts tried for a label, and the only ones the selector may choose:
    centre_level(N) - 2 .. + 1."""
    Lc = centre_level(n)
    return [L for L in range(Lc - 2, Lc + 2) if LMIN <= L <= min(LMAX, max_levels(n))]


def candidate_ps(tol: float):
    if tol < MIXED_FLOOR:
        return [20, 24, 26, 28, 30, 32]
    return list(range(PMIN, PMAX + 1, 2))


def time_params(inst: Instance, L: int, p: int, tol: float, reps: int = 2):
    return run_table(inst, [L], [p], tol, reps)[0]


# ---- the network ----------------------------------------------------------------------------

def init_params(seed: int) -> np.ndarray:
    """He-normal weights, zero biases (the random numbers are drawn on the host)."""
    g = np.random.default_rng(seed)
    parts = []
    for nout, nin in ((fmm.FMM_MLP_HIDDEN, fmm.FMM_MLP_IN), (fmm.FMM_MLP_HIDDEN, fmm.FMM_MLP_HIDDEN),
                      (NCLASS, fmm.FMM_MLP_HIDDEN)):
        parts.append(g.normal(0.0, math.sqrt(2.0 / nin), nout * nin))
        parts.append(np.zeros(nout))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == fmm.FMM_MLP_PARAMS
    return p


class Selector:
    """The network on the GPU (library kernels) plus the feature computation."""

    def __init__(self, params=None, device=None, batch_max: int = 4096):
        self.dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.batch_max = batch_max
        self.m = fmm.fmm_mlp_create(batch_max)
        self.meta = {}
        self.set_params(init_params(0) if params is None else params)

    def set_params(self, params):
        self.params = _t(np.asarray(params, np.float32), self.dev, torch.float32)
        fmm.fmm_mlp_set_params(self.m, self.params)

    def get_params(self) -> np.ndarray:
        out = torch.empty(fmm.FMM_MLP_PARAMS, dtype=torch.float32, device=self.dev)
        fmm.fmm_mlp_get_params(self.m, out)
        return out.cpu().numpy()

    @staticmethod
    def features(x, y, tol: float, levels: int | None = None) -> torch.Tensor:
        """The 64 inputs of one point set (x, y: CUDA float64) from a probe tree."""
        n = x.numel()
        L = probe_levels(n) if levels is None else levels
        t = fmm.fmm_tree_create(n, L)
        try:
            fmm.fmm_build_tree(t, x, y)
            out = torch.empty(64, dtype=torch.float32, device=x.device)
            fmm.fmm_selector_features(t, tol, out)
            torch.cuda.synchronize(x.device)
        finally:
            fmm.fmm_tree_destroy(t)
        return out

    def select_features(self, feats: torch.Tensor):
        """(levels, p) for each row of feats (CUDA float32 [B][64])."""
        B = feats.shape[0]
        out = torch.empty((B, 2), dtype=torch.int32, device=feats.device)
        fmm.fmm_select_params(self.m, feats.contiguous(), out)
        return [tuple(r) for r in out.cpu().tolist()]

    def select(self, x, y, tol: float):
        return self.select_features(self.features(x, y, tol)[None, :])[0]

    def train(self, X: np.ndarray, y: np.ndarray, epochs: int = 400, batch: int = 64, lr: float = 1e-3,
              seed: int = 0, X_val=None, y_val=None):
        """Mini-batch Adam on the GPU; returns the per-epoch mean training loss."""
        Xd = _t(X.astype(np.float32), self.dev, torch.float32)
        yd = _t(y.astype(np.int32), self.dev, torch.int32)
        g = np.random.default_rng(seed)
        loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
        hist = []
        for _ in range(epochs):
            order = torch.as_tensor(g.permutation(X.shape[0]), device=self.dev)
            tot = torch.zeros(1, dtype=torch.float32, device=self.dev)
            nb = 0
            for s in range(0, X.shape[0], batch):
                idx = order[s:s + batch]
                xb = Xd[idx].contiguous()
                lb = yd[idx].contiguous()
                fmm.fmm_mlp_train_step(self.m, xb, lb, lr, loss)
                tot += loss
                nb += 1
            hist.append(float(tot.item()) / nb)
        return hist

    def accuracy(self, X: np.ndarray, y: np.ndarray) -> float:
        feats = _t(X.astype(np.float32), self.dev, torch.float32)
        got = self.select_features(feats)
        return float(np.mean([class_of(L, p) == int(c) for (L, p), c in zip(got, y)]))

    def save(self, path: str = WEIGHTS, meta: dict | None = None):
        self.get_params().astype("<f4").tofile(path + ".f32")
        with open(path + ".json", "w") as fh:
            json.dump(meta or self.meta, fh, indent=1, sort_keys=True)

    @classmethod
    def load(cls, path: str = WEIGHTS, device=None):
        p = np.fromfile(path + ".f32", dtype="<f4")
        if p.size != fmm.FMM_MLP_PARAMS:
            raise ValueError(f"{path}.f32 holds {p.size} values, expected {fmm.FMM_MLP_PARAMS}")
        s = cls(p, device)
        if os.path.exists(path + ".json"):
            with open(path + ".json") as fh:
                s.meta = json.load(fh)
        return s

    def close(self):
        if self.m:
            fmm.fmm_mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- data -----------------------------------------------------------------------------------

KINDS = ("uniform", "normal", "circle", "clusters", "rings")
TOLS = (1e-3, 1e-6, 1e-9)


def make_cloud(i: int, seed: int, nmin: float, nmax: float):
    """Point set i of a family: N log-uniform in [nmin, nmax], the distributions of the
    benchmark workloads in turn."""
    g = np.random.default_rng(seed * 7919 + i)
    n = int(round(math.exp(g.uniform(math.log(nmin), math.log(nmax)))))
    kind = KINDS[i % len(KINDS)]
    s = seed * 100003 + i
    if kind == "uniform":
        return W.uniform(n, s)
    if kind == "normal":
        return W.normal(n, s)
    if kind == "circle":
        return W.circle(n, s)
    if kind == "clusters":
        return W.clusters(n, s)
    return W.rings_plummer(n, s)


def generate(count: int, seed: int, dev, nmin: float = 1e4, nmax: float = 1e6, tols=TOLS, log=None,
             time_budget: float | None = None, save=None):
    """Features X[count * len(tols)][64], labels y and the run tables, from `count` point sets (or
    as many as `time_budget` seconds allow); save(X, y) is called after every tenth set."""
    X, y, tables = [], [], []
    t0 = time.time()
    for i in range(count):
        if time_budget is not None and time.time() - t0 > time_budget:
            if log:
                log(f"time budget reached after {i} point sets")
            break
        c = make_cloud(i, seed, nmin, nmax)
        inst = Instance(c, dev, seed=seed * 31 + i)
        tab = {}
        for tol in tols:
            key = "split" if tol < MIXED_FLOOR else "mixed"
            if key not in tab:
                tab[key] = run_table(inst, candidate_levels(inst.n), candidate_ps(tol), tol, reps=2)
            f = Selector.features(inst.x, inst.y, tol).cpu().numpy()
            X.append(f)
            y.append(label(tab[key], tol, LABEL_MARGIN))
        tables.append({"n": inst.n, "kind": c.name, "tables": tab})
        if log:
            log(f"instance {i}: n={inst.n} {c.name} labels={[params_of(v) for v in y[-len(tols):]]}")
        if save is not None and (i + 1) % 10 == 0:
            save(np.array(X, np.float32), np.array(y, np.int32))
    return np.array(X, np.float32), np.array(y, np.int32), tables


def gain(selector: Selector, count: int, seed: int, dev, nmin: float = 1e4, nmax: float = 1e6, tols=TOLS):
    """Selector against the fallback rule on fresh point sets: per case the chosen parameters,
    their run time and error; totals over all cases."""
    cases = []
    for i in range(count):
        c = make_cloud(i, seed, nmin, nmax)
        inst = Instance(c, dev, seed=seed * 31 + i)
        for tol in tols:
            Ls, ps = selector.select(inst.x, inst.y, tol)
            Lf, pf = fallback_params(inst.n, tol)
            rs = time_params(inst, Ls, ps, tol)
            rf = time_params(inst, Lf, pf, tol)
            cases.append({"n": inst.n, "kind": c.name, "tol": tol, "selector": [Ls, ps, rs[2], rs[3]],
                          "fallback": [Lf, pf, rf[2], rf[3]]})
    ok_s = [c["selector"][3] <= c["tol"] for c in cases]
    ok_f = [c["fallback"][3] <= c["tol"] for c in cases]
    both = [k for k, c in enumerate(cases) if ok_s[k] and ok_f[k]]
    return {
        "cases": cases,
        "met_tol_selector": float(np.mean(ok_s)),
        "met_tol_fallback": float(np.mean(ok_f)),
        "ms_selector": float(sum(c["selector"][2] for c in cases)),
        "ms_fallback": float(sum(c["fallback"][2] for c in cases)),
        "speedup_where_both_met": (float(sum(cases[k]["fallback"][2] for k in both) /
                                         max(sum(cases[k]["selector"][2] for k in both), 1e-9)) if both else None),
    }


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(prog="python -m paper_1006_2269_gb300.selector")
    sub = ap.add_subparsers(dest="cmd", required=True)
    tr = sub.add_parser("train", help="generate runs, train, report the gain, write the weights")
    tr.add_argument("--instances", type=int, default=300)
    tr.add_argument("--test-instances", type=int, default=30)
    tr.add_argument("--nmax", type=float, default=1e6)
    tr.add_argument("--epochs", type=int, default=400)
    tr.add_argument("--seed", type=int, default=1)
    tr.add_argument("--out", default=WEIGHTS)
    tr.add_argument("--report", default=None)
    tr.add_argument("--time-budget", type=float, default=None,
                    help="seconds of data generation at most (the point sets made by then are used)")
    tr.add_argument("--data", default=None, help="npz file the features and labels are saved to as they grow")
    a = ap.parse_args(argv)
    from . import build
    build.build()
    fmm.load_library()
    dev = torch.device("cuda", 0)
    t0 = time.time()
    save = (lambda X_, y_: np.savez(a.data, X=X_, y=y_)) if a.data else None
    X, y, tables = generate(a.instances, a.seed, dev, nmax=a.nmax, log=lambda m: print(m, flush=True),
                            time_budget=a.time_budget, save=save)
    if save is not None:
        save(X, y)
    t_gen = time.time() - t0
    nval = max(1, len(y) // 10)
    perm = np.random.default_rng(a.seed).permutation(len(y))
    va, trn = perm[:nval], perm[nval:]
    sel = Selector(init_params(a.seed), dev)
    hist = sel.train(X[trn], y[trn], epochs=a.epochs, seed=a.seed)
    acc_tr, acc_va = sel.accuracy(X[trn], y[trn]), sel.accuracy(X[va], y[va])
    g = gain(sel, a.test_instances, a.seed + 1000, dev, nmax=a.nmax)
    meta = {
        "instances": int(len(y)) // len(TOLS), "samples": int(len(y)), "tolerances": list(TOLS), "theta": THETA,
        "label_margin": LABEL_MARGIN,
        "n_range": [1e4, a.nmax], "kinds": list(KINDS), "epochs": a.epochs, "seed": a.seed,
        "loss_first_last": [hist[0], hist[-1]], "accuracy_train": acc_tr, "accuracy_val": acc_va,
        "generation_s": t_gen,
        "gain": {k: v for k, v in g.items() if k != "cases"},
    }
    sel.save(a.out, meta)
    print(json.dumps(meta, indent=1))
    if a.report:
        with open(a.report, "w") as fh:
            json.dump({"meta": meta, "gain_cases": g["cases"], "tables": tables}, fh)
    sel.close()


if __name__ == "__main__":
    main()
