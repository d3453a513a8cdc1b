"""Benchmark: 2D FMM potentials/sec at relative error <= 1e-6, mixed precision vs the FP64 GPU path.

Workload (default): N = 2^20 points, half uniform in [0,1]^2 and half from 8 Gaussian clusters
(sigma 0.01), strengths N(0,1), 8 levels (16 points per leaf), theta = 1/2, p = 20.

One step = one pass of the whole method on one input resident in HBM: build the tree, build the
interaction lists, evaluate (P2M, M2M, M2L, L2L, L2P + near field), potentials in input order.
The L2 cache (129 MB) is flushed between steps by writing a 256 MB buffer outside the timed
events.  Per-stage device times come from CUDA events recorded by the library on its stream.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica (the method has no exchange step on one
instance here); value = points of all ranks / max over ranks of the timed region.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2D FMM potentials/sec at rel err <=1e-6, mixed-prec vs FP64 GPU path"
UNIT = "potentials/s"
SM_COUNT = 152
SM_MAX_MHZ = 2070.0


def measured_bf16_tflops():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except Exception:
        return 1900.0


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---- clocks sampled during the timed region ------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0:  # sampling has started
                time.sleep(0.01)
            self.lines.clear()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- the FP64 CPU oracle as it stands, on one core and on every host core ----------------------

def cpu_model() -> str:
    """The host CPU's model name (lscpu / /proc/cpuinfo), or the platform's processor string."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


_ORC_SAMPLE = None


def _orc_worker_init(ns, Ls, p, theta):
    os.environ["OMP_NUM_THREADS"] = "1"
    global _ORC_SAMPLE
    import oracle
    from paper_1006_2269_gb300 import workloads as W
    oracle.build()
    _ORC_SAMPLE = (oracle, W.mixed_1m_cloud(ns), Ls, p, theta)


def _orc_worker_run(_):
    orc, c, Ls, p, theta = _ORC_SAMPLE
    t0 = time.perf_counter()
    orc.fmm(c.x, c.y, c.q, Ls, p, theta)
    return time.perf_counter() - t0


class OraclePool:
    """One process per host core (spawned, so it is safe beside a CUDA context), each holding the
    same bounded sample of the workload; a round runs the unmodified oracle FMM once on every core
    at the same time."""

    def __init__(self, cores, ns, Ls, p, theta):
        import multiprocessing as mp
        self.cores = cores
        self.pool = mp.get_context("spawn").Pool(cores, initializer=_orc_worker_init, initargs=(ns, Ls, p, theta))

    def round(self, limit_s: float = 600.0) -> float:
        # a worker that dies is replaced by the pool and its task never returns: the time limit
        # turns that into an error instead of a wait without end
        t0 = time.perf_counter()
        self.pool.map_async(_orc_worker_run, range(self.cores), chunksize=1).get(timeout=limit_s)
        return time.perf_counter() - t0

    def close(self):
        self.pool.terminate()
        self.pool.join()


# ---- the reference arm: the FP64 CPU oracle as it stands ----------------------------------------

def run_reference(args, rank):
    """The oracle as it stands on the host cores: every step runs the oracle FMM once on each
    core at the same time, each on the same bounded sample of the benchmark workload."""
    if rank != 0:
        return None
    import oracle
    from paper_1006_2269_gb300 import workloads as W
    oracle.build()
    w = W.MIXED_1M
    ns, Ls = 1 << 16, 6  # bounded sample of the workload: same distribution, 16 points per leaf
    cores = host_cores()
    pool = OraclePool(cores, ns, Ls, w.p, w.theta)
    try:
        for _ in range(args.warmup):
            pool.round()
        t = [pool.round() for _ in range(args.steps)]
    finally:
        pool.close()
    dt = sum(t) / args.steps
    v = cores * ns / dt
    sample = (f"oracle FMM on N={ns} points of the same distribution, L={Ls}, p={w.p}, one run per core "
              f"on all {cores} host cores at once ({cpu_model()})")
    return {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"clusters N={ns}, L={Ls}, theta=1/2, p={w.p} (bounded sample of {w.name})",
                   "sample_of": w.name, "points_per_step": cores * ns},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "nproc": cores, "cpu_model": cpu_model()},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ---- replicas: one per GPU, the slowest rank's time, whole-job throughput ---------------------------

def max_over_ranks(ms: float, world: int, device="cpu") -> float:
    """The slowest rank's time: every rank takes part (world 1: the value itself)."""
    if world == 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_replica: int, ms_total: float, steps: int) -> float:
    """Units of all replicas per second, each step of every replica within the slowest's time."""
    return world * units_per_replica / (ms_total / steps * 1e-3)


def shard_instances(sizes, world: int, rank: int):
    """Indices of the independent instances rank `rank` of `world` runs: largest first to the
    least loaded rank (ties to the lower rank), each rank's indices ascending.  One rank takes
    every instance in order."""
    if world == 1:
        return list(range(len(sizes)))
    load = [0] * world
    mine = []
    for i in sorted(range(len(sizes)), key=lambda j: (-sizes[j], j)):
        r = min(range(world), key=lambda k: (load[k], k))
        load[r] += sizes[i]
        if r == rank:
            mine.append(i)
    return sorted(mine)


# ---- our arm -----------------------------------------------------------------------------------

# dram__bytes_read.sum + dram__bytes_write.sum of the SIMT M2L kernel per launch on the 1M
# clustered workload, from one ncu capture each; valid while that kernel is unchanged
M2L_TRAFFIC = {(21, 1 << 20, "parents"): 85135872 + 3795712}


def pair_counts(f):
    """Algorithmic units of the current tree/lists: weak pairs per level and near-field pair
    evaluations (sum over leaves of n_t * sum of strong n_s)."""
    from paper_1006_2269_gb300 import fmm
    _, L, nbox = fmm.fmm_tree_info(f.tree)
    woff, widx, soff, sidx = (a.cpu().numpy().astype(np.int64) for a in f.export_lists())
    _, _, lb = f.export_tree()
    lb = lb.cpu().numpy().astype(np.int64)
    nweak = int(woff[-1])
    base = (4 ** L - 1) // 3
    sizes = np.diff(lb)
    so = soff[base:base + 4 ** L + 1] - soff[base]
    s_idx = sidx[soff[base]:soff[base + 4 ** L]]
    src = np.add.reduceat(sizes[s_idx], so[:-1]) if s_idx.size else np.zeros(4 ** L)
    pairs = int(np.sum(sizes * src))
    return nweak, pairs


def bench_batched(dev, steps, warmup, sequential=True, world=1, rank=0):
    """The batched workload: 512 independent instances, N log-uniform in [1e3, 2e5] (uniform
    square / 2D normal / jittered unit circle), theta = 1/2, p = 16, leaves of ~32 points.  One
    step = tree, lists and evaluation of every instance, all instances in the same launches,
    replayed as one CUDA graph with the launch shapes chosen by the library's autotuner.  Under
    several ranks the instances are shared out (shard_instances; no exchange between ranks) and
    the value counts the points of all ranks over the slowest rank's time.  For comparison the
    same instances are also run one after another through single-instance handles (one step,
    plain launches)."""
    import torch
    from paper_1006_2269_gb300 import fmm, workloads as W
    inst_all = W.batched_instances()
    n_all = int(sum(c.x.shape[0] for c, _ in inst_all))
    inst = [inst_all[i] for i in shard_instances([c.x.shape[0] for c, _ in inst_all], world, rank)]
    sizes = [c.x.shape[0] for c, _ in inst]
    levels = [L for _, L in inst]
    x = torch.as_tensor(np.concatenate([c.x for c, _ in inst]), device=dev)
    y = torch.as_tensor(np.concatenate([c.y for c, _ in inst]), device=dev)
    q = torch.as_tensor(np.concatenate([c.q for c, _ in inst]), device=dev)
    n = int(sum(sizes))
    theta, p = 0.5, 16
    b = fmm.FMMBatch(x, y, sizes, levels, theta)
    phi = torch.empty(n, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    m2l_blocks, p2p_blocks = b.autotune(q, p)

    def step():
        fmm.fmm_step(b.tree, b.lists, x, y, theta, q, p, fmm.FMM_MODE_MIXED, phi)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    fmm.fmm_sync_status(b.tree, b.lists)
    l0 = fmm.fmm_launch_count()
    step()
    launches = fmm.fmm_launch_count() - l0
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, e in ev:
        flush.zero_()
        a.record(stream)
        g.replay()
        e.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(sum(a.elapsed_time(e) for a, e in ev) / steps, world, dev)
    fmm.fmm_sync_status(b.tree, b.lists)
    # accuracy: 16 sampled targets of every instance against the binary64 direct sum
    worst = 0.0
    for i, d in enumerate(b.inst):
        a0, m = d["p0"], d["n"]
        tg = torch.as_tensor(W.sample_targets(m, 16, W.SEED_BASE + 500 + i), device=dev)
        ref = torch.empty(tg.numel(), dtype=torch.float64, device=dev)
        fmm.fmm_direct(x[a0:a0 + m], y[a0:a0 + m], q[a0:a0 + m], tg, ref)
        err = ((phi[a0:a0 + m][tg] - ref).abs().max() / ref.abs().max()).item()
        worst = max(worst, err)
    worst = max_over_ranks(worst, world, dev)
    out = {"workload": "512 instances, N log-uniform in [1e3, 2e5], uniform/normal/circle, "
                       "theta=1/2, p=16, ~32 points per leaf",
           "instances": len(inst_all), "points": n_all, "value": n_all / (ms * 1e-3), "unit": UNIT,
           "ms_per_step": ms, "gpu_launches_per_step": launches, "cuda_graph": True,
           "autotuned_blocks_per_instance": {"m2l": m2l_blocks, "near_field": p2p_blocks},
           "rel_err_max_sampled": worst, "n_check_per_instance": 16}
    if world > 1:  # a fixed set of instances shared out: strong scaling for this sub-result
        out["ranks"] = world
        out["scaling"] = "strong"
        out["instances_per_rank"] = "largest first to the least loaded rank"
    b.close()
    if sequential:
        # the same instances one by one through single-instance handles
        fs = []
        try:
            for i, (c, L) in enumerate(inst):
                a0 = int(sum(sizes[:i]))
                fs.append((fmm.FMM(x[a0:a0 + sizes[i]], y[a0:a0 + sizes[i]], L, theta), a0, sizes[i]))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.zero_()
            e0.record(stream)
            for f, a0, m in fs:
                fmm.fmm_build_tree(f.tree, x[a0:a0 + m], y[a0:a0 + m])
                fmm.fmm_interaction_lists(f.tree, f.lists, theta)
                fmm.fmm_evaluate(f.tree, f.lists, q[a0:a0 + m], p, fmm.FMM_MODE_MIXED, phi[a0:a0 + m])
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1)
            out["one_by_one"] = {"value": n / (t * 1e-3), "ms_per_step": t,
                                 "note": f"the same {len(inst)} instances through single-instance handles, "
                                         "plain launches" + ("" if world == 1 else " (this rank's share)")}
        finally:
            for f, _, _ in fs:
                f.close()
    return out


def cpu_baseline(w, W, seconds=8.0):
    """The oracle FMM as it stands on a bounded sample of the benchmark workload (2^16 points of
    the same distribution, 16 per leaf): about `seconds` on one core, then about `seconds` with one
    run per host core at once.  value/cores describe the all-core run."""
    import oracle
    oracle.build()
    ns, Ls = 1 << 16, 6
    cs = W.mixed_1m_cloud(ns)
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.fmm(cs.x, cs.y, cs.q, Ls, w.p, w.theta)
        reps += 1
        if time.perf_counter() - t0 > seconds:
            break
    one = ns * reps / (time.perf_counter() - t0)
    cores = host_cores()
    pool = OraclePool(cores, ns, Ls, w.p, w.theta)
    try:
        pool.round()  # warm-up: every worker has loaded the oracle and its sample
        t0 = time.perf_counter()
        rounds = 0
        while True:
            pool.round()
            rounds += 1
            if time.perf_counter() - t0 > seconds:
                break
        allc = cores * ns * rounds / (time.perf_counter() - t0)
    finally:
        pool.close()
    model = cpu_model()
    return {"value": allc, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"oracle FMM, N={ns} points of the same distribution, L={Ls}, p={w.p}: one run per "
                      f"core on all {cores} host cores at once, {rounds} rounds",
            "nproc": cores, "cpu_model": model,
            "single_core": {"value": one, "unit": UNIT, "cores": 1, "runs": reps}}


def profile_run(a):
    """A fixed workload run a few times as a profiler's target (see --profile-run)."""
    import torch
    from paper_1006_2269_gb300 import build, fmm, workloads as W
    build.build()
    fmm.load_library()
    dev = torch.device("cuda", 0)
    p = a.p
    if a.workload == "clusters-1m":
        c, L, theta, p = W.mixed_1m_cloud(), W.MIXED_1M.levels, W.MIXED_1M.theta, p or W.MIXED_1M.p
    elif a.workload == "uniform-1m":
        c, L, theta, p = W.uniform(1 << 20, W.SEED_BASE + 7), 8, 0.5, p or 20
    elif a.workload == "rings-1m":  # the 2^24-point workload's distribution at 2^20 points, 64 per leaf
        c, L, theta, p = W.rings_plummer(1 << 20, W.SEED_BASE + 8), 7, 0.5, p or W.LARGE_16M.p
    else:
        c, L, theta, p = W.large_16m_cloud(), W.LARGE_16M.levels, W.LARGE_16M.theta, p or W.LARGE_16M.p
    lists = a.lists if a.lists != "auto" else "parents"
    x, y, q = (torch.as_tensor(np.ascontiguousarray(v), device=dev) for v in (c.x, c.y, c.q))
    f = fmm.FMM(x, y, L, theta, parents="parents" in lists, exchange="exchange" in lists)
    try:
        fmm.fmm_set_m2l_kernel(f.tree, {"auto": fmm.FMM_M2L_AUTO, "simt": fmm.FMM_M2L_SIMT,
                                        "tensor": fmm.FMM_M2L_TENSOR}[a.m2l])
        fmm.fmm_set_m2l_shape(f.tree, *(int(v) for v in a.m2l_shape.split(",")))
        if a.blocks:
            fmm.fmm_set_launch(f.tree, *(int(v) for v in a.blocks.split(",")))
        mode = {"mixed": fmm.FMM_MODE_MIXED, "fp64": fmm.FMM_MODE_FP64, "split": fmm.FMM_MODE_SPLIT}[a.mode]
        phi = torch.empty(c.x.shape[0], dtype=torch.float64, device=dev)
        if a.stage_times:  # one untimed run first, then the library's per-stage CUDA events
            fmm.fmm_evaluate(f.tree, f.lists, q, p, mode, phi)
            torch.cuda.synchronize()
            fmm.fmm_profile_read()
            fmm.fmm_profile_enable(True)
        for _ in range(a.profile_run):
            if a.profile_steps:
                fmm.fmm_build_tree(f.tree, x, y)
                fmm.fmm_interaction_lists(f.tree, f.lists, theta)
            fmm.fmm_evaluate(f.tree, f.lists, q, p, mode, phi)
        torch.cuda.synchronize()
        if a.stage_times:
            fmm.fmm_profile_enable(False)
            prof = fmm.fmm_profile_read()
            print(json.dumps({k: round(v[0] / v[1], 4) for k, v in prof.items() if v[1]}))
        fmm.fmm_sync_status(f.tree, f.lists)
        nweak, nstrong = fmm.fmm_lists_sync(f.lists)
        print(f"{a.workload}: {a.profile_run} {'steps' if a.profile_steps else 'evaluations'}, p = {p}, "
              f"{a.mode}, lists {lists} ({nweak} weak, {nstrong} strong entries), phi[0] = {float(phi[0]):.6e}")
    finally:
        f.close()


def bench_large(dev, steps=3, warmup=2):
    """The large nonuniform workload: N = 2^24 points on 20 rings plus a Plummer-like core,
    strengths U[0, 1], 9 levels (64 points per leaf), theta = 1/2, p = 30, tolerance 1e-10, with
    the parent-level and role-exchange lists.  A step is tree, lists and evaluation (fmm_step) in
    two precisions: every stage in binary64, and the split mode (binary64 expansions, binary32
    near-field terms in float-float sums, far and near joined in binary64).  Errors against the
    binary64 direct sum at 2,048 sampled targets; per-stage device times from one more step run
    stage by stage."""
    import torch
    from paper_1006_2269_gb300 import fmm, workloads as W
    w = W.LARGE_16M
    c = W.large_16m_cloud()
    x, y, q = (torch.as_tensor(a, device=dev) for a in (c.x, c.y, c.q))
    n, tol = w.n, 1e-10
    f = fmm.FMM(x, y, w.levels, w.theta, parents=True, exchange=True)
    phi = torch.empty(n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    tg = torch.as_tensor(W.sample_targets(n, w.n_check, W.SEED_BASE + 4 + 100), device=dev)
    ref = torch.empty(tg.numel(), dtype=torch.float64, device=dev)
    fmm.fmm_direct(x, y, q, tg, ref)
    out = {"workload": w.name + ", TOL 1e-10, rings + Plummer core", "points": n, "tol": tol,
           "n_check": int(tg.numel()), "lists": "parents+exchange (Section 4's optional optimisations)",
           "steps": steps}
    try:
        for name, mode in (("binary64", fmm.FMM_MODE_FP64), ("split", fmm.FMM_MODE_SPLIT)):
            def step():
                fmm.fmm_step(f.tree, f.lists, x, y, w.theta, q, w.p, mode, phi, tol)

            for _ in range(warmup):
                step()
            torch.cuda.synchronize()
            fmm.fmm_sync_status(f.tree, f.lists)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(steps):
                step()
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / steps
            err = ((phi[tg] - ref).abs().max() / ref.abs().max()).item()
            fmm.fmm_profile_read()
            fmm.fmm_profile_enable(True)
            fmm.fmm_build_tree(f.tree, x, y)
            fmm.fmm_interaction_lists(f.tree, f.lists, w.theta)
            fmm.fmm_evaluate(f.tree, f.lists, q, w.p, mode, phi, tol)
            torch.cuda.synchronize()
            fmm.fmm_profile_enable(False)
            prof = fmm.fmm_profile_read()
            fmm.fmm_sync_status(f.tree, f.lists)
            out[name] = {"value": n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "rel_err": err,
                         "met_tol": err <= tol, "stages_ms": {k: v[0] / v[1] for k, v in prof.items() if v[1]}}
        out["precision"] = {"binary64": "every stage in binary64",
                            "split": "binary64 P2M, M2M, M2L, L2L, L2P; near field in float-float (pairs of "
                                     "binary32, terms and sums); far and near joined in binary64"}
        return out
    finally:
        f.close()


def bench_selector(dev, x, y, q, tg, ref, steps, warmup, fixed_ms, tol=1e-6):
    """The learned-parameter path on the benchmark cloud: every timed step computes the
    selector's features on a probe tree (the library's feature kernel), runs the network and its
    masked arg-max (fmm_select_params), reads the chosen (levels, p) back, then builds the lists
    and evaluates at those parameters (the probe tree is reused when its levels were chosen,
    otherwise a tree of the chosen levels is built).  Compared with the fixed parameters of the
    benchmark workload; both errors against the same binary64 direct sums."""
    import torch
    from paper_1006_2269_gb300 import fmm
    from paper_1006_2269_gb300 import selector as S
    w_theta = 0.5
    n = x.numel()
    sel = S.Selector.load(device=dev)
    L0 = S.probe_levels(n)
    trees = {L0: fmm.FMM(x, y, L0, w_theta, parents=True)}
    feats = torch.empty((1, 64), dtype=torch.float32, device=dev)
    choice = torch.empty((1, 2), dtype=torch.int32, device=dev)
    phi = torch.empty(n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    chosen = {}

    def sel_step():
        probe = trees[L0]
        fmm.fmm_build_tree(probe.tree, x, y)
        fmm.fmm_selector_features(probe.tree, tol, feats)
        fmm.fmm_select_params(sel.m, feats, choice)
        L, p = (int(v) for v in choice[0].tolist())  # the host needs the choice: one sync
        chosen[(L, p)] = chosen.get((L, p), 0) + 1
        f = trees.get(L)
        if f is None:  # first time only (warm-up): a tree of these levels
            f = trees[L] = fmm.FMM(x, y, L, w_theta, parents=True)
        if L != L0:
            fmm.fmm_build_tree(f.tree, x, y)
        fmm.fmm_interaction_lists(f.tree, f.lists, w_theta)
        fmm.fmm_evaluate(f.tree, f.lists, q, p, fmm.FMM_MODE_MIXED, phi, tol)

    try:
        for _ in range(warmup):
            sel_step()
        torch.cuda.synchronize()
        for f in trees.values():
            fmm.fmm_sync_status(f.tree, f.lists)
        chosen.clear()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            sel_step()
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        err = ((phi[tg] - ref).abs().max() / ref.abs().max()).item()
        L, p = max(chosen, key=chosen.get)  # the same choice every step on the same input
        return {"tol": tol, "value": n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                "chosen": {"levels": L, "p": p}, "rel_err": err, "met_tol": err <= tol,
                "fixed_parameters": {"levels": 8, "p": 20, "ms_per_step": fixed_ms, "value": n / (fixed_ms * 1e-3)},
                "rule_parameters": dict(zip(("levels", "p"), S.fallback_params(n, tol))),
                "note": "timed step = probe tree + features + network + arg-max + host read of the choice + "
                        "lists + evaluation (plain launches); the fixed-parameter step is the headline's graph"}
    finally:
        for f in trees.values():
            f.close()
        sel.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--no-graph", action="store_true", help="launch kernels one by one instead of replaying a CUDA graph")
    ap.add_argument("--no-batched", action="store_true", help="skip the 512-instance batched workload")
    ap.add_argument("--no-selector", action="store_true", help="skip the learned-parameter sub-result")
    ap.add_argument("--no-large", action="store_true", help="skip the 2^24-point workload at TOL 1e-10")
    ap.add_argument("--blocks", default=None, metavar="M2L,NEAR",
                    help="grid sizes of the binary32 M2L and near-field kernels instead of the autotuner's "
                         "(e.g. to profile the plain run's launch configuration under a profiler)")
    ap.add_argument("--lists", default="auto", choices=["auto", "plain", "parents", "exchange", "parents+exchange"],
                    help="interaction lists: the plain rule, with Section 4's parent-level interactions and/or "
                         "finest-level role exchange, or the fastest variant on this workload")
    ap.add_argument("--profile-run", type=int, default=0, metavar="K",
                    help="profiler target: build the tree and lists of --workload once, run K evaluations "
                         "(whole steps with --profile-steps) on plain launches, print one line and exit; "
                         "no timing, so a profiler's -s/-c counts select the same kernels on every run")
    ap.add_argument("--profile-steps", action="store_true")
    ap.add_argument("--stage-times", action="store_true",
                    help="with --profile-run: print the mean per-stage device time (ms) of the K runs")
    ap.add_argument("--workload", default="clusters-1m", choices=["clusters-1m", "uniform-1m", "rings-1m", "rings-16m"],
                    help="workload of --profile-run")
    ap.add_argument("--p", type=int, default=None, help="expansion order of --profile-run (workload's default)")
    ap.add_argument("--mode", default="mixed", choices=["mixed", "fp64", "split"], help="precision of --profile-run")
    ap.add_argument("--m2l", default="auto", choices=["auto", "simt", "tensor"], help="M2L kernel of --profile-run")
    ap.add_argument("--m2l-shape", default="0,0", metavar="CHUNK,STAGES",
                    help="tensor-core M2L tile shape of --profile-run: consecutive weak entries per row and TMEM "
                         "accumulator stages (0: defaults)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.profile_run:
        profile_run(args)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        out = run_reference(args, rank)
        if out is not None:
            print(json.dumps(out), flush=True)
        return

    import torch
    import torch.distributed as dist
    from paper_1006_2269_gb300 import build, fmm, workloads as W

    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    build.build()
    fmm.load_library()

    w = W.MIXED_1M
    c = W.mixed_1m_cloud()
    n = w.n
    xh, yh, qh = (torch.from_numpy(a).pin_memory() for a in (c.x, c.y, c.q))
    x, y, q = (a.to(dev) for a in (xh, yh, qh))
    phi = torch.empty(n, dtype=torch.float64, device=dev)
    phi_h = torch.empty(n, dtype=torch.float64).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    f = fmm.FMM(x, y, w.levels, w.theta)

    def step(mode, serial=False):
        # tree, lists and evaluation in one call; the lists and the binary32 near field run on
        # the tree's second stream, overlapped with the upward and the far-field passes.  The
        # stage profile takes the three calls one after another, so that every stage's time is
        # its own (overlapped stages stretch each other).
        if serial:
            fmm.fmm_build_tree(f.tree, x, y)
            fmm.fmm_interaction_lists(f.tree, f.lists, w.theta)
            fmm.fmm_evaluate(f.tree, f.lists, q, w.p, mode, phi)
        else:
            fmm.fmm_step(f.tree, f.lists, x, y, w.theta, q, w.p, mode, phi)

    def capture(mode):
        """The whole step (tree, lists, evaluation: ~140 kernels) as one CUDA graph."""
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            step(mode)
        torch.cuda.current_stream().wait_stream(side)
        with torch.cuda.graph(g):
            step(mode)
        torch.cuda.synchronize()
        return g

    # warm-up, launch tuning of each path, then the accuracy check against the binary64 direct
    # sum at sampled targets
    for _ in range(args.warmup):
        step(fmm.FMM_MODE_MIXED)
    fmm.fmm_sync_status(f.tree, f.lists)
    fmm.fmm_lists_sync(f.lists)

    # Section 4's optional optimisations (parent-level interactions: fewer M2L shifts; role
    # exchange: P2L / M2P instead of some near-field pairs) change the lists, not the accuracy
    # class; "auto" keeps whichever variant runs the whole step fastest here
    def time_lists(mode_lists, k=20):
        fmm.fmm_lists_set_mode(f.lists, mode_lists)
        step(fmm.FMM_MODE_MIXED)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            step(fmm.FMM_MODE_MIXED)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / k

    variants = {"plain": fmm.FMM_LISTS_PLAIN, "parents": fmm.FMM_LISTS_PARENTS,
                "exchange": fmm.FMM_LISTS_EXCHANGE,
                "parents+exchange": fmm.FMM_LISTS_PARENTS | fmm.FMM_LISTS_EXCHANGE}
    lists_ms = {}
    if args.lists == "auto":
        lists_ms = {name: time_lists(m) for name, m in variants.items()}
        lists_kind = min(lists_ms, key=lists_ms.get)
    else:
        lists_kind = args.lists
    fmm.fmm_lists_set_mode(f.lists, variants[lists_kind])
    step(fmm.FMM_MODE_MIXED)
    fmm.fmm_sync_status(f.tree, f.lists)
    tuned = {fmm.FMM_MODE_FP64: fmm.fmm_autotune(f.tree, f.lists, q, w.p, fmm.FMM_MODE_FP64, phi),
             fmm.FMM_MODE_SPLIT: fmm.fmm_autotune(f.tree, f.lists, q, w.p, fmm.FMM_MODE_SPLIT, phi)}
    if args.blocks:
        tuned[fmm.FMM_MODE_MIXED] = tuple(int(v) for v in args.blocks.split(","))
    else:
        tuned[fmm.FMM_MODE_MIXED] = fmm.fmm_autotune(f.tree, f.lists, q, w.p, fmm.FMM_MODE_MIXED, phi)

    def use(mode):
        fmm.fmm_set_launch(f.tree, *tuned[mode])

    # The autotuner times evaluations; inside a whole step the M2L shares the GPU with the near
    # field and the tree's tail, so the binary32 M2L kernel (SIMT or tensor cores, with the
    # tensor-core kernel's tile shapes) is also chosen on whole steps, as the lists are
    m2l_trial = {}
    if not args.blocks and w.p + 1 <= 32:
        def time_steps(k=12):
            step(fmm.FMM_MODE_MIXED)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(k):
                step(fmm.FMM_MODE_MIXED)
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / k

        use(fmm.FMM_MODE_MIXED)
        auto = (fmm.fmm_get_m2l_kernel(f.tree), fmm.fmm_get_m2l_shape(f.tree), tuned[fmm.FMM_MODE_MIXED])
        best = (time_steps(), auto)
        m2l_trial["autotuned"] = best[0]
        near_blocks = tuned[fmm.FMM_MODE_MIXED][1]
        for blocks in (SM_COUNT * 2, SM_COUNT * 3, SM_COUNT * 4):
            for chunk in (8, 16, 32):
                for stages in (1, 2):
                    fmm.fmm_set_m2l_kernel(f.tree, fmm.FMM_M2L_TENSOR)
                    fmm.fmm_set_m2l_shape(f.tree, chunk, stages)
                    fmm.fmm_set_launch(f.tree, blocks, near_blocks)
                    ms = time_steps()
                    m2l_trial[f"tensor {blocks}x{chunk}x{stages}"] = ms
                    if ms < best[0]:
                        best = (ms, (fmm.FMM_M2L_TENSOR, (chunk, stages), (blocks, near_blocks)))
        kind, shape, tuned[fmm.FMM_MODE_MIXED] = best[1]
        fmm.fmm_set_m2l_kernel(f.tree, kind)
        fmm.fmm_set_m2l_shape(f.tree, *shape)
        use(fmm.FMM_MODE_MIXED)

    use(fmm.FMM_MODE_MIXED)
    tg = torch.as_tensor(W.sample_targets(n, w.n_check, W.SEED_BASE + 101), device=dev)
    ref = torch.empty(tg.numel(), dtype=torch.float64, device=dev)
    fmm.fmm_direct(x, y, q, tg, ref)
    step(fmm.FMM_MODE_MIXED)
    torch.cuda.synchronize()
    scale = ref.abs().max().item()
    err_mixed = (phi[tg] - ref).abs().max().item() / scale
    use(fmm.FMM_MODE_FP64)
    step(fmm.FMM_MODE_FP64)
    torch.cuda.synchronize()
    err_fp64 = (phi[tg] - ref).abs().max().item() / scale
    use(fmm.FMM_MODE_SPLIT)
    step(fmm.FMM_MODE_SPLIT)
    torch.cuda.synchronize()
    err_split = (phi[tg] - ref).abs().max().item() / scale
    nweak, npairs = pair_counts(f)

    graphs = {}
    if not args.no_graph:
        try:
            for m in (fmm.FMM_MODE_MIXED, fmm.FMM_MODE_FP64):
                use(m)
                graphs[m] = capture(m)
        except Exception as exc:  # report and time plain launches instead
            print(f"graph capture failed: {exc}", file=sys.stderr)
            graphs = {}

    def timed(mode, steps, e2e=False, profile=False):
        use(mode)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        fmm.fmm_profile_read()
        fmm.fmm_profile_enable(profile)
        l0 = fmm.fmm_launch_count()
        for i in range(steps):
            flush.zero_()
            starts[i].record(stream)
            if e2e:
                x.copy_(xh, non_blocking=True)
                y.copy_(yh, non_blocking=True)
                q.copy_(qh, non_blocking=True)
            if mode in graphs and not profile:
                graphs[mode].replay()
            else:
                step(mode, serial=profile)
            if e2e:
                phi_h.copy_(phi, non_blocking=True)
            ends[i].record(stream)
        torch.cuda.synchronize()
        launches = fmm.fmm_launch_count() - l0
        if mode in graphs and not profile:
            launches = per_step_launches * steps
        fmm.fmm_profile_enable(False)
        prof = fmm.fmm_profile_read()
        if world > 1:
            dist.barrier()
        ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
        return max_over_ranks(ms, world, dev), launches, prof

    use(fmm.FMM_MODE_MIXED)
    l0 = fmm.fmm_launch_count()
    step(fmm.FMM_MODE_MIXED)
    per_step_launches = fmm.fmm_launch_count() - l0
    _, _, prof = timed(fmm.FMM_MODE_MIXED, args.steps, profile=True)
    # The sampler's window: about one second of the same graph-replayed steps (untimed) right
    # before the timed K steps, then the timed steps themselves, so that a short timed region
    # still gets many clock samples under the same load
    with ClockSampler(local) as clk:
        use(fmm.FMM_MODE_MIXED)
        t_soak = time.perf_counter()
        while time.perf_counter() - t_soak < 1.0:
            for _ in range(20):
                flush.zero_()
                if fmm.FMM_MODE_MIXED in graphs:
                    graphs[fmm.FMM_MODE_MIXED].replay()
                else:
                    step(fmm.FMM_MODE_MIXED)
            torch.cuda.synchronize()
        ms_mixed_plain, launches, _ = timed(fmm.FMM_MODE_MIXED, args.steps)
    ms_e2e, _, _ = timed(fmm.FMM_MODE_MIXED, args.steps, e2e=True)
    ms_fp64, _, prof64 = timed(fmm.FMM_MODE_FP64, args.fp64_steps, profile=True)
    ms_split, _, prof_split = timed(fmm.FMM_MODE_SPLIT, args.fp64_steps, profile=True)
    fmm.fmm_sync_status(f.tree, f.lists)

    K = args.steps
    per_step = ms_mixed_plain / K
    value = job_throughput(world, n, ms_mixed_plain, K)
    stage_ms = {k: v[0] / max(v[1], 1) for k, v in prof.items() if v[1]}
    stage_ms64 = {k: v[0] / max(v[1], 1) for k, v in prof64.items() if v[1]}
    top = max(stage_ms, key=stage_ms.get)

    # roofline of the dominant kernel (per launch): algorithmic work / measured duration.  The
    # binary32 FMA and special-function (lg2) peaks come from the library's probes on this GPU;
    # the unit-count figures (128 FMA and 16 lg2 per SM per clock at the maximum SM clock) are
    # kept beside them
    P = w.p + 1
    hbm, hbm_kind = peaks()
    mufu_derived = 16 * SM_COUNT * SM_MAX_MHZ * 1e6  # log2 evaluations / s
    fp32_derived = 128 * 2 * SM_COUNT * SM_MAX_MHZ * 1e6  # flop / s
    probed = {"ffma_tflops": fmm.fmm_probe_throughput(fmm.FMM_PROBE_FFMA, 4096) / 1e12,
              "lg2_per_s": fmm.fmm_probe_throughput(fmm.FMM_PROBE_LG2, 1024),
              "dfma_tflops": fmm.fmm_probe_throughput(fmm.FMM_PROBE_DFMA, 256) / 1e12}
    mufu_peak = probed["lg2_per_s"]
    fp32_peak = probed["ffma_tflops"] * 1e12
    t_top = stage_ms[top] * 1e-3
    m2l_kind = fmm.fmm_get_m2l_kernel(f.tree)
    if m2l_kind == fmm.FMM_M2L_AUTO:
        m2l_kind = fmm.FMM_M2L_TENSOR if 24 <= P <= 32 else fmm.FMM_M2L_SIMT
    if top == "near":
        roof = {"bound": "alu", "achieved": npairs / t_top / 1e12, "peak": mufu_peak / 1e12,
                "unit": "Tlog2/s (MUFU)", "traffic": None}
    elif top == "m2l" and m2l_kind == fmm.FMM_M2L_TENSOR:
        # tcgen05 split-tf32: three tf32 products per element of the contraction (4 P^2 flop per
        # weak pair each); peak = tf32 dense rate, the measured bf16 rate x the nominal tf32/bf16
        # ratio 1/2
        bf16 = measured_bf16_tflops()
        roof = {"bound": "tensor", "achieved": 3 * nweak * 4 * P * P / t_top / 1e12, "peak": bf16 / 2,
                "unit": "TFLOP/s (tf32 tensor)", "traffic": None}
    elif top == "m2l":
        # dram__bytes_read.sum + dram__bytes_write.sum of k_m2l_pairs<float, 21> on this workload,
        # from one ncu capture; valid while that kernel is unchanged
        traffic = M2L_TRAFFIC.get((P, n, lists_kind))
        roof = {"bound": "alu", "achieved": nweak * 4 * P * P / t_top / 1e12, "peak": fp32_peak / 1e12,
                "unit": "TFLOP/s (FP32 FMA pipe)", "traffic": traffic}
    elif top == "tree_sort":
        byts = n * (32 + 16 * 24)
        roof = {"bound": "hbm", "achieved": byts / t_top / 1e9, "peak": hbm, "unit": "GB/s",
                "traffic": None}
    else:
        byts = n * 30 * w.levels
        roof = {"bound": "hbm", "achieved": byts / t_top / 1e9, "peak": hbm, "unit": "GB/s",
                "traffic": None}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["kernel"] = top
    roof["peak_kind"] = (hbm_kind if roof["bound"] == "hbm" else
                         "measured (bf16 dense burst) x 1/2 for tf32" if roof["bound"] == "tensor" else
                         "measured: the library's throughput probe on this GPU")

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "n": n, "levels": w.levels, "theta": w.theta, "p": w.p,
                   "mode": "mixed", "l2": "flushed between steps (256 MB write outside the events)",
                   "replicas": world, "cuda_graph": bool(graphs),
                   ("launch_blocks" if args.blocks else "autotuned_blocks"): {
                       "m2l": tuned[fmm.FMM_MODE_MIXED][0], "near_field": tuned[fmm.FMM_MODE_MIXED][1]},
                   "m2l_kernel": "tensor cores (tcgen05, split tf32)" if m2l_kind == fmm.FMM_M2L_TENSOR
                   else "SIMT binary32",
                   "near_targets_per_lane": fmm.fmm_get_near_shape(f.tree) or 2,
                   "lists": lists_kind + ("" if lists_kind == "plain" else " (Section 4's optional optimisations)"),
                   "lists_trial_ms_per_step": lists_ms or None,
                   "m2l_trial_ms_per_step": m2l_trial or None},
        "rel_err": err_mixed, "rel_err_fp64": err_fp64, "n_check": w.n_check,
        "fp64_path": {"value": job_throughput(world, n, ms_fp64, args.fp64_steps),
                      "ms_per_step": ms_fp64 / args.fp64_steps, "stages_ms": stage_ms64},
        "split_path": {"value": job_throughput(world, n, ms_split, args.fp64_steps),
                       "ms_per_step": ms_split / args.fp64_steps, "rel_err": err_split,
                       "precision": "binary64 expansions, float-float near field, binary64 join",
                       "stages_ms": {k: v[0] / max(v[1], 1) for k, v in prof_split.items() if v[1]}},
        "speedup_vs_fp64": (ms_fp64 / args.fp64_steps) / per_step,
        "stages_ms": stage_ms, "weak_pairs": nweak, "near_pair_evals": npairs,
        "e2e": {"value": job_throughput(world, n, ms_e2e, K), "unit": UNIT,
                "h2d_bytes_per_step": 24 * n, "d2h_bytes_per_step": 8 * n},
        "gpu_launches": launches,
        "roofline": roof,
        "peaks_probed": dict(probed, ffma_tflops_derived=fp32_derived / 1e12, lg2_per_s_derived=mufu_derived),
        "clocks": dict(clk.summary(), window="~1 s of identical untimed steps, then the timed steps"),
    }
    if not args.no_large:
        out["large"] = bench_large(dev)
    if not args.no_selector:
        out["selector"] = bench_selector(dev, x, y, q, tg, ref, max(3, min(K, 10)), args.warmup, per_step)
    if not args.no_batched:
        out["batched"] = bench_batched(dev, max(3, min(K, 10)), args.warmup, sequential=(rank == 0),
                                       world=world, rank=rank)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w, W)
    if rank == 0:
        print(json.dumps(out), flush=True)
    f.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
