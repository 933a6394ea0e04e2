#!/usr/bin/env python3
"""Benchmark of the GB300 facility-location hot path (one JSON line on rank 0).

A step is one pass of the whole path over one instance: bottom-k sketches and
ADS (phase i), radii (phase ii), key sort and greedy-MIS facility selection
(phase iii), assignment BFS and objective.  Inputs are resident in HBM when the
timed region starts (they are larger than L2 for the default workload).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl gpu|reference]

Metric: sketch edge-merges per second (an edge-merge is one CSR entry (v, u)
processed at a hop whose u gained sketch entries at the previous hop), whole
job over all ranks.  Under torchrun each rank solves its own replica of the
workload (the method has no exchange step on one GPU per instance), so the
scaling is weak.  `--impl reference` times the CPU oracle on a bounded sample
of the same workload (the first hops of its sketch build) on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import flsynth  # noqa: E402

METRIC = "sketch edge-merges/sec and HBM GB/s (% peak); solves/sec batched vs plain; p50/p99"
UNIT = "edge-merges/s"
DEFAULT_WORKLOAD = "rmat26"
# bounded oracle samples (hops of its sketch build) per workload: ~10-30 s of CPU work
CPU_SAMPLE_HOPS = {"er10k": 64, "rmat20": 64, "rmat26": 1}
PROFILE_DIR = os.path.join(ROOT, "profiles")
# exact-size workload: sampled sources, facilities and the k of the accuracy study
EXACT_SEED = 13
EXACT_SOURCES = 4096
EXACT_FACILITIES = 16384
EXACT_CPU_SOURCES = 256
ACCURACY_K = (4, 8, 16, 32)


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def source_hash(path):
    with open(path, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def ncu_traffic(kernel, workload):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    p = os.path.join(PROFILE_DIR, "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    e = d.get(kernel, {}).get(workload)
    if not e:
        return None
    src = os.path.join(ROOT, "paper_1503_03635_gb300", "csrc", e["source"])
    if not os.path.exists(src) or source_hash(src) != e["source_sha256_16"]:
        return None
    return e["dram_bytes_per_launch"]


class Clocks:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for ln in fh:
                parts = [x.strip() for x in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, val in zip(names, r[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def cpu_sample(w, hops, steps=1):
    """Time the CPU oracle's sketch build for `hops` hops of the same workload."""
    import oracle

    g = oracle.Graph(w.rowp, w.cols)
    times, merges = [], 0
    for _ in range(steps):
        t0 = time.perf_counter()
        g.build_sketches(w.k, w.seed, max_hops=hops)
        times.append(time.perf_counter() - t0)
        merges = g.edge_merges
        done_hops = g.hops
    g.close()
    t = statistics.median(times)
    return {"value": merges / t, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": f"oracle sketch build (phase i), first {min(hops, done_hops)} hop(s) on the full "
                      f"{w.name} graph: {merges} edge-merges in {t:.2f} s"}


def workload_config(w):
    return {"workload": w.name, "n": w.n, "nnz": w.nnz, "k": w.k, "rank_seed": w.seed,
            "clients": int(w.client.sum()), "facilities": int(np.isfinite(w.cost).sum()),
            "l2": "inputs larger than L2 (no flush)" if (w.nnz * 4 + w.n * 8) > 129e6 else
                  "inputs smaller than L2",
            "parallelism": "replicas (one instance per GPU)"}


def run_reference_exact(args):
    """The oracle's BFS ball sizes on the exact workload's graph: a bounded
    sample of its sources per step (sources/s on the host cores)."""
    import oracle

    w = flsynth.config("rmat20")
    rng = np.random.default_rng(EXACT_SEED)
    src = rng.choice(w.n, size=EXACT_SOURCES, replace=False).astype(np.int32)[:EXACT_CPU_SOURCES]
    g = oracle.Graph(w.rowp, w.cols)
    for _ in range(args.warmup):
        g.ball_sizes(src, 20)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        g.ball_sizes(src, 20)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = len(src) * len(times) / total
    unit = "sources/s"
    line = {"impl": "reference", "metric": "exact neighbourhood sizes (sources/s) and ADS accuracy vs k",
            "value": value, "unit": unit, "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "exact", "graph": f"rmat20 (n={w.n}, nnz={w.nnz})", "sources": len(src),
                       "max_dist": 20},
            "cpu_baseline": {"value": value, "unit": unit, "cores": oracle.threads(), "kind": "oracle",
                             "sample": f"oracle BFS ball sizes of the first {len(src)} of the "
                                       f"{EXACT_SOURCES} sampled sources per step"},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    rank = env_int("RANK", 0)
    if rank != 0:
        return 0
    if args.workload == "exact":
        return run_reference_exact(args)
    w = flsynth.config(args.workload)
    hops = CPU_SAMPLE_HOPS.get(args.workload, 1)
    import oracle

    g = oracle.Graph(w.rowp, w.cols)
    for _ in range(args.warmup):
        g.build_sketches(w.k, w.seed, max_hops=hops)
    times = []
    merges = 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        g.build_sketches(w.k, w.seed, max_hops=hops)
        times.append(time.perf_counter() - t0)
        merges = g.edge_merges
    total = sum(times)
    value = merges * len(times) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": workload_config(w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": f"oracle sketch build, first {hops} hop(s) of {w.name} per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def mis_summary(rows):
    """Per greedy round of the last step's MIS: undecided facilities at its
    start, those it decided, its largest ball radius T, host ms, the bucket
    sizes by ball radius, and per cover / gather round [step, frontier,
    pulled, ms] (fl_mis_log rows)."""
    if rows is None or len(rows) == 0:
        return None
    out = []
    for rd in sorted(set(int(x) for x in rows[:, 0])):
        R = rows[rows[:, 0] == rd]
        tot = R[R[:, 1] == 3]
        d = {"round": rd}
        if len(tot):
            d.update(undecided=int(tot[0, 3]), decided=int(tot[0, 4]), T=int(tot[0, 2]),
                     ms=round(tot[0, 5] / 1e3, 2))
        d["buckets"] = {int(b): int(c) for b, c in R[R[:, 1] == 2][:, 2:4]}
        for kind, name in ((0, "cover"), (1, "gather")):
            d[name] = [[int(x[2]), int(x[3]), int(x[4]), round(x[5] / 1e3, 2)] for x in R[R[:, 1] == kind]]
        out.append(d)
    return out


def run_gpu(args):
    import torch

    import paper_1503_03635_gb300 as fl

    rank, world, local = env_int("RANK", 0), env_int("WORLD_SIZE", 1), env_int("LOCAL_RANK", 0)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    fl.load()
    w = flsynth.config(args.workload)
    stream = torch.cuda.Stream(device=dev)

    # ---------------- device-resident inputs and outputs
    rowp_d = torch.from_numpy(w.rowp).to(dev)
    cols_d = torch.from_numpy(w.cols).to(dev)
    cost_d = torch.from_numpy(w.cost).to(dev)
    client_d = torch.from_numpy(w.client).to(dev)
    radii_d = torch.empty(w.n, dtype=torch.float64, device=dev)
    open_d = torch.empty(w.n, dtype=torch.uint8, device=dev)
    assign_d = torch.empty(w.n, dtype=torch.int32, device=dev)
    dist_d = torch.empty(w.n, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    g = fl.Graph(rowp_d, cols_d, stream=stream)
    info = {}
    tune = None
    if not args.no_autotune:
        # the graph's launch and round-switch schedule, picked by timing the
        # path on it (results do not depend on it)
        tune = g.autotune(w.k, w.seed, cost_d, client_d, max_trials=args.tune_trials)
        tune["trials"] = args.tune_trials

    def step():
        g.build_sketches(w.k, w.seed)
        s = fl.Solve(g)
        s.compute_radii(cost_d, client_d, radii_d)
        _, nopen = s.open_facilities(open_d)
        s.assign_clients(assign_d, dist_d)
        obj = s.objective()
        info["n_open"] = nopen
        info["objective"] = obj[0]
        info["mis"] = s.stats()
        info["mis_log"] = s.mis_log()
        s.close()

    for _ in range(args.warmup):
        step()

    # ---------------- timed region (device-resident inputs)
    g.profile(True)
    g.profile_reset()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    if dist:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    torch.cuda.synchronize()
    stats = g.stats()
    g_schedule = g.schedule
    prof = {name: g.profile_query(name) for name in fl.PROF_CLASSES}
    launches = g.profile_query(-1)["launches"]
    # the per-hop census (scanned / mask-merged entries) takes extra kernels:
    # one more build outside the timed region collects it
    g.profile(True, census=True)
    g.build_sketches(w.k, w.seed)
    g.profile(False)
    model = g.hop_model()
    hop_detail = [{"hop": h["hop"], "ms": round(h["ms"], 3), "scanned": h["scanned"],
                   "mask_share": round(h["mask"] / h["scanned"], 4) if h["scanned"] else 0.0,
                   "changed": h["changed"], "E": m["edge_merges"], "A": m["merging"], "delta_sum": m["delta_sum"],
                   "delta_read": m["delta_read"], "new": m["new_entries"]}
                  for h, m in zip(g.hop_stats(), model)]
    # algorithmic bytes of one build by the per-hop model: row offsets and own
    # sketch (read + write) per merging vertex, a column and the neighbour's
    # delta ranks per edge-merge, an ADS id + weight per new entry
    model_bytes = sum(8 * m["merging"] + 4 * m["edge_merges"] + 8 * m["delta_sum"] + 16 * w.k * m["merging"]
                      + 12 * m["new_entries"] for m in model)
    g.profile(False)
    merges_step = stats["edge_merges"]
    value = world * merges_step * args.steps / (ms / 1e3)

    # ---------------- end to end through the C ABI with pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        rowp_h = torch.from_numpy(w.rowp).pin_memory()
        cols_h = torch.from_numpy(w.cols).pin_memory()
        cost_h = torch.from_numpy(w.cost).pin_memory()
        client_h = torch.from_numpy(w.client).pin_memory()
        open_h = torch.empty(w.n, dtype=torch.uint8).pin_memory()
        assign_h = torch.empty(w.n, dtype=torch.int32).pin_memory()
        dist_h = torch.empty(w.n, dtype=torch.int32).pin_memory()
        g.close()
        times = []
        parts = {}
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            marks = []
            g2 = fl.Graph(rowp_h, cols_h, stream=stream)      # H2D of the CSR
            marks.append(("graph_create", time.perf_counter()))
            g2.set_schedule(**g_schedule)                        # the schedule tuned above
            g2.build_sketches(w.k, w.seed)
            marks.append(("build_sketches", time.perf_counter()))
            s2 = fl.Solve(g2)
            s2.compute_radii(cost_h, client_h)                  # H2D of costs and mask
            marks.append(("radii", time.perf_counter()))
            s2.open_facilities(open_h)                          # D2H of the open set
            marks.append(("open_facilities", time.perf_counter()))
            s2.assign_clients(assign_h, dist_h)                 # D2H of assignment and distance
            marks.append(("assign", time.perf_counter()))
            s2.objective()
            s2.close()
            g2.close()
            marks.append(("objective_close", time.perf_counter()))
            dt = time.perf_counter() - t0
            if i > 0:  # the first pass warms allocations
                times.append(dt)
                prev = t0
                for name, t in marks:  # host wall time of each call (each returns with its work done)
                    parts[name] = parts.get(name, 0.0) + 1e3 * (t - prev) / args.e2e_steps
                    prev = t
        t_e2e = sum(times) / len(times)
        if dist:
            t = torch.tensor([t_e2e], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            t_e2e = float(t.item())
        e2e = {"value": world * merges_step / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": int(w.rowp.nbytes + w.cols.nbytes + w.cost.nbytes + w.client.nbytes),
               "d2h_bytes_per_step": int(open_h.numel() + 4 * assign_h.numel() + 4 * dist_h.numel()),
               "ms_per_step": 1e3 * t_e2e, "steps": len(times),
               "calls_ms": {k: round(v, 2) for k, v in parts.items()}}
    else:
        g.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    # ---------------- roofline of the dominant kernel (the sketch merge)
    peak, peak_kind = measured_peaks()
    mp = prof["sketch_merge"]
    # numerator: the model's bytes of every timed build (the same graph and
    # seed each step); beside it, the bytes the merge kernels' loads touched
    alg_bytes = model_bytes * args.steps
    achieved = alg_bytes / (mp["ms"] / 1e3) / 1e9 if mp["ms"] > 0 else None
    achieved_reads = mp["alg_bytes"] / (mp["ms"] / 1e3) / 1e9 if mp["ms"] > 0 else None
    per_launch_bytes = alg_bytes / mp["launches"] if mp["launches"] else None
    traffic = ncu_traffic("k_merge_hop", w.name)
    roofline = {"kernel": "k_merge_hop", "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "peak_kind": f"{peak_kind} copy bandwidth", "alg_bytes_per_launch": per_launch_bytes,
                "alg_bytes_per_build": model_bytes,
                "alg_model": "per hop: 8 A + 4 E + 8 sum|D_{h-1}(u)| + 16 k A + 12 |D_h| (hop_detail terms)",
                "achieved_reads": achieved_reads, "frac_reads": (achieved_reads / peak) if achieved_reads else None,
                "reads_bytes_per_build": mp["alg_bytes"] / args.steps,
                "reads_model": "as alg_model with the neighbour-delta ranks the kernels' loads read (delta_read) "
                               "in place of sum|D_{h-1}(u)|",
                "launches": mp["launches"], "kernel_ms": mp["ms"],
                "share_of_step": mp["ms"] / ms if ms > 0 else None}

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_sample(w, CPU_SAMPLE_HOPS.get(w.name, 1))

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": workload_config(w),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "solves_per_sec": world * args.steps / (ms / 1e3),
            "phases_ms_per_step": {k: v["ms"] / args.steps for k, v in prof.items()},
            "schedule": g_schedule, "autotune": tune,
            "hops": stats["hops"], "edge_merges_per_step": merges_step, "ads_entries": stats["ads_entries"],
            "n_open": info.get("n_open"), "objective": info.get("objective"),
            "mis_rounds": info.get("mis", {}).get("mis_rounds"), "hop_detail": hop_detail,
            "mis_detail": mis_summary(info.get("mis_log"))}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_exact(args):
    """Exact neighbourhood sizes (bit-parallel BFS) on the R-MAT scale-20
    graph: sources/s of fl_ball_sizes to distance 20, the ADS accuracy study
    of Section 5.1 (Fig. 1: relative error of the HIP estimate against the
    exact size, per k), and exact-count radii against the sketch radii."""
    import torch

    import paper_1503_03635_gb300 as fl

    rank = env_int("RANK", 0)
    local = env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fl.load()
    w = flsynth.config("rmat20")
    n = w.n
    D = 20
    rng = np.random.default_rng(EXACT_SEED)
    src = rng.choice(n, size=EXACT_SOURCES, replace=False).astype(np.int32)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        g = fl.Graph(torch.from_numpy(w.rowp).to(dev), torch.from_numpy(w.cols).to(dev), stream=stream)
        src_d = torch.from_numpy(src).to(dev)
        out_d = torch.empty((len(src), D + 1), dtype=torch.int64, device=dev)
    torch.cuda.synchronize()

    def step():
        g.ball_sizes(src_d, D, None, out=out_d)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    g.profile(True)
    g.profile_reset()
    clocks = Clocks(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    px = g.profile_query("exact")
    launches = g.profile_query(-1)["launches"]
    g.profile(False)
    peak, peak_kind = measured_peaks()
    achieved = px["alg_bytes"] / (px["ms"] / 1e3) / 1e9 if px["ms"] > 0 else None
    roofline = {"kernel": "exact-size class: bit-parallel BFS levels (k_x_heavy, k_x_light, k_x_td, k_x_td_finish)", "bound": "hbm",
                "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": ncu_traffic("k_x_level", "exact"),
                "peak_kind": f"{peak_kind} copy bandwidth",
                "alg_bytes_per_launch": px["alg_bytes"] / max(1, px["launches"]), "launches": px["launches"],
                "kernel_ms": px["ms"], "share_of_step": px["ms"] / (ms * args.steps) if ms > 0 else None}
    exact = out_d.cpu().numpy()

    # ---- ADS accuracy vs k: 100 sampled vertices per distance 1..20
    samp = np.stack([rng.choice(n, size=100, replace=False) for _ in range(D)]).astype(np.int32)
    flat = samp.reshape(-1)
    ex = g.ball_sizes(flat, D)
    accuracy = {}
    for k in ACCURACY_K:
        g.build_sketches(k, w.seed)
        est = g.ball_estimates(flat, D)
        errs = []
        for d in range(1, D + 1):
            rows = slice((d - 1) * 100, d * 100)
            se = ex[rows, d].astype(np.float64)
            errs.append(np.abs(se - est[rows, d]) / se)
        e = np.concatenate(errs)
        accuracy[str(k)] = {"mean_rel_err": float(e.mean()), "var_rel_err": float(e.var()),
                            "per_distance_mean": [round(float(x.mean()), 5) for x in errs]}

    # ---- exact-count radii of sampled facilities vs the sketch radii
    fac = rng.choice(n, size=EXACT_FACILITIES, replace=False).astype(np.int32)
    cost = np.full(n, np.inf)
    cost[fac] = w.cost[fac]
    radii = {}
    g.build_sketches(w.k, w.seed)
    s = fl.Solve(g)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r_exact = s.compute_radii_exact(cost, w.client)
    t_exact = time.perf_counter() - t0
    s.open_facilities()
    s.assign_clients()
    obj_exact = s.objective()[0]
    s.close()
    for k in ACCURACY_K:
        g.build_sketches(k, w.seed)
        s = fl.Solve(g)
        r = s.compute_radii(cost, w.client)
        s.open_facilities()
        s.assign_clients()
        obj = s.objective()[0]
        s.close()
        fin = np.isfinite(r_exact[fac]) & np.isfinite(r[fac])
        rel = np.abs(r[fac][fin] - r_exact[fac][fin]) / r_exact[fac][fin]
        radii[str(k)] = {"mean_rel_err": float(rel.mean()), "p90_rel_err": float(np.percentile(rel, 90)),
                         "objective_vs_exact": obj / obj_exact}
    g.close()
    if rank != 0:
        return 0
    line = {"metric": "exact neighbourhood sizes (sources/s) and ADS accuracy vs k", "value": len(src) / (ms / 1e3),
            "unit": "sources/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "exact", "graph": f"rmat20 (n={n}, nnz={w.nnz})", "sources": len(src),
                       "max_dist": D, "l2": "bit arrays (96 MB) mostly L2-resident; no flush"},
            "roofline": roofline, "gpu_launches": launches, "clocks": clk,
            "accuracy_vs_k": {"samples": "100 vertices per distance 1..20 (Section 5.1)", "by_k": accuracy},
            "exact_radii": {"facilities": len(fac), "seconds": t_exact, "facilities_per_s": len(fac) / t_exact,
                            "sketch_vs_exact_by_k": radii}}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """Batched workload: solves/s of the batch form vs the plain form (one
    instance per fl_* sequence) on the same GPU, and whether they agree."""
    import torch

    import paper_1503_03635_gb300 as fl

    rank = env_int("RANK", 0)
    local = env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fl.load()
    bw = flsynth.batch_config()
    base = bw.resident
    R, n = len(bw.inst_cost), base.n
    k, seed = base.k, base.seed
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        # resident graphs, costs and client sets (device memory, built once)
        g = fl.Graph(torch.from_numpy(base.rowp).to(dev), torch.from_numpy(base.cols).to(dev), stream=stream)
        cost_r = torch.from_numpy(np.concatenate(bw.inst_cost)).to(dev)
        client_r = torch.from_numpy(np.concatenate(bw.inst_client)).to(dev)
        tune = None
        if not args.no_autotune:
            # tuned on the resident graph with the first instance's inputs
            tune = g.autotune(k, seed, cost_r[:n], client_r[:n], max_trials=args.tune_trials)
        g.build_sketches(k, seed)
        er_csr = [(torch.from_numpy(x.rowp).to(dev), torch.from_numpy(x.cols).to(dev)) for x in bw.graphs]
        cost_u = torch.from_numpy(np.concatenate([x.cost for x in bw.graphs])).to(dev)
        client_u = torch.from_numpy(np.concatenate([x.client for x in bw.graphs])).to(dev)
        er_graphs = [fl.Graph(r, c, stream=stream) for r, c in er_csr]
        brep = fl.Batch.replicas(g, R)
        brep.set_schedule(g.schedule)
        buni = fl.Batch.union(er_csr, stream=stream)
        buni_sched = dict(hop_group=0, sparse_div=16, dense_div=8, edge_div=16, graph_bfs=0, level_cap=0)
        N_r, N_u = brep.n_total, buni.n_total
        out = {f: torch.empty(N_r + N_u, dtype=dt, device=dev)
               for f, dt in (("open", torch.uint8), ("assign", torch.int32), ("dist", torch.int32))}
        plain = {f: torch.empty_like(t) for f, t in out.items()}
        uoff = np.concatenate([[0], np.cumsum([x.n for x in bw.graphs])])
        plain_obj = np.zeros(R + len(bw.graphs))
        batch_obj = np.zeros(R + len(bw.graphs))

    def batched():
        r1 = brep.solve(k, seed, cost_r, client_r, out["open"][:N_r], out["assign"][:N_r], out["dist"][:N_r])
        r2 = buni.solve(k, seed, cost_u, client_u, out["open"][N_r:], out["assign"][N_r:], out["dist"][N_r:])
        batch_obj[:R] = r1["objective"]
        batch_obj[R:] = r2["objective"]

    def one_by_one():
        for i in range(R):
            s = fl.Solve(g)
            sl = slice(i * n, (i + 1) * n)
            s.compute_radii(cost_r[sl], client_r[sl])
            s.open_facilities(plain["open"][sl])
            s.assign_clients(plain["assign"][sl], plain["dist"][sl])
            plain_obj[i] = s.objective()[0]
            s.close()
        for j, gj in enumerate(er_graphs):
            gj.build_sketches(k, seed)
            s = fl.Solve(gj)
            sl = slice(N_r + int(uoff[j]), N_r + int(uoff[j + 1]))
            s.compute_radii(cost_u[int(uoff[j]):int(uoff[j + 1])], client_u[int(uoff[j]):int(uoff[j + 1])])
            s.open_facilities(plain["open"][sl])
            s.assign_clients(plain["assign"][sl], plain["dist"][sl])
            plain_obj[R + j] = s.objective()[0]
            s.close()

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    clocks = Clocks(local)
    clocks.start()
    ms_batch = timed(batched)
    ms_plain = timed(one_by_one)
    # the same batches with the assignment BFS as one CUDA graph (device-side level loop)
    host_out = {f: t.clone() for f, t in out.items()}
    sched_graph = dict(g.schedule, graph_bfs=1)
    brep.set_schedule(sched_graph)
    buni.set_schedule(dict(buni_sched, graph_bfs=1))
    ms_graph = timed(batched)
    graph_same = all(torch.equal(out[f], host_out[f]) for f in out)
    clk = clocks.stop()
    same = all(torch.equal(host_out[f], plain[f]) for f in out)
    obj_ok = bool(np.all(np.abs(batch_obj - plain_obj) <= 1e-9 * np.abs(plain_obj)))
    n_inst = R + len(bw.graphs)
    if rank == 0:
        line = {"metric": METRIC, "value": n_inst / (ms_batch / 1e3), "unit": "solves/s", "n_gpus": 1,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_batch, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": {"workload": "batch", "instances": n_inst,
                           "resident": f"{R} instances on rmat20 (n={n}, nnz={base.nnz}), k={k}",
                           "graphs": f"{len(bw.graphs)} ER graphs, {N_u} vertices in all, "
                                     f"{sum(x.nnz for x in bw.graphs)} CSR entries, k={k}",
                           "step": "every instance solved once (radii, keys, MIS, assignment, objective; "
                                   "the ER graphs' sketches built too)"},
                "plain": {"value": n_inst / (ms_plain / 1e3), "unit": "solves/s", "ms_per_step": ms_plain,
                          "form": "one fl_* sequence per instance on one stream"},
                "speedup_vs_plain": ms_plain / ms_batch,
                "graph_form": {"value": n_inst / (ms_graph / 1e3), "unit": "solves/s", "ms_per_step": ms_graph,
                               "form": "the same batches, the assignment BFS as one CUDA graph (conditional WHILE "
                                       "node: the level loop on the device)",
                               "identical_to_host_driven": bool(graph_same)},
                "identical_to_plain": bool(same and obj_ok), "schedule": g.schedule, "autotune": tune,
                "clocks": clk}
        print(json.dumps(line), flush=True)
    for x in er_graphs:
        x.close()
    brep.close()
    buni.close()
    g.close()
    return 0


def run_serve(args):
    """Serving workload: a resident R-MAT graph with built sketches (k=32),
    a Poisson stream of queries (client set of log-uniform size, one
    log-uniform cost), continuous batching over two workers; p50/p99 latency
    (arrival -> results on the host) and solves/s, beside the same queries
    run plain one after another."""
    import threading

    import torch

    import paper_1503_03635_gb300 as fl
    from paper_1503_03635_gb300 import serve

    local = env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fl.load()
    scale = args.serve_scale
    rowp, cols = flsynth.rmat(scale, 16, 42 + 5)
    n = len(rowp) - 1
    k, seed = 32, flsynth.SKETCH_SEED
    g = fl.Graph(torch.from_numpy(rowp).to(dev), torch.from_numpy(cols).to(dev))
    g.build_sketches(k, seed)
    torch.cuda.synchronize()
    rate, warm, dur = args.rate, args.serve_warmup, args.serve_seconds
    m = int((warm + dur) * rate * 1.2) + 16
    gaps = -np.log1p(-flsynth.uniform(m, flsynth.QUERY_SEED, 0.0, 1.0)) / rate
    arrivals = np.cumsum(gaps)
    arrivals = arrivals[arrivals < warm + dur]
    sizes = flsynth.loguniform(len(arrivals), flsynth.QUERY_SEED + 1, 1.0e3, 1.0e6)
    costs = flsynth.loguniform(len(arrivals), flsynth.QUERY_SEED + 2, 10.0, 1.0e3)
    qs = [serve.Query(costs[i], client_seed=flsynth.QUERY_SEED * 1000003 + i, client_frac=min(1.0, sizes[i] / n))
          for i in range(len(arrivals))]
    tune = None
    if not args.no_autotune:
        # the resident graph's schedule, tuned on one query's inputs
        m0 = torch.empty(n, dtype=torch.uint8, device=dev)
        serve.client_mask_on_device(torch, n, qs[0].client_seed, qs[0].client_frac, dev, m0)
        tune = g.autotune(k, seed, torch.full((n,), qs[0].cost, dtype=torch.float64, device=dev), m0,
                          max_trials=args.tune_trials)
        torch.cuda.synchronize()
    sched = g.schedule
    srv = serve.Server(g, k, seed, workers=args.serve_workers, max_slots=args.serve_slots, keep_open_mask=True,
                       schedule=sched)
    clocks = Clocks(local)
    clocks.start()
    t0 = time.perf_counter()
    for q, ta in zip(qs, arrivals):
        delay = t0 + ta - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        srv.submit(q)
    t_end = t0 + warm + dur
    for q in qs:
        q._done.wait()
    t_drain = time.perf_counter()
    clk = clocks.stop()
    srv.close()
    measured = [q for q, ta in zip(qs, arrivals) if ta >= warm]
    served = [q for q in measured if q.error is None]
    done_in_window = [q for q in served if q.t_done <= t_end]
    lat = serve.latency_summary(served)
    batch_sizes = [q.batch_size for q in served]

    # the same queries run plain, one fl_* sequence at a time (a bounded prefix)
    plain_q = measured[:args.serve_plain]
    t_plain = []
    mask = torch.empty(n, dtype=torch.uint8, device=dev)
    cost_d = torch.empty(n, dtype=torch.float64, device=dev)
    open_d = torch.empty(n, dtype=torch.uint8, device=dev)
    same = True
    for q in plain_q:
        torch.cuda.synchronize()
        ts = time.perf_counter()
        cost_d.fill_(q.cost)
        serve.client_mask_on_device(torch, n, q.client_seed, q.client_frac, dev, mask)
        s = fl.Solve(g)
        s.compute_radii(cost_d, mask)
        _, no = s.open_facilities(open_d)
        s.assign_clients()
        obj = s.objective()[0]
        op_h = open_d.cpu().numpy()
        s.close()
        t_plain.append(time.perf_counter() - ts)
        if q.error is None:
            same = same and no == q.result["n_open"] and np.array_equal(op_h, q.result["open"]) and \
                abs(obj - q.result["objective"]) <= 1e-9 * abs(obj)
    g.close()
    line = {"metric": METRIC, "value": len(done_in_window) / dur, "unit": "solves/s", "n_gpus": 1,
            "steps": len(measured), "warmup": len(qs) - len(measured), "ms_per_step": lat.get("mean_ms"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": f"serve: resident R-MAT scale {scale} (n={n}, nnz={len(cols)}), k={k}",
                       "arrivals": f"Poisson {rate} req/s, {warm} s warm-up + {dur} s measured",
                       "query": "clients: each vertex with probability m/n, m log-uniform in [1e3, 1e6]; "
                                "every vertex a facility, one cost log-uniform in [10, 1000]",
                       "workers": args.serve_workers, "slots_per_worker": srv.slots,
                       "max_pending": srv.max_pending, "admission": "per query, by free device memory",
                       "waited_for_memory": srv.waited_for_memory, "schedule": sched, "autotune": tune},
            "latency_ms": {"p50": lat.get("p50_ms"), "p99": lat.get("p99_ms"), "mean": lat.get("mean_ms"),
                           "max": lat.get("max_ms")},
            "offered": len(measured), "served": len(served), "refused": srv.rejected,
            "served_in_window": len(done_in_window), "drain_s": t_drain - t_end,
            "mean_batch": float(np.mean(batch_sizes)) if batch_sizes else None,
            "plain": {"queries": len(plain_q), "solves_per_sec": len(t_plain) / sum(t_plain) if t_plain else None,
                      "p50_ms": float(np.percentile(t_plain, 50) * 1e3) if t_plain else None,
                      "form": "one fl_* sequence per query, back to back"},
            "identical_to_plain": bool(same), "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_eps(args):
    """The opening phase with eps > 0 (Algorithms 3-6) on the R-MAT scale-20
    workload (k = 32, costs log-uniform in [5, 500], every vertex a client
    and a facility): solves/s of fl_open_facilities_eps + assignment +
    objective for eps in {0.01, 0.1, 1} (sketches built once beforehand),
    beside the eps -> 0 path on the same instance, and the oracle's time for
    eps = 1 on the host cores."""
    import torch

    import paper_1503_03635_gb300 as fl

    if env_int("RANK", 0) != 0:
        return 0
    local = env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fl.load()
    w = flsynth.config("rmat20")
    stream = torch.cuda.Stream(device=dev)
    g = fl.Graph(torch.from_numpy(w.rowp).to(dev), torch.from_numpy(w.cols).to(dev), stream=stream)
    g.build_sketches(w.k, w.seed)
    cost_d = torch.from_numpy(w.cost).to(dev)
    client_d = torch.from_numpy(w.client).to(dev)
    open_d = torch.empty(w.n, dtype=torch.uint8, device=dev)
    fi_d = torch.empty(w.n, dtype=torch.int32, device=dev)
    ci_d = torch.empty(w.n, dtype=torch.int32, device=dev)
    asg_d = torch.empty(w.n, dtype=torch.int32, device=dev)
    dist_d = torch.empty(w.n, dtype=torch.int32, device=dev)
    radii_d = torch.empty(w.n, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    rows = []
    clocks = Clocks(local)
    clocks.start()
    for eps in (0.01, 0.1, 1.0):
        s = fl.Solve(g)
        out = {}

        def one():
            _, out["n_open"], _, _ = s.open_facilities_eps(eps, cost_d, client_d, open_d, fi_d, ci_d)
            s.assign_clients(asg_d, dist_d)
            out["objective"] = s.objective()[0]

        ms = timed(one)
        rows.append({"eps": eps, "ms_per_solve": ms, "solves_per_sec": 1e3 / ms, "n_open": out["n_open"],
                     "objective": out["objective"], **s.eps_stats()})
        s.close()
    s = fl.Solve(g)
    out = {}

    def limit():
        s.compute_radii(cost_d, client_d, radii_d)
        _, out["n_open"] = s.open_facilities(open_d)
        s.assign_clients(asg_d, dist_d)
        out["objective"] = s.objective()[0]

    ms0 = timed(limit)
    s.close()
    clk = clocks.stop()
    g.close()
    cpu = None
    small = None
    if not args.no_cpu_baseline:
        # a bounded sample: the 10^4-vertex ER workload at eps = 1, on the
        # host cores (the oracle evaluates every iteration of the grid) and on
        # the GPU
        import oracle

        we = flsynth.config("er10k")
        og = oracle.Graph(we.rowp, we.cols)
        og.build_sketches(we.k, we.seed)
        t0 = time.perf_counter()
        o = og.eps_open(1.0, we.cost, we.client)
        og.eps_select(1.0, o["alpha0"], o["fac_iter"], o["cli_iter"], we.seed)
        t = time.perf_counter() - t0
        og.close()
        cpu = {"value": 1.0 / t, "unit": "solves/s", "cores": oracle.threads(), "kind": "oracle",
               "sample": f"oracle opening phase and selection, eps = 1, on the er10k workload: {t:.3f} s "
                         f"({o['iterations']} iterations, every one evaluated)"}
        ge = fl.Graph(we.rowp, we.cols)
        ge.build_sketches(we.k, we.seed)
        se = fl.Solve(ge)
        se.open_facilities_eps(1.0, we.cost, we.client)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            se.open_facilities_eps(1.0, we.cost, we.client)
        small = {"workload": "er10k, eps = 1, host arrays", "gpu_ms_per_solve": (time.perf_counter() - t0) / 5 * 1e3,
                 "oracle_ms_per_solve": t * 1e3}
        se.close()
        ge.close()
    line = {"metric": METRIC, "value": rows[1]["solves_per_sec"], "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": rows[1]["ms_per_solve"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "eps: opening phase with eps > 0 on rmat20", "n": w.n, "nnz": w.nnz, "k": w.k,
                       "value_is": "eps = 0.1",
                       "step": "fl_open_facilities_eps + assignment + objective (sketches built once)"},
            "by_eps": rows,
            "eps_to_zero": {"ms_per_solve": ms0, "n_open": out["n_open"], "objective": out["objective"],
                            "form": "fl_compute_radii + fl_open_facilities + assignment + objective"},
            "cpu_baseline": cpu, "same_instance_gpu_vs_oracle": small, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_weighted(args):
    """Weighted graphs (Section 3.3 after Algorithm 2; weights uniform in
    [1, 100] as in Section 5): the whole path on the rmat20 graph with edge
    lengths from flsynth.edge_weights (k = 16, the rmat20 costs and clients),
    device-resident inputs: the ADS build in Dijkstra order, the radii, the
    greedy MIS with balls by weighted distance, the assignment and the
    objective.  Value: ADS entries per second of the step.  The oracle's
    definitional build (one Dijkstra per vertex) on a 2000-vertex ER graph is
    the CPU baseline."""
    import torch

    import paper_1503_03635_gb300 as fl

    if env_int("RANK", 0) != 0:
        return 0
    local = env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fl.load()
    w = flsynth.config("rmat20")
    k = 16
    lengths = flsynth.edge_weights(w.rowp, w.cols, 5)
    stream = torch.cuda.Stream(device=dev)
    g = fl.Graph(torch.from_numpy(w.rowp).to(dev), torch.from_numpy(w.cols).to(dev), stream=stream,
                 lengths=torch.from_numpy(lengths).to(dev))
    cost_d = torch.from_numpy(w.cost).to(dev)
    client_d = torch.from_numpy(w.client).to(dev)
    radii_d = torch.empty(w.n, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()

    open_d = torch.empty(w.n, dtype=torch.uint8, device=dev)
    assign_d = torch.empty(w.n, dtype=torch.int32, device=dev)
    dist_d = torch.empty(w.n, dtype=torch.int32, device=dev)
    out = {}

    def step():
        g.build_sketches(k, w.seed)
        s = fl.Solve(g)
        s.compute_radii(cost_d, client_d, radii_d)
        _, out["n_open"] = s.open_facilities(open_d)
        s.assign_clients(assign_d, dist_d)
        out["objective"] = s.objective()
        out["mis"] = s.stats()
        log = s.mis_log()
        out["largest_ball"] = int(log[log[:, 1] == 3][:, 2].max()) if len(log) else 0
        out["sweep_steps"] = int(log[log[:, 1] != 3][:, 3].sum()) if len(log) else 0
        out["sweeps"] = {name: {"sweeps": int((log[:, 1] == kind).sum()),
                                "steps": int(log[log[:, 1] == kind][:, 3].sum()),
                                "host_ms": round(float(log[log[:, 1] == kind][:, 5].sum()) / 1e3, 3)}
                         for name, kind in (("cover", 0), ("gather", 1), ("kill", 4))} if len(log) else {}
        s.close()

    for _ in range(args.warmup):
        step()
    g.profile(True)
    g.profile_reset()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    st = g.stats()
    prof = {name: g.profile_query(name) for name in fl.PROF_CLASSES}
    launches = g.profile_query(-1)["launches"]
    g.close()
    cpu = None
    if not args.no_cpu_baseline:
        import oracle

        we = flsynth.small_er(2000, 6.0, 81)
        wl = flsynth.edge_weights(we.rowp, we.cols, 7)
        og = oracle.Graph(we.rowp, we.cols)
        og.set_weights(wl)
        t0 = time.perf_counter()
        og.build_sketches_weighted(k, 1)
        t = time.perf_counter() - t0
        entries = int(og.ads(ranks=False)["eofs"][-1])
        og.close()
        cpu = {"value": entries / t, "unit": "ADS entries/s", "cores": oracle.threads(), "kind": "oracle",
               "sample": f"oracle weighted build (a Dijkstra per vertex) of a 2000-vertex ER graph with lengths "
                         f"in [1, 100], k = 16: {entries} entries in {t:.3f} s"}
    line = {"metric": METRIC, "value": st["ads_entries"] / (ms / 1e3), "unit": "ADS entries/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "weighted: rmat20 with edge lengths uniform in [1, 100]", "n": w.n, "nnz": w.nnz,
                       "k": k, "step": "fl_build_sketches (weighted, Dijkstra order) + fl_compute_radii + "
                                        "fl_open_facilities + fl_assign_clients + fl_objective"},
            "ads_entries": st["ads_entries"], "ads_groups": st["ads_groups"], "largest_distance": st["hops"],
            "n_open": out["n_open"], "objective": out["objective"][0], "unserved": out["objective"][2],
            "mis_rounds": out["mis"]["mis_rounds"], "candidates": out["mis"]["candidates"],
            "largest_ball_radius": out["largest_ball"], "mis_sweep_steps": out["sweep_steps"],
            "mis_sweeps": out["sweeps"],
            "phases_ms_per_step": {kk: v["ms"] / args.steps for kk, v in prof.items()},
            "gpu_launches": launches, "cpu_baseline": cpu, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_quality(args):
    """Quality of the GPU path against the oracle's references (Section 5.2,
    Table 2 compares the method with a sequential local search).  Enumerable
    instances (24 ER graphs, 16 vertices): objective / optimum for the sketch
    radii with k = 4 and k = 32 (exact sketches at this size) and the
    exact-count radii.  Graphs of 1-2 thousand vertices (R-MAT scales 10, 11
    with the workloads' recipe; ER with average degree 10), all vertices
    clients and facilities, costs log-uniform [5, 500]: objective / the
    add/drop/swap local search from the cheapest facility, and that local
    search restarted from the GPU's k = 32 solution."""
    import oracle
    import paper_1503_03635_gb300 as fl

    if env_int("RANK", 0) != 0:
        return 0
    fl.load()
    tiny_n, max_moves = 24, 5000

    def ours(rowp, cols, k, cost, client, exact=False):
        g = fl.Graph(rowp, cols)
        g.build_sketches(k, 1)
        s = fl.Solve(g)
        (s.compute_radii_exact if exact else s.compute_radii)(cost, client)
        op, _ = s.open_facilities()
        s.assign_clients()
        obj = s.objective()[0]
        s.close()
        g.close()
        return op, obj

    def ours_eps(rowp, cols, k, eps, cost, client):
        r = fl.solve_eps(rowp, cols, k, 1, eps, cost, client)
        r["solve"].close()
        r["graph"].close()
        return r["objective"]

    t0 = time.perf_counter()
    modes = (("k4", 4, False), ("k32", 32, False), ("exact", 32, True))
    eps_modes = (("eps0.01", 0.01), ("eps0.1", 0.1), ("eps1", 1.0))
    tiny = {key: [] for key, _, _ in modes}
    tiny.update({key: [] for key, _ in eps_modes})
    for seed in range(tiny_n):
        w = flsynth.small_er(16, 2.2, 4000 + seed)
        cost = flsynth.loguniform(16, 4100 + seed, 0.5, 12.0)
        client = flsynth.bernoulli(16, 4200 + seed, 0.85)
        _, opt = oracle.Graph(w.rowp, w.cols).optimum(cost, client)
        for key, k, ex in modes:
            tiny[key].append(ours(w.rowp, w.cols, k, cost, client, ex)[1] / opt)
        for key, eps in eps_modes:
            tiny[key].append(ours_eps(w.rowp, w.cols, 32, eps, cost, client) / opt)
    table = []
    graphs = [("rmat10", flsynth.rmat(10, 16, 52)), ("rmat11", flsynth.rmat(11, 16, 53))]
    for n in (1000, 2000):
        w = flsynth.small_er(n, 10.0, 54 + n)
        graphs.append((f"er{n}", (w.rowp, w.cols)))
    for name, (rowp, cols) in graphs:
        n = len(rowp) - 1
        cost = flsynth.loguniform(n, 7, 5.0, 500.0)
        client = np.ones(n, np.uint8)
        orc = oracle.Graph(rowp, cols)
        _, ls, moves = orc.local_search(cost, client, max_moves=max_moves)
        row = {"graph": name, "n": n, "nnz": int(len(cols)), "local_search": ls, "local_search_moves": moves}
        for key, k, ex in modes:
            op, obj = ours(rowp, cols, k, cost, client, ex)
            row[key] = {"objective": obj, "vs_local_search": obj / ls}
            if key == "k32":
                _, ls2, _ = orc.local_search(cost, client, start=op, max_moves=max_moves)
                row["local_search_from_k32"] = ls2
        for key, eps in eps_modes:
            obj = ours_eps(rowp, cols, 32, eps, cost, client)
            row[key] = {"objective": obj, "vs_local_search": obj / ls}
        table.append(row)
    print(json.dumps({"workload": "quality", "seconds": time.perf_counter() - t0,
                      "vs_optimum": {"instances": f"{tiny_n} ER graphs, n = 16",
                                     **{key: {"mean": float(np.mean(v)), "max": float(np.max(v))}
                                        for key, v in tiny.items()}},
                      "vs_local_search": table}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    help="er10k, rmat20, rmat26 (the named workloads), batch (solves/s batched vs plain), "
                         "serve (Poisson query stream: p50/p99 latency, solves/s), "
                         "exact (exact neighbourhood sizes, ADS accuracy vs k, exact-count radii), "
                         "quality (objective against the optimum and a local search), "
                         "eps (the opening phase with eps > 0), weighted (the weighted ADS build and radii) "
                         "or rmatS for the rmat20 recipe at scale S")
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default schedule (no tuning pass)")
    ap.add_argument("--tune-trials", type=int, default=15, help="timed schedules of the autotuner, at most")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: Poisson arrival rate (req/s)")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="serve: measured seconds")
    ap.add_argument("--serve-warmup", type=float, default=5.0, help="serve: warm-up seconds")
    ap.add_argument("--serve-scale", type=int, default=23, help="serve: R-MAT scale of the resident graph")
    ap.add_argument("--serve-plain", type=int, default=20, help="serve: queries also run plain")
    ap.add_argument("--serve-workers", type=int, default=4, help="serve: worker threads (streams)")
    ap.add_argument("--serve-slots", type=int, default=2, help="serve: most queries per batch solve")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gpu":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "exact":
        return run_exact(args)
    if args.workload == "quality":
        return run_quality(args)
    if args.workload == "eps":
        return run_eps(args)
    if args.workload == "weighted":
        return run_weighted(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
