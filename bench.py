#!/usr/bin/env python
"""Benchmark: exact butterfly counting on one GB300 (or N replicas).

One step = the whole counting path over one synthetic graph:
  pb_graph_from_edges (device-resident edge list: dedupe + CSR)
  -> pb_rank (PREPROCESS: ranking, relabelling, adjacency by decreasing rank,
     deg_x(y), wedge work split)
  -> pb_count_all (wedge retrieval + aggregation; global, per-vertex and
     per-edge counts in one pass)
Metric: wedges aggregated per second, W / step time, where W is the exact
number of wedges the ranking retrieves (Algorithm 2).  Counts are exact uint64.

Default workload: the largest single-GPU configuration, a Chung-Lu
bipartite graph |U|=20M, |V|=60M, m=300M distinct edges, expected-degree
exponent 2.0 on both sides (capped at 1e5), degree ranking, exact global and
per-edge counts, batch aggregation (simple batching) within a 16 GiB scratch
budget.  `--workload cl2` selects the 1M x 4M graph (all outputs, automatic
aggregation).

Multi-GPU (torchrun): every rank counts its own replica of the workload (the
path has no exchange step), so per-GPU work is fixed: weak scaling, value =
N * W / max-over-ranks time.

--impl reference times the CPU oracle (the plain implementation the tests
check against) on the host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "wedges aggregated/sec and % HBM roofline, exact counts; batched/served p50/p99 vs plain"
UNIT = "wedges/s"

# Each workload with the counting configuration it is measured in (ranking,
# aggregation, outputs, scratch budget); command-line options override them.
WORKLOADS = {
    "er1": dict(desc="ER |U|=2000 |V|=3000 m=2e4", idx=1, agg="hash", outputs="vertex", scratch=0),
    "cl2": dict(desc="Chung-Lu |U|=1M |V|=4M m=5e7, exponents 2.1/2.5, cap 1e5", idx=2, agg="auto",
                outputs="all", scratch=0),
    "cl3": dict(desc="Chung-Lu |U|=20M |V|=60M m=3e8, exponents 2.0/2.0, cap 1e5", idx=3, agg="batch",
                outputs="edge", scratch=16 << 30),
    # quarter-scale copy of cl2 for profiler captures (a few GB on the device)
    "cl2s": dict(desc="Chung-Lu |U|=250k |V|=1M m=1.25e7, exponents 2.1/2.5, cap 1e5", idx=-2, agg="auto",
                 outputs="all", scratch=0),
    # 1/16-scale copy of cl3 for profiler captures (same recipe and counting configuration)
    "cl3s": dict(desc="Chung-Lu |U|=1.25M |V|=3.75M m=1.875e7, exponents 2.0/2.0, cap 1e5", idx=-3, agg="batch",
                 outputs="edge", scratch=1 << 30),
}
# CPU samples of each workload for the oracle: the same generator recipe at a
# reduced scale.  "baseline" is the cpu_baseline of the GPU line (about 10-30 s
# of oracle time on the host cores); "step" is one step of the reference arm,
# small enough that warm-up plus timed steps end within a few minutes.
SAMPLES = {
    "er1": dict(baseline=dict(kind="er", nU=2000, nV=3000, m=20000),
                step=dict(kind="er", nU=2000, nV=3000, m=20000)),
    "cl2": dict(baseline=dict(kind="cl", nU=400_000, nV=1_600_000, m=20_000_000, gu=2.1, gv=2.5, cap=1e5),
                step=dict(kind="cl", nU=200_000, nV=800_000, m=10_000_000, gu=2.1, gv=2.5, cap=1e5)),
    "cl3": dict(baseline=dict(kind="cl", nU=1_200_000, nV=3_600_000, m=18_000_000, gu=2.0, gv=2.0, cap=1e5),
                step=dict(kind="cl", nU=400_000, nV=1_200_000, m=6_000_000, gu=2.0, gv=2.0, cap=1e5)),
    "cl2s": dict(baseline=dict(kind="cl", nU=200_000, nV=800_000, m=10_000_000, gu=2.1, gv=2.5, cap=1e5),
                 step=dict(kind="cl", nU=100_000, nV=400_000, m=5_000_000, gu=2.1, gv=2.5, cap=1e5)),
    "cl3s": dict(baseline=dict(kind="cl", nU=1_200_000, nV=3_600_000, m=18_000_000, gu=2.0, gv=2.0, cap=1e5),
                 step=dict(kind="cl", nU=400_000, nV=1_200_000, m=6_000_000, gu=2.0, gv=2.0, cap=1e5)),
}

# Algorithmic bytes per wedge of a pass producing global, per-vertex and
# per-edge counts: 4 B to read the second endpoint, and an 8 B read + 8 B write
# of the per-edge counter it updates ("streaming, no reuse" model).
BYTES_PER_WEDGE = {"all": 20, "edge": 20, "global": 4, "vertex": 8}
OUTPUT_DESC = {"all": "global+per-vertex+per-edge", "edge": "global+per-edge", "global": "global",
               "vertex": "global+per-vertex"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--mode", default="plain", choices=["plain", "batched", "serving", "noalloc"],
                    help="plain: one graph per step (default); batched: 1,024 graphs in one CUDA-graph launch "
                         "vs one launch per graph; serving: Poisson request stream")
    ap.add_argument("--graphs", type=int, default=1024)
    ap.add_argument("--workload", default="cl3", choices=sorted(WORKLOADS))
    ap.add_argument("--rank", default="degree", choices=["side", "degree", "approx_degree", "complement_degeneracy",
                                                        "approx_complement_degeneracy"])
    ap.add_argument("--agg", default=None, choices=["sort", "hash", "hist", "batch", "auto"],
                    help="wedge aggregation (default: the workload's)")
    ap.add_argument("--outputs", default=None, choices=["all", "edge", "global", "vertex"],
                    help="counts produced (default: the workload's)")
    ap.add_argument("--scratch-gib", type=float, default=None,
                    help="aggregation scratch budget in GiB (default: the workload's; 0 = library default)")
    ap.add_argument("--cpu-sample", default="bounded", choices=["bounded", "full"],
                    help="cpu_baseline on the bounded sample (default) or on the full workload graph")
    ap.add_argument("--retrieval", default="auto", choices=["low", "high", "auto"])
    ap.add_argument("--butterfly", default="atomic", choices=["atomic", "sort"],
                    help="butterfly aggregation: atomic adds or sort re-aggregation (needs --agg sort)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    if args.agg is None:
        args.agg = wl["agg"]
    if args.outputs is None:
        args.outputs = wl["outputs"]
    args.scratch = wl["scratch"] if args.scratch_gib is None else int(args.scratch_gib * (1 << 30))
    return args


# ---------------------------------------------------------------------------
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi samples every 200 ms while running."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, enabled: bool = True):
        self.index, self.enabled, self.proc, self.lines = index, enabled, None, []

    def __enter__(self):
        if self.enabled:
            try:
                self.proc = subprocess.Popen(
                    ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                     "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
                self.t = threading.Thread(target=self._read, daemon=True)
                self.t.start()
            except OSError:
                self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, val in zip(names, f[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def measured_traffic(workload: str, phase: str, wedges_per_launch: float):
    """DRAM bytes per launch of the tier kernel of `phase` from the committed
    ncu capture of this workload (or of its reduced-scale copy), scaled by
    wedges; None when no capture covers it or the kernel source has changed
    since the capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
    except Exception:
        return None
    for cap in t.get("captures", []):
        if workload not in (cap.get("workload"), cap.get("scales_to")):
            continue
        k = cap.get("kernels", {}).get(phase)
        if k is None:
            continue
        try:
            with open(os.path.join(ROOT, cap["source_file"]), "rb") as f:
                sha = hashlib.sha256(f.read()).hexdigest()
        except OSError:
            continue
        if sha == cap.get("source_sha256"):
            return k["dram_bytes_per_wedge"] * wedges_per_launch
    return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
def _sample_graph(workload: str, which: str):
    import synth
    if which == "full":
        return synth.workload(WORKLOADS[workload]["idx"]), f"the full {WORKLOADS[workload]['desc']} graph"
    sp = SAMPLES[workload][which]
    seed = synth.SEED_BASE + 100 + WORKLOADS[workload]["idx"]
    if sp["kind"] == "er":
        g = synth.er_graph(seed, sp["nU"], sp["nV"], sp["m"])
    else:
        g = synth.chung_lu_graph(seed, sp["nU"], sp["nV"], sp["m"], sp["gu"], sp["gv"], cap_u=sp["cap"],
                                 cap_v=sp["cap"])
    return g, f"{sp['kind']} |U|={sp['nU']} |V|={sp['nV']} m={sp['m']} (same recipe, reduced scale)"


def cpu_baseline(workload: str, nthreads: int | None = None, which: str = "baseline", outputs: str | None = None,
                 rank: str = "degree") -> dict:
    """The oracle as it stands, on a sample of the workload ("baseline":
    bounded sample for the GPU line; "step": one reference-arm step; "full":
    the workload graph itself).  Dedupe, PREPROCESS and counting are timed."""
    import oracle
    outputs = outputs or WORKLOADS[workload]["outputs"]
    g, gdesc = _sample_graph(workload, which)
    threads = nthreads or oracle.threads()
    pv = outputs in ("all", "vertex")
    pe = outputs in ("all", "edge")
    t0 = time.perf_counter()
    c = oracle.count(g.nU, g.nV, g.u, g.v, kind=rank, per_vertex=pv, per_edge=pe, nthreads=threads)
    dt = time.perf_counter() - t0
    desc = f"{gdesc}, {rank} ranking, {OUTPUT_DESC[outputs]}, dedupe+preprocess+count timed, W={c.W}"
    return {"value": c.W / dt, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc,
            "seconds": dt, "W": c.W}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        cpu_baseline(args.workload, which="step", outputs=args.outputs, rank=args.rank)
    vals, secs = [], []
    for _ in range(args.steps):
        r = cpu_baseline(args.workload, which="step", outputs=args.outputs, rank=args.rank)
        vals.append(r["value"])
        secs.append(r["seconds"])
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["desc"], "sample": r["sample"], "rank": args.rank,
                       "outputs": OUTPUT_DESC[args.outputs]},
            "cpu_baseline": {"kind": "oracle", "cores": r["cores"], "sample": r["sample"], "value": value,
                             "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
def run_gb300(args):
    import numpy as np
    import torch

    import synth
    import paper_1907_08607_gb300 as pb
    from paper_1907_08607_gb300 import build as pbuild

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    pbuild.build()
    pb.load_library()

    # CPU baseline first (host threads only, before heavy GPU work).
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, which="baseline" if args.cpu_sample == "bounded" else "full",
                           outputs=args.outputs, rank=args.rank)

    g = synth.workload(WORKLOADS[args.workload]["idx"])
    du = torch.from_numpy(g.u.view(np.int32)).to(dev)
    dv = torch.from_numpy(g.v.view(np.int32)).to(dev)
    want_v = args.outputs in ("all", "vertex")
    want_e = args.outputs in ("all", "edge")
    outs = {}
    if want_v:
        outs["U"] = torch.empty(g.nU, dtype=torch.int64, device=dev)
        outs["V"] = torch.empty(g.nV, dtype=torch.int64, device=dev)
    if want_e:
        outs["E"] = torch.empty(g.m, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()

    state = {}

    def step():
        G = pb.Graph.from_edges(g.nU, g.nV, du, dv)
        G.rank(args.rank)
        G.set_retrieval(args.retrieval).set_butterfly_aggregation(args.butterfly)
        c = G.count_all(args.agg, scratch_bytes=args.scratch, on_device=True, out=outs, vertex=want_v,
                        edge=want_e)
        state["W"] = G.wedges
        state["global"] = c.global_count
        G.free()

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    # the L2 atomic ceiling for the roofline (a few ms, before the timed region)
    try:
        atomics_peak = pb.calibrate_atomics(False)
    except Exception:
        atomics_peak = None

    # ---- timed region: device-resident inputs
    pb.profile(enable=True, reset=True)
    l0 = pb.kernel_launches()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(dev, enabled=not args.no_clocks) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms_total = ev0.elapsed_time(ev1)
    launches = pb.kernel_launches() - l0
    prof = pb.profile(enable=False)
    if dist is not None:
        t = torch.tensor([ms_total], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    W = state["W"]
    value = world * W / (ms_step / 1e3)

    # ---- end to end through host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        # Page-locked buffers allocated as such and touched once: on the GPU
        # box, pinned copies of pageable tensors (.pin_memory()) ran at 50-60
        # GB/s even when warm, these at 190-210 GB/s.
        def pinned(n, dtype, src=None):
            t = torch.empty(n, dtype=dtype, pin_memory=True)
            if src is not None:
                t.copy_(torch.from_numpy(src))
            else:
                t.zero_()
            return t

        hu = pinned(g.m, torch.int32, g.u.view(np.int32))
        hv = pinned(g.m, torch.int32, g.v.view(np.int32))
        hout = {}
        if want_v:
            hout["U"] = pinned(g.nU, torch.int64)
            hout["V"] = pinned(g.nV, torch.int64)
        if want_e:
            hout["E"] = pinned(g.m, torch.int64)

        def step_host():
            G = pb.Graph.from_edges(g.nU, g.nV, hu, hv)
            G.rank(args.rank)
            G.set_retrieval(args.retrieval).set_butterfly_aggregation(args.butterfly)
            G.count_all(args.agg, scratch_bytes=args.scratch, on_device=False, out=hout, vertex=want_v,
                        edge=want_e)
            G.free()

        for _ in range(max(3, args.warmup)):
            step_host()
        barrier()
        torch.cuda.synchronize()
        pb.profile(enable=True, reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0 = time.perf_counter()
        e0.record(stream)
        for _ in range(args.steps):
            step_host()
        e1.record(stream)
        torch.cuda.synchronize()
        host_s = time.perf_counter() - h0
        barrier()
        eprof = pb.profile(enable=False)
        ems = e0.elapsed_time(e1)
        if dist is not None:
            t = torch.tensor([ems], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ems = float(t.item())
        e2e = {"value": world * W / (ems / args.steps / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": 8 * g.m,
               "d2h_bytes_per_step": 8 * ((g.nU + g.nV if want_v else 0) + (g.m if want_e else 0)) + 8,
               "ms_per_step": ems / args.steps,
               # where the end-to-end step goes: the library's phases (build
               # includes the upload, output the download) and the host clock
               "phases_ms_per_step": {k: v["ms"] / args.steps for k, v in eprof.items() if v["records"]},
               "host_ms_per_step": 1e3 * host_s / args.steps}

    # ---- roofline of the dominant kernel (CUDA events inside the library)
    kern = max(["light", "medium", "large", "heavy", "sort"], key=lambda k: prof[k]["ms"])
    kp = prof[kern]
    peak, peak_src = measured_peaks()
    roof = None
    if kp["records"] > 0 and kp["ms"] > 0:
        per_launch_ms = kp["ms"] / kp["records"]
        per_launch_bytes = BYTES_PER_WEDGE[args.outputs] * kp["wedges"] / kp["records"]
        achieved = per_launch_bytes / (per_launch_ms / 1e3) / 1e9
        traffic = measured_traffic(args.workload, kern, kp["wedges"] / kp["records"])
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": kern, "peak_source": peak_src,
                "launch_ms": per_launch_ms, "algorithmic_bytes_per_launch": per_launch_bytes}
        if traffic:  # the DRAM bytes the kernel moves (ncu), over the same launch time
            roof["traffic_gbs"] = traffic / (per_launch_ms / 1e3) / 1e9
            roof["traffic_frac"] = roof["traffic_gbs"] / peak
        # Second ceiling: the device's 64-bit L2 atomic-add throughput (measured
        # by the library's calibration kernel in this process).  Per-edge counts
        # take one counter update per wedge, per-vertex one per wedge (centre)
        # in the streaming model; global counts need none per wedge.
        if atomics_peak:
            per_wedge = {"all": 2, "edge": 1, "vertex": 1, "global": 0}[args.outputs]
            if per_wedge:
                ops = per_wedge * kp["wedges"] / kp["records"] / (per_launch_ms / 1e3)
                roof["l2_atomic"] = {"achieved_ops_per_s": ops, "peak_ops_per_s": atomics_peak,
                                     "frac": ops / atomics_peak, "updates_per_wedge": per_wedge,
                                     "peak_pattern": "coalesced 64-bit reductions, 32 consecutive counters per warp"}
        roof["l2_atomic_frac"] = roof.get("l2_atomic", {}).get("frac")

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    clocks = clk.summary() if not args.no_clocks else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload]["desc"], "rank": args.rank, "agg": args.agg,
                   "scratch_bytes": args.scratch or "library default (16 GiB)",
                   "retrieval": args.retrieval, "butterfly_aggregation": args.butterfly,
                   "outputs": OUTPUT_DESC[args.outputs], "W": W, "butterflies": state["global"],
                   "parallelism": f"replicas{world}",
                   "l2": f"inputs larger than L2 ({8 * g.m / 1e6:.0f} MB edge list)"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "phases_ms_per_step": {k: v["ms"] / args.steps for k, v in prof.items() if v["records"]},
        "phases_wedges_per_step": {k: v["wedges"] // args.steps for k, v in prof.items() if v["wedges"]},
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_serving(args):
    from paper_1907_08607_gb300 import serve
    print(json.dumps(serve.bench(args)), flush=True)
    return 0


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(round(q / 100.0 * (len(xs) - 1))))]


def run_batched(args):
    """Batched workload: graphs with m log-uniform in [1e3, 1e6], ER or
    Chung-Lu by coin flip, |V|/|U| log-uniform in [0.1, 10]; global + per-vertex
    counts.  Counting only (graphs built and ranked beforehand): one CUDA-graph
    launch for the whole batch vs one pb_count_all per graph."""
    import numpy as np
    import torch

    import synth
    import paper_1907_08607_gb300 as pb
    from paper_1907_08607_gb300 import build as pbuild

    torch.cuda.set_device(0)
    pbuild.build()
    pb.load_library()
    gs = [synth.batch_graph(i) for i in range(args.graphs)]
    Gs = []
    for g in gs:
        G = pb.Graph.from_edges(g.nU, g.nV, g.u, g.v).rank("degree")
        G.set_retrieval("auto")
        Gs.append(G)
    W = sum(G.wedges for G in Gs)
    outs = [{"U": torch.empty(G.nU, dtype=torch.int64, device="cuda"),
             "V": torch.empty(G.nV, dtype=torch.int64, device="cuda")} for G in Gs]
    stream = torch.cuda.current_stream()

    def plain_pass(lat=None):
        for G, o in zip(Gs, outs):
            t0 = time.perf_counter()
            G.count_all("auto", edge=False, on_device=True, out=o)
            if lat is not None:
                lat.append(time.perf_counter() - t0)

    B = pb.Batch(Gs, vertex=True)
    for _ in range(max(3, args.warmup)):
        plain_pass()
        B.run()
    torch.cuda.synchronize()
    lat = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plain_pass(lat)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1) / args.steps
    blat = []
    l0 = pb.kernel_launches()
    e0.record(stream)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        B.run()
        blat.append(time.perf_counter() - t0)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = pb.kernel_launches() - l0
    batch_ms = e0.elapsed_time(e1) / args.steps
    glob = B.globals()
    same = all(int(glob[i]) == G.count_global("auto") for i, G in enumerate(Gs[:64]))
    B.free()
    # The autotuner's per-graph choices, and the same batch with every graph
    # pinned to one fixed plan (no large tier, dense heavy slots: the plan
    # before per-graph tuning), timed the same way.
    plans = [G.autotune() for G in Gs]
    chosen = {}
    for p in plans:
        key = f"agg={p['agg']},med_max={p['med_max']},large_max={p['large_max']},hot={p['hot']}"
        chosen[key] = chosen.get(key, 0) + 1
    for G, p in zip(Gs, plans):
        G.set_plan(dict(p, agg="batch", light_max=768, med_max=4096, large_max=4096, hot=16384))
    Bf = pb.Batch(Gs, vertex=True)
    for _ in range(max(3, args.warmup)):
        Bf.run()
    e0.record(stream)
    for _ in range(args.steps):
        Bf.run()
    e1.record(stream)
    torch.cuda.synchronize()
    fixed_ms = e0.elapsed_time(e1) / args.steps
    same = same and all(int(a) == int(b) for a, b in zip(Bf.globals(), glob))
    Bf.free()
    for G in Gs:
        G.set_plan(None)
    line = {"metric": METRIC, "mode": "batched", "value": W / (batch_ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": batch_ms, "higher_is_better": True,
            "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"{args.graphs} graphs, m log-uniform [1e3,1e6], ER or Chung-Lu (gamma 1.8-2.8), "
                                   "|V|/|U| log-uniform [0.1,10]", "outputs": "global+per-vertex", "W": W,
                       "edges": int(sum(g.m for g in gs)), "rank": "degree", "agg": "auto (autotuned)"},
            "plain": {"value": W / (plain_ms / 1e3), "ms_per_pass": plain_ms,
                      "per_graph_latency_ms": {"p50": 1e3 * _pct(lat, 50), "p99": 1e3 * _pct(lat, 99)}},
            "batched_latency_ms": {"p50": 1e3 * _pct(blat, 50), "p99": 1e3 * _pct(blat, 99)},
            "speedup_vs_plain": plain_ms / batch_ms, "gpu_launches": launches,
            "autotuned_plans": chosen,
            "fixed_plan": {"value": W / (fixed_ms / 1e3), "ms_per_step": fixed_ms,
                           "plan": "light_max 768, med_max 4096, no large tier, dense heavy slots, hot 16384"},
            "speedup_vs_fixed_plan": fixed_ms / batch_ms,
            "results_equal_alone_and_in_batch": same}
    print(json.dumps(line), flush=True)
    for G in Gs:
        G.free()
    return 0


def noalloc_workload(workload: str) -> str:
    """The allocation-free entry point's scratch takes sides of at most
    16,777,184 vertices: the 20M x 60M default runs the 1M x 4M graph."""
    return "cl2" if workload == "cl3" else workload


def run_noalloc(args):
    """pb_count_noalloc, the allocation-free entry point, on caller-owned
    device buffers holding the library's own PREPROCESS output (global +
    per-vertex counts; a step is one call).  Its fixed scratch takes sides of
    at most 16,777,184 vertices, so the 20M x 60M default runs the 1M x 4M
    graph instead.  The counts are checked against the regular entry point."""
    import numpy as np
    import torch

    import synth
    import paper_1907_08607_gb300 as pb
    from paper_1907_08607_gb300 import build as pbuild

    torch.cuda.set_device(0)
    pbuild.build()
    pb.load_library()
    wl = noalloc_workload(args.workload)
    g = synth.workload(WORKLOADS[wl]["idx"])
    G = pb.Graph.from_edges(g.nU, g.nV, g.u, g.v).rank("degree")
    W, n = G.wedges, g.nU + g.nV
    L = G.layout()
    out_g = torch.zeros(1, dtype=torch.int64, device="cuda")
    out_pv = torch.zeros(n, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    call = lambda: pb.count_noalloc(n, g.nU, L["off"], L["adj"], L["cpos"], L["degp"], out_g, out_pv)  # noqa: E731
    for _ in range(max(3, args.warmup)):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = pb.kernel_launches()
    e0.record(stream)
    for _ in range(args.steps):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = pb.kernel_launches() - l0
    ms = e0.elapsed_time(e1) / args.steps
    ref = G.count_all("auto", vertex=True, edge=False)
    lab = L["label_of"].cpu().numpy().view(np.uint32).astype(np.int64)
    pv = out_pv.cpu().numpy().view(np.uint64)[lab]
    same = int(out_g.cpu().numpy().view(np.uint64)[0]) == ref.global_count and \
        np.array_equal(pv[:g.nU], ref.per_vertex_U) and np.array_equal(pv[g.nU:], ref.per_vertex_V)
    line = {"metric": METRIC, "mode": "noalloc", "value": W / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
            "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOADS[wl]["desc"], "outputs": "global+per-vertex", "W": W, "rank": "degree",
                       "step": "one pb_count_noalloc call on a preprocessed graph in caller-owned device memory"},
            "gpu_launches": launches, "results_equal_regular_entry_point": bool(same)}
    print(json.dumps(line), flush=True)
    G.free()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "batched":
        return run_batched(args)
    if args.mode == "serving":
        return run_serving(args)
    if args.mode == "noalloc":
        return run_noalloc(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
