#!/usr/bin/env python3
"""Benchmark: Jet refinement throughput (Medges/s) and partition time at k=64.

Workload: the 128^3 7-point mesh (2,097,152 vertices, 6,242,304 edges),
vertex weights U[1,4], edge weights U[1,10], k = 64, eps = 0.03, seed 1 —
the paper's artificial-mesh class (its 200^3 cube), generated synthetically.

A step is one jet_partition call: heavy-edge coarsening, greedy initial
partition and Jet refinement (Jetlp + Jetrw/Jetrs) on every level.  `value`
is refinement edges per second: sum over levels of (iterations x edges of
the level) divided by the refinement time (CUDA events on the library's
stream), with the graph resident in HBM.  `e2e` is the same numerator over
the time of jet_partition_host (host arrays in pinned memory; copies in).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU: the path does not shard (one graph per GPU); N ranks run N
independent replicas (weak scaling) and rank 0 prints one JSON line.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Jet refinement Medges/s & partition ms at k=64; cutsize vs CPU oracle"
UNIT = "Medges/s"
K_PARTS, EPS, SEED = 64, 0.03, 1
WORKLOAD = "grid3d 128x128x128 (7-point), vwgt U[1,4], adjwgt U[1,10], k=64, eps=0.03, seed=1"
FLUSH_BYTES = 512 << 20          # written between steps (L2 is 129 MB)
G3_WORKLOAD = ("rmat s22 (4,194,304 vertices, edge factor 16, a=.57 b=c=.19 d=.05, symmetrised, isolated vertices "
               "kept), unit weights, k=64, eps=0.03, seed=1")
PROFILES = os.path.join(ROOT, "profiles")


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing (debug runs)")
    p.add_argument("--no-g3", action="store_true", help="skip the R-MAT scale-22 workload (debug runs)")
    p.add_argument("--scale", type=int, default=128, help="mesh side (128 is the benchmark workload)")
    p.add_argument("--hostloop", action="store_true",
                   help="drive refinement iterations from the host (same kernels and launch configuration; "
                        "used for profiler launch lists)")
    p.add_argument("--no-pdl", action="store_true",
                   help="launch every refinement kernel after the previous one finishes (no programmatic "
                        "dependent launch); results are identical")
    p.add_argument("--grid-loop", action="store_true",
                   help="refine levels above the cluster threshold in one cooperative launch each "
                        "(grid barriers between phases) instead of the CUDA-graph loop; results are identical")
    p.add_argument("--cluster-max-n", type=int, default=None,
                   help="largest level refined by the one-cluster loop (library default if omitted; 0 = never)")
    p.add_argument("--kernel-probe", action="store_true",
                   help="run one profiled partition and report per-level select launches (profiler target)")
    p.add_argument("--probe-graph", choices=["mesh", "rmat22"], default="mesh",
                   help="with --kernel-probe: the mesh workload (--scale) or R-MAT scale 22")
    p.add_argument("--max-levels", type=int, default=None,
                   help="with --kernel-probe: at most this many levels (1 = refine the input graph only, so "
                        "that its first refinement kernels come after a few dozen launches: a profiler target)")
    p.add_argument("--rmat-k", type=int, default=None, help="with --sweep rmat: only this k")
    p.add_argument("--two-hop", action="store_true", help="with --sweep rmat: coarsen with two-hop matches")
    p.add_argument("--sweep", choices=["lp_versions", "batched", "rmat", "shapes"], default=None,
                   help="the Jetlp versions of the paper's component study and the phi trade-off, on the "
                        "mesh, power-law and large-grid workloads (one JSON line per run and a summary)")
    return p.parse_args(argv)


def workload_graph(scale):
    import graphgen
    return graphgen.grid3d(scale, scale, scale, vw=(1, 4), ew=(1, 10), seed=SEED)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------------------
# multi-process plumbing (torchrun): one replica per rank
# --------------------------------------------------------------------------
def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(ws, backend):
    if ws <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend=backend)
    return dist


def aggregate(units, seconds, extra_max=(), dist=None, device=None):
    """Whole-job throughput over ranks: (sum of units) / (max of seconds).
    Returns (total_units, max_seconds, [max of each extra value])."""
    if dist is None:
        return float(units), float(seconds), [float(x) for x in extra_max]
    import torch
    t = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    m = torch.tensor([float(seconds)] + [float(x) for x in extra_max], dtype=torch.float64, device=device)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return float(t.item()), float(m[0].item()), [float(x) for x in m[1:].tolist()]


def barrier(dist):
    if dist is not None:
        dist.barrier()


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="jet_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------
# the oracle (CPU baseline / reference arm): a bounded sample of refinement
# --------------------------------------------------------------------------
def oracle_sample(g, iters, repeats=1):
    """Oracle Jet refinement of the finest level, starting from the greedy
    initial partition of the whole mesh, capped at `iters` iterations.
    Returns (edge passes, seconds, iterations run)."""
    import oracle
    part0 = oracle.initial_partition(g, K_PARTS)
    opts = oracle.Options(max_iters=iters)
    units = secs = its = 0
    for _ in range(repeats):
        t0 = time.perf_counter()
        r = oracle.refine(g, K_PARTS, part0, eps=EPS, is_finest=True, seed=SEED, opts=opts, trace_cap=1)
        secs += time.perf_counter() - t0
        units += r.iters * g.m
        its += r.iters
    return units, secs, its


def run_reference(args):
    """The oracle as it stands, on one host core, on the same workload and
    metric: each timed step is one whole oracle partition of the mesh (every
    stage and level, about 8 s on a Grace core); value = its refinement edge
    passes / its refinement seconds, as in our arm.  Warm-up steps are one
    capped refinement iteration each (a CPU program has nothing to warm)."""
    ws, rank, _ = dist_info()
    if rank != 0:
        return 0
    import oracle
    g = workload_graph(args.scale)
    for _ in range(args.warmup):
        oracle_sample(g, 1)
    units = secs = 0.0
    per_step = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.partition(g, K_PARTS, EPS, SEED)
        per_step.append(time.perf_counter() - t0)
        units += r.stats["edge_iters"]
        secs += r.stats["sec_refine"]
    value = units / secs / 1e6 if secs > 0 else 0.0
    sample = ("oracle partition of the whole workload per step (coarsening, initial partition, refinement of "
              "every level), single thread")
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * statistics.mean(per_step), 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
           "data": "synthetic", "config": {"workload": WORKLOAD, "n": g.n, "m": g.m, "sample": sample,
                                           "same_config": True},
           "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
KERNEL_SOURCES = ("jet_refine.cu", "jet_phases.cuh", "jet_internal.cuh")


def kernel_source_hash():
    """Hash of the refinement kernels' sources (the profile summary is only
    used for the source it was captured on)."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2304_13194_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic_per_launch(kernel, workload_tag):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    profiles/<kernel>_<workload_tag>.txt, if it was taken on the current
    kernel sources (else None)."""
    try:
        kv = {}
        with open(os.path.join(PROFILES, f"{kernel}_{workload_tag}.txt")) as f:
            for line in f:
                if ":" in line:
                    a, b = line.split(":", 1)
                    kv[a.strip()] = b.strip()
        if kv.get("kernel_source_sha256_16") != kernel_source_hash():
            return None
        return int(float(kv["traffic_bytes_per_launch"]))
    except Exception:
        return None


def kernel_table(pst, names, peak):
    """Per refinement kernel over the whole partition, from the profiled run:
    launches, CUDA-event ms, share of the kernel time, algorithmic bytes and
    GB/s.  Returns (table, name of the kernel with the largest time)."""
    tot_ms = [0.0] * len(names)
    tot_b = [0] * len(names)
    tot_l = [0] * len(names)
    for lv in range(pst.levels):
        for i in range(len(names)):
            tot_ms[i] += pst.kern_ms[lv][i]
            tot_b[i] += pst.kern_bytes[lv][i]
            tot_l[i] += pst.kern_launches[lv][i]
    all_ms = sum(tot_ms) or 1.0
    table = {}
    for i, name in enumerate(names):
        if tot_l[i] == 0:
            continue
        gbs = tot_b[i] / (tot_ms[i] / 1e3) / 1e9 if tot_ms[i] > 0 else 0.0
        table[name] = {"launches": tot_l[i], "ms": round(tot_ms[i], 3), "share": round(tot_ms[i] / all_ms, 4),
                       "bytes": tot_b[i], "gbs": round(gbs, 1), "frac": round(gbs / peak, 4)}
    top = max(table, key=lambda k: table[k]["ms"])
    return table, top


def roofline_of(table, top, peak, peak_kind, workload_tag):
    t = table[top]
    return {"bound": "hbm", "kernel": top, "achieved": t["gbs"], "peak": peak, "peak_kind": peak_kind,
            "unit": "GB/s", "frac": t["frac"], "traffic": ncu_traffic_per_launch(top, workload_tag),
            "bytes_per_launch": int(t["bytes"] / max(t["launches"], 1)),
            "ms_per_launch": round(t["ms"] / max(t["launches"], 1), 5), "launches": t["launches"],
            "time_share": t["share"],
            "how": "algorithmic bytes of the kernel's launches (byte model of jet_stats.kern_bytes) / their "
                   "CUDA-event time on the library stream, host-driven loop with the same kernels and launch "
                   "configuration (JET_FLAG_PROFILE)"}


def run_probe(args):
    """One profiled partition (CUDA events around every refinement kernel) of
    the mesh workload, or of R-MAT scale 22 with --probe-graph rmat22; prints
    per-level kernel times (a target for profiler launch lists)."""
    import torch
    import paper_2304_13194_gb300 as jet
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    if args.probe_graph == "rmat22":
        import graphgen
        g = graphgen.rmat(22, seed=SEED)
        t = [torch.from_numpy(g.xadj).to(dev), torch.from_numpy(g.adjncy).to(dev), None, None]
    else:
        g = workload_graph(args.scale)
        t = [torch.from_numpy(a).to(dev) for a in (g.xadj, g.adjncy, g.vwgt, g.adjwgt)]
    copts = {} if args.max_levels is None else {"max_levels": args.max_levels}
    with jet.Context(0, flags=jet.FLAG_PROFILE, **copts) as ctx:
        _, cut, st = ctx.partition(*t, k=K_PARTS, eps=EPS, seed=SEED, return_stats=True)
    skip = sum(st.sel_launches[1:])
    names = jet.kernel_names()
    per_level = [{nm: [lv_l[i], round(lv_ms[i], 4)] for i, nm in enumerate(names) if lv_l[i]}
                 for lv_l, lv_ms in zip(st.kern_launches, st.kern_ms)]
    print(json.dumps({"probe": "kernels", "cut": cut, "levels": st.levels, "n": st.n, "kernels_per_level": per_level,
                      "iters": [a + b + c for a, b, c in zip(st.iters_lp, st.iters_rw, st.iters_rs)],
                      "ms_level": [round(x, 3) for x in st.ms_level], "sel_launches": st.sel_launches,
                      "sel_ms": [round(x, 4) for x in st.sel_ms], "sel_bytes": st.sel_bytes,
                      "skip_before_finest": skip}), flush=True)
    return 0


def run_ours(args):
    import torch
    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    dist = dist_init(ws, "nccl")
    device = torch.device("cuda", local)
    import paper_2304_13194_gb300 as jet

    g = workload_graph(args.scale)
    xadj = torch.from_numpy(g.xadj).to(device)
    adj = torch.from_numpy(g.adjncy).to(device)
    vw = torch.from_numpy(g.vwgt).to(device)
    ew = torch.from_numpy(g.adjwgt).to(device)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=device)
    copts = {} if args.cluster_max_n is None else {"cluster_max_n": args.cluster_max_n}
    pdl_off = jet.FLAG_NO_PDL if args.no_pdl else 0
    loop = (jet.FLAG_HOSTLOOP if args.hostloop else 0) | (jet.FLAG_GRID_LOOP if args.grid_loop else 0)
    ctx = jet.Context(local, flags=loop | pdl_off, **copts)
    stream = torch.cuda.current_stream(device)

    def step():
        return ctx.partition(xadj, adj, vw, ew, k=K_PARTS, eps=EPS, seed=SEED, return_stats=True)

    for _ in range(max(args.warmup, 0)):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    # ---- timed region: K device-resident partitions ----------------------
    sampler = ClockSampler(local)
    barrier(dist)
    torch.cuda.synchronize()
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats, cuts, parts = [], [], None
    for i in range(args.steps):
        flush.zero_()                          # evict L2 between steps (outside the step's events)
        ev[i][0].record(stream)
        part, cut, st = step()
        ev[i][1].record(stream)
        stats.append(st); cuts.append(cut); parts = part
    torch.cuda.synchronize()
    barrier(dist)
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    units = sum(s.edge_iters for s in stats)
    refine_s = sum(s.ms_refine for s in stats) / 1e3
    launches = sum(s.kernel_launches for s in stats)
    tot_units, max_refine_s, (max_step_ms,) = aggregate(units, refine_s, [statistics.mean(step_ms)], dist, device)
    value = tot_units / max_refine_s / 1e6

    # ---- end to end through the host-pointer entry point -----------------
    hx = torch.from_numpy(g.xadj).pin_memory(); ha = torch.from_numpy(g.adjncy).pin_memory()
    hv = torch.from_numpy(g.vwgt).pin_memory(); hw = torch.from_numpy(g.adjwgt).pin_memory()
    hp = torch.empty(g.n, dtype=torch.int32).pin_memory()
    ctx.partition_host(hx, ha, hv, hw, k=K_PARTS, eps=EPS, seed=SEED, part_out=hp)   # warm
    e2e_units = 0
    e2e_ev = []
    barrier(dist)
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, _, st = ctx.partition_host(hx, ha, hv, hw, k=K_PARTS, eps=EPS, seed=SEED, part_out=hp, return_stats=True)
        b.record(stream)
        e2e_units += st.edge_iters
        e2e_ev.append((a, b))
    torch.cuda.synchronize()
    e2e_s = sum(a.elapsed_time(b) for a, b in e2e_ev) / 1e3
    e2e_tot, e2e_max, _ = aggregate(e2e_units, e2e_s, [], dist, device)
    h2d = g.xadj.nbytes + g.adjncy.nbytes + g.vwgt.nbytes + g.adjwgt.nbytes
    d2h = g.n * 4

    # ---- per-kernel CUDA-event times (profiling mode drives the same kernels
    # with the same launch configuration from the host); the roofline names
    # the kernel with the largest share of the time ---------------------------
    peak, peak_kind = peaks()
    names = jet.kernel_names()
    pctx = jet.Context(local, flags=jet.FLAG_PROFILE | pdl_off)
    flush.zero_()
    _, pcut, pst = pctx.partition(xadj, adj, vw, ew, k=K_PARTS, eps=EPS, seed=SEED, return_stats=True)
    pctx.close()
    table, top = kernel_table(pst, names, peak)
    st0 = stats[-1]
    refine_gbs = st0.bytes_model / (st0.ms_refine / 1e3) / 1e9

    # ---- CPU baseline: the oracle over the same stages (rank 0, N = 1) ------
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_partition_baseline(g, K_PARTS, SEED)

    # ---- the power-law workload (R-MAT scale 22, k = 64) --------------------
    g3 = None
    if not args.no_g3 and ws == 1:
        g3 = run_g3(args, jet, device, stream, flush, loop | pdl_off, copts, peak, peak_kind, names, rank == 0)

    if rank == 0:
        out = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(max_step_ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": g.n, "m": g.m, "k": K_PARTS, "eps": EPS, "seed": SEED,
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "l2": f"{FLUSH_BYTES >> 20} MB buffer written before every step",
                       "levels": st0.levels, "cut": cuts[-1], "max_part_w": st0.max_part_w,
                       "refine_ms": round(st0.ms_refine, 3), "coarsen_ms": round(st0.ms_coarsen, 3),
                       "initpart_ms": round(st0.ms_init, 3), "finest_refine_ms": round(st0.ms_refine_finest, 3),
                       "edge_iters_per_step": st0.edge_iters, "bytes_model_per_step": st0.bytes_model,
                       "ms_level": [round(x, 3) for x in st0.ms_level],
                       "iters_level": [a + b + c for a, b, c in zip(st0.iters_lp, st0.iters_rw, st0.iters_rs)],
                       "cluster_blocks": st0.cluster_blocks},
            "roofline": roofline_of(table, top, peak, peak_kind, "grid3d_128_k64"),
            "roofline_refine": {"bound": "hbm", "achieved": round(refine_gbs, 1), "peak": peak,
                                "peak_kind": peak_kind, "unit": "GB/s", "frac": round(refine_gbs / peak, 4),
                                "how": "algorithmic bytes of every refinement kernel of one partition "
                                       "(jet_stats.bytes_model) / the refinement time of the timed steps "
                                       "(CUDA-graph loop)"},
            "kernels": table,
            "cpu_baseline": cpu,
            "e2e": {"value": round(e2e_tot / e2e_max / 1e6, 3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clocks,
            "step_ms": [round(x, 3) for x in step_ms],
            "refine_ms_steps": [round(s.ms_refine, 3) for s in stats],
            "g3": g3,
        }
        print(json.dumps(out), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def oracle_partition_baseline(g, k, seed):
    """The oracle's whole partition of the workload (coarsening, initial
    partition, refinement of every level: the same stages as a step), one
    run on one host core.  value = its refinement edge passes per second."""
    import oracle
    t0 = time.perf_counter()
    r = oracle.partition(g, k, EPS, seed)
    secs = time.perf_counter() - t0
    st = r.stats
    return {"value": round(st["edge_iters"] / st["sec_refine"] / 1e6, 3), "unit": UNIT, "cores": 1,
            "kind": "oracle", "partition_ms": round(1e3 * secs, 1),
            "refine_ms": round(1e3 * st["sec_refine"], 1), "coarsen_ms": round(1e3 * st["sec_coarsen"], 1),
            "initpart_ms": round(1e3 * st["sec_init"], 1), "cut": r.cut, "same_config": True,
            "sample": "oracle partition of the whole workload (all stages, every level), one run, single thread"}


def run_g3(args, jet, device, stream, flush, flags, copts, peak, peak_kind, names, with_cpu):
    """The power-law workload: R-MAT scale 22, unit weights, k = 64.  The
    same step, timing and flush as the mesh; its own per-kernel profile and
    rooflines.  Heavy-edge matching stalls at the first level, so the whole
    64M-edge graph is refined."""
    import torch
    import graphgen
    g = graphgen.rmat(22, seed=SEED)
    xadj = torch.from_numpy(g.xadj).to(device)
    adj = torch.from_numpy(g.adjncy).to(device)
    ctx = jet.Context(device.index, flags=flags, **copts)

    def step():
        return ctx.partition(xadj, adj, None, None, k=K_PARTS, eps=EPS, seed=SEED, return_stats=True)

    for _ in range(max(args.warmup, 0)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        _, cut, st = step()
        ev[i][1].record(stream)
        stats.append(st)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ctx.close()
    units = sum(s.edge_iters for s in stats)
    refine_s = sum(s.ms_refine for s in stats) / 1e3
    st0 = stats[-1]
    pctx = jet.Context(device.index, flags=jet.FLAG_PROFILE | (flags & jet.FLAG_NO_PDL))
    flush.zero_()
    _, _, pst = pctx.partition(xadj, adj, None, None, k=K_PARTS, eps=EPS, seed=SEED, return_stats=True)
    pctx.close()
    table, top = kernel_table(pst, names, peak)
    refine_gbs = st0.bytes_model / (st0.ms_refine / 1e3) / 1e9
    cpu = None
    if with_cpu and not args.no_cpu_baseline:
        import oracle
        iters = 2
        part0 = oracle.initial_partition(g, K_PARTS)
        t0 = time.perf_counter()
        r = oracle.refine(g, K_PARTS, part0, eps=EPS, is_finest=True, seed=oracle.level_seed(SEED, 0),
                          opts=oracle.Options(max_iters=iters), trace_cap=1)
        secs = time.perf_counter() - t0
        cpu = {"value": round(r.iters * g.m / secs / 1e6, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"oracle Jet refinement of the whole graph (the only level) from the greedy initial "
                         f"partition, {r.iters} iterations ({secs:.1f} s), single thread"}
    del xadj, adj
    return {"workload": G3_WORKLOAD, "n": g.n, "m": g.m, "metric": METRIC, "unit": UNIT,
            "value": round(units / refine_s / 1e6, 3), "ms_per_step": round(statistics.mean(step_ms), 3),
            "refine_ms": round(st0.ms_refine, 3), "coarsen_ms": round(st0.ms_coarsen, 3),
            "initpart_ms": round(st0.ms_init, 3), "levels": st0.levels, "cut": cut, "max_part_w": st0.max_part_w,
            "edge_iters_per_step": st0.edge_iters, "bytes_model_per_step": st0.bytes_model,
            "roofline": roofline_of(table, top, peak, peak_kind, "rmat22_k64"),
            "roofline_refine": {"bound": "hbm", "achieved": round(refine_gbs, 1), "peak": peak,
                                "peak_kind": peak_kind, "unit": "GB/s", "frac": round(refine_gbs / peak, 4)},
            "kernels": table, "cpu_baseline": cpu}


# Jetlp versions of the component study (Sec. 6.1.4, Table 2) as library flags
LP_VERSIONS = [("baseline", "BASELINE_LP"), ("baseline+locks", "STRICT_GAIN|NO_AFTERBURN"),
               ("baseline+weak_afterburner", "WEAK_AFTERBURN|NO_LOCKS"), ("baseline+full_afterburner", "NO_LOCKS"),
               ("full_jetlp", "")]


def sweep_graphs():
    """Meshes, a power-law graph and the paper's two large synthetic grids."""
    import graphgen
    return [
        ("grid2d_64x64", lambda: graphgen.grid2d(64, 64), 8),
        ("grid3d_128", lambda: graphgen.grid3d(128, 128, 128, vw=(1, 4), ew=(1, 10), seed=SEED), 64),
        ("rmat_s22", lambda: graphgen.rmat(22, seed=SEED), 64),
        ("grid2d_2000x4000", lambda: graphgen.grid2d(2000, 4000), 64),
        ("grid3d_200", lambda: graphgen.grid3d(200, 200, 200), 64),
    ]


def run_sweep(args):
    import math
    import torch
    import paper_2304_13194_gb300 as jet
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    flag = lambda spec: sum(getattr(jet, "FLAG_" + f) for f in spec.split("|") if f)
    runs = [(name, flag(spec), 0.999) for name, spec in LP_VERSIONS] + [("phi_0.99", 0, 0.99), ("phi_0.9999", 0, 0.9999)]
    results = {}
    for gname, make, k in sweep_graphs():
        g = make()
        t = [torch.from_numpy(a).to(dev) if a is not None else None for a in (g.xadj, g.adjncy, g.vwgt, g.adjwgt)]
        for rname, flags, phi in runs:
            with jet.Context(0, flags=flags, phi=phi) as ctx:
                ctx.partition(*t, k=k, eps=EPS, seed=SEED)                       # warm-up
                _, cut, st = ctx.partition(*t, k=k, eps=EPS, seed=SEED, return_stats=True)
            results[(gname, rname)] = (cut, st.ms_refine, st.ms_total, st.max_part_w)
            print(json.dumps({"sweep": "lp_versions", "graph": gname, "n": g.n, "m": g.m, "k": k, "version": rname,
                              "phi": phi, "cut": cut, "uncoarsen_ms": round(st.ms_refine, 3),
                              "total_ms": round(st.ms_total, 3), "max_part_w": st.max_part_w}), flush=True)
        del t
    gnames = [x[0] for x in sweep_graphs()]

    def geo(rname, idx):
        return math.exp(sum(math.log(results[(gn, rname)][idx]) for gn in gnames) / len(gnames))
    base = geo("baseline", 0)
    summary = {"sweep": "lp_versions", "summary": "geomean(baseline cut) / geomean(version cut)",
               "ratios": {rname: round(base / geo(rname, 0), 4) for rname, _, _ in runs},
               "phi_vs_default": {r: {"uncoarsen_time": round(geo(r, 1) / geo("full_jetlp", 1), 3),
                                      "cut": round(geo(r, 0) / geo("full_jetlp", 0), 4)}
                                  for r in ("phi_0.99", "phi_0.9999")}}
    print(json.dumps(summary), flush=True)
    return 0


def batched_graphs(count=512):
    """The batched workload: random geometric graphs in the unit square, n
    log-uniform in [1k, 200k], mean degree 8, unit weights, each with its own
    k uniform in {2, 4, ..., 64}; seeded."""
    import numpy as np
    import graphgen
    rng = np.random.default_rng(SEED)
    ns = np.exp(rng.uniform(np.log(1000), np.log(200000), count)).astype(np.int64)
    ks = rng.choice(np.arange(2, 65, 2), count)
    return [(graphgen.rgg(int(n), seed=i + 1), int(k)) for i, (n, k) in enumerate(zip(ns, ks))]


def run_batched(args):
    """Sequential plain partitions vs the batched form on the same graphs
    (cuts must agree); wall time around each whole set."""
    import time
    import torch
    import paper_2304_13194_gb300 as jet
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    gks = batched_graphs()
    items = [dict(xadj=torch.from_numpy(g.xadj).to(dev), adjncy=torch.from_numpy(g.adjncy).to(dev), k=k, eps=EPS,
                  seed=SEED + i) for i, (g, k) in enumerate(gks)]
    n_tot = sum(g.n for g, _ in gks)
    m_tot = sum(g.m for g, _ in gks)
    with jet.Context(0) as ctx:
        for it in items[:8]:                                          # warm-up
            ctx.partition(it["xadj"], it["adjncy"], k=it["k"], eps=EPS, seed=it["seed"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        seq = [ctx.partition(it["xadj"], it["adjncy"], k=it["k"], eps=EPS, seed=it["seed"])[1] for it in items]
        torch.cuda.synchronize()
        t_seq = time.perf_counter() - t0
        print(json.dumps({"sweep": "batched", "mode": "sequential", "graphs": len(items), "n_total": n_tot,
                          "m_total": m_tot, "seconds": round(t_seq, 4)}), flush=True)
        for workers in (4, 8, 16):
            ctx.partition_batch(items[:16], workers=workers)          # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = ctx.partition_batch(items, workers=workers)
            torch.cuda.synchronize()
            t_b = time.perf_counter() - t0
            same = all(o[1] == c for o, c in zip(out, seq))
            print(json.dumps({"sweep": "batched", "mode": "batched", "workers": workers, "graphs": len(items),
                              "seconds": round(t_b, 4), "speedup_vs_sequential": round(t_seq / t_b, 3),
                              "cuts_equal_to_sequential": same}), flush=True)
        # autotuned: execution choices timed on a sample of 64 graphs, then the whole set
        t0 = time.perf_counter()
        rep = ctx.autotune(items[::8], reps=1)
        t_tune = time.perf_counter() - t0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = ctx.partition_batch(items, workers=rep["workers"])
        torch.cuda.synchronize()
        t_b = time.perf_counter() - t0
        same = all(o[1] == c for o, c in zip(out, seq))
        chosen = {k: v for k, v in rep.items() if k not in ("candidates", "parts")}
        print(json.dumps({"sweep": "batched", "mode": "autotuned", "chosen": chosen,
                          "tune_seconds": round(t_tune, 3), "graphs": len(items),
                          "seconds": round(t_b, 4), "speedup_vs_sequential": round(t_seq / t_b, 3),
                          "cuts_equal_to_sequential": same,
                          "candidates": [[c["stage"], c["value"], round(c["ms"], 2)] for c in rep["candidates"]]}),
              flush=True)
    return 0


def run_rmat(args):
    """The power-law configuration: R-MAT scale 22 (edge factor 16, a=.57,
    b=c=.19, d=.05, symmetrised, unit weights), k in {2, 8, 64, 256}: partition
    time (CUDA events, median of 3 after one warm-up), refinement throughput,
    cut (checked against jet_cut) and balance."""
    import torch
    import graphgen
    import paper_2304_13194_gb300 as jet
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    g = graphgen.rmat(22, seed=SEED)
    xadj, adj = torch.from_numpy(g.xadj).to(dev), torch.from_numpy(g.adjncy).to(dev)
    flags = (jet.FLAG_TWO_HOP if args.two_hop else 0) | (jet.FLAG_HOSTLOOP if args.hostloop else 0)
    with jet.Context(0, flags=flags) as ctx:
        for k in ((args.rmat_k,) if args.rmat_k else (2, 8, 64, 256)):
            ctx.partition(xadj, adj, k=k, eps=EPS, seed=SEED)                    # warm-up
            runs = [ctx.partition(xadj, adj, k=k, eps=EPS, seed=SEED, return_stats=True) for _ in range(3)]
            part, cut, st = runs[0]
            assert all(r[1] == cut for r in runs)
            c2, pw = ctx.cut(xadj, adj, None, None, k, part)
            ms = sorted(r[2].ms_total for r in runs)[1]
            L = (-(-g.n // k)) * (1000000 + round(EPS * 1e6)) // 1000000
            print(json.dumps({"sweep": "rmat", "graph": "rmat22", "two_hop": bool(args.two_hop), "n": g.n, "m": g.m,
                              "k": k, "levels": st.levels,
                              "coarsest_n": st.n[-1], "partition_ms": round(ms, 2),
                              "coarsen_ms": round(st.ms_coarsen, 2), "init_ms": round(st.ms_init, 2),
                              "refine_ms": round(st.ms_refine, 2),
                              "refine_medges_per_s": round(st.edge_iters / st.ms_refine / 1e3, 1),
                              "cut": cut, "cut_recomputed": c2, "max_part_w": int(pw.max().item()), "limit": L}),
                  flush=True)
    return 0


SHAPE_CANDIDATES = [("list_blocks_per_sm", (2, 8)), ("apply_blocks_per_sm", (1, 2)),
                    ("list_items_per_block", (32, 128, 256)), ("scan_blocks_per_sm", (4, 16)),
                    ("hub_degree", (256, 4096))]


def run_shapes(args):
    """Launch shapes of the refinement kernels, one option at a time from the
    defaults, on the mesh and the power-law workloads: median refinement ms
    of three partitions after one warm-up (CUDA-graph loop), cut checked
    against the default's (execution choices never change results)."""
    import torch
    import graphgen
    import paper_2304_13194_gb300 as jet
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for gname, g in (("grid3d_128_w", workload_graph(128)), ("rmat22", graphgen.rmat(22, seed=SEED))):
        t = [torch.from_numpy(a).to(dev) if a is not None else None for a in (g.xadj, g.adjncy, g.vwgt, g.adjwgt)]
        if gname == "rmat22":
            t[2] = t[3] = None
        runs = [("default", None, 0)] + [(opt, opt, v) for opt, vals in SHAPE_CANDIDATES for v in vals]
        ref_cut = None
        for label, opt, val in runs:
            kw = {opt: val} if opt else {}
            with jet.Context(0, **kw) as ctx:
                ctx.partition(*t, k=K_PARTS, eps=EPS, seed=SEED)
                res = []
                for _ in range(3):
                    flush.zero_()
                    res.append(ctx.partition(*t, k=K_PARTS, eps=EPS, seed=SEED, return_stats=True))
            cut = res[0][1]
            if ref_cut is None:
                ref_cut = cut
            ms = sorted(r[2].ms_refine for r in res)[1]
            tot = sorted(r[2].ms_total for r in res)[1]
            print(json.dumps({"sweep": "shapes", "graph": gname, "option": label, "value": val,
                              "refine_ms": round(ms, 3), "total_ms": round(tot, 3), "cut": cut,
                              "cut_equal": cut == ref_cut}), flush=True)
        del t
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.sweep == "batched":
        return run_batched(args)
    if args.sweep == "shapes":
        return run_shapes(args)
    if args.sweep == "rmat":
        return run_rmat(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.kernel_probe:
        return run_probe(args)
    if args.sweep:
        return run_sweep(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
