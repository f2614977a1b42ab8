#!/usr/bin/env python3
"""Benchmark of the GB300 mapping path.

One step = one complete multilevel mapping (GPU-IM, Section 4.2): label-
propagation coarsening with sort-based contraction, initial mapping, then
Alg. 6 refinement (label propagation + rebalancing + J evaluation) on every
level from the coarsest to the input graph.

Default workload (``--workload rmat``): R-MAT power-law graph of scale 22
(4,194,304 vertices, edge factor 16, (a, b, c) = (.57, .19, .19), self-loops
and duplicates removed, seeded relabelling: 64,152,350 undirected edges),
unit weights, hierarchy 4:16:8 (k = 512), distances 1:10:100, eps = 0.03.
``--workload rgg``: random geometric graph with 2^20 vertices, mean degree
12, edge weights 1..10, hierarchy 4:8:8.  ``--workload grid64``: the 64x64
grid, hierarchy 4:8, distances 1:10, 10 fixed refinement rounds from a
seeded random mapping plus J, no coarsening (L2- and launch-bound).

Metric: mapped edges per second: the undirected edges of the input graph
divided by the end-to-end map time (``ms_per_step``), so coarsening,
contraction, initial mapping, projection and refinement all count; for
grid64 the edges of the grid times the 10 rounds over the time of the 10
rounds.  J is bit-equal to the CPU oracle (tests).  ``refine_round`` gives
the edges/s of one refinement round on the input graph (m_undirected /
t_round) and its fraction of the HBM peak.  ``e2e`` measures the same metric
through the C ABI with host buffers (graph upload, validation, mapping,
download of P).

``--impl reference`` times the CPU oracle (plain serial C, one core); on
R-MAT each step is a bounded sample: the map of R-MAT of scale
``--cpu-sample-scale`` (default 13) from the same generator and settings.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "edges/s per refine round, end-to-end map time at equal J, % HBM peak"
UNIT = "edges/s"
L2_FLUSH_BYTES = 512 << 20
# DRAM bytes per algorithmic byte of a kernel class from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of one launch on the input
# graph of the RGG 2^20 workload;
# profiles/k_eval_tile_k_lp_gain_tile_k_cluster_tile_rgg2e20_level0.md and
# profiles/k_match_prefer_rgg2e20_level0.md),
# valid only while the kernel's source hash matches.
TRAFFIC = {
    ("rgg2d", "lp_gain"): {"kernel": "k_lp_gain_tile", "kernel_hash": "6b701f37fb0860d6", "dram_bytes": 120026880,
                "alg_bytes": 178028552, "dram_per_alg_byte": 120026880 / 178028552},
    ("rgg2d", "cluster"): {"kernel": "k_cluster_tile", "kernel_hash": "03b2663e5efeed5a", "dram_bytes": 129838592,
                           "alg_bytes": 167542792, "dram_per_alg_byte": 129838592 / 167542792},
    ("rgg2d", "match_prefer"): {"kernel": "k_match_prefer", "kernel_hash": "8f3c2a530fe7cd2d", "dram_bytes": 121675776,
                     "alg_bytes": 221992288, "dram_per_alg_byte": 121675776 / 221992288},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--log2n", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-samples", type=int, default=4)
    ap.add_argument("--coarsener", default="lp", choices=["lp", "match"],
                    help="lp: label-propagation clustering (default); match: two-hop matching (Section 4.2)")
    ap.add_argument("--initial", default="bfs", choices=["bfs", "hm"],
                    help="mapping of the coarsest graph: bfs: breadth-first chunks (default); hm: hierarchical "
                         "multisection (Section 4.2, initial partitioning)")
    ap.add_argument("--lp-relax", default="0/1",
                    help="relaxed label-propagation filter c = num/den (0/1: the paper's G >= 0 filter)")
    ap.add_argument("--reb-objective", default="cut", choices=["cut", "j"],
                    help="rebalancing gains: cut (the paper's) or j (Eq. 1)")
    ap.add_argument("--launch-mode", type=int, default=0, choices=[0, 1],
                    help="0: refinement / clustering loops as CUDA graphs; 1: stream launches")
    ap.add_argument("--profile-steps", type=int, default=3,
                    help="steps re-run with per-kernel CUDA events after the timed region")
    ap.add_argument("--workload", default="rmat", choices=["rmat", "rgg", "grid64", "batch", "serve", "hm"],
                    help="rmat: the R-MAT scale-22 full map, 4:16:8 (default); rgg: the RGG 2^20 multilevel job; "
                         "grid64: 10 fixed refinement rounds + J on the 64x64 grid; batch: 64 RGGs of "
                         "2^12..2^18 vertices, 10 fixed refinement rounds each, one persistent launch vs one job at "
                         "a time; serve: a Poisson stream of mapping requests through the server; hm: hierarchical "
                         "multisection (GPU-HM) of the RGG 2^20 workload")
    ap.add_argument("--rmat-scale", type=int, default=22)
    ap.add_argument("--cpu-sample-scale", type=int, default=13,
                    help="R-MAT scale of the oracle's bounded sample (cpu_baseline and --impl reference)")
    ap.add_argument("--hm-workers", type=int, default=8, help="host threads partitioning one level's subgraphs")
    ap.add_argument("--serve-requests", type=int, default=400,
                    help="requests of the capacity run (all queued at once)")
    ap.add_argument("--serve-seconds", type=float, default=5.0,
                    help="length of each Poisson stream (requests = rate x seconds)")
    ap.add_argument("--serve-pool", type=int, default=48,
                    help="distinct requests generated; the stream cycles through them")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-lanes", type=int, default=0,
                    help="level batcher threads of the server (0: the library default, -1: no batching)")
    ap.add_argument("--probe", action="store_true",
                    help="one map_run, then one label-propagation step and one J evaluation on the input "
                         "graph inside the NVTX range 'probe', the coarsening again inside 'probe_coarsen' and "
                         "the matching coarsening inside 'probe_match' (for ncu captures of single launches)")
    return ap.parse_args()


def slowest_rank(pg, x, dev):
    """The largest x over the ranks (a job's time is its slowest rank's);
    x itself without a process group.  dev: where the reduction tensor lives
    (the rank's GPU under NCCL, "cpu" under gloo)."""
    if pg is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, ranks, seconds):
    """Whole-job throughput: the units every rank processed (each rank maps
    its own replica of the workload: weak scaling) over the job's time."""
    return units_per_rank * ranks / seconds


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(args, kind=None):
    from paper_2510_12196_gb300 import inputs as I
    kind = kind or args.workload
    if kind == "rmat":
        return I.workload_rmat(args.rmat_scale)
    if kind == "grid64":
        return I.workload_grid64()
    return I.workload_rgg(args.log2n)


def cpu_sample(args, w):
    """The oracle's bounded sample of workload w: the workload itself, except
    for R-MAT, whose serial map takes tens of minutes at scale 22: there the
    map of a smaller R-MAT from the same generator and settings."""
    from paper_2510_12196_gb300 import inputs as I
    if w.name.startswith("rmat") and args.cpu_sample_scale < args.rmat_scale:
        s = I.workload_rmat(args.cpu_sample_scale)
        return s, (f"R-MAT scale {args.cpu_sample_scale} (n={s.graph.n}, {s.graph.m} undirected edges) from the "
                   f"same generator and settings, one complete multilevel map per sample (a serial map at scale "
                   f"{args.rmat_scale} takes tens of minutes)")
    if not w.multilevel:
        return w, f"the full workload: {w.rounds} fixed refinement rounds + J per sample"
    return w, "the full workload, one complete multilevel map per sample"


COARSENERS = {"lp": 0, "match": 1}
INITIALS = {"bfs": 0, "hm": 1}


def variant_settings(args):
    """(lp_relax_num, lp_relax_den, reb_objective) of the command line."""
    num, den = (int(x) for x in args.lp_relax.split("/"))
    return num, den, 1 if args.reb_objective == "j" else 0


def config_of(w, extra=None, coarsener="lp", initial="bfs", variants=(0, 1, 0)):
    g, t = w.graph, w.topo
    if not w.multilevel:
        cfg = {"workload": "grid2d 64x64 4-neighbour, unit weights, H=4:8 D=1:10 eps=0.03, "
                           f"{w.rounds} fixed refinement rounds + J from P0(v) = h(v) mod {t.k}, no coarsening",
               "n": g.n, "m_undirected": g.m, "m_dir": g.m_dir, "k": t.k, "seed": w.seed, "rounds": w.rounds,
               "parallelism": "replicas",
               "l2": "not flushed: the working set (~0.2 MB) is L2-resident by design; reported as L2/launch-bound"}
        if variants != (0, 1, 0):
            cfg["variants"] = list(variants)
        if extra:
            cfg.update(extra)
        return cfg
    tail = "" if coarsener == "lp" else " two-hop-matching-coarsener"
    tail += "" if initial == "bfs" else " multisection-initial-mapping"
    tail += "" if variants[0] == 0 else f" relaxed-lp-filter-{variants[0]}/{variants[1]}"
    tail += "" if variants[2] == 0 else " j-objective-rebalancing"
    if w.name.startswith("rmat"):
        fam = (f"rmat scale {int(np.log2(g.n))} edge-factor 16 (a,b,c)=(.57,.19,.19) self-loops/duplicates removed, "
               f"unit weights n={g.n} ")
        l2 = "flushed between timed steps (512 MiB write); the CSR is larger than the 129 MB L2"
    else:
        fam = f"rgg2d n=2^{int(np.log2(g.n))} mean-degree-12 edge-weights-1..10 "
        l2 = "flushed between timed steps (512 MiB write); the CSR (~112 MB) is below the 129 MB L2"
    cfg = {"workload": fam + f"H={':'.join(map(str, t.hier))} D={':'.join(map(str, t.dist))} eps={t.eps} "
                             "full-multilevel" + tail,
           "n": g.n, "m_undirected": g.m, "m_dir": g.m_dir, "k": t.k, "seed": w.seed, "l2": l2,
           "parallelism": "replicas"}
    if extra:
        cfg.update(extra)
    return cfg


def edge_rounds(stats_levels, n_list, m_dir_list, iters_list):
    return int(sum(it * (m // 2) for m, it in zip(m_dir_list, iters_list)))


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ["index", "pci.bus_id", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, bus_id=None):
        self.bus_id = (bus_id or "").lower()
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS),
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        rows = [[x.strip() for x in l.split(",")] for l in self.lines if l.count(",") >= len(self.FIELDS) - 1]
        if self.bus_id:
            mine = [r for r in rows if r[1].lower().endswith(self.bus_id[-12:])]
            rows = mine or rows
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[6:10]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _code_only(src):
    """Source text without // comments and blank lines: a comment edit does
    not change what a kernel does, so it must not invalidate its counters."""
    lines = (line.split("//", 1)[0].rstrip() for line in src.split("\n"))
    return "\n".join(line for line in lines if line)


def kernel_hash(kernel="k_eval_tile"):
    """Hash of the code (comments left out) of one kernel: its definition
    (launch bounds and body, from refine.cu, coarsen.cu or match.cu), the row
    helper, the tile-staging functions of tile.cuh that it calls, and
    common.cuh."""
    import re
    csrc = os.path.join(ROOT, "paper_2510_12196_gb300", "csrc")
    text = "".join(open(os.path.join(csrc, f)).read() for f in ("refine.cu", "coarsen.cu", "match.cu"))
    tile = open(os.path.join(csrc, "tile.cuh")).read()

    def body(src, name):
        m = re.search(r"\n[^\n]*\b" + name + r"\(.*?\n}\n", src, re.S)
        return m.group(0) if m else ""

    h = hashlib.sha256()
    kbody = body(text, kernel)
    for part in (kbody, body(text, "row_cost")):
        h.update(_code_only(part).encode())
    # the staging helpers and constants of tile.cuh: constants always, each
    # function only if the kernel names it
    h.update(_code_only("\n".join(l for l in tile.split("\n") if l.startswith("constexpr"))).encode())
    for fn in ("stage_tile", "stage_tile_packed", "tile_worker", "tile_worker_ranked"):
        if re.search(r"\b" + fn + r"\b", kbody):
            h.update(_code_only(body(tile, fn)).encode())
    h.update(_code_only(open(os.path.join(csrc, "common.cuh")).read()).encode())
    return h.hexdigest()[:16]


# ----------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ----------------------------------------------------------------------------
def units_per_step(w):
    """The metric's units in one step of workload w: the undirected edges of
    the input graph (one complete map), or edges x rounds for a fixed-round
    refinement workload."""
    return w.graph.m * (w.rounds if not w.multilevel else 1)


def oracle_params(w, coarsener="lp", initial="bfs", variants=(0, 1, 0)):
    import oracle as O
    prm = O.default_params(w.seed)
    prm.coarsener = COARSENERS[coarsener]
    prm.initial = INITIALS[initial]
    prm.lp_relax_num, prm.lp_relax_den, prm.reb_objective = variants
    return prm


def oracle_run(w, samples, coarsener="lp", initial="bfs", variants=(0, 1, 0)):
    """The oracle on workload w `samples` times: (seconds per sample, J, P)."""
    import oracle as O
    g, t = w.graph, w.topo
    prm = oracle_params(w, coarsener, initial, variants)
    times, J, pi = [], None, None
    for _ in range(samples):
        t0 = time.perf_counter()
        if w.multilevel:
            pi, J, _ = O.map_run(g, t.hier, t.dist, t.eps, prm)
        else:
            L = O.lmax(int(g.vw.sum()), t.k, t.eps)
            pi, J, *_ = O.refine(g, t.hier, t.dist, L, w.pi0, rounds=w.rounds, params=prm)
        times.append(time.perf_counter() - t0)
    return times, J, pi


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    w = workload(args)
    s, sample = cpu_sample(args, w)
    var = variant_settings(args)
    for _ in range(max(0, args.warmup)):
        oracle_run(s, 1, args.coarsener, args.initial, var)
    times, J, _ = oracle_run(s, max(1, args.steps), args.coarsener, args.initial, var)
    tot = sum(times)
    val = units_per_step(s) * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": len(times), "warmup": args.warmup, "ms_per_step": 1000 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": config_of(w, coarsener=args.coarsener, initial=args.initial,
                                                     variants=var), "J_sample": J,
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample + " per step (serial C oracle)"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(args, w, J_gpu, cfg):
    """The oracle timed on its bounded sample of w (one host core).  Where the
    sample is a smaller graph, the GPU maps it too and both must agree."""
    from paper_2510_12196_gb300 import gpumap as G
    s, sample = cpu_sample(args, w)
    var = variant_settings(args)
    times, Jc, pic = oracle_run(s, args.cpu_samples, args.coarsener, args.initial, var)
    if s is w:
        assert Jc == J_gpu, "oracle and GPU disagree on the bench workload"
    else:
        gs, ts = s.graph, s.topo
        cs = G.map_config_default(s.seed)
        for f in ("coarsener", "initial", "lp_relax_num", "lp_relax_den", "reb_objective"):
            setattr(cs, f, getattr(cfg, f))
        c2 = G.map_create(gs.xadj, gs.adj, gs.adjw, gs.vw, gs.n, ts.hier, ts.dist, ts.eps, cs)
        pi2 = np.zeros(gs.n, np.int32)
        J2 = G.map_run(c2, pi2)
        G.map_destroy(c2)
        assert J2 == Jc and np.array_equal(pi2, pic), "oracle and GPU disagree on the CPU sample"
    return {"value": units_per_step(s) * len(times) / sum(times), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{sample}; {len(times)} samples (serial C oracle, one host core)",
            "ms_per_sample": 1000 * sum(times) / len(times), "J_sample": Jc}


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def run_ours(args, ws, rank, local):
    import torch
    import ctypes as C
    from paper_2510_12196_gb300 import gpumap as G

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    w = workload(args)
    g, t = w.graph, w.topo
    stream = torch.cuda.current_stream(dev)
    d_in = [torch.from_numpy(a).to(dev) for a in (g.xadj, g.adj, g.adjw, g.vw)]
    cfg = G.map_config_default(w.seed)
    cfg.launch_mode = args.launch_mode
    cfg.coarsener = COARSENERS[args.coarsener]
    cfg.initial = INITIALS[args.initial]
    cfg.lp_relax_num, cfg.lp_relax_den, cfg.reb_objective = variant_settings(args)
    ctx = G.map_create(*d_in, g.n, t.hier, t.dist, t.eps, cfg, stream=stream, inputs_on_device=True)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    Js = []
    for _ in range(max(0, args.warmup)):
        Js.append(G.map_run(ctx))
    props = torch.cuda.get_device_properties(dev)
    sampler = ClockSampler(getattr(props, "pci_bus_id", None))
    sampler.start()
    time.sleep(0.3)
    launches0 = G.map_launch_count()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(i)  # evict L2 between timed steps (outside the events)
        evs[i][0].record(stream)
        Js.append(G.map_run(ctx))
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    launches = G.map_launch_count() - launches0
    clocks = sampler.stop()
    st = G.map_stats(ctx)  # every step maps the same graph identically
    levels = st.levels
    er = edge_rounds(levels, [st.n[i] for i in range(levels)], [st.m_dir[i] for i in range(levels)],
                     [st.iters[i] for i in range(levels)])
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = float(sum(step_ms))
    # Per-kernel CUDA-event timing cannot see inside the refinement graphs, so
    # the same steps run again with stream launches and events around the
    # profiled kernels (same kernels, same work, same results).
    G.map_profile_enable(ctx, 1)
    for i in range(args.profile_steps):
        flush.fill_(i)
        Js.append(G.map_run(ctx))
    prof = {}
    for kid, nm in G.KERNEL_CLASSES.items():
        l0, ms0, by0 = G.map_profile_read(ctx, kid, 0)      # input-graph level
        lr, msr, byr = G.map_profile_read(ctx, kid, -1)     # the coarser levels
        prof[nm] = {"launches": l0 + lr, "ms": ms0 + msr, "bytes": by0 + byr,
                    "level0": {"launches": l0, "ms": ms0, "bytes": by0}}
    G.map_profile_enable(ctx, 0)
    assert len(set(Js)) == 1, f"nondeterministic J: {set(Js)}"
    total_ms = slowest_rank(pg, total_ms, dev)
    units = units_per_step(w)
    value = job_throughput(units * args.steps, ws, total_ms / 1000.0)

    # roofline of the dominant profiled kernel (largest device time over the
    # job), on its launches over the input graph
    peak, peak_kind = measured_peak()
    tn, tall = max(prof.items(), key=lambda kv: kv[1]["ms"])
    tv = tall["level0"]
    achieved = tv["bytes"] / (tv["ms"] / 1000.0) / 1e9 if tv["ms"] > 0 else 0.0
    tr = TRAFFIC.get((w.name.split("_")[0], tn))
    traffic = None
    if tr and tr.get("kernel_hash") == kernel_hash(tr["kernel"]) and tv["launches"]:
        traffic = tr["dram_per_alg_byte"] * tv["bytes"] / tv["launches"]
    roof = {"bound": "hbm", "kernel": tn, "kernel_name": G.KERNEL_OF_CLASS.get(tn),
            "scope": "launches on the input graph (level 0), CUDA events on the library stream during "
                     f"{args.profile_steps} profiled steps that follow the timed region",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
            "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)",
            "bytes_per_launch": tv["bytes"] / max(1, tv["launches"]), "launches": tv["launches"],
            "avg_launch_us": 1000 * tv["ms"] / max(1, tv["launches"]),
            "all_levels_GBps": tall["bytes"] / (tall["ms"] / 1000.0) / 1e9 if tall["ms"] > 0 else 0.0}

    # refinement rounds on the input graph against both per-round byte models
    # (compulsory streams 37 m_dir + 58 n; strict CSR-twice minimum 16 m_dir + 58 n)
    r0 = st.iters[0]
    ms0 = st.ms_refine_level[0]
    refine_round = None
    if r0 > 0 and ms0 > 0:
        us = 1000.0 * ms0 / r0
        alg_b = 37 * g.m_dir + 58 * g.n
        strict_b = 16 * g.m_dir + 58 * g.n
        refine_round = {"level": 0, "rounds": int(r0), "us_per_round": us,
                        "edges_per_s": g.m / (us * 1e-6), "m_undirected": g.m, "m_dir": g.m_dir,
                        "frac": strict_b / us / 1e3 / peak, "frac_model": "strict (16 m_dir + 58 n bytes per round)",
                        "strict_bytes": strict_b, "strict_GBps": strict_b / us / 1e3,
                        "strict_frac": strict_b / us / 1e3 / peak,
                        "alg_bytes": alg_b, "alg_GBps": alg_b / us / 1e3, "alg_frac": alg_b / us / 1e3 / peak,
                        "peak": peak,
                        "scope": "host wall time of Alg. 6 on the input graph in the last timed step (graph "
                                 "launches, result read-back), over its iterations: label-propagation and "
                                 "rebalancing rounds together"}

    # end to end through the C ABI with host buffers (pinned), P read back
    e2e = None
    if not args.no_e2e and args.e2e_steps > 0:
        h = [torch.from_numpy(a).pin_memory() for a in (g.xadj, g.adj, g.adjw, g.vw)]
        out = torch.empty(g.n, dtype=torch.int32).pin_memory()
        hbytes = sum(x.numel() * x.element_size() for x in h)
        e2e_t = []
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            c2 = G.map_create(*[x.data_ptr() for x in h], g.n, t.hier, t.dist, t.eps, cfg, stream=stream)
            J2 = G.lib().map_run(c2, C.c_void_p(out.data_ptr()), None)
            G.map_sync(c2)
            dt = time.perf_counter() - t0
            G.map_destroy(c2)
            assert J2 == 0
            if i > 0:  # first one warms the allocator
                e2e_t.append(dt)
        e2e_s = sum(e2e_t)
        e2e_s = slowest_rank(pg, e2e_s, dev)
        e2e = {"value": job_throughput(units * len(e2e_t), ws, e2e_s), "unit": UNIT, "h2d_bytes_per_step": hbytes,
               "d2h_bytes_per_step": g.n * 4, "ms_per_step": 1000 * e2e_s / len(e2e_t),
               "path": "map_create(host CSR) + map_run + download of P + map_destroy"}

    G.map_destroy(ctx)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, w, Js[0], cfg)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                "config": config_of(w, {"levels": levels, "level_n": [st.n[i] for i in range(levels)],
                                        "refine_rounds": [st.iters[i] for i in range(levels)],
                                        "refine_kinds_lp_weak_strong": [[st.lp_iters[i], st.weak_iters[i],
                                                                         st.strong_iters[i]] for i in range(levels)],
                                        "schedule": {"mid_deg": [st.mid_deg[i] for i in range(levels)],
                                                     "split_deg": [st.split_deg[i] for i in range(levels)],
                                                     "autotuned": [st.tuned[i] for i in range(levels)],
                                                     "tune_ms": st.ms_tune}},
                                    args.coarsener, args.initial, variant_settings(args)),
                "edge_rounds_per_s": job_throughput(er * args.steps, ws, total_ms / 1000.0),
                "J": Js[0], "e2e": e2e, "roofline": roof, "refine_round": refine_round, "cpu_baseline": cpu,
                "clocks": clocks,
                "gpu_launches": int(launches), "kernels": prof,
                "phase_ms": {"coarsen": st.ms_coarsen, "initial": st.ms_initial, "refine": st.ms_refine,
                             "project": st.ms_project}}
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


def run_grid64(args, ws, rank, local):
    """The 64x64 grid: 10 synchronous refinement rounds (Alg. 6 body, fixed
    count) + J from the seeded random mapping, no coarsening.  The working
    set (~0.2 MB) lives in L2: the rounds are launch- and latency-bound."""
    import torch
    import ctypes as C
    from paper_2510_12196_gb300 import gpumap as G

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    w = workload(args)
    g, t = w.graph, w.topo
    stream = torch.cuda.current_stream(dev)
    cfg = G.map_config_default(w.seed)
    cfg.launch_mode = args.launch_mode
    cfg.lp_relax_num, cfg.lp_relax_den, cfg.reb_objective = variant_settings(args)
    ctx = G.map_create(g.xadj, g.adj, g.adjw, g.vw, g.n, t.hier, t.dist, t.eps, cfg, stream=stream)
    Js = []
    for _ in range(max(0, args.warmup)):
        G.map_set_mapping(ctx, 0, w.pi0)
        Js.append(G.map_refine(ctx, 0, w.rounds)[0])
    props = torch.cuda.get_device_properties(dev)
    sampler = ClockSampler(getattr(props, "pci_bus_id", None))
    sampler.start()
    time.sleep(0.3)
    launches0 = G.map_launch_count()
    step_ms = []
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    for i in range(args.steps):
        G.map_set_mapping(ctx, 0, w.pi0)  # the same start every step (outside the events)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Js.append(G.map_refine(ctx, 0, w.rounds)[0])  # returns J: synchronises
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    if pg:
        pg.barrier()
    launches = G.map_launch_count() - launches0
    clocks = sampler.stop()
    assert len(set(Js)) == 1, f"nondeterministic J: {set(Js)}"
    total_ms = slowest_rank(pg, float(sum(step_ms)), dev)
    units = units_per_step(w)
    value = job_throughput(units * args.steps, ws, total_ms / 1000.0)
    us_round = 1000.0 * total_ms / args.steps / w.rounds
    peak, peak_kind = measured_peak()
    alg_b = 37 * g.m_dir + 58 * g.n
    roof = {"bound": "hbm", "kernel": "one refinement round (fused engine or graph of kernels)",
            "achieved": alg_b / us_round / 1e3, "peak": peak, "unit": "GB/s",
            "frac": alg_b / us_round / 1e3 / peak, "traffic": None,
            "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)",
            "note": "the working set (about 0.2 MB) fits in L2: L2- and launch-bound, the HBM fraction does not "
                    "apply; bytes by the per-round model 37 m_dir + 58 n"}
    e2e = None
    if not args.no_e2e and args.e2e_steps > 0:
        pin = [torch.from_numpy(a).pin_memory() for a in (g.xadj, g.adj, g.adjw, g.vw)]
        p0 = torch.from_numpy(w.pi0).pin_memory()
        out = torch.empty(g.n, dtype=torch.int32).pin_memory()
        hb = sum(x.numel() * x.element_size() for x in pin) + p0.numel() * 4
        tt = []
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            c2 = G.map_create(*[x.data_ptr() for x in pin], g.n, t.hier, t.dist, t.eps, cfg, stream=stream)
            assert G.lib().map_set_mapping(c2, 0, C.c_void_p(p0.data_ptr())) == 0
            J2 = G.map_refine(c2, 0, w.rounds)[0]
            assert G.lib().map_get_mapping(c2, 0, C.c_void_p(out.data_ptr())) == 0
            dt = time.perf_counter() - t0
            G.map_destroy(c2)
            assert J2 == Js[0]
            if i > 0:
                tt.append(dt)
        e2e_s = slowest_rank(pg, sum(tt), dev)
        e2e = {"value": job_throughput(units * len(tt), ws, e2e_s), "unit": UNIT, "h2d_bytes_per_step": hb,
               "d2h_bytes_per_step": g.n * 4 + 8, "ms_per_step": 1000 * e2e_s / len(tt),
               "path": "map_create(host CSR) + map_set_mapping + map_refine(10 rounds) + map_get_mapping + "
                       "map_destroy"}
    G.map_destroy(ctx)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, w, Js[0], cfg)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                "config": config_of(w, variants=variant_settings(args)),
                "us_per_round": us_round, "J": Js[0], "e2e": e2e, "roofline": roof, "cpu_baseline": cpu,
                "clocks": clocks, "gpu_launches": int(launches)}
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


def run_probe(args, local):
    import torch
    from paper_2510_12196_gb300 import gpumap as G
    torch.cuda.set_device(local)
    w = workload(args)
    g, t = w.graph, w.topo
    cfg = G.map_config_default(w.seed)
    cfg.launch_mode = 1  # stream launches: a profiler sees every kernel
    ctx = G.map_create(g.xadj, g.adj, g.adjw, g.vw, g.n, t.hier, t.dist, t.eps, cfg)
    J = G.map_run(ctx)
    st0 = G.map_stats(ctx)
    sched0 = {"mid_deg": st0.mid_deg[0], "split_deg": st0.split_deg[0], "autotuned": st0.tuned[0]}
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("probe_coarsen")
    G.map_coarsen(ctx)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    J = G.map_run(ctx)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("probe")
    moved = G.map_lp_step(ctx, 0)
    J2, mw = G.map_objective(ctx, 0)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    G.map_destroy(ctx)
    # the matching coarsener on the same graph (its first launches are level 0's heavy-edge rounds)
    cfg.coarsener = 1
    ctx = G.map_create(g.xadj, g.adj, g.adjw, g.vw, g.n, t.hier, t.dist, t.eps, cfg)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("probe_match")
    nl = G.map_coarsen(ctx)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    G.map_destroy(ctx)
    print(json.dumps({"probe": "coarsening (range probe_coarsen); lp_step + objective on level 0 after "
                               "map_run (range probe); matching coarsening (range probe_match)", "J_map": J,
                      "moved": moved, "J_after_step": J2, "n": g.n, "m_dir": g.m_dir, "match_levels": nl,
                      "level0_schedule": sched0}))
    return 0


# ----------------------------------------------------------------------------
# batched refinement: 64 graphs in one persistent launch vs one at a time
# ----------------------------------------------------------------------------
def run_batch(args, ws, rank, local):
    import torch
    from paper_2510_12196_gb300 import gpumap as G
    from paper_2510_12196_gb300 import inputs as I

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = I.workload_batch()
    ctxs = []
    for w in wl:
        g, t = w.graph, w.topo
        cfg = G.map_config_default(w.seed)
        ctxs.append(G.map_create(g.xadj, g.adj, g.adjw, g.vw, g.n, t.hier, t.dist, t.eps, cfg))

    def reset():
        for c, w in zip(ctxs, wl):
            G.map_set_mapping(c, 0, w.pi0)

    rounds = wl[0].rounds
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    nj = len(ctxs)
    # batched: autotune + capture on the first launch (untimed)
    reset()
    b = G.map_batch_create(ctxs, G.map_batch_opts_default(rounds=rounds), stream=stream)
    G.map_batch_launch(b)
    Jb, _, itb = G.map_batch_results(b, nj)
    sched = G.map_batch_schedule(b)
    for _ in range(max(0, args.warmup)):
        reset()
        G.map_batch_launch(b)
        G.map_batch_results(b, nj)
    er = int(sum(int(it) * w.graph.m for it, w in zip(itb, wl)))

    def timed(fn):
        evs = []
        for i in range(args.steps):
            reset()
            flush.fill_(i)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            evs.append(e0.elapsed_time(e1))
        return evs

    def batched():
        G.map_batch_launch(b)

    plain_J = []

    def plain():
        plain_J.clear()
        for c in ctxs:
            plain_J.append(G.map_refine(c, 0, rounds)[0])

    props = torch.cuda.get_device_properties(dev)
    sampler = ClockSampler(getattr(props, "pci_bus_id", None))
    sampler.start()
    time.sleep(0.3)
    launches0 = G.map_launch_count()
    tb = timed(batched)
    launches = (G.map_launch_count() - launches0) / max(1, args.steps)
    clocks = sampler.stop()
    Jb2, _, itb2 = G.map_batch_results(b, nj)
    for _ in range(max(0, args.warmup)):
        reset()
        plain()
    tp = timed(plain)
    assert list(Jb2) == list(Jb) == plain_J and list(itb2) == list(itb), "batched and plain results differ"
    G.map_batch_destroy(b)
    for c in ctxs:
        G.map_destroy(c)
    ms_b, ms_p = sum(tb) / len(tb), sum(tp) / len(tp)
    peak, peak_kind = measured_peak()
    alg_bytes = sum(int(it) * (37 * w.graph.m_dir + 58 * w.graph.n) for it, w in zip(itb, wl))
    achieved = alg_bytes / (ms_b / 1000.0) / 1e9
    if rank == 0:
        line = {"metric": METRIC, "workload": "batch", "value": er / (ms_b / 1000.0), "unit": UNIT, "n_gpus": 1,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                "config": {"workload": "64 RGGs, n log-uniform in 2^12..2^18, mean degree 10, edge weights "
                                       "1..10, H from {4:8, 4:8:8, 2:4:16:8}, D prefix of 1:10:100:1000, "
                                       "eps 0.03, 10 fixed Alg. 6 rounds from h(v) mod k",
                           "jobs": nj, "n_total": int(sum(w.graph.n for w in wl)),
                           "m_dir_total": int(sum(w.graph.m_dir for w in wl)),
                           "l2": "flushed between timed steps (512 MiB write)",
                           "schedule": {"ctas_per_job": sched[0], "tile_entries": sched[1],
                                        "clusters": sched[2], "autotune_ms": sched[3]}},
                "plain": {"value": er / (ms_p / 1000.0), "ms_per_step": ms_p,
                          "path": "map_refine on each context in turn (one job at a time)"},
                "speedup_vs_plain": ms_p / ms_b,
                "roofline": {"bound": "hbm", "kernel": "k_engine (whole batch launch)",
                             "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                             "traffic": None, "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)",
                             "bytes_model": "per round and job 37 m_dir + 58 n"},
                "clocks": clocks, "gpu_launches": launches, "J_total": int(sum(Jb))}
        print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# serving: Poisson arrivals through the request loop
# ----------------------------------------------------------------------------
def run_serve(args, ws, rank, local):
    """Serving: the capacity of the server (all requests queued at once,
    `--serve-slots` slots, small levels batched across requests) and of one
    slot, then Poisson streams offered at about 50 % and 90 % of that
    capacity and at the configured 200 req/s: throughput, latency (submit to
    result) and service time (start to result) percentiles.  Every served
    result is checked against the same request alone."""
    import queue as Q
    import torch
    from paper_2510_12196_gb300 import gpumap as G
    from paper_2510_12196_gb300 import inputs as I

    torch.cuda.set_device(local)
    pool = [I.serve_request(i) for i in range(args.serve_pool)]
    cfgs = [G.map_config_default(w.seed) for w in pool]
    alone = []  # each pool request alone (reference results, also the warm-up)
    for w, cfg in zip(pool, cfgs):
        g, t = w.graph, w.topo
        ctx = G.map_create(g.xadj, g.adj, g.adjw, g.vw, g.n, t.hier, t.dist, t.eps, cfg)
        J = G.map_run(ctx)
        st = G.map_stats(ctx)
        er = edge_rounds(st.levels, None, [st.m_dir[i] for i in range(st.levels)],
                         [st.iters[i] for i in range(st.levels)])
        G.map_destroy(ctx)
        alone.append((J, er))

    def stream(slots, R, arr, lanes=0):
        """R requests (pool order cycled) at arrival times arr (None: all at
        once); returns the run's figures."""
        srv = G.MapServer(slots=slots, lookahead=8, batch_lanes=lanes)
        tq = Q.Queue()
        out = [None] * R

        def collect():
            for _ in range(R):
                i, t = tq.get()
                r, _ = srv.wait(t)
                out[i] = (r.status, r.J, r.t_submit_ms, r.t_start_ms, r.t_done_ms)

        th = threading.Thread(target=collect)
        th.start()
        t0 = time.perf_counter()
        for i in range(R):
            if arr is not None:
                dt = t0 + arr[i] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
            w = pool[i % len(pool)]
            tq.put((i, srv.submit(w.graph, w.topo.hier, w.topo.dist, w.topo.eps, cfg=cfgs[i % len(pool)],
                                  user=i)))
        th.join()
        st = srv.stats()
        srv.close()
        bad = [i for i in range(R) if out[i][0] != 0 or out[i][1] != alone[i % len(pool)][0]]
        assert not bad, f"served results differ from the jobs alone: {bad[:5]}"
        lat = np.array([o[4] - o[2] for o in out])
        svc = np.array([o[4] - o[3] for o in out])
        span = max(o[4] for o in out) - min(o[2] for o in out)
        er = sum(alone[i % len(pool)][1] for i in range(R))
        return {"slots": slots, "requests": R, "jobs_per_s": 1000.0 * R / span,
                "offered_jobs_per_s": (R / float(arr[-1])) if arr is not None else None,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "service_p50_ms": float(np.percentile(svc, 50)),
                "service_p99_ms": float(np.percentile(svc, 99)), "service_mean_ms": float(svc.mean()),
                "edges_per_s": 1000.0 * er / span, "peak_running": st.peak_running,
                "peak_bytes_in_flight": st.peak_bytes_in_flight, "mem_budget": st.mem_budget,
                "batcher_launches": st.engine_launches, "batched_levels": st.engine_jobs,
                "peak_batch": st.peak_batch, "makespan_ms": span}

    props = torch.cuda.get_device_properties(local)
    sampler = ClockSampler(getattr(props, "pci_bus_id", None))
    sampler.start()
    time.sleep(0.3)
    launches0 = G.map_launch_count()
    R = args.serve_requests
    lanes = args.serve_lanes
    cap = stream(args.serve_slots, R, None, lanes)
    one = stream(1, max(len(pool), R // 2), None, lanes)
    loads = {}
    for frac in (0.5, 0.9):
        rate = frac * cap["jobs_per_s"]
        n = max(len(pool), int(round(rate * args.serve_seconds)))
        loads[f"{int(frac * 100)}pct"] = stream(args.serve_slots, n,
                                                I.poisson_arrivals(n, 1.0 / rate, I.SEED_ITEM + 0x20000), lanes)
    n200 = max(len(pool), int(round(200.0 * args.serve_seconds)))
    cfg200 = stream(args.serve_slots, n200, I.poisson_arrivals(n200, 0.005, I.SEED_ITEM + 0x20000), lanes)
    launches = G.map_launch_count() - launches0
    clocks = sampler.stop()
    if rank == 0:
        line = {"metric": METRIC, "workload": "serve", "value": cfg200["jobs_per_s"], "unit": "jobs/s",
                "n_gpus": 1, "steps": n200, "warmup": len(pool), "ms_per_step": cfg200["mean_ms"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
                "data": "synthetic",
                "config": {"workload": "Poisson stream (mean 200 req/s offered); 50% 3D 6-neighbour grids "
                                       "2^10..2^21 cells, 50% RGGs 2^12..2^20 vertices mean degree 12; H from "
                                       "{4:8, 4:8:8, 4:16:8, 4:16:16}, D prefix of 1:10:100, eps 0.03, full "
                                       "multilevel per request",
                           "distinct_requests": len(pool), "slots": args.serve_slots, "batch_lanes": lanes,
                           "l2": "not flushed (a stream of different graphs)"},
                "p50_ms": cfg200["p50_ms"], "p99_ms": cfg200["p99_ms"], "edges_per_s": cfg200["edges_per_s"],
                "capacity": cap, "capacity_one_slot": one,
                "capacity_ratio": cap["jobs_per_s"] / one["jobs_per_s"],
                "load_50pct": loads["50pct"], "load_90pct": loads["90pct"], "offered_200": cfg200,
                "clocks": clocks, "gpu_launches": launches}
        print(json.dumps(line), flush=True)
    return 0


def run_hm(args, ws, rank, local):
    """Hierarchical multisection of the RGG workload: wall time of map_run_hm
    (it synchronises; its partitioner calls run on several streams)."""
    import torch
    from paper_2510_12196_gb300 import gpumap as G
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload(args, "rgg")
    g, t = w.graph, w.topo
    stream = torch.cuda.current_stream(dev)
    d_in = [torch.from_numpy(a).to(dev) for a in (g.xadj, g.adj, g.adjw, g.vw)]
    cfg = G.map_config_default(w.seed)
    cfg.coarsener = COARSENERS[args.coarsener]
    cfg.launch_mode = args.launch_mode
    ctx = G.map_create(*d_in, g.n, t.hier, t.dist, t.eps, cfg, stream=stream, inputs_on_device=True)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    Js = [G.map_run_hm(ctx, workers=args.hm_workers) for _ in range(max(0, args.warmup))]
    props = torch.cuda.get_device_properties(dev)
    sampler = ClockSampler(getattr(props, "pci_bus_id", None))
    sampler.start()
    time.sleep(0.3)
    launches0 = G.map_launch_count()
    times, parts, builds = [], [], []
    for i in range(args.steps):
        flush.fill_(i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Js.append(G.map_run_hm(ctx, workers=args.hm_workers))
        times.append(time.perf_counter() - t0)
        st = G.map_hm_stats(ctx)
        parts.append(st.ms_partition)
        builds.append(st.ms_build)
    launches = G.map_launch_count() - launches0
    clocks = sampler.stop()
    st = G.map_hm_stats(ctx)
    G.map_destroy(ctx)
    assert len(set(Js)) == 1, f"nondeterministic J: {set(Js)}"
    ms = 1000 * sum(times) / len(times)
    cpu = None
    if not args.no_cpu_baseline:
        import oracle as O
        t0 = time.perf_counter()
        _, Jc, _ = O.hm_run(g, t.hier, t.dist, t.eps, O.default_params(w.seed) if args.coarsener == "lp" else
                            _oracle_params_match(w.seed))
        dt = time.perf_counter() - t0
        assert Jc == Js[0], "oracle and GPU disagree on the hierarchical multisection"
        cpu = {"value": 1000 * dt, "unit": "ms", "cores": 1, "kind": "oracle",
               "sample": "one complete hierarchical multisection of the workload (serial C oracle)"}
    line = {"metric": "end-to-end map time (hierarchical multisection, GPU-HM)", "value": ms, "unit": "ms",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": config_of(w, {"method": "GPU-HM (Alg. 3), partitioner = the library's multilevel pipeline "
                                              "on a_i with distance 1", "workers": args.hm_workers,
                                    "calls_per_level": [st.calls[i] for i in range(st.levels)]}, args.coarsener),
            "J": Js[0], "ms_partition": sum(parts) / len(parts), "ms_build": sum(builds) / len(builds),
            "ms_level": [st.ms_level[i] for i in range(st.levels)],
            "ms_calls": {"create": st.ms_create, "run": st.ms_run, "destroy": st.ms_destroy},
            "cpu_baseline": cpu, "clocks": clocks, "gpu_launches": int(launches)}
    print(json.dumps(line), flush=True)
    return 0


def _oracle_params_match(seed):
    import oracle as O
    p = O.default_params(seed)
    p.coarsener = 1
    return p


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.probe:
        return run_probe(args, local)
    if args.workload == "batch" and args.impl == "ours":
        return run_batch(args, ws, rank, local)
    if args.workload == "serve" and args.impl == "ours":
        return run_serve(args, ws, rank, local)
    if args.workload == "hm" and args.impl == "ours":
        return run_hm(args, ws, rank, local)
    if args.workload == "grid64" and args.impl == "ours":
        return run_grid64(args, ws, rank, local)
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    return run_ours(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
