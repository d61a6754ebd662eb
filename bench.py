#!/usr/bin/env python
"""Benchmark of the all-edge effective-resistance sweep (PEERS implicit-inverse walk).

One step = peers_query over every edge of the 1M-node 3-layer PDN mesh (3 x 577 x 577 5-point
grids, vias every 4th node, conductances log-uniform 1e-2..1e2, seed 2, node 0 grounded):
2 036 162 queries, each walked from its starting supernode to the root (§8 rows A1-A4).  The
factor is resident before the timed region; `value` is edge queries per second of the device
sweep, `e2e` the same metric through the public API with host buffers (conductances uploaded
and factored, results copied back) inside the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 (torchrun) every rank runs an independent replica on its own GPU (weak scaling);
the sweep itself needs no collective.  `--impl reference` times the CPU oracle (tests'
oracle/) on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "edge queries/s, all-edge sweep (1M-node PDN grid, FP64)"


def metric_of(workload):
    """The metric's name for a single-graph workload (the default one is the headline)."""
    return {"pdn1m": METRIC,
            "grid512": "edge queries/s, all-edge sweep (512x512 grid, FP64)",
            "grid32": "edge queries/s, all-edge sweep (32x32 grid, FP64)"}.get(workload, METRIC)
UNIT = "queries/s"
WORKLOAD = "pdn3x577x577_vias4_loguniform_1e-2_1e2_seed2_all_edges"
HBM_FALLBACK_GBS = 6400.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="pdn1m",
                    choices=["pdn1m", "grid32", "grid512", "batch256", "serve"])
    ap.add_argument("--requests", type=int, default=80,
                    help="serving stream: requests in the stream (the full stream is 500)")
    ap.add_argument("--rho", default="0.7,1.3",
                    help="serving stream: offered loads as fractions of the GPU's one-at-a-time "
                         "service rate, comma separated")
    ap.add_argument("--extras", default="batch,serve",
                    help="with the default workload at N=1, also measure the 256-graph batch "
                         "and the serving stream (comma list of batch, serve; empty: neither)")
    ap.add_argument("--cpu-sample", type=int, default=16000,
                    help="edges in the oracle's CPU-baseline sample (0 = skip)")
    ap.add_argument("--ref-sample", type=int, default=8000,
                    help="edges per step of --impl reference")
    ap.add_argument("--ref-threads", type=int, default=None,
                    help="host threads of --impl reference (default: all cores)")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--routes", default="blockinv,selinv",
                    help="other exact routes to time on the same queries after the walk: a "
                         "comma list of blockinv, selinv (empty: none)")
    ap.add_argument("--no-blockinv", action="store_true",
                    help="same as --routes ''")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the largest tiles instead of running the tile autotuner")
    return ap.parse_args()


def make_graph(name):
    from paper_2606_31535_b300 import inputs as I
    if name == "pdn1m":
        return I.pdn1m()
    if name == "grid512":
        return I.grid2d(512, 512, seed=3, law="loguniform", lo=1e-2, hi=1e2)
    return I.grid32()


def workload_name(name):
    return {"pdn1m": WORKLOAD, "grid32": "grid32x32_uniform_0.5_2_seed1_all_edges",
            "grid512": "grid512x512_loguniform_seed3_all_edges",
            "batch256": "batch256_grids_5pct_deleted_and_rgg6_1k_64k_loguniform_seeds3000+i_all_edges",
            "serve": "serve_stream_n10k_500k_grid_or_rgg_all_or_10pct_edges_poisson_seed4"}[name]


# ------------------------------------------------------------------ CPU oracle (host cores)

def _oracle_sample(workload, sample, steps, warmup, seed, out_q, threads=None):
    """Runs in a spawned process: factors with the oracle (untimed), then times the per-query
    path solves on `sample` seeded edges per step, on `threads` host cores (default all)."""
    import oracle
    g = make_graph(workload)
    t0 = time.time()
    F = oracle.Factor.of(g)
    t_fact = time.time() - t0
    u, v = g.all_edges()
    rng = np.random.default_rng(seed)
    idx = rng.choice(u.size, min(sample, u.size), replace=False)
    cores = threads or os.cpu_count() or 1
    times = []
    for i in range(warmup + steps):
        t0 = time.perf_counter()
        F.resistance(u[idx], v[idx], threads=cores)
        dt = time.perf_counter() - t0
        if i >= warmup:
            times.append(dt)
    out_q.put({"t_factor_s": t_fact, "times": times, "sample": int(idx.size), "cores": cores})


def start_oracle(workload, sample, steps, warmup, seed, threads=None):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_oracle_sample,
                    args=(workload, sample, steps, warmup, seed, q, threads))
    p.start()
    return p, q


# ------------------------------------------------------------------ clocks

CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def start_clocks(dev):
    f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    try:
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}",
                              "--format=csv,noheader,nounits", "-i", str(dev), "-lms", "200"],
                             stdout=f, stderr=subprocess.DEVNULL)
    except OSError:
        p = None
    return p, f


def stop_clocks(p, f):
    if p is None:
        return None
    p.terminate()
    try:
        p.wait(timeout=5)
    except subprocess.TimeoutExpired:
        p.kill()
    f.flush()
    f.seek(0)
    rows = [r.split(",") for r in f.read().strip().splitlines() if r.count(",") >= 8]
    f.close()
    os.unlink(f.name)
    if not rows:
        return None
    sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i]
                      and "Not" not in r[5 + i]})
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def k_sweep_source_sha(text):
    """Hash of the k_sweep kernel source: sweep.cu from kSweepThreads through the end of
    k_sweep_multi (the device code the DRAM counters were taken on; host helpers excluded)."""
    import hashlib
    a = text.index("constexpr int kSweepThreads")
    b = text.index("\n}\n", text.index("k_sweep_multi(const SweepItem")) + 3
    return hashlib.sha256(text[a:b].encode()).hexdigest()[:16]


def profiled_traffic(info, launches_per_step):
    """DRAM bytes per k_sweep launch of this plan, scaled from the committed ncu capture of a
    smaller sweep (the 512x512 grid) by the query-front bytes each sweep carries between
    levels (the DRAM traffic of the walk is those fronts, written at one level and read at
    the next; the panels are re-read from L2).  None when there is no capture or the kernel
    source has changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "k_sweep_dram_grid512.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
        with open(os.path.join(ROOT, "paper_2606_31535_b300", "csrc", "sweep.cu")) as fh:
            sha = k_sweep_source_sha(fh.read())
    except (OSError, ValueError):
        return None
    if rec.get("k_sweep_source_sha256_16") != sha or not info.get("front_bytes"):
        return None
    per_front_byte = rec["dram_bytes_per_sweep"] / rec["front_bytes"]
    return per_front_byte * info["front_bytes"] / max(1, launches_per_step)

def tuning_cache():
    """Tile-autotuner cache file: $PEERS_TUNING_CACHE, else one in the system temp dir."""
    return os.environ.get("PEERS_TUNING_CACHE",
                          os.path.join(tempfile.gettempdir(), "peers_tiles.txt"))


def dist_max(value, dist=None, device=None):
    """Largest `value` over all ranks (the job's time is its slowest rank's); the local value
    when not distributed.  Works with gloo (CPU tensors) and nccl (device tensors)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, seconds):
    """Whole-job throughput of `world` replicas that each process `units_per_rank` units, when
    the slowest took `seconds`."""
    return units_per_rank * world / seconds


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    p, q = start_oracle(args.workload, args.ref_sample, args.steps, args.warmup, seed=7,
                        threads=args.ref_threads)
    res = q.get()
    p.join()
    t = sum(res["times"])
    value = res["sample"] * args.steps / t
    line = {
        "impl": "reference", "metric": metric_of(args.workload), "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.workload), "queries_per_step": res["sample"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": res["cores"], "kind": "oracle",
                         "sample": f"{res['sample']} seeded edges per step (oracle factor "
                                   f"{res['t_factor_s']:.1f} s, untimed)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm

def run_ours(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    oracle_proc = None
    if rank == 0 and world == 1 and args.cpu_sample > 0:
        # spawned before the first GPU call; runs on the host cores while the GPU works
        oracle_proc = start_oracle(args.workload, args.cpu_sample, 1, 0, seed=11)

    import torch
    from paper_2606_31535_b300 import peers as P

    g = make_graph(args.workload)
    t0 = time.time()
    sym = P.Symbolic.of(g)
    t_analyze = time.time() - t0
    info = sym.info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    ctx = P.Context(local, stream)
    peaks64 = ctx.fp64_peaks()
    shapes64 = ctx.fp64_mma_shapes()
    fp64_peak = peaks64["dfma"]
    num = P.Numeric(ctx, sym)
    nq = sym.nq
    R = torch.empty(nq, dtype=torch.float64, device=f"cuda:{local}")
    tiles = None
    if not args.no_autotune:
        t0 = time.time()
        tiles = P.autotune(ctx, sym, num, tuning_cache())
        tiles["seconds"] = time.time() - t0

    for _ in range(args.warmup):
        P.query(ctx, sym, num, R)
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()

    barrier()
    torch.cuda.synchronize()
    clk = start_clocks(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    launches = 0
    for _ in range(args.steps):
        P.query(ctx, sym, num, R)
        launches += ctx.last_stats()["sweep_launches"]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = stop_clocks(*clk)
    t = dist_max(e0.elapsed_time(e1) * 1e-3, dist, f"cuda:{local}")
    step_s = t / args.steps
    value = job_throughput(nq * args.steps, world, t)

    sweep_stats = ctx.last_stats()
    # the same queries by the block implicit inverse (the paper's order of work)
    routes = set() if args.no_blockinv else {r for r in args.routes.split(",") if r}
    blockinv = None
    if "blockinv" in routes:
        cost = P.blockinv_cost(sym)
        Rb = torch.empty(nq, dtype=torch.float64, device=f"cuda:{local}")
        for _ in range(args.warmup):
            P.query_blockinv(ctx, sym, num, Rb)
        torch.cuda.synchronize()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for _ in range(args.steps):
            P.query_blockinv(ctx, sym, num, Rb)
        b1.record(stream)
        torch.cuda.synchronize()
        tb = b0.elapsed_time(b1) * 1e-3 / args.steps
        rel = float(((Rb - R).abs() / R.abs()).max().item()) if nq else 0.0
        blockinv = {"value": nq / tb, "unit": UNIT, "ms_per_step": 1e3 * tb,
                    "gemm_fma": cost["fma"], "gemm_tflops": 2.0 * cost["fma"] / tb / 1e12,
                    "frac_of_dfma_peak": 2.0 * cost["fma"] / tb / 1e12 / fp64_peak,
                    "device_bytes": cost["bytes"], "max_rel_vs_walk": rel,
                    "speedup_vs_walk": step_s / tb}
        del Rb
    # and from the selected inverse (Sigma on the pattern of L, Takahashi recurrences)
    selinv = None
    if "selinv" in routes:
        fma_si = int(P.load().peers_selinv_fma(sym._h))
        Rs = torch.empty(nq, dtype=torch.float64, device=f"cuda:{local}")
        for _ in range(args.warmup):
            P.query_selinv(ctx, sym, num, Rs)
        torch.cuda.synchronize()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for _ in range(args.steps):
            P.query_selinv(ctx, sym, num, Rs)
        b1.record(stream)
        torch.cuda.synchronize()
        ts = b0.elapsed_time(b1) * 1e-3 / args.steps
        rel = float(((Rs - R).abs() / R.abs()).max().item()) if nq else 0.0
        selinv = {"value": nq / ts, "unit": UNIT, "ms_per_step": 1e3 * ts, "fma": fma_si,
                  "tflops": 2.0 * fma_si / ts / 1e12,
                  "frac_of_dfma_peak": 2.0 * fma_si / ts / 1e12 / fp64_peak,
                  "max_rel_vs_walk": rel, "speedup_vs_walk": step_s / ts}
        del Rs
    num.close()
    # end to end through the public API: pinned conductances -> factor -> sweep -> host R
    w_pin = torch.from_numpy(g.w).pin_memory()
    r_pin = torch.empty(nq, dtype=torch.float64).pin_memory()
    e2e_times, h2d, d2h = [], 0, 0
    for _ in range(args.e2e_steps):
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        num2 = P.Numeric(ctx, sym, w_pin.numpy())
        h2d = ctx.last_stats()["h2d_bytes"]
        P.query(ctx, sym, num2, r_pin.numpy())
        st = ctx.last_stats()
        d2h = st["d2h_bytes"]
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
        num2.close()
        del num2
    t_e2e = dist_max(max(e2e_times), dist, f"cuda:{local}")
    # the e2e result must equal the device-resident result
    same = bool(np.array_equal(r_pin.numpy(), R.cpu().numpy()))
    del R
    # the other two patterns of the path on the same GPU (one replica only: they are
    # measured once, not per rank)
    extras = {x for x in args.extras.split(",") if x} if (world == 1 and
                                                         args.workload == "pdn1m") else set()
    batch256 = serve = None
    if "batch" in extras:
        torch.cuda.empty_cache()
        batch256 = measure_batch(args, ctx, stream, fp64_peak)
    if "serve" in extras:
        torch.cuda.empty_cache()
        serve = measure_serve(args, ctx, tiles["qcap"] if tiles else None)

    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    algo_flops = 2.0 * info["walk_entries"]          # per step
    achieved_tf = algo_flops / step_s / 1e12
    walk_gbs = 8.0 * info["walk_entries"] / step_s / 1e9
    line = {
        "metric": metric_of(args.workload), "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * step_s,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(args.workload), "n": g.n, "edges": nq,
                   "queries_per_step": nq, "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2: %.2f GB factor panels + %.1f GB query fronts"
                         % (8e-9 * info["nnz_l"], 1e-9 * info["device_bytes"])},
        "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": fp64_peak,
                     "unit": "TFLOP/s", "frac": achieved_tf / fp64_peak if fp64_peak else None,
                     "traffic": profiled_traffic(info, launches // args.steps),
                     "traffic_note": "DRAM bytes per k_sweep launch: the ncu capture of the "
                                     "512x512 grid's sweep (profiles/), scaled by the query-"
                                     "front bytes carried between levels",
                     "kernel": "k_sweep (FP64 DFMA; peak = DFMA throughput measured live; "
                               "mma.sync f64 m8n8k4 %.3f, m16n8k4 %.3f, m16n8k8 %.3f, "
                               "m16n8k16 %.3f TFLOP/s, DFMA and m8n8k4 at once %.3f)"
                               % (shapes64["m8n8k4"], shapes64["m16n8k4"], shapes64["m16n8k8"],
                                  shapes64["m16n8k16"], peaks64["dfma_with_dmma"]),
                     "fp64_tflops": {"dfma": fp64_peak, **{"mma_" + k: v
                                                           for k, v in shapes64.items()},
                                     "dfma_with_mma_m8n8k4": peaks64["dfma_with_dmma"]},
                     "algorithmic": "2 flops x W walk entries per step, W = %d" % info["walk_entries"]},
        "hbm_walk": {"achieved_gbs": walk_gbs, "peak_gbs": hbm or HBM_FALLBACK_GBS,
                     "frac": walk_gbs / (hbm or HBM_FALLBACK_GBS),
                     "peak_source": "measured" if hbm else "fallback",
                     "bytes_per_step": 8 * info["walk_entries"]},
        "e2e": {"value": job_throughput(nq, world, t_e2e), "unit": UNIT,
                "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "includes": "factor + sweep",
                "matches_device_result": same,
                "e2e_with_analyze": {"value": job_throughput(nq, world, t_e2e + t_analyze),
                                     "unit": UNIT, "t_analyze_s": t_analyze,
                                     "includes": "host analysis (peers_analyze) + factor + "
                                                 "sweep"}},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "tiles": tiles,
        "next1_blockinv": blockinv,
        "next2_selinv": selinv,
        "batch256": batch256,
        "serve": serve,
        "analysis": {"t_analyze_s": t_analyze, "nsuper": info["nsuper"],
                     "levels": info["levels"], "nnz_l": info["nnz_l"],
                     "walk_fma": info["walk_fma"]},
    }
    if oracle_proc is not None:
        p, q = oracle_proc
        res = q.get()
        p.join()
        tq = res["times"][0]
        line["cpu_baseline"] = {"value": res["sample"] / tq, "unit": UNIT, "cores": res["cores"],
                                "kind": "oracle",
                                "sample": f"{res['sample']} seeded edges of the same workload, "
                                          f"per-query path solves timed (oracle factor "
                                          f"{res['t_factor_s']:.1f} s untimed)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ batched graphs

def measure_batch(args, ctx, stream, dfma_peak, tiles_cache=True):
    """256 independent graphs swept together (one persistent launch per aligned level, CUDA
    graph replay), against the same graphs swept one at a time on the same GPU.  Returns the
    measurement as a dict (the `batch256` object of the default line)."""
    import torch
    from paper_2606_31535_b300 import inputs as I
    from paper_2606_31535_b300 import peers as P

    t0 = time.time()
    graphs = I.batch_graphs()
    t_gen = time.time() - t0
    t0 = time.time()
    syms = [P.Symbolic.of(g) for g in graphs]
    t_analyze = time.time() - t0
    t0 = time.time()
    nums = [P.Numeric(ctx, s) for s in syms]
    torch.cuda.synchronize()
    t_factor = time.time() - t0
    tiles = None
    if not args.no_autotune:
        # tune on the largest graph (cached per GPU and size class), then tile every plan alike
        big = max(range(len(syms)), key=lambda i: syms[i].info()["walk_entries"])
        tiles = P.autotune(ctx, syms[big], nums[big], tuning_cache())
        for s, m in zip(syms, nums):
            P.retile(ctx, s, m, tiles["qcap"])
    batch = P.Batch(ctx, syms, nums, cuda_graph=True)
    binfo = batch.info()
    nq = sum(s.nq for s in syms)
    W = sum(s.info()["walk_entries"] for s in syms)
    levels = sum(s.info()["levels"] for s in syms)
    outs = [torch.empty(s.nq, dtype=torch.float64, device="cuda:0") for s in syms]

    def timed(fn, k):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e-3 / k

    def batched():
        batch.query(outs)

    def one_at_a_time():
        for s, m, o in zip(syms, nums, outs):
            P.query(ctx, s, m, o)

    for _ in range(args.warmup):
        batched()
    clk = start_clocks(0)
    t_batch = timed(batched, args.steps)
    clocks = stop_clocks(*clk)
    ref = [o.clone() for o in outs]
    for _ in range(max(1, args.warmup // 2)):
        one_at_a_time()
    t_single = timed(one_at_a_time, args.steps)
    same = all(bool(torch.equal(a, b)) for a, b in zip(ref, outs))

    # end to end: pinned conductances -> factor every graph -> batched sweep -> host results
    pins = [torch.from_numpy(g.w).pin_memory() for g in graphs]
    hosts = [torch.empty(s.nq, dtype=torch.float64).pin_memory().numpy() for s in syms]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nums2, h2d = [], 0
    for s, w in zip(syms, pins):
        nums2.append(P.Numeric(ctx, s, w.numpy()))
        h2d += ctx.last_stats()["h2d_bytes"]
    b2 = P.Batch(ctx, syms, nums2, cuda_graph=False)
    b2.query(hosts)
    d2h = ctx.last_stats()["d2h_bytes"]
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    b2.close()
    for m in nums2:
        m.close()
    same_e2e = all(bool(np.array_equal(h, r.cpu().numpy())) for h, r in zip(hosts, ref))
    batch.close()
    for m in nums:
        m.close()
    del outs, ref

    achieved_tf = 2.0 * W / t_batch / 1e12
    return {
        "workload": workload_name("batch256"), "graphs": len(graphs),
        "nodes": int(sum(g.n for g in graphs)), "edges": nq,
        "value": nq / t_batch, "unit": UNIT, "ms_per_step": 1e3 * t_batch,
        "steps": args.steps, "warmup": args.warmup,
        "one_at_a_time": {"value": nq / t_single, "ms_per_step": 1e3 * t_single,
                          "launches": levels},
        "speedup_vs_one_at_a_time": t_single / t_batch,
        "same_results": same,
        "batched": {"launches": binfo["launches"], "items": binfo["items"], "cuda_graph": True},
        "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": dfma_peak,
                     "unit": "TFLOP/s", "frac": achieved_tf / dfma_peak,
                     "kernel": "k_sweep_multi (2 flops x W walk entries per step, W = %d)" % W},
        "e2e": {"value": nq / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "includes": "factor all 256 + batched sweep",
                "matches_device_result": same_e2e},
        "gpu_launches": int(binfo["launches"] * args.steps),
        "clocks": clocks,
        "tiles": tiles,
        "l2": "inputs larger than L2: %.2f GB of factors and fronts" % (1e-9 * binfo["device_bytes"]),
        "analysis": {"t_generate_s": t_gen, "t_analyze_s": t_analyze, "t_factor_s": t_factor,
                     "walk_entries": W},
    }


def run_batch(args):
    import torch
    from paper_2606_31535_b300 import peers as P
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    ctx = P.Context(0, stream)
    res = measure_batch(args, ctx, stream, ctx.fp64_peaks()["dfma"])
    line = {
        "metric": "edge queries/s, batched all-edge sweep of 256 graphs (FP64)",
        "value": res["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": res["workload"], "graphs": res["graphs"], "nodes": res["nodes"],
                   "edges": res["edges"], "l2": res["l2"]},
    }
    line.update({k: res[k] for k in ("one_at_a_time", "speedup_vs_one_at_a_time",
                                     "same_results", "batched", "roofline", "e2e",
                                     "gpu_launches", "clocks", "tiles", "analysis")})
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ serving stream

def _replay(P, reqs, arrivals, server_kw):
    """Submits each request at its arrival time (relative to now) to a fresh server and
    waits for all; returns (latencies, server stats)."""
    import threading
    sv = P.Server(0, **server_kw)
    tickets = [None] * len(reqs)
    t0 = time.perf_counter()

    def submitter():
        for i, (g, qu, qv) in enumerate(reqs):
            delay = arrivals[i] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets[i] = sv.submit(g, qu, qv)

    th = threading.Thread(target=submitter)
    th.start()
    lat = []
    for i in range(len(reqs)):
        while tickets[i] is None:
            time.sleep(0.001)
        _, l = sv.wait(tickets[i])
        lat.append(l)
    th.join()
    st = sv.stats()
    sv.close()
    return np.array(lat), st


def _replay_plain(P, ctx, reqs, arrivals):
    """The same stream served one request at a time through the plain API (analyse, factor,
    sweep), in arrival order; latency = completion - arrival."""
    t0 = time.perf_counter()
    lat, nq = [], 0
    for i, (g, qu, qv) in enumerate(reqs):
        now = time.perf_counter() - t0
        if arrivals[i] > now:
            time.sleep(arrivals[i] - now)
        sym = P.Symbolic.of(g, 0, qu, qv)
        num = P.Numeric(ctx, sym)
        R = P.query(ctx, sym, num)
        nq += R.size
        lat.append(time.perf_counter() - t0 - arrivals[i])
        num.close()
        sym.close()
    wall = time.perf_counter() - t0 - arrivals[0]
    return np.array(lat), nq / wall


def _lat(lat, qps, extra=None):
    d = {"qps": qps, "p50_s": float(np.percentile(lat, 50)),
         "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
         "max_s": float(lat.max())}
    d.update(extra or {})
    return d


def measure_serve(args, ctx, qcap=None):
    """The serving stream (Poisson arrivals of graph + query-set requests) at the offered
    loads of --rho, served three ways on the same GPU: the server with continuous batching,
    the same server admitting one request at a time, and the plain API one request at a time
    in arrival order.  The load is a fraction of the GPU's one-at-a-time service rate: rho =
    arrival rate x mean device seconds of a request's factorization + sweep, measured first,
    request by request, with the library's own CUDA-event timing.  Returns a dict (the
    `serve` object of the default line)."""
    from paper_2606_31535_b300 import inputs as I
    from paper_2606_31535_b300 import peers as P

    t0 = time.time()
    reqs = [I.serve_request(i) for i in range(args.requests)]
    t_gen = time.time() - t0
    opt = None
    if qcap is not None:
        opt = P.Options()
        opt.qcap[:] = list(qcap)
    # calibration: every request alone, device time of its factorization and sweep
    ctx.set_timing(True)
    gpu_s, host_s, nq_total = [], [], 0
    for g, qu, qv in reqs:
        t0 = time.perf_counter()
        sym = P.Symbolic.of(g, 0, qu, qv, options=opt)
        host_s.append(time.perf_counter() - t0)
        num = P.Numeric(ctx, sym)
        f_s = ctx.last_stats()["factor_s"]
        P.query(ctx, sym, num)
        gpu_s.append(f_s + ctx.last_stats()["sweep_s"])
        nq_total += sym.nq
        num.close()
        sym.close()
    ctx.set_timing(False)
    mean_gpu = float(np.mean(gpu_s))
    workers = max(2, min(8, (os.cpu_count() or 4) // 2))
    loads = []
    for rho in [float(x) for x in args.rho.split(",") if x]:
        rate = rho / mean_gpu
        arrivals = I.poisson_arrivals(len(reqs), rate, seed=4)
        arrivals -= arrivals[0]
        lat_b, st_b = _replay(P, reqs, arrivals, {"max_active": 64, "workers": workers,
                                                  "options": opt})
        lat_1, st_1 = _replay(P, reqs, arrivals, {"max_active": 1, "workers": workers,
                                                  "options": opt})
        lat_p, qps_p = _replay_plain(P, ctx, reqs, arrivals)
        loads.append({
            "rho": rho, "arrival_rate_per_s": rate,
            "continuous_batching": _lat(lat_b, st_b["qps"], {
                "steps": st_b["steps"], "max_step_requests": st_b["max_step_requests"],
                "request_steps": st_b["request_steps"], "peak_bytes": st_b["peak_bytes"]}),
            "one_at_a_time_on_gpu": _lat(lat_1, st_1["qps"], {
                "steps": st_1["steps"],
                "note": "same server and workers, one admitted request at a time"}),
            "plain_api_fifo": _lat(lat_p, qps_p, {
                "note": "analyse + factor + sweep per request through the plain API, in "
                        "arrival order"}),
        })
    return {
        "workload": workload_name("serve"), "requests": len(reqs), "queries": int(nq_total),
        "gpu_service_s": {"mean": mean_gpu, "p50": float(np.median(gpu_s)),
                          "max": float(np.max(gpu_s)), "sum": float(np.sum(gpu_s)),
                          "what": "device seconds of peers_factor + peers_query per request, "
                                  "one request at a time (CUDA events)"},
        "host_analyze_s": {"mean": float(np.mean(host_s)), "max": float(np.max(host_s))},
        "workers": workers, "t_generate_s": t_gen, "loads": loads,
    }


def run_serve(args):
    import torch
    from paper_2606_31535_b300 import peers as P
    torch.cuda.set_device(0)
    ctx = P.Context(0)
    qcap = None
    if not args.no_autotune:
        from paper_2606_31535_b300 import inputs as I
        g0, qu0, qv0 = max((I.serve_request(i) for i in range(min(8, args.requests))),
                           key=lambda r: r[0].n)
        s0 = P.Symbolic.of(g0, 0, qu0, qv0)
        qcap = P.autotune(ctx, s0, P.Numeric(ctx, s0), tuning_cache())["qcap"]
    res = measure_serve(args, ctx, qcap)
    main_load = res["loads"][0]
    line = {
        "metric": "edge queries/s and p50/p99 request latency, served request stream (FP64)",
        "value": main_load["continuous_batching"]["qps"], "unit": UNIT, "n_gpus": 1,
        "steps": 1, "warmup": 0, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": res["workload"], "requests": res["requests"],
                   "queries": res["queries"], "workers": res["workers"]},
        "latency": {"p50_s": main_load["continuous_batching"]["p50_s"],
                    "p99_s": main_load["continuous_batching"]["p99_s"]},
        "serve": res,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.warmup < 0 or args.steps < 1:
        raise SystemExit("need --steps >= 1 and --warmup >= 0")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch256":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
