#!/usr/bin/env python3
"""Benchmark: Contour connected components (MM^h sweeps) on GB300.

Default workload: R-MAT scale 24 (16,777,216 vertices, 268,435,456 edges,
a/b/c/d = .57/.19/.19/.05, permuted ids), operator order 2, asynchronous,
convergence check every sweep -- the paper's default C-2 variant.  One step
is one complete ``cc_run`` (label init, sweeps to convergence, compress) on a
device-resident graph.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
(serial union-find) on the host instead.  Under torchrun every rank solves
its own replica graph (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import graphgen as gg  # noqa: E402

FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="rmat24",
                   help="rmat<scale> (default rmat24), grid4096, caterpillar, components64, batch<G> or delaunay-scaling")
    p.add_argument("--order", type=int, default=2)
    p.add_argument("--mode", choices=["async", "sync"], default="async")
    p.add_argument("--interval", type=int, default=1)
    p.add_argument("--no-variants", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-config3", action="store_true",
                   help="skip the R-MAT scale 27 and caterpillar lines of the default run")
    p.add_argument("--batch-graphs", type=int, default=4096,
                   help="also compare batched + learned vs plain on a batch-mix of this many graphs (0: off)")
    p.add_argument("--layout", choices=["coo", "csr", "csr-sym"], default="coo",
                   help="main handle: edge list, or the same graph kept as CSR (each edge once / both directions)")
    p.add_argument("--launch", choices=["graph", "host"], default="graph",
                   help="sweep loop as a conditional CUDA graph, or host-polled blocks (for profilers)")
    p.add_argument("--reorder", choices=["none", "src", "lowdeg", "hub", "degree"], default="hub",
                   help="cc_graph_reorder layout step once before timing (included in e2e)")
    p.add_argument("--config3-reorder", choices=["none", "lowdeg", "hub", "degree"], default="degree",
                   help="layout of the R-MAT 27 and caterpillar handles")
    p.add_argument("--entry", choices=["cc_run", "noalloc"], default="cc_run",
                   help="cc_run (conditional CUDA-graph loop) or cc_run_noalloc (host-polled "
                        "plain launches of the same sweep kernel; profilers can see each sweep)")
    return p.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------

def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def whole_job_rate(units_per_rank: float, ms_local: float, world: int):
    """(units of all ranks per second, max ms over ranks): every rank solves the
    same amount of work; the job takes as long as its slowest rank."""
    ms = max_over_ranks(ms_local, world)
    return units_per_rank * world / (ms * 1e-3), ms


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def REORDER(cc):
    return {"none": 0, "src": cc.CC_REORDER_SRC, "lowdeg": cc.CC_REORDER_LOWDEG, "hub": cc.CC_REORDER_HUB,
            "degree": cc.CC_REORDER_DEGREE}


def main_config(args, cfg, n, m):
    """The workload description both arms print (identical for the same flags)."""
    return dict(cfg, n=n, m=m, order=args.order, mode=args.mode, check_interval=args.interval,
                layout={"coo": "edge list", "csr": "native CSR, each edge in its src row",
                        "csr-sym": "native CSR, each edge in both rows"}[args.layout],
                ids="int32", parallelism=f"replicas x{args.gpus}" if args.gpus > 1 else "single GPU",
                l2="inputs larger than L2: edge list %.2f GB streamed every sweep" % (8 * m / 1e9))


class OracleJob:
    """The oracle's serial union-find on a background thread (the C call
    releases the GIL), timed; its labels check the GPU labels of the same
    graph."""

    def __init__(self, n, s_host, d_host):
        import threading

        import oracle
        oracle.build()
        self.result = None
        self.error = None

        def run():
            try:
                t0 = time.perf_counter()
                lab = oracle.uf_labels(n, s_host, d_host)
                self.result = (lab, time.perf_counter() - t0)
            except Exception as e:  # noqa: BLE001
                self.error = repr(e)

        self.thread = threading.Thread(target=run, daemon=True)
        self.thread.start()

    def get(self):
        self.thread.join()
        if self.error:
            raise RuntimeError(f"oracle failed: {self.error}")
        return self.result


def make_workload(name: str, device, seed: int):
    if name.startswith("rmat"):
        scale = int(name[4:])
        s, d = gg.rmat(scale, seed=seed, device=device)
        return (1 << scale), s, d, {"workload": f"rmat-scale{scale}",
                                    "graph": "R-MAT a/b/c/d=.57/.19/.19/.05, edge factor 16, ids permuted"}
    if name == "caterpillar":
        s, d = gg.caterpillar(1 << 24, seed=seed, device=device)
        return 1 << 28, s, d, {"workload": "caterpillar-2^24",
                               "graph": "2^24-vertex path backbone + 15 leaves per backbone vertex, ids permuted"}
    if name == "grid4096":
        s, d = gg.grid(4096, 4096, seed=seed, device=device)
        return 4096 * 4096, s, d, {"workload": "grid-4096x4096", "graph": "4-neighbour grid, 5% edges deleted, ids permuted"}
    n, s, d = gg.components64(seed=seed, device=device)
    return n, s, d, {"workload": "components64", "graph": "32 paths + 32 ER(deg 8)+spanning path, 1024 vertices each"}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, local_rank: int):
        self.proc = None
        self.index = self._physical_index(local_rank)

    @staticmethod
    def _physical_index(local_rank):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            parts = [p.strip() for p in vis.split(",") if p.strip()]
            if local_rank < len(parts) and parts[local_rank].isdigit():
                return parts[local_rank]
        return str(local_rank)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.index, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                rows.append((float(f[0]), float(f[1]), f[3:7], float(f[7]) if f[7] not in ("", "[N/A]") else 0.0))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [r for r in rows if r[3] > 0] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in loaded for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(loaded)}


# ---------------------------------------------------------------------------
# CPU baseline (the oracle, as it stands)
# ---------------------------------------------------------------------------

def cpu_oracle_rate(n, s_host, d_host, target_s: float):
    """Serial union-find on a prefix of the edge list sized to ~target_s seconds."""
    import oracle
    oracle.build()
    m = s_host.numel()
    probe = max(1, m // 64)
    t0 = time.perf_counter()
    oracle.uf_labels(n, s_host[:probe], d_host[:probe])
    dt = max(time.perf_counter() - t0, 1e-6)
    k = int(min(m, probe * max(1.0, target_s / dt)))
    t0 = time.perf_counter()
    oracle.uf_labels(n, s_host[:k], d_host[:k])
    dt = time.perf_counter() - t0
    return k / dt, k, dt


def cpu_contour_rate(n, s_host, d_host, order):
    """The multicore CPU form of the method (asynchronous Contour with OpenMP,
    the paper's own setting) on all host cores, whole graph, one solve."""
    import oracle
    try:
        oracle.build_omp()
    except Exception as e:  # noqa: BLE001
        return {"unavailable": f"gcc -fopenmp failed: {e}"}
    s_np, d_np = s_host.numpy(), d_host.numpy()
    oracle.omp_contour(1024, s_np[:0], d_np[:0], order=order)  # load the library outside the timing
    t0 = time.perf_counter()
    _, iters, used = oracle.omp_contour(n, s_np, d_np, order=order)
    dt = time.perf_counter() - t0
    m = s_np.size
    return {"value": m / dt, "unit": "edges/s", "cores": used, "kind": "contour-async-openmp",
            "sample": f"whole graph ({m:,} edges, as generated), order {order}, asynchronous, "
                      f"{iters} iterations, {dt:.2f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    n, s, d, cfg = make_workload(args.workload, dev, gg.BASE_SEED)
    s_h, d_h = s.cpu(), d.cpu()
    del s, d
    m = s_h.numel()
    per_step = max(2.0, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    rates = []
    for i in range(args.warmup + args.steps):
        r, k, dt = cpu_oracle_rate(n, s_h, d_h, per_step)
        if i >= args.warmup:
            rates.append((r, k, dt))
    tot_edges = sum(k for _, k, _ in rates)
    tot_t = sum(dt for _, _, dt in rates)
    value = tot_edges / tot_t
    sample = f"serial union-find over the first {rates[-1][1]:,} of {m:,} edges (all {n:,} vertices) per step"
    cfg = main_config(args, cfg, n, m)
    line = {"impl": "reference", "metric": "CC edges/sec (m / solve time)", "value": value,
            "unit": "edges/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_t / len(rates), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def _source_sha(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2311_02811_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def _traffic_for(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary of this kernel on
    this workload, if it matches the kernel's sources (the files listed in the
    entry, default mm_kernels.cuh)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        ent = json.load(open(path)).get(f"{kernel}@{workload}")
        if ent and ent.get("source_sha256") == _source_sha(ent.get("sources", ["mm_kernels.cuh"])):
            return ent.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        pass
    return None


def _peaks():
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return FALLBACK_HBM_GBS, "fallback"


class _NoallocStats:
    def __init__(self, sweeps):
        self.sweeps = sweeps
        self.loop_ms = float("nan")


def timed_runs(cc, g, out, n_steps, order, mode, interval, stream, edges=None):
    """n_steps solves between two CUDA events on the launching stream.

    ``edges`` = (n, src, dst) switches to cc_run_noalloc (plain launches)."""
    stats = []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(n_steps):
        if edges is None:
            stats.append(cc.cc_run(g, out, order, mode, interval))
        else:
            n, s, d, m = edges
            stats.append(_NoallocStats(cc.cc_run_noalloc(n, s, d, out, order, mode, interval,
                                                         stream=stream.cuda_stream, m=m)))
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1), stats


def run_ours(args, rank, world, local):
    import paper_2311_02811_gb300 as cc
    assert torch.cuda.is_available(), "bench needs a CUDA device"
    dev = torch.device("cuda", torch.cuda.current_device())
    mode = cc.CC_ASYNC if args.mode == "async" else cc.CC_SYNC
    seed = gg.BASE_SEED + rank
    n, s, d, cfg = make_workload(args.workload, dev, seed)
    torch.cuda.empty_cache()  # release the generator's temporaries
    m = s.numel()
    stream = torch.cuda.current_stream()
    cpu_leg = rank == 0 and world == 1 and not args.no_cpu
    job = None
    if cpu_leg:
        # the oracle on the whole graph, on a host thread while the GPU works
        s_h, d_h = s.cpu(), d.cpu()
        job = OracleJob(n, s_h, d_h)
    if args.layout == "coo":
        g = cc.cc_init(n, s, d, stream=stream.cuda_stream)
    else:
        sym = args.layout == "csr-sym"
        off, cols = gg.to_csr(n, s, d, symmetric=sym)
        g = cc.cc_init(n, off, cols, m=cols.numel(), id_bits=32, on_device=True, stream=stream.cuda_stream,
                       layout=cc.CC_CSR_NATIVE_SYM if sym else cc.CC_CSR_NATIVE)
        if args.reorder != "none":
            raise SystemExit("--layout csr keeps the row order: use --reorder none")
    reorder = REORDER(cc)[args.reorder]
    if args.layout != "coo" and args.entry == "noalloc":
        raise SystemExit("--entry noalloc takes edge lists: use --layout coo")
    if reorder in (cc.CC_REORDER_HUB, cc.CC_REORDER_DEGREE) and args.entry == "noalloc":
        raise SystemExit("--entry noalloc takes plain edge lists in the caller's ids; use --reorder none/src/lowdeg")
    reorder_ms = None
    if reorder:
        t0 = time.perf_counter()
        cc.cc_graph_reorder(g, reorder)
        reorder_ms = 1e3 * (time.perf_counter() - t0)
    if args.launch == "host":
        cc.cc_graph_set_launch(g, cc.CC_LAUNCH_HOST)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    # the no-alloc entry runs the same sweep kernel on the handle's (possibly
    # reordered) edge arrays with host-polled plain launches
    edges = (n, *cc.cc_graph_edges(g), m) if args.entry == "noalloc" else None
    timed_runs(cc, g, out, args.warmup, args.order, mode, args.interval, stream, edges)

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    ms, stats = timed_runs(cc, g, out, args.steps, args.order, mode, args.interval, stream, edges)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    value, ms_max = whole_job_rate(m * args.steps, ms, world)
    timed_labels = out.cpu().numpy() if cpu_leg else None  # the last timed step's output

    sweeps = [st.sweeps for st in stats]
    loop_ms = sum(st.loop_ms for st in stats) if edges is None else ms
    tot_sweeps = sum(sweeps)
    B = 4
    if args.layout == "coo":
        per_sweep = 2 * B * m + B * n + (3 * B * n if mode == cc.CC_SYNC else 0)
        kernel = ("mm_sweep_prefix_kernel" if cc.cc_graph_perm(g)[0] else
                  "mm_sweep_hub_kernel" if cc.cc_graph_hubs(g)[1] > 0 else "mm_sweep_kernel")
    else:  # native CSR: columns, offsets and labels once per sweep
        nnz = m * (2 if args.layout == "csr-sym" else 1)
        per_sweep = B * nnz + 8 * (n + 1) + B * n + (3 * B * n if mode == cc.CC_SYNC else 0)
        kernel = "csr_sweep_kernel"
    sweep_ms = loop_ms / max(1, tot_sweeps)
    achieved = per_sweep / (sweep_ms * 1e-3) / 1e9
    peak, peak_kind = _peaks()
    kname = f"{kernel}<{args.order},{'sync' if mode == cc.CC_SYNC else 'async'},int32>"
    launches_per_run = [3 + sw * (2 if mode == cc.CC_SYNC else 1) + sw // args.interval for sw in sweeps]

    line = {
        "metric": "CC edges/sec (m / solve time)", "value": value, "unit": "edges/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": main_config(args, cfg, n, m),
        "run": {"sweep_loop": ("conditional CUDA graph" if args.launch == "graph" else "host-polled blocks"),
                "entry": args.entry,
                "edge_order": ("as generated (shuffled)" if not reorder else
                               f"cc_graph_reorder({args.reorder}) once before timing, "
                               f"{reorder_ms:.1f} ms host-timed; inside e2e_handle_reorder's timing"),
                "sweeps_per_step": statistics.median(sweeps)},
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": _traffic_for(kname, cfg["workload"]),
                     "alg_bytes_per_launch": per_sweep,
                     "launch_ms": sweep_ms,
                     "timing": "sweep-loop CUDA events on the launching stream / sweeps (includes the per-block check kernel)"},
        "clocks": clocks,
        "gpu_launches": sum(launches_per_run),
    }

    if not args.no_e2e:
        # the one-shot call a user with host edges makes, then the handle
        # pipelines (upload, [the timed handle's layout step], solve) for context
        line["e2e"] = e2e(cc, n, s, d, args, mode, world, stream, 0, "solve_host")
        line["e2e_handle"] = e2e(cc, n, s, d, args, mode, world, stream, 0, "handle")
        if reorder:
            line["e2e_handle_reorder"] = e2e(cc, n, s, d, args, mode, world, stream, reorder, "handle")
        e2e_labels = [line[k].pop("labels") for k in ("e2e", "e2e_handle", "e2e_handle_reorder") if k in line]

    if not args.no_variants and rank == 0:
        line["variants"] = variants(cc, g, out, n, m, args, dev, seed, stream, s, d)
    cc.cc_free(g)
    del out
    if rank == 0 and world == 1 and not args.no_config3 and args.workload.startswith("rmat"):
        line["config1"] = config1(cc, dev, stream, with_oracle=cpu_leg)
    cc.cc_release_memory()  # the handles' pooled memory goes back before the larger graphs
    if rank == 0 and world == 1 and not args.no_config3 and args.workload.startswith("rmat"):
        del s, d
        torch.cuda.empty_cache()
        line["config3"] = config3(cc, args, dev, stream, with_oracle=cpu_leg)
        cc.cc_release_memory()
        torch.cuda.empty_cache()
    if args.batch_graphs > 0 and rank == 0:
        line["batch"] = batch_compare(cc, args.batch_graphs, args, dev, stream, gg.BASE_SEED + 3)
    if rank == 0 and world == 1 and not args.no_config3 and args.workload.startswith("rmat"):
        # Section IV's delaunay_n10..n24 experiment on the Delaunay-style generator
        d = delaunay_scaling(cc, args, dev)
        line["delaunay_scaling"] = {"growth_n10_to_n24": d["growth"],
                                    "paper_growth_20_core_xeon": d["paper_growth_20_core_xeon"],
                                    "n24": {k: v for k, v in d["rows"][-1].items()}}

    if "config3" in line:
        finish_config3(line["config3"])
    if cpu_leg:
        want, dt = job.get()
        line["labels_match_oracle"] = bool(np.array_equal(timed_labels, want))
        if not args.no_e2e:
            line["e2e_labels_match_oracle"] = all(bool(np.array_equal(x, want)) for x in e2e_labels)
        line["cpu_baseline"] = {"value": m / dt, "unit": "edges/s", "cores": 1, "kind": "oracle",
                                "sample": f"serial union-find over all {m:,} edges and {n:,} vertices "
                                          f"of the timed graph, {dt:.1f} s; its labels are compared "
                                          "with the last timed step's (labels_match_oracle)"}
        line["cpu_parallel"] = cpu_contour_rate(n, s_h, d_h, args.order if args.order > 0 else 1024)
    if rank == 0:
        print(json.dumps(line), flush=True)


def e2e(cc, n, s, d, args, mode, world, stream, reorder=0, pipeline="solve_host"):
    """Same metric through the public API from pinned host buffers, copies
    included.  pipeline "solve_host": one cc_solve_host call (the upload
    overlapped with sweeps); "handle": cc_init (upload) + [cc_graph_reorder] +
    cc_run + cc_free.  Labels come back to pinned host memory."""
    s_h = s.cpu().pin_memory()
    d_h = d.cpu().pin_memory()
    out_h = torch.empty(n, dtype=torch.int32).pin_memory()
    m = s_h.numel()

    def one():
        if pipeline == "solve_host":
            cc.cc_solve_host(n, s_h, d_h, out_h, args.order, mode, args.interval, out_on_device=False,
                             stream=stream.cuda_stream)
            return
        g = cc.cc_init(n, s_h, d_h, on_device=False, stream=stream.cuda_stream)
        if reorder:
            cc.cc_graph_reorder(g, reorder)
        cc.cc_run(g, out_h, args.order, mode, args.interval, out_on_device=False)
        cc.cc_free(g)

    one()
    one()  # the library's memory pool has grown to the step's size
    steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    barrier(world)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        one()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    call = ("cc_solve_host" if pipeline == "solve_host" else
            "cc_init + " + ("cc_graph_reorder + " if reorder else "") + "cc_run + cc_free")
    return {"value": m * steps * world / (ms * 1e-3), "unit": "edges/s",
            "h2d_bytes_per_step": 2 * 4 * m, "d2h_bytes_per_step": 4 * n, "steps": steps,
            "ms_per_step": ms / steps, "call": call, "labels": out_h.numpy().copy()}


def measure_solves(cc, gh, o, mm, order, mode, c, stream, reps=3):
    """reps solves after one untimed one: edges/s, and the sweep loop's
    algorithmic bytes over its CUDA-event time as a fraction of the peak."""
    cc.cc_run(gh, o, order, mode, c)
    ms, st = timed_runs(cc, gh, o, reps, order, mode, c, stream)
    loop_ms = sum(x.loop_ms for x in st)
    alg = sum(x.alg_bytes for x in st)
    peak, _ = _peaks()
    return {"edges_per_s": mm * reps / (ms * 1e-3), "ms": ms / reps, "sweeps": st[-1].sweeps,
            "loop_ms": loop_ms / reps, "alg_bytes_per_solve": alg / reps,
            "roofline_frac": alg / (loop_ms * 1e-3) / 1e9 / peak}


def variants(cc, g, out, n, m, args, dev, seed, stream, s=None, d=None):
    res = {}

    def measure(gh, o, nn, mm, order, mode, c, reps=3):
        return measure_solves(cc, gh, o, mm, order, mode, c, stream, reps)

    for order, mode, name in [(2, cc.CC_SYNC, "o2-sync"), (4, cc.CC_ASYNC, "o4-async"),
                              (4, cc.CC_SYNC, "o4-sync"), (0, cc.CC_ASYNC, "full-async"),
                              (1, cc.CC_ASYNC, "o1-async"), (cc.CC_ORDER_11MM, cc.CC_ASYNC, "c11mm-async"),
                              (cc.CC_ORDER_1M1M, cc.CC_ASYNC, "c1m1m-async")]:
        res[f"{args.workload}/{name}"] = measure(g, out, n, m, order, mode, 1)
    if s is not None:
        # compaction takes plain edge lists: a lowdeg-reordered handle of the same graph
        gl = cc.cc_init(n, s, d, stream=stream.cuda_stream)
        cc.cc_graph_reorder(gl, cc.CC_REORDER_LOWDEG)
        for order, mode, name in [(0, cc.CC_ASYNC, "full-async-lowdeg"), (0, cc.CC_ASYNC_COMPACT, "full-compact-lowdeg"),
                                  (2, cc.CC_ASYNC, "o2-async-lowdeg")]:
            res[f"{args.workload}/{name}"] = measure(gl, out, n, m, order, mode, 1)
        cc.cc_free(gl)
    if s is not None and args.reorder != "degree":
        # the same graph renumbered by degree (labels mapped back to the caller's ids)
        gd = cc.cc_init(n, s, d, stream=stream.cuda_stream)
        cc.cc_graph_reorder(gd, cc.CC_REORDER_DEGREE)
        for order, mode, name in [(2, cc.CC_SYNC, "o2-sync"), (2, cc.CC_ASYNC, "o2-async"),
                                  (0, cc.CC_ASYNC, "full-async")]:
            res[f"{args.workload}-degree/{name}"] = measure(gd, out, n, m, order, mode, 1)
        cc.cc_free(gd)
    if os.path.exists(cc.SCHED_WEIGHTS_PATH):
        cc.load_default_scheduler()
        r = measure(g, out, n, m, cc.CC_ORDER_AUTO, cc.CC_ASYNC, 0)
        st = cc.cc_run(g, out, cc.CC_ORDER_AUTO, cc.CC_ASYNC, 0)
        r["schedule"] = [st.order, st.mode, st.check_interval]
        res[f"{args.workload}/learned"] = r
        cc.unload_scheduler()
    if s is not None and args.workload.startswith("rmat"):
        # the same graph kept as CSR (native row walk, no edge-list expansion):
        # each edge once in its src row, and stored in both rows (symmetric)
        for sym, name in [(False, "csr"), (True, "csr-sym")]:
            off, cols = gg.to_csr(n, s, d, symmetric=sym)
            layout = cc.CC_CSR_NATIVE_SYM if sym else cc.CC_CSR_NATIVE
            gc = cc.cc_init(n, off, cols, m=cols.numel(), id_bits=32, layout=layout, on_device=True,
                            stream=stream.cuda_stream)
            for order, mode, oname in [(2, cc.CC_ASYNC, "o2-async"), (0, cc.CC_ASYNC, "full-async"),
                                       (2, cc.CC_SYNC, "o2-sync")]:
                r = measure(gc, out, n, m, order, mode, 1)
                r["entries"] = int(cols.numel())
                res[f"{args.workload}-{name}/{oname}"] = r
            cc.cc_free(gc)
            del off, cols
            torch.cuda.empty_cache()
    if args.workload.startswith("rmat"):
        n2, s2, d2, _ = make_workload("grid4096", dev, seed)
        g2 = cc.cc_init(n2, s2, d2, stream=stream.cuda_stream)
        if args.reorder != "none":
            # the same one-time layout step as the main handle (a grid has no
            # vertex of degree >= 16, so the hub layout is the lowdeg one)
            cc.cc_graph_reorder(g2, REORDER(cc)[args.reorder])
        o2 = torch.empty(n2, dtype=torch.int32, device=dev)
        for order, mode, name in [(2, cc.CC_ASYNC, "o2-async"), (2, cc.CC_SYNC, "o2-sync"),
                                  (4, cc.CC_ASYNC, "o4-async"), (0, cc.CC_ASYNC, "full-async"),
                                  (0, cc.CC_ASYNC_COMPACT, "full-compact")]:
            res[f"grid4096/{name}"] = measure(g2, o2, n2, s2.numel(), order, mode, 1)
        cc.cc_free(g2)
    return res


def config1(cc, dev, stream, with_oracle):
    """The plain form of config 1: 64 components of 1,024 vertices (32 paths,
    32 ER with a spanning path), order 2, synchronous, check every sweep, on
    the edges as generated and after each layout step.  Its labels are
    compared with union-find and its sweep count with the Alg. 1 simulator
    (both on the host, a fraction of a second at this size).  The labels
    (256 KB) and edges (2.4 MB) fit in L2 and a solve takes 13 sweeps of a
    few microseconds each, so the time is launch and latency, not HBM."""
    n, s, d = gg.components64(device="cpu")
    sd, dd = s.to(dev), d.to(dev)
    res = {"graph": "components64", "n": n, "m": int(s.numel())}
    want = it = None
    if with_oracle:
        import oracle
        want = oracle.uf_labels(n, s, d)
        _, it, _, _ = oracle.contour_sync(n, s, d, 2)
        res["simulator_sweeps"] = it
    peak, _ = _peaks()
    out = torch.empty(n, dtype=torch.int32, device=dev)
    for layout in ("none", "lowdeg", "hub", "degree"):
        g = cc.cc_init(n, sd, dd, stream=stream.cuda_stream)
        if layout != "none":
            cc.cc_graph_reorder(g, REORDER(cc)[layout])
        r = measure_solves(cc, g, out, int(s.numel()), 2, cc.CC_SYNC, 1, stream, reps=5)
        if want is not None:
            r["labels_match_oracle"] = bool(np.array_equal(out.cpu().numpy(), want))
            if layout != "degree":  # renumbered ids take their own sequence of states (reading 20)
                r["sweeps_match_simulator"] = r["sweeps"] == it
        res[f"o2-sync/{layout}"] = r
        cc.cc_free(g)
    return res


def config3(cc, args, dev, stream, with_oracle):
    """The two largest single graphs: R-MAT scale 27 (2^31 edges, so 64-bit
    edge indices; labels 537 MB, larger than L2) and the caterpillar (2^24
    backbone vertices with 15 leaves each: n = 2^28, diameter 2^24 + 1, the
    d_max stress case of Lemma 2 and the Theorem).  Each is solved on the same
    layout as the main handle.  R-MAT 27's labels are compared with the
    oracle's union-find (run on a host thread; resolved by finish_config3);
    the caterpillar is connected, so every label must be 0."""
    reorder = REORDER(cc)[args.config3_reorder]
    res = {}
    for name in ("rmat27", "caterpillar"):
        t0 = time.perf_counter()
        if name == "rmat27":
            n = 1 << 27
            s, d = gg.rmat(27, seed=gg.BASE_SEED, device=dev)
            graph = "R-MAT a/b/c/d=.57/.19/.19/.05, scale 27, edge factor 16, ids permuted"
        else:
            B = 1 << 24
            n = 16 * B
            s, d = gg.caterpillar(B, seed=gg.BASE_SEED, device=dev)
            graph = "caterpillar: 2^24-vertex path backbone + 15 leaves per backbone vertex, ids permuted"
        torch.cuda.synchronize()
        gen_s = time.perf_counter() - t0
        torch.cuda.empty_cache()
        m = s.numel()
        job = OracleJob(n, s.cpu(), d.cpu()) if (with_oracle and name == "rmat27") else None
        g = cc.cc_init(n, s, d, stream=stream.cuda_stream)
        reorder_ms = None
        if reorder:
            t0 = time.perf_counter()
            cc.cc_graph_reorder(g, reorder)
            reorder_ms = 1e3 * (time.perf_counter() - t0)
        del s, d  # the reordered handle owns its edges
        torch.cuda.empty_cache()
        out = torch.empty(n, dtype=torch.int32, device=dev)
        ent = {"graph": graph, "n": n, "m": m, "edge_index_bits": 64 if m >= 1 << 31 else 32,
               "generation_s": gen_s, "layout": args.config3_reorder, "reorder_ms": reorder_ms,
               "labels_bytes": 4 * n, "alg_bytes_per_async_sweep": 8 * m + 4 * n}
        forms = {}
        for order, mode, fname in [(2, cc.CC_ASYNC, "o2-async"), (0, cc.CC_ASYNC, "full-async"),
                                   (2, cc.CC_SYNC, "o2-sync")]:
            forms[fname] = measure_solves(cc, g, out, m, order, mode, 1, stream, reps=2)
            if fname == "o2-async":
                labels = out.cpu().numpy()
        ent["forms"] = forms
        kern = {"degree": "mm_sweep_prefix_kernel", "hub": "mm_sweep_hub_kernel"}.get(args.config3_reorder,
                                                                                     "mm_sweep_kernel")
        wl = "rmat-scale27" if name == "rmat27" else "caterpillar-2^24"
        forms["o2-async"]["kernel"] = f"{kern}<2,async,int32>"
        forms["o2-async"]["traffic_per_sweep"] = _traffic_for(f"{kern}<2,async,int32>", wl)
        forms["o2-sync"]["kernel"] = f"{kern}<2,sync,int32>"
        forms["o2-sync"]["traffic_per_sweep"] = _traffic_for(f"{kern}<2,sync,int32>", wl)
        if name == "caterpillar":
            d_max = B + 1
            bound = math.ceil(math.log(d_max) / math.log(1.5)) + 1
            ent["theorem_bound_sync_o2"] = {"d_max": d_max, "bound": bound,
                                            "sweeps_with_detection": forms["o2-sync"]["sweeps"],
                                            "within_bound": forms["o2-sync"]["sweeps"] <= bound + 1}
            ent["labels_match_closed_form"] = bool((labels == 0).all())
        else:
            ent["_pending"] = (job, labels) if job is not None else None
        cc.cc_free(g)
        del out, labels
        torch.cuda.empty_cache()
        res[name] = ent
    return res


def finish_config3(res):
    """Join the oracle runs of config3() and record their checks."""
    for ent in res.values():
        pend = ent.pop("_pending", None)
        if pend is None:
            continue
        job, labels = pend
        want, dt = job.get()
        ent["labels_match_oracle"] = bool(np.array_equal(labels, want))
        ent["cpu_baseline"] = {"value": ent["m"] / dt, "unit": "edges/s", "cores": 1, "kind": "oracle",
                               "sample": f"serial union-find over all {ent['m']:,} edges, {dt:.1f} s"}


def make_batch(n_graphs: int, device, seed: int):
    t0 = time.perf_counter()
    vo, eo, s, d, params = gg.batch_mix(n_graphs, seed=seed, device=device)
    torch.cuda.synchronize()
    return vo.numpy(), eo.numpy(), s, d, params, time.perf_counter() - t0


def batch_compare(cc, G, args, dev, stream, seed):
    """The batch mix solved four ways with identical output: one cc_run per
    graph (the plain form) and one batched launch, each with the plain
    order-2 synchronous schedule and with the paper's C-2 (order 2, async);
    plus the batched launch with the learned per-graph schedule."""
    vo, eo, s, d, params, gen_s = make_batch(G, dev, seed)
    torch.cuda.empty_cache()
    total_n, total_m = int(vo[-1]), int(eo[-1])
    t0 = time.perf_counter()
    plan = cc.cc_batch_init(vo, eo, s, d, autotune=1, stream=stream.cuda_stream)
    tune_s = time.perf_counter() - t0
    reorder_s = None
    if args.reorder != "none":
        t0 = time.perf_counter()
        cc.cc_batch_reorder(plan)
        reorder_s = time.perf_counter() - t0
    out_b = torch.empty(total_n, dtype=torch.int32, device=dev)
    res = {}

    def ev_ms(fn, reps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    reps = max(1, min(args.steps, 5))
    peak, _ = _peaks()
    nv, me = np.diff(vo).astype(np.float64), np.diff(eo).astype(np.float64)

    def batch_frac(sweeps, ms, sync):
        # algorithmic bytes of every graph's sweeps (sync: plus L_u and the copy)
        per = 8 * me + 4 * nv + (12 * nv if sync else 0)
        alg = float((np.asarray(sweeps, np.float64) * per).sum())
        return alg, alg / (ms * 1e-3) / 1e9 / peak

    for name, (order, md, c) in [("batched-plain-o2-sync", (2, cc.CC_SYNC, 1)),
                                 ("batched-c2-async", (2, cc.CC_ASYNC, 1)),
                                 ("batched-full-async", (0, cc.CC_ASYNC, 1))]:
        first = ev_ms(lambda: cc.cc_batch_run(plan, out_b, order, md, c), 1)
        ms = ev_ms(lambda: cc.cc_batch_run(plan, out_b, order, md, c), reps)
        sw = cc.cc_batch_run(plan, out_b, order, md, c)[0]
        alg, frac = batch_frac(sw, ms, md == cc.CC_SYNC)
        res[name] = {"ms": ms, "first_call_ms": first, "edges_per_s": total_m / (ms * 1e-3),
                     "alg_bytes": alg, "roofline_frac": frac}
    ref = out_b.clone()
    learned = os.path.exists(cc.SCHED_WEIGHTS_PATH)
    per_kind = None
    if learned:
        cc.load_default_scheduler()
        first = ev_ms(lambda: cc.cc_batch_run(plan, out_b, cc.CC_ORDER_AUTO, cc.CC_ASYNC, 0), 1)
        ms = ev_ms(lambda: cc.cc_batch_run(plan, out_b, cc.CC_ORDER_AUTO, cc.CC_ASYNC, 0), reps)
        sweeps = np.asarray(cc.cc_batch_run(plan, out_b, cc.CC_ORDER_AUTO, cc.CC_ASYNC, 0)[0])
        kinds = np.array([p["kind"] for p in params])
        ns, ms_ = np.diff(vo), np.diff(eo)
        budget = cc.cc_batch_tuning(plan)[0]
        per_kind = {k: {"graphs": int((kinds == k).sum()), "edges": int(ms_[kinds == k].sum()),
                        "in_shared_memory": int(((kinds == k) & (ns * 4 <= budget)).sum()),
                        "sweeps_mean": float(sweeps[kinds == k].mean()), "sweeps_max": int(sweeps[kinds == k].max())}
                    for k in sorted(set(kinds.tolist()))}
        alg, frac = batch_frac(sweeps, ms, False)
        res["batched-learned"] = {"ms": ms, "first_call_ms": first, "edges_per_s": total_m / (ms * 1e-3),
                                  "alg_bytes": alg, "roofline_frac": frac,
                                  "note": "first call includes the feature pass and inference; bytes counted "
                                          "as asynchronous sweeps (the batch model picks asynchronous orders)"}
        identical_learned = bool(torch.equal(out_b, ref))
        cc.unload_scheduler()
    handles = []
    ps, pd = cc.cc_batch_edges(plan)  # the same (possibly reordered) edges as the batched form
    for g in range(G):
        a, b = int(eo[g]), int(eo[g + 1])
        handles.append((cc.cc_init(int(vo[g + 1] - vo[g]), ps + 4 * a, pd + 4 * a, m=b - a, id_bits=32,
                                   on_device=True, stream=stream.cuda_stream),
                        int(vo[g]), int(vo[g + 1])))
    out_p = torch.empty(total_n, dtype=torch.int32, device=dev)

    def plain(order, md):
        for h, v0, v1 in handles:
            cc.cc_run(h, out_p[v0:v1], order, md, 1)

    for name, (order, md) in [("plain-o2-sync", (2, cc.CC_SYNC)), ("plain-c2-async", (2, cc.CC_ASYNC))]:
        plain(order, md)
        ms = ev_ms(lambda: plain(order, md), max(1, min(reps, 2)))
        res[name] = {"ms": ms, "edges_per_s": total_m / (ms * 1e-3)}
    identical = bool(torch.equal(out_p, ref)) and (identical_learned if learned else True)
    for h, _, _ in handles:
        cc.cc_free(h)
    tuning = cc.cc_batch_tuning(plan)
    cc.cc_batch_free(plan)
    best_batched = "batched-learned" if learned else "batched-c2-async"
    return {"workload": f"batch-mix-{G}", "graphs": G, "n": total_n, "m": total_m, "per_kind_learned": per_kind,
            "generation_s": gen_s, "plan_and_autotune_s": tune_s,
            "edge_order": ("as generated (shuffled)" if reorder_s is None else
                           f"cc_batch_reorder once before timing ({reorder_s:.2f} s); the plain "
                           "per-graph handles use the same reordered edges"),
            "tuning": {"smem_budget": tuning[0], "threads": tuning[1], "edges_per_thread": tuning[2]},
            "forms": res, "identical_output": identical,
            "speedup_batched_learned_vs_plain": res["plain-o2-sync"]["ms"] / res[best_batched]["ms"],
            "speedup_batched_learned_vs_plain_c2": res["plain-c2-async"]["ms"] / res[best_batched]["ms"]}


def run_batch(args, rank, world, local):
    """Config-4 style line: the batch mix, batched + learned vs plain."""
    import paper_2311_02811_gb300 as cc
    dev = torch.device("cuda", torch.cuda.current_device())
    G = int(args.workload[5:])
    stream = torch.cuda.current_stream()
    b = batch_compare(cc, G, args, dev, stream, gg.BASE_SEED + 3 + rank)
    key = "batched-learned" if "batched-learned" in b["forms"] else "batched-c2-async"
    ms = b["forms"][key]["ms"]
    value, ms_max = whole_job_rate(b["m"], ms, world)
    line = {"metric": "CC edges/sec (m / solve time), batched + learned vs plain", "value": value,
            "unit": "edges/s", "n_gpus": world, "steps": args.steps, "warmup": 1,
            "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": b["workload"], "graphs": G, "n": b["n"], "m": b["m"], "form": key},
            "batch": b}
    if rank == 0:
        print(json.dumps(line), flush=True)


PAPER_DELAUNAY_GROWTH = {"C-2": 895, "C-1m1m": 1072, "C-m": 1268, "C-11mm": 1329, "C-Syn": 2705}


def delaunay_scaling(cc, args, dev):
    """Solve time of each Contour variant on Delaunay-style graphs n = 2^10..2^24
    and its growth from n10 to n24 (the paper's delaunay_n10..n24 experiment)."""
    variants = {"C-Syn": (2, cc.CC_SYNC), "C-1": (1, cc.CC_ASYNC), "C-2": (2, cc.CC_ASYNC),
                "C-m": (0, cc.CC_ASYNC), "C-11mm": (cc.CC_ORDER_11MM, cc.CC_ASYNC),
                "C-1m1m": (cc.CC_ORDER_1M1M, cc.CC_ASYNC)}
    rows = []
    for k in range(10, 25):
        n, s, d = gg.delaunay_like(k, device=dev)
        g = cc.cc_init(n, s, d)
        out = torch.empty(n, dtype=torch.int32, device=dev)
        row = {"k": k, "n": n, "m": int(s.numel())}
        for name, (order, mode) in variants.items():
            best, sweeps = float("inf"), 0
            for _ in range(1 + max(1, min(args.steps, 3))):
                st = cc.cc_run(g, out, order, mode, 1)
                if st.solve_ms < best:
                    best, sweeps = st.solve_ms, st.sweeps
            row[name] = {"ms": best, "sweeps": sweeps}
        cc.cc_free(g)
        rows.append(row)
        del s, d, out
    growth = {v: rows[-1][v]["ms"] / rows[0][v]["ms"] for v in variants}
    return {"growth": growth, "paper_growth_20_core_xeon": PAPER_DELAUNAY_GROWTH, "rows": rows}


def run_delaunay_scaling(args, rank):
    import paper_2311_02811_gb300 as cc
    dev = torch.device("cuda", torch.cuda.current_device())
    res = delaunay_scaling(cc, args, dev)
    line = {"metric": "Delaunay-style scaling n=2^10..2^24: solve-time growth n10 -> n24",
            "value": res["growth"]["C-2"], "unit": "x", "higher_is_better": False, "n_gpus": 1,
            "data": "synthetic", "dtype": "int32",
            "config": {"workload": "delaunay-like-2^10..2^24", "edges": "jittered grid with Delaunay diagonals"},
            **res}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_init()
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        elif args.workload == "delaunay-scaling":
            run_delaunay_scaling(args, rank)
        elif args.workload.startswith("batch"):
            run_batch(args, rank, world, local)
        else:
            run_ours(args, rank, world, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
