"""Benchmark of the grid-filtered P2P / PIP join on GB300.

Workloads (--workload):
  p2p    (default) P2P, 10,000,000 clustered points, 100,000 random-walk
         polylines (2-40 vertices), window D = 100 m, grid 512 x 512
  pip    PIP, 1,000,000 uniform points, 1,024 star polygons, grid 256 x 256
  pip3   PIP at scale, 100,000,000 clustered points against the 40,000-tile
         layer (--layer 1), the 14,000-tile heavy-tail layer (--layer 2) or the
         multi-ring layer (--layer 3: layer 1 with island holes, ~70,000 polygons)
  p2p4   P2P at scale, 170,000,000 clustered points, 150,000 lognormal walks,
         D = --D (50, 100 or 200 m)
  serve  continuous batching: a Poisson stream of GPS batches (1k-5M points,
         70 % PIP against the 40,000-tile layer, 30 % P2P against the 150,000
         walks), batched rounds vs one join call per request; p50 / p99 latency

One step = one join against the resident layer: cell ids (a1), bucketing (a2),
work items (a5), refinement (a6 / a7) with the scatter of results (a8).  The
layer's MBBs and candidate lists (a3, a4) are built once before the timed
region, as in serving; that build time is reported as config.layer_build_ms.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload ...] [--form fp32x|fp64]

Rank 0 prints one JSON line.  Under torchrun (N > 1) every rank joins its own
points against a replica of the layer (weak scaling, no data-path collective);
the timed region is bracketed by barriers and the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOPS_PER_SEGMENT = 12      # algorithmic FP ops of one point-segment distance test
FLOPS_PER_EDGE = 2          # algorithmic FP ops of one point-edge straddle test (2 compares)
FP32_LANES_PER_SM = 128
FP64_LANES_PER_SM = 2       # GB300: FP64 FMA issue per SM per clock (measured: 1.97)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["p2p", "pip", "pip3", "p2p4", "serve"], default="p2p")
    ap.add_argument("--layer", type=int, default=1, choices=[1, 2, 3],
                    help="pip3: tiling layer 1, 2 or 3 (multi-ring)")
    ap.add_argument("--D", type=float, default=100.0, help="p2p4: window")
    ap.add_argument("--points", type=int, default=0, help="override the workload's point count")
    ap.add_argument("--form", choices=["fp32x", "fp64"], default="fp32x")
    ap.add_argument("--grid", type=int, default=0, help="filter grid cells per axis (0: the workload's)")
    ap.add_argument("--ppi", type=int, default=0, help="points per work item, 1..128 (0: library default 128)")
    ap.add_argument("--requests", type=int, default=10000, help="serve: stream length")
    ap.add_argument("--no-baselines", action="store_true", help="skip the FP64, e2e and CPU comparison legs")
    ap.add_argument("--oracle-full", action="store_true",
                    help="--impl reference: join the whole workload once instead of bounded steps")
    ap.add_argument("--oracle-threads", type=int, default=0, help="--impl reference: host threads (0: all)")
    return ap.parse_args()


def workload(args, rank: int = 0):
    from paper_1403_0802_gb300 import synth
    n = args.points or None
    g = {"grid_n": args.grid} if getattr(args, "grid", 0) else {}
    if args.workload == "p2p":
        return synth.p2p_walks(n_points=n or 10_000_000, shard=rank, **g)
    if args.workload == "pip":
        return synth.pip_stars(n_points=n or 1_000_000, shard=rank, **g)
    if args.workload == "pip3":
        return synth.pip_tiles(n_points=n or 100_000_000, layer=args.layer, shard=rank, **g)
    if args.workload == "p2p4":
        return synth.p2p_walks_lognormal(n_points=n or 170_000_000, D=args.D, shard=rank, **g)
    raise ValueError(args.workload)


def default_ppi(args) -> int:
    """Points per work item: --ppi, else the autotuner's best for the workload
    at its full size (128, the library default, except 64 on the heavy-tail
    tiling, whose boundary cells stage long near-edge lists per item)."""
    if args.ppi:
        return args.ppi
    return 64 if (args.workload == "pip3" and args.layer == 2) else 0


def dist_env():
    return int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def oracle_join_fn(w):
    """The oracle's grid-filtered join for workload w (candidate lists built
    here, outside any timing)."""
    from oracle import oracle as O
    O.build()
    if w.kind == "p2p":
        L = w.polylines
        cs, ci = O.cand_csr(w.grid, O.p2p_mbb(w.grid, L.verts, L.line_off), w.D, expand=True)
        return lambda pts: O.p2p_grid(w.grid, pts, L.verts, L.line_off, w.D, cs, ci)
    P = w.polygons
    cs, ci = O.cand_csr(w.grid, O.pip_mbb(w.grid, P.verts, P.ring_off, P.poly_ring_off))
    return lambda pts: O.pip_grid(w.grid, pts, P.verts, P.ring_off, P.poly_ring_off, cs, ci)


def cpu_baseline(w, target_wall_s: float = 1.0):
    """The oracle on all host cores, on a bounded prefix of the workload's points
    sized from a short probe to about target_wall_s of wall time (10-30 core-s)."""
    from oracle import oracle as O
    n_thr = O.set_threads(None)
    join = oracle_join_fn(w)
    probe = min(len(w.points), 100_000)
    t0 = time.perf_counter()
    join(np.ascontiguousarray(w.points[:probe]))
    rate = probe / max(time.perf_counter() - t0, 1e-6)
    sample = int(min(len(w.points), max(probe, rate * target_wall_s)))
    pts = np.ascontiguousarray(w.points[:sample])
    t0 = time.perf_counter()
    join(pts)
    dt = time.perf_counter() - t0
    return {"value": sample / dt, "unit": "points/s", "cores": n_thr, "kind": "oracle",
            "sample": f"first {sample} points of the workload, grid-filtered oracle join on {n_thr} threads, "
                      f"{dt:.2f} s wall ({dt * n_thr:.0f} core-s)"}


def metric_name(kind):
    return ("P2P points/s (grid-filtered nearest polyline within D)" if kind == "p2p"
            else "PIP points/s (grid-filtered point-in-polygon)")


def config_of(w, args):
    c = {"workload": w.name, "points": int(len(w.points)), "grid": f"{w.grid['nx']}x{w.grid['ny']}",
         "form": args.form, "launch": "per_request", "pts_per_item": default_ppi(args) or 128}
    big = len(w.points) * 16 > 129e6
    c["l2"] = ("inputs larger than L2 (points %d MB > 129 MB); no flush" % (len(w.points) * 16 // 10 ** 6) if big
               else "points %d MB fit in L2; steps re-read them (no flush)" % (len(w.points) * 16 // 10 ** 6))
    if w.kind == "p2p":
        c.update(polylines=w.polylines.n_lines, vertices=int(len(w.polylines.verts)), D=w.D)
    else:
        c.update(polygons=w.polygons.n_polygons, vertices=int(len(w.polygons.verts)))
    return c


def run_reference(args):
    """The oracle on the host cores: each step joins a bounded slice of the same
    workload (rank 0 only)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    if args.workload == "serve":
        args.workload = "p2p"
    w = workload(args)
    n = O.set_threads(args.oracle_threads or None)
    t_idx = time.perf_counter()
    join = oracle_join_fn(w)
    if args.oracle_full:      # the whole workload, once (the layer's filter lists built outside the timing)
        t_idx = time.perf_counter() - t_idx
        t0 = time.perf_counter()
        join(w.points)
        dt = time.perf_counter() - t0
        v = len(w.points) / dt
        print(json.dumps({
            "impl": "reference", "metric": metric_name(w.kind), "value": v, "unit": "points/s",
            "n_gpus": args.gpus, "steps": 1, "warmup": 0, "ms_per_step": 1000 * dt, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(w, args),
            "cpu_baseline": {"value": v, "unit": "points/s", "cores": n, "kind": "oracle",
                             "sample": f"all {len(w.points)} points once, grid-filtered oracle join on {n} "
                                       f"threads ({dt:.1f} s; filter lists {t_idx:.1f} s before)"},
            "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    per_step = 50_000
    N = len(w.points)
    slices = [np.ascontiguousarray(w.points[(k * per_step) % N:(k * per_step) % N + per_step])
              for k in range(args.warmup + args.steps)]
    for k in range(args.warmup):
        join(slices[k])
    t0 = time.perf_counter()
    for k in range(args.steps):
        join(slices[args.warmup + k])
    dt = time.perf_counter() - t0
    v = per_step * args.steps / dt
    print(json.dumps({
        "impl": "reference", "metric": metric_name(w.kind), "value": v, "unit": "points/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(w, args),
        "cpu_baseline": {"value": v, "unit": "points/s", "cores": n, "kind": "oracle",
                         "sample": f"{per_step} points per step, grid-filtered oracle join"},
        "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def time_joins(api, layer, w, pts, form, steps, warmup, world, stream, timed=True, ppi=0):
    import torch
    n = pts.shape[0]
    out_id = torch.empty(n, dtype=torch.int32, device=pts.device)
    out_d = torch.empty(n, dtype=torch.float64, device=pts.device)

    def one(time_refine):
        if w.kind == "p2p":
            api.p2p_join(layer, pts, out_id, out_d, form=form, stream=stream, time_refine=time_refine,
                         pts_per_item=ppi)
        else:
            api.pip_join(layer, pts, out_id, form=form, stream=stream, time_refine=time_refine, pts_per_item=ppi)

    for _ in range(warmup):
        one(False)
    torch.cuda.synchronize()
    layer.reset_stats()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        one(timed)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    return e0.elapsed_time(e1), layer.stats()


def build_layer(api, w, dev, stream):
    import torch
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    if w.kind == "p2p":
        L = w.polylines
        v = torch.as_tensor(L.verts, device=dev)
        off = torch.as_tensor(L.line_off, device=dev)
        torch.cuda.synchronize()
        t0.record(stream)
        layer = api.p2p_layer(v, off, w.D, w.grid, stream=stream)
    else:
        P = w.polygons
        v = torch.as_tensor(P.verts, device=dev)
        ro = torch.as_tensor(P.ring_off, device=dev)
        pro = torch.as_tensor(P.poly_ring_off, device=dev)
        torch.cuda.synchronize()
        t0.record(stream)
        layer = api.pip_layer(v, ro, pro, w.grid, stream=stream)
    t1.record(stream)
    torch.cuda.synchronize()
    return layer, t0.elapsed_time(t1)


HERE = os.path.dirname(os.path.abspath(__file__))
REFINE_SOURCES = {"p2p": ("paper_1403_0802_gb300/csrc/sj_p2p.cu",), "pip": ("paper_1403_0802_gb300/csrc/sj_pip.cu",)}


def sources_sha(kind):
    h = hashlib.sha256()
    for f in REFINE_SOURCES[kind]:
        with open(os.path.join(HERE, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(kernel, workload, kind):
    """DRAM bytes (read + write) per launch of `kernel` on `workload` from the
    committed ncu summary profiles/traffic.txt (lines: kernel workload bytes
    sha256-of-the-kernel's-source-file), or None when absent or when that file
    changed since the counters were taken."""
    path = os.path.join(HERE, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    sha = sources_sha(kind)
    for line in open(path):
        f = line.split()
        if len(f) == 4 and not line.startswith("#") and f[0] == kernel and f[1] == workload and f[3] == sha:
            return float(f[2])
    return None


def roofline_of(w, form, st, props, peaks):
    """Dominant kernel = the refinement launch, timed with CUDA events on the
    join's stream.  Work per launch = the (point, edge or segment) tests the
    kernel executes (the candidate lists' tests minus the exact staging prune)
    x the algorithmic FP ops of one test; achieved = that / launch time.  The
    unpruned count (points x segments or edges of the candidate objects) is
    reported as effective_tflops."""
    refine_ms = st["refine_ms"] / max(st["refine_launches"], 1)
    joins = max(st["joins"], 1)
    algo = st["algo_tests"] / joins
    executed = st["edge_tests"] / joins
    fpt = FLOPS_PER_SEGMENT if w.kind == "p2p" else FLOPS_PER_EDGE
    lanes = FP32_LANES_PER_SM if form == "fp32x" else FP64_LANES_PER_SM
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = props.multi_processor_count * lanes * 2 * sm_mhz * 1e6 / 1e12
    achieved = executed * fpt / (refine_ms / 1e3) / 1e12 if refine_ms > 0 else None
    kernel = f"k_{w.kind}_refine<{form}>"
    return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak if achieved else None,
            "traffic": measured_traffic(kernel, w.name, w.kind),
            "peak_source": f"derived: {props.multi_processor_count} SMs x {lanes} "
                           f"{'FP32' if form == 'fp32x' else 'FP64'} lanes x 2 flops x {sm_mhz:.0f} MHz "
                           f"(MEASURED_PEAKS sm_max_mhz)",
            "refine_ms_per_launch": refine_ms, "executed_tests_per_launch": executed,
            "algorithmic_tests_per_launch": algo, "flops_per_test": fpt,
            "effective_tflops": algo * fpt / (refine_ms / 1e3) / 1e12 if refine_ms > 0 else None}


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_1403_0802_gb300 import api, build
    build.build()
    w = workload(args, rank)
    stream = torch.cuda.current_stream(dev)
    layer, layer_ms = build_layer(api, w, dev, stream)
    pts = torch.as_tensor(w.points, device=dev)
    n = pts.shape[0]
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0]
    gpu_index = int(vis) if vis.isdigit() else local
    with ClockSampler(gpu_index) as clk:
        ms, st = time_joins(api, layer, w, pts, args.form, args.steps, args.warmup, world, stream,
                            ppi=default_ppi(args))
    clocks = clk.summary()
    ms_max = max_over_ranks(ms, world, dev)
    value = n * world * args.steps / (ms_max / 1000.0)
    props = torch.cuda.get_device_properties(dev)
    roofline = roofline_of(w, args.form, st, props, measured_peaks())

    extra = {"fallbacks_per_join": st["fallbacks"] / max(st["joins"], 1),
             "edge_tests_per_s_algorithmic": st["algo_tests"] / (ms / 1000.0)}
    if not args.no_baselines and rank == 0 and args.form != "fp64":
        k64 = max(3, min(args.steps, 20))
        ms64, st64 = time_joins(api, layer, w, pts, "fp64", k64, 2, 1, stream, ppi=default_ppi(args))
        extra["fp64_plain"] = {"value": n * k64 / (ms64 / 1000.0), "unit": "points/s", "ms_per_step": ms64 / k64,
                               "roofline": roofline_of(w, "fp64", st64, props, measured_peaks())}
        extra["speedup_vs_fp64_plain"] = value / extra["fp64_plain"]["value"]

    e2e = None
    if rank == 0 and not args.no_baselines:
        hp = torch.empty((n, 2), dtype=torch.float64, pin_memory=True)
        hp.copy_(torch.from_numpy(w.points))
        hid = torch.empty(n, dtype=torch.int32, pin_memory=True)
        hd = torch.empty(n, dtype=torch.float64, pin_memory=True)
        ke = max(3, min(args.steps, 20))
        if w.kind == "p2p":
            join_host = lambda: api.p2p_join_host(layer, hp, hid, hd, form=args.form, stream=stream,
                                                  pts_per_item=default_ppi(args))
        else:
            join_host = lambda: api.pip_join_host(layer, hp, hid, form=args.form, stream=stream,
                                                  pts_per_item=default_ppi(args))
        for _ in range(2):
            join_host()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            join_host()      # synchronous: copies in, join, copies out
        ems = (time.perf_counter() - t0) * 1e3
        e2e = {"value": n * ke / (ems / 1000.0), "unit": "points/s", "h2d_bytes_per_step": n * 16,
               "d2h_bytes_per_step": n * (4 + (8 if w.kind == "p2p" else 0)), "steps": ke,
               "api": "sj_p2p_join_host" if w.kind == "p2p" else "sj_pip_join_host",
               "timing": "host wall clock around synchronous calls (pinned buffers)"}

    cpu = cpu_baseline(w) if (rank == 0 and world == 1 and not args.no_baselines) else None
    # cell_hist, 3 scan phases, scatter; refine; FP32X P2P recheck; unsort
    kernels_per_join = 5 + 1 + (1 if (w.kind == "p2p" and args.form == "fp32x") else 0) + 1
    if rank == 0:
        line = {
            "metric": metric_name(w.kind), "value": value, "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.form == "fp32x" else "f64", "data": "synthetic",
            "config": dict(config_of(w, args), layer_build_ms=layer_ms,
                           parallelism=f"points sharded, layer replicated x{world}"),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": kernels_per_join * args.steps, **extra,
        }
        print(json.dumps(line))
    layer.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_serve(args):
    """Continuous batching (native server, batched engine rounds) against one
    join call per request in the same native loop -- in the same form and in
    the plain FP64 form -- on one Poisson stream of requests."""
    import torch
    world, rank, local = dist_env()
    if rank != 0:
        return
    from paper_1403_0802_gb300 import api, build, serve, synth
    build.build()
    torch.cuda.set_device(local)
    wp = synth.pip_tiles(n_points=20_000_000, layer=1)
    wl = synth.p2p_walks_lognormal(n_points=20_000_000, n_lines=150_000, D=100.0)
    pip = api.pip_layer(wp.polygons.verts, wp.polygons.ring_off, wp.polygons.poly_ring_off, wp.grid)
    p2p = api.p2p_layer(wl.polylines.verts, wl.polylines.line_off, wl.D, wl.grid)
    pool_p = torch.from_numpy(wp.points).pin_memory()
    pool_l = torch.from_numpy(wl.points).pin_memory()
    outs = {serve.PIP: (torch.empty(len(pool_p), dtype=torch.int32, pin_memory=True), None),
            serve.P2P: (torch.empty(len(pool_l), dtype=torch.int32, pin_memory=True),
                        torch.empty(len(pool_l), dtype=torch.float64, pin_memory=True))}
    srv = serve.Server(pip, p2p, form=args.form, round_points=6_000_000, max_requests=4096)
    arms = [("batched", args.form), ("per_request", args.form), ("per_request", "fp64")]
    for mode, form in arms:      # warm-up: workspaces, graphs, allocator pools
        srv.run(serve.make_stream(32, 0.0, pool_p, pool_l, seed=1), mode=mode, form=form, out_pools=outs)
    # capacity of each arm with every request queued at t = 0
    sat = {f"{m}_{f}": srv.run(serve.make_stream(min(args.requests, 300), 0.0, pool_p, pool_l, seed=3),
                               mode=m, form=f, out_pools=outs) for m, f in arms}
    mean_pts = sat[f"batched_{args.form}"]["points"] / sat[f"batched_{args.form}"]["requests"]
    base = sat["per_request_fp64"]["points_per_s"]          # the plain FP64 one-launch-per-request form
    res = {}
    for rho in (0.5, 0.8):
        rate = rho * base / mean_pts
        for m, f in arms:
            reqs = serve.make_stream(args.requests, rate, pool_p, pool_l, seed=7)
            res[f"{m}_{f}_rho{rho}"] = srv.run(reqs, mode=m, form=f, out_pools=outs)
    fast = sat[f"per_request_{args.form}"]["points_per_s"]  # a load the FP64 form cannot sustain
    for m, f in arms[:2]:
        reqs = serve.make_stream(args.requests, 0.8 * fast / mean_pts, pool_p, pool_l, seed=7)
        res[f"{m}_{f}_rho0.8_of_{args.form}_capacity"] = srv.run(reqs, mode=m, form=f, out_pools=outs)
    b, p64 = res[f"batched_{args.form}_rho0.8"], res["per_request_fp64_rho0.8"]
    line = {"metric": "serving p50/p99 latency (ms) and points/s, continuous batching", "value": b["p99_ms"],
            "unit": "ms (p99)", "n_gpus": 1, "steps": args.requests, "warmup": 32, "ms_per_step": b["mean_ms"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.form == "fp32x" else "f64", "data": "synthetic",
            "config": {"workload": f"serve_{args.requests}req_pip40k_p2p150k", "requests": args.requests,
                       "sizes": "log-uniform 1e3..5e6 points", "mix": "70% PIP / 30% P2P (D=100 m)",
                       "arrivals": "Poisson, rate = rho x capacity of the plain FP64 one-join-per-request form",
                       "form": args.form, "server": "native (sj_server_*), batched engine rounds"},
            "p50_ms": b["p50_ms"], "p99_ms": b["p99_ms"], "points_per_s": b["points_per_s"],
            "plain_fp64_per_request_p50_ms": p64["p50_ms"], "plain_fp64_per_request_p99_ms": p64["p99_ms"],
            "plain_fp64_per_request_points_per_s": p64["points_per_s"], "capacity": sat, "runs": res}
    print(json.dumps(line))
    srv.close()
    pip.close()
    p2p.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
