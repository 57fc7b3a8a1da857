"""Benchmark of the grid-filtered P2P / PIP join on GB300.

Default workload (N = 1): P2P, 10,000,000 clustered points against 100,000
random-walk polylines (2-40 vertices), window D = 100 m, grid 1024 x 1024.
One step = one join against the resident polyline layer: cell ids (a1),
bucketing (a2), work items (a5), refinement (a7) and the scatter of results
(a8); the layer's MBBs and candidate lists (a3, a4) are built once before the
timed region, as in serving, and their build time is reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload p2p|pip] [--form fp32x|fp64]

Rank 0 prints one JSON line.  Under torchrun (N > 1) every rank joins its own
points against a replica of the layer (weak scaling, no data-path collective);
the timed region is bracketed by barriers and the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import json
import math
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
FP64_LANES_PER_SM = 2       # GB300: FP64 issue rate per SM per clock (1/64 of FP32)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["p2p", "pip"], default="p2p")
    ap.add_argument("--form", choices=["fp32x", "fp64"], default="fp32x")
    ap.add_argument("--no-baselines", action="store_true", help="skip the FP64, e2e and CPU comparison legs")
    return ap.parse_args()


def workload(name: str, rank: int = 0):
    from paper_1403_0802_gb300 import synth
    if name == "p2p":
        return synth.p2p_walks(seed=synth.SEED_BASE + 2 + 1000 * rank)
    return synth.pip_stars(seed=synth.SEED_BASE + 1 + 1000 * rank)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


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
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
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
        for l in getattr(self, "lines", []):
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


def cpu_baseline(w, sample: int, threads: int | None = None):
    """The oracle's grid-filtered join on the host cores, on the first `sample`
    points of the workload (candidate lists built outside the timing)."""
    from oracle import oracle as O
    O.build()
    n = O.set_threads(threads)
    pts = np.ascontiguousarray(w.points[:sample])
    if w.kind == "p2p":
        L = w.polylines
        mbb = O.p2p_mbb(w.grid, L.verts, L.line_off)
        cs, ci = O.cand_csr(w.grid, mbb, w.D, expand=True)
        t0 = time.perf_counter()
        O.p2p_grid(w.grid, pts, L.verts, L.line_off, w.D, cs, ci)
    else:
        P = w.polygons
        mbb = O.pip_mbb(w.grid, P.verts, P.ring_off, P.poly_ring_off)
        cs, ci = O.cand_csr(w.grid, mbb)
        t0 = time.perf_counter()
        O.pip_grid(w.grid, pts, P.verts, P.ring_off, P.poly_ring_off, cs, ci)
    dt = time.perf_counter() - t0
    return {"value": sample / dt, "unit": "points/s", "cores": n, "kind": "oracle",
            "sample": f"first {sample} points of the workload, grid-filtered oracle join, {n} threads, "
                      f"{dt:.2f} s wall"}


def run_reference(args):
    """The oracle on the host cores: each step joins a bounded slice of the same
    workload (rank 0 only)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    w = workload(args.workload)
    from oracle import oracle as O
    O.build()
    n = O.set_threads(None)
    per_step = 50_000
    if w.kind == "p2p":
        L = w.polylines
        cs, ci = O.cand_csr(w.grid, O.p2p_mbb(w.grid, L.verts, L.line_off), w.D, expand=True)
        step = lambda pts: O.p2p_grid(w.grid, pts, L.verts, L.line_off, w.D, cs, ci)
    else:
        P = w.polygons
        cs, ci = O.cand_csr(w.grid, O.pip_mbb(w.grid, P.verts, P.ring_off, P.poly_ring_off))
        step = lambda pts: O.pip_grid(w.grid, pts, P.verts, P.ring_off, P.poly_ring_off, cs, ci)
    N = len(w.points)
    slices = [np.ascontiguousarray(w.points[(k * per_step) % N:(k * per_step) % N + per_step])
              for k in range(args.warmup + args.steps)]
    for k in range(args.warmup):
        step(slices[k])
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(slices[args.warmup + k])
    dt = time.perf_counter() - t0
    v = per_step * args.steps / dt
    print(json.dumps({
        "impl": "reference", "metric": metric_name(w), "value": v, "unit": "points/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(w, args),
        "cpu_baseline": {"value": v, "unit": "points/s", "cores": n, "kind": "oracle",
                         "sample": f"{per_step} points per step, grid-filtered oracle join"},
        "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def metric_name(w):
    return ("P2P points/s (grid-filtered nearest polyline within D)" if w.kind == "p2p"
            else "PIP points/s (grid-filtered point-in-polygon)")


def config_of(w, args):
    c = {"workload": w.name, "points": int(len(w.points)), "grid": f"{w.grid['nx']}x{w.grid['ny']}",
         "form": args.form, "launch": "per_request", "pts_per_item": 64,
         "l2": "inputs larger than L2 (points alone 160 MB for the P2P workload); no flush"}
    if w.kind == "p2p":
        c.update(polylines=w.polylines.n_lines, vertices=int(len(w.polylines.verts)), D=w.D)
    else:
        c.update(polygons=w.polygons.n_polygons, vertices=int(len(w.polygons.verts)))
        c["l2"] = "points 16 MB fit in L2; no flush between steps"
    return c


def time_joins(api, layer, w, pts, form, steps, warmup, world, dev, stream, timed=True):
    import torch
    n = pts.shape[0]
    out_id = torch.empty(n, dtype=torch.int32, device=dev)
    out_d = torch.empty(n, dtype=torch.float64, device=dev)

    def one(time_refine):
        if w.kind == "p2p":
            api.p2p_join(layer, pts, out_id, out_d, form=form, stream=stream, time_refine=time_refine)
        else:
            api.pip_join(layer, pts, out_id, form=form, stream=stream, time_refine=time_refine)

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
    ms = e0.elapsed_time(e1)
    return ms, layer.stats(), (out_id, out_d)


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
    w = workload(args.workload, rank)
    stream = torch.cuda.current_stream(dev)

    t0 = torch.cuda.Event(enable_timing=True); t1 = torch.cuda.Event(enable_timing=True)
    if w.kind == "p2p":
        L = w.polylines
        v = torch.as_tensor(L.verts, device=dev); off = torch.as_tensor(L.line_off, device=dev)
        torch.cuda.synchronize(); t0.record(stream)
        layer = api.p2p_layer(v, off, w.D, w.grid, stream=stream)
    else:
        P = w.polygons
        v = torch.as_tensor(P.verts, device=dev)
        ro = torch.as_tensor(P.ring_off, device=dev); pro = torch.as_tensor(P.poly_ring_off, device=dev)
        torch.cuda.synchronize(); t0.record(stream)
        layer = api.pip_layer(v, ro, pro, w.grid, stream=stream)
    t1.record(stream); torch.cuda.synchronize()
    layer_ms = t0.elapsed_time(t1)

    pts = torch.as_tensor(w.points, device=dev)
    n = pts.shape[0]
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0]) if os.environ.get(
        "CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local
    with ClockSampler(gpu_index) as clk:
        ms, st, _ = time_joins(api, layer, w, pts, args.form, args.steps, args.warmup, world, dev, stream)
    clocks = clk.summary()
    ms_max = max_over_ranks(ms, world, dev)
    value = n * world * args.steps / (ms_max / 1000.0)

    # dominant kernel: the refinement launch, timed with events on the join's stream
    refine_ms = st["refine_ms"] / max(st["refine_launches"], 1)
    tests_per_launch = st["edge_tests"] / max(st["joins"], 1)
    props = torch.cuda.get_device_properties(dev)
    peaks = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    if w.kind == "p2p":
        flops = tests_per_launch * FLOPS_PER_SEGMENT
        lanes = FP32_LANES_PER_SM if args.form == "fp32x" else FP64_LANES_PER_SM
    else:
        flops = tests_per_launch * FLOPS_PER_EDGE
        lanes = FP32_LANES_PER_SM if args.form == "fp32x" else FP64_LANES_PER_SM
    peak_tflops = props.multi_processor_count * lanes * 2 * sm_mhz * 1e6 / 1e12
    achieved = flops / (refine_ms / 1000.0) / 1e12 if refine_ms > 0 else None
    roofline = {"bound": "alu", "kernel": f"k_{w.kind}_refine<{args.form}>", "achieved": achieved,
                "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": (achieved / peak_tflops) if achieved else None, "traffic": None,
                "peak_source": f"derived: {props.multi_processor_count} SMs x {lanes} "
                               f"{'FP32' if args.form == 'fp32x' else 'FP64'} lanes x 2 x {sm_mhz:.0f} MHz",
                "refine_ms_per_launch": refine_ms, "tests_per_launch": tests_per_launch,
                "flops_per_test": FLOPS_PER_SEGMENT if w.kind == "p2p" else FLOPS_PER_EDGE}

    extra = {}
    if not args.no_baselines and rank == 0:
        # the plain FP64 form, same workload, fewer steps
        if args.form != "fp64":
            k64 = max(3, min(args.steps, 20))
            ms64, st64, _ = time_joins(api, layer, w, pts, "fp64", k64, 2, 1, dev, stream)
            extra["fp64_plain"] = {"value": n * k64 / (ms64 / 1000.0), "unit": "points/s",
                                   "ms_per_step": ms64 / k64,
                                   "refine_ms_per_launch": st64["refine_ms"] / max(st64["refine_launches"], 1)}
            extra["speedup_vs_fp64_plain"] = value / extra["fp64_plain"]["value"]
        extra["fallbacks_per_join"] = st["fallbacks"] / max(st["joins"], 1)
        extra["edge_tests_per_s"] = tests_per_launch * args.steps / (ms / 1000.0)

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if rank == 0 and not args.no_baselines:
        hp = torch.empty((n, 2), dtype=torch.float64, pin_memory=True)
        hp.copy_(torch.from_numpy(w.points))
        hid = torch.empty(n, dtype=torch.int32, pin_memory=True)
        hd = torch.empty(n, dtype=torch.float64, pin_memory=True)
        ke = max(3, min(args.steps, 20))
        join_host = (lambda: api.p2p_join_host(layer, hp, hid, hd, form=args.form, stream=stream)) if w.kind == "p2p" \
            else (lambda: api.pip_join_host(layer, hp, hid, form=args.form, stream=stream))
        for _ in range(2):
            join_host()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ke):
            join_host()
        e1.record(stream)
        torch.cuda.synchronize()
        ems = e0.elapsed_time(e1)
        e2e = {"value": n * ke / (ems / 1000.0), "unit": "points/s", "h2d_bytes_per_step": n * 16,
               "d2h_bytes_per_step": n * (4 + (8 if w.kind == "p2p" else 0)), "steps": ke,
               "api": "sj_p2p_join_host" if w.kind == "p2p" else "sj_pip_join_host"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_baselines:
        cpu = cpu_baseline(w, 1_000_000 if w.kind == "p2p" else 1_000_000)

    kernels_per_join = 5 + 1 + (1 if (w.kind == "p2p" and args.form == "fp32x") else 0)
    if rank == 0:
        line = {
            "metric": metric_name(w), "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if args.form == "fp32x" else "f64",
            "data": "synthetic", "config": dict(config_of(w, args), layer_build_ms=layer_ms,
                                                 parallelism=f"points sharded, layer replicated x{world}"),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": kernels_per_join * args.steps, **extra,
        }
        print(json.dumps(line))
    layer.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
