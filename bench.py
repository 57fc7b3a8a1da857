"""Benchmark of the grid-filtered P2P / PIP join on GB300.

Workloads (--workload):
  p2p    (default) P2P, 10,000,000 clustered points, 100,000 random-walk
         polylines (2-40 vertices), window D = 100 m, grid 448 x 448
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

The default run (the P2P workload at one GPU) prints ONE JSON line: the P2P
headline, plus the other halves of the metric as extra keys, each timed the
same way (CUDA events on the join's stream, its own clock record, roofline,
CPU baseline with the GPU's measured error against the oracle, and plain FP64
comparison): "pip_stars" (the PIP workload), "pip_at_scale_layer1" and
"pip_at_scale_layer2" (100 M points against the 40,000-tile and the
heavy-tail tilings), "p2p_at_scale_D50" / "_D100" / "_D200" (170 M points,
150,000 walks) and "serve" (the serving workload); --no-extra leaves them
out.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload ...] [--form fp32x|fp64]

Rank 0 prints one JSON line.  Under torchrun (N > 1) every rank joins its own
points against a replica of the layer (weak scaling, no data-path collective);
the timed region is bracketed by barriers and the slowest rank's time is used.

Roofline (the join has no dense contraction, so no tensor-core peak applies):
the dominant kernel is the refinement, bound by plain arithmetic.  Its work
is the algorithmic test count the candidate lists imply -- P2P: every
(point, segment of a candidate polyline) pair, 12 flops each; PIP: every
(point, edge of a candidate polygon) pair, 2 compares each plus 7 flops for
the fraction of edges that straddle the point's y (counted by sj_pip_census)
-- divided by the refinement launch time (CUDA events on the join's stream)
and by the FP32 (or FP64) peak measured by sj_peaks_measure.  The HBM side is
the algorithmic bytes of the join (points in, results out, the layer once)
over the whole join time against MEASURED_PEAKS' copy bandwidth.
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
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
FLOPS_PER_COMPARE = 2       # PIP: the two straddle compares of every edge test
FLOPS_PER_STRADDLE = 7      # PIP: the orientation test of an edge that straddles
FP32_LANES_PER_SM = 128
FP64_LANES_PER_SM = 2       # GB300: FP64 FMA issue per SM per clock (measured: 1.97)
SUB_LEG_MIN_S = 0.25        # extra legs time enough joins to fill at least this much


def parse(argv=None):
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
    ap.add_argument("--serve-grid-pip", type=int, default=1024, help="serve: grid cells per axis, polygon layer")
    ap.add_argument("--serve-grid-p2p", type=int, default=512, help="serve: grid cells per axis, polyline layer")
    ap.add_argument("--no-baselines", action="store_true", help="skip the FP64, e2e and CPU comparison legs")
    ap.add_argument("--no-extra", action="store_true", help="default run: leave out the PIP and serving legs")
    ap.add_argument("--oracle-full", action="store_true",
                    help="--impl reference: join the whole workload once instead of bounded steps")
    ap.add_argument("--oracle-threads", type=int, default=0, help="--impl reference: host threads (0: all)")
    ap.add_argument("--ref-budget-s", type=float, default=60.0,
                    help="--impl reference: wall-time budget of the warm-up and timed steps together")
    return ap.parse_args(argv)


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


# Launch settings per workload at full size: the fastest row of
# paper_1403_0802_gb300.autotune on GB300 (points per item x warps per block x
# edges per chunk; 0 = the library default).
TUNED = {"p2p": dict(ppi=128, block=4, edges=0), "pip": dict(ppi=128, block=4, edges=0),
         "pip3_1": dict(ppi=128, block=4, edges=64), "pip3_2": dict(ppi=128, block=2, edges=64),
         "pip3_3": dict(ppi=128, block=8, edges=64), "p2p4": dict(ppi=128, block=4, edges=0)}


def tuned(args) -> dict:
    key = f"pip3_{args.layer}" if args.workload == "pip3" else args.workload
    t = dict(TUNED.get(key, dict(ppi=0, block=0, edges=0)))
    if args.ppi:
        t["ppi"] = args.ppi
    return t


def default_ppi(args) -> int:
    """Points per work item: --ppi, else the autotuned setting."""
    return tuned(args)["ppi"]


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
    """nvidia-smi clocks and throttle reasons sampled every period_ms (10 ms by
    default: several samples even in a 17 ms timed region) with their
    timestamps; summary() reports the samples inside the timed regions marked
    with region() (host wall clock), widened by one sampling period."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 10):
        self.idx = gpu_index
        self.PERIOD_MS = period_ms
        self.proc = None
        self.lines = []
        self.regions = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)                    # the first samples arrive before the timed region
        except OSError:
            self.proc = None
        return self

    def region(self, t0: float, t1: float):
        self.regions.append((t0, t1))

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.05)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    @staticmethod
    def _epoch(ts: str):
        try:
            return datetime.datetime.strptime(ts.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def summary(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 10:
                continue
            try:
                rows.append((self._epoch(f[0]), float(f[2]), float(f[3]),
                             {n for n, v in zip(names, f[6:10]) if v.lower() == "active"}))
            except ValueError:
                continue
        pad = self.PERIOD_MS / 1e3
        inside = [r for r in rows if r[0] is not None and
                  any(t0 - pad <= r[0] <= t1 + pad for t0, t1 in self.regions)]
        use = inside or rows
        sm = [r[1] for r in use]
        reasons = set().union(*[r[3] for r in use]) if use else set()
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max((r[2] for r in rows), default=None),
                "reasons": sorted(reasons), "samples": len(sm), "samples_in_timed_region": len(inside),
                "samples_total": len(rows), "period_ms": self.PERIOD_MS,
                "timed_region_s": round(sum(t1 - t0 for t0, t1 in self.regions), 4)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def alu_peaks(api):
    """FP32 / FP64 flop rates of this GPU measured by sj_peaks_measure (2 flops
    per FMA), with the lanes x clock figure as a cross-check."""
    import ctypes as C
    import torch
    from paper_1403_0802_gb300 import _lib
    r = _lib.sj_peak_rates()
    rc = _lib.lib().sj_peaks_measure(C.byref(r))
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    mhz = float(measured_peaks().get("sm_max_mhz", 2070.0))
    derived = {"fp32": props.multi_processor_count * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12,
               "fp64": props.multi_processor_count * FP64_LANES_PER_SM * 2 * mhz * 1e6 / 1e12}
    if rc != 0:
        return {"fp32": derived["fp32"], "fp64": derived["fp64"], "source": "derived (sj_peaks_measure failed)",
                "derived": derived}
    return {"fp32": 2 * r.ffma_per_s / 1e12, "fp64": 2 * r.dfma_per_s / 1e12,
            "ffma_per_clk_sm": r.ffma_per_clk_sm, "dfma_per_clk_sm": r.dfma_per_clk_sm,
            "source": "measured: sj_peaks_measure (FFMA / DFMA rate x 2 flops)", "derived": derived}


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


def cpu_baseline(w, target_wall_s: float = 1.0, gpu=None, form="fp32x"):
    """The oracle on all host cores, on a bounded prefix of the workload's points
    sized from a short probe to about target_wall_s of wall time (10-30 core-s).
    With gpu = (ids, distances) of the GPU join of the whole workload, the
    sample is also the GPU's error measurement against the oracle."""
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
    ref = join(pts)
    dt = time.perf_counter() - t0
    out = {"value": sample / dt, "unit": "points/s", "cores": n_thr, "kind": "oracle",
           "sample": f"first {sample} points of the workload, grid-filtered oracle join on {n_thr} threads, "
                     f"{dt:.2f} s wall ({dt * n_thr:.0f} core-s)"}
    if gpu is not None:
        out["error_vs_oracle"] = error_vs_oracle(w, pts, ref, gpu[0][:sample], None if gpu[1] is None
                                                 else gpu[1][:sample], form)
    return out


def error_vs_oracle(w, pts, ref, gid, gd, form):
    """The GPU's results on the oracle's sample, measured against it with the
    bar of the parity tests (tests/parity.py)."""
    from oracle import oracle as O
    if w.kind == "pip":
        return {"points": int(len(pts)), "id_mismatches": int((gid != ref).sum())}
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from parity import P2PRef, tie_or_edge
    rid, rd, d1, d2 = ref
    exempt = tie_or_edge(d1, d2, w.D)
    both = (gid >= 0) & (rid >= 0)
    err = np.abs(gd[both] - rd[both])
    rel = err / np.maximum(rd[both], 1.0)
    res = {"points": int(len(pts)), "id_mismatches_unexplained": int(((gid != rid) & ~exempt).sum()),
           "id_mismatches_at_ties_or_window_edge": int(((gid != rid) & exempt).sum()),
           "max_abs_err_m": float(err.max()) if err.size else 0.0,
           "max_rel_err": float(rel.max()) if rel.size else 0.0,
           "mean_abs_err_m": float(err.mean()) if err.size else 0.0}
    if form == "fp32x":
        bound = P2PRef(O, w.grid, w.polylines.verts, w.polylines.line_off, w.D).fp32x_bound(pts)[both]
        res["over_certified_bound"] = int((err > bound).sum())
        res["max_err_over_bound"] = float((err / bound).max()) if err.size else 0.0
    else:
        res["over_1e-12_relative"] = int((err > 1e-12 * np.maximum(rd[both], 1.0)).sum())
    return res


def metric_name(kind):
    return ("P2P points/s (grid-filtered nearest polyline within D)" if kind == "p2p"
            else "PIP points/s (grid-filtered point-in-polygon)")


def config_of(w, args):
    t = tuned(args)
    c = {"workload": w.name, "points": int(len(w.points)), "grid": f"{w.grid['nx']}x{w.grid['ny']}",
         "form": args.form, "launch": "per_request", "pts_per_item": t["ppi"] or 128,
         "warps_per_block": t["block"] or 4, "edges_per_chunk": t["edges"] or ("64" if w.kind == "pip" else "none")}
    big = len(w.points) * 16 > 129e6
    c["l2"] = ("inputs larger than L2 (points %d MB > 129 MB); no flush" % (len(w.points) * 16 // 10 ** 6) if big
               else "points %d MB fit in L2; steps re-read them (no flush)" % (len(w.points) * 16 // 10 ** 6))
    if w.kind == "p2p":
        c.update(polylines=w.polylines.n_lines, vertices=int(len(w.polylines.verts)), D=w.D)
    else:
        c.update(polygons=w.polygons.n_polygons, vertices=int(len(w.polygons.verts)))
    return c


def run_reference(args):
    """The oracle on the host cores, each step a slice of the same workload
    (rank 0 only): the slice is the whole workload when warm-up and timed steps
    together fit --ref-budget-s at the rate a short probe measures, else the
    largest prefix that does."""
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
    N = len(w.points)
    if args.oracle_full:      # the whole workload, once (the layer's filter lists built outside the timing)
        t_idx = time.perf_counter() - t_idx
        t0 = time.perf_counter()
        join(w.points)
        dt = time.perf_counter() - t0
        v = N / dt
        print(json.dumps({
            "impl": "reference", "metric": metric_name(w.kind), "value": v, "unit": "points/s",
            "n_gpus": args.gpus, "steps": 1, "warmup": 0, "ms_per_step": 1000 * dt, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(w, args),
            "cpu_baseline": {"value": v, "unit": "points/s", "cores": n, "kind": "oracle",
                             "sample": f"all {N} points once, grid-filtered oracle join on {n} "
                                       f"threads ({dt:.1f} s; filter lists {t_idx:.1f} s before)"},
            "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    probe = min(N, 100_000)
    t0 = time.perf_counter()
    join(np.ascontiguousarray(w.points[:probe]))
    rate = probe / max(time.perf_counter() - t0, 1e-6)
    per_step = int(min(N, max(10_000, rate * args.ref_budget_s / max(args.steps + args.warmup, 1))))
    whole = per_step == N
    if whole:
        slices = [w.points] * (args.warmup + args.steps)
    else:
        slices = [np.ascontiguousarray(w.points[(k * per_step) % N:(k * per_step) % N + per_step])
                  for k in range(args.warmup + args.steps)]
    for k in range(args.warmup):
        join(slices[k])
    t0 = time.perf_counter()
    done = 0
    for k in range(args.steps):
        join(slices[args.warmup + k])
        done += len(slices[args.warmup + k])
    dt = time.perf_counter() - t0
    v = done / dt
    sample = (f"the whole workload ({N} points) per step, grid-filtered oracle join on {n} threads" if whole else
              f"{per_step} of the workload's {N} points per step (consecutive slices), grid-filtered oracle "
              f"join on {n} threads; slice sized to the {args.ref_budget_s:.0f} s budget")
    print(json.dumps({
        "impl": "reference", "metric": metric_name(w.kind), "value": v, "unit": "points/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(w, args), "same_config": whole,
        "cpu_baseline": {"value": v, "unit": "points/s", "cores": n, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def time_joins(api, layer, w, pts, form, steps, warmup, world, stream, timed=True, ppi=0, clk=None, outs=None,
               knobs=None):
    """Mean CUDA-event time over `steps` joins after `warmup` untimed ones (the
    layer's counters cover the timed joins only); returns (total ms, stats,
    (out_id, out_d))."""
    import torch
    n = pts.shape[0]
    out_id = torch.empty(n, dtype=torch.int32, device=pts.device) if outs is None else outs[0]
    out_d = (torch.empty(n, dtype=torch.float64, device=pts.device) if outs is None else outs[1]) \
        if w.kind == "p2p" else None

    kn = knobs or {}

    def one(time_refine):
        if w.kind == "p2p":
            api.p2p_join(layer, pts, out_id, out_d, form=form, stream=stream, time_refine=time_refine,
                         pts_per_item=ppi, **kn)
        else:
            api.pip_join(layer, pts, out_id, form=form, stream=stream, time_refine=time_refine, pts_per_item=ppi,
                         **kn)

    for _ in range(warmup):
        one(False)
    torch.cuda.synchronize()
    layer.reset_stats()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.time()
    e0.record(stream)
    for _ in range(steps):
        one(timed)
    e1.record(stream)
    torch.cuda.synchronize()
    if clk is not None:
        clk.region(t0, time.time())
    barrier(world)
    return e0.elapsed_time(e1), layer.stats(), (out_id, out_d)


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
# the sources a refine kernel is compiled from: its file and the shared header
REFINE_SOURCES = {"p2p": ("paper_1403_0802_gb300/csrc/sj_p2p.cu", "paper_1403_0802_gb300/csrc/sj_internal.cuh"),
                  "pip": ("paper_1403_0802_gb300/csrc/sj_pip.cu", "paper_1403_0802_gb300/csrc/sj_internal.cuh")}


def sources_sha(kind):
    h = hashlib.sha256()
    for f in REFINE_SOURCES[kind]:
        with open(os.path.join(HERE, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(kernel, workload, kind):
    """DRAM bytes (read + write) per launch of `kernel` on `workload` from the
    committed ncu summary profiles/traffic.txt (lines: kernel workload bytes
    sha256-of-the-kernel's-sources), or None when absent or when those sources
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


def layer_bytes(w) -> int:
    """The layer read once: FP64 vertices and the offset arrays."""
    if w.kind == "p2p":
        return int(w.polylines.verts.nbytes + w.polylines.line_off.nbytes)
    P = w.polygons
    return int(P.verts.nbytes + P.ring_off.nbytes + P.poly_ring_off.nbytes)


def roofline_of(w, form, st, ms_per_join, peaks, census=None):
    """Roofline of the refinement launch (the dominant kernel), in the units of
    the algorithmic work the candidate lists imply (see the module docstring),
    with the executed-test rate and the join's HBM bound beside it."""
    hbm_peak = float(measured_peaks().get("hbm_gbs", 6800.0))
    refine_ms = st["refine_ms"] / max(st["refine_launches"], 1)
    joins = max(st["joins"], 1)
    algo = st["algo_tests"] / joins
    executed = st["edge_tests"] / joins
    if w.kind == "p2p":
        fpt = float(FLOPS_PER_SEGMENT)
        work_note = "unpruned (point, candidate-polyline segment) tests x 12 flops"
    else:
        frac_s = (census[1] / census[0]) if census and census[0] else 0.0
        fpt = FLOPS_PER_COMPARE + FLOPS_PER_STRADDLE * frac_s
        work_note = (f"unpruned (point, candidate-polygon edge) tests x (2 + 7 x {frac_s:.4f}: the straddling "
                     f"fraction counted by sj_pip_census)")
    peak = peaks["fp32"] if form == "fp32x" else peaks["fp64"]
    refine_s = refine_ms / 1e3
    achieved = algo * fpt / refine_s / 1e12 if refine_ms > 0 else None
    n = len(w.points)
    io = n * (16 + (12 if w.kind == "p2p" else 4))
    algo_bytes = io + layer_bytes(w)
    hbm_ach = algo_bytes / (ms_per_join / 1e3) / 1e9
    kernel = f"k_{w.kind}_refine<{form}>"
    r = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
         "frac": achieved / peak if achieved else None,
         "traffic": measured_traffic(kernel, w.name, w.kind),
         "peak_source": peaks["source"] + ("; FP32" if form == "fp32x" else "; FP64"),
         "peak_derived_cross_check": peaks["derived"]["fp32" if form == "fp32x" else "fp64"],
         "work": work_note, "flops_per_test": fpt,
         "refine_ms_per_launch": refine_ms, "algorithmic_tests_per_launch": algo,
         "executed_tests_per_launch": executed,
         "executed_frac": executed * fpt / refine_s / 1e12 / peak if refine_ms > 0 else None,
         "hbm": {"algorithmic_bytes_per_join": algo_bytes, "achieved_gbs": hbm_ach, "peak_gbs": hbm_peak,
                 "frac": hbm_ach / hbm_peak, "over": "the whole join (ms_per_step)",
                 "peak_source": "MEASURED_PEAKS.json hbm_gbs"}}
    if census:
        r["census"] = {"tests": census[0], "straddles": census[1], "points": census[2]}
    return r


def gpu_index(local):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0]
    return int(vis) if vis.isdigit() else local


def join_leg(api, args, w, dev, stream, world, steps, warmup, peaks, baselines=True, clocks_own=True):
    """Time `steps` joins of workload w (and, with baselines, the plain FP64
    form, the host-buffer form and the oracle on the host cores)."""
    import torch
    layer, layer_ms = build_layer(api, w, dev, stream)
    pts = torch.as_tensor(w.points, device=dev)
    n = pts.shape[0]
    t = tuned(args)
    ppi = t["ppi"]
    kn = dict(block=t["block"], edges_per_chunk=t["edges"])
    with ClockSampler(gpu_index(dist_env()[2])) as clk:
        ms, st, outs = time_joins(api, layer, w, pts, args.form, steps, warmup, world, stream, ppi=ppi, clk=clk,
                                  knobs=kn)
    clocks = clk.summary()
    ms_max = max_over_ranks(ms, world, dev)
    census = None
    if w.kind == "pip":
        k = min(n, 10_000_000)
        e_, s_ = api.pip_census(layer, pts[:k], stream=stream)
        census = (e_, s_, k)
    res = {"value": n * world * steps / (ms_max / 1000.0), "unit": "points/s", "steps": steps, "warmup": warmup,
           "ms_per_step": ms_max / steps, "dtype": "f32+f64" if args.form == "fp32x" else "f64",
           "config": dict(config_of(w, args), layer_build_ms=layer_ms,
                          parallelism=f"points sharded, layer replicated x{world}"),
           "roofline": roofline_of(w, args.form, st, ms / steps, peaks, census), "clocks": clocks,
           "fallbacks_per_join": st["fallbacks"] / max(st["joins"], 1),
           "edge_tests_per_s_algorithmic": st["algo_tests"] / (ms / 1000.0)}
    gid = outs[0].cpu().numpy()
    gd = outs[1].cpu().numpy() if outs[1] is not None else None
    if baselines and args.form != "fp64":
        k64 = max(3, min(steps, 20))
        with ClockSampler(gpu_index(dist_env()[2])) as clk64:
            ms64, st64, _ = time_joins(api, layer, w, pts, "fp64", k64, 2, 1, stream, ppi=ppi, clk=clk64, knobs=kn)
        res["fp64_plain"] = {"value": n * k64 / (ms64 / 1000.0), "unit": "points/s", "ms_per_step": ms64 / k64,
                             "steps": k64, "roofline": roofline_of(w, "fp64", st64, ms64 / k64, peaks, census),
                             "clocks": clk64.summary()}
        res["speedup_vs_fp64_plain"] = res["value"] / res["fp64_plain"]["value"]
    if baselines:
        hp = torch.empty((n, 2), dtype=torch.float64, pin_memory=True)
        hp.copy_(torch.from_numpy(w.points))
        hid = torch.empty(n, dtype=torch.int32, pin_memory=True)
        hd = torch.empty(n, dtype=torch.float64, pin_memory=True)
        ke = max(3, min(steps, 20))
        if w.kind == "p2p":
            join_host = lambda: api.p2p_join_host(layer, hp, hid, hd, form=args.form, stream=stream,
                                                  pts_per_item=ppi, **kn)
        else:
            join_host = lambda: api.pip_join_host(layer, hp, hid, form=args.form, stream=stream, pts_per_item=ppi,
                                                  **kn)
        for _ in range(2):
            join_host()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            join_host()      # synchronous: copies in, join, copies out
        ems = (time.perf_counter() - t0) * 1e3
        res["e2e"] = {"value": n * ke / (ems / 1000.0), "unit": "points/s", "h2d_bytes_per_step": n * 16,
                      "d2h_bytes_per_step": n * (4 + (8 if w.kind == "p2p" else 0)), "steps": ke,
                      "api": "sj_p2p_join_host" if w.kind == "p2p" else "sj_pip_join_host",
                      "timing": "host wall clock around synchronous calls (pinned buffers)"}
        del hp, hid, hd
        res["cpu_baseline"] = cpu_baseline(w, gpu=(gid, gd), form=args.form)
    layer.close()
    del pts, outs
    torch.cuda.empty_cache()
    return res


def sub_steps(ms_hint: float, steps: int) -> int:
    """Joins to time in an extra leg: the run's step count, raised so that the
    timed region lasts at least SUB_LEG_MIN_S (several clock samples)."""
    return int(min(2000, max(steps, math.ceil(SUB_LEG_MIN_S * 1e3 / max(ms_hint, 1e-3)))))


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
    peaks = alu_peaks(api)
    w = workload(args, rank)
    stream = torch.cuda.current_stream(dev)
    baselines = rank == 0 and world == 1 and not args.no_baselines
    head = join_leg(api, args, w, dev, stream, world, args.steps, args.warmup, peaks, baselines=baselines)
    # cell_hist, the scan (2 phases up to 256 tiles of 1,024 cells, else 3), scatter; refine; FP32X P2P
    # recheck; unsort
    scan_tiles = (int(w.grid["nx"]) * int(w.grid["ny"]) + 1023) // 1024
    kernels_per_join = 1 + (2 if scan_tiles <= 256 else 3) + 1 + 1 + (1 if (w.kind == "p2p" and args.form == "fp32x") else 0) + 1
    extra = {}
    if rank == 0 and world == 1 and args.workload == "p2p" and not args.no_extra and not args.points:
        import copy
        # serving first: its host-bound loop measured the same on a fresh box
        # whatever ran before, but its tail latencies grew 3-10x (both modes)
        # minutes into a call on this shared machine
        extra["serve"] = serve_leg_child(args)
        a1 = copy.copy(args)
        a1.workload, a1.ppi = "pip", 0
        ws = workload(a1)
        extra["pip_stars"] = join_leg(api, a1, ws, dev, stream, 1, sub_steps(0.12, args.steps), 3, peaks,
                                      baselines=not args.no_baselines)
        del ws
        for layer in (1, 2):      # the PIP-at-scale layers (the same 100 M points)
            a2 = copy.copy(args)
            a2.workload, a2.layer, a2.ppi = "pip3", layer, 0
            wt = workload(a2)
            extra[f"pip_at_scale_layer{layer}"] = join_leg(api, a2, wt, dev, stream, 1, sub_steps(7.0, args.steps),
                                                           3, peaks, baselines=not args.no_baselines)
            del wt
        a4 = copy.copy(args)
        a4.workload, a4.ppi = "p2p4", 0
        w4 = workload(a4)
        base_name = w4.name
        for D in (50.0, 100.0, 200.0):   # P2P at scale: one layer per window, the same 170 M points
            w4.D = D
            w4.name = base_name.replace("_D100_", f"_D{int(D)}_")
            extra[f"p2p_at_scale_D{int(D)}"] = join_leg(api, a4, w4, dev, stream, 1, sub_steps(15.0, args.steps), 3,
                                                        peaks, baselines=not args.no_baselines)
        del w4
    if rank == 0:
        line = {
            "metric": metric_name(w.kind), "value": head["value"], "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": head["dtype"], "data": "synthetic", "config": head["config"],
            "roofline": head["roofline"], "cpu_baseline": head.get("cpu_baseline"), "e2e": head.get("e2e"),
            "clocks": head["clocks"], "gpu_launches": kernels_per_join * args.steps,
            "alu_peaks_tflops": {k: peaks[k] for k in ("fp32", "fp64", "source")},
            **{k: head[k] for k in ("fallbacks_per_join", "edge_tests_per_s_algorithmic", "fp64_plain",
                                    "speedup_vs_fp64_plain") if k in head},
            **extra,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def serve_leg_child(args):
    """The serving leg in a process of its own (python bench.py --workload
    serve): the earlier legs leave host state behind -- multi-GB pinned
    buffers, the oracle's host threads -- that slows a host-bound serving loop
    run after them in the same process."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "serve", "--requests", str(args.requests),
           "--form", args.form, "--serve-grid-pip", str(args.serve_grid_pip), "--serve-grid-p2p",
           str(args.serve_grid_p2p)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    if r.returncode != 0 or not lines:
        return {"error": f"serving leg exited {r.returncode}: {r.stderr[-500:]}"}
    return json.loads(lines[-1])


def serve_leg(args):
    """Continuous batching (native server, batched engine rounds) against one
    join call per request in the same native loop -- in the same form and in
    the plain FP64 form -- on one Poisson stream of requests."""
    import torch
    world, rank, local = dist_env()
    from paper_1403_0802_gb300 import api, build, serve, synth
    build.build()
    torch.cuda.set_device(local)
    # serving grids: every join pays for a scan over the grid's cells, which
    # dominates requests of a few thousand points, so the serving layers use
    # coarser grids than the 100 M-point joins
    wp = synth.pip_tiles(n_points=20_000_000, layer=1, grid_n=args.serve_grid_pip)
    wl = synth.p2p_walks_lognormal(n_points=20_000_000, n_lines=150_000, D=100.0, grid_n=args.serve_grid_p2p)
    pip = api.pip_layer(wp.polygons.verts, wp.polygons.ring_off, wp.polygons.poly_ring_off, wp.grid)
    p2p = api.p2p_layer(wl.polylines.verts, wl.polylines.line_off, wl.D, wl.grid)
    pool_p = torch.from_numpy(wp.points).pin_memory()
    pool_l = torch.from_numpy(wl.points).pin_memory()
    outs = {serve.PIP: (torch.empty(len(pool_p), dtype=torch.int32, pin_memory=True), None),
            serve.P2P: (torch.empty(len(pool_l), dtype=torch.int32, pin_memory=True),
                        torch.empty(len(pool_l), dtype=torch.float64, pin_memory=True))}
    srv = serve.Server(pip, p2p, form=args.form, round_points=6_000_000, max_requests=4096)
    arms = [("batched", args.form), ("per_request", args.form), ("per_request", "fp64")]
    # a coarser period here: the serving loop is host-bound (copies, a worker
    # thread) and its timed regions last seconds
    with ClockSampler(gpu_index(local), period_ms=200) as clk:
        for mode, form in arms:      # warm-up: workspaces, graphs, allocator pools
            srv.run(serve.make_stream(32, 0.0, pool_p, pool_l, seed=1), mode=mode, form=form, out_pools=outs)

        def timed(reqs, mode, form):
            t0 = time.time()
            r = srv.run(reqs, mode=mode, form=form, out_pools=outs)
            clk.region(t0, time.time())
            return r

        # capacity of each arm with every request queued at t = 0
        sat = {f"{m}_{f}": timed(serve.make_stream(min(args.requests, 300), 0.0, pool_p, pool_l, seed=3), m, f)
               for m, f in arms}
        mean_pts = sat[f"batched_{args.form}"]["points"] / sat[f"batched_{args.form}"]["requests"]
        base = sat["per_request_fp64"]["points_per_s"]          # the plain FP64 one-launch-per-request form
        res = {}
        for rho in (0.5, 0.8):
            rate = rho * base / mean_pts
            for m, f in arms:
                reqs = serve.make_stream(args.requests, rate, pool_p, pool_l, seed=7)
                res[f"{m}_{f}_rho{rho}"] = timed(reqs, m, f)
        fast = sat[f"per_request_{args.form}"]["points_per_s"]  # a load the FP64 form cannot sustain
        for m, f in arms[:2]:
            reqs = serve.make_stream(args.requests, 0.8 * fast / mean_pts, pool_p, pool_l, seed=7)
            res[f"{m}_{f}_rho0.8_of_{args.form}_capacity"] = timed(reqs, m, f)
    b, p64 = res[f"batched_{args.form}_rho0.8"], res["per_request_fp64_rho0.8"]
    pr = res[f"per_request_{args.form}_rho0.8"]
    line = {"metric": "serving p50/p99 latency (ms) and points/s, continuous batching", "value": b["p99_ms"],
            "unit": "ms (p99)", "n_gpus": 1, "steps": args.requests, "warmup": 32, "ms_per_step": b["mean_ms"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.form == "fp32x" else "f64", "data": "synthetic",
            "config": {"workload": f"serve_{args.requests}req_pip40k_p2p150k", "requests": args.requests,
                       "grids": f"PIP {args.serve_grid_pip}^2, P2P {args.serve_grid_p2p}^2",
                       "sizes": "log-uniform 1e3..5e6 points", "mix": "70% PIP / 30% P2P (D=100 m)",
                       "arrivals": "Poisson, rate = rho x capacity of the plain FP64 one-join-per-request form",
                       "form": args.form, "server": "native (sj_server_*), batched engine rounds",
                       "bounded": "nothing: 10,000 requests per stream as stated; point pools of 20 M points "
                                  "per kind (requests are slices of them)"},
            "p50_ms": b["p50_ms"], "p99_ms": b["p99_ms"], "points_per_s": b["points_per_s"],
            "per_request_p50_ms": pr["p50_ms"], "per_request_p99_ms": pr["p99_ms"],
            "plain_fp64_per_request_p50_ms": p64["p50_ms"], "plain_fp64_per_request_p99_ms": p64["p99_ms"],
            "plain_fp64_per_request_points_per_s": p64["points_per_s"],
            "capacity_points_per_s": {k: v["points_per_s"] for k, v in sat.items()},
            "clocks": clk.summary(), "capacity": sat, "runs": res}
    srv.close()
    pip.close()
    p2p.close()
    del pool_p, pool_l, outs
    torch.cuda.empty_cache()
    return line


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serve":
        world, rank, _ = dist_env()
        if rank == 0:
            print(json.dumps(serve_leg(args)))
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
