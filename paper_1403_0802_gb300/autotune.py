"""Autotuner for the join's launch knobs.

Knobs: points per work item (how many points of a cell one warp refines
against the cell's staged candidates), the filter grid resolution (Sec. III.A:
a finer grid gives fewer false candidates but more cells and smaller items --
the paper's own trade-off, left to tuning), and the arithmetic form.  Each
setting is timed with CUDA events over a few joins of the given points after a
warm-up; the fastest setting is returned with the whole table.

    python -m paper_1403_0802_gb300.autotune --workload p2p --points 2000000
"""
from __future__ import annotations

import argparse
import itertools
import json
import time

import torch

from . import api, synth


def time_join(layer, pts, kind: str, form: str, ppi: int, steps: int = 8, warmup: int = 2) -> float:
    """Mean milliseconds per join."""
    n = pts.shape[0]
    out_id = torch.empty(n, dtype=torch.int32, device=pts.device)
    out_d = torch.empty(n, dtype=torch.float64, device=pts.device)
    stream = torch.cuda.current_stream()

    def one():
        if kind == "p2p":
            api.p2p_join(layer, pts, out_id, out_d, form=form, pts_per_item=ppi, stream=stream)
        else:
            api.pip_join(layer, pts, out_id, form=form, pts_per_item=ppi, stream=stream)

    for _ in range(warmup):
        one()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        one()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def autotune(w: synth.Workload, grids=(512, 1024, 2048), ppis=(16, 32, 64, 128), forms=("fp32x",),
             steps: int = 8) -> dict:
    pts = torch.as_tensor(w.points, device="cuda")
    table = []
    for g in grids:
        grid = synth.grid(g)
        if w.kind == "p2p":
            L = w.polylines
            t0 = time.perf_counter()
            layer = api.p2p_layer(L.verts, L.line_off, w.D, grid)
        else:
            P = w.polygons
            t0 = time.perf_counter()
            layer = api.pip_layer(P.verts, P.ring_off, P.poly_ring_off, grid)
        build_ms = (time.perf_counter() - t0) * 1e3
        with layer:
            for form, ppi in itertools.product(forms, ppis):
                ms = time_join(layer, pts, w.kind, form, ppi, steps=steps)
                table.append({"grid": g, "pts_per_item": ppi, "form": form, "ms": ms,
                              "points_per_s": len(w.points) / (ms / 1e3), "layer_build_ms": build_ms})
    best = min(table, key=lambda r: r["ms"])
    return {"workload": w.name, "best": best, "table": table}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["p2p", "pip", "pip3", "p2p4"], default="p2p")
    ap.add_argument("--points", type=int, default=2_000_000)
    ap.add_argument("--layer", type=int, default=1)
    ap.add_argument("--grids", default="512,1024,2048")
    ap.add_argument("--ppis", default="16,32,64,128")
    ap.add_argument("--forms", default="fp32x")
    a = ap.parse_args()
    if a.workload == "p2p":
        w = synth.p2p_walks(n_points=a.points)
    elif a.workload == "pip":
        w = synth.pip_stars(n_points=a.points)
    elif a.workload == "pip3":
        w = synth.pip_tiles(n_points=a.points, layer=a.layer)
    else:
        w = synth.p2p_walks_lognormal(n_points=a.points)
    res = autotune(w, grids=[int(x) for x in a.grids.split(",")], ppis=[int(x) for x in a.ppis.split(",")],
                   forms=a.forms.split(","))
    print(json.dumps(res))


if __name__ == "__main__":
    main()
