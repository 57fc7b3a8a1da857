"""Autotuner for the join's launch knobs.

Knobs (none changes a result):
  * points per work item -- how many points of a cell one warp refines
    against the cell's staged candidates;
  * edges per chunk -- the edge budget of a work item: a cell whose points
    each test more edges is cut into smaller items, so heavy cells (complex
    polygons, Sec. IV.C; dense polyline cells) spread over more warps;
  * block -- warps per refinement block (2, 4 or 8);
  * the filter grid resolution (Sec. III.A: a finer grid gives fewer false
    candidates but more cells and smaller items -- the paper's own
    trade-off, left to tuning);
  * the arithmetic form.
Each setting is timed with CUDA events over a few joins of the given points
after a warm-up; the fastest setting is returned with the whole table.

    python -m paper_1403_0802_gb300.autotune --workload pip3 --layer 2 --points 10000000
"""
from __future__ import annotations

import argparse
import itertools
import json
import time

import torch

from . import api, synth


def time_join(layer, pts, kind: str, form: str, ppi: int, steps: int = 8, warmup: int = 2, block: int = 0,
              edges_per_chunk: int = 0) -> float:
    """Mean milliseconds per join."""
    n = pts.shape[0]
    out_id = torch.empty(n, dtype=torch.int32, device=pts.device)
    out_d = torch.empty(n, dtype=torch.float64, device=pts.device)
    stream = torch.cuda.current_stream()
    kw = dict(form=form, pts_per_item=ppi, stream=stream, block=block, edges_per_chunk=edges_per_chunk)

    def one():
        if kind == "p2p":
            api.p2p_join(layer, pts, out_id, out_d, **kw)
        else:
            api.pip_join(layer, pts, out_id, **kw)

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
             blocks=(4,), edges=(0,), steps: int = 8) -> dict:
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
            for form, ppi, nw, epc in itertools.product(forms, ppis, blocks, edges):
                ms = time_join(layer, pts, w.kind, form, ppi, steps=steps, block=nw, edges_per_chunk=epc)
                table.append({"grid": g, "pts_per_item": ppi, "block": nw, "edges_per_chunk": epc, "form": form,
                              "ms": ms, "points_per_s": len(w.points) / (ms / 1e3), "layer_build_ms": build_ms})
    best = min(table, key=lambda r: r["ms"])
    return {"workload": w.name, "best": best, "table": table}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["p2p", "pip", "pip3", "p2p4"], default="p2p")
    ap.add_argument("--points", type=int, default=2_000_000)
    ap.add_argument("--layer", type=int, default=1)
    ap.add_argument("--grids", default="512,1024,2048")
    ap.add_argument("--ppis", default="16,32,64,128")
    ap.add_argument("--blocks", default="2,4,8")
    ap.add_argument("--edges", default="0,64,256,1024")
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
    ints = lambda x: [int(v) for v in x.split(",")]
    res = autotune(w, grids=ints(a.grids), ppis=ints(a.ppis), forms=a.forms.split(","), blocks=ints(a.blocks),
                   edges=ints(a.edges))
    print(json.dumps(res))


if __name__ == "__main__":
    main()
