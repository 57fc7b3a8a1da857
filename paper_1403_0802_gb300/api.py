"""Python front end of libsj.so: argument marshalling only.

Every step of the join runs in the library's CUDA kernels; this module turns
torch tensors (device memory, streams) and numpy arrays into the pointers and
sizes of the C ABI in include/sj.h.

    layer = pip_layer(verts, ring_off, poly_ring_off, grid)      # resident polygon layer
    ids = pip_join(layer, pts)                                     # torch int32 [N] on the GPU
    layer = p2p_layer(verts, line_off, D, grid)                    # resident polyline layer
    ids, d = p2p_join(layer, pts, form="fp32x")                    # nearest polyline within D
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L

FORMS = {"fp64": L.SJ_FP64, "fp32x": L.SJ_FP32X}
LAUNCHES = {"per_request": L.SJ_PER_REQUEST, "persistent": L.SJ_PERSISTENT}


def _grid(g) -> L.sj_grid:
    return L.sj_grid(float(g["x0"]), float(g["y0"]), float(g["x1"]), float(g["y1"]), int(g["nx"]), int(g["ny"]))


def _stream(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if isinstance(stream, torch.cuda.Stream) else int(stream)


def _opts(form="fp64", launch="per_request", pts_per_item=0, time_refine=False, subcell=None, block=0,
          edges_per_chunk=0) -> L.sj_opts:
    flags = L.SJ_FLAG_TIME_REFINE if time_refine else 0
    if subcell is not None:
        flags |= L.SJ_FLAG_SUBCELL_ON if subcell else L.SJ_FLAG_SUBCELL_OFF
    return L.sj_opts(FORMS[form], LAUNCHES[launch], int(block), int(pts_per_item), int(edges_per_chunk), flags)


def _dev(a, dtype, device="cuda") -> torch.Tensor:
    if isinstance(a, torch.Tensor):
        t = a.to(device=device, dtype=dtype)
    else:
        t = torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=device)
    return t.contiguous()


def _ptr(t: torch.Tensor | None):
    return None if t is None or t.numel() == 0 else t.data_ptr()


class Layer:
    """A resident polygon (kind 0) or polyline (kind 1) layer with its grid index."""

    def __init__(self, handle: int, grid: dict, kind: int, D: float = 0.0):
        self._h = C.c_void_p(handle)
        self.grid = dict(grid)
        self.kind = kind
        self.D = D

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("layer destroyed")
        return self._h

    def info(self) -> dict:
        inf = L.sj_layer_info()
        L.check(L.lib().sj_layer_get_info(self.handle, C.byref(inf)), "sj_layer_get_info")
        return {f: getattr(inf, f) for f, _ in inf._fields_}

    def candidates(self):
        """Per-cell candidate lists: (cand_start int32 [G+1], cand_ids int32 [M])."""
        inf = self.info()
        start = np.empty(inf["n_cells"] + 1, np.int32)
        ids = np.empty(max(inf["n_candidates"], 1), np.int32)
        L.check(L.lib().sj_layer_get_candidates(self.handle, start.ctypes.data, ids.ctypes.data),
                "sj_layer_get_candidates")
        return start, ids[:inf["n_candidates"]]

    def stats(self) -> dict:
        st = L.sj_run_stats()
        L.check(L.lib().sj_layer_get_stats(self.handle, C.byref(st)), "sj_layer_get_stats")
        return {f: getattr(st, f) for f, _ in st._fields_}

    def reset_stats(self):
        L.check(L.lib().sj_layer_reset_stats(self.handle), "sj_layer_reset_stats")

    def close(self):
        if self._h:
            L.lib().sj_layer_destroy(self._h)
            self._h = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def pip_layer(verts, ring_off, poly_ring_off, grid: dict, stream=None) -> Layer:
    v = _dev(verts, torch.float64).reshape(-1, 2)
    ro = _dev(ring_off, torch.int64)
    pro = _dev(poly_ring_off, torch.int64)
    h = C.c_void_p()
    g = _grid(grid)
    L.check(L.lib().sj_pip_layer_create(_ptr(v), v.shape[0], ro.data_ptr(), ro.numel() - 1, pro.data_ptr(),
                                        pro.numel() - 1, C.byref(g), _stream(stream), C.byref(h)),
            "sj_pip_layer_create")
    return Layer(h.value, grid, 0)


def p2p_layer(verts, line_off, D: float, grid: dict, stream=None) -> Layer:
    v = _dev(verts, torch.float64).reshape(-1, 2)
    lo = _dev(line_off, torch.int64)
    h = C.c_void_p()
    g = _grid(grid)
    L.check(L.lib().sj_p2p_layer_create(_ptr(v), v.shape[0], lo.data_ptr(), lo.numel() - 1, float(D), C.byref(g),
                                        _stream(stream), C.byref(h)), "sj_p2p_layer_create")
    return Layer(h.value, grid, 1, float(D))


def _points(pts) -> torch.Tensor:
    p = pts if isinstance(pts, torch.Tensor) and pts.is_cuda else _dev(pts, torch.float64)
    if p.dtype != torch.float64 or p.dim() != 2 or p.shape[1] != 2:
        raise ValueError("points must be a float64 [N, 2] tensor")
    return p.contiguous()


def pip_join(layer: Layer, pts, out: torch.Tensor | None = None, form: str = "fp64", launch: str = "per_request",
             pts_per_item: int = 0, stream=None, time_refine: bool = False, subcell: bool | None = None,
             block: int = 0, edges_per_chunk: int = 0) -> torch.Tensor:
    """Polygon id (or -1) per point, int32 on the points' device (Sec. III.C).
    Launch knobs (results do not depend on them): subcell orders points by
    sub-cell inside their cells (None: the library's choice), block = warps per
    refinement block (0: 4), edges_per_chunk = the edge budget of a work item
    (0: the library default, 64 for polygon layers)."""
    p = _points(pts)
    out = torch.empty(p.shape[0], dtype=torch.int32, device=p.device) if out is None else out
    o = _opts(form, launch, pts_per_item, time_refine, subcell, block, edges_per_chunk)
    L.check(L.lib().sj_pip_join(layer.handle, _ptr(p), p.shape[0], _ptr(out), C.byref(o), _stream(stream)),
            "sj_pip_join")
    return out


def p2p_join(layer: Layer, pts, out_id: torch.Tensor | None = None, out_d: torch.Tensor | None = None,
             form: str = "fp64", launch: str = "per_request", pts_per_item: int = 0, stream=None,
             time_refine: bool = False, window: float | None = None, subcell: bool | None = None,
             block: int = 0, edges_per_chunk: int = 0):
    """(nearest polyline id or -1, distance or +inf) per point (Sec. III.B); window (<= the layer's D)
    replaces D for this call (sj_p2p_join_window); launch knobs as in pip_join."""
    p = _points(pts)
    n = p.shape[0]
    out_id = torch.empty(n, dtype=torch.int32, device=p.device) if out_id is None else out_id
    out_d = torch.empty(n, dtype=torch.float64, device=p.device) if out_d is None else out_d
    o = _opts(form, launch, pts_per_item, time_refine, subcell, block, edges_per_chunk)
    if window is None:
        L.check(L.lib().sj_p2p_join(layer.handle, _ptr(p), n, _ptr(out_id), _ptr(out_d), C.byref(o),
                                    _stream(stream)), "sj_p2p_join")
    else:
        L.check(L.lib().sj_p2p_join_window(layer.handle, _ptr(p), n, float(window), _ptr(out_id), _ptr(out_d),
                                           C.byref(o), _stream(stream)), "sj_p2p_join_window")
    return out_id, out_d


def p2p_join_noalloc(layer: Layer, pts, out_id: torch.Tensor, out_d: torch.Tensor | None = None,
                     form: str = "fp64", stream=None):
    """p2p_join for callers that must not allocate device memory: the caller
    supplies the outputs and the library takes its scratch from a fixed
    built-in device array (at most 524,288 points and 1,048,576 grid cells per
    call; calls must not overlap on the GPU).  Nothing here allocates either:
    the points must already be a float64 [N, 2] CUDA tensor."""
    if not (isinstance(pts, torch.Tensor) and pts.is_cuda and pts.dtype == torch.float64 and pts.is_contiguous()):
        raise ValueError("points must be a contiguous float64 [N, 2] CUDA tensor")
    o = _opts(form)
    L.check(L.lib().sj_p2p_join_noalloc(layer.handle, _ptr(pts), pts.shape[0], _ptr(out_id), _ptr(out_d), C.byref(o),
                                        _stream(stream)), "sj_p2p_join_noalloc")
    return out_id, out_d


def pip_census(layer: Layer, pts, stream=None) -> tuple[int, int]:
    """(edges of the candidate polygons, edges straddling the point's y),
    summed over the points: the algorithmic PIP work (sj_pip_census)."""
    p = _points(pts)
    out = (C.c_int64 * 2)()
    L.check(L.lib().sj_pip_census(layer.handle, _ptr(p), p.shape[0], out, _stream(stream)), "sj_pip_census")
    return int(out[0]), int(out[1])


def pip_join_host(layer: Layer, pts: np.ndarray, out: np.ndarray | None = None, form: str = "fp64",
                  stream=None, pts_per_item: int = 0, block: int = 0, edges_per_chunk: int = 0) -> np.ndarray:
    """Same as pip_join from host memory (copies in and out; synchronous)."""
    p = np.ascontiguousarray(pts, dtype=np.float64) if not isinstance(pts, torch.Tensor) else pts
    n = p.shape[0]
    out = np.empty(n, np.int32) if out is None else out
    o = _opts(form, pts_per_item=pts_per_item, block=block, edges_per_chunk=edges_per_chunk)
    pp = p.data_ptr() if isinstance(p, torch.Tensor) else p.ctypes.data
    op = out.data_ptr() if isinstance(out, torch.Tensor) else out.ctypes.data
    L.check(L.lib().sj_pip_join_host(layer.handle, pp, n, op, C.byref(o), _stream(stream)), "sj_pip_join_host")
    return out


def p2p_join_host(layer: Layer, pts, out_id=None, out_d=None, form: str = "fp64", stream=None,
                  pts_per_item: int = 0, window: float | None = None, block: int = 0, edges_per_chunk: int = 0):
    """Same as p2p_join from host memory (copies in and out; synchronous); window as in p2p_join."""
    p = np.ascontiguousarray(pts, dtype=np.float64) if not isinstance(pts, torch.Tensor) else pts
    n = p.shape[0]
    out_id = np.empty(n, np.int32) if out_id is None else out_id
    out_d = np.empty(n, np.float64) if out_d is None else out_d
    o = _opts(form, pts_per_item=pts_per_item, block=block, edges_per_chunk=edges_per_chunk)
    ptr = lambda a: a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data
    if window is None:
        L.check(L.lib().sj_p2p_join_host(layer.handle, ptr(p), n, ptr(out_id), ptr(out_d), C.byref(o),
                                         _stream(stream)), "sj_p2p_join_host")
    else:
        L.check(L.lib().sj_p2p_join_window_host(layer.handle, ptr(p), n, float(window), ptr(out_id), ptr(out_d),
                                                C.byref(o), _stream(stream)), "sj_p2p_join_window_host")
    return out_id, out_d


def bucket_points(pts, grid: dict, stream=None):
    """Cell bucketing alone (Sec. III.A): (cell_start int32 [G+1], perm int32 [N])."""
    p = _points(pts)
    G = int(grid["nx"]) * int(grid["ny"])
    cs = torch.empty(G + 1, dtype=torch.int32, device=p.device)
    perm = torch.full((p.shape[0],), -1, dtype=torch.int32, device=p.device)
    g = _grid(grid)
    L.check(L.lib().sj_bucket_points(_ptr(p), p.shape[0], C.byref(g), cs.data_ptr(), _ptr(perm), _stream(stream)),
            "sj_bucket_points")
    return cs, perm


def pip_join_once(points, verts, ring_off, poly_ring_off, grid: dict, form: str = "fp64") -> torch.Tensor:
    """pip_join(points, polygons, grid): build the layer, join, free it."""
    with pip_layer(verts, ring_off, poly_ring_off, grid) as layer:
        out = pip_join(layer, points, form=form)
        torch.cuda.current_stream().synchronize()
        return out


def p2p_join_once(points, verts, line_off, D: float, grid: dict, form: str = "fp64"):
    """p2p_join(points, polylines, D, grid): build the layer, join, free it."""
    with p2p_layer(verts, line_off, D, grid) as layer:
        res = p2p_join(layer, points, form=form)
        torch.cuda.current_stream().synchronize()
        return res


class Engine:
    """Batched rounds (continuous batching) over resident layers.

        eng = Engine(max_points=8_000_000, max_requests=256, form="fp32x")
        eng.round([(pip_layer, pts_a, ids_a, None), (p2p_layer, pts_b, ids_b, d_b)], stream)

    Each request is (layer, points [N, 2] f64 CUDA tensor, out_id int32 [N],
    out_d f64 [N] or None[, window]); outputs are written asynchronously on
    `stream`.  A window (polyline layers, <= the layer's D) replaces D for that
    request alone.
    """

    def __init__(self, max_points: int, max_requests: int = 1024, form: str = "fp64", pts_per_item: int = 0,
                 graph: bool = True):
        o = L.sj_opts(FORMS[form], L.SJ_PERSISTENT, 0, int(pts_per_item), 0, 0 if graph else L.SJ_FLAG_NO_GRAPH)
        h = C.c_void_p()
        L.check(L.lib().sj_engine_create(int(max_points), int(max_requests), C.byref(o), C.byref(h)),
                "sj_engine_create")
        self._h = h
        self.max_points = int(max_points)
        self.max_requests = int(max_requests)
        self.form = form

    def round(self, requests, stream=None):
        arr = (L.sj_request * max(len(requests), 1))()
        for k, req in enumerate(requests):
            layer, pts, out_id, out_d = req[:4]
            window = req[4] if len(req) > 4 else None
            arr[k] = L.sj_request(layer.handle.value, _ptr(pts), pts.shape[0], _ptr(out_id),
                                  _ptr(out_d) if out_d is not None else None, 0 if window is None else 1, 0,
                                  0.0 if window is None else float(window))
        L.check(L.lib().sj_engine_round(self._h, arr, len(requests), _stream(stream)), "sj_engine_round")

    def close(self):
        if self._h:
            L.lib().sj_engine_destroy(self._h)
            self._h = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def version() -> str:
    return L.lib().sj_version().decode()
