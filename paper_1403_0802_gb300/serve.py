"""Continuous-batching serving over resident layers (Python side).

Requests (a batch of GPS points and a kind: PIP against the resident polygon
layer or P2P against the resident polyline layer) arrive over time.  The
serving loop itself is native (include/sj_serve.h, csrc/sj_serve.cu): a worker
thread admits queued requests in arrival order while their device memory fits
a fixed budget, copies their points in on one stream, runs them in rounds
through the batched engine (one graph replay per layer per round, so requests
that arrive while a round runs join the next one) and copies results back on
another stream.  This module generates request streams, hands them to the
server with their arrival times (the worker admits each request no earlier
than its arrival), and reports latency (results in host memory minus
arrival) and throughput.

mode="per_request" runs the same native loop with one join call per request
in arrival order -- the baseline the batched form is measured against -- in
the server's form or another one (form="fp64" gives the plain FP64 form).
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L
from . import api

PIP, P2P = 0, 1


@dataclass
class Request:
    rid: int
    arrival: float          # seconds from the start of the run
    kind: int               # PIP or P2P
    pts: torch.Tensor       # pinned host float64 [N, 2]
    t_done: float = math.nan
    out_id: torch.Tensor | None = None    # pinned host int32 [N]
    out_d: torch.Tensor | None = None     # pinned host float64 [N] (P2P)
    window: float | None = None           # P2P: window of this request (None = the layer's D)
    off: int = 0                          # first point's index in its pool

    @property
    def n(self) -> int:
        return int(self.pts.shape[0])

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


def make_stream(n_requests: int, rate_per_s: float, pool_pip: torch.Tensor, pool_p2p: torch.Tensor,
                size_min: int = 1_000, size_max: int = 5_000_000, pip_frac: float = 0.7,
                seed: int = 20140309, p2p_windows: tuple[float, ...] | None = None) -> list[Request]:
    """Poisson arrivals (all at t = 0 when rate_per_s is 0); sizes log-uniform in
    [size_min, size_max]; points are slices of pinned host pools of clustered
    points (one pool per kind); each P2P request asks for a window drawn
    uniformly from p2p_windows (None: the layer's D)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, n_requests)) if rate_per_s > 0 else np.zeros(n_requests)
    reqs = []
    for k in range(n_requests):
        kind = PIP if rng.random() < pip_frac else P2P
        pool = pool_pip if kind == PIP else pool_p2p
        n = int(round(math.exp(rng.uniform(math.log(size_min), math.log(size_max)))))
        n = min(n, pool.shape[0])
        off = int(rng.integers(0, pool.shape[0] - n + 1))
        win = float(p2p_windows[int(rng.integers(0, len(p2p_windows)))]) if (p2p_windows and kind == P2P) else None
        reqs.append(Request(k, float(t[k]), kind, pool[off:off + n], window=win, off=off))
    return reqs


class Server:
    """Resident layers and a native continuous-batching server (sj_server_*)."""

    def __init__(self, pip_layer: api.Layer, p2p_layer: api.Layer, form: str = "fp32x",
                 round_points: int = 16_000_000, max_requests: int = 1024, hbm_budget: int | None = None,
                 pts_per_item: int = 0):
        self.layers = {PIP: pip_layer, P2P: p2p_layer}
        self.form = form
        self.round_points = int(round_points)
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info()
            hbm_budget = int(0.25 * free)
        o = api._opts(form, "persistent", pts_per_item)
        h = C.c_void_p()
        L.check(L.lib().sj_server_create(pip_layer.handle if pip_layer else None,
                                         p2p_layer.handle if p2p_layer else None, C.byref(o),
                                         L.SJ_SERVE_BATCHED, int(hbm_budget), self.round_points,
                                         int(max_requests), C.byref(h)), "sj_server_create")
        self.handle = h

    def close(self):
        if self.handle:
            L.lib().sj_server_destroy(self.handle)
            self.handle = None

    def stats(self) -> dict:
        s = L.sj_server_stats()
        L.check(L.lib().sj_server_get_stats(self.handle, C.byref(s)), "sj_server_get_stats")
        return {k: getattr(s, k) for k, _ in s._fields_}

    def run(self, requests: list[Request], mode: str = "batched", form: str | None = None,
            out_pools: dict | None = None) -> dict:
        """Replay `requests` on the server: each is submitted up front with its
        arrival time (seconds from now) as not_before, so the native worker
        admits it then; returns latency (results in host memory - arrival) and
        throughput statistics.  out_pools ({kind: (ids, distances or None)},
        pinned host tensors as long as the point pools) makes each request's
        outputs the slice of the pool at its points' offset instead of buffers
        of its own: requests that share points then write the same values to
        the same bytes, so long streams need no memory per request."""
        assert mode in ("batched", "per_request")
        lib = L.lib()
        L.check(lib.sj_server_set_mode(self.handle, L.SJ_SERVE_BATCHED if mode == "batched" else
                                       L.SJ_SERVE_PER_REQUEST, api.FORMS[form or self.form]), "sj_server_set_mode")
        order = sorted(requests, key=lambda r: r.arrival)
        for r in order:
            if out_pools is not None:
                ids, ds = out_pools[r.kind]
                r.out_id = ids[r.off:r.off + r.n]
                r.out_d = ds[r.off:r.off + r.n] if (r.kind == P2P and ds is not None) else None
            else:
                r.out_id = torch.empty(r.n, dtype=torch.int32, pin_memory=True)
                r.out_d = torch.empty(r.n, dtype=torch.float64, pin_memory=True) if r.kind == P2P else None
            r.t_done = math.nan
        st0 = self.stats()
        L.check(lib.sj_server_reset_maxima(self.handle), "sj_server_reset_maxima")
        req = L.sj_serve_request()
        tk = C.c_int64()
        tickets = []
        t0 = lib.sj_server_now(self.handle) + 2e-3    # leaves time to queue the early arrivals
        for r in order:
            req.kind = L.SJ_SERVE_PIP if r.kind == PIP else L.SJ_SERVE_P2P
            req.pts = r.pts.data_ptr()
            req.n = r.n
            req.out_id = r.out_id.data_ptr()
            req.out_d = r.out_d.data_ptr() if r.out_d is not None else None
            req.not_before = t0 + r.arrival
            req.use_window = 0 if r.window is None else 1
            req.window = 0.0 if r.window is None else r.window
            L.check(lib.sj_server_submit(self.handle, C.byref(req), C.byref(tk)), "sj_server_submit")
            tickets.append(tk.value)
        late = max(lib.sj_server_now(self.handle) - t0 - order[-1].arrival, 0.0)   # submission behind schedule
        lat = C.c_double()
        for r, t in zip(order, tickets):
            L.check(lib.sj_server_wait(self.handle, t, C.byref(lat)), "sj_server_wait")
            r.t_done = r.arrival + lat.value       # seconds from t0
        wall = max(r.t_done for r in order)
        lat_all = np.array([r.latency for r in order])
        pts = sum(r.n for r in order)
        return {"mode": mode, "form": form or self.form, "requests": len(order),
                "rounds": self.stats()["rounds"] - st0["rounds"], "points": pts, "wall_s": wall,
                "max_launch_ms": self.stats()["max_launch_s"] * 1e3,
                "max_round_ms": self.stats()["max_round_s"] * 1e3,
                "points_per_s": pts / wall, "p50_ms": float(np.percentile(lat_all, 50) * 1e3),
                "p99_ms": float(np.percentile(lat_all, 99) * 1e3), "mean_ms": float(lat_all.mean() * 1e3),
                "submit_behind_ms": float(late * 1e3)}
