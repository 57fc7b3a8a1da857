"""Continuous-batching serving loop over resident layers.

Requests (a batch of GPS points and a kind: PIP against the resident polygon
layer or P2P against the resident polyline layer) arrive over time.  The loop

  * admits queued requests, in arrival order, while their device memory
    (points, ids, distances) fits in a fixed device arena -- the HBM budget --
    and copies each admitted request's points to the GPU on a copy stream;
  * whenever fewer than two rounds are in flight, forms a round from every
    admitted request whose points have arrived (up to round_points points)
    and submits it to the batched engine (one graph replay per layer, however
    many requests), so requests that arrive while a round runs join the next;
  * copies each round's results back on a second copy stream and records each
    request's latency = (results in host memory) - (arrival).

mode="per_request" runs the same loop with one join call (its own kernel
launches) per request in arrival order -- the baseline the batched form is
measured against.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

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
    _dev: tuple | None = field(default=None, repr=False)   # (block, pts, id, d) views into the arena

    @property
    def n(self) -> int:
        return int(self.pts.shape[0])

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


def make_stream(n_requests: int, rate_per_s: float, pool_pip: torch.Tensor, pool_p2p: torch.Tensor,
                size_min: int = 1_000, size_max: int = 5_000_000, pip_frac: float = 0.7,
                seed: int = 20140309) -> list[Request]:
    """Poisson arrivals (all at t = 0 when rate_per_s is 0); sizes log-uniform in
    [size_min, size_max]; points are slices of pinned host pools of clustered
    points (one pool per kind)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, n_requests)) if rate_per_s > 0 else np.zeros(n_requests)
    reqs = []
    for k in range(n_requests):
        kind = PIP if rng.random() < pip_frac else P2P
        pool = pool_pip if kind == PIP else pool_p2p
        n = int(round(math.exp(rng.uniform(math.log(size_min), math.log(size_max)))))
        n = min(n, pool.shape[0])
        off = int(rng.integers(0, pool.shape[0] - n + 1))
        reqs.append(Request(k, float(t[k]), kind, pool[off:off + n]))
    return reqs


class Arena:
    """Ring allocator over one device buffer.  Blocks are handed out in order;
    a freed block is reclaimed once every older block is free as well."""
    ALIGN = 256

    def __init__(self, nbytes: int):
        self.cap = int(nbytes) // self.ALIGN * self.ALIGN
        self.buf = torch.empty(self.cap, dtype=torch.uint8, device="cuda")
        self.live = deque()       # [start, size, freed] in allocation order
        self.head = 0

    def alloc(self, size: int):
        size = -(-size // self.ALIGN) * self.ALIGN
        if size > self.cap:
            return None
        if not self.live:
            self.head = 0
            start = 0
        else:
            tail = self.live[0][0]
            if self.head >= tail:                       # free space: [head, cap) and [0, tail)
                if self.cap - self.head >= size:
                    start = self.head
                elif tail >= size:
                    start = 0
                else:
                    return None
            else:                                       # free space: [head, tail)
                if tail - self.head >= size:
                    start = self.head
                else:
                    return None
        blk = [start, size, False]
        self.live.append(blk)
        self.head = start + size
        return blk

    def free(self, blk):
        blk[2] = True
        while self.live and self.live[0][2]:
            self.live.popleft()

    def view(self, blk, offset: int, dtype, shape):
        nbytes = int(np.prod(shape)) * torch.tensor([], dtype=dtype).element_size()
        return self.buf[blk[0] + offset: blk[0] + offset + nbytes].view(dtype).view(shape)


class Server:
    """Resident layers, the batched engine, the device arena and the streams."""

    def __init__(self, pip_layer: api.Layer, p2p_layer: api.Layer, form: str = "fp32x",
                 round_points: int = 16_000_000, max_requests: int = 1024, hbm_budget: int | None = None):
        self.layers = {PIP: pip_layer, P2P: p2p_layer}
        self.form = form
        self.round_points = int(round_points)
        self.engine = api.Engine(max_points=round_points, max_requests=max_requests, form=form)
        self.copy_in = torch.cuda.Stream()
        self.compute = torch.cuda.Stream()
        self.copy_out = torch.cuda.Stream()
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info()
            hbm_budget = int(0.25 * free)
        self.arena = Arena(hbm_budget)

    @staticmethod
    def request_bytes(r: Request) -> int:
        n = r.n
        return 16 * n + 256 + 4 * n + 256 + (8 * n if r.kind == P2P else 0)

    def close(self):
        self.engine.close()

    def _place(self, r: Request):
        blk = self.arena.alloc(self.request_bytes(r))
        if blk is None:
            return False
        n = r.n
        o_id = -(-16 * n // 256) * 256
        o_d = o_id + -(-4 * n // 256) * 256
        pts = self.arena.view(blk, 0, torch.float64, (n, 2))
        ids = self.arena.view(blk, o_id, torch.int32, (n,))
        d = self.arena.view(blk, o_d, torch.float64, (n,)) if r.kind == P2P else None
        r._dev = (blk, pts, ids, d)
        return True

    # ------------------------------------------------------------------ the loop
    def run(self, requests: list[Request], mode: str = "batched", max_rounds_in_flight: int = 2) -> dict:
        assert mode in ("batched", "per_request")
        pending = sorted(requests, key=lambda r: r.arrival)
        for r in pending:
            r.out_id = torch.empty(r.n, dtype=torch.int32, pin_memory=True)
            r.out_d = torch.empty(r.n, dtype=torch.float64, pin_memory=True) if r.kind == P2P else None
            r.t_done = math.nan
        queue: deque[Request] = deque()
        copying: deque[tuple[torch.cuda.Event, list[Request]]] = deque()   # admitted, copy in flight
        ready: deque[Request] = deque()                                      # on the device
        rounds: deque[tuple[torch.cuda.Event, list[Request]]] = deque()
        done = n_rounds = i = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while done < len(requests):
            t = time.perf_counter() - t0
            while i < len(pending) and pending[i].arrival <= t:
                queue.append(pending[i])
                i += 1
            # admission: arrival order, while the request fits in the arena
            batch = []
            while queue and self._place(queue[0]):
                batch.append(queue.popleft())
            if batch:
                with torch.cuda.stream(self.copy_in):
                    for r in batch:
                        r._dev[1].copy_(r.pts, non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(self.copy_in)
                copying.append((ev, batch))
            while copying and copying[0][0].query():
                ready.extend(copying.popleft()[1])
            # rounds
            if len(rounds) < max_rounds_in_flight and ready:
                rnd, tot = [], 0
                while ready and (not rnd or (mode == "batched" and tot + ready[0].n <= self.round_points)):
                    r = ready.popleft()
                    rnd.append(r)
                    tot += r.n
                self._submit(rnd, mode)
                ev = torch.cuda.Event()
                ev.record(self.copy_out)
                rounds.append((ev, rnd))
                n_rounds += 1
            # completions, in order
            while rounds and rounds[0][0].query():
                t_done = time.perf_counter() - t0
                for r in rounds.popleft()[1]:
                    r.t_done = t_done
                    self.arena.free(r._dev[0])
                    r._dev = None
                    done += 1
        wall = time.perf_counter() - t0
        lat = np.array([r.latency for r in requests])
        pts = sum(r.n for r in requests)
        return {"mode": mode, "requests": len(requests), "rounds": n_rounds, "points": pts, "wall_s": wall,
                "points_per_s": pts / wall, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3)}

    def _submit(self, rnd: list[Request], mode: str):
        comp = self.compute
        with torch.cuda.stream(comp):
            if mode == "batched":
                self.engine.round([(self.layers[r.kind], r._dev[1], r._dev[2], r._dev[3]) for r in rnd], comp)
            else:
                for r in rnd:
                    if r.kind == PIP:
                        api.pip_join(self.layers[PIP], r._dev[1], r._dev[2], form=self.form, stream=comp)
                    else:
                        api.p2p_join(self.layers[P2P], r._dev[1], r._dev[2], r._dev[3], form=self.form, stream=comp)
        out = self.copy_out
        out.wait_stream(comp)
        with torch.cuda.stream(out):
            for r in rnd:
                r.out_id.copy_(r._dev[2], non_blocking=True)
                if r.out_d is not None:
                    r.out_d.copy_(r._dev[3], non_blocking=True)
