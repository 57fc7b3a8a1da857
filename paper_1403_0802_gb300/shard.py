"""Point sharding across GPUs with replicated layers.

A point's result depends only on the point and the layer (Sec. III: the
join is data-parallel over points), so a large request splits into
contiguous point ranges, one per GPU, each joined against that GPU's replica
of the layer, and the results concatenate back in input order.  No exchange
of data is needed during the join; only the outputs are gathered.

Two forms:
  * MultiDeviceJoin -- one process, every visible device: a layer replica
    per device and one host thread per device running the host-buffer join
    (sj_pip_join_host / sj_p2p_join_host) on its slice of the caller's
    arrays, so the slices are joined concurrently and written in place.
  * join_distributed -- one process per GPU (torch.distributed, any
    backend): each rank joins its shard with its own join function and the
    shards are all-gathered into the full result, in input order, on every
    rank.

shard_bounds() is the partition both use.
"""
from __future__ import annotations

import threading

import numpy as np

from . import api


def shard_bounds(n: int, parts: int) -> list[tuple[int, int]]:
    """Contiguous ranges [lo, hi) covering 0..n, sizes differing by at most 1."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    q, r = divmod(int(n), parts)
    out, lo = [], 0
    for k in range(parts):
        hi = lo + q + (1 if k < r else 0)
        out.append((lo, hi))
        lo = hi
    return out


class MultiDeviceJoin:
    """A layer replicated on several devices (default: every visible one) and
    joins of host point arrays split across them.

        mj = MultiDeviceJoin.p2p(verts, line_off, D, grid)
        ids, d = mj.join(points, form="fp32x")
    """

    def __init__(self, kind: str, make_layer, devices=None):
        import torch
        self.kind = kind
        self.devices = list(range(torch.cuda.device_count())) if devices is None else list(devices)
        if not self.devices:
            raise RuntimeError("no CUDA device")
        self.layers = {}
        for dev in self.devices:
            with torch.cuda.device(dev):
                self.layers[dev] = make_layer()

    @classmethod
    def pip(cls, verts, ring_off, poly_ring_off, grid, devices=None):
        return cls("pip", lambda: api.pip_layer(verts, ring_off, poly_ring_off, grid), devices)

    @classmethod
    def p2p(cls, verts, line_off, D, grid, devices=None):
        return cls("p2p", lambda: api.p2p_layer(verts, line_off, D, grid), devices)

    def join(self, pts, form: str = "fp64", **kw):
        """Results of every point, in input order: PIP ids, or P2P (ids,
        distances).  pts: host float64 [N, 2] (numpy or pinned torch)."""
        import torch
        n = pts.shape[0]
        ids = np.empty(n, np.int32)
        dist = np.empty(n, np.float64) if self.kind == "p2p" else None
        errors = []

        def run(dev, lo, hi):
            try:
                with torch.cuda.device(dev):
                    sl = pts[lo:hi]
                    if self.kind == "pip":
                        api.pip_join_host(self.layers[dev], sl, ids[lo:hi], form=form, **kw)
                    else:
                        api.p2p_join_host(self.layers[dev], sl, ids[lo:hi], dist[lo:hi], form=form, **kw)
            except Exception as e:     # re-raised in the caller's thread
                errors.append(e)

        threads = [threading.Thread(target=run, args=(dev, lo, hi))
                   for dev, (lo, hi) in zip(self.devices, shard_bounds(n, len(self.devices))) if hi > lo]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        if errors:
            raise errors[0]
        return ids if self.kind == "pip" else (ids, dist)

    def close(self):
        for layer in self.layers.values():
            layer.close()
        self.layers = {}

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def join_distributed(join_fn, pts, group=None):
    """One process per GPU: rank r joins shard r of pts with join_fn (returns
    an array, or a tuple of arrays, one entry per point) and every rank
    receives the full results in input order (all_gather of the shards,
    padded to the largest shard).  pts is the whole point array on every rank
    (the partition is shard_bounds(N, world_size))."""
    import torch
    import torch.distributed as dist
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    bounds = shard_bounds(pts.shape[0], world)
    lo, hi = bounds[rank]
    local = join_fn(pts[lo:hi])
    parts = local if isinstance(local, tuple) else (local,)
    width = max(h - l for l, h in bounds)
    full = []
    for arr in parts:
        arr = np.asarray(arr)
        pad = np.zeros(width, arr.dtype)
        pad[:len(arr)] = arr
        mine = torch.from_numpy(pad)
        got = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(got, mine, group=group)
        full.append(np.concatenate([g.numpy()[:h - l] for g, (l, h) in zip(got, bounds)]))
    return tuple(full) if isinstance(local, tuple) else full[0]
