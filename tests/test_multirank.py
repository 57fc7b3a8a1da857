"""The N > 1 host path of bench.py on CPU with two gloo ranks: every rank gets
its own shard of points (weak scaling, no data-path collective) and the timed
region is reduced with the slowest rank's time."""
import os
import socket
import sys
import types

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, _ = bench.dist_env()
    slowest = bench.max_over_ranks(10.0 * (rank + 1), w, device="cpu")
    args = types.SimpleNamespace(workload="p2p", points=2000, layer=1, D=100.0)
    wl = bench.workload(args, r)
    bench.barrier(w)
    q.put((rank, w, slowest, wl.points[:3].tolist(), wl.polylines.line_off[-1]))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_points_and_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, s0, p0, v0), (r1, w1, s1, p1, v1) = out
    assert (w0, w1) == (2, 2)
    assert s0 == s1 == 20.0                 # max over ranks
    assert p0 != p1                         # each rank joins its own points
    assert v0 == v1                         # against a replica of the same layer


def test_shard_bounds_partition():
    from paper_1403_0802_gb300.shard import shard_bounds
    for n, k in ((0, 1), (10, 3), (7, 8), (1_000_003, 4)):
        b = shard_bounds(n, k)
        assert len(b) == k and b[0][0] == 0 and b[-1][1] == n
        assert all(b[i][1] == b[i + 1][0] for i in range(k - 1))
        sizes = [h - l for l, h in b]
        assert max(sizes) - min(sizes) <= 1


def _join_worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np
    from oracle import oracle as O
    from paper_1403_0802_gb300 import synth
    from paper_1403_0802_gb300.shard import join_distributed
    w = synth.p2p_walks(n_points=30_011, n_lines=3_000)
    L = w.polylines
    # each rank joins its shard (here with the CPU oracle standing in for the
    # GPU join of that rank), the shards are gathered in input order
    fn = lambda p: O.p2p_join(w.grid, p, L.verts, L.line_off, w.D)[:2]
    ids, d = join_distributed(fn, w.points)
    wp = synth.pip_stars(n_points=20_007, n_side=8)
    P = wp.polygons
    pid = join_distributed(lambda p: O.pip_join(wp.grid, p, P.verts, P.ring_off, P.poly_ring_off), wp.points)
    if rank == 0:
        rid, rd = O.p2p_join(w.grid, w.points, L.verts, L.line_off, w.D)[:2]
        ref_pip = O.pip_join(wp.grid, wp.points, P.verts, P.ring_off, P.poly_ring_off)
        q.put((bool(np.array_equal(ids, rid)), bool(np.array_equal(d, rd)), bool(np.array_equal(pid, ref_pip))))
    else:
        q.put(None)
    dist.destroy_process_group()


def test_two_gloo_ranks_join_shards_equal_one_rank_join():
    """The multi-GPU path's partition and gather: two ranks each join a
    contiguous shard of one request's points and all-gather the results; the
    gathered results equal a one-rank join of all points, P2P and PIP."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_join_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res = [o for o in out if o is not None]
    assert res == [(True, True, True)]
