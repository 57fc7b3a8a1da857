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
