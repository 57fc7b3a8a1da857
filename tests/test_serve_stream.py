"""Host logic of the serving stream generator (no GPU): arrival order, request
sizes and pool offsets, and per-request P2P windows."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_stream_offsets_sizes_and_windows():
    from paper_1403_0802_gb300 import serve
    pool_p = torch.arange(2 * 50_000, dtype=torch.float64).reshape(-1, 2)
    pool_l = -torch.arange(2 * 40_000, dtype=torch.float64).reshape(-1, 2)
    reqs = serve.make_stream(400, 1000.0, pool_p, pool_l, size_min=10, size_max=30_000, seed=3,
                             p2p_windows=(0.0, 25.0, 100.0))
    arr = [r.arrival for r in reqs]
    assert arr == sorted(arr) and arr[0] > 0
    kinds = np.array([r.kind for r in reqs])
    assert 0.55 < (kinds == serve.PIP).mean() < 0.85
    for r in reqs:
        pool = pool_p if r.kind == serve.PIP else pool_l
        assert 10 <= r.n <= 30_000
        assert torch.equal(r.pts, pool[r.off:r.off + r.n])          # offsets locate the slice
        if r.kind == serve.PIP:
            assert r.window is None
        else:
            assert r.window in (0.0, 25.0, 100.0)
    assert len({r.window for r in reqs if r.kind == serve.P2P}) == 3
    # no windows asked: none drawn; all at t = 0 when the rate is 0
    plain = serve.make_stream(50, 0.0, pool_p, pool_l, seed=4)
    assert all(r.window is None for r in plain) and all(r.arrival == 0.0 for r in plain)
