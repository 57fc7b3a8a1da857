"""Batched rounds (sj_engine_*): every request's result inside a round equals
its result when joined alone, round after round (graph replay), for PIP and
P2P requests mixed in one round, empty requests included.  P2P results are
also checked against the oracle at each request's window (the bar of
tests/parity.py); FP32X ids must equal those of the join alone wherever the
oracle's answer is unique."""
import numpy as np
import pytest

from paper_1403_0802_gb300 import synth
from parity import P2PRef, PIPRef

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup(oracle):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_0802_gb300 import api, build
    build.build()
    wp = synth.pip_tiles(n_points=400_000, layer=1)
    wl = synth.p2p_walks(n_points=400_000, n_lines=30_000)
    pip = api.pip_layer(wp.polygons.verts, wp.polygons.ring_off, wp.polygons.poly_ring_off, wp.grid)
    p2p = api.p2p_layer(wl.polylines.verts, wl.polylines.line_off, wl.D, wl.grid)
    p2p.ref = P2PRef(oracle, wl.grid, wl.polylines.verts, wl.polylines.line_off, wl.D)
    pip.ref = PIPRef(oracle, wp.grid, wp.polygons.verts, wp.polygons.ring_off, wp.polygons.poly_ring_off)
    yield api, pip, p2p, torch.as_tensor(wp.points, device="cuda"), torch.as_tensor(wl.points, device="cuda")
    pip.close()
    p2p.close()


def check_p2p_round(layer, pts, a_id, a_d, b_id, b_d, form, window=None):
    """A request's round result (a) against the oracle and against its join
    alone (b): FP64 bit for bit; FP32X ids equal wherever the oracle's answer
    is unique (a point's FP32 certificate depends on the other points of its
    work item, and an uncertified point is redone in FP64)."""
    p = pts.cpu().numpy()
    ref = layer.ref.join(p, window)
    layer.ref.check(p, a_id, a_d, form, window=window, ref=ref)
    if form == "fp64":
        np.testing.assert_array_equal(a_id, b_id)
        np.testing.assert_array_equal(a_d, b_d)
    else:
        u = layer.ref.unique(p, window, ref=ref)
        np.testing.assert_array_equal(a_id[u], b_id[u])


def make_requests(rng, pip, p2p, ptsP, ptsL, n):
    reqs = []
    for _ in range(n):
        kind = rng.random() < 0.7
        pool = ptsP if kind else ptsL
        size = int(rng.choice([0, 1, 7, 1000, 20_000, 60_000]))
        off = int(rng.integers(0, pool.shape[0] - size)) if size else 0
        pts = pool[off:off + size].contiguous()
        out_id = torch.full((size,), 99, dtype=torch.int32, device="cuda")
        out_d = None if kind else torch.full((size,), -5.0, dtype=torch.float64, device="cuda")
        reqs.append((pip if kind else p2p, pts, out_id, out_d))
    return reqs


@pytest.mark.parametrize("form", ["fp64", "fp32x"])
@pytest.mark.parametrize("graph", [True, False])
def test_rounds_match_single_joins(setup, form, graph):
    api, pip, p2p, ptsP, ptsL = setup
    rng = np.random.default_rng(3)
    stream = torch.cuda.Stream()
    with api.Engine(max_points=600_000, max_requests=64, form=form, graph=graph) as eng:
        for rnd in range(4):
            reqs = make_requests(rng, pip, p2p, ptsP, ptsL, int(rng.integers(1, 12)))
            stream.wait_stream(torch.cuda.current_stream())     # inputs / outputs were made there
            with torch.cuda.stream(stream):
                eng.round(reqs, stream)
            stream.synchronize()
            for layer, pts, out_id, out_d in reqs:
                if layer is pip:
                    ref = api.pip_join(layer, pts, form=form) if pts.shape[0] else out_id
                    torch.cuda.synchronize()
                    assert torch.equal(out_id, ref), (rnd, pts.shape)
                    if pts.shape[0]:
                        np.testing.assert_array_equal(out_id.cpu().numpy(), pip.ref.join(pts.cpu().numpy()))
                else:
                    if pts.shape[0] == 0:
                        continue
                    rid, rd = api.p2p_join(layer, pts, form=form)
                    torch.cuda.synchronize()
                    a_id, a_d, b_id, b_d = (t.cpu().numpy() for t in (out_id, out_d, rid, rd))
                    check_p2p_round(layer, pts, a_id, a_d, b_id, b_d, form)


@pytest.mark.parametrize("form", ["fp64", "fp32x"])
def test_rounds_with_per_request_windows(setup, form):
    """P2P requests of one round ask for different windows (none, 0, 20 m,
    60 m, the layer's D): each equals sj_p2p_join_window at its window alone.
    Rounds alternate between windowed and unwindowed, so one captured graph
    serves both."""
    api, pip, p2p, ptsP, ptsL = setup
    D = p2p.D
    rng = np.random.default_rng(8)
    stream = torch.cuda.Stream()
    wins = [None, 0.0, 20.0, 60.0, D]
    with api.Engine(max_points=600_000, max_requests=64, form=form) as eng:
        for rnd in range(4):
            reqs = []
            for k in range(8):
                size = int(rng.choice([1, 999, 30_000]))
                off = int(rng.integers(0, ptsL.shape[0] - size))
                win = wins[(k + rnd) % len(wins)] if rnd % 2 == 0 else None
                reqs.append((p2p, ptsL[off:off + size].contiguous(),
                             torch.full((size,), 99, dtype=torch.int32, device="cuda"),
                             torch.full((size,), -5.0, dtype=torch.float64, device="cuda"), win))
            stream.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(stream):
                eng.round(reqs, stream)
            stream.synchronize()
            for layer, pts, out_id, out_d, win in reqs:
                rid, rd = api.p2p_join(layer, pts, form=form, window=win)
                torch.cuda.synchronize()
                a_id, a_d, b_id, b_d = (t.cpu().numpy() for t in (out_id, out_d, rid, rd))
                check_p2p_round(layer, pts, a_id, a_d, b_id, b_d, form, window=win)
                if win is not None:
                    assert np.all(a_d[a_id >= 0] <= win)


def test_round_limits(setup):
    api, pip, p2p, ptsP, ptsL = setup
    from paper_1403_0802_gb300._lib import SJError, SJ_ERR_INVALID
    with api.Engine(max_points=1000, max_requests=2) as eng:
        big = ptsP[:1001].contiguous()
        with pytest.raises(SJError) as e:
            eng.round([(pip, big, torch.empty(1001, dtype=torch.int32, device="cuda"), None)])
        assert e.value.status == SJ_ERR_INVALID
        small = ptsP[:10].contiguous()
        outs = [torch.empty(10, dtype=torch.int32, device="cuda") for _ in range(3)]
        with pytest.raises(SJError):
            eng.round([(pip, small, o, None) for o in outs])         # 3 requests > max_requests
        ls = ptsL[:10].contiguous()
        oi, od = outs[0], torch.empty(10, dtype=torch.float64, device="cuda")
        for bad in ((pip, small, oi, None, 5.0), (p2p, ls, oi, od, -1.0), (p2p, ls, oi, od, 1e9)):
            with pytest.raises(SJError) as e:
                eng.round([bad])                                    # windows: P2P only, within [0, D]
            assert e.value.status == SJ_ERR_INVALID


def test_rounds_on_the_multi_ring_layer(setup):
    """PIP rounds against the multi-ring layer (tiles with island holes and the
    islands) equal direct joins bit for bit in both forms, island points included."""
    api = setup[0]
    w = synth.pip_tiles(n_points=300_000, layer=3)
    P = w.polygons
    pts_all = torch.as_tensor(w.points, device="cuda")
    stream = torch.cuda.Stream()
    with api.pip_layer(P.verts, P.ring_off, P.poly_ring_off, w.grid) as layer:
        for form in ("fp64", "fp32x"):
            with api.Engine(max_points=300_000, max_requests=16, form=form) as eng:
                cuts = [0, 1, 1000, 50_000, 120_000, 300_000]
                reqs = [(layer, pts_all[a:b].contiguous(), torch.full((b - a,), 99, dtype=torch.int32, device="cuda"),
                         None) for a, b in zip(cuts[:-1], cuts[1:])]
                stream.wait_stream(torch.cuda.current_stream())
                with torch.cuda.stream(stream):
                    eng.round(reqs, stream)
                stream.synchronize()
                got = torch.cat([r[2] for r in reqs])
                ref = api.pip_join(layer, pts_all, form=form)
                torch.cuda.synchronize()
                assert torch.equal(got, ref), form
                assert int((ref >= 40_000).sum()) > 0           # some points answer an island
