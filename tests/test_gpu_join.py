"""GPU parity of the CUDA path (through the C ABI) against the CPU oracle.

PIP ids and the filter's candidate lists must match the oracle bit for bit in
both arithmetic forms.  P2P ids must match except where the oracle's best and
second-best distances tie within 1e-9 (relative) or the best distance sits
within 1e-9 of D; FP64 distances must agree to 1e-12 * max(d, 1 m); FP32X
distances must stay inside the per-point bound the kernel certifies
(64 * 2^-24 * the largest cell-relative coordinate involved, plus 1e-9 m).
"""
import math

import numpy as np
import pytest

from paper_1403_0802_gb300 import synth
from parity import P2PRef

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FORMS = ("fp64", "fp32x")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_0802_gb300 import api as A
    from paper_1403_0802_gb300 import build
    build.build()
    return A


# ------------------------------------------------------------------ helpers

def pip_ref(oracle, w):
    P = w.polygons
    return oracle.pip_join(w.grid, w.points, P.verts, P.ring_off, P.poly_ring_off)


def check_p2p(oracle, w, gid, gd, form, verts=None, line_off=None, D_layer=None):
    """The P2P bar of tests/parity.py for workload w (its grid, points and
    window w.D) on a layer built for D_layer (default w.D)."""
    L = w.polylines if verts is None else None
    verts = L.verts if verts is None else verts
    line_off = L.line_off if line_off is None else line_off
    ref = P2PRef(oracle, w.grid, verts, line_off, w.D if D_layer is None else D_layer)
    return ref.check(w.points, gid, gd, form, window=w.D)


def to_np(t):
    return t.cpu().numpy()


# ------------------------------------------------------------------ filter

def test_candidate_lists_match_oracle(api, oracle):
    w = synth.pip_stars(n_points=10)
    P = w.polygons
    with api.pip_layer(P.verts, P.ring_off, P.poly_ring_off, w.grid) as layer:
        gs, gi = layer.candidates()
        info = layer.info()
    mbb = oracle.pip_mbb(w.grid, P.verts, P.ring_off, P.poly_ring_off)
    rs, ri = oracle.cand_csr(w.grid, mbb)
    np.testing.assert_array_equal(gs, rs)
    np.testing.assert_array_equal(gi, ri)
    assert info["n_candidates"] == len(ri) and info["n_objects"] == P.n_polygons

    w = synth.p2p_walks(n_points=10, n_lines=30_000)
    Lw = w.polylines
    with api.p2p_layer(Lw.verts, Lw.line_off, w.D, w.grid) as layer:
        gs, gi = layer.candidates()
    mbb = oracle.p2p_mbb(w.grid, Lw.verts, Lw.line_off)
    rs, ri = oracle.cand_csr(w.grid, mbb, w.D, expand=True)
    np.testing.assert_array_equal(gs, rs)
    np.testing.assert_array_equal(gi, ri)


def test_bucketing_matches_oracle_counts(api, oracle):
    rng = np.random.default_rng(5)
    g = synth.grid(512)
    pts = synth.points_mixture(300_001, rng)
    pts[:50] = [-1.0, 5.0]                 # outside the grid
    pts[50:60] = np.nan
    pts[60:70] = [1e5, 1.0]                # on the open edge
    cs, perm = api.bucket_points(pts, g)
    cs, perm = to_np(cs), to_np(perm)
    counts = oracle.cell_counts(g, pts)
    np.testing.assert_array_equal(cs, np.concatenate([[0], np.cumsum(counts[:-1])]))
    n_in = cs[-1]
    sorted_idx = perm[:n_in]
    assert len(np.unique(sorted_idx)) == n_in
    cells = oracle.point_cells(g, pts)
    slot_cell = np.repeat(np.arange(len(cs) - 1), np.diff(cs))
    np.testing.assert_array_equal(cells[sorted_idx], slot_cell)


# ------------------------------------------------------------------ PIP

@pytest.mark.parametrize("form", FORMS)
def test_pip_stars_full_size(api, oracle, form):
    """1,000,000 uniform points, 1,024 star polygons, grid 256 x 256."""
    w = synth.pip_stars()
    ref = pip_ref(oracle, w)
    P = w.polygons
    with api.pip_layer(P.verts, P.ring_off, P.poly_ring_off, w.grid) as layer:
        pts = torch.as_tensor(w.points, device="cuda")
        got = to_np(api.pip_join(layer, pts, form=form))
        st = layer.stats()
    np.testing.assert_array_equal(got, ref)
    assert st["hits"] == (ref >= 0).sum()
    assert 0 < st["resolved"] < len(ref)           # classified cells answered without refinement


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("ppi", [1, 7, 32, 128])
def test_pip_ragged_items_and_dense_cells(api, oracle, form, ppi):
    """Few cells holding hundreds of points (several items per cell, ragged
    tails) and polygons larger than one staging chunk (5,000 vertices)."""
    rng = np.random.default_rng(ppi)
    verts, sizes = [], []
    for k, n in enumerate([5000, 300, 3]):
        ang = np.sort(rng.uniform(0, 2 * np.pi, n))
        r = rng.uniform(200, 450, n)
        cx, cy = 500 + 1000 * k, 500
        verts.append(np.stack([cx + r * np.cos(ang), cy + r * np.sin(ang)], 1))
        sizes.append(n)
    verts = np.concatenate(verts)
    ring_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pro = np.arange(len(sizes) + 1, dtype=np.int64)
    g = dict(x0=0.0, y0=0.0, x1=4000.0, y1=1000.0, nx=8, ny=2)
    pts = np.concatenate([rng.uniform([0, 0], [4000, 1000], (20000, 2)), rng.normal(500, 30, (3001, 2))])
    ref = oracle.pip_join(g, pts, verts, ring_off, pro)
    with api.pip_layer(verts, ring_off, pro, g) as layer:
        got = to_np(api.pip_join(layer, pts, form=form, pts_per_item=ppi))
    np.testing.assert_array_equal(got, ref)


def layer_from_rings(polys):
    verts, ring_off, pro = [], [0], [0]
    for rings in polys:
        for ring in rings:
            verts.extend(ring)
            ring_off.append(len(verts))
        pro.append(len(ring_off) - 1)
    return np.asarray(verts, np.float64).reshape(-1, 2), np.asarray(ring_off, np.int64), np.asarray(pro, np.int64)


@pytest.mark.parametrize("form", FORMS)
def test_pip_degenerate_integer_tiling(api, oracle, form):
    """Triangles with integer corners tiling a square, queried on a half-unit
    lattice: thousands of points on edges and vertices, FP32 y ties and zero
    orientations -- the FP32X form must take its FP64 fallback and agree."""
    from tests.test_oracle_pip import jittered_triangulation, dyadic_lattice
    rng = np.random.default_rng(21)
    polys = jittered_triangulation(rng, 10, 4, jitter=1)
    verts, ro, pro = layer_from_rings(polys)
    g = dict(x0=-8.0, y0=-8.0, x1=48.0, y1=48.0, nx=7, ny=7)
    pts = dyadic_lattice(-2.0, 42.0, 0.5)
    ref, nh = oracle.pip_join(g, pts, verts, ro, pro, with_hits=True)
    with api.pip_layer(verts, ro, pro, g) as layer:
        got = to_np(api.pip_join(layer, pts, form=form))
        st = layer.stats()
    np.testing.assert_array_equal(got, ref)
    if form == "fp32x":
        assert st["fallbacks"] > 0


@pytest.mark.parametrize("form", FORMS)
def test_pip_long_near_lists_window_search(api, oracle, form):
    """A polygon whose right side is a 2,048-vertex zigzag inside one grid
    column: every cell of that column has a near list of ~256 edges (longer
    than the refinement stages), searched per point in its sorted window.
    Points on the zigzag's vertices and edge midpoints, at the vertices' exact
    y values (FP32 ties) and uniform points: ids bit-identical to the oracle,
    with far fewer tests than points x list length."""
    n, W, A, H = 2048, 32.0, 7.0, 64.0
    ys = np.arange(n + 1) * (H / n)                          # dyadic steps of 1/32
    xs = W + A * (np.arange(n + 1) % 2)
    ring = np.concatenate([[[0.0, 0.0]], np.stack([xs, ys], 1), [[0.0, H]]])
    verts = np.ascontiguousarray(ring, np.float64)
    ring_off = np.array([0, len(verts)], np.int64)
    poly_off = np.array([0, 1], np.int64)
    g = dict(x0=0.0, y0=0.0, x1=128.0, y1=128.0, nx=16, ny=16)
    rng = np.random.default_rng(11)
    mids = 0.5 * (verts[1:n + 1] + verts[2:n + 2])
    tie = np.stack([rng.uniform(W, W + A, n + 1), ys], 1)
    pts = np.concatenate([rng.uniform(0, 128, (60_000, 2)), verts, mids, tie,
                          np.stack([np.full(n + 1, W + 0.5 * A), ys], 1)])
    ref = oracle.pip_join(g, pts, verts, ring_off, poly_off)
    assert 0 < (ref == 0).sum() < len(pts)
    with api.pip_layer(verts, ring_off, poly_off, g) as layer:
        got = to_np(api.pip_join(layer, pts, form=form))
        st = layer.stats()
    np.testing.assert_array_equal(got, ref)
    assert st["edge_tests"] < 0.1 * (st["points"] - st["resolved"]) * 256


@pytest.mark.parametrize("form", FORMS)
def test_pip_holes_overlaps_and_translation(api, oracle, form):
    sq = [[(0, 0), (4, 0), (4, 4), (0, 4)], [(1, 1), (1, 3), (3, 3), (3, 1)]]     # square with a hole
    comb = [[(0, 0), (7, 0), (7, 4), (6, 4), (6, 1), (4, 1), (4, 4), (3, 4), (3, 1), (1, 1), (1, 4), (0, 4)]]
    big = [[(-1, -1), (9, -1), (9, 9), (-1, 9)]]
    base_polys = [sq, comb, big]
    pts0 = np.stack(np.meshgrid(np.arange(-2, 10, 0.25), np.arange(-2, 10, 0.25)), -1).reshape(-1, 2)
    for shift in (0.0, 65536.0, 3 * 65536.0):
        verts, ro, pro = layer_from_rings(base_polys)
        verts = verts + shift
        pts = pts0 + shift
        g = dict(x0=shift - 16, y0=shift - 16, x1=shift + 16, y1=shift + 16, nx=8, ny=8)
        ref = oracle.pip_join(g, pts, verts, ro, pro)
        with api.pip_layer(verts, ro, pro, g) as layer:
            got = to_np(api.pip_join(layer, pts, form=form))
        np.testing.assert_array_equal(got, ref)


def test_pip_empty_and_outside(api, oracle):
    w = synth.pip_stars(n_points=1000, n_side=4)
    P = w.polygons
    with api.pip_layer(P.verts, P.ring_off, P.poly_ring_off, w.grid) as layer:
        out = api.pip_join(layer, np.zeros((0, 2)))
        assert out.numel() == 0
        pts = np.array([[-1.0, 5.0], [np.nan, 1.0], [1e5, 1e5], [2e5, 0.0]])
        np.testing.assert_array_equal(to_np(api.pip_join(layer, pts)), -1)
    # a layer without polygons
    with api.pip_layer(np.zeros((0, 2)), np.zeros(1, np.int64), np.zeros(1, np.int64), w.grid) as layer:
        np.testing.assert_array_equal(to_np(api.pip_join(layer, w.points)), -1)


@pytest.mark.parametrize("form", FORMS)
def test_p2p_empty_and_outside(api, oracle, form):
    """No points; points outside the grid or NaN; a layer without polylines;
    a window of 0 on points off every polyline."""
    w = synth.p2p_walks(n_points=2000, n_lines=50)
    Lw = w.polylines
    with api.p2p_layer(Lw.verts, Lw.line_off, w.D, w.grid) as layer:
        gid, gd = api.p2p_join(layer, np.zeros((0, 2)), form=form)
        assert gid.numel() == 0 and gd.numel() == 0
        pts = np.array([[-1.0, 5.0], [np.nan, 1.0], [1e5, 1e5], [2e5, 0.0]])
        gid, gd = api.p2p_join(layer, pts, form=form)
        np.testing.assert_array_equal(to_np(gid), -1)
        assert np.isinf(to_np(gd)).all()
        gid, gd = api.p2p_join(layer, w.points, form=form, window=0.0)
        rid, rd, _, _ = oracle.p2p_join(w.grid, w.points, Lw.verts, Lw.line_off, 0.0)
        np.testing.assert_array_equal(to_np(gid), rid)
    with api.p2p_layer(np.zeros((0, 2)), np.zeros(1, np.int64), w.D, w.grid) as layer:
        gid, gd = api.p2p_join(layer, w.points, form=form)
        np.testing.assert_array_equal(to_np(gid), -1)
        assert np.isinf(to_np(gd)).all()


def test_layer_errors(api):
    from paper_1403_0802_gb300._lib import SJError, SJ_ERR_INVALID, SJ_ERR_GRID_COVER
    g = dict(x0=0.0, y0=0.0, x1=10.0, y1=10.0, nx=4, ny=4)
    verts, ro, pro = layer_from_rings([[[(1, 1), (2, 1), (2, 2)]]])
    with pytest.raises(SJError) as e:
        api.pip_layer(verts + 20.0, ro, pro, g)
    assert e.value.status == SJ_ERR_GRID_COVER
    with pytest.raises(SJError) as e:
        api.pip_layer(verts[:2], np.array([0, 2]), pro, g)            # ring of two vertices
    assert e.value.status == SJ_ERR_INVALID
    bad = verts.copy()
    bad[0, 0] = np.nan
    with pytest.raises(SJError) as e:
        api.pip_layer(bad, ro, pro, g)
    assert e.value.status == SJ_ERR_INVALID
    with pytest.raises(SJError) as e:
        api.p2p_layer(verts, np.array([0, 3]), -1.0, g)
    assert e.value.status == SJ_ERR_INVALID


# ------------------------------------------------------------------ P2P

@pytest.mark.parametrize("form", FORMS)
def test_p2p_walks_full_size(api, oracle, form):
    """10,000,000 mixture points, 100,000 random-walk polylines, D = 100 m,
    grid 512 x 512 -- the benchmark's workload and launch configuration."""
    w = synth.p2p_walks()
    Lw = w.polylines
    with api.p2p_layer(Lw.verts, Lw.line_off, w.D, w.grid) as layer:
        pts = torch.as_tensor(w.points, device="cuda")
        gid, gd = api.p2p_join(layer, pts, form=form)
        gid, gd = to_np(gid), to_np(gd)
    r = check_p2p(oracle, w, gid, gd, form)
    assert 0.5 < r["hit_frac"] < 0.99


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("ppi", [1, 13, 64, 128])
def test_p2p_subset_ragged_items(api, oracle, form, ppi):
    w = synth.p2p_walks(n_points=200_003, n_lines=20_000)
    Lw = w.polylines
    with api.p2p_layer(Lw.verts, Lw.line_off, w.D, w.grid) as layer:
        gid, gd = api.p2p_join(layer, w.points, form=form, pts_per_item=ppi)
    check_p2p(oracle, w, to_np(gid), to_np(gd), form)


@pytest.mark.parametrize("form", FORMS)
def test_p2p_degenerate_polylines(api, oracle, form):
    """One-vertex polylines, zero-length segments, duplicated polylines (exact
    ties go to the smaller id), points on polylines and at exactly D, long
    polylines spanning several staging chunks."""
    rng = np.random.default_rng(3)
    lines = [
        [(100.0, 100.0)],                                  # a point
        [(200.0, 200.0), (200.0, 200.0), (260.0, 200.0)],  # zero-length first segment
        [(300.0, 300.0), (340.0, 300.0)],
        [(300.0, 300.0), (340.0, 300.0)],                  # duplicate of the previous one
        [(500.0, 500.0), (500.0, 600.0), (600.0, 600.0)],
    ]
    t = np.linspace(0, 2 * np.pi, 600)
    lines.append(list(zip(700 + 150 * np.cos(t), 700 + 150 * np.sin(t))))   # 600 vertices, > 1 chunk
    verts = np.concatenate([np.asarray(l, np.float64) for l in lines])
    off = np.concatenate([[0], np.cumsum([len(l) for l in lines])]).astype(np.int64)
    D = 16.0
    pts = np.concatenate([
        np.array([[100.0, 116.0], [100.0, 116.0001], [230.0, 216.0], [320.0, 310.0], [320.0, 300.0],
                  [500.0, 550.0], [550.0, 600.0], [100.0, 100.0], [700.0, 700.0], [850.0, 700.0]]),
        rng.uniform(0, 1024, (50000, 2))])
    g = dict(x0=0.0, y0=0.0, x1=1024.0, y1=1024.0, nx=32, ny=32)

    class W:
        pass
    w = W()
    w.grid, w.points, w.D, w.polylines = g, pts, D, None
    with api.p2p_layer(verts, off, D, g) as layer:
        gid, gd = api.p2p_join(layer, pts, form=form)
    gid, gd = to_np(gid), to_np(gd)
    check_p2p(oracle, w, gid, gd, form, verts=verts, line_off=off)
    assert gid[0] == 0 and gd[0] == 16.0                # exactly D: inclusive window
    assert gid[1] == -1
    assert gid[3] == 2                                   # tie between ids 2 and 3
    assert gid[4] == 2 and gd[4] == 0.0
    assert gid[7] == 0 and gd[7] == 0.0


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("D", [0.0, 50.0, 100.0])
def test_p2p_window_across_cell_boundaries(api, oracle, form, D):
    """Per-cell segment lists at their edges: axis-aligned segments on a 25 m
    lattice (cells are 100 m, so segment ends and ends +- D fall on cell
    boundaries), points at distance just under and just over D from a segment
    end or side, in the neighbouring cells.  A segment missing from a cell's
    list changes an id against the oracle, which filters whole polylines."""
    rng = np.random.default_rng(int(D) + 11)
    g = dict(x0=0.0, y0=0.0, x1=6400.0, y1=6400.0, nx=64, ny=64)
    lines = []
    for _ in range(400):
        x, y = 25.0 * rng.integers(8, 248, 2)
        k = int(rng.integers(1, 5))
        if rng.random() < 0.5:
            lines.append([(x, y), (x + 25.0 * k, y)])
        else:
            lines.append([(x, y), (x, y + 25.0 * k)])
    verts = np.concatenate([np.asarray(l, np.float64) for l in lines])
    off = np.arange(0, 2 * len(lines) + 1, 2, dtype=np.int64)
    pts = []
    for s_ in (1.0 - 1e-7, 1.0 + 1e-7):
        r = D * s_
        for (ax, ay), (bx, by) in lines:
            for (px, py) in ((ax, ay), (bx, by), (0.5 * (ax + bx), 0.5 * (ay + by))):
                for (ux, uy) in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                    pts.append((px + r * ux, py + r * uy))
                q = r / math.sqrt(2.0)
                for (ux, uy) in ((1, 1), (1, -1), (-1, 1), (-1, -1)):
                    pts.append((px + q * ux, py + q * uy))
    pts = np.asarray(pts, np.float64)

    class W:
        pass
    w = W()
    w.grid, w.points, w.D, w.polylines = g, pts, D, None
    with api.p2p_layer(verts, off, D, g) as layer:
        gid, gd = api.p2p_join(layer, pts, form=form)
    check_p2p(oracle, w, to_np(gid), to_np(gd), form, verts=verts, line_off=off)


@pytest.mark.parametrize("form", FORMS)
def test_p2p_window_larger_than_the_extent(api, oracle, form):
    """D larger than the grid's extent: every polyline is a candidate of every
    cell and every segment is in every cell's list (the longest lists the
    layer build sorts and the refinement stages)."""
    rng = np.random.default_rng(17)
    layer = synth.random_walks(rng, rng.integers(2, 41, size=800), extent=2048.0)
    g = dict(x0=0.0, y0=0.0, x1=2048.0, y1=2048.0, nx=16, ny=16)
    pts = rng.uniform(-100.0, 2148.0, (20_000, 2))

    class W:
        pass
    w = W()
    w.grid, w.points, w.D, w.polylines = g, pts, 3000.0, layer
    with api.p2p_layer(layer.verts, layer.line_off, w.D, g) as L:
        info = L.info()
        assert info["n_candidates"] == 16 * 16 * 800
        gid, gd = api.p2p_join(L, pts, form=form)
    r = check_p2p(oracle, w, to_np(gid), to_np(gd), form)
    inside = (pts[:, 0] >= 0) & (pts[:, 0] < 2048) & (pts[:, 1] >= 0) & (pts[:, 1] < 2048)
    assert (to_np(gid)[inside] >= 0).all() and (to_np(gid)[~inside] < 0).all()


@pytest.mark.parametrize("form", FORMS)
def test_p2p_window_per_call(api, oracle, form):
    """One resident layer built for D = 100 m answers windows 0, 10, 37.5 and
    100 m per call (sj_p2p_join_window); each equals the oracle's join at that
    window, and the window D equals sj_p2p_join bit for bit."""
    w = synth.p2p_walks(n_points=200_003, n_lines=20_000)
    Lw = w.polylines
    D = w.D
    with api.p2p_layer(Lw.verts, Lw.line_off, D, w.grid) as layer:
        pts = torch.as_tensor(w.points, device="cuda")
        fid, fd = api.p2p_join(layer, pts, form=form)
        hits = []
        for win in (0.0, 10.0, 37.5, D):
            gid, gd = api.p2p_join(layer, pts, form=form, window=win)
            w.D = win
            r = check_p2p(oracle, w, to_np(gid), to_np(gd), form, D_layer=D)
            hits.append(r["hit_frac"])
            if win == D:
                assert torch.equal(gid, fid) and torch.equal(gd, fd)
        w.D = D
        for bad in (-1.0, D * (1 + 1e-9), float("nan")):
            with pytest.raises(Exception) as e:
                api.p2p_join(layer, pts, form=form, window=bad)
            assert "window" in str(e.value)
    assert hits[0] < hits[1] < hits[2] < hits[3]


@pytest.mark.parametrize("form", FORMS)
def test_p2p_window_from_host_buffers(api, oracle, form):
    """sj_p2p_join_window_host (two pipelined chunks at 3 M points) against the
    oracle at each window (ids to near-ties, distances within the bound of the
    form), and against the device window join: FP64 bit for bit; FP32X ids
    equal wherever the oracle's answer is unique (a point's FP64 recheck can
    depend on the other points of its work item, which the chunks change)."""
    w = synth.p2p_walks(n_points=3_000_000, n_lines=20_000)
    Lw = w.polylines
    ref = P2PRef(oracle, w.grid, Lw.verts, Lw.line_off, w.D)
    with api.p2p_layer(Lw.verts, Lw.line_off, w.D, w.grid) as layer:
        for win in (30.0, w.D):
            hid, hd = api.p2p_join_host(layer, w.points, form=form, window=win)
            gid, gd = api.p2p_join(layer, w.points, form=form, window=win)
            gid, gd = to_np(gid), to_np(gd)
            r = ref.join(w.points, win)
            ref.check(w.points, hid, hd, form, window=win, ref=r)
            ref.check(w.points, gid, gd, form, window=win, ref=r)
            if form == "fp64":
                np.testing.assert_array_equal(hid, gid)
                np.testing.assert_array_equal(hd, gd)
            else:
                u = ref.unique(w.points, win, ref=r)
                np.testing.assert_array_equal(hid[u], gid[u])
        with pytest.raises(Exception):
            api.p2p_join_host(layer, w.points[:10], form=form, window=w.D * 2)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("win", [25.0, 50.0])
def test_p2p_window_per_call_at_cell_boundaries(api, oracle, form, win):
    """Windows smaller than the layer's D = 100 m on the axis-aligned 25 m
    lattice, points just inside and just outside the window: the layer's
    lists, built for D, must give exactly the window's answers."""
    rng = np.random.default_rng(int(win) + 5)
    g = dict(x0=0.0, y0=0.0, x1=6400.0, y1=6400.0, nx=64, ny=64)
    lines = []
    for _ in range(400):
        x, y = 25.0 * rng.integers(8, 248, 2)
        k = int(rng.integers(1, 5))
        lines.append([(x, y), (x + 25.0 * k, y)] if rng.random() < 0.5 else [(x, y), (x, y + 25.0 * k)])
    verts = np.concatenate([np.asarray(l, np.float64) for l in lines])
    off = np.arange(0, 2 * len(lines) + 1, 2, dtype=np.int64)
    pts = []
    for s_ in (1.0 - 1e-7, 1.0 + 1e-7):
        r = win * s_
        for (ax, ay), (bx, by) in lines:
            for (px, py) in ((ax, ay), (bx, by), (0.5 * (ax + bx), 0.5 * (ay + by))):
                for (ux, uy) in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                    pts.append((px + r * ux, py + r * uy))
    pts = np.asarray(pts, np.float64)

    class W:
        pass
    w = W()
    w.grid, w.points, w.D, w.polylines = g, pts, win, None
    with api.p2p_layer(verts, off, 100.0, g) as layer:
        gid, gd = api.p2p_join(layer, pts, form=form, window=win)
    check_p2p(oracle, w, to_np(gid), to_np(gd), form, verts=verts, line_off=off, D_layer=100.0)


@pytest.mark.parametrize("form", FORMS)
def test_host_buffers_match_device(api, oracle, form):
    w = synth.p2p_walks(n_points=50_000, n_lines=10_000)
    Lw = w.polylines
    with api.p2p_layer(Lw.verts, Lw.line_off, w.D, w.grid) as layer:
        did, dd = api.p2p_join(layer, w.points, form=form)
        hid, hd = api.p2p_join_host(layer, w.points, form=form)
    np.testing.assert_array_equal(to_np(did), hid)
    np.testing.assert_array_equal(to_np(dd), hd)
    w = synth.pip_stars(n_points=50_000)
    P = w.polygons
    with api.pip_layer(P.verts, P.ring_off, P.poly_ring_off, w.grid) as layer:
        np.testing.assert_array_equal(to_np(api.pip_join(layer, w.points, form=form)),
                                      api.pip_join_host(layer, w.points, form=form))


@pytest.mark.parametrize("form", FORMS)
def test_host_join_pipelined_chunks(api, oracle, form):
    """Host joins of more than 2 M points run as chunks on two streams; every
    point's result is checked against the oracle, and equals the device join's
    (FP64 bit for bit; FP32X ids equal wherever the oracle's answer is unique,
    since a point's FP64 recheck can depend on the other points of its work
    item)."""
    w = synth.p2p_walks(n_points=5_000_001, n_lines=20_000)
    Lw = w.polylines
    ref = P2PRef(oracle, w.grid, Lw.verts, Lw.line_off, w.D)
    with api.p2p_layer(Lw.verts, Lw.line_off, w.D, w.grid) as layer:
        did, dd = api.p2p_join(layer, w.points, form=form)
        hid, hd = api.p2p_join_host(layer, w.points, form=form)
    did, dd = to_np(did), to_np(dd)
    r = ref.join(w.points)
    ref.check(w.points, hid, hd, form, ref=r)
    if form == "fp64":
        np.testing.assert_array_equal(did, hid)
        np.testing.assert_array_equal(dd, hd)
    else:
        u = ref.unique(w.points, ref=r)
        np.testing.assert_array_equal(did[u], hid[u])
    w = synth.pip_stars(n_points=4_500_000)
    P = w.polygons
    with api.pip_layer(P.verts, P.ring_off, P.poly_ring_off, w.grid) as layer:
        np.testing.assert_array_equal(to_np(api.pip_join(layer, w.points, form=form)),
                                      api.pip_join_host(layer, w.points, form=form))


@pytest.mark.parametrize("form", FORMS)
def test_subcell_order_gives_the_same_results(api, oracle, form):
    """Points ordered by sub-cell inside their cells (SJ_FLAG_SUBCELL_ON) on
    dense grids: P2P (2 M clustered points, 128 x 128 cells, 32 points per
    work item: several items per cell) and PIP (the heavy-tail tiling, 1 M
    points, 256 x 256 cells, 16 points per item) against the oracle, and
    against arrival order within cells (FP64 bit for bit); the exact per-item
    prunes then leave fewer tests."""
    w = synth.p2p_walks(n_points=2_000_003, n_lines=20_000, grid_n=128)
    Lw = w.polylines
    ref = P2PRef(oracle, w.grid, Lw.verts, Lw.line_off, w.D)
    r = ref.join(w.points)
    res, tests = {}, {}
    with api.p2p_layer(Lw.verts, Lw.line_off, w.D, w.grid) as layer:
        pts = torch.as_tensor(w.points, device="cuda")
        for sub in (False, True):
            layer.reset_stats()
            gid, gd = api.p2p_join(layer, pts, form=form, subcell=sub, pts_per_item=32)
            res[sub] = (to_np(gid), to_np(gd))
            tests[sub] = layer.stats()["edge_tests"]
            ref.check(w.points, *res[sub], form, ref=r)
    if form == "fp64":
        np.testing.assert_array_equal(res[False][0], res[True][0])
        np.testing.assert_array_equal(res[False][1], res[True][1])
    assert tests[True] < 0.9 * tests[False]
    w = synth.pip_tiles(n_points=1_000_003, layer=2, grid_n=256)
    P = w.polygons
    want = oracle.pip_join(w.grid, w.points, P.verts, P.ring_off, P.poly_ring_off)
    with api.pip_layer(P.verts, P.ring_off, P.poly_ring_off, w.grid) as layer:
        for sub in (False, True):
            layer.reset_stats()
            got = to_np(api.pip_join(layer, w.points, form=form, subcell=sub, pts_per_item=16))
            np.testing.assert_array_equal(got, want)
            tests[sub] = layer.stats()["edge_tests"]
    assert tests[True] < tests[False]


def test_fp32x_fallback_rate_is_small(api, oracle):
    w = synth.p2p_walks(n_points=1_000_000)
    Lw = w.polylines
    with api.p2p_layer(Lw.verts, Lw.line_off, w.D, w.grid) as layer:
        api.p2p_join(layer, w.points, form="fp32x")
        st = layer.stats()
    assert st["fallbacks"] < 1e-3 * st["points"]


@pytest.mark.parametrize("g", [
    dict(x0=-123.456, y0=7.89, x1=99876.54, y1=100007.1, nx=1013, ny=997),
    dict(x0=4.5e6, y0=5.3e6, x1=4.5e6 + 37123.3, y1=5.3e6 + 411.7, nx=100_003, ny=7),   # UTM-like, 0.37 m cells
    dict(x0=0.0, y0=0.0, x1=1e5, y1=1e5, nx=1024, ny=1024),
], ids=["odd", "utm", "bench"])
def test_cell_ids_exact_at_cell_boundaries(api, oracle, g):
    """The threshold-table cell id must equal the FP64 rule floor(fl(fl(x-x0)/cw))
    exactly, including points on, and one ulp around, every cell boundary."""
    rng = np.random.default_rng(1)
    cw = (g["x1"] - g["x0"]) / g["nx"]
    ch = (g["y1"] - g["y0"]) / g["ny"]
    kx = np.unique(np.concatenate([np.arange(0, g["nx"] + 1, max(1, g["nx"] // 3000)), [0, g["nx"]]]))
    bx = g["x0"] + kx * cw
    xs = np.concatenate([bx, np.nextafter(bx, -np.inf), np.nextafter(bx, np.inf),
                         rng.uniform(g["x0"] - cw, g["x1"] + cw, 2000), [g["x0"], g["x1"], -0.0, 0.0]])
    ky = np.arange(0, g["ny"] + 1, max(1, g["ny"] // 40))
    by = g["y0"] + ky * ch
    ys = np.concatenate([by, np.nextafter(by, -np.inf), np.nextafter(by, np.inf), [g["y0"], g["y1"]]])
    X, Y = np.meshgrid(xs, ys[:60])
    pts = np.stack([X.ravel(), Y.ravel()], 1)
    pts = np.concatenate([pts, np.stack([np.full(len(ys), xs[5]), ys], 1), [[np.nan, g["y0"]], [np.inf, g["y0"]]]])
    cs, perm = api.bucket_points(pts, g)
    cs, perm = to_np(cs), to_np(perm)
    G = g["nx"] * g["ny"]
    gpu_cell = np.full(len(pts), G, np.int64)
    gpu_cell[perm[:cs[-1]]] = np.repeat(np.arange(G), np.diff(cs))
    np.testing.assert_array_equal(gpu_cell, oracle.point_cells(g, pts))


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("layer", [1, 2, 3])
def test_pip_tiles_subset(api, oracle, form, layer):
    """PIP at scale on a 1,000,003-point subset: the clustered mixture against
    the 40,000-tile layer (median 19, max 5,004 vertices), the 14,000-tile
    layer (median ~500, max 100,004 vertices, edges staged in many chunks) and
    the multi-ring layer (layer 1 with island holes and their islands)."""
    w = synth.pip_tiles(n_points=1_000_003, layer=layer)
    P = w.polygons
    ref, nh = oracle.pip_join(w.grid, w.points, P.verts, P.ring_off, P.poly_ring_off, with_hits=True)
    assert nh.max() == 1 and (ref >= 0).all()          # a tiling: every point in exactly one tile
    with api.pip_layer(P.verts, P.ring_off, P.poly_ring_off, w.grid) as layer_:
        got = to_np(api.pip_join(layer_, w.points, form=form))
    np.testing.assert_array_equal(got, ref)


# ------------------------------------------------------------------ full-size at-scale configurations
# The GPU joins every point, in the launch configuration bench.py times; the
# oracle recomputes a seeded sample of the outputs one by one (it cannot join
# 1e8 points in seconds).

SAMPLE = 200_000


@pytest.fixture(scope="module")
def tiles_points():
    """The 100,000,000 clustered points of the PIP-at-scale workloads (the
    same points for every layer), generated once for the module."""
    return synth.pip_tiles(layer=1).points


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("layer", [1, 2, 3])
def test_pip_at_scale_full_size_sampled(api, oracle, tiles_points, layer, form):
    """100,000,000 clustered points against the 40,000-tile (layer 1), the
    heavy-tail 14,000-tile (layer 2) or the multi-ring (layer 3: layer 1 with
    island holes) tiling, grid 1024 x 1024, in both forms with the launch
    settings the benchmark uses: ids of a 200,000-point sample bit-identical
    to the oracle; every point in exactly one polygon."""
    import bench
    w = synth.pip_tiles(n_points=1, layer=layer)
    P = w.polygons
    t = bench.TUNED[f"pip3_{layer}"]
    with api.pip_layer(P.verts, P.ring_off, P.poly_ring_off, w.grid) as layer_:
        pts = torch.as_tensor(tiles_points, device="cuda")
        got = api.pip_join(layer_, pts, form=form, pts_per_item=t["ppi"], block=t["block"],
                           edges_per_chunk=t["edges"])
        del pts
        got = to_np(got)
    assert (got >= 0).all()                              # a tiling covers the extent
    idx = np.random.default_rng(layer).choice(len(tiles_points), SAMPLE, replace=False)
    ref = oracle.pip_join(w.grid, np.ascontiguousarray(tiles_points[idx]), P.verts, P.ring_off, P.poly_ring_off)
    np.testing.assert_array_equal(got[idx], ref)
    if layer == 3:                                       # points in holes answer the island
        assert (ref >= 40_000).sum() > 1000


@pytest.fixture(scope="module")
def walks_at_scale():
    """The P2P-at-scale workload (170,000,000 clustered points, 150,000
    lognormal walks), generated once for the module; D varies per test."""
    return synth.p2p_walks_lognormal()


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("D", [50.0, 100.0, 200.0])
def test_p2p_at_scale_full_size_sampled(api, oracle, walks_at_scale, D, form):
    """170,000,000 clustered points against 150,000 lognormal random walks,
    grid 512 x 512, D = 50, 100 and 200 m, both forms: a 200,000-point sample
    against the oracle (ids exact up to near-ties, FP64 distances within
    1e-12 relative, FP32X within the certified bound)."""
    w = walks_at_scale
    Lw = w.polylines
    with api.p2p_layer(Lw.verts, Lw.line_off, D, w.grid) as layer:
        pts = torch.as_tensor(w.points, device="cuda")
        gid, gd = api.p2p_join(layer, pts, form=form)
        del pts
        gid, gd = to_np(gid), to_np(gd)
    idx = np.random.default_rng(4).choice(len(w.points), SAMPLE, replace=False)
    sample = np.ascontiguousarray(w.points[idx])
    ref = P2PRef(oracle, w.grid, Lw.verts, Lw.line_off, D)
    r = ref.check(sample, gid[idx], gd[idx], form)
    assert 0.02 < r["hit_frac"] < 1.0


def test_pip_at_the_maximum_point_count(api, oracle):
    """N = 2^31 - 2^22 points, the largest count a join accepts (34 GB of
    points, about 90 GB on the device in all), against the 1,024 stars: the
    32-bit indices of every kernel reach their limit.  A seeded 200,000-point
    sample is checked against the oracle one by one; one point more is
    rejected before any device work."""
    N = (1 << 31) - (1 << 22)
    free, _ = torch.cuda.mem_get_info()
    if free < 120e9:
        pytest.skip("needs about 120 GB of free device memory")
    w = synth.pip_stars(n_points=1000)
    P = w.polygons
    gen = torch.Generator(device="cuda").manual_seed(20140304)
    with api.pip_layer(P.verts, P.ring_off, P.poly_ring_off, w.grid) as layer:
        pts = torch.rand((N, 2), dtype=torch.float64, device="cuda", generator=gen).mul_(1e5)
        out = torch.empty(N, dtype=torch.int32, device="cuda")
        api.pip_join(layer, pts, out, form="fp32x")
        idx = torch.as_tensor(np.random.default_rng(7).choice(N, SAMPLE, replace=False), device="cuda")
        sample = pts[idx].cpu().numpy()
        got = out[idx].cpu().numpy()
        tail = out[-SAMPLE:].cpu().numpy()
        tail_pts = pts[-SAMPLE:].cpu().numpy()
        hit_frac = float((out[: 1 << 24] >= 0).float().mean())
        from paper_1403_0802_gb300 import _lib
        assert _lib.lib().sj_pip_join(layer.handle, pts.data_ptr(), N + 1, out.data_ptr(), None,
                                      None) == _lib.SJ_ERR_INVALID
        del pts, out
        torch.cuda.empty_cache()
    np.testing.assert_array_equal(got, oracle.pip_join(w.grid, np.ascontiguousarray(sample), P.verts, P.ring_off,
                                                       P.poly_ring_off))
    np.testing.assert_array_equal(tail, oracle.pip_join(w.grid, np.ascontiguousarray(tail_pts), P.verts,
                                                        P.ring_off, P.poly_ring_off))
    assert 0.3 < hit_frac < 0.45
