"""Pins of the oracle's point-to-polyline distance and nearest-polyline search
(Sec. III.B, Fig. 2) against closed forms, exact rational arithmetic, dense
sampling of the polyline, and invariants."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_1403_0802_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
SHAPES = json.load(open(os.path.join(HERE, "golden", "p2p_shapes.json")))["polylines"]
G = dict(x0=-64.0, y0=-64.0, x1=64.0, y1=64.0, nx=16, ny=16)


def layer(*lines):
    verts = np.concatenate([np.asarray(l, np.float64).reshape(-1, 2) for l in lines])
    off = np.zeros(len(lines) + 1, np.int64)
    off[1:] = np.cumsum([len(l) for l in lines])
    return verts, off


def test_segment_closed_forms(oracle):
    """Segment (0,0)-(8,0): |y| above the segment, Euclidean distance to the
    nearer end beyond it (Pythagorean triples keep every value exact)."""
    cases = [((4, 3), 3.0), ((4, -6), 6.0), ((0, 5), 5.0), ((8, -5), 5.0), ((-3, 4), 5.0), ((11, 4), 5.0),
             ((-6, -8), 10.0), ((14, 8), 10.0), ((4, 0), 0.0), ((0, 0), 0.0), ((8, 0), 0.0), ((-1, 0), 1.0),
             ((9.5, 0), 1.5), ((2.25, -0.5), 0.5)]
    for (px, py), d in cases:
        for (ax, ay, bx, by, x, y) in [(0, 0, 8, 0, px, py), (8, 0, 0, 0, px, py),     # both directions
                                       (0, 0, 0, 8, py, px), (0, 8, 0, 0, py, px),     # 90-degree turns
                                       (0, 0, -8, 0, -px, -py)]:                       # half turn
            assert oracle.seg_dist(x, y, ax, ay, bx, by) == d, (x, y, ax, ay, bx, by)


def test_golden_polylines(oracle):
    verts, off = layer(*SHAPES.values())
    names = list(SHAPES)
    idx = {n: i for i, n in enumerate(names)}
    d = lambda name, x, y: oracle.line_dist(x, y, verts, off, idx[name])
    assert d("l_shape", 4, 3) == 3.0          # above the first leg
    assert d("l_shape", 11, 3) == 3.0         # right of the second leg
    assert d("l_shape", 12, 9) == 5.0         # beyond the far end: (4, 3) triple
    assert d("l_shape", 8, 6) == 0.0
    assert d("diag_8", 3, 3) == 0.0           # on a 45-degree segment
    assert d("diag_8", 11, 12) == 5.0         # (3, 4) from the end (8, 8)
    assert d("zero_length", 6, 7) == 5.0      # zero-length segment is a point
    assert d("single_vertex", 8, -3) == 5.0   # one-vertex polyline is a point
    assert d("y_axis_8", -2.5, 4) == 2.5


def exact_seg_dist2(p, a, b):
    """Independent reference: exact squared distance to the closest point
    a + t (b - a), t clamped to [0, 1], in rational arithmetic."""
    p, a, b = [tuple(Fraction(float(v)) for v in q) for q in (p, a, b)]
    ex, ey = b[0] - a[0], b[1] - a[1]
    L2 = ex * ex + ey * ey
    t = Fraction(0) if L2 == 0 else min(max(((p[0] - a[0]) * ex + (p[1] - a[1]) * ey) / L2, Fraction(0)),
                                        Fraction(1))
    qx, qy = a[0] + t * ex, a[1] + t * ey
    return (p[0] - qx) ** 2 + (p[1] - qy) ** 2


def test_random_segments_against_exact_rationals(oracle):
    rng = np.random.default_rng(5)
    worst = 0.0
    for _ in range(3000):
        a, b, p = rng.uniform(-1000, 1000, size=(3, 2))
        if rng.random() < 0.2:
            b = a + rng.uniform(-1, 1, 2) * 1e-3          # very short segments
        ref = math.sqrt(exact_seg_dist2(p, a, b))
        got = oracle.seg_dist(*p, *a, *b)
        err = abs(got - ref) / max(ref, 1.0)
        worst = max(worst, err)
    assert worst < 1e-12, worst


def test_polyline_distance_brackets_dense_sampling(oracle):
    """Dense sampling of the polyline gives an upper bound and, minus half the
    sample spacing, a lower bound on the true distance."""
    rng = np.random.default_rng(9)
    L = synth.random_walks(rng, rng.integers(2, 12, size=40), extent=2000.0)
    for l in range(L.n_lines):
        v = L.verts[L.line_off[l]:L.line_off[l + 1]]
        samples, h = [v[:1]], 0.0
        for a, b in zip(v[:-1], v[1:]):
            seg = np.linalg.norm(b - a)
            k = max(int(seg / 0.01), 1)
            h = max(h, seg / k)
            t = np.linspace(0, 1, k + 1)[:, None]
            samples.append(a + t * (b - a))
        S = np.concatenate(samples)
        for p in rng.uniform(v.min(0) - 50, v.max(0) + 50, size=(5, 2)):
            d = oracle.line_dist(p[0], p[1], L.verts, L.line_off, l)
            ds = np.hypot(S[:, 0] - p[0], S[:, 1] - p[1]).min()
            assert ds - h / 2 - 1e-9 <= d <= ds + 1e-9, (l, p, d, ds)


def test_window_is_inclusive_and_ties_go_to_smaller_id(oracle):
    verts, off = layer([(0, 0), (8, 0)], [(0, 0), (8, 0)], [(0, 5), (8, 5)])
    pts = np.array([[4.0, 2.0], [4.0, -2.0], [4.0, 2.5], [4.0, 8.0], [4.0, 9.0], [40.0, 40.0]])
    oid, od, d1, d2 = oracle.p2p_join(G, pts, verts, off, 3.0)
    np.testing.assert_array_equal(oid, [0, 0, 0, 2, -1, -1])
    np.testing.assert_array_equal(od, [2.0, 2.0, 2.5, 3.0, np.inf, np.inf])
    assert d2[0] == 2.0        # the identical copy (id 1) ties with the winner
    assert d2[2] == 2.5        # (4, 2.5) is equidistant from ids 0, 1 and 2: id 0 wins
    oid_b, od_b, _, _ = oracle.p2p_brute(G, pts, verts, off, 3.0)
    np.testing.assert_array_equal(oid_b, oid)
    np.testing.assert_array_equal(od_b, od)


def test_points_on_polylines_are_at_distance_zero(oracle):
    rng = np.random.default_rng(2)
    L = synth.random_walks(rng, rng.integers(2, 30, size=200), extent=100.0)
    verts = np.round(L.verts * 64) / 64
    pts = verts[rng.integers(0, len(verts), 500)]
    g = dict(x0=0.0, y0=0.0, x1=128.0, y1=128.0, nx=32, ny=32)
    oid, od, _, _ = oracle.p2p_join(g, pts, verts, L.line_off, 1.0)
    assert (od == 0.0).all() and (oid >= 0).all()
    # axis-aligned dyadic segments: every dyadic point on them is at distance 0
    v2, off2 = layer([(1, 1), (9, 1), (9, 7)])
    on = np.array([[3.25, 1.0], [9.0, 2.5], [9.0, 7.0], [1.0, 1.0]])
    oid, od, _, _ = oracle.p2p_join(G, on, v2, off2, 0.0)
    np.testing.assert_array_equal(od, 0.0)
    np.testing.assert_array_equal(oid, 0)


def test_translation_invariance_dyadic(oracle):
    rng = np.random.default_rng(4)
    L = synth.random_walks(rng, rng.integers(2, 20, size=500), extent=8192.0)
    q = lambda a: np.round(a * 1024) / 1024
    verts = q(L.verts)
    pts = q(synth.points_mixture(20000, rng, extent=8192.0))
    g0 = dict(x0=0.0, y0=0.0, x1=8192.0, y1=8192.0, nx=64, ny=64)
    base = oracle.p2p_join(g0, pts, verts, L.line_off, 100.0)
    t = np.array([65536.0, 131072.0])
    g = dict(x0=t[0], y0=t[1], x1=t[0] + 8192.0, y1=t[1] + 8192.0, nx=64, ny=64)
    got = oracle.p2p_join(g, pts + t, verts + t, L.line_off, 100.0)
    np.testing.assert_array_equal(got[0], base[0])
    np.testing.assert_array_equal(got[1], base[1])


def test_walk_workload_brute_equals_filtered(oracle):
    w = synth.p2p_walks(n_points=3000, n_lines=20000)
    L = w.polylines
    oid, od, d1, d2 = oracle.p2p_join(w.grid, w.points, L.verts, L.line_off, w.D)
    bid, bd, _, _ = oracle.p2p_brute(w.grid, w.points, L.verts, L.line_off, w.D)
    np.testing.assert_array_equal(oid, bid)
    np.testing.assert_array_equal(od, bd)
    assert ((od <= w.D) == (oid >= 0)).all()
    assert (d1[oid >= 0] == od[oid >= 0]).all() and (d2 >= d1).all()
    assert 0.3 < (oid >= 0).mean() < 0.99


def test_layer_validation(oracle):
    verts, off = layer([(0, 0), (1, 1)])
    oracle.p2p_mbb(G, verts, off)
    with pytest.raises(oracle.OracleError):
        oracle.p2p_mbb(G, verts, np.array([0, 0, 2]))          # empty polyline
    with pytest.raises(oracle.OracleError) as e:
        oracle.p2p_mbb(G, verts + 100.0, off)
    assert e.value.code == oracle.GRID_COVER
