"""Pins of the oracle's point-in-polygon test (Sec. III.C) against facts that
do not come from the oracle itself: closed-form regions, an independent
winding-number computation, an exact tiling invariant on degenerate integer
inputs, and translation invariance."""
import json
import math
import os

import numpy as np
import pytest

from paper_1403_0802_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def layer_from_rings(polys):
    """polys: list of polygons, each a list of rings (lists of (x, y))."""
    verts, ring_off, poly_ring_off = [], [0], [0]
    for rings in polys:
        for ring in rings:
            verts.extend(ring)
            ring_off.append(len(verts))
        poly_ring_off.append(len(ring_off) - 1)
    return (np.asarray(verts, np.float64).reshape(-1, 2), np.asarray(ring_off, np.int64),
            np.asarray(poly_ring_off, np.int64))


def in_region(region, x, y):
    """Closed-form membership: union of convex pieces of (a, b, c, strict)."""
    inside = np.zeros(len(x), bool)
    for piece in region:
        ok = np.ones(len(x), bool)
        for a, b, c, strict in piece:
            v = a * x + b * y + c
            ok &= (v > 0) if strict else (v >= 0)
        inside |= ok
    return inside


def dyadic_lattice(lo, hi, step):
    xs = np.arange(lo, hi + step / 2, step)
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    return np.stack([X.ravel(), Y.ravel()], 1)


GRID_SMALL = dict(x0=-16.0, y0=-16.0, x1=16.0, y1=16.0, nx=8, ny=8)


@pytest.mark.parametrize("shape", json.load(open(os.path.join(HERE, "golden", "pip_shapes.json")))["shapes"],
                         ids=lambda s: s["name"])
def test_closed_form_regions(oracle, shape):
    verts, ro, pro = layer_from_rings([shape["rings"]])
    pts = dyadic_lattice(-1.0, 8.0, 0.25)
    expect = np.where(in_region(shape["region"], pts[:, 0], pts[:, 1]), 0, -1)
    got_b = oracle.pip_brute(GRID_SMALL, pts, verts, ro, pro)
    got_g = oracle.pip_join(GRID_SMALL, pts, verts, ro, pro)
    bad = np.flatnonzero(got_b != expect)
    assert bad.size == 0, (shape["name"], pts[bad[:5]], got_b[bad[:5]], expect[bad[:5]])
    np.testing.assert_array_equal(got_g, expect)


def test_multiple_hits_take_smallest_id(oracle):
    sq = [[(0, 0), (4, 0), (4, 4), (0, 4)]]
    small = [[(1, 1), (2, 1), (2, 2), (1, 2)]]
    verts, ro, pro = layer_from_rings([small, sq, sq])
    pts = np.array([[1.5, 1.5], [3.0, 3.0], [5.0, 5.0]])
    ids, nh = oracle.pip_join(GRID_SMALL, pts, verts, ro, pro, with_hits=True)
    np.testing.assert_array_equal(ids, [0, 1, -1])
    np.testing.assert_array_equal(nh, [3, 2, 0])


def test_points_outside_grid_are_minus_one(oracle):
    sq = [[(0, 0), (16, 0), (16, 16), (0, 16)]]
    verts, ro, pro = layer_from_rings([sq])
    pts = np.array([[8.0, 8.0], [16.0, 8.0], [8.0, 16.0], [np.nan, 1.0], [-16.0, -16.0]])
    ids = oracle.pip_join(GRID_SMALL, pts, verts, ro, pro)
    np.testing.assert_array_equal(ids, [0, -1, -1, -1, -1])


def winding_number(px, py, ring):
    """Independent reference: winding number by summing the signed angles the
    ring's edges subtend at p (atan2), rounded to an integer."""
    r = np.asarray(ring, np.float64)
    a = r - (px, py)
    b = np.roll(r, -1, axis=0) - (px, py)
    ang = np.arctan2(a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0], (a * b).sum(1))
    return int(round(ang.sum() / (2 * math.pi)))


def boundary_distance(px, py, ring):
    r = np.asarray(ring, np.float64)
    a, b = r, np.roll(r, -1, axis=0)
    e = b - a
    t = np.clip(((px - a[:, 0]) * e[:, 0] + (py - a[:, 1]) * e[:, 1]) / np.maximum((e * e).sum(1), 1e-300), 0, 1)
    q = a + t[:, None] * e
    return float(np.hypot(q[:, 0] - px, q[:, 1] - py).min())


def test_star_polygons_agree_with_winding_number(oracle):
    """For simple polygons, even-odd parity and a non-zero winding number are
    the same set away from the boundary."""
    rng = np.random.default_rng(7)
    layer = synth.star_polygons(rng, n_side=4, extent=1000.0)
    g = synth.grid(16, extent=1000.0)
    pts = synth.points_uniform(3000, rng, extent=1000.0)
    got = oracle.pip_brute(g, pts, layer.verts, layer.ring_off, layer.poly_ring_off)
    checked = 0
    for i, (px, py) in enumerate(pts):
        expect = -1
        near = False
        for p in range(layer.n_polygons):
            ring = layer.verts[layer.ring_off[p]:layer.ring_off[p + 1]]
            if boundary_distance(px, py, ring) < 1e-6:
                near = True
                break
            if winding_number(px, py, ring) != 0 and expect < 0:
                expect = p
        if near:
            continue
        checked += 1
        assert got[i] == expect, (i, px, py, got[i], expect)
    assert checked > 2900
    assert (got >= 0).mean() > 0.2


def jittered_triangulation(rng, n, step, jitter):
    """Triangles tiling [0, n*step]^2 exactly: lattice corners, interior ones
    moved by integer jitter, each quad split along a random diagonal.  Shared
    edges use identical coordinates."""
    P = np.zeros((n + 1, n + 1, 2))
    for i in range(n + 1):
        for j in range(n + 1):
            x, y = i * step, j * step
            if 0 < i < n:
                x += rng.integers(-jitter, jitter + 1)
            if 0 < j < n:
                y += rng.integers(-jitter, jitter + 1)
            P[i, j] = (x, y)
    polys = []
    for i in range(n):
        for j in range(n):
            a, b, c, d = P[i, j], P[i + 1, j], P[i + 1, j + 1], P[i, j + 1]
            if rng.integers(2):
                tris = [(a, b, c), (a, c, d)]
            else:
                tris = [(a, b, d), (b, c, d)]
            for t in tris:
                if rng.integers(2):
                    t = t[::-1]
                polys.append([[tuple(v) for v in t]])
    return polys


def test_exact_tiling_covers_each_point_once(oracle):
    """Integer coordinates make every FP64 step exact, and shared edges are
    bit-identical, so the half-open rule must put every point of the square
    [0, W) x [0, W) in exactly one triangle and every other point in none --
    including the many points that sit on edges and vertices."""
    rng = np.random.default_rng(11)
    n, step = 8, 4
    polys = jittered_triangulation(rng, n, step, jitter=1)
    verts, ro, pro = layer_from_rings(polys)
    W = n * step
    g = dict(x0=-8.0, y0=-8.0, x1=40.0, y1=40.0, nx=12, ny=12)
    pts = dyadic_lattice(-2.0, W + 2.0, 0.5)
    ids, nh = oracle.pip_join(g, pts, verts, ro, pro, with_hits=True)
    inside = (pts[:, 0] >= 0) & (pts[:, 0] < W) & (pts[:, 1] >= 0) & (pts[:, 1] < W)
    np.testing.assert_array_equal(nh, inside.astype(np.int32))
    ids_b, nh_b = oracle.pip_brute(g, pts, verts, ro, pro, with_hits=True)
    np.testing.assert_array_equal(ids, ids_b)
    np.testing.assert_array_equal(nh, nh_b)


def test_translation_invariance_dyadic(oracle):
    """Coordinates on a 2^-10 lattice below 2^17, translated by k * 2^16, stay
    exact, so results must not change."""
    rng = np.random.default_rng(3)
    layer = synth.star_polygons(rng, n_side=8, extent=65536.0)
    q = lambda a: np.round(a * 1024.0) / 1024.0
    verts = q(layer.verts)
    pts = q(synth.points_uniform(20000, rng, extent=65536.0))
    g0 = dict(x0=0.0, y0=0.0, x1=65536.0, y1=65536.0, nx=64, ny=64)
    base = oracle.pip_join(g0, pts, verts, layer.ring_off, layer.poly_ring_off)
    for kx, ky in [(1, 0), (0, 1), (1, 1)]:
        t = np.array([kx * 65536.0, ky * 65536.0])
        g = dict(x0=t[0], y0=t[1], x1=t[0] + 65536.0, y1=t[1] + 65536.0, nx=64, ny=64)
        got = oracle.pip_join(g, pts + t, verts + t, layer.ring_off, layer.poly_ring_off)
        np.testing.assert_array_equal(got, base)
    assert (base >= 0).mean() > 0.3


def test_star_workload_brute_equals_filtered_and_is_disjoint(oracle):
    w = synth.pip_stars(n_points=200_000)
    L = w.polygons
    ids_g, nh = oracle.pip_join(w.grid, w.points, L.verts, L.ring_off, L.poly_ring_off, with_hits=True)
    assert nh.max() <= 1
    sub = slice(0, 5000)
    ids_b = oracle.pip_brute(w.grid, w.points[sub], L.verts, L.ring_off, L.poly_ring_off)
    np.testing.assert_array_equal(ids_g[sub], ids_b)
    frac = (ids_g >= 0).mean()
    assert 0.2 < frac < 0.6


def test_layer_validation(oracle):
    g = GRID_SMALL
    verts, ro, pro = layer_from_rings([[[(0, 0), (1, 0), (1, 1)]]])
    oracle.pip_mbb(g, verts, ro, pro)
    with pytest.raises(oracle.OracleError) as e:   # ring with two vertices
        oracle.pip_mbb(g, verts[:2], np.array([0, 2]), pro)
    assert e.value.code == oracle.INVALID
    bad = verts.copy()
    bad[1, 0] = np.inf
    with pytest.raises(oracle.OracleError):
        oracle.pip_mbb(g, bad, ro, pro)
    far = verts + 100.0
    with pytest.raises(oracle.OracleError) as e:
        oracle.pip_mbb(g, far, ro, pro)
    assert e.value.code == oracle.GRID_COVER


@pytest.mark.parametrize("side_median,cap", [(2.6, 50), (30.0, 400)])
def test_synthetic_tiling_covers_every_point_once(oracle, side_median, cap):
    """The tiling generator shares each side's vertices between neighbours, so
    every point of the extent lies in exactly one tile -- an invariant on both
    the generator and the crossing rule (shared edges evaluate identically)."""
    rng = np.random.default_rng(17)
    P = synth.tiling(rng, 12, 9, side_median=side_median, side_cap=cap, extent=1000.0, n_giant=1)
    g = synth.grid(32, extent=1000.0)
    pts = np.concatenate([synth.points_uniform(20000, rng, extent=1000.0), P.verts[::7]])
    pts = pts[(pts < 1000.0).all(1)]
    ids, nh = oracle.pip_join(g, pts, P.verts, P.ring_off, P.poly_ring_off, with_hits=True)
    np.testing.assert_array_equal(nh, 1)
    assert P.polygon_sizes().max() >= 4 * cap
