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


@pytest.mark.parametrize("exact", [False, True], ids=["fp64", "exact"])
@pytest.mark.parametrize("shape", json.load(open(os.path.join(HERE, "golden", "pip_shapes.json")))["shapes"],
                         ids=lambda s: s["name"])
def test_closed_form_regions(oracle, shape, exact):
    """The closed-form regions hold under both predicate modes (the dyadic
    lattice makes every FP64 step exact, so the two rules must agree)."""
    verts, ro, pro = layer_from_rings([shape["rings"]])
    pts = dyadic_lattice(-1.0, 8.0, 0.25)
    expect = np.where(in_region(shape["region"], pts[:, 0], pts[:, 1]), 0, -1)
    oracle._load().or_set_exact(1 if exact else 0)
    try:
        got_b = oracle.pip_brute(GRID_SMALL, pts, verts, ro, pro)
        got_g = oracle.pip_join(GRID_SMALL, pts, verts, ro, pro)
    finally:
        oracle._load().or_set_exact(0)
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


def test_islands_layer_covers_every_point_once(oracle):
    """Holes of multi-ring tiles are also the rings of island polygons (the
    WWF-like layer): every point lies in exactly one polygon, hole vertices
    included; points in a hole take the island's id, not the tile's."""
    rng = np.random.default_rng(23)
    T = synth.tiling(rng, 12, 9, side_median=2.6, side_cap=50, extent=1000.0, n_giant=1)
    P = synth.with_islands(rng, T, 12, 9, hole_frac=0.6, extent=1000.0)
    n_tiles = 12 * 9
    assert P.n_polygons > n_tiles and (np.diff(P.poly_ring_off)[:n_tiles] > 1).any()
    g = synth.grid(32, extent=1000.0)
    pts = np.concatenate([synth.points_uniform(40000, rng, extent=1000.0), P.verts[::5]])
    pts = pts[(pts < 1000.0).all(1)]
    ids, nh = oracle.pip_join(g, pts, P.verts, P.ring_off, P.poly_ring_off, with_hits=True)
    np.testing.assert_array_equal(nh, 1)
    assert (ids >= n_tiles).mean() > 0.005
    # island i's ring is a hole of the tile whose lattice cell holds it
    isl = np.flatnonzero(ids >= n_tiles)
    cw, ch = 1000.0 / 12, 1000.0 / 9
    for k in isl[:200]:
        ring = P.ring_off[P.poly_ring_off[ids[k]]]
        vx, vy = P.verts[ring]
        t = int(vy // ch) * 12 + int(vx // cw)
        r0, r1 = P.poly_ring_off[t], P.poly_ring_off[t + 1]
        assert any(np.array_equal(P.verts[P.ring_off[r]:P.ring_off[r + 1]],
                                  P.verts[ring:P.ring_off[P.poly_ring_off[ids[k]] + 1]]) for r in range(r0 + 1, r1))


def _near_degenerate(rng, n):
    """Points within a couple of ulps of the line through l and h, with l and h
    of different magnitudes (so the FP64 differences round and the FP64 sign
    is often zero or wrong)."""
    l = rng.uniform(0.0, 1e5, (n, 2)) * rng.choice([1e-4, 1e-2, 1.0], (n, 1))
    h = rng.uniform(0.0, 1e5, (n, 2))
    t = rng.uniform(0.0, 1.0, n)
    p = l + t[:, None] * (h - l)
    k = rng.integers(-2, 3, n)
    p[:, 0] = p[:, 0] + k * np.spacing(p[:, 0])
    return l, h, p


def test_exact_predicate_matches_rational_arithmetic(oracle):
    """The exact mode's crossing sign equals the sign of the determinant in
    exact rational arithmetic (Python fractions of the same doubles) on points
    within a few ulps of the edge's line; the FP64 sign is wrong on some of
    them (so the cases reach the expansion arithmetic)."""
    from fractions import Fraction as F
    rng = np.random.default_rng(31)
    l, h, p = _near_degenerate(rng, 4000)
    wrong64 = flipped64 = 0
    with oracle.exact_predicates():
        for i in range(len(p)):
            hx, hy, lx, ly, px, py = (F(float(v)) for v in (h[i, 0], h[i, 1], l[i, 0], l[i, 1], p[i, 0], p[i, 1]))
            d = (hx - lx) * (py - ly) - (hy - ly) * (px - lx)
            want = (d > 0) - (d < 0)
            got = oracle.cross_sign(h[i, 0], h[i, 1], l[i, 0], l[i, 1], p[i, 0], p[i, 1])
            assert got == want, i
    for i in range(len(p)):
        hx, hy, lx, ly, px, py = (F(float(v)) for v in (h[i, 0], h[i, 1], l[i, 0], l[i, 1], p[i, 0], p[i, 1]))
        d = (hx - lx) * (py - ly) - (hy - ly) * (px - lx)
        f = oracle.cross_sign(h[i, 0], h[i, 1], l[i, 0], l[i, 1], p[i, 0], p[i, 1])
        wrong64 += f != (d > 0) - (d < 0)
        flipped64 += f * ((d > 0) - (d < 0)) < 0
    assert wrong64 > 100 and flipped64 > 10          # zero and opposite FP64 signs both occur


def test_exact_predicate_special_values(oracle):
    """Closed forms: points exactly on an edge give 0; one ulp off gives the
    side; exact arithmetic on integers far above 2^26 (where FP64 products
    round) still decides."""
    with oracle.exact_predicates():
        assert oracle.cross_sign(3.0, 7.0, 0.0, 0.0, 1.5, 3.5) == 0
        assert oracle.cross_sign(3.0, 7.0, 0.0, 0.0, np.nextafter(1.5, 0.0), 3.5) == 1
        assert oracle.cross_sign(3.0, 7.0, 0.0, 0.0, np.nextafter(1.5, 9.0), 3.5) == -1
        big = float(2 ** 40)
        # l = (0, 0), h = (big + 1, big - 1), p = (big + 3, big - 1): d = -2 (big - 1) exactly
        assert oracle.cross_sign(big + 1, big - 1, 0.0, 0.0, big + 3, big - 1) == -1
        # collinear with integer coordinates beyond 2^53 / 2 products: d = 0
        a = float(2 ** 30 + 3)
        assert oracle.cross_sign(3 * a, 5 * a, 0.0, 0.0, 6 * a, 10 * a) == 0
    assert oracle.cross_sign(3.0, 7.0, 0.0, 0.0, 1.5, 3.5) == 0      # FP64 mode is exact here too


def test_exact_mode_tiling_and_workloads(oracle):
    """Exact predicates keep the tiling invariant on points within ulps of the
    shared edges, and agree with the FP64 rule on the synthetic workloads'
    points (so ids equal to the FP64 oracle are also the exact answers)."""
    rng = np.random.default_rng(41)
    P = synth.with_islands(rng, synth.tiling(rng, 12, 9, side_median=8.0, side_cap=60, extent=1000.0), 12, 9,
                           hole_frac=0.5, extent=1000.0)
    g = synth.grid(32, extent=1000.0)
    # points within a few ulps of edges: on the chord between consecutive vertices
    v = P.verts
    i = rng.integers(0, len(v) - 1, 20000)
    t = rng.uniform(0.0, 1.0, len(i))
    pe = v[i] + t[:, None] * (v[i + 1] - v[i])
    pe = pe[(pe >= 0.0).all(1) & (pe < 1000.0).all(1)]
    with oracle.exact_predicates():
        ids_x, nh = oracle.pip_join(g, pe, P.verts, P.ring_off, P.poly_ring_off, with_hits=True)
    np.testing.assert_array_equal(nh, 1)
    ids_f = oracle.pip_join(g, pe, P.verts, P.ring_off, P.poly_ring_off)
    assert (ids_x != ids_f).sum() > 0            # the two rules differ on some edge points
    w = synth.pip_tiles(n_points=200_000, layer=3)
    Q = w.polygons
    with oracle.exact_predicates():
        ex = oracle.pip_join(w.grid, w.points, Q.verts, Q.ring_off, Q.poly_ring_off)
    np.testing.assert_array_equal(ex, oracle.pip_join(w.grid, w.points, Q.verts, Q.ring_off, Q.poly_ring_off))
