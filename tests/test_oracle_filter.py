"""Pins of the oracle's grid filter (Sec. III.A): cell ids against exact
rational floors, candidate lists against exact rectangle intersection, and
completeness (no true hit is ever filtered out)."""
import math
from fractions import Fraction

import numpy as np

from paper_1403_0802_gb300 import synth

GD = dict(x0=-512.0, y0=-256.0, x1=512.0, y1=768.0, nx=64, ny=32)   # dyadic: cw = 16, ch = 32


def exact_cell(g, x, y):
    G = g["nx"] * g["ny"]
    if not (math.isfinite(x) and math.isfinite(y)):
        return G
    cw = (Fraction(g["x1"]) - Fraction(g["x0"])) / g["nx"]
    ch = (Fraction(g["y1"]) - Fraction(g["y0"])) / g["ny"]
    ix = math.floor((Fraction(x) - Fraction(g["x0"])) / cw)
    iy = math.floor((Fraction(y) - Fraction(g["y0"])) / ch)
    if 0 <= ix < g["nx"] and 0 <= iy < g["ny"]:
        return iy * g["nx"] + ix
    return G


def test_cell_ids_match_exact_floor(oracle):
    rng = np.random.default_rng(1)
    pts = np.round(rng.uniform(-600, 800, size=(20000, 2)) * 8) / 8        # many on cell boundaries
    edge = np.array([[-512, -256], [511.875, 767.9], [512, 0], [0, 768], [-512.125, 0], [np.nan, 0],
                     [0, np.inf], [16, 32], [15.999, 31.999]])
    pts = np.concatenate([pts, edge])
    got = oracle.point_cells(GD, pts)
    ref = np.array([exact_cell(GD, x, y) for x, y in pts])
    np.testing.assert_array_equal(got, ref)
    counts = oracle.cell_counts(GD, pts)
    assert counts.sum() == len(pts)
    np.testing.assert_array_equal(counts, np.bincount(ref, minlength=GD["nx"] * GD["ny"] + 1))


def test_cell_ids_monotone_on_decimal_grid(oracle):
    g = synth.grid(1024)
    x = np.sort(np.random.default_rng(3).uniform(0, 1e5, 200000))
    pts = np.stack([x, np.full_like(x, 5.0)], 1)
    c = oracle.point_cells(g, pts)
    assert (np.diff(c) >= 0).all()
    ix = c % 1024
    cw = 1e5 / 1024
    assert (np.abs(x - (ix + 0.5) * cw) <= 0.5 * cw * (1 + 1e-9)).all()


def exact_cells_of_box(g, xlo, ylo, xhi, yhi):
    """Cells whose half-open rectangle meets the closed box, exactly."""
    cw = (g["x1"] - g["x0"]) / g["nx"]
    ch = (g["y1"] - g["y0"]) / g["ny"]
    out = set()
    for iy in range(g["ny"]):
        for ix in range(g["nx"]):
            cx0, cy0 = g["x0"] + ix * cw, g["y0"] + iy * ch
            if cx0 <= xhi and xlo < cx0 + cw and cy0 <= yhi and ylo < cy0 + ch:
                out.add(iy * g["nx"] + ix)
    # cells past the grid edge clamp to the border cells
    return out


def test_candidate_lists_are_exact_rectangle_intersections(oracle):
    rng = np.random.default_rng(8)
    boxes = []
    for _ in range(60):
        x0 = np.round(rng.uniform(-512, 400) * 4) / 4
        y0 = np.round(rng.uniform(-256, 650) * 4) / 4
        w, h = np.round(rng.uniform(0, 120, 2) * 4) / 4
        boxes.append((x0, y0, min(x0 + w, 512.0), min(y0 + h, 768.0)))
    boxes += [(-512, -256, -512, -256), (512, 768, 512, 768), (0, 0, 16, 32), (-512, -256, 512, 768)]
    mbb = np.array(boxes, np.float64)
    start, ids = oracle.cand_csr(GD, mbb)
    got = {}
    for c in range(len(start) - 1):
        for k in range(start[c], start[c + 1]):
            got.setdefault(int(ids[k]), set()).add(c)
        assert (np.diff(ids[start[c]:start[c + 1]]) > 0).all()       # sorted, no duplicates
    for o, (a, b, c_, d) in enumerate(boxes):
        ref = exact_cells_of_box(GD, a, b, c_, d)
        if not ref:   # a box on the far grid edge clamps to the border cell
            ref = {min(int((b - GD["y0"]) // 32), 31) * 64 + min(int((a - GD["x0"]) // 16), 63)}
        assert got.get(o, set()) == ref, o


def test_expanded_candidate_lists_bracket_exact_window(oracle):
    rng = np.random.default_rng(12)
    R = 20.0
    mbb = []
    for _ in range(40):
        x0 = np.round(rng.uniform(-480, 400) * 4) / 4
        y0 = np.round(rng.uniform(-220, 650) * 4) / 4
        w, h = np.round(rng.uniform(0, 60, 2) * 4) / 4
        mbb.append((x0, y0, x0 + w, y0 + h))
    mbb = np.array(mbb)
    start, ids = oracle.cand_csr(GD, mbb, R, expand=True)
    for o, (a, b, c, d) in enumerate(mbb):
        cells = {cc for cc in range(len(start) - 1) if o in ids[start[cc]:start[cc + 1]]}
        inner = exact_cells_of_box(GD, a - R, b - R, c + R, d + R)
        outer = exact_cells_of_box(GD, a - R - 1e-6, b - R - 1e-6, c + R + 1e-6, d + R + 1e-6)
        assert inner <= cells <= outer, o


def test_filter_is_complete_for_pip_and_p2p(oracle):
    w = synth.pip_stars(n_points=20000)
    L = w.polygons
    mbb = oracle.pip_mbb(w.grid, L.verts, L.ring_off, L.poly_ring_off)
    cs, ci = oracle.cand_csr(w.grid, mbb)
    ids = oracle.pip_brute(w.grid, w.points, L.verts, L.ring_off, L.poly_ring_off)
    cells = oracle.point_cells(w.grid, w.points)
    for i in np.flatnonzero(ids >= 0):
        assert ids[i] in ci[cs[cells[i]]:cs[cells[i] + 1]]
    w = synth.p2p_walks(n_points=2000, n_lines=5000)
    L = w.polylines
    mbb = oracle.p2p_mbb(w.grid, L.verts, L.line_off)
    cs, ci = oracle.cand_csr(w.grid, mbb, w.D, expand=True)
    oid, od, _, _ = oracle.p2p_brute(w.grid, w.points, L.verts, L.line_off, w.D)
    cells = oracle.point_cells(w.grid, w.points)
    assert (oid >= 0).sum() > 100
    for i in np.flatnonzero(oid >= 0):
        assert oid[i] in ci[cs[cells[i]]:cs[cells[i] + 1]]
