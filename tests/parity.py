"""Parity against the CPU oracle, shared by the GPU tests (P2P bar below;
PIP ids are bit-exact).

The bar (Sec. III.B: the nearest polyline within the window, ties to the
smaller id):
  * ids equal the oracle's, except where the oracle's best and second-best
    distances differ by at most 1e-9 relative (either id is then right), or
    where the best distance lies within 1e-9 of the window (inside or outside
    is then decided by rounding);
  * a miss has distance +inf;
  * FP64 distances within 1e-12 * max(d, 1 m) of the oracle's;
  * FP32X distances within the per-point bound the kernel certifies: 64 u
    (u = 2^-24) times the largest |coordinate - cell corner| among the point
    and the MBB corners of its cell's candidates (the lists built for the
    layer's D, which is what the kernel stages), plus 1e-9 m.

P2PRef and PIPRef cache the oracle's MBBs and candidate lists of one layer,
so that many requests against the same layer are checked without rebuilding
them.
"""
from __future__ import annotations

import numpy as np

U = 2.0 ** -24


def tie_or_edge(d1, d2, window):
    """Points whose oracle answer is not unique: a near-tie of the two best
    polylines, or a best distance within 1e-9 of the window."""
    with np.errstate(invalid="ignore"):
        tie = (d2 - d1) <= 1e-9 * np.maximum(d1, 1.0)
    edge = np.abs(d1 - window) <= 1e-9 * max(window, 1.0)
    return tie | edge


class P2PRef:
    def __init__(self, oracle, grid, verts, line_off, D_layer):
        self.o = oracle
        self.grid = grid
        self.verts = np.ascontiguousarray(verts, np.float64)
        self.line_off = np.ascontiguousarray(line_off, np.int64)
        self.D = float(D_layer)
        self.mbb = oracle.p2p_mbb(grid, self.verts, self.line_off)
        self._csr = {}
        self._box = None

    def csr(self, R):
        R = float(R)
        if R not in self._csr:
            self._csr[R] = self.o.cand_csr(self.grid, self.mbb, R, expand=True)
        return self._csr[R]

    def join(self, pts, window=None):
        """Oracle (id, d, best, second best) at `window` (None: the layer's D)."""
        R = self.D if window is None else float(window)
        cs, ci = self.csr(R)
        return self.o.p2p_grid(self.grid, np.ascontiguousarray(pts, np.float64), self.verts, self.line_off, R, cs,
                               ci)

    def _cell_boxes(self):
        if self._box is None:
            g = self.grid
            G = g["nx"] * g["ny"]
            cs, ci = self.csr(self.D)
            counts = np.diff(cs)
            xlo = np.full(G, np.inf); xhi = np.full(G, -np.inf)
            ylo = np.full(G, np.inf); yhi = np.full(G, -np.inf)
            if len(ci):
                ne = np.flatnonzero(counts > 0)
                starts = cs[:-1][ne]
                xlo[ne] = np.minimum.reduceat(self.mbb[ci, 0], starts)
                xhi[ne] = np.maximum.reduceat(self.mbb[ci, 2], starts)
                ylo[ne] = np.minimum.reduceat(self.mbb[ci, 1], starts)
                yhi[ne] = np.maximum.reduceat(self.mbb[ci, 3], starts)
            self._box = (xlo, xhi, ylo, yhi)
        return self._box

    def fp32x_bound(self, pts):
        g = self.grid
        pts = np.asarray(pts, np.float64)
        cells = self.o.point_cells(g, pts)
        G = g["nx"] * g["ny"]
        cw = (g["x1"] - g["x0"]) / g["nx"]
        ch = (g["y1"] - g["y0"]) / g["ny"]
        c = np.where(cells < G, cells, 0)
        ox = g["x0"] + (c % g["nx"]) * cw
        oy = g["y0"] + (c // g["nx"]) * ch
        xlo, xhi, ylo, yhi = self._cell_boxes()
        with np.errstate(invalid="ignore"):
            m = np.maximum.reduce([np.abs(pts[:, 0] - ox), np.abs(pts[:, 1] - oy), np.abs(xlo[c] - ox),
                                   np.abs(xhi[c] - ox), np.abs(ylo[c] - oy), np.abs(yhi[c] - oy)])
        m = np.where(np.isfinite(m), m, 0.0)
        return 64.0 * U * m * 1.0001 + 1e-9

    def check(self, pts, gid, gd, form, window=None, ref=None):
        """Assert the bar above for the GPU results (gid, gd) of `pts` at
        `window`; returns the hit fraction, the largest absolute and relative
        distance errors and the counts of exempt points."""
        pts = np.asarray(pts, np.float64)
        gid = np.asarray(gid)
        gd = np.asarray(gd)
        W = self.D if window is None else float(window)
        rid, rd, d1, d2 = self.join(pts, window) if ref is None else ref
        exempt = tie_or_edge(d1, d2, W)
        bad = np.flatnonzero((gid != rid) & ~exempt)
        assert bad.size == 0, (form, W, bad[:5], gid[bad[:5]], rid[bad[:5]], gd[bad[:5]], rd[bad[:5]])
        assert np.all(np.isinf(gd[gid < 0])), (form, W)
        assert np.all(gd[gid >= 0] <= W), (form, W)
        both = (gid >= 0) & (rid >= 0)
        err = np.abs(gd[both] - rd[both])
        if form == "fp64":
            lim = 1e-12 * np.maximum(rd[both], 1.0)
        else:
            lim = self.fp32x_bound(pts)[both]
        worst = np.flatnonzero(err > lim)
        assert worst.size == 0, (form, W, err[worst[:5]], lim[worst[:5]])
        rel = err / np.maximum(rd[both], 1.0)
        return {"hit_frac": float((gid >= 0).mean()) if gid.size else 0.0,
                "max_abs_err": float(err.max()) if err.size else 0.0,
                "max_rel_err": float(rel.max()) if rel.size else 0.0,
                "exempt": int(exempt.sum()), "n": int(gid.size)}

    def unique(self, pts, window=None, ref=None):
        """Mask of the points whose oracle id is unique (no near-tie, not at
        the window's edge): any two correct results agree on their ids there."""
        W = self.D if window is None else float(window)
        rid, rd, d1, d2 = self.join(pts, window) if ref is None else ref
        return ~tie_or_edge(d1, d2, W)


class PIPRef:
    """Oracle PIP ids (Sec. III.C) for one polygon layer, its candidate lists
    built once."""

    def __init__(self, oracle, grid, verts, ring_off, poly_ring_off):
        self.o = oracle
        self.grid = grid
        self.args = (np.ascontiguousarray(verts, np.float64), np.ascontiguousarray(ring_off, np.int64),
                     np.ascontiguousarray(poly_ring_off, np.int64))
        self.cs, self.ci = oracle.cand_csr(grid, oracle.pip_mbb(grid, *self.args))

    def join(self, pts):
        return self.o.pip_grid(self.grid, np.ascontiguousarray(pts, np.float64), *self.args, self.cs, self.ci)
