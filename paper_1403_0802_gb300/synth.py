"""Seeded synthetic workloads shaped like the paper's data sets.

The paper joins taxi pick-ups against street polylines (P2P, Sec. IV.A) and
species occurrences against ecoregion polygons (PIP, Sec. IV.A).  Those data
sets are not available here, so these generators produce inputs with the same
structure: clustered point clouds, short random-walk polylines, and disjoint
polygon tilings with uneven vertex counts.

This module holds no arithmetic of the join itself (no cell ids, no
crossing tests, no distances).  Both the CUDA path and the CPU oracle consume
its arrays; neither imports the other.

Layer formats (all numpy, C-contiguous):
  points         float64 [N, 2]          (x, y) in metres
  polygon layer  verts float64 [V, 2], ring_off int64 [R + 1],
                 poly_ring_off int64 [P + 1]; ring r owns vertices
                 ring_off[r] .. ring_off[r + 1] - 1 (implicitly closed),
                 polygon p owns rings poly_ring_off[p] .. poly_ring_off[p + 1] - 1
  polyline layer verts float64 [V, 2], line_off int64 [L + 1]
  grid           dict(x0, y0, x1, y1, nx, ny)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

EXTENT = 100_000.0          # metres; every workload lives on [0, EXTENT]^2
SEED_BASE = 20140304        # seed of workload k is SEED_BASE + k


def grid(nx: int, ny: int | None = None, extent: float = EXTENT) -> dict:
    ny = nx if ny is None else ny
    return dict(x0=0.0, y0=0.0, x1=float(extent), y1=float(extent), nx=int(nx), ny=int(ny))


# --------------------------------------------------------------------------- points

def points_uniform(n: int, rng: np.random.Generator, extent: float = EXTENT) -> np.ndarray:
    """Uniform points on [0, extent)^2."""
    return np.ascontiguousarray(rng.uniform(0.0, extent, size=(n, 2)))


def points_mixture(n: int, rng: np.random.Generator, n_centres: int = 64,
                   sigma_frac: float = 0.02, uniform_frac: float = 0.2,
                   extent: float = EXTENT) -> np.ndarray:
    """Clustered GPS-like points: a Gaussian mixture plus a uniform background.

    (1 - uniform_frac) of the points come from n_centres isotropic Gaussians
    (centres uniform on the extent, sigma = sigma_frac * extent); samples that
    fall outside [0, extent)^2 are redrawn.  The rest are uniform.
    """
    sigma = sigma_frac * extent
    centres = rng.uniform(0.0, extent, size=(n_centres, 2))
    n_mix = int(round(n * (1.0 - uniform_frac)))
    out = np.empty((n, 2), dtype=np.float64)
    which = rng.integers(0, n_centres, size=n_mix)
    pts = centres[which] + rng.normal(0.0, sigma, size=(n_mix, 2))
    bad = np.flatnonzero((pts < 0.0).any(1) | (pts >= extent).any(1))
    while bad.size:
        pts[bad] = centres[which[bad]] + rng.normal(0.0, sigma, size=(bad.size, 2))
        sub = pts[bad]
        bad = bad[(sub < 0.0).any(1) | (sub >= extent).any(1)]
    out[:n_mix] = pts
    out[n_mix:] = rng.uniform(0.0, extent, size=(n - n_mix, 2))
    perm = rng.permutation(n)
    return np.ascontiguousarray(out[perm])


# --------------------------------------------------------------------------- polygons

@dataclass
class PolygonLayer:
    verts: np.ndarray
    ring_off: np.ndarray
    poly_ring_off: np.ndarray

    @property
    def n_polygons(self) -> int:
        return len(self.poly_ring_off) - 1

    @property
    def n_rings(self) -> int:
        return len(self.ring_off) - 1

    def ring_sizes(self) -> np.ndarray:
        return np.diff(self.ring_off)

    def polygon_sizes(self) -> np.ndarray:
        return np.diff(self.ring_off[self.poly_ring_off])


@dataclass
class PolylineLayer:
    verts: np.ndarray
    line_off: np.ndarray

    @property
    def n_lines(self) -> int:
        return len(self.line_off) - 1

    def line_sizes(self) -> np.ndarray:
        return np.diff(self.line_off)


def _sorted_angles(n: int, rng: np.random.Generator) -> np.ndarray:
    """n distinct sorted angles in [0, 2pi) whose largest circular gap is < pi.

    The gap rule keeps the centre inside the kernel of the polygon, so the
    polygon built from these angles is star-shaped and therefore simple.
    """
    while True:
        a = np.sort(rng.uniform(0.0, 2.0 * math.pi, size=n))
        gaps = np.diff(np.concatenate([a, [a[0] + 2.0 * math.pi]]))
        if np.all(gaps > 0.0) and gaps.max() < math.pi:
            return a


def star_polygons(rng: np.random.Generator, n_side: int = 32, extent: float = EXTENT,
                  nmin: int = 8, nmax: int = 64, jitter: float = 0.05,
                  rmin: float = 0.25, rmax: float = 0.45) -> PolygonLayer:
    """One star-shaped polygon per cell of an n_side x n_side lattice.

    Polygon id = row * n_side + col (row along y).  Centre = lattice-cell centre
    jittered by U(-jitter, jitter) * s per axis; n ~ U{nmin..nmax} vertices at
    sorted uniform angles with radius U(rmin, rmax) * s.  With jitter + rmax <=
    0.5 every polygon stays inside its own lattice cell, so the layer is
    disjoint.
    """
    s = extent / n_side
    verts, sizes = [], []
    for row in range(n_side):
        for col in range(n_side):
            cx = (col + 0.5) * s + rng.uniform(-jitter, jitter) * s
            cy = (row + 0.5) * s + rng.uniform(-jitter, jitter) * s
            n = int(rng.integers(nmin, nmax + 1))
            ang = _sorted_angles(n, rng)
            r = rng.uniform(rmin, rmax, size=n) * s
            verts.append(np.stack([cx + r * np.cos(ang), cy + r * np.sin(ang)], 1))
            sizes.append(n)
    v = np.ascontiguousarray(np.concatenate(verts))
    ring_off = np.zeros(len(sizes) + 1, np.int64)
    ring_off[1:] = np.cumsum(sizes)
    return PolygonLayer(v, ring_off, np.arange(len(sizes) + 1, dtype=np.int64))


def tiling(rng: np.random.Generator, nx: int, ny: int, side_median: float, side_sigma: float = 1.0,
           side_cap: int = 1250, extent: float = EXTENT, corner_jitter: float = 0.1,
           bulge: float = 0.1, n_giant: int = 0) -> PolygonLayer:
    """Disjoint polygons tiling [0, extent]^2 exactly, with heavy-tailed vertex counts.

    Corners of an nx x ny lattice are jittered by U(-corner_jitter, corner_jitter)
    cells (boundary corners only along the boundary).  Every lattice side gets
    k ~ round(lognormal(ln side_median, side_sigma)) interior points, k <= side_cap,
    at sorted positions t along its chord, displaced perpendicular to the chord by
    U(-1, 1) * bulge * cell * sin(pi t) (sides on the extent boundary stay straight).
    Each side is a graph over its chord that vanishes at the corners, so tiles are
    simple; neighbouring tiles share the identical vertex arrays of a side
    (traversed in opposite directions), so the tiling has no gaps or overlaps.
    The n_giant tiles drawn at random get side_cap points on all four sides, so
    the vertex-count tail reaches about 4 * side_cap.  Polygon id = row * nx + col.
    """
    cw, ch = extent / nx, extent / ny
    giant = set(map(tuple, np.stack([rng.integers(0, nx, n_giant), rng.integers(0, ny, n_giant)], 1)))
    giant_h = {(i, j + d) for i, j in giant for d in (0, 1)}
    giant_v = {(i + d, j) for i, j in giant for d in (0, 1)}
    P = np.zeros((nx + 1, ny + 1, 2))
    gx, gy = np.meshgrid(np.arange(nx + 1) * cw, np.arange(ny + 1) * ch, indexing="ij")
    jx = rng.uniform(-corner_jitter, corner_jitter, gx.shape) * cw
    jy = rng.uniform(-corner_jitter, corner_jitter, gy.shape) * ch
    jx[0, :] = jx[-1, :] = 0.0
    jy[:, 0] = jy[:, -1] = 0.0
    P[..., 0] = gx + jx
    P[..., 1] = gy + jy
    scale = min(cw, ch)

    def side(a, b, on_boundary, big=False):
        k = side_cap if big else int(min(side_cap, max(0, round(rng.lognormal(math.log(side_median), side_sigma)))))
        if k == 0:
            return np.zeros((0, 2))
        t = np.sort(rng.uniform(0.0, 1.0, k))
        t = np.unique(t)
        d = b - a
        nrm = np.array([-d[1], d[0]]) / np.hypot(*d)
        off = np.zeros(len(t)) if on_boundary else rng.uniform(-1.0, 1.0, len(t)) * bulge * scale * np.sin(np.pi * t)
        return a + t[:, None] * d + off[:, None] * nrm

    hside = {(i, j): side(P[i, j], P[i + 1, j], j in (0, ny), (i, j) in giant_h)
             for i in range(nx) for j in range(ny + 1)}
    vside = {(i, j): side(P[i, j], P[i, j + 1], i in (0, nx), (i, j) in giant_v)
             for i in range(nx + 1) for j in range(ny)}
    verts, sizes = [], []
    for j in range(ny):
        for i in range(nx):
            ring = [P[i, j][None], hside[i, j], P[i + 1, j][None], vside[i + 1, j],
                    P[i + 1, j + 1][None], hside[i, j + 1][::-1], P[i, j + 1][None], vside[i, j][::-1]]
            r = np.concatenate(ring)
            verts.append(r)
            sizes.append(len(r))
    v = np.ascontiguousarray(np.concatenate(verts))
    ring_off = np.zeros(len(sizes) + 1, np.int64)
    ring_off[1:] = np.cumsum(sizes)
    return PolygonLayer(v, ring_off, np.arange(len(sizes) + 1, dtype=np.int64))


def with_islands(rng: np.random.Generator, tiles: PolygonLayer, nx: int, ny: int, hole_frac: float = 0.3,
                 max_holes: int = 4, hole_median: float = 12.0, hole_sigma: float = 0.8, hole_cap: int = 400,
                 extent: float = EXTENT) -> PolygonLayer:
    """Multi-ring version of an nx x ny tiling (WWF-like enclaves): a fraction
    hole_frac of the tiles get 1..max_holes holes, and each hole is also the
    single ring of a new "island" polygon, so the layer still tiles the extent
    without gaps or overlaps.  Holes are star-shaped (sorted angles, largest gap
    below pi) with k = clamp(round(lognormal(ln hole_median, hole_sigma)), 4,
    hole_cap) vertices, one per quarter of the tile's lattice cell, centred at
    (0.375 or 0.625) +- 0.02 cells with radius U(0.05, 0.10) cells: inside
    [0.25, 0.75]^2 of the cell, which the jittered and bulged tile sides
    (at most 0.2 cells from the lattice lines) never reach, and disjoint.
    Polygon ids: tiles keep row * nx + col; islands follow in tile order."""
    cw, ch = extent / nx, extent / ny
    n_tiles = tiles.n_polygons
    verts = [tiles.verts]
    ring_sizes = [tiles.ring_sizes()]
    tile_rings = np.ones(n_tiles, np.int64)        # rings per tile polygon (outer + holes)
    holes = []                                      # (tile, ring vertices) in tile order
    quarters = np.array([(0.375, 0.375), (0.625, 0.375), (0.375, 0.625), (0.625, 0.625)])
    chosen = np.flatnonzero(rng.random(n_tiles) < hole_frac)
    for t in chosen:
        col, row = t % nx, t // nx
        nh = int(rng.integers(1, max_holes + 1))
        for q in rng.permutation(4)[:nh]:
            cx = (col + quarters[q, 0] + rng.uniform(-0.02, 0.02)) * cw
            cy = (row + quarters[q, 1] + rng.uniform(-0.02, 0.02)) * ch
            k = int(min(hole_cap, max(4, round(rng.lognormal(math.log(hole_median), hole_sigma)))))
            ang = _sorted_angles(k, rng)
            r = rng.uniform(0.05, 0.10, size=k)
            holes.append((int(t), np.stack([cx + r * cw * np.cos(ang), cy + r * ch * np.sin(ang)], 1)))
        tile_rings[t] += nh
    # rings in polygon order: each tile's outer ring then its holes, then the islands
    by_tile: dict[int, list[np.ndarray]] = {}
    for t, h in holes:
        by_tile.setdefault(t, []).append(h)
    rings = []
    off = tiles.ring_off
    for t in range(n_tiles):
        rings.append(tiles.verts[off[t]:off[t + 1]])
        rings.extend(by_tile.get(t, ()))
    island_rings = [h for t in sorted(by_tile) for h in by_tile[t]]
    rings.extend(island_rings)
    sizes = np.array([len(r) for r in rings], np.int64)
    ring_off = np.zeros(len(rings) + 1, np.int64)
    ring_off[1:] = np.cumsum(sizes)
    rings_per_poly = np.concatenate([tile_rings, np.ones(len(island_rings), np.int64)])
    poly_ring_off = np.zeros(len(rings_per_poly) + 1, np.int64)
    poly_ring_off[1:] = np.cumsum(rings_per_poly)
    del verts, ring_sizes
    return PolygonLayer(np.ascontiguousarray(np.concatenate(rings)), ring_off, poly_ring_off)


# --------------------------------------------------------------------------- polylines

def _segmented_cumsum(vals: np.ndarray, starts: np.ndarray) -> np.ndarray:
    cs = np.cumsum(vals)
    base = cs[starts] - vals[starts]
    lens = np.diff(np.append(starts, len(vals)))
    return cs - np.repeat(base, lens)


def random_walks(rng: np.random.Generator, sizes: np.ndarray, extent: float = EXTENT,
                 step_mean: float = 50.0, step_sd: float = 15.0, step_min: float = 1.0,
                 turn_sd: float = math.pi / 6.0) -> PolylineLayer:
    """Street-like polylines as seeded random walks.

    Polyline l has sizes[l] vertices: start uniform on the extent, initial
    heading U[0, 2pi), each later step turns by N(0, turn_sd) and has length
    N(step_mean, step_sd) clipped below at step_min.  Vertices are clamped to
    the closed extent; clamping can create zero-length segments, which are kept.
    """
    sizes = np.asarray(sizes, dtype=np.int64)
    L = len(sizes)
    off = np.zeros(L + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    V = int(off[-1])
    starts = off[:-1]
    first = np.zeros(V, bool)
    first[starts] = True
    turn = rng.normal(0.0, turn_sd, size=V)
    turn[first] = 0.0
    turn[starts[sizes > 1] + 1] = 0.0  # the first step uses the initial heading
    head0 = rng.uniform(0.0, 2.0 * math.pi, size=L)
    heading = np.repeat(head0, sizes) + _segmented_cumsum(turn, starts)
    step = np.maximum(rng.normal(step_mean, step_sd, size=V), step_min)
    step[first] = 0.0
    dx = step * np.cos(heading)
    dy = step * np.sin(heading)
    start = rng.uniform(0.0, extent, size=(L, 2))
    x = np.repeat(start[:, 0], sizes) + _segmented_cumsum(dx, starts)
    y = np.repeat(start[:, 1], sizes) + _segmented_cumsum(dy, starts)
    v = np.stack([np.clip(x, 0.0, extent), np.clip(y, 0.0, extent)], 1)
    return PolylineLayer(np.ascontiguousarray(v), off)


# --------------------------------------------------------------------------- named workloads

@dataclass
class Workload:
    name: str
    kind: str                       # "pip" or "p2p"
    points: np.ndarray
    grid: dict
    polygons: PolygonLayer | None = None
    polylines: PolylineLayer | None = None
    D: float = 0.0
    meta: dict = field(default_factory=dict)


def _count(n: int) -> str:
    """10_000_000 -> "10M", 100_000 -> "100k", 1_500 -> "1500" (workload names)."""
    if n >= 1_000_000 and n % 1_000_000 == 0:
        return f"{n // 1_000_000}M"
    return f"{n // 1000}k" if n >= 1000 and n % 1000 == 0 else str(n)


def _point_rng(rng: np.random.Generator, seed: int, shard: int) -> np.random.Generator:
    """Points of shard 0 continue the layer's generator; shard k > 0 (another
    rank of a weak-scaling run) draws its own points from (seed, k), so every
    rank joins different points against an identical layer."""
    return rng if shard == 0 else np.random.default_rng((seed, shard))


def pip_stars(n_points: int = 1_000_000, seed: int = SEED_BASE + 1, n_side: int = 32,
              grid_n: int = 256, shard: int = 0) -> Workload:
    """PIP, plain FP64 method: uniform points against a jittered lattice of
    1,024 star polygons (8-64 vertices), filter grid 256 x 256."""
    rng = np.random.default_rng(seed)
    layer = star_polygons(rng, n_side=n_side)
    pts = points_uniform(n_points, _point_rng(rng, seed, shard))
    return Workload(f"pip_{_count(n_points)}_stars{n_side * n_side}_grid{grid_n}", "pip", pts, grid(grid_n),
                    polygons=layer)


def p2p_walks(n_points: int = 10_000_000, n_lines: int = 100_000, seed: int = SEED_BASE + 2,
              D: float = 100.0, grid_n: int = 448, shard: int = 0) -> Workload:
    """P2P, plain FP64 method: mixture points against random-walk polylines with
    2-40 vertices, window D = 100 m, filter grid 448 x 448 (the fastest of
    384..768 per axis on GB300 with the current kernels: 0.796 ms per join
    against 0.820 at 512)."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(2, 41, size=n_lines)
    layer = random_walks(rng, sizes)
    pts = points_mixture(n_points, _point_rng(rng, seed, shard))
    return Workload(f"p2p_{_count(n_points)}_walks{_count(n_lines)}_D{int(D)}_grid{grid_n}", "p2p", pts,
                    grid(grid_n), polylines=layer, D=float(D))


def pip_tiles(n_points: int = 100_000_000, layer: int = 1, seed: int = SEED_BASE + 3,
              grid_n: int | None = None, shard: int = 0) -> Workload:
    """PIP at scale: clustered points against a disjoint tiling.  Layer 1: 200 x 200
    tiles, side counts lognormal(median 2.6, sigma 1) capped at 1,250, three giant
    tiles (polygon median ~19, max ~5,000).  Layer 2: 140 x 100 tiles, side median
    90, cap 25,000, three giant tiles (polygon median ~500, max ~100,000).  Layer 3
    (multi-ring, WWF-like): layer 1's tiling with island holes in 30 % of the
    tiles (with_islands), about 70,000 polygons.  Filter grid per layer: the
    fastest of 768..1536 per axis at 100 M points on GB300 -- 1536 x 1536 for
    layers 1 and 2 (layer 2: 5.3 ms per join against 6.5 at 1024), 1280 x 1280
    for layer 3."""
    if grid_n is None:
        grid_n = {1: 1536, 2: 1536, 3: 1280}[layer]
    rng = np.random.default_rng(seed + 10 * layer)
    if layer == 1:
        P = tiling(rng, 200, 200, side_median=2.6, side_cap=1250, n_giant=3)
    elif layer == 3:
        P = with_islands(rng, tiling(np.random.default_rng(seed + 10), 200, 200, side_median=2.6, side_cap=1250,
                                     n_giant=3), 200, 200)
    else:
        P = tiling(rng, 140, 100, side_median=90.0, side_cap=25000, n_giant=3)
    pts = points_mixture(n_points, _point_rng(np.random.default_rng(seed), seed, shard))
    return Workload(f"pip_{_count(n_points)}_tiles{P.n_polygons}_L{layer}_grid{grid_n}", "pip", pts, grid(grid_n), polygons=P)


def p2p_walks_lognormal(n_points: int = 170_000_000, n_lines: int = 150_000,
                        seed: int = SEED_BASE + 4, D: float = 100.0,
                        grid_n: int = 512, shard: int = 0) -> Workload:
    """P2P at scale: mixture points against random walks whose vertex counts are
    clamp(round(lognormal(ln 8, 0.8)), 2, 200); filter grid 512 x 512 (faster
    than 1024 x 1024 on GB300 with per-cell segment lists)."""
    rng = np.random.default_rng(seed)
    sizes = np.clip(np.round(rng.lognormal(math.log(8.0), 0.8, size=n_lines)), 2, 200).astype(np.int64)
    layer = random_walks(rng, sizes)
    pts = points_mixture(n_points, _point_rng(rng, seed, shard))
    return Workload(f"p2p_{_count(n_points)}_walks{_count(n_lines)}_D{int(D)}_grid{grid_n}", "p2p", pts,
                    grid(grid_n), polylines=layer, D=float(D))
