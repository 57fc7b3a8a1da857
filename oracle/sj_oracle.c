/*
 * sj_oracle.c -- plain, slow, obviously-correct CPU oracle for the grid-filtered
 * spatial join of Zhang & You, "Large-Scale Geospatial Processing on Multi-Core
 * and Many-Core Processors" (arXiv 1403.0802).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header or constant with the CUDA path.
 *
 * Build: gcc -O2 -ffp-contract=off (no fast-math) so that every FP64 operation
 * below is a single IEEE round-to-nearest operation in source order.
 *
 * What it computes:
 *   - cell of a point on a uniform grid                         (Sec. III.A, Fig. 1)
 *   - minimum bounding box (MBB) per polygon / polyline          (Sec. III.A)
 *   - rasterisation of MBBs (expanded by R for P2P) to cells,
 *     giving per-cell candidate lists                             (Sec. III.A)
 *   - point-to-segment distance, two cases                       (Sec. III.B, Fig. 2)
 *   - nearest polyline within the window R                       (Sec. II, Sec. III.B)
 *   - ray-crossing point-in-polygon test, rings with holes       (Sec. III.C, Fig. 3)
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - cell: ix = floor((x - x0) / cw) with cw = (x1 - x0) / nx; a point is in the
 *     join domain iff 0 <= ix < nx and 0 <= iy < ny (half-open grid box).
 *   - crossing rule: edge (a, b) straddles p iff (a.y > p.y) != (b.y > p.y);
 *     with lo = the endpoint whose y <= p.y and hi = the other,
 *     d = (hi.x - lo.x) * (p.y - lo.y) - (hi.y - lo.y) * (p.x - lo.x) and the
 *     edge counts iff d > 0.  Inside iff the count over all rings is odd.
 *     d's sign is taken from its FP64 evaluation (the default, the method's
 *     arithmetic) or, in the exact-predicate mode (or_set_exact(1)), from the
 *     exact value of d for the given doubles (Shewchuk's adaptive orientation
 *     predicate: an FP64 filter, then error-free expansion arithmetic).
 *   - a point inside several polygons gets the smallest id.
 *   - P2P window is inclusive (d <= R); exact distance ties go to the smaller id.
 *   - the P2P cell range uses lo = nextafter(xmin - R, -inf),
 *     hi = nextafter(xmax + R, +inf) so that rounding never drops a cell.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double x0, y0, x1, y1;
    int32_t nx, ny;
} or_grid;

enum { OR_OK = 0, OR_INVALID = -1, OR_OOM = -2, OR_GRID_COVER = -3 };

static int g_threads = 1;

void or_set_threads(int n) { g_threads = n > 0 ? n : 1; }

int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_num_procs();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ grid (Sec. III.A) */

static int grid_ok(const or_grid *g) {
    if (!(g->nx >= 1 && g->ny >= 1)) return 0;
    if ((int64_t)g->nx * (int64_t)g->ny > 2147483646LL) return 0;
    if (!(isfinite(g->x0) && isfinite(g->x1) && isfinite(g->y0) && isfinite(g->y1))) return 0;
    if (!(g->x1 > g->x0 && g->y1 > g->y0)) return 0;
    return 1;
}

static double cell_w(const or_grid *g) { return (g->x1 - g->x0) / (double)g->nx; }
static double cell_h(const or_grid *g) { return (g->y1 - g->y0) / (double)g->ny; }

/* Cell id of one point; G = nx * ny for points outside the half-open grid box
 * (NaN coordinates included). */
int64_t or_point_cell(const or_grid *g, double x, double y) {
    int64_t G = (int64_t)g->nx * (int64_t)g->ny;
    double tx = (x - g->x0) / cell_w(g);
    double ty = (y - g->y0) / cell_h(g);
    if (!(tx >= 0.0 && tx < (double)g->nx)) return G;
    if (!(ty >= 0.0 && ty < (double)g->ny)) return G;
    int64_t ix = (int64_t)floor(tx);
    int64_t iy = (int64_t)floor(ty);
    return iy * (int64_t)g->nx + ix;
}

void or_point_cells(const or_grid *g, const double *pts, int64_t n, int64_t *cid) {
    for (int64_t i = 0; i < n; ++i) cid[i] = or_point_cell(g, pts[2 * i], pts[2 * i + 1]);
}

/* Number of points per cell; counts has G + 1 entries, the last one counts the
 * points outside the grid.  Sorting points by cell (VGC/VGI of Fig. 1) is the
 * exclusive prefix sum of these counts. */
int or_cell_counts(const or_grid *g, const double *pts, int64_t n, int64_t *counts) {
    if (!grid_ok(g)) return OR_INVALID;
    int64_t G = (int64_t)g->nx * (int64_t)g->ny;
    memset(counts, 0, (size_t)(G + 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) counts[or_point_cell(g, pts[2 * i], pts[2 * i + 1])] += 1;
    return OR_OK;
}

/* floor((v - lo) / w) clamped to [0, n - 1]. */
static int32_t clamped_cell(double v, double lo, double w, int32_t n) {
    double f = floor((v - lo) / w);
    if (!(f >= 0.0)) return 0;
    if (f > (double)(n - 1)) return n - 1;
    return (int32_t)f;
}

/* ------------------------------------------------------------------ layers */

static int check_finite(const double *v, int64_t nv) {
    for (int64_t i = 0; i < 2 * nv; ++i)
        if (!isfinite(v[i])) return 0;
    return 1;
}

/* MBB of vertices [b, e) -> out[4] = (xmin, ymin, xmax, ymax). */
static void range_mbb(const double *v, int64_t b, int64_t e, double *out) {
    double xmin = v[2 * b], xmax = v[2 * b], ymin = v[2 * b + 1], ymax = v[2 * b + 1];
    for (int64_t i = b + 1; i < e; ++i) {
        double x = v[2 * i], y = v[2 * i + 1];
        if (x < xmin) xmin = x;
        if (x > xmax) xmax = x;
        if (y < ymin) ymin = y;
        if (y > ymax) ymax = y;
    }
    out[0] = xmin; out[1] = ymin; out[2] = xmax; out[3] = ymax;
}

static int mbb_covered(const or_grid *g, const double *m) {
    return m[0] >= g->x0 && m[2] <= g->x1 && m[1] >= g->y0 && m[3] <= g->y1;
}

/* Validate a polygon layer and compute its MBBs (Sec. III.A).  Rings need at
 * least 3 vertices, polygons at least one ring, every coordinate finite, and
 * every MBB inside the closed grid box. */
int or_pip_mbb(const or_grid *g, const double *verts, int64_t V, const int64_t *ring_off, int64_t R,
               const int64_t *poly_ring_off, int32_t P, double *mbb) {
    if (!grid_ok(g) || V < 0 || R < 0 || P < 0) return OR_INVALID;
    if (ring_off[0] != 0 || ring_off[R] != V || poly_ring_off[0] != 0 || poly_ring_off[P] != R)
        return OR_INVALID;
    for (int64_t r = 0; r < R; ++r)
        if (ring_off[r + 1] - ring_off[r] < 3) return OR_INVALID;
    for (int32_t p = 0; p < P; ++p)
        if (poly_ring_off[p + 1] - poly_ring_off[p] < 1) return OR_INVALID;
    if (!check_finite(verts, V)) return OR_INVALID;
    for (int32_t p = 0; p < P; ++p) {
        range_mbb(verts, ring_off[poly_ring_off[p]], ring_off[poly_ring_off[p + 1]], mbb + 4 * p);
        if (!mbb_covered(g, mbb + 4 * p)) return OR_GRID_COVER;
    }
    return OR_OK;
}

/* Same for a polyline layer (each polyline at least one vertex). */
int or_p2p_mbb(const or_grid *g, const double *verts, int64_t V, const int64_t *line_off, int32_t L,
               double *mbb) {
    if (!grid_ok(g) || V < 0 || L < 0) return OR_INVALID;
    if (line_off[0] != 0 || line_off[L] != V) return OR_INVALID;
    for (int32_t l = 0; l < L; ++l)
        if (line_off[l + 1] - line_off[l] < 1) return OR_INVALID;
    if (!check_finite(verts, V)) return OR_INVALID;
    for (int32_t l = 0; l < L; ++l) {
        range_mbb(verts, line_off[l], line_off[l + 1], mbb + 4 * l);
        if (!mbb_covered(g, mbb + 4 * l)) return OR_GRID_COVER;
    }
    return OR_OK;
}

/* Cell index box of one MBB.  For P2P (expand != 0) the MBB is widened by R on
 * every side, rounded outward by one ulp (Sec. III.A, expanded MBB). */
static void mbb_cells(const or_grid *g, const double *m, double R, int expand, int32_t *ix0, int32_t *iy0,
                      int32_t *ix1, int32_t *iy1) {
    double xlo = m[0], ylo = m[1], xhi = m[2], yhi = m[3];
    if (expand) {
        xlo = nextafter(xlo - R, -INFINITY);
        ylo = nextafter(ylo - R, -INFINITY);
        xhi = nextafter(xhi + R, INFINITY);
        yhi = nextafter(yhi + R, INFINITY);
    }
    double cw = cell_w(g), ch = cell_h(g);
    *ix0 = clamped_cell(xlo, g->x0, cw, g->nx);
    *ix1 = clamped_cell(xhi, g->x0, cw, g->nx);
    *iy0 = clamped_cell(ylo, g->y0, ch, g->ny);
    *iy1 = clamped_cell(yhi, g->y0, ch, g->ny);
}

/* Per-cell candidate lists (the VPP relation of Fig. 1) in CSR form:
 * cand_start[G + 1] and, when cand_ids is not NULL, the object ids of each cell
 * in increasing order.  Call once with cand_ids == NULL to size it. */
int or_cand_csr(const or_grid *g, const double *mbb, int32_t nobj, double R, int expand, int64_t *cand_start,
                int32_t *cand_ids) {
    if (!grid_ok(g)) return OR_INVALID;
    int64_t G = (int64_t)g->nx * (int64_t)g->ny;
    memset(cand_start, 0, (size_t)(G + 1) * sizeof(int64_t));
    for (int32_t o = 0; o < nobj; ++o) {
        int32_t ix0, iy0, ix1, iy1;
        mbb_cells(g, mbb + 4 * o, R, expand, &ix0, &iy0, &ix1, &iy1);
        for (int32_t iy = iy0; iy <= iy1; ++iy)
            for (int32_t ix = ix0; ix <= ix1; ++ix) cand_start[(int64_t)iy * g->nx + ix + 1] += 1;
    }
    for (int64_t c = 0; c < G; ++c) cand_start[c + 1] += cand_start[c];
    if (!cand_ids) return OR_OK;
    int64_t *cur = (int64_t *)malloc((size_t)G * sizeof(int64_t));
    if (!cur) return OR_OOM;
    memcpy(cur, cand_start, (size_t)G * sizeof(int64_t));
    for (int32_t o = 0; o < nobj; ++o) {
        int32_t ix0, iy0, ix1, iy1;
        mbb_cells(g, mbb + 4 * o, R, expand, &ix0, &iy0, &ix1, &iy1);
        for (int32_t iy = iy0; iy <= iy1; ++iy)
            for (int32_t ix = ix0; ix <= ix1; ++ix) cand_ids[cur[(int64_t)iy * g->nx + ix]++] = o;
    }
    free(cur);
    return OR_OK;
}

/* ------------------------------------------------------------------ PIP (Sec. III.C) */

/* Exact sign of the crossing determinant, after J. R. Shewchuk, "Adaptive
 * Precision Floating-Point Arithmetic and Fast Robust Geometric Predicates"
 * (Discrete Comput. Geom. 18, 1997).  An expansion is a list of doubles,
 * nonoverlapping and ordered by increasing magnitude, whose exact sum is the
 * value it stands for; its sign is the sign of its largest nonzero
 * component.  Inputs are assumed far from overflow and underflow (true for
 * coordinates of a bounded grid). */
static int g_exact = 0;
void or_set_exact(int on) { g_exact = on ? 1 : 0; }

/* s + t = a + b exactly, s = fl(a + b) (Knuth's two-sum, Shewchuk Thm. 7). */
static void two_sum(double a, double b, double *s, double *t) {
    double x = a + b;
    double bv = x - a;
    double av = x - bv;
    *s = x;
    *t = (a - av) + (b - bv);
}

/* p + t = a * b exactly, p = fl(a * b): the fused multiply-add rounds once,
 * so a * b - p is exact. */
static void two_prod(double a, double b, double *p, double *t) {
    double x = a * b;
    *p = x;
    *t = fma(a, b, -x);
}

/* Add the double b to the expansion h[0..m) in place (Shewchuk's
 * Grow-Expansion, Thm. 10); returns the new length m + 1. */
static int grow(double *h, int m, double b) {
    double q = b;
    for (int i = 0; i < m; ++i) {
        double s, t;
        two_sum(q, h[i], &s, &t);
        h[i] = t;
        q = s;
    }
    h[m] = q;
    return m + 1;
}

/* Exact sign of (hx - lx) * (py - ly) - (hy - ly) * (px - lx). */
static int cross_sign_exact(double hx, double hy, double lx, double ly, double px, double py) {
    double dl = (hx - lx) * (py - ly), dr = (hy - ly) * (px - lx);
    double d = dl - dr;
    /* filter: the FP64 value's error is below (3 eps + 16 eps^2)(|dl| + |dr|),
     * eps = 2^-53 (Shewchuk's bound for this orientation form) */
    const double eps = 1.1102230246251565e-16;
    double bound = (3.0 * eps + 16.0 * eps * eps) * (fabs(dl) + fabs(dr));
    if (d > bound) return 1;
    if (-d > bound) return -1;
    /* each difference as an exact two-term sum, each product of two such sums
     * as four exact two-term products: sixteen doubles summing to d exactly */
    double a[2], b[2], c[2], e[2];
    two_sum(hx, -lx, &a[1], &a[0]);
    two_sum(py, -ly, &b[1], &b[0]);
    two_sum(hy, -ly, &c[1], &c[0]);
    two_sum(px, -lx, &e[1], &e[0]);
    double h[16];
    int m = 0;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double p, t;
            two_prod(a[i], b[j], &p, &t);
            m = grow(h, m, t);
            m = grow(h, m, p);
            two_prod(c[i], e[j], &p, &t);
            m = grow(h, m, -t);
            m = grow(h, m, -p);
        }
    for (int i = m - 1; i >= 0; --i)
        if (h[i] != 0.0) return h[i] > 0.0 ? 1 : -1;
    return 0;
}

/* Exported for tests: the sign the crossing rule takes for d (-1, 0, 1) in the
 * current mode. */
int or_cross_sign(double hx, double hy, double lx, double ly, double px, double py) {
    if (g_exact) return cross_sign_exact(hx, hy, lx, ly, px, py);
    double d = (hx - lx) * (py - ly) - (hy - ly) * (px - lx);
    return (d > 0.0) - (d < 0.0);
}

/* Crossing parity of point p against ring [b, e) (implicitly closed). */
static int ring_parity(double px, double py, const double *v, int64_t b, int64_t e) {
    int odd = 0;
    for (int64_t i = b; i < e; ++i) {
        int64_t j = (i + 1 < e) ? i + 1 : b;
        double ax = v[2 * i], ay = v[2 * i + 1];
        double bx = v[2 * j], by = v[2 * j + 1];
        int a_above = ay > py;
        int b_above = by > py;
        if (a_above == b_above) continue;
        double lx, ly, hx, hy;
        if (a_above) { hx = ax; hy = ay; lx = bx; ly = by; }
        else         { lx = ax; ly = ay; hx = bx; hy = by; }
        if (g_exact) {
            if (cross_sign_exact(hx, hy, lx, ly, px, py) > 0) odd ^= 1;
        } else {
            double d = (hx - lx) * (py - ly) - (hy - ly) * (px - lx);
            if (d > 0.0) odd ^= 1;
        }
    }
    return odd;
}

/* Even-odd rule over all rings of polygon p, so holes need no orientation. */
int or_pip_polygon(double px, double py, const double *verts, const int64_t *ring_off,
                   const int64_t *poly_ring_off, int32_t p) {
    int odd = 0;
    for (int64_t r = poly_ring_off[p]; r < poly_ring_off[p + 1]; ++r)
        odd ^= ring_parity(px, py, verts, ring_off[r], ring_off[r + 1]);
    return odd;
}

/* Brute force: every in-grid point against every polygon; the smallest id
 * containing the point, else -1.  out_nhit (may be NULL) counts the polygons
 * that contain each point. */
int or_pip_brute(const or_grid *g, const double *pts, int64_t n, const double *verts, const int64_t *ring_off,
                 const int64_t *poly_ring_off, int32_t P, int32_t *out_id, int32_t *out_nhit) {
    if (!grid_ok(g)) return OR_INVALID;
    int64_t G = (int64_t)g->nx * (int64_t)g->ny;
#pragma omp parallel for schedule(dynamic, 256) num_threads(g_threads)
    for (int64_t i = 0; i < n; ++i) {
        double px = pts[2 * i], py = pts[2 * i + 1];
        int32_t best = -1, nh = 0;
        if (or_point_cell(g, px, py) != G) {
            for (int32_t p = 0; p < P; ++p)
                if (or_pip_polygon(px, py, verts, ring_off, poly_ring_off, p)) {
                    if (best < 0) best = p;
                    ++nh;
                }
        }
        out_id[i] = best;
        if (out_nhit) out_nhit[i] = nh;
    }
    return OR_OK;
}

/* Grid-filtered: each in-grid point is tested only against the candidates of
 * its cell (cand_ids sorted by id, so the first hit is the smallest id). */
int or_pip_grid(const or_grid *g, const double *pts, int64_t n, const double *verts, const int64_t *ring_off,
                const int64_t *poly_ring_off, const int64_t *cand_start, const int32_t *cand_ids,
                int32_t *out_id, int32_t *out_nhit) {
    if (!grid_ok(g)) return OR_INVALID;
    int64_t G = (int64_t)g->nx * (int64_t)g->ny;
#pragma omp parallel for schedule(dynamic, 1024) num_threads(g_threads)
    for (int64_t i = 0; i < n; ++i) {
        double px = pts[2 * i], py = pts[2 * i + 1];
        int64_t c = or_point_cell(g, px, py);
        int32_t best = -1, nh = 0;
        if (c != G) {
            for (int64_t k = cand_start[c]; k < cand_start[c + 1]; ++k) {
                int32_t p = cand_ids[k];
                if (or_pip_polygon(px, py, verts, ring_off, poly_ring_off, p)) {
                    if (best < 0) best = p;
                    ++nh;
                }
            }
        }
        out_id[i] = best;
        if (out_nhit) out_nhit[i] = nh;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ P2P (Sec. III.B) */

/* Shortest distance from p to segment ab, the two cases of Fig. 2: the
 * perpendicular distance when the projection of p falls strictly inside the
 * segment, else the distance to the nearer end. */
double or_seg_dist(double px, double py, double ax, double ay, double bx, double by) {
    double ex = bx - ax, ey = by - ay;
    double dx = px - ax, dy = py - ay;
    double dot = ex * dx + ey * dy;
    double L2 = ex * ex + ey * ey;
    if (L2 == 0.0 || dot <= 0.0) return sqrt(dx * dx + dy * dy);
    if (dot >= L2) {
        double fx = px - bx, fy = py - by;
        return sqrt(fx * fx + fy * fy);
    }
    double c = ex * dy - ey * dx;
    return fabs(c) / sqrt(L2);
}

/* Distance from p to polyline l: the minimum over its segments; a one-vertex
 * polyline is a point. */
double or_line_dist(double px, double py, const double *verts, const int64_t *line_off, int32_t l) {
    int64_t b = line_off[l], e = line_off[l + 1];
    if (e - b == 1) {
        double dx = px - verts[2 * b], dy = py - verts[2 * b + 1];
        return sqrt(dx * dx + dy * dy);
    }
    double best = INFINITY;
    for (int64_t i = b; i + 1 < e; ++i) {
        double d = or_seg_dist(px, py, verts[2 * i], verts[2 * i + 1], verts[2 * i + 2], verts[2 * i + 3]);
        if (d < best) best = d;
    }
    return best;
}

/* Nearest polyline of one point among ids[0..k) (or all when ids == NULL):
 * lexicographic minimum of (distance, id); out_d2 gets the smallest distance
 * among the other polylines (for the tie tolerance of the tests). */
static void nearest(double px, double py, const double *verts, const int64_t *line_off, const int32_t *ids,
                    int64_t k, double *d1, int32_t *i1, double *d2) {
    double bd = INFINITY, sd = INFINITY;
    int32_t bi = -1;
    for (int64_t t = 0; t < k; ++t) {
        int32_t l = ids ? ids[t] : (int32_t)t;
        double d = or_line_dist(px, py, verts, line_off, l);
        if (d < bd || (d == bd && l < bi)) {
            if (bi >= 0) sd = bd < sd ? bd : sd;
            bd = d;
            bi = l;
        } else if (d < sd) {
            sd = d;
        }
    }
    *d1 = bd; *i1 = bi; *d2 = sd;
}

static void p2p_emit(double R, double bd, int32_t bi, double sd, int64_t i, int32_t *out_id, double *out_d,
                     double *out_d1, double *out_d2) {
    if (bi >= 0 && bd <= R) { out_id[i] = bi; out_d[i] = bd; }
    else                    { out_id[i] = -1; out_d[i] = INFINITY; }
    if (out_d1) out_d1[i] = bd;
    if (out_d2) out_d2[i] = sd;
}

/* Brute force: every in-grid point against every polyline. */
int or_p2p_brute(const or_grid *g, const double *pts, int64_t n, const double *verts, const int64_t *line_off,
                 int32_t L, double R, int32_t *out_id, double *out_d, double *out_d1, double *out_d2) {
    if (!grid_ok(g)) return OR_INVALID;
    int64_t G = (int64_t)g->nx * (int64_t)g->ny;
#pragma omp parallel for schedule(dynamic, 64) num_threads(g_threads)
    for (int64_t i = 0; i < n; ++i) {
        double px = pts[2 * i], py = pts[2 * i + 1];
        double bd = INFINITY, sd = INFINITY;
        int32_t bi = -1;
        if (or_point_cell(g, px, py) != G) nearest(px, py, verts, line_off, NULL, L, &bd, &bi, &sd);
        p2p_emit(R, bd, bi, sd, i, out_id, out_d, out_d1, out_d2);
    }
    return OR_OK;
}

/* Grid-filtered: each in-grid point against the candidates of its cell. */
int or_p2p_grid(const or_grid *g, const double *pts, int64_t n, const double *verts, const int64_t *line_off,
                double R, const int64_t *cand_start, const int32_t *cand_ids, int32_t *out_id, double *out_d,
                double *out_d1, double *out_d2) {
    if (!grid_ok(g)) return OR_INVALID;
    int64_t G = (int64_t)g->nx * (int64_t)g->ny;
#pragma omp parallel for schedule(dynamic, 1024) num_threads(g_threads)
    for (int64_t i = 0; i < n; ++i) {
        double px = pts[2 * i], py = pts[2 * i + 1];
        double bd = INFINITY, sd = INFINITY;
        int32_t bi = -1;
        int64_t c = or_point_cell(g, px, py);
        if (c != G)
            nearest(px, py, verts, line_off, cand_ids + cand_start[c], cand_start[c + 1] - cand_start[c], &bd,
                    &bi, &sd);
        p2p_emit(R, bd, bi, sd, i, out_id, out_d, out_d1, out_d2);
    }
    return OR_OK;
}
