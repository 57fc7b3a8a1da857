/*
 * sj.h -- C ABI of the GB300 grid-filtered spatial join (libsj.so).
 *
 * The library implements the data-parallel spatial join of Zhang & You,
 * "Large-Scale Geospatial Processing on Multi-Core and Many-Core Processors"
 * (arXiv 1403.0802):
 *   - a uniform-grid filter (Sec. III.A, Fig. 1): points are bucketed by grid
 *     cell, and polygon / polyline minimum bounding boxes (MBBs) are rasterised
 *     to the same grid, giving per-cell candidate lists;
 *   - PIP refinement (Sec. III.C, Fig. 3): ray-crossing point-in-polygon test
 *     over every ring of a candidate polygon (holes allowed);
 *   - P2P refinement (Sec. III.B, Fig. 2): nearest polyline within a window
 *     R (called D here), by the minimum point-to-segment distance.
 *
 * Conventions shared by every entry point:
 *   - Coordinates are FP64 metres, points and vertices are interleaved
 *     (x, y) pairs, i.e. [n, 2] row-major arrays; point / vertex arrays must be
 *     16-byte aligned.
 *   - "dev" pointers are CUDA device pointers, "host" pointers are host memory.
 *     The caller owns every buffer it passes in.  The library owns sj_layer
 *     objects and the scratch memory of each call (stream-ordered allocations
 *     on the caller's stream).
 *   - stream is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  Joins are asynchronous on it; argument errors are returned
 *     synchronously and leave the outputs untouched.
 *   - Ids are 0-based int32.  The join domain is the half-open grid box
 *     [x0, x1) x [y0, y1): points outside it get id -1 (and distance +inf).
 *   - Readings of the paper used here (the paper is silent on them):
 *       cell of (x, y): ix = floor((x - x0) / cw), cw = (x1 - x0) / nx, in FP64;
 *       an edge (a, b) straddles p iff (a.y > p.y) != (b.y > p.y); with lo the
 *       end at or below p.y and hi the other, it counts iff
 *       (hi.x - lo.x) * (p.y - lo.y) - (hi.y - lo.y) * (p.x - lo.x) > 0
 *       (FP64, each operation rounded, no fused multiply-add); inside iff the
 *       count over all rings is odd; a point inside several polygons gets the
 *       smallest id; the P2P window is inclusive (d <= D) and equal distances
 *       go to the smaller id.
 *   - Every function returns an sj_status; on failure sj_last_error() gives a
 *     message (thread-local, valid until the next call on that thread).
 */
#ifndef SJ_H
#define SJ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Uniform grid over [x0, x1) x [y0, y1) with nx * ny cells (Sec. III.A).
 * Requires finite x0 < x1, y0 < y1, 1 <= nx, ny <= 2^20 and nx * ny <= 2^31 - 2^22.
 * Every element count of the library (cells, points, vertices, rings,
 * candidate and list entries) is at most 2^31 - 2^22, so that 32-bit indices
 * of the kernels' grid-stride loops never overflow; a layer whose lists would
 * be longer is rejected with SJ_ERR_INVALID. */
typedef struct {
    double x0, y0, x1, y1;
    int32_t nx, ny;
} sj_grid;

typedef enum {
    SJ_OK = 0,
    SJ_ERR_INVALID = -1,    /* bad argument, bad layer topology, NaN / inf vertex  */
    SJ_ERR_OOM = -2,        /* device allocation failed                            */
    SJ_ERR_GRID_COVER = -3, /* an MBB is not inside the closed grid box            */
    SJ_ERR_CUDA = -4,       /* a CUDA call failed (message in sj_last_error)       */
    SJ_ERR_TIMEOUT = -5,    /* a bounded wait gave up (sj_server_wait_for)         */
    SJ_ERR_BUSY = -6,       /* resource in use, or a request refused (admission)   */
    SJ_ERR_CANCELLED = -7   /* the request was cancelled before it ran             */
} sj_status;

/* Refinement arithmetic. */
enum {
    SJ_FP64 = 0,  /* plain FP64 refinement                                        */
    SJ_FP32X = 1  /* cell-relative FP32 with FP64 fallback: PIP ids are identical
                     to the FP64 rule; P2P ids are exact (ties aside) and the
                     distance error is bounded per point                           */
};

/* Launch form.  Every join's refinement is one persistent launch whose warps
 * take work items from a device counter (cost-balanced); both values select
 * that code and give the same results.  Batched rounds of many requests are
 * the sj_engine_* calls below. */
enum {
    SJ_PER_REQUEST = 0, /* one pass of kernels per call                           */
    SJ_PERSISTENT = 1   /* same kernels (accepted for callers that ask for it)    */
};

/* Join options; a zeroed struct (or NULL) selects the defaults.  The launch
 * knobs (block, pts_per_item, edges_per_chunk) change speed only, never a
 * result; paper_1403_0802_gb300/autotune.py times their combinations. */
typedef struct {
    int32_t form;            /* SJ_FP64 (default) or SJ_FP32X                       */
    int32_t launch;          /* SJ_PER_REQUEST (default) or SJ_PERSISTENT           */
    int32_t block;           /* warps per refinement block: 2, 4 or 8; 0 = 4.  The
                                grid keeps the same number of resident warps (SMs x
                                the occupancy of 4-warp blocks, in warps)          */
    int32_t pts_per_item;    /* points per work item, 1..128, 0 = default (128)    */
    int32_t edges_per_chunk; /* edge budget of a work item: a cell whose points
                                each test w > edges_per_chunk edges (PIP: the near
                                edges of its boundary candidates; P2P: its segment
                                list) is cut into items of
                                max(min(pts_per_item, 8),
                                    pts_per_item * edges_per_chunk / w) points, so
                                that heavy cells yield more, smaller items (the work
                                queue split by candidate-edge count).  0 = the
                                default: 64 for polygon layers, no split for
                                polyline layers; a value above every cell's work
                                (e.g. INT32_MAX) turns the split off              */
    int32_t flags;           /* SJ_FLAG_* bits                                      */
} sj_opts;

/* opts.flags: record CUDA events on the call's stream around the refinement
 * kernels; their summed elapsed time is reported by sj_layer_get_stats. */
#define SJ_FLAG_TIME_REFINE 1
/* opts.flags of the joins: order the points inside each grid cell by sub-cell
 * (P2P: 4 x 4 sub-cells in Z-order; PIP: 8 horizontal bands) before they are
 * cut into work items (SJ_FLAG_SUBCELL_ON), or keep them in arrival order
 * (the default; SJ_FLAG_SUBCELL_OFF says so explicitly).  Results do not
 * depend on it (a point's result depends on the point and the layer only).
 * Work items of dense cells then cover compact parts of their cell, so the
 * exact per-item prunes leave fewer tests, at the price of a per-sub-cell
 * start table (4 bytes per sub-cell) in the bucketing. */
#define SJ_FLAG_SUBCELL_ON 4
#define SJ_FLAG_SUBCELL_OFF 8

typedef struct sj_layer sj_layer;

typedef struct {
    int32_t kind;         /* 0 = polygon layer (PIP), 1 = polyline layer (P2P)  */
    int32_t n_objects;    /* polygons or polylines                              */
    int64_t n_vertices;
    int64_t n_rings;      /* polygon layers; = n_objects for polyline layers    */
    int64_t n_cells;      /* G = nx * ny                                        */
    int64_t n_candidates; /* M = number of (cell, object) candidate pairs       */
    double D;             /* P2P window (0 for polygon layers)                  */
} sj_layer_info;

/* Counters accumulated by the joins run on a layer since the last reset. */
typedef struct {
    int64_t joins;
    int64_t points;        /* points submitted                                  */
    int64_t items;         /* (cell, point-chunk) work items                    */
    int64_t pairs;         /* (point, candidate object) pairs refined            */
    int64_t edge_tests;    /* PIP: point x edge tests; P2P: point x segment tests */
    int64_t fallbacks;     /* SJ_FP32X: PIP edges / P2P points redone in FP64   */
    int64_t hits;          /* points given an id                                 */
    int64_t refine_launches; /* refinement launches timed (SJ_FLAG_TIME_REFINE)  */
    double refine_ms;        /* their summed device time, milliseconds           */
    int64_t algo_tests;      /* edge / segment tests the candidate lists imply;
                                edge_tests is what remains after the exact
                                per-item prune (edges that cannot straddle /
                                segments farther than D from every point)        */
    int64_t census_tests;     /* sj_pip_census totals since the last reset: the  */
    int64_t census_straddles; /* edges of the points' candidate polygons, and how
                                 many of them straddle the point's y              */
    int64_t resolved;         /* PIP: points whose cell's candidates are all
                                 classified inside / outside, answered by the
                                 cell-id pass without refinement (counted in
                                 hits, not in items, pairs or algo_tests)         */
} sj_run_stats;

/* Build a resident polygon layer and its candidate lists (Sec. III.A: MBB of
 * each polygon rasterised to the grid; Sec. III.C: no expansion for PIP).
 *   verts          dev  [V, 2] f64 vertices; ring r owns ring_off[r] .. ring_off[r+1]-1,
 *                       implicitly closed (a repeated closing vertex is harmless)
 *   ring_off       dev  [R + 1] int64, ring_off[0] = 0, ring_off[R] = V, rings >= 3 vertices
 *   poly_ring_off  dev  [P + 1] int64, polygon p owns rings poly_ring_off[p] .. [p+1]-1
 *                       (outer ring and holes alike: even-odd rule), >= 1 ring each
 *   g              host grid; every polygon MBB must lie in the closed grid box
 * The input arrays are copied; the caller may free them after return.  The
 * call synchronises `stream` (it reads validation results back).
 * Errors: SJ_ERR_INVALID (topology, NaN/inf, V > 2^31 - 2^22), SJ_ERR_GRID_COVER,
 * SJ_ERR_OOM, SJ_ERR_CUDA. */
sj_status sj_pip_layer_create(const double *verts, int64_t V, const int64_t *ring_off, int64_t R,
                              const int64_t *poly_ring_off, int32_t P, const sj_grid *g, void *stream,
                              sj_layer **out);

/* Build a resident polyline layer for window D (Sec. III.A: expanded MBB
 * (x1 - D, y1 - D, x2 + D, y2 + D), rounded outward by one ulp).
 *   verts     dev [V, 2] f64; polyline l owns line_off[l] .. line_off[l+1]-1 (>= 1 vertex;
 *                 a one-vertex polyline is a point)
 *   line_off  dev [L + 1] int64
 *   D         window, finite and >= 0
 * Same ownership, synchronisation and errors as sj_pip_layer_create. */
sj_status sj_p2p_layer_create(const double *verts, int64_t V, const int64_t *line_off, int32_t L, double D,
                              const sj_grid *g, void *stream, sj_layer **out);

/* Free a layer (synchronises the device before freeing).  NULL is a no-op. */
sj_status sj_layer_destroy(sj_layer *layer);

sj_status sj_layer_get_info(const sj_layer *layer, sj_layer_info *out);

/* Copy the layer's candidate lists to host memory (Fig. 1, VPP relation in
 * CSR form): cand_start [G + 1] int32, cand_ids [M] int32 sorted by id within
 * each cell.  Synchronous. */
sj_status sj_layer_get_candidates(const sj_layer *layer, int32_t *cand_start, int32_t *cand_ids);

/* Point-in-polygon join (Sec. III.C): out_id[i] = smallest polygon id whose
 * even-odd ray-crossing count for point i is odd, else -1.
 *   pts     dev [N, 2] f64, 16-byte aligned
 *   out_id  dev [N] int32
 *   opts    may be NULL
 * N <= 2^31 - 2^22.  Asynchronous on stream. */
sj_status sj_pip_join(const sj_layer *layer, const double *pts, int64_t N, int32_t *out_id, const sj_opts *opts,
                      void *stream);

/* Point-to-polyline join (Sec. III.B): for each point the polyline with the
 * smallest distance (ties: smaller id) if that distance is <= D:
 * out_id[i] = its id, out_d[i] = the distance; else -1 and +inf.
 *   pts     dev [N, 2] f64; out_id dev [N] int32; out_d dev [N] f64 (may be NULL)
 * SJ_FP64 distances agree with the FP64 two-case formula to 1e-12 * max(d, 1 m);
 * SJ_FP32X distances are within a per-point bound (about 64 * 2^-24 times the
 * largest cell-relative coordinate involved).  Asynchronous on stream. */
sj_status sj_p2p_join(const sj_layer *layer, const double *pts, int64_t N, int32_t *out_id, double *out_d,
                      const sj_opts *opts, void *stream);

/* sj_p2p_join with a window chosen per call (Sec. III.B fixes the distance D
 * when the polylines are indexed; this entry point answers any smaller
 * distance query on the same resident layer): the nearest polyline within
 * `window` instead of the layer's D, with the same outputs, precision and
 * streams as sj_p2p_join.  The layer's grid lists, built for D, stay valid for
 * every window <= D; a smaller window prunes no more cells, so the call costs
 * what sj_p2p_join costs.  Errors: SJ_ERR_INVALID when window is NaN, negative
 * or larger than the layer's D. */
sj_status sj_p2p_join_window(const sj_layer *layer, const double *pts, int64_t N, double window, int32_t *out_id,
                             double *out_d, const sj_opts *opts, void *stream);

/* Same joins from HOST buffers: the library copies the points to the device,
 * joins, copies the results back, and synchronises `stream` before returning
 * (the work starts after what is already queued on `stream`).  Inputs of more
 * than 2 M points are split into two or three chunks, pipelined on three
 * library-owned streams (copy in, join, copy out), so that copies and joins of
 * different chunks overlap; every point's result is the one sj_*_join gives.  pts / out_id /
 * out_d are host pointers (pinned memory gives asynchronous full-bandwidth
 * copies; pageable memory works too). */
sj_status sj_pip_join_host(const sj_layer *layer, const double *pts, int64_t N, int32_t *out_id,
                           const sj_opts *opts, void *stream);
sj_status sj_p2p_join_host(const sj_layer *layer, const double *pts, int64_t N, int32_t *out_id, double *out_d,
                           const sj_opts *opts, void *stream);

/* sj_p2p_join_window from HOST buffers (as sj_p2p_join_host, with the
 * window of sj_p2p_join_window).  Errors: those of both. */
sj_status sj_p2p_join_window_host(const sj_layer *layer, const double *pts, int64_t N, double window,
                                  int32_t *out_id, double *out_d, const sj_opts *opts, void *stream);

/* Point bucketing alone (Sec. III.A, Fig. 1 top-left: sort points by cell id,
 * VGC/VGI vectors): cell_start [G + 1] int32 dev gets the exclusive prefix sum
 * of per-cell point counts (cell_start[G] = in-grid points) and perm [N] int32
 * dev the input index of each sorted slot (order within a cell unspecified;
 * slots past cell_start[G] are left untouched).  Asynchronous on stream. */
sj_status sj_bucket_points(const double *pts, int64_t N, const sj_grid *g, int32_t *cell_start, int32_t *perm,
                           void *stream);

/* Census of the algorithmic PIP work (a measurement pass, not a join; used
 * for the arithmetic roofline of the refinement, whose per-edge cost is the
 * straddle test of Sec. III.C plus the orientation test for the edges that
 * straddle the point's y).  For every in-grid point of pts (dev [N, 2] f64)
 * against the candidate polygons of its cell: out[0] = their edges (every
 * ring), out[1] = how many of those edges straddle the point's y, i.e.
 * (a.y > p.y) != (b.y > p.y).  out is a HOST int64 [2]; both are also added to
 * the layer's census_tests / census_straddles counters.  Synchronises
 * `stream`.  Errors: SJ_ERR_INVALID (NULL, not a polygon layer, N out of
 * range), SJ_ERR_CUDA. */
sj_status sj_pip_census(const sj_layer *layer, const double *pts, int64_t N, int64_t *out, void *stream);

/* Counters of the joins run on `layer` (synchronises the device). */
sj_status sj_layer_get_stats(const sj_layer *layer, sj_run_stats *out);
sj_status sj_layer_reset_stats(sj_layer *layer);

/* ------------------------------------------------------------------ batched rounds
 *
 * Continuous batching: an engine joins many requests per call ("round").
 * Requests against the same layer are joined as one point set -- one cell-id
 * pass, one scan, one scatter, ONE refinement launch over their merged work
 * items and one pass that writes each request's outputs -- so a round costs
 * a fixed number of launches per layer whatever the number of requests.  The
 * per-layer kernel sequence has a fixed shape (sizes live in device memory),
 * is captured into a CUDA graph on its first round and replayed afterwards.
 * Results are exactly those of joining each request alone (Sec. III.B-C:
 * a point's result depends only on the point and the layer). */

typedef struct sj_engine sj_engine;

typedef struct {
    const sj_layer *layer;   /* polygon layer (PIP) or polyline layer (P2P)      */
    const double *pts;       /* dev [N, 2] f64, 16-byte aligned                   */
    int64_t N;
    int32_t *out_id;         /* dev [N] int32                                     */
    double *out_d;           /* dev [N] f64 for polyline layers (may be NULL)     */
    int32_t use_window;      /* polyline layers: nonzero = join within `window`
                                (as sj_p2p_join_window); 0 = the layer's D        */
    int32_t pad;
    double window;           /* 0 <= window <= the layer's D when use_window      */
} sj_request;

/* opts.flags for sj_engine_create: launch the round's kernels directly instead
 * of replaying a captured graph. */
#define SJ_FLAG_NO_GRAPH 2

/* Create an engine for rounds of at most max_points points and max_requests
 * requests per layer.  opts selects form and points per work item (as for the
 * joins; NULL = defaults).  The engine allocates one workspace per layer on
 * the first round that uses the layer (about 36 bytes per point for a
 * polygon layer, 60 for a polyline layer, plus 8 bytes per grid cell) and captures that layer's graph then; later rounds allocate
 * nothing.  Layers must outlive the engine.  Errors: SJ_ERR_INVALID. */
sj_status sj_engine_create(int64_t max_points, int32_t max_requests, const sj_opts *opts, sj_engine **out);

/* One round over reqs[0..n): asynchronous on stream (a non-NULL stream is
 * needed for graph replay; the legacy stream runs the kernels directly).  The
 * host blocks only if the request table of the round-before-last for the same
 * layer has not been copied to the device yet.  Rounds on one engine must be
 * issued on one stream (or ordered by the caller).  Requests against one
 * polyline layer may ask for different windows: each point is joined within
 * its request's window (a round with windows below D also writes one window
 * per point, 8 bytes).  Errors: SJ_ERR_INVALID (sizes beyond the engine's
 * limits, bad buffers, a window outside [0, D] or on a polygon layer),
 * SJ_ERR_CUDA, SJ_ERR_OOM. */
sj_status sj_engine_round(sj_engine *engine, const sj_request *reqs, int32_t n, void *stream);

/* Free the engine (synchronises the device first).  NULL is a no-op. */
sj_status sj_engine_destroy(sj_engine *engine);

/* P2P join that allocates nothing.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory when they join
 * -- code on a hard latency budget (an allocation can stall), code living in
 * a pre-sized memory arena, or hosts whose allocator is owned by another
 * component.  It computes exactly what sj_p2p_join computes (same kernels,
 * same results), but every byte of scratch comes from one fixed device array
 * built into the library (about 32 MB, held on every GPU that loads the
 * library until the process exits).  The caller still passes the points and
 * the outputs (same layout and meaning as sj_p2p_join).
 *   N <= SJ_NOALLOC_MAX_POINTS and the layer's grid <= SJ_NOALLOC_MAX_CELLS
 *   cells, else SJ_ERR_INVALID with a message; pts_per_item and flags in opts
 *   are ignored (64 points per item, no timing events).
 * The first call on a device looks up the array's device address (once per
 * device, with that device current) and keeps it for the life of the process;
 * make that first call before any stream capture.  A device reset
 * (cudaDeviceReset) invalidates the kept address: do not call this entry point
 * again in a process that has reset the device.  All calls share the array and it keeps the previous call's
 * contents (the counters that must start at zero are cleared on `stream` at
 * the start of each call): calls whose kernels overlap on the GPU race, so
 * issue them on one stream or order them with events.  Asynchronous on
 * stream. */
#define SJ_NOALLOC_MAX_POINTS 524288
#define SJ_NOALLOC_MAX_CELLS 1048576
sj_status sj_p2p_join_noalloc(const sj_layer *layer, const double *pts, int64_t N, int32_t *out_id, double *out_d,
                              const sj_opts *opts, void *stream);

/* Host-side fault injection, for tests of the failure paths (the paper has
 * no counterpart).  Nothing here touches a GPU: a fault makes a host-side
 * call report the failure it would report for real.
 *   SJ_FAULT_ALLOC  device allocations of the library (layer builds, join
 *                   scratch, engine workspaces, server arenas) fail as out of
 *                   memory: the call returns SJ_ERR_OOM, frees what it had
 *                   allocated and leaves its outputs and the layer untouched;
 *   SJ_FAULT_ADMIT  sj_server_submit refuses the request with SJ_ERR_BUSY (as
 *                   a full server would); the server keeps serving.
 * After `after` calls that would trigger it succeed, the next `count` fail;
 * count 0 (or SJ_FAULT_NONE) disarms.  Process-wide, thread-safe. */
enum { SJ_FAULT_NONE = 0, SJ_FAULT_ALLOC = 1, SJ_FAULT_ADMIT = 2 };
sj_status sj_fault_inject(int32_t kind, int32_t after, int32_t count);
/* Failures still armed (0 when disarmed). */
int32_t sj_fault_pending(void);

/* 1 in a bounds-checked build of the library, else 0.  A checked build
 * (paper_1403_0802_gb300.build.build(checked=True), compiled with
 * -DSJ_CHECK_BOUNDS) tests the index of the kernels' main indexed accesses
 * (point gathers, list records, counters, slots, results) before each access;
 * an out-of-range access is skipped and recorded in an error word, and the
 * join then returns SJ_ERR_CUDA ("bounds check: ...") after synchronising its
 * stream.  No guard traps: the context stays usable.  Normal builds compile
 * the guards away. */
int32_t sj_bounds_checked(void);

/* Message of the last failing call on this thread ("" if none). */
const char *sj_last_error(void);

/* Library version string. */
const char *sj_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SJ_H */
