// sj_internal.cuh -- device-side building blocks shared by the CUDA
// translation units of libsj.so (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sj.h"

namespace sj {

constexpr unsigned FULL = 0xffffffffu;
constexpr int MAX_CH = 128;        // largest point chunk per work item
// Largest element count of any array the kernels index with 32-bit ints
// (points, vertices, candidate and list entries): every grid-stride loop with
// a 32-bit index advances by at most 2^22 (grids are capped below that), so an
// index i < MAX_COUNT never passes 2^31 - 1 when it advances; loops with a
// larger step (the unrolled bucketing and unsort kernels) count in 64 bits.
constexpr long long MAX_COUNT = (1LL << 31) - (1LL << 22);
constexpr float U32 = 5.9604644775390625e-08f;   // 2^-24, unit roundoff of FP32

// Grid with derived cell sizes (computed once on the host, FP64, rounded) and
// the per-axis threshold tables of point_cell.
struct GridDev {
    double x0, y0, x1, y1;
    double cw, ch;     // (x1 - x0) / nx, (y1 - y0) / ny
    int nx, ny, G;
    const unsigned long long *kx;   // [nx + 1] order keys of the x thresholds
    const unsigned long long *ky;   // [ny + 1]
    float x0f, y0f, icwf, ichf;     // FP32 estimates of x0, y0, 1 / cw, 1 / ch
};

// Cell of one coordinate: floor((v - lo) / w) as a double (may be out of range
// or NaN).  Every operation is a single IEEE round-to-nearest step.
__device__ __forceinline__ double axis_floor(double v, double lo, double w) {
    return floor(__ddiv_rn(__dsub_rn(v, lo), w));
}

// Order-preserving map of a double to an unsigned 64-bit key (x < y iff
// key(x) < key(y) for non-NaN values; -0 sorts just below +0).
__device__ __forceinline__ unsigned long long order_key(double v) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}
__device__ __forceinline__ double key_value(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffULL) : ~k));
}

// FP32 value of a finite double, truncated, from its bit pattern with integer
// operations only (no FP64 instruction); magnitudes outside the FP32 normal
// range are clamped.  Only used as an estimate.
__device__ __forceinline__ float approx_float(double v) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    unsigned hi = (unsigned)(b >> 32);
    int e = (int)((hi >> 20) & 0x7ff) - 896;          // FP32 biased exponent
    unsigned m = (unsigned)(b >> 29) & 0x7fffffu;
    unsigned bits = (e <= 0) ? 0u : (e >= 255 ? 0x7f7fffffu : (((unsigned)e << 23) | m));
    return __uint_as_float(bits | (hi & 0x80000000u));
}

// Split a finite double v into FP32 hi + lo with integer and FP32 operations
// only: hi = v truncated toward zero to FP32 (a monotone map), lo = fl32(v - hi)
// (the 29 mantissa bits the truncation drops, converted and scaled by a power
// of two).  |v - hi| < ulp32(hi) <= 2^-23 |v|; magnitudes below 2^-126 give
// hi = lo = 0 and magnitudes beyond the FP32 range are clamped (callers keep
// coordinates below 1e30).
__device__ __forceinline__ void split_double(double v, float &hi, float &lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    hi = approx_float(v);
    const int pe = (int)((b >> 52) & 0x7ff) - 948;   // FP32 biased exponent of 2^(e - 52)
    const float scale = (pe >= 1 && pe <= 254) ? __int_as_float(pe << 23) : 0.0f;
    const float l = __uint2float_rn((unsigned)(b & 0x1fffffffULL)) * scale;
    lo = (b >> 63) ? -l : l;
}

// Cell-relative FP32 coordinate (hi - origin) + lo of a split value.
__device__ __forceinline__ float rel_coord(float hi, float lo, float origin) {
    return __fadd_rn(__fsub_rn(hi, origin), lo);
}

// Bit pattern of the double equal to a float (exact widening) with integer
// operations only; finite normal or zero inputs, infinities kept.
__device__ __forceinline__ double widen(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
    const unsigned e = (u >> 23) & 0xff, m = u & 0x7fffffu;
    unsigned long long bits;
    if (e == 0) bits = s;                                        // zero (FP32 subnormals flushed)
    else if (e == 0xff) bits = s | 0x7ff0000000000000ULL | ((unsigned long long)m << 29);
    else bits = s | ((unsigned long long)(e + 896) << 52) | ((unsigned long long)m << 29);
    return __longlong_as_double((long long)bits);
}

// Cell index along one axis by threshold table: keys[k] is the order key of the
// smallest double whose cell, floor(fl(fl(v - lo) / w)), is >= k, so the cell
// of v is the k with keys[k] <= key(v) < keys[k + 1] (exactly the FP64 rule:
// the rule is monotone in v).  An FP32 estimate picks the start; integer key
// compares walk to the exact cell.  Returns -1 outside [keys[0], keys[n]).
__device__ __forceinline__ int axis_cell(double v, const unsigned long long *keys, int n, float lof, float iwf) {
    const unsigned long long k = order_key(v);
    if (k < keys[0] || k >= keys[n]) return -1;
    float t = floorf((approx_float(v) - lof) * iwf);
    int i = (t >= (float)(n - 1)) ? n - 1 : (t > 0.0f ? (int)t : 0);
    while (k < keys[i]) --i;          // keys[0] <= k, so this stops at i >= 0
    while (k >= keys[i + 1]) ++i;     // k < keys[n], so this stops at i <= n - 1
    return i;
}

// Cell id of a point (Sec. III.A), G when it lies outside the half-open grid
// box or has a NaN or infinite coordinate; (ix, iy) its column and row.
__device__ __forceinline__ int point_cell_xy(const GridDev &g, double x, double y, int &ix, int &iy) {
    const unsigned long long EXP = 0x7ff0000000000000ULL;
    ix = iy = -1;
    if (((unsigned long long)__double_as_longlong(x) & EXP) == EXP ||
        ((unsigned long long)__double_as_longlong(y) & EXP) == EXP)
        return g.G;
    ix = axis_cell(x, g.kx, g.nx, g.x0f, g.icwf);
    iy = axis_cell(y, g.ky, g.ny, g.y0f, g.ichf);
    if (ix < 0 || iy < 0) return g.G;
    return iy * g.nx + ix;
}
__device__ __forceinline__ int point_cell(const GridDev &g, double x, double y) {
    int ix, iy;
    return point_cell_xy(g, x, y, ix, iy);
}

// floor((v - lo) / w) clamped to [0, n - 1] (rasterisation of MBB corners).
__device__ __forceinline__ int clamped_axis(double v, double lo, double w, int n) {
    double f = axis_floor(v, lo, w);
    if (!(f >= 0.0)) return 0;
    if (f > (double)(n - 1)) return n - 1;
    return (int)f;
}

// FP32 frame origin of cell c: the lower-left corner x0 + ix * cw rounded to
// FP32, read from per-axis tables built with the layer (frame_x[nx], frame_y[ny]).
__device__ __forceinline__ float2 cell_frame(const float *fx, const float *fy, int nx, int c) {
    const int iy = c / nx;
    return make_float2(fx[c - iy * nx], fy[iy]);
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Bounds-checked builds (compiled with -DSJ_CHECK_BOUNDS): a guarded access
// first tests its index; out of range, it is skipped and the guard's code is
// OR-ed into this translation unit's error word, which the host reads back
// after the call (bounds_take()) -- no trap, the context stays usable.  In
// normal builds a guard is `true` and costs nothing.
enum {
    BND_BUCKET = 1, BND_SCATTER = 2, BND_UNSORT = 4, BND_P2P_POINT = 8, BND_P2P_REC = 16, BND_P2P_RES = 32,
    BND_PIP_POINT = 64, BND_PIP_REC = 128, BND_PIP_RES = 256
};
#ifdef SJ_CHECK_BOUNDS
static __device__ unsigned g_bounds_err;
#define SJ_IN_BOUNDS(cond, code) ((cond) || (atomicOr(&g_bounds_err, (unsigned)(code)), false))
// This translation unit's error word, read and cleared (host).
static inline unsigned bounds_take() {
    unsigned v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_bounds_err, sizeof(v)) != cudaSuccess) return 0x80000000u;
    cudaMemcpyToSymbol(g_bounds_err, &z, sizeof(z));
    return v;
}
#else
#define SJ_IN_BOUNDS(cond, code) true
static inline unsigned bounds_take() { return 0; }
#endif

// 16-byte asynchronous copy global -> shared (cp.async), cached in L2 only:
// the copied data is read once, from shared memory, and allocating it in L1
// would evict the segment records that consecutive items of a cell re-read
// (P2P refine at 170 M points: 4.72 -> 4.23 ms).  Both addresses 16-byte
// aligned.  The copying thread sees the data after copy_async_wait_all().
__device__ __forceinline__ void copy16_async(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void copy_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Points per work item of cell c: the join's chunk size ch, reduced for cells
// whose points each test many edges / segments (work = the cell's list
// length) so that points x work stays within ch x budget -- the work queue is
// split by candidate-edge count, heavy cells yielding more, smaller items --
// but never below min(ch, 8) points (budget 0: ch for every cell).
__host__ __device__ __forceinline__ int cell_chunk(int ch, int work, int budget) {
    if (budget <= 0 || work <= budget) return ch;
    const long long c = (long long)ch * budget / work;
    const int lo = ch < 8 ? ch : 8;
    return c < lo ? lo : (c > ch ? ch : (int)c);
}

// Lanes per point group for a chunk of `nw` work units (edges / segments) and
// `np` points: the power of two SG in {1..32} that minimises the number of
// warp iterations ceil(np / (32 / SG)) * (ceil(nw / SG) + reduction steps).
__device__ __forceinline__ int choose_group(int np, int nw, int red_cost) {
    int best_sg = 1, best = 0x7fffffff;
#pragma unroll
    for (int lg = 0; lg <= 5; ++lg) {
        // powers of two: shifts, not divisions
        const int rounds = (np + (32 >> lg) - 1) >> (5 - lg);
        const int cost = rounds * (((nw + (1 << lg) - 1) >> lg) + lg * red_cost);
        if (cost < best) { best = cost; best_sg = 1 << lg; }
    }
    return best_sg;
}

// Minimum bounding box of an object.
struct Box {
    double xmin, ymin, xmax, ymax;
};

// Layer kinds.
enum { KIND_PIP = 0, KIND_P2P = 1 };

// Per-layer device counters (index into sj_run_stats order after `joins`).
enum { ST_POINTS = 0, ST_ITEMS, ST_PAIRS, ST_TESTS, ST_FALLBACK, ST_HITS, ST_ALGO, ST_RESOLVED, ST_N };

// cell_res value of a polygon-layer cell whose points need the refinement.
constexpr int CELL_REFINE = -2;

// Adds counters to the layer's statistics with one global atomic per counter
// and block: every lane 0 of the block's warps passes its warp's values
// (others pass zeros), the block sums them in shared memory first.  Every
// thread of the block must call it (it synchronises the block).  Thousands of
// warps adding to the same few addresses would otherwise queue at the L2.
__device__ __forceinline__ void flush_stats(unsigned long long *stats, const unsigned long long *v) {
    __shared__ unsigned long long blk[ST_N];
    if (threadIdx.x < ST_N) blk[threadIdx.x] = 0;
    __syncthreads();
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < ST_N; ++k)
            if (v[k]) atomicAdd(&blk[k], v[k]);
    __syncthreads();
    if (threadIdx.x < ST_N && blk[threadIdx.x]) atomicAdd(&stats[threadIdx.x], blk[threadIdx.x]);
}

// Cell-ordered P2P results of a per-request join, one record per slot so that
// the final gather to input order reads one place per point.
struct ResF {            // FP32X: id and the certified FP32 distance (+inf on a miss)
    int id;
    float d;
};
struct alignas(16) ResD {  // FP64
    int id;
    int pad;
    double d;
};

// Arguments of the refinement kernels.
struct RefineArgs {
    GridDev g;
    const int2 *items;       // (cell, first point of the chunk within the cell)
    const int *n_items;      // device count
    int *work_next;          // zeroed device counter handing out items (or null: fixed stride)
    int claim;               // consecutive items a warp takes per counter update (>= 1)
    const int *cell_start;   // [G + 1] sorted point ranges
    const int *perm;         // sorted slot -> input index
    const double2 *spts;     // sorted points (FP64), or null: the point of slot j is pts[perm[j]]
    const double2 *pts;      // input points (used when spts is null)
    const int *cand_start;   // [G + 1]
    const int *cand_ids;     // [M]
    const int *obj_voff;     // [nobj + 1] first vertex of each polygon / polyline
    const int *nxt;          // PIP: next vertex of the same ring
    const double2 *verts;    // [V] FP64 vertices
    const float4 *vsplit;    // [V] (fl32(x), fl32(y), fl32(x - fl32(x)), fl32(y - fl32(y)))
    const double2 *seg_e64;  // P2P: [V] b - a of the segment starting at vertex i
    const double *seg_inv64; // P2P: [V] 1 / |b - a|^2 (0 for a degenerate segment)
    const float4 *seg32;     // P2P: (fl32(ex), fl32(ey), fl32(1 / |e|^2), owner polyline id bits)
    const int *cseg_start;   // P2P: [G + 1] per-cell segment lists
    const int *cseg_ids;     //      segment (= first vertex) indices, ascending per cell
    const int *cell_algo;    //      [G] segments of the cell's candidate polylines
    const float4 *cseg_rec;  //      [2 MS] staging records of the list entries (see sj_filter.cu)
    const int *prow_base;    // PIP: [P + 1] first (polygon, row) slot of each polygon
    const int *prow_r0;      //      [P] first grid row of each polygon's MBB
    const int *prow_start;   //      [slots + 1] edge list range of each (polygon, row)
    const int *pedge_ids;    //      edge (= first vertex) indices
    const float4 *pedge_rec; //      [2 entries] vsplit of the entry's edge ends (FP32X staging)
    const unsigned char *cand_cls;   // PIP: per candidate entry 0 = boundary (test its edges),
                                     //      1 = cell inside the polygon, 2 = outside
    const int *bnear_start;  // PIP boundary entries: near edge lists [M + 1]
    const int *bnear_ids;
    const float4 *bnear_rec; //      [2 per edge] vsplit of both ends
    const float *bnear_key;  //      per near edge: min of its ends' FP32 truncated y (ascending per entry)
    const float *bnear_h;    //      [M] largest (max - min) truncated y of an entry's edges, rounded up
    const int *bflip_start;  //      far-right parity flips: [M + 1] starts,
    const int *bflip_len;    //      [M] lengths,
    const unsigned long long *bflip_keys;   // ascending order keys of the flip y-values
    double D;                // P2P window
    float Ddn, Dup;          // FP32 D rounded down / up with a 1e-12 relative margin
    float Df;                // D rounded to FP32 (staging prune)
    // per-point windows (batched rounds whose requests ask for windows below
    // D): when win_on and *win_on != 0, point slot j is joined within win[j]
    // (<= D) instead of D; the lists and the staging prune stay those of D
    const double *win;
    const int *win_on;
    float eps_abs;           // absolute term of the split-coordinate rounding bound
    const float *frame_x;    // [nx] FP32 cell frame origins along x
    const float *frame_y;    // [ny]
    int npts;                // input points (slot indices and perm values stay below it)
    int ch;                  // points per work item (at most; see cell_chunk)
    const int *cell_work;    // [G] per-point edge / segment work of each cell (or null)
    int budget;              // edge budget per point of an item (0: none)
    int *out_id;
    double *out_d;
    int *res_id;             // when set: results in sorted order for every slot
    double *res_d;           //   (hits and misses); out_id / perm unused
    ResF *resf;              // P2P FP32X: packed sorted results (instead of res_id / res_d);
                             //   the FP64 recheck then writes out_id / out_d through perm
    ResD *resd;              // P2P FP64: packed sorted results
    int2 *fb;                // P2P FP32X: points to redo in FP64 (sorted slot, cell)
    int *n_fb;
    unsigned long long *stats;
};

// FP64 point of sorted slot j.
__device__ __forceinline__ double2 slot_point(const RefineArgs &a, int j) {
    return a.spts ? a.spts[j] : a.pts[a.perm[j]];
}

// Order key of a y-value with -0 folded onto +0 (IEEE compares treat them as
// equal; the order key alone would not).
__device__ __forceinline__ unsigned long long y_key(double v) { return order_key(v == 0.0 ? 0.0 : v); }

// PIP boundary-entry lists (layer build): count (emit = 0) or emit (emit = 1).
struct BoundaryArgs {
    GridDev g;
    const int *cand_start, *cand_ids;
    const unsigned char *cls;
    const int *prow_base, *prow_r0, *prow_start, *pedge_ids, *nxt, *prv;
    const double2 *verts;
    double delta;
    int *near_cnt, *flip_cnt;                 // count pass: [M]
    const int *near_start, *flip_start;       // emit pass
    int *near_ids;
    unsigned long long *flip_keys;
};
cudaError_t launch_pip_boundary(const BoundaryArgs &a, int emit, cudaStream_t s);
cudaError_t launch_pip_flips(const int *flip_start, int M, unsigned long long *keys, int *len, cudaStream_t s);
cudaError_t launch_pip_near_sort(const int *near_start, int M, int *ids, const int *nxt, const float4 *vsplit,
                                 float *keys, float *h, cudaStream_t s);

// PIP cell classification (layer build): one class per candidate entry.
cudaError_t launch_cell_work_pip(const int *cand_start, const unsigned char *cls, const int *near_start, int G,
                                 int *work, cudaStream_t s);
cudaError_t launch_cell_work_p2p(const int *cseg_start, int G, int *work, cudaStream_t s);
cudaError_t launch_cell_result(const int *cand_start, const int *cand_ids, const unsigned char *cls, int G, int *res,
                               cudaStream_t s);
cudaError_t launch_pip_classify(const GridDev &g, const int *cand_start, const int *cand_ids, const int *prow_base,
                                const int *prow_r0, const int *prow_start, const int *pedge_ids, const int *nxt,
                                const double2 *verts, double delta, unsigned char *cls, cudaStream_t s);

// The error words of the bounds-checked build, per translation unit, read
// and cleared (0 in normal builds).
unsigned bounds_take_filter();
unsigned bounds_take_p2p();
unsigned bounds_take_pip();

// Host-side launchers (defined in the .cu files).
cudaError_t launch_pip_refine(const RefineArgs &a, int form, int warps_per_block, int blocks, cudaStream_t s);
cudaError_t launch_p2p_refine(const RefineArgs &a, int form, int warps_per_block, int blocks, cudaStream_t s);
cudaError_t launch_p2p_recheck(const RefineArgs &a, int blocks, cudaStream_t s);
cudaError_t launch_pip_census(const RefineArgs &a, const double2 *pts, int n, unsigned long long *out,
                              cudaStream_t s);

struct BucketArgs {
    GridDev g;
    const double2 *pts;
    int n;
    int *cnt;            // [G + 1] zeroed
    int2 *key_rank;      // [n] (cell, rank within cell)
    int *cell_start;     // [G + 1]
    int *perm;           // [n]
    double2 *spts;       // [n] cell-ordered copy of the points, or null (not written)
    const int *cand_start;  // layer candidates (null: no work items)
    int ch;
    const int *cell_work;   // with budget > 0: work items of cell_chunk(ch, cell_work[c], budget) points
    int budget;
    int2 *items;         // work items or null
    int2 *block_sums;    // scan scratch
    size_t bs_cap;       // its capacity in int2 (launches fail when it is too small)
    int *totals;         // [2]: in-grid points, items
    int *out_id;         // initialised to -1 (or null)
    double *out_d;       // initialised to +inf (or null)
    int *pos;            // [n] sorted slot of each input point, -1 when its cell has no
                         //     candidates or it lies outside the grid (or null)
    int *cell_base;      // [G] with pos: cell_start of cells that yield work items, else -1
    // Sub-cell order (sub_lx + sub_ly > 0): inside each cell the points are
    // ordered by sub-cell, 2^sub_lx x 2^sub_ly sub-cells in Z-order, so that
    // consecutive points of a cell -- one work item -- cover a compact part of
    // it.  cnt then holds G * S + 1 counters (S = 2^(sub_lx + sub_ly)) and
    // sub_start [G * S] the first slot of each sub-cell (-1 with pos for cells
    // without work items).  The order is a pure permutation within cells: no
    // result depends on it.
    int sub_lx, sub_ly;
    int *sub_start;
    // PIP: per cell the result of every point of a cell whose candidates are
    // all classified inside / outside, else CELL_REFINE (or null).  Such a
    // point's result is written to out_id by the cell-id pass itself; it gets
    // no slot (pos = POS_DONE) and no work item.
    const int *cell_res;
    unsigned long long *stats;   // ST_RESOLVED counts those points (or null)
};
constexpr int POS_DONE = -2;   // pos of a point whose result the cell-id pass wrote

// Z-order index of sub-cell (sx, sy) with lx / ly bits per axis (at most 3).
__device__ __forceinline__ int sub_index(int sx, int sy, int lx, int ly) {
    int sub = 0, bit = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        if (b < lx) sub |= ((sx >> b) & 1) << bit++;
        if (b < ly) sub |= ((sy >> b) & 1) << bit++;
    }
    return sub;
}
size_t bucket_scan_blocks(int G);
cudaError_t launch_bucket(const BucketArgs &a, cudaStream_t s);
// a8 for cell-ordered results: out[i] = res[pos[i]], or -1 / +inf where
// pos[i] < 0 (one pass; out_d and res_d may be null).
cudaError_t launch_unsort(const int *pos, const int *res_id, const double *res_d, int n, int *out_id, double *out_d,
                          cudaStream_t s);
cudaError_t launch_unsort_f(const int *pos, const ResF *res, int n, int *out_id, double *out_d, cudaStream_t s);
cudaError_t launch_unsort_d(const int *pos, const ResD *res, int n, int *out_id, double *out_d, cudaStream_t s);

struct LayerBuildArgs {
    GridDev g;
    int kind;
    double D;
    int nobj, V;
    const double2 *verts;
    const int *obj_voff;     // [nobj + 1]
    Box *mbb;                // [nobj]
    int *cell_cnt;           // [G + 1] zeroed
    int *cand_start;         // [G + 1]
    int *cursor;             // [G] zeroed
    int *obj_cells;          // [nobj + 1]
    int2 *block_sums;
    size_t bs_cap;           // capacity of block_sums in int2
    int *totals;
    int *bad;                // validation flags
};

}  // namespace sj
