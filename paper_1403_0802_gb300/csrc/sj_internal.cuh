// sj_internal.cuh -- device-side building blocks shared by the CUDA
// translation units of libsj.so (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sj.h"

namespace sj {

constexpr unsigned FULL = 0xffffffffu;
constexpr int MAX_CH = 128;        // largest point chunk per work item
constexpr float U32 = 5.9604644775390625e-08f;   // 2^-24, unit roundoff of FP32

// Grid with derived cell sizes (computed once on the host, FP64, rounded).
struct GridDev {
    double x0, y0, x1, y1;
    double cw, ch;     // (x1 - x0) / nx, (y1 - y0) / ny
    int nx, ny, G;
};

// Cell of one coordinate: floor((v - lo) / w) as a double (may be out of range
// or NaN).  Every operation is a single IEEE round-to-nearest step.
__device__ __forceinline__ double axis_floor(double v, double lo, double w) {
    return floor(__ddiv_rn(__dsub_rn(v, lo), w));
}

// Cell id of a point (Sec. III.A), G when it lies outside the half-open grid
// box or has a NaN coordinate.  ix is in range iff 0 <= floor(t) < n, which is
// the same as 0 <= t < n for the rounded quotient t.
__device__ __forceinline__ int point_cell(const GridDev &g, double x, double y) {
    double fx = axis_floor(x, g.x0, g.cw);
    double fy = axis_floor(y, g.y0, g.ch);
    if (!(fx >= 0.0 && fx < (double)g.nx && fy >= 0.0 && fy < (double)g.ny)) return g.G;
    return (int)fy * g.nx + (int)fx;
}

// floor((v - lo) / w) clamped to [0, n - 1] (rasterisation of MBB corners).
__device__ __forceinline__ int clamped_axis(double v, double lo, double w, int n) {
    double f = axis_floor(v, lo, w);
    if (!(f >= 0.0)) return 0;
    if (f > (double)(n - 1)) return n - 1;
    return (int)f;
}

// FP32-representable frame origin of cell c: the lower-left corner rounded to
// FP32 (stored as a double so that FP64 code can use it exactly).
__device__ __forceinline__ double2 cell_frame(const GridDev &g, int c) {
    int iy = c / g.nx, ix = c - iy * g.nx;
    double ox = __dadd_rn(g.x0, __dmul_rn((double)ix, g.cw));
    double oy = __dadd_rn(g.y0, __dmul_rn((double)iy, g.ch));
    return make_double2((double)__double2float_rn(ox), (double)__double2float_rn(oy));
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Lanes per point group for a chunk of `nw` work units (edges / segments) and
// `np` points: the power of two SG in {1..32} that minimises the number of
// warp iterations ceil(np / (32 / SG)) * (ceil(nw / SG) + reduction steps).
__device__ __forceinline__ int choose_group(int np, int nw, int red_cost) {
    int best_sg = 1, best = 0x7fffffff;
#pragma unroll
    for (int lg = 0; lg <= 5; ++lg) {
        int sg = 1 << lg, pg = 32 >> lg;
        int rounds = (np + pg - 1) / pg;
        int cost = rounds * ((nw + sg - 1) / sg + lg * red_cost);
        if (cost < best) { best = cost; best_sg = sg; }
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
enum { ST_POINTS = 0, ST_ITEMS, ST_PAIRS, ST_TESTS, ST_FALLBACK, ST_HITS, ST_N };

// Arguments of the refinement kernels.
struct RefineArgs {
    GridDev g;
    const int2 *items;       // (cell, first point of the chunk within the cell)
    const int *n_items;      // device count
    const int *cell_start;   // [G + 1] sorted point ranges
    const int *perm;         // sorted slot -> input index
    const double2 *spts;     // sorted points (FP64)
    const int *cand_start;   // [G + 1]
    const int *cand_ids;     // [M]
    const int *obj_voff;     // [nobj + 1] first vertex of each polygon / polyline
    const int *nxt;          // PIP: next vertex of the same ring
    const double2 *verts;    // [V] FP64 vertices
    const float4 *vsplit;    // [V] (fl32(x), fl32(y), fl32(x - fl32(x)), fl32(y - fl32(y)))
    const double2 *seg_e64;  // P2P: [V] b - a of the segment starting at vertex i
    const double *seg_inv64; // P2P: [V] 1 / |b - a|^2 (0 for a degenerate segment)
    const float2 *seg_e32;   // P2P: fl32 of seg_e64
    const float *seg_inv32;  // P2P: fl32 of seg_inv64
    double D;                // P2P window
    float eps_abs;           // absolute term of the vertex rounding bound
    int ch;                  // points per work item
    int *out_id;
    double *out_d;
    int2 *fb;                // P2P FP32X: points to redo in FP64 (sorted slot, cell)
    int *n_fb;
    unsigned long long *stats;
};

// Host-side launchers (defined in the .cu files).
cudaError_t launch_pip_refine(const RefineArgs &a, int form, int warps_per_block, int blocks, cudaStream_t s);
cudaError_t launch_p2p_refine(const RefineArgs &a, int form, int warps_per_block, int blocks, cudaStream_t s);
cudaError_t launch_p2p_recheck(const RefineArgs &a, int blocks, cudaStream_t s);

struct BucketArgs {
    GridDev g;
    const double2 *pts;
    int n;
    int *cnt;            // [G + 1] zeroed
    int2 *key_rank;      // [n] (cell, rank within cell)
    int *cell_start;     // [G + 1]
    int *perm;           // [n]
    double2 *spts;       // [n] or null
    const int *cand_start;  // layer candidates (null: no work items)
    int ch;
    int2 *items;         // work items or null
    int2 *block_sums;    // scan scratch
    int *totals;         // [2]: in-grid points, items
    int *out_id;         // initialised to -1 (or null)
    double *out_d;       // initialised to +inf (or null)
};
size_t bucket_scan_blocks(int G);
cudaError_t launch_bucket(const BucketArgs &a, cudaStream_t s);

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
    int *totals;
    int *bad;                // validation flags
};

}  // namespace sj
