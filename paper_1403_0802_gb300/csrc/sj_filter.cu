// sj_filter.cu -- the uniform-grid filter of Sec. III.A (Fig. 1):
//   - point bucketing: cell id per point, per-cell counts, exclusive scan,
//     scatter into cell order (the VGC / VGI vectors of Fig. 1), plus the
//     (cell, point-chunk) work items of cells that have candidates;
//   - layer side: per-object MBB, rasterisation of (expanded) MBBs to cells,
//     and the per-cell candidate lists (the VPP relation) in CSR form.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sj_internal.cuh"

namespace sj {

unsigned bounds_take_filter() { return bounds_take(); }

// ------------------------------------------------------------------ block scan helpers

constexpr int SCAN_T = 256;
constexpr int SCAN_V = 4;     // 1,024 elements per tile: >= 256 tiles for a 512 x 512 grid
constexpr int SCAN_TILE = SCAN_T * SCAN_V;

__device__ __forceinline__ int2 add2(int2 a, int2 b) { return make_int2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ int2 sub2(int2 a, int2 b) { return make_int2(a.x - b.x, a.y - b.y); }

__device__ __forceinline__ int2 warp_incl_scan(int2 v) {
    int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int x = __shfl_up_sync(FULL, v.x, o), y = __shfl_up_sync(FULL, v.y, o);
        if (lane >= o) { v.x += x; v.y += y; }
    }
    return v;
}

// Inclusive scan over the block (blockDim.x = NT, a multiple of 32); also
// returns the block total.
template <int NT>
__device__ __forceinline__ int2 block_incl_scan(int2 v, int2 &total) {
    __shared__ int2 wsum[NT / 32];
    int lane = lane_id(), w = threadIdx.x >> 5;
    int2 inc = warp_incl_scan(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        int2 s = lane < NT / 32 ? wsum[lane] : make_int2(0, 0);
        s = warp_incl_scan(s);
        if (lane < NT / 32) wsum[lane] = s;
    }
    __syncthreads();
    if (w > 0) inc = add2(inc, wsum[w - 1]);
    total = wsum[NT / 32 - 1];
    __syncthreads();
    return inc;
}

// Phase 1: per-tile sums.
template <class Load>
__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(Load ld, int n, int2 *block_sums) {
    int base = blockIdx.x * SCAN_TILE;
    int2 s = make_int2(0, 0);
#pragma unroll
    for (int k = threadIdx.x; k < SCAN_TILE; k += SCAN_T) {
        int c = base + k;
        if (c < n) s = add2(s, ld(c));
    }
    int2 total;
    block_incl_scan<SCAN_T>(s, total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// Phase 2: exclusive scan of the tile sums in one block; block_sums[nb] and
// totals[0..1] get the grand total.
__global__ void __launch_bounds__(1024) k_scan_top(int2 *block_sums, int nb, int *totals) {
    int2 carry = make_int2(0, 0);
    for (int base = 0; base < nb; base += 1024) {
        int i = base + threadIdx.x;
        int2 v = i < nb ? block_sums[i] : make_int2(0, 0);
        int2 total;
        int2 inc = block_incl_scan<1024>(v, total);
        if (i < nb) block_sums[i] = add2(carry, sub2(inc, v));
        carry = add2(carry, total);
    }
    if (threadIdx.x == 0) {
        block_sums[nb] = carry;
        if (totals) { totals[0] = carry.x; totals[1] = carry.y; }
    }
}

// Phase 3: rescan each tile with its offset; ap(c, exclusive prefix, value).
template <class Load, class Apply>
__global__ void __launch_bounds__(SCAN_T) k_scan_apply(Load ld, Apply ap, int n, const int2 *block_sums) {
    int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_V;
    int2 v[SCAN_V];
    int2 tsum = make_int2(0, 0);
#pragma unroll
    for (int j = 0; j < SCAN_V; ++j) {
        int c = base + j;
        v[j] = c < n ? ld(c) : make_int2(0, 0);
        tsum = add2(tsum, v[j]);
    }
    int2 total;
    int2 inc = block_incl_scan<SCAN_T>(tsum, total);
    int2 ex = add2(sub2(inc, tsum), block_sums[blockIdx.x]);
#pragma unroll
    for (int j = 0; j < SCAN_V; ++j) {
        int c = base + j;
        if (c < n) ap(c, ex, v[j], n);
        ex = add2(ex, v[j]);
    }
}

// Phases 2 and 3 in one launch for at most SCAN_FUSE tiles: each block sums
// the (raw) sums of the tiles before it itself -- at most SCAN_FUSE - 1 loads
// over the block -- and the last tile writes the grand totals.
constexpr int SCAN_FUSE = 256;

template <class Load, class Apply>
__global__ void __launch_bounds__(SCAN_T) k_scan_apply_fused(Load ld, Apply ap, int n, int2 *block_sums, int nb,
                                                             int *totals) {
    int2 pre = make_int2(0, 0);
    for (int k = threadIdx.x; k < (int)blockIdx.x; k += SCAN_T) pre = add2(pre, block_sums[k]);
    int2 offset;
    block_incl_scan<SCAN_T>(pre, offset);   // its total: the tile's exclusive prefix
    int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_V;
    int2 v[SCAN_V];
    int2 tsum = make_int2(0, 0);
#pragma unroll
    for (int j = 0; j < SCAN_V; ++j) {
        int c = base + j;
        v[j] = c < n ? ld(c) : make_int2(0, 0);
        tsum = add2(tsum, v[j]);
    }
    int2 total;
    int2 inc = block_incl_scan<SCAN_T>(tsum, total);
    int2 ex = add2(sub2(inc, tsum), offset);
#pragma unroll
    for (int j = 0; j < SCAN_V; ++j) {
        int c = base + j;
        if (c < n) ap(c, ex, v[j], n);
        ex = add2(ex, v[j]);
    }
    if ((int)blockIdx.x == nb - 1 && threadIdx.x == 0) {
        const int2 grand = add2(offset, total);
        block_sums[nb] = grand;
        if (totals) { totals[0] = grand.x; totals[1] = grand.y; }
    }
}

// block_sums must hold at least nb + 1 entries (bucket_scan_blocks(n) does);
// a smaller capacity is an error, not an out-of-bounds write.
template <class Load, class Apply>
static cudaError_t run_scan(Load ld, Apply ap, int n, int2 *block_sums, size_t cap, int *totals, cudaStream_t s) {
    int nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 0) nb = 1;
    if ((size_t)nb + 1 > cap) return cudaErrorInvalidValue;
    k_scan_reduce<Load><<<nb, SCAN_T, 0, s>>>(ld, n, block_sums);
    if (nb <= SCAN_FUSE) {
        k_scan_apply_fused<Load, Apply><<<nb, SCAN_T, 0, s>>>(ld, ap, n, block_sums, nb, totals);
    } else {
        k_scan_top<<<1, 1024, 0, s>>>(block_sums, nb, totals);
        k_scan_apply<Load, Apply><<<nb, SCAN_T, 0, s>>>(ld, ap, n, block_sums);
    }
    return cudaGetLastError();
}

size_t bucket_scan_blocks(int G) { return (size_t)((G + SCAN_TILE - 1) / SCAN_TILE) + 2; }

// Loader / writer for a plain int array -> exclusive offsets (with the total in out[n]).
struct IntLoad {
    const int *a;
    __device__ int2 operator()(int c) const { return make_int2(a[c], 0); }
};
struct OffsetApply {
    int *out;
    __device__ void operator()(int c, int2 ex, int2 v, int n) const {
        out[c] = ex.x;
        if (c == n - 1) out[n] = ex.x + v.x;
    }
};

// ------------------------------------------------------------------ cell threshold tables

// keys[k] = order key of the smallest double v with floor(fl(fl(v - lo) / w)) >= k,
// k = 0..n, by binary search over the order keys of [-inf, +inf] (the rule is
// monotone in v, false at -inf and true at +inf).  64 steps per threshold.
__global__ void k_axis_thresholds(double lo, double w, int n, unsigned long long *keys) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > n) return;
    const double INF = __longlong_as_double(0x7ff0000000000000LL);
    unsigned long long a = order_key(-INF), b = order_key(INF);
    while (b - a > 1) {
        const unsigned long long m = a + (b - a) / 2;
        if (axis_floor(key_value(m), lo, w) >= (double)k) b = m; else a = m;
    }
    keys[k] = b;
}

cudaError_t launch_thresholds(const GridDev &g, unsigned long long *kx, unsigned long long *ky, cudaStream_t s) {
    k_axis_thresholds<<<(g.nx + 1 + 127) / 128, 128, 0, s>>>(g.x0, g.cw, g.nx, kx);
    k_axis_thresholds<<<(g.ny + 1 + 127) / 128, 128, 0, s>>>(g.y0, g.ch, g.ny, ky);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ point bucketing

// a1: cell id per point and per-cell count; the atomic's return value is the
// point's rank inside its cell, so the scatter needs no second pass.  Points
// whose result is known here (PIP whole-cell results, or the one-pass result
// form's initial -1 / +inf) get their outputs written here.
// Each thread handles UNR points per step so that several independent
// load -> atomic -> store chains are in flight at once: UNR / 2 pairs of
// consecutive points (2q, 2q + 1), q = q0, q0 + T, ... (T = total threads),
// whose keys move as one 16-byte access (the scatter and the result gathers
// take pairs the same way).
constexpr int UNR = 4;

// The step of the strided kernels can exceed the 2^22 headroom below 2^31
// that the element cap leaves, so they count in unsigned 32 bits: an index
// below the cap plus a step below 2^31 stays below 2^32.
// Counter of a point: its cell, or with sub-cell order the cell's sub-cell
// (from FP32 estimates of the position inside the cell: any deterministic
// choice is a valid order); the sentinel G (G * S) outside the grid.
__device__ __forceinline__ int bucket_key(const BucketArgs &a, double x, double y) {
    int ix, iy;
    const int c = point_cell_xy(a.g, x, y, ix, iy);
    if (a.sub_lx + a.sub_ly == 0) return c;
    const int S = 1 << (a.sub_lx + a.sub_ly);
    if (c >= a.g.G) return a.g.G * S;
    const float fx = (approx_float(x) - a.g.x0f) * a.g.icwf - (float)ix;
    const float fy = (approx_float(y) - a.g.y0f) * a.g.ichf - (float)iy;
    const int nx = 1 << a.sub_lx, ny = 1 << a.sub_ly;
    const int sx = min(max((int)(fx * (float)nx), 0), nx - 1);
    const int sy = min(max((int)(fy * (float)ny), 0), ny - 1);
    return c * S + sub_index(sx, sy, a.sub_lx, a.sub_ly);
}

__global__ void k_cell_hist(BucketArgs a) {
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    const unsigned T = gridDim.x * blockDim.x;
    const int lS = a.sub_lx + a.sub_ly;
    const int sentinel = a.g.G << lS;
    unsigned resolved = 0, rhits = 0;
    // A thread takes the pairs of points (2q, 2q + 1), q = q0, q0 + T, ...: the
    // keys of a pair leave in one 16-byte store.
    const unsigned pairs = ((unsigned)a.n + 1u) / 2u;
    for (unsigned q0 = blockIdx.x * blockDim.x + threadIdx.x; q0 < pairs; q0 += (UNR / 2) * T) {
        auto elem = [&](int u) { return 2u * (q0 + (unsigned)(u >> 1) * T) + (unsigned)(u & 1); };
        double2 p[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const unsigned i = elem(u);
            if (i < (unsigned)a.n) p[u] = a.pts[i];
        }
        // key (sentinel outside the grid), rank in its counter; a point of a
        // cell whose result is known (cell_res) gets key sentinel, rank 1
        int c[UNR], r[UNR], v[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const unsigned i = elem(u);
            c[u] = sentinel;
            r[u] = 0;
            v[u] = CELL_REFINE;
            if (i < (unsigned)a.n) {
                c[u] = bucket_key(a, p[u].x, p[u].y);
                if (a.cell_res && c[u] < sentinel) {
                    v[u] = a.cell_res[c[u] >> lS];
                    if (v[u] != CELL_REFINE) {
                        c[u] = sentinel;
                        r[u] = 1;
                    }
                }
                if (c[u] < sentinel && SJ_IN_BOUNDS(c[u] >= 0, BND_BUCKET)) r[u] = atomicAdd(&a.cnt[c[u]], 1);
            }
        }
#pragma unroll
        for (int u = 0; u < UNR; u += 2) {
            const unsigned i = elem(u);
            if (i + 1u < (unsigned)a.n)
                *reinterpret_cast<int4 *>(a.key_rank + i) = make_int4(c[u], r[u], c[u + 1], r[u + 1]);
            else if (i < (unsigned)a.n)
                a.key_rank[i] = make_int2(c[u], r[u]);
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const unsigned i = elem(u);
            if (i < (unsigned)a.n) {
                if (a.cell_res) {
                    if (v[u] != CELL_REFINE) {
                        a.out_id[i] = v[u];
                        ++resolved;
                        rhits += v[u] >= 0;
                    }
                } else {
                    if (a.out_id) a.out_id[i] = -1;
                    if (a.out_d) a.out_d[i] = inf;
                }
            }
        }
    }
    if (a.stats) {
        unsigned long long v[ST_N] = {};
        v[ST_RESOLVED] = __reduce_add_sync(FULL, resolved);
        v[ST_HITS] = __reduce_add_sync(FULL, rhits);
        flush_stats(a.stats, v);
    }
}

// Per cell: (points, work items).  A cell yields ceil(points / ch) items when
// it has both points and candidates.
struct BucketLoad {
    const int *cnt;
    const int *cand_start;
    int ch;
    int lS;           // log2 of the sub-cells per cell (0: none)
    const int *cell_work;
    int budget;
    __device__ int2 operator()(int c) const {
        int np = 0;
        if (lS == 0) {
            np = cnt[c];
        } else {
            const int *q = cnt + ((size_t)c << lS);
            for (int k = 0; k < (1 << lS); ++k) np += q[k];
        }
        int ni = 0;
        if (cand_start && np > 0 && cand_start[c + 1] > cand_start[c]) {
            const int cc = cell_chunk(ch, budget > 0 ? cell_work[c] : 0, budget);
            ni = (np + cc - 1) / cc;
        }
        return make_int2(np, ni);
    }
};
struct BucketApply {
    int *cell_start;
    int2 *items;
    int ch;
    int *cell_base;   // optional: cell_start of cells that yield items, else -1
    const int *cnt;   // with sub-cells: their counters and first slots
    int *sub_start;
    int lS;
    const int *cell_work;
    int budget;
    __device__ void operator()(int c, int2 ex, int2 v, int n) const {
        cell_start[c] = ex.x;
        if (cell_base) cell_base[c] = v.y > 0 ? ex.x : -1;
        if (c == n - 1) cell_start[n] = ex.x + v.x;
        if (items && v.y > 0) {
            const int cc = cell_chunk(ch, budget > 0 ? cell_work[c] : 0, budget);
            for (int t = 0; t < v.y; ++t) items[ex.y + t] = make_int2(c, t * cc);
        }
        if (lS > 0) {
            const size_t b = (size_t)c << lS;
            const bool none = cell_base && v.y == 0;
            int run = ex.x;
            for (int k = 0; k < (1 << lS); ++k) {
                sub_start[b + k] = none ? -1 : run;
                run += cnt[b + k];
            }
        }
    }
};

__global__ void k_scatter(BucketArgs a) {
    const unsigned T = gridDim.x * blockDim.x;
    // pairs of points as in k_cell_hist: one 16-byte load of their keys, one
    // 8-byte store of their slots
    const unsigned pairs = ((unsigned)a.n + 1u) / 2u;
    for (unsigned q0 = blockIdx.x * blockDim.x + threadIdx.x; q0 < pairs; q0 += (UNR / 2) * T) {
        auto elem = [&](int u) { return 2u * (q0 + (unsigned)(u >> 1) * T) + (unsigned)(u & 1); };
        int2 k[UNR];
        double2 p[UNR];
#pragma unroll
        for (int u = 0; u < UNR; u += 2) {
            const unsigned i = elem(u);
            k[u] = k[u + 1] = make_int2(a.g.G << (a.sub_lx + a.sub_ly), 0);
            if (i + 1u < (unsigned)a.n) {
                const int4 kk = *reinterpret_cast<const int4 *>(a.key_rank + i);
                k[u] = make_int2(kk.x, kk.y);
                k[u + 1] = make_int2(kk.z, kk.w);
            } else if (i < (unsigned)a.n) {
                k[u] = a.key_rank[i];
            }
        }
        if (a.spts) {
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                const unsigned i = elem(u);
                if (i < (unsigned)a.n) p[u] = a.pts[i];
            }
        }
        // With a.pos (cell_base set): only points of cells that yield work
        // items get a slot; the others, like points outside the grid, get -1.
        // With sub-cells the key is the sub-cell, whose first slot (or -1) is
        // in sub_start.
        const int lS = a.sub_lx + a.sub_ly;
        const int *base = lS ? a.sub_start : (a.pos ? a.cell_base : a.cell_start);
        const int sentinel = a.g.G << lS;
        int pos[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            pos[u] = (k[u].x >= sentinel && k[u].y == 1) ? POS_DONE : -1;   // result already written, or outside
            if (k[u].x < sentinel) {
                const int b = base[k[u].x];
                pos[u] = b >= 0 ? b + k[u].y : -1;
            }
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            if (pos[u] >= 0 && SJ_IN_BOUNDS(pos[u] < a.n, BND_SCATTER)) {
                a.perm[pos[u]] = (int)elem(u);
                if (a.spts) a.spts[pos[u]] = p[u];
            }
        }
        if (a.pos) {
#pragma unroll
            for (int u = 0; u < UNR; u += 2) {
                const unsigned i = elem(u);
                if (i + 1u < (unsigned)a.n) *reinterpret_cast<int2 *>(a.pos + i) = make_int2(pos[u], pos[u + 1]);
                else if (i < (unsigned)a.n) a.pos[i] = pos[u];
            }
        }
    }
}

// a8 for cell-ordered results (see launch_unsort).
__global__ void k_unsort(const int *pos, const int *res_id, const double *res_d, int n, int *out_id,
                         double *out_d) {
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    const unsigned T = gridDim.x * blockDim.x;
    for (unsigned i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < (unsigned)n; i0 += UNR * T) {
        int j[UNR], id[UNR];
        double d[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) j[u] = (i0 + u * T < (unsigned)n) ? pos[i0 + u * T] : -1;
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            if (j[u] >= 0 && !SJ_IN_BOUNDS(j[u] < n, BND_UNSORT)) j[u] = -1;
            id[u] = j[u] >= 0 ? res_id[j[u]] : -1;
            if (out_d) d[u] = j[u] >= 0 ? res_d[j[u]] : inf;
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const unsigned i = i0 + u * T;
            if (i < (unsigned)n && j[u] != POS_DONE) {
                out_id[i] = id[u];
                if (out_d) out_d[i] = d[u];
            }
        }
    }
}

// Ids only, two consecutive points per thread and step (one 8-byte load of
// their slots, one 8-byte store of their ids unless one of them was answered
// by the cell-id pass); out_id 8-byte aligned.
__global__ void k_unsort_ids2(const int *pos, const int *res_id, int n, int *out_id) {
    const unsigned T = gridDim.x * blockDim.x;
    const unsigned pairs = ((unsigned)n + 1u) / 2u;
    for (unsigned p0 = blockIdx.x * blockDim.x + threadIdx.x; p0 < pairs; p0 += UNR * T) {
        int2 j[UNR], id[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const unsigned p = p0 + u * T, i = 2u * p;
            j[u] = make_int2(POS_DONE, POS_DONE);
            if (p < pairs) {
                if (i + 1u < (unsigned)n) j[u] = *reinterpret_cast<const int2 *>(pos + i);
                else j[u].x = pos[i];
            }
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            if (j[u].x >= 0 && !SJ_IN_BOUNDS(j[u].x < n, BND_UNSORT)) j[u].x = -1;
            if (j[u].y >= 0 && !SJ_IN_BOUNDS(j[u].y < n, BND_UNSORT)) j[u].y = -1;
            id[u].x = j[u].x >= 0 ? res_id[j[u].x] : -1;
            id[u].y = j[u].y >= 0 ? res_id[j[u].y] : -1;
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const unsigned p = p0 + u * T, i = 2u * p;
            if (p >= pairs) continue;
            if (i + 1u < (unsigned)n && j[u].x != POS_DONE && j[u].y != POS_DONE) {
                *reinterpret_cast<int2 *>(out_id + i) = id[u];
            } else {
                if (j[u].x != POS_DONE) out_id[i] = id[u].x;
                if (i + 1u < (unsigned)n && j[u].y != POS_DONE) out_id[i + 1] = id[u].y;
            }
        }
    }
}

static int stream_blocks(long long n, int per_block, int cap) {
    long long b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

// The scan alone (per-cell counts already in a.cnt): cell_start, work items
// and totals.  Grid size depends only on G, so the launch can be replayed.
cudaError_t launch_bucket_scan(const BucketArgs &a, cudaStream_t s) {
    const int lS = a.sub_lx + a.sub_ly;
    return run_scan(BucketLoad{a.cnt, a.cand_start, a.ch, lS, a.cell_work, a.budget},
                    BucketApply{a.cell_start, a.items, a.ch, a.cell_base, a.cnt, a.sub_start, lS, a.cell_work, a.budget},
                    a.g.G, a.block_sums, a.bs_cap, a.totals, s);
}

// Packed records: one gather per point.  FP32X distances widen exactly.
template <typename R>
__global__ void k_unsort_rec(const int *pos, const R *res, int n, int *out_id, double *out_d) {
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    const unsigned T = gridDim.x * blockDim.x;
    for (unsigned i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < (unsigned)n; i0 += UNR * T) {
        int j[UNR];
        R r[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) j[u] = (i0 + u * T < (unsigned)n) ? pos[i0 + u * T] : -1;
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            if (j[u] >= 0 && !SJ_IN_BOUNDS(j[u] < n, BND_UNSORT)) j[u] = -1;
            if (j[u] >= 0) r[u] = res[j[u]];
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const unsigned i = i0 + u * T;
            if (i < (unsigned)n) {
                out_id[i] = j[u] >= 0 ? r[u].id : -1;
                if (out_d) out_d[i] = j[u] >= 0 ? (double)r[u].d : inf;
            }
        }
    }
}

// The same with two consecutive points per thread and step: one 8-byte load of
// their slots and 8- / 16-byte stores of their results, half the memory
// instructions of the form above (whose load / store queue fills first).
// out_id 8-byte and out_d 16-byte aligned.
template <typename R>
__global__ void k_unsort_rec2(const int *pos, const R *res, int n, int *out_id, double *out_d) {
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    const unsigned T = gridDim.x * blockDim.x;
    const unsigned pairs = ((unsigned)n + 1u) / 2u;
    for (unsigned p0 = blockIdx.x * blockDim.x + threadIdx.x; p0 < pairs; p0 += UNR * T) {
        int2 j[UNR];
        R r0[UNR], r1[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const unsigned p = p0 + u * T, i = 2u * p;
            j[u] = make_int2(-1, -1);
            if (p < pairs) {
                if (i + 1u < (unsigned)n) j[u] = *reinterpret_cast<const int2 *>(pos + i);
                else j[u].x = pos[i];
            }
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            if (j[u].x >= 0 && !SJ_IN_BOUNDS(j[u].x < n, BND_UNSORT)) j[u].x = -1;
            if (j[u].y >= 0 && !SJ_IN_BOUNDS(j[u].y < n, BND_UNSORT)) j[u].y = -1;
            if (j[u].x >= 0) r0[u] = res[j[u].x];
            if (j[u].y >= 0) r1[u] = res[j[u].y];
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const unsigned p = p0 + u * T, i = 2u * p;
            if (p >= pairs) continue;
            const int id0 = j[u].x >= 0 ? r0[u].id : -1, id1 = j[u].y >= 0 ? r1[u].id : -1;
            const double d0 = j[u].x >= 0 ? (double)r0[u].d : inf, d1 = j[u].y >= 0 ? (double)r1[u].d : inf;
            if (i + 1u < (unsigned)n) {
                *reinterpret_cast<int2 *>(out_id + i) = make_int2(id0, id1);
                if (out_d) *reinterpret_cast<double2 *>(out_d + i) = make_double2(d0, d1);
            } else {
                out_id[i] = id0;
                if (out_d) out_d[i] = d0;
            }
        }
    }
}

template <typename R>
static cudaError_t launch_unsort_rec(const int *pos, const R *res, int n, int *out_id, double *out_d,
                                     cudaStream_t s) {
    const bool paired = ((uintptr_t)out_id & 7) == 0 && ((uintptr_t)out_d & 15) == 0;
    if (paired) {
        const int nb = stream_blocks(((n + 1) / 2 + UNR - 1) / UNR, 256, 152 * 16);
        k_unsort_rec2<R><<<nb, 256, 0, s>>>(pos, res, n, out_id, out_d);
    } else {
        const int nb = stream_blocks((n + UNR - 1) / UNR, 256, 152 * 16);
        k_unsort_rec<R><<<nb, 256, 0, s>>>(pos, res, n, out_id, out_d);
    }
    return cudaGetLastError();
}

cudaError_t launch_unsort_f(const int *pos, const ResF *res, int n, int *out_id, double *out_d, cudaStream_t s) {
    return launch_unsort_rec(pos, res, n, out_id, out_d, s);
}

cudaError_t launch_unsort_d(const int *pos, const ResD *res, int n, int *out_id, double *out_d, cudaStream_t s) {
    return launch_unsort_rec(pos, res, n, out_id, out_d, s);
}

cudaError_t launch_unsort(const int *pos, const int *res_id, const double *res_d, int n, int *out_id, double *out_d,
                          cudaStream_t s) {
    if (!res_d && !out_d && ((uintptr_t)out_id & 7) == 0) {
        const int nb = stream_blocks(((n + 1) / 2 + UNR - 1) / UNR, 256, 152 * 16);
        k_unsort_ids2<<<nb, 256, 0, s>>>(pos, res_id, n, out_id);
        return cudaGetLastError();
    }
    const int nb = stream_blocks((n + UNR - 1) / UNR, 256, 152 * 16);
    k_unsort<<<nb, 256, 0, s>>>(pos, res_id, res_d, n, out_id, out_d);
    return cudaGetLastError();
}

cudaError_t launch_bucket(const BucketArgs &a, cudaStream_t s) {
    int nb = stream_blocks(a.n, 256, 152 * 32);
    if (a.sub_lx < 0 || a.sub_ly < 0 || a.sub_lx > 3 || a.sub_ly > 3 || ((a.sub_lx + a.sub_ly) && !a.sub_start) ||
        (a.budget > 0 && !a.cell_work))
        return cudaErrorInvalidValue;
    k_cell_hist<<<nb, 256, 0, s>>>(a);
    cudaError_t e = launch_bucket_scan(a, s);
    if (e != cudaSuccess) return e;
    k_scatter<<<nb, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ layer build

// Offsets must start at `first`, end at `last`, and give runs of at least
// `min_size`; a copy narrowed to int32 is written to out.
__global__ void k_check_offsets(const int64_t *off, int64_t n, int64_t min_size, int64_t first, int64_t last,
                                int *out, int *bad) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= n; k += (int64_t)gridDim.x * blockDim.x) {
        int64_t v = off[k];
        if (k == 0 && v != first) atomicOr(bad, 1);
        if (k == n && v != last) atomicOr(bad, 1);
        if (k < n && off[k + 1] - v < min_size) atomicOr(bad, 1);
        if (v < 0 || v > 2147483647LL) atomicOr(bad, 1);
        if (out) out[k] = (int)v;
    }
}

__global__ void k_check_finite(const double2 *v, int n, int *bad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double2 p = v[i];
        if (!(isfinite(p.x) && isfinite(p.y))) atomicOr(bad, 1);
    }
}

// Vertex range of polygon p = rings poly_ring_off[p] .. poly_ring_off[p + 1].
__global__ void k_poly_voff(const int *ring_off, const int *poly_ring_off, int P, int *poly_voff) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p <= P; p += gridDim.x * blockDim.x)
        poly_voff[p] = ring_off[poly_ring_off[p]];
}

// Next and previous vertex within the same ring (the closing edge wraps).
__global__ void k_ring_next(const int *ring_off, int R, int *nxt, int *prv) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
        int b = ring_off[r], e = ring_off[r + 1];
        for (int i = b; i < e; ++i) {
            nxt[i] = (i + 1 < e) ? i + 1 : b;
            prv[i] = (i > b) ? i - 1 : e - 1;
        }
    }
}

// (hi, lo) FP32 split of each vertex, the same split the kernels apply to
// points: hi = x truncated to FP32, lo = fl32(x - hi).
__global__ void k_split(const double2 *v, int n, float4 *vs) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double2 p = v[i];
        float xh, xl, yh, yl;
        split_double(p.x, xh, xl);
        split_double(p.y, yh, yl);
        vs[i] = make_float4(xh, yh, xl, yl);
    }
}

// FP32 frame origins: frame[k] = fl32(lo + k * w), k = 0..n-1.
__global__ void k_frames(double lo, double w, int n, float *frame) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        frame[k] = __double2float_rn(__dadd_rn(lo, __dmul_rn((double)k, w)));
}

cudaError_t launch_frames(const GridDev &g, float *fx, float *fy, cudaStream_t s) {
    k_frames<<<(g.nx + 255) / 256, 256, 0, s>>>(g.x0, g.cw, g.nx, fx);
    k_frames<<<(g.ny + 255) / 256, 256, 0, s>>>(g.y0, g.ch, g.ny, fy);
    return cudaGetLastError();
}

// P2P segment table: for the segment that starts at vertex i of polyline l,
// e = v[i+1] - v[i] and 1 / |e|^2 (0 for a zero-length segment, and for the
// single vertex of a one-vertex polyline, which then acts as a point); the
// fourth component holds l as int bits, or -1 for the last vertex of a
// polyline of two or more vertices (which starts no segment).
__global__ void k_seg_table(const double2 *v, const int *line_off, int L, double2 *e64, double *inv64,
                            float4 *seg32) {
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < L; l += gridDim.x * blockDim.x) {
        int b = line_off[l], e = line_off[l + 1];
        for (int i = b; i < e; ++i) {
            double ex = 0.0, ey = 0.0, inv = 0.0;
            if (i + 1 < e) {
                ex = __dsub_rn(v[i + 1].x, v[i].x);
                ey = __dsub_rn(v[i + 1].y, v[i].y);
                double L2 = __dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey));
                inv = L2 > 0.0 ? __ddiv_rn(1.0, L2) : 0.0;
            }
            e64[i] = make_double2(ex, ey);
            inv64[i] = inv;
            const int owner = (i + 1 < e || e - b == 1) ? l : -1;
            seg32[i] = make_float4(__double2float_rn(ex), __double2float_rn(ey), __double2float_rn(inv),
                                   __int_as_float(owner));
        }
    }
}

// a3: MBB per object, one warp per object; flags an MBB outside the closed
// grid box (bit 2 of *bad).
__global__ void k_mbb(LayerBuildArgs a) {
    int lane = lane_id();
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int o = warp; o < a.nobj; o += nwarps) {
        int b = a.obj_voff[o], e = a.obj_voff[o + 1];
        double xmin = INFINITY, ymin = INFINITY, xmax = -INFINITY, ymax = -INFINITY;
        for (int i = b + lane; i < e; i += 32) {
            double2 p = a.verts[i];
            xmin = fmin(xmin, p.x); xmax = fmax(xmax, p.x);
            ymin = fmin(ymin, p.y); ymax = fmax(ymax, p.y);
        }
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            xmin = fmin(xmin, __shfl_xor_sync(FULL, xmin, s));
            ymin = fmin(ymin, __shfl_xor_sync(FULL, ymin, s));
            xmax = fmax(xmax, __shfl_xor_sync(FULL, xmax, s));
            ymax = fmax(ymax, __shfl_xor_sync(FULL, ymax, s));
        }
        if (lane == 0) {
            a.mbb[o] = Box{xmin, ymin, xmax, ymax};
            if (!(xmin >= a.g.x0 && xmax <= a.g.x1 && ymin >= a.g.y0 && ymax <= a.g.y1)) atomicOr(a.bad, 2);
        }
    }
}

// Largest double below x / smallest above x (x not NaN; infinities kept).
__device__ __forceinline__ double next_down(double x) {
    if (isinf(x)) return x;
    if (x == 0.0) return -4.9406564584124654e-324;
    long long b = __double_as_longlong(x);
    return __longlong_as_double(x > 0.0 ? b - 1 : b + 1);
}
__device__ __forceinline__ double next_up(double x) { return -next_down(-x); }

// a4: cell box of an MBB (P2P: widened by D and rounded outward by one ulp).
__device__ __forceinline__ int4 mbb_cell_box(const LayerBuildArgs &a, Box m) {
    double xlo = m.xmin, ylo = m.ymin, xhi = m.xmax, yhi = m.ymax;
    if (a.kind == KIND_P2P) {
        xlo = next_down(__dsub_rn(xlo, a.D));
        ylo = next_down(__dsub_rn(ylo, a.D));
        xhi = next_up(__dadd_rn(xhi, a.D));
        yhi = next_up(__dadd_rn(yhi, a.D));
    }
    return make_int4(clamped_axis(xlo, a.g.x0, a.g.cw, a.g.nx), clamped_axis(ylo, a.g.y0, a.g.ch, a.g.ny),
                     clamped_axis(xhi, a.g.x0, a.g.cw, a.g.nx), clamped_axis(yhi, a.g.y0, a.g.ch, a.g.ny));
}

__global__ void k_raster_count(LayerBuildArgs a, unsigned long long *total) {
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < a.nobj; o += gridDim.x * blockDim.x) {
        int4 b = mbb_cell_box(a, a.mbb[o]);
        long long n = (long long)(b.z - b.x + 1) * (long long)(b.w - b.y + 1);
        a.obj_cells[o] = n > 2147483647LL ? 2147483647 : (int)n;
        atomicAdd(total, (unsigned long long)n);
    }
}

// Emit (cell, object) pairs and count candidates per cell.
__global__ void k_raster_emit(LayerBuildArgs a, int2 *pairs) {
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < a.nobj; o += gridDim.x * blockDim.x) {
        int4 b = mbb_cell_box(a, a.mbb[o]);
        int k = a.obj_cells[o];
        for (int iy = b.y; iy <= b.w; ++iy)
            for (int ix = b.x; ix <= b.z; ++ix) {
                int c = iy * a.g.nx + ix;
                pairs[k++] = make_int2(c, o);
                atomicAdd(&a.cell_cnt[c], 1);
            }
    }
}

// (cell, id) pairs -> CSR lists (order within a cell fixed by k_cand_sort).
__global__ void k_pair_scatter(const int2 *pairs, int M, const int *start, int *cursor, int *ids) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
        int2 p = pairs[k];
        ids[start[p.x] + atomicAdd(&cursor[p.x], 1)] = p.y;
    }
}

// Sort each cell's ids ascending: Shell sort with Ciura's gap sequence
// (1, 4, 10, 23, 57, 132, 301, 701, then x 2.25), one thread per cell.  Lists
// are short in the common case (one or two gap passes), and a long
// one (a large D makes every object a candidate of every cell) stays near
// n^1.3 instead of the n^2 of plain insertion.
__global__ void k_cand_sort(const int *cand_start, int G, int *cand_ids) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < G; c += gridDim.x * blockDim.x) {
        const int b = cand_start[c], n = cand_start[c + 1] - b;
        int *v = cand_ids + b;
        const int ciura[8] = {1, 4, 10, 23, 57, 132, 301, 701};
        int gaps[32];
        int ng = 0;
        while (ng < 8 && ciura[ng] < n) { gaps[ng] = ciura[ng]; ++ng; }
        if (ng == 8) {
            long long g = 701;
            while (ng < 32 && (g = g * 9 / 4) < n) gaps[ng++] = (int)g;
        }
        for (int t = ng - 1; t >= 0; --t) {
            const int h = gaps[t];
            for (int i = h; i < n; ++i) {
                const int x = v[i];
                int j = i;
                while (j >= h && v[j - h] > x) { v[j] = v[j - h]; j -= h; }
                v[j] = x;
            }
        }
    }
}

// ---- P2P per-cell segment lists.  A point p of cell c is within D of segment
// [a, b] only if p lies in the segment's box widened by D; the cells of that
// box (outward-rounded like the MBB filter above, and the same monotone FP64
// cell rule as the points) therefore include c.  Listing, per cell, the
// segments whose widened box meets it drops only segments farther than D from
// every point of the cell, so the refinement may walk this list instead of all
// segments of the cell's candidate polylines without changing any result.

// Box of the segment starting at vertex i (b = a when e = b - a is zero, which
// in IEEE arithmetic means b == a; a one-vertex polyline is its vertex).
__device__ __forceinline__ Box seg_box(const double2 *v, const double2 *e64, int i) {
    const double2 a = v[i], e = e64[i];
    const double2 b = (e.x == 0.0 && e.y == 0.0) ? a : v[i + 1];
    return Box{fmin(a.x, b.x), fmin(a.y, b.y), fmax(a.x, b.x), fmax(a.y, b.y)};
}

__device__ __forceinline__ long long seg_cell_count(const LayerBuildArgs &a, const float4 *seg32,
                                                    const double2 *e64, int i, int4 &b) {
    if (__float_as_int(seg32[i].w) < 0) return 0;
    b = mbb_cell_box(a, seg_box(a.verts, e64, i));
    return (long long)(b.z - b.x + 1) * (long long)(b.w - b.y + 1);
}

__global__ void k_segcell_count(LayerBuildArgs a, const float4 *seg32, const double2 *e64, int *seg_cells,
                                unsigned long long *total) {
    const int stride = gridDim.x * blockDim.x;
    for (int i0 = blockIdx.x * blockDim.x; i0 < a.V; i0 += stride) {   // warp-uniform trip count
        const int i = i0 + threadIdx.x;
        unsigned long long n = 0;
        if (i < a.V) {
            int4 b;
            const long long c = seg_cell_count(a, seg32, e64, i, b);
            seg_cells[i] = c > 2147483647LL ? 2147483647 : (int)c;
            n = (unsigned long long)c;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(FULL, n, o);
        if (lane_id() == 0 && n) atomicAdd(total, n);
    }
}

__global__ void k_segcell_emit(LayerBuildArgs a, const float4 *seg32, const double2 *e64, const int *seg_off,
                               int *cell_cnt, int2 *pairs) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.V; i += gridDim.x * blockDim.x) {
        int4 b;
        if (seg_cell_count(a, seg32, e64, i, b) == 0) continue;
        int k = seg_off[i];
        for (int iy = b.y; iy <= b.w; ++iy)
            for (int ix = b.x; ix <= b.z; ++ix) {
                const int c = iy * a.g.nx + ix;
                pairs[k++] = make_int2(c, i);
                atomicAdd(&cell_cnt[c], 1);
            }
    }
}

// FP32X staging records of the segment lists, two float4 per entry g of cell c:
//   rec[2g]     = (ax, ay, ex, ey): a relative to the cell's FP32 frame origin
//                 (rel_coord of the (hi, lo) split, the refinement's own rule)
//                 and fl32(b - a);
//   rec[2g + 1] = (fl32(1 / |e|^2), owner polyline id bits,
//                  max(|ax|, |ay|, |ax + ex|, |ay + ey|), segment index bits).
__global__ void k_cseg_records(const int *cseg_start, const int *cseg_ids, int G, int nx, const float *frame_x,
                               const float *frame_y, const float4 *vsplit, const float4 *seg32, float4 *rec) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < G; c += gridDim.x * blockDim.x) {
        const float2 fo = cell_frame(frame_x, frame_y, nx, c);
        for (int g = cseg_start[c]; g < cseg_start[c + 1]; ++g) {
            const int i = cseg_ids[g];
            const float4 v = vsplit[i], e = seg32[i];
            const float ax = rel_coord(v.x, v.z, fo.x), ay = rel_coord(v.y, v.w, fo.y);
            const float bx = ax + e.x, by = ay + e.y;
            const float mag = fmaxf(fmaxf(fabsf(ax), fabsf(ay)), fmaxf(fabsf(bx), fabsf(by)));
            rec[2 * (size_t)g] = make_float4(ax, ay, e.x, e.y);
            rec[2 * (size_t)g + 1] = make_float4(e.z, e.w, mag, __int_as_float(i));
        }
    }
}

// Per-point segment work of each cell of a polyline layer: its list length.
__global__ void k_cell_work_p2p(const int *cseg_start, int G, int *work) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < G; c += gridDim.x * blockDim.x)
        work[c] = cseg_start[c + 1] - cseg_start[c];
}

cudaError_t launch_cell_work_p2p(const int *cseg_start, int G, int *work, cudaStream_t s) {
    k_cell_work_p2p<<<stream_blocks(G, 256, 8192), 256, 0, s>>>(cseg_start, G, work);
    return cudaGetLastError();
}

// Per cell: the number of segments of its candidate polylines (the tests the
// unfiltered refinement of Sec. III.B performs per point; statistics only).
__global__ void k_cell_algo(const int *cand_start, const int *cand_ids, const int *obj_voff, int G, int *cell_algo) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < G; c += gridDim.x * blockDim.x) {
        long long n = 0;
        for (int k = cand_start[c]; k < cand_start[c + 1]; ++k) {
            const int l = cand_ids[k], nv = obj_voff[l + 1] - obj_voff[l];
            n += nv > 1 ? nv - 1 : 1;
        }
        cell_algo[c] = n > 2147483647LL ? 2147483647 : (int)n;
    }
}

// ---- PIP per-(polygon, row) edge lists.  A point p of grid row r has p.y in
// the row's band under the FP64 cell rule; an edge straddles p's horizontal
// line only if min(ay, by) <= p.y < max(ay, by), and the row rule is monotone,
// so r lies between the rows of the edge's two y values.  Listing, for each
// candidate polygon and row, the edges whose row span includes the row drops
// only edges that cannot cross the ray of any point in that row: the parity,
// hence the result, is unchanged.

// Rows of each polygon's MBB: prow_n[P] = r1 - r0 + 1 (scanned into the slot
// bases afterwards), prow_r0[P] = r0, and the total in *total.
__global__ void k_prow_count(LayerBuildArgs a, int *prow_n, int *prow_r0, unsigned long long *total) {
    const int stride = gridDim.x * blockDim.x;
    for (int p0 = blockIdx.x * blockDim.x; p0 < a.nobj; p0 += stride) {   // warp-uniform trip count
        const int P = p0 + threadIdx.x;
        unsigned long long n = 0;
        if (P < a.nobj) {
            const Box m = a.mbb[P];
            const int r0 = clamped_axis(m.ymin, a.g.y0, a.g.ch, a.g.ny);
            const int r1 = clamped_axis(m.ymax, a.g.y0, a.g.ch, a.g.ny);
            prow_r0[P] = r0;
            prow_n[P] = r1 - r0 + 1;
            n = (unsigned long long)(r1 - r0 + 1);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(FULL, n, o);
        if (lane_id() == 0 && n) atomicAdd(total, n);
    }
}

// One warp per polygon, lanes over its edges (vertex i -> nxt[i]).  Count pass
// (ids == nullptr): cnt[slot] += 1 for every row of the edge, total in *total.
// Emit pass: ids[start[slot] + cursor[slot]++] = i.
__global__ void k_prow_edges(LayerBuildArgs a, const int *nxt, const int *prow_base, const int *prow_r0, int *cnt,
                             unsigned long long *total, const int *start, int *cursor, int *ids) {
    const int lane = lane_id();
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int P = warp; P < a.nobj; P += nwarps) {
        const int b = a.obj_voff[P], e = a.obj_voff[P + 1];
        const int base = prow_base[P] - prow_r0[P];
        unsigned long long n = 0;
        for (int i = b + lane; i < e; i += 32) {
            const double ya = a.verts[i].y, yb = a.verts[nxt[i]].y;
            const int ra = clamped_axis(fmin(ya, yb), a.g.y0, a.g.ch, a.g.ny);
            const int rb = clamped_axis(fmax(ya, yb), a.g.y0, a.g.ch, a.g.ny);
            for (int r = ra; r <= rb; ++r) {
                if (ids) ids[start[base + r] + atomicAdd(&cursor[base + r], 1)] = i;
                else atomicAdd(&cnt[base + r], 1);
            }
            n += (unsigned long long)(rb - ra + 1);
        }
        if (!ids) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(FULL, n, o);
            if (lane == 0) atomicAdd(total, n);
        }
    }
}

// Host side of the layer build steps that the API file sequences.
cudaError_t launch_check_offsets(const int64_t *off, int64_t n, int64_t min_size, int64_t first, int64_t last, int *out,
                                 int *bad, cudaStream_t s) {
    k_check_offsets<<<stream_blocks(n + 1, 256, 4096), 256, 0, s>>>(off, n, min_size, first, last, out, bad);
    return cudaGetLastError();
}
cudaError_t launch_check_finite(const double2 *v, int n, int *bad, cudaStream_t s) {
    k_check_finite<<<stream_blocks(n, 256, 4096), 256, 0, s>>>(v, n, bad);
    return cudaGetLastError();
}
cudaError_t launch_pip_topology(const int *ring_off, int R, const int *poly_ring_off, int P, int *poly_voff, int *nxt,
                                int *prv, cudaStream_t s) {
    k_poly_voff<<<stream_blocks(P + 1, 256, 4096), 256, 0, s>>>(ring_off, poly_ring_off, P, poly_voff);
    k_ring_next<<<stream_blocks(R, 128, 4096), 128, 0, s>>>(ring_off, R, nxt, prv);
    return cudaGetLastError();
}
cudaError_t launch_split(const double2 *v, int n, float4 *vs, cudaStream_t s) {
    k_split<<<stream_blocks(n, 256, 4096), 256, 0, s>>>(v, n, vs);
    return cudaGetLastError();
}
cudaError_t launch_seg_table(const double2 *v, const int *line_off, int L, double2 *e64, double *inv64, float4 *seg32,
                             cudaStream_t s) {
    k_seg_table<<<stream_blocks(L, 128, 4096), 128, 0, s>>>(v, line_off, L, e64, inv64, seg32);
    return cudaGetLastError();
}
cudaError_t launch_mbb(const LayerBuildArgs &a, cudaStream_t s) {
    k_mbb<<<stream_blocks((long long)a.nobj * 32, 256, 4096), 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_raster_count(const LayerBuildArgs &a, unsigned long long *total, cudaStream_t s) {
    k_raster_count<<<stream_blocks(a.nobj, 256, 4096), 256, 0, s>>>(a, total);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // Counts -> exclusive offsets in place: every tile loads its counts into
    // registers before it writes, and tiles write only their own indices.
    return run_scan(IntLoad{a.obj_cells}, OffsetApply{a.obj_cells}, a.nobj, a.block_sums, a.bs_cap, a.totals, s);
}
cudaError_t launch_raster_emit(const LayerBuildArgs &a, int2 *pairs, int M, int *cand_ids, cudaStream_t s) {
    k_raster_emit<<<stream_blocks(a.nobj, 128, 4096), 128, 0, s>>>(a, pairs);
    cudaError_t e = run_scan(IntLoad{a.cell_cnt}, OffsetApply{a.cand_start}, a.g.G, a.block_sums, a.bs_cap, a.totals, s);
    if (e != cudaSuccess) return e;
    k_pair_scatter<<<stream_blocks(M, 256, 4096), 256, 0, s>>>(pairs, M, a.cand_start, a.cursor, cand_ids);
    k_cand_sort<<<stream_blocks(a.g.G, 128, 8192), 128, 0, s>>>(a.cand_start, a.g.G, cand_ids);
    return cudaGetLastError();
}

// Segment lists, step 1: cells per segment (into seg_off[V + 1]), their total,
// and the exclusive offsets in place (V > 0; a.block_sums sized for V).
cudaError_t launch_segcell_count(const LayerBuildArgs &a, const float4 *seg32, const double2 *e64, int *seg_off,
                                 unsigned long long *total, cudaStream_t s) {
    k_segcell_count<<<stream_blocks(a.V, 256, 4096), 256, 0, s>>>(a, seg32, e64, seg_off, total);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return run_scan(IntLoad{seg_off}, OffsetApply{seg_off}, a.V, a.block_sums, a.bs_cap, a.totals, s);
}

// Step 2: (cell, segment) pairs, per-cell counts (a.cell_cnt zeroed), CSR
// offsets cseg_start, the lists (a.cursor zeroed) sorted by segment index, and
// the per-cell candidate segment counts.
cudaError_t launch_segcell_emit(const LayerBuildArgs &a, const float4 *seg32, const double2 *e64, const int *seg_off,
                                int2 *pairs, int MS, const int *cand_ids, int *cseg_start, int *cseg_ids,
                                int *cell_algo, cudaStream_t s) {
    k_segcell_emit<<<stream_blocks(a.V, 128, 4096), 128, 0, s>>>(a, seg32, e64, seg_off, a.cell_cnt, pairs);
    cudaError_t e = run_scan(IntLoad{a.cell_cnt}, OffsetApply{cseg_start}, a.g.G, a.block_sums, a.bs_cap, a.totals, s);
    if (e != cudaSuccess) return e;
    k_pair_scatter<<<stream_blocks(MS, 256, 4096), 256, 0, s>>>(pairs, MS, cseg_start, a.cursor, cseg_ids);
    k_cand_sort<<<stream_blocks(a.g.G, 128, 8192), 128, 0, s>>>(cseg_start, a.g.G, cseg_ids);
    k_cell_algo<<<stream_blocks(a.g.G, 128, 8192), 128, 0, s>>>(a.cand_start, cand_ids, a.obj_voff, a.g.G, cell_algo);
    return cudaGetLastError();
}

// PIP row lists, step 1: rows per polygon and the slot bases (prow_base[P + 1],
// exclusive scan in place); a.block_sums sized for max(G, P, slots).
cudaError_t launch_prow_count(const LayerBuildArgs &a, int *prow_base, int *prow_r0, unsigned long long *total,
                              cudaStream_t s) {
    k_prow_count<<<stream_blocks(a.nobj, 256, 4096), 256, 0, s>>>(a, prow_base, prow_r0, total);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return run_scan(IntLoad{prow_base}, OffsetApply{prow_base}, a.nobj, a.block_sums, a.bs_cap, a.totals, s);
}

// Step 2 (count): edges per slot into cnt (zeroed), total entries in *total.
cudaError_t launch_prow_edge_count(const LayerBuildArgs &a, const int *nxt, const int *prow_base, const int *prow_r0,
                                   int *cnt, unsigned long long *total, cudaStream_t s) {
    k_prow_edges<<<stream_blocks((long long)a.nobj * 32, 256, 4096), 256, 0, s>>>(a, nxt, prow_base, prow_r0, cnt,
                                                                                 total, nullptr, nullptr, nullptr);
    return cudaGetLastError();
}

// Step 3 (emit): slot ranges prow_start[slots + 1] from cnt, then the lists
// (cursor zeroed).  Order within a list is not fixed (parity is a XOR).
cudaError_t launch_prow_edge_emit(const LayerBuildArgs &a, const int *nxt, const int *prow_base, const int *prow_r0,
                                  const int *cnt, int slots, int *prow_start, int *cursor, int *pedge_ids,
                                  cudaStream_t s) {
    cudaError_t e = run_scan(IntLoad{cnt}, OffsetApply{prow_start}, slots, a.block_sums, a.bs_cap, a.totals, s);
    if (e != cudaSuccess) return e;
    k_prow_edges<<<stream_blocks((long long)a.nobj * 32, 256, 4096), 256, 0, s>>>(a, nxt, prow_base, prow_r0, nullptr,
                                                                                 nullptr, prow_start, cursor,
                                                                                 pedge_ids);
    return cudaGetLastError();
}

cudaError_t launch_cseg_records(const int *cseg_start, const int *cseg_ids, const GridDev &g, const float *frame_x,
                                const float *frame_y, const float4 *vsplit, const float4 *seg32, float4 *rec,
                                cudaStream_t s) {
    k_cseg_records<<<stream_blocks(g.G, 128, 8192), 128, 0, s>>>(cseg_start, cseg_ids, g.G, g.nx, frame_x, frame_y,
                                                                vsplit, seg32, rec);
    return cudaGetLastError();
}

// FP32X staging records of the PIP row lists: the (hi, lo) splits of both ends
// of each listed edge, so that staging reads one contiguous record per entry.
__global__ void k_prow_records(const int *pedge_ids, long long ME, const int *nxt, const float4 *vsplit, float4 *rec) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ME;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = pedge_ids[e];
        rec[2 * e] = vsplit[i];
        rec[2 * e + 1] = vsplit[nxt[i]];
    }
}

cudaError_t launch_prow_records(const int *pedge_ids, long long ME, const int *nxt, const float4 *vsplit,
                                float4 *rec, cudaStream_t s) {
    k_prow_records<<<stream_blocks(ME, 256, 8192), 256, 0, s>>>(pedge_ids, ME, nxt, vsplit, rec);
    return cudaGetLastError();
}

// 64-bit sum of cnt[0..n) added to *total (checks a list's size before its
// 32-bit offsets are taken).
__global__ void k_sum64(const int *cnt, int n, unsigned long long *total) {
    unsigned long long v = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v += (unsigned)cnt[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(total, v);
}

cudaError_t launch_sum64(const int *cnt, int n, unsigned long long *total, cudaStream_t s) {
    k_sum64<<<stream_blocks(n, 256, 4096), 256, 0, s>>>(cnt, n, total);
    return cudaGetLastError();
}

// Exclusive offsets out[0..n] of the counts cnt[0..n) (out[n] = total, also in
// totals[0]); block_sums holds cap entries (bucket_scan_blocks(n)).
cudaError_t launch_offsets(const int *cnt, int n, int *out, int2 *block_sums, size_t cap, int *totals,
                           cudaStream_t s) {
    return run_scan(IntLoad{cnt}, OffsetApply{out}, n, block_sums, cap, totals, s);
}

}  // namespace sj
