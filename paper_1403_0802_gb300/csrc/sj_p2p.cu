// sj_p2p.cu -- P2P refinement (Sec. III.B, Fig. 2): for every point of a work
// item, the candidate polyline at the smallest distance, accepted when the
// distance is within the window D.
//
// Work decomposition: one warp per (cell, point-chunk) item.  For each
// candidate polyline, in id order, the warp stages its segments in shared
// memory (start point a, direction e = b - a, 1 / |e|^2) and splits its lanes
// into point groups of SG lanes; a group's lanes stride over the segments,
// keep a running minimum of the squared distance, and fold it with SG-lane
// shuffles (the cross-lane min of the paper's vertex-per-lane alternative,
// Sec. III.B).  Per point the warp keeps the best (distance, id) and the
// second-best distance of another polyline in shared memory.
//
// The point-to-segment distance is the two-case distance of Fig. 2 written as
// the clamped projection: t = clamp(((p - a) . e) / |e|^2, 0, 1) and
// d^2 = |p - a - t e|^2 (t = 0 or 1 gives the nearer end, 0 < t < 1 the
// perpendicular foot; a zero-length segment has 1 / |e|^2 = 0, hence t = 0).
//
// Two arithmetic forms:
//   FP64   -- the formula in FP64; agrees with the two-case FP64 evaluation to
//             a few ulps of the coordinates' magnitude.
//   FP32X  -- cell-relative FP32 coordinates; every (point, polyline) distance
//             carries a bound E = 64 u max|coordinate| + 4 eps.  A point is
//             final only when its best polyline is separated from the runner-up
//             by more than the two bounds and its distance from D by more than
//             its bound; otherwise it is queued and redone in FP64
//             (k_p2p_recheck).
#include <cuda_runtime.h>

#include <type_traits>

#include "sj_internal.cuh"

namespace sj {

constexpr int P2P_WARPS = 4;
constexpr int SMAX32 = 256, SMAX64 = 128;

template <bool FP32>
struct P2PSmem;

template <>
struct P2PSmem<true> {
    float ax[SMAX32], ay[SMAX32], ex[SMAX32], ey[SMAX32], inv[SMAX32];
    float px[MAX_CH], py[MAX_CH], cur[MAX_CH], d1[MAX_CH], d2[MAX_CH], e1[MAX_CH], e2[MAX_CH];
    int id1[MAX_CH];
};

template <>
struct P2PSmem<false> {
    double ax[SMAX64], ay[SMAX64], ex[SMAX64], ey[SMAX64], inv[SMAX64];
    double px[MAX_CH], py[MAX_CH], cur[MAX_CH], d1[MAX_CH];
    int id1[MAX_CH];
};

// Squared distance from p to the segment (a, a + e) by the clamped projection.
__device__ __forceinline__ float seg_d2(float px, float py, float ax, float ay, float ex, float ey, float inv) {
    float dx = px - ax, dy = py - ay;
    float t = __saturatef(fmaf(ex, dx, ey * dy) * inv);
    float qx = fmaf(-t, ex, dx), qy = fmaf(-t, ey, dy);
    return fmaf(qx, qx, qy * qy);
}

__device__ __forceinline__ double seg_d2(double px, double py, double ax, double ay, double ex, double ey,
                                         double inv) {
    double dx = __dsub_rn(px, ax), dy = __dsub_rn(py, ay);
    double t = __dmul_rn(__fma_rn(ex, dx, __dmul_rn(ey, dy)), inv);
    t = fmin(fmax(t, 0.0), 1.0);
    double qx = __fma_rn(-t, ex, dx), qy = __fma_rn(-t, ey, dy);
    return __fma_rn(qx, qx, __dmul_rn(qy, qy));
}

template <typename T>
__device__ __forceinline__ T tmin(T a, T b);
template <>
__device__ __forceinline__ float tmin(float a, float b) { return fminf(a, b); }
template <>
__device__ __forceinline__ double tmin(double a, double b) { return fmin(a, b); }

template <bool FP32>
__global__ void __launch_bounds__(P2P_WARPS * 32) k_p2p_refine(RefineArgs a) {
    using T = typename std::conditional<FP32, float, double>::type;
    constexpr int SMAX = FP32 ? SMAX32 : SMAX64;
    __shared__ P2PSmem<FP32> smem[P2P_WARPS];
    const int lane = lane_id(), w = threadIdx.x >> 5;
    P2PSmem<FP32> &s = smem[w];
    const int n_items = *a.n_items;
    const T INF = (T)__longlong_as_double(0x7ff0000000000000LL);
    unsigned long long c_pairs = 0, c_tests = 0;
    unsigned long long c_items = 0;
    unsigned c_fb = 0, c_hits = 0;

    for (int it = blockIdx.x * P2P_WARPS + w; it < n_items; it += gridDim.x * P2P_WARPS) {
        ++c_items;
        const int2 item = a.items[it];
        const int c = item.x;
        const int j0 = a.cell_start[c] + item.y;
        const int np = min(a.ch, a.cell_start[c + 1] - j0);
        double2 fr = make_double2(0.0, 0.0);
        if (FP32) fr = cell_frame(a.g, c);
        const float fox = (float)fr.x, foy = (float)fr.y;

        for (int q = lane; q < np; q += 32) {
            double2 p = a.spts[j0 + q];
            if constexpr (FP32) {
                s.px[q] = __double2float_rn(__dsub_rn(p.x, fr.x));
                s.py[q] = __double2float_rn(__dsub_rn(p.y, fr.y));
                s.d2[q] = INF;
                s.e1[q] = 0.0f;
                s.e2[q] = 0.0f;
            } else {
                s.px[q] = p.x;
                s.py[q] = p.y;
            }
            s.cur[q] = INF;
            s.d1[q] = INF;
            s.id1[q] = -1;
        }
        __syncwarp();

        const int k1 = a.cand_start[c + 1];
        for (int k = a.cand_start[c]; k < k1; ++k) {
            const int lid = a.cand_ids[k];
            const int vb = a.obj_voff[lid], nv = a.obj_voff[lid + 1] - vb;
            const int nseg = nv > 1 ? nv - 1 : 1;
            c_pairs += np;
            c_tests += (unsigned long long)np * (unsigned long long)nseg;
            float mag = 0.0f;   // FP32X: largest |cell-relative coordinate| of the polyline
            for (int s0 = 0; s0 < nseg; s0 += SMAX) {
                const int ns = min(SMAX, nseg - s0);
                for (int t = lane; t < ns; t += 32) {
                    const int i = vb + s0 + t;
                    if constexpr (FP32) {
                        const float4 v = a.vsplit[i];
                        const float2 e = a.seg_e32[i];
                        const float ax = __fadd_rn(__fsub_rn(v.x, fox), v.z);
                        const float ay = __fadd_rn(__fsub_rn(v.y, foy), v.w);
                        s.ax[t] = ax; s.ay[t] = ay; s.ex[t] = e.x; s.ey[t] = e.y;
                        s.inv[t] = a.seg_inv32[i];
                        mag = fmaxf(mag, fmaxf(fmaxf(fabsf(ax), fabsf(ay)),
                                               fmaxf(fabsf(ax + e.x), fabsf(ay + e.y))));
                    } else {
                        const double2 v = a.verts[i];
                        const double2 e = a.seg_e64[i];
                        s.ax[t] = v.x; s.ay[t] = v.y; s.ex[t] = e.x; s.ey[t] = e.y;
                        s.inv[t] = a.seg_inv64[i];
                    }
                }
                __syncwarp();
                const int sg = choose_group(np, ns, 1);
                const int lg = __ffs(sg) - 1, pg = 32 >> lg;
                const int sub = lane & (sg - 1), grp = lane >> lg;
                for (int q0 = 0; q0 < np; q0 += pg) {
                    const int q = q0 + grp;
                    T m = INF;
                    if (q < np) {
                        const T px = s.px[q], py = s.py[q];
                        for (int t = sub; t < ns; t += sg)
                            m = tmin(m, seg_d2(px, py, s.ax[t], s.ay[t], s.ex[t], s.ey[t], s.inv[t]));
                    }
                    for (int o = sg >> 1; o > 0; o >>= 1) m = tmin(m, __shfl_xor_sync(FULL, m, o));
                    if (sub == 0 && q < np) s.cur[q] = tmin(s.cur[q], m);
                }
                __syncwarp();
            }
            if constexpr (FP32) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) mag = fmaxf(mag, __shfl_xor_sync(FULL, mag, o));
            }
            for (int q = lane; q < np; q += 32) {
                const T d = sqrt(s.cur[q]);
                s.cur[q] = INF;
                if constexpr (FP32) {
                    const float m = fmaxf(mag, fmaxf(fabsf(s.px[q]), fabsf(s.py[q])));
                    const float e = fmaf(64.0f * U32, m, 4.0f * a.eps_abs);
                    if (d < s.d1[q]) {
                        s.d2[q] = s.d1[q]; s.e2[q] = s.e1[q];
                        s.d1[q] = d; s.e1[q] = e; s.id1[q] = lid;
                    } else if (d < s.d2[q]) {
                        s.d2[q] = d; s.e2[q] = e;
                    }
                } else {
                    if (d < s.d1[q]) { s.d1[q] = d; s.id1[q] = lid; }
                }
            }
            __syncwarp();
        }
        for (int q = lane; q < np; q += 32) {
            const int id = s.id1[q];
            if (id < 0) continue;
            const double d = (double)s.d1[q];
            if constexpr (FP32) {
                const double e1 = s.e1[q], e2 = s.e2[q];
                const double tiny = 1e-12 * (a.D + 1.0);
                if (d - e1 > a.D + tiny) continue;                                  // certainly outside the window
                const bool in_window = d + e1 < a.D - tiny;
                const bool separated = (double)s.d2[q] - d > e1 + e2 + tiny;       // d2 = inf: no runner-up
                if (!(in_window && separated)) {
                    const int slot = atomicAdd(a.n_fb, 1);
                    a.fb[slot] = make_int2(j0 + q, c);
                    ++c_fb;
                    continue;
                }
            } else {
                if (!(d <= a.D)) continue;
            }
            const int i = a.perm[j0 + q];
            a.out_id[i] = id;
            if (a.out_d) a.out_d[i] = d;
            ++c_hits;
        }
        __syncwarp();
    }
    if (a.stats) {
        c_fb = __reduce_add_sync(FULL, c_fb);
        c_hits = __reduce_add_sync(FULL, c_hits);
        if (lane == 0) {
            atomicAdd(&a.stats[ST_ITEMS], c_items);
            atomicAdd(&a.stats[ST_PAIRS], c_pairs);
            atomicAdd(&a.stats[ST_TESTS], c_tests);
            atomicAdd(&a.stats[ST_FALLBACK], (unsigned long long)c_fb);
            atomicAdd(&a.stats[ST_HITS], (unsigned long long)c_hits);
        }
    }
}

// FP64 recomputation of the points the FP32X pass could not certify: one warp
// per point, lanes over each candidate's segments, warp min per polyline.
__global__ void __launch_bounds__(256) k_p2p_recheck(RefineArgs a) {
    const int lane = lane_id();
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int n = *a.n_fb;
    const double INF = __longlong_as_double(0x7ff0000000000000LL);
    unsigned c_hits = 0;
    for (int f = warp; f < n; f += nwarps) {
        const int2 e = a.fb[f];
        const int j = e.x, c = e.y;
        const double2 p = a.spts[j];
        double best = INF;
        int bid = -1;
        for (int k = a.cand_start[c]; k < a.cand_start[c + 1]; ++k) {
            const int lid = a.cand_ids[k];
            const int vb = a.obj_voff[lid], nv = a.obj_voff[lid + 1] - vb;
            const int nseg = nv > 1 ? nv - 1 : 1;
            double m = INF;
            for (int t = lane; t < nseg; t += 32) {
                const int i = vb + t;
                const double2 v = a.verts[i], ev = a.seg_e64[i];
                m = fmin(m, seg_d2(p.x, p.y, v.x, v.y, ev.x, ev.y, a.seg_inv64[i]));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(FULL, m, o));
            const double d = sqrt(m);
            if (d < best) { best = d; bid = lid; }
        }
        if (lane == 0 && bid >= 0 && best <= a.D) {
            const int i = a.perm[j];
            a.out_id[i] = bid;
            if (a.out_d) a.out_d[i] = best;
            ++c_hits;
        }
    }
    if (a.stats) {
        c_hits = __reduce_add_sync(FULL, c_hits);
        if (lane == 0 && c_hits) atomicAdd(&a.stats[ST_HITS], (unsigned long long)c_hits);
    }
}

cudaError_t launch_p2p_refine(const RefineArgs &a, int form, int warps_per_block, int blocks, cudaStream_t s) {
    (void)warps_per_block;
    if (form == SJ_FP32X)
        k_p2p_refine<true><<<blocks, P2P_WARPS * 32, 0, s>>>(a);
    else
        k_p2p_refine<false><<<blocks, P2P_WARPS * 32, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_p2p_recheck(const RefineArgs &a, int blocks, cudaStream_t s) {
    k_p2p_recheck<<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

int p2p_blocks_per_sm(int form) {
    int n = 0;
    if (form == SJ_FP32X)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_p2p_refine<true>, P2P_WARPS * 32, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_p2p_refine<false>, P2P_WARPS * 32, 0);
    return n > 0 ? n : 1;
}

}  // namespace sj
