// sj_p2p.cu -- P2P refinement (Sec. III.B, Fig. 2): for every point of a work
// item, the candidate polyline at the smallest distance, accepted when the
// distance is within the window D.
//
// Work decomposition: one warp per (cell, point-chunk) item.  The warp first
// reads the metadata of up to 32 candidate polylines at once (one per lane),
// warp-scans their segment counts, and stages the concatenated segments of
// all of them in shared memory in one strided pass (start point a, direction
// e = b - a, 1 / |e|^2, polyline id) -- so the L2 round trips of different
// candidates overlap instead of forming a chain per candidate.  It then splits
// its lanes into point groups of SG lanes (SG chosen so that np points x S
// segments fill the warp); each lane strides over the segments keeping a
// running "top-2" -- the best (squared distance, polyline) and the best
// distance of any *other* polyline -- and the SG lanes of a group fold their
// top-2s with shuffles (the cross-lane min of the vertex-per-lane alternative
// of Sec. III.B).  Per point the result lives in shared memory across chunks.
//
// The point-to-segment distance is the two-case distance of Fig. 2 written as
// the clamped projection: t = clamp(((p - a) . e) / |e|^2, 0, 1) and
// d^2 = |p - a - t e|^2 (t = 0 or 1 gives the nearer end, 0 < t < 1 the
// perpendicular foot; a zero-length segment has 1 / |e|^2 = 0, hence t = 0).
//
// Two arithmetic forms:
//   FP64   -- the formula in FP64 (ties of equal squared distance go to the
//             smaller id); agrees with the two-case FP64 evaluation to a few
//             ulps of the coordinates' magnitude.
//   FP32X  -- cell-relative FP32 coordinates; every (point, polyline) distance
//             carries the bound E = 64 u max|coordinate| + 4 eps (u = 2^-24,
//             max over the point and every staged vertex of the item).  A
//             point is final only when its best polyline is ahead of the
//             runner-up by more than 2E and its distance differs from D by
//             more than E; otherwise it is queued and redone in FP64
//             (k_p2p_recheck), so ids agree with FP64 up to exact ties.
#include <cuda_runtime.h>

#include <type_traits>

#include "sj_internal.cuh"

namespace sj {

constexpr int P2P_WARPS = 4;

template <bool FP32>
struct P2PCfg {
    using T = float;
    static constexpr int SMAX = 512;   // staged segments per chunk per warp
};
template <>
struct P2PCfg<false> {
    using T = double;
    static constexpr int SMAX = 256;
};

template <bool FP32>
struct P2PSmem {
    using T = typename P2PCfg<FP32>::T;
    static constexpr int SMAX = P2PCfg<FP32>::SMAX;
    T ax[SMAX], ay[SMAX], ex[SMAX], ey[SMAX], inv[SMAX];
    int sid[SMAX];
    int coff[33], cid[32], cvb[32];   // candidate group: segment offsets, ids, first vertices
    T px[MAX_CH], py[MAX_CH], b1[MAX_CH], b2[MAX_CH];
    int i1[MAX_CH];
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

// Running result of one point over a set of segments: b1 = smallest squared
// distance, i1 = its polyline, b2 = smallest squared distance of any segment of
// another polyline (FP32X certificate; unused in FP64).
template <typename T>
struct Best {
    T b1, b2;
    int i1;
};

template <bool FP32, typename T>
__device__ __forceinline__ void consider(Best<T> &s, T d, int l) {
    if constexpr (FP32) {
        if (d < s.b1) {
            s.b2 = (l != s.i1) ? s.b1 : s.b2;
            s.b1 = d;
            s.i1 = l;
        } else if (d < s.b2 && l != s.i1) {
            s.b2 = d;
        }
    } else {
        if (d < s.b1 || (d == s.b1 && l < s.i1)) {
            s.b1 = d;
            s.i1 = l;
        }
    }
}

// Result over the union of two segment sets (commutative and associative).
template <bool FP32, typename T>
__device__ __forceinline__ Best<T> merge(Best<T> A, Best<T> B) {
    Best<T> r;
    if constexpr (FP32) {
        if (A.i1 == B.i1) {
            r.b1 = fminf(A.b1, B.b1); r.i1 = A.i1; r.b2 = fminf(A.b2, B.b2);
        } else if (B.b1 < A.b1 || (B.b1 == A.b1 && B.i1 < A.i1)) {
            r.b1 = B.b1; r.i1 = B.i1; r.b2 = fminf(B.b2, A.b1);
        } else {
            r.b1 = A.b1; r.i1 = A.i1; r.b2 = fminf(A.b2, B.b1);
        }
    } else {
        r = (B.b1 < A.b1 || (B.b1 == A.b1 && B.i1 < A.i1)) ? B : A;
    }
    return r;
}

template <bool FP32, typename T>
__device__ __forceinline__ Best<T> shfl_best(const Best<T> &s, int o) {
    Best<T> r;
    r.b1 = __shfl_xor_sync(FULL, s.b1, o);
    r.i1 = __shfl_xor_sync(FULL, s.i1, o);
    r.b2 = FP32 ? __shfl_xor_sync(FULL, s.b2, o) : s.b2;
    return r;
}

template <bool FP32>
__global__ void __launch_bounds__(P2P_WARPS * 32) k_p2p_refine(RefineArgs a) {
    using T = typename P2PCfg<FP32>::T;
    constexpr int SMAX = P2PCfg<FP32>::SMAX;
    extern __shared__ __align__(16) unsigned char p2p_smem_raw[];
    const int lane = lane_id(), w = threadIdx.x >> 5;
    P2PSmem<FP32> &s = reinterpret_cast<P2PSmem<FP32> *>(p2p_smem_raw)[w];
    const int n_items = *a.n_items;
    const T INF = (T)__longlong_as_double(0x7ff0000000000000LL);
    unsigned long long c_pairs = 0, c_tests = 0, c_items = 0;
    unsigned c_fb = 0, c_hits = 0;

    for (int it = blockIdx.x * P2P_WARPS + w; it < n_items; it += gridDim.x * P2P_WARPS) {
        ++c_items;
        const int2 item = a.items[it];
        const int c = item.x;
        const int j0 = a.cell_start[c] + item.y;
        const int np = min(a.ch, a.cell_start[c + 1] - j0);
        const int k0 = a.cand_start[c], k1 = a.cand_start[c + 1];
        double2 fr = make_double2(0.0, 0.0);
        if (FP32) fr = cell_frame(a.g, c);
        const float fox = (float)fr.x, foy = (float)fr.y;

        for (int q = lane; q < np; q += 32) {
            double2 p = a.spts[j0 + q];
            if constexpr (FP32) {
                s.px[q] = __double2float_rn(__dsub_rn(p.x, fr.x));
                s.py[q] = __double2float_rn(__dsub_rn(p.y, fr.y));
            } else {
                s.px[q] = p.x;
                s.py[q] = p.y;
            }
            s.b1[q] = INF;
            s.b2[q] = INF;
            s.i1[q] = -1;
        }
        float mag = 0.0f;   // FP32X: largest |cell-relative coordinate| staged for this item
        c_pairs += (unsigned long long)np * (unsigned long long)(k1 - k0);

        for (int kg = k0; kg < k1; kg += 32) {
            // candidate group: one polyline per lane, segment counts scanned
            const int nc = min(32, k1 - kg);
            int lid = 0, vb = 0, nseg = 0;
            if (lane < nc) {
                lid = a.cand_ids[kg + lane];
                vb = a.obj_voff[lid];
                const int nv = a.obj_voff[lid + 1] - vb;
                nseg = nv > 1 ? nv - 1 : 1;
            }
            int incl = nseg;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += v;
            }
            const int S = __shfl_sync(FULL, incl, 31);
            __syncwarp();   // previous chunk's readers are done with the staging area
            if (lane < nc) {
                s.coff[lane] = incl - nseg;
                s.cid[lane] = lid;
                s.cvb[lane] = vb;
            }
            if (lane == 0) s.coff[nc] = S;
            __syncwarp();
            c_tests += (unsigned long long)np * (unsigned long long)S;

            for (int s0 = 0; s0 < S; s0 += SMAX) {
                const int ns = min(SMAX, S - s0);
                for (int t = lane; t < ns; t += 32) {
                    const int g = s0 + t;
                    int lo = 0, hi = nc;   // coff[lo] <= g < coff[hi]
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (s.coff[mid] <= g) lo = mid; else hi = mid;
                    }
                    const int i = s.cvb[lo] + (g - s.coff[lo]);
                    s.sid[t] = s.cid[lo];
                    if constexpr (FP32) {
                        const float4 v = a.vsplit[i];
                        const float2 e = a.seg_e32[i];
                        const float ax = __fadd_rn(__fsub_rn(v.x, fox), v.z);
                        const float ay = __fadd_rn(__fsub_rn(v.y, foy), v.w);
                        s.ax[t] = ax; s.ay[t] = ay; s.ex[t] = e.x; s.ey[t] = e.y;
                        s.inv[t] = a.seg_inv32[i];
                        mag = fmaxf(mag, fmaxf(fmaxf(fabsf(ax), fabsf(ay)), fmaxf(fabsf(ax + e.x), fabsf(ay + e.y))));
                    } else {
                        const double2 v = a.verts[i];
                        const double2 e = a.seg_e64[i];
                        s.ax[t] = v.x; s.ay[t] = v.y; s.ex[t] = e.x; s.ey[t] = e.y;
                        s.inv[t] = a.seg_inv64[i];
                    }
                }
                __syncwarp();
                const int sg = choose_group(np, ns, 2);
                const int lg = __ffs(sg) - 1, pg = 32 >> lg;
                const int sub = lane & (sg - 1), grp = lane >> lg;
                for (int q0 = 0; q0 < np; q0 += pg) {
                    const int q = q0 + grp;
                    Best<T> st{INF, INF, -1};
                    if (q < np) {
                        const T px = s.px[q], py = s.py[q];
                        for (int t = sub; t < ns; t += sg)
                            consider<FP32>(st, seg_d2(px, py, s.ax[t], s.ay[t], s.ex[t], s.ey[t], s.inv[t]), s.sid[t]);
                    }
                    for (int o = sg >> 1; o > 0; o >>= 1) st = merge<FP32>(st, shfl_best<FP32>(st, o));
                    if (sub == 0 && q < np) {
                        Best<T> cur{s.b1[q], s.b2[q], s.i1[q]};
                        cur = merge<FP32>(cur, st);
                        s.b1[q] = cur.b1; s.b2[q] = cur.b2; s.i1[q] = cur.i1;
                    }
                }
                __syncwarp();
            }
        }
        if constexpr (FP32) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mag = fmaxf(mag, __shfl_xor_sync(FULL, mag, o));
        }
        for (int q = lane; q < np; q += 32) {
            const int id = s.i1[q];
            if (id < 0) continue;
            const double d = (double)sqrt(s.b1[q]);
            if constexpr (FP32) {
                const double e = (double)fmaf(64.0f * U32, fmaxf(mag, fmaxf(fabsf(s.px[q]), fabsf(s.py[q]))),
                                              4.0f * a.eps_abs);
                const double d2 = (double)sqrtf(s.b2[q]);
                const double tiny = 1e-12 * (a.D + 1.0);
                if (d - e > a.D + tiny) continue;                      // certainly outside the window
                const bool in_window = d + e < a.D - tiny;
                const bool separated = d2 - d > 2.0 * e + tiny;         // d2 = inf: no runner-up
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

template <bool FP32>
static size_t p2p_smem_bytes() {
    return sizeof(P2PSmem<FP32>) * P2P_WARPS;
}

template <bool FP32>
static cudaError_t p2p_prepare() {
    static bool done = false;   // per process; the attribute is per function
    if (!done) {
        cudaError_t e = cudaFuncSetAttribute(k_p2p_refine<FP32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)p2p_smem_bytes<FP32>());
        if (e != cudaSuccess) return e;
        done = true;
    }
    return cudaSuccess;
}

cudaError_t launch_p2p_refine(const RefineArgs &a, int form, int warps_per_block, int blocks, cudaStream_t s) {
    (void)warps_per_block;
    cudaError_t e;
    if (form == SJ_FP32X) {
        if ((e = p2p_prepare<true>()) != cudaSuccess) return e;
        k_p2p_refine<true><<<blocks, P2P_WARPS * 32, p2p_smem_bytes<true>(), s>>>(a);
    } else {
        if ((e = p2p_prepare<false>()) != cudaSuccess) return e;
        k_p2p_refine<false><<<blocks, P2P_WARPS * 32, p2p_smem_bytes<false>(), s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_p2p_recheck(const RefineArgs &a, int blocks, cudaStream_t s) {
    k_p2p_recheck<<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

int p2p_blocks_per_sm(int form) {
    int n = 0;
    if (form == SJ_FP32X) {
        if (p2p_prepare<true>() != cudaSuccess) return 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_p2p_refine<true>, P2P_WARPS * 32, p2p_smem_bytes<true>());
    } else {
        if (p2p_prepare<false>() != cudaSuccess) return 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_p2p_refine<false>, P2P_WARPS * 32,
                                                      p2p_smem_bytes<false>());
    }
    return n > 0 ? n : 1;
}

}  // namespace sj
