// sj_pip.cu -- PIP refinement (Sec. III.C, Fig. 3): ray-crossing parity of
// each point of a work item against every ring of each candidate polygon of
// its cell.
//
// Work decomposition (GB300 design, not the paper's block-per-cell mapping):
// one warp per (cell, point-chunk) item.  For each candidate polygon, in id
// order, the warp stages the polygon's edges in shared memory in chunks, then
// splits its 32 lanes into point groups of SG lanes (SG chosen per chunk so
// that np points x ne edges fill the warp); the lanes of a group stride over
// the edges and a single ballot folds the groups' parities.  A point leaves
// the candidate loop once a polygon contains it (ids are visited in
// increasing order, so the first hit is the smallest id).
//
// Two arithmetic forms:
//   FP64   -- the crossing rule in FP64, each operation rounded, no FMA.
//   FP32X  -- the straddle test on the FP32 roundings of y (monotone, so a
//             strict FP32 inequality implies the FP64 one; equal values fall
//             back), the orientation on cell-relative FP32 coordinates with a
//             forward error bound (after Shewchuk's orient2d bound plus the
//             input-rounding terms); a test whose |d| does not exceed the
//             bound is redone in FP64 from the original vertices, so the
//             result is the FP64 rule's, bit for bit.
#include <cuda_runtime.h>

#include "sj_internal.cuh"

namespace sj {

constexpr int PIP_WARPS = 4;
constexpr int PIP_SMAX = 256;   // edges per staging chunk per warp

template <bool FP32>
struct PipSmem;

template <>
struct PipSmem<false> {
    double ax[PIP_SMAX], ay[PIP_SMAX], bx[PIP_SMAX], by[PIP_SMAX];
    double px[MAX_CH], py[MAX_CH];
    int found[MAX_CH], par[MAX_CH];
};

template <>
struct PipSmem<true> {
    float2 yh[PIP_SMAX];    // fl32(y) of the edge's two ends
    float4 rel[PIP_SMAX];   // cell-relative (ax, ay, bx, by)
    int vi[PIP_SMAX];       // global index of the edge's first end
    float px[MAX_CH], py[MAX_CH], pyh[MAX_CH];
    int found[MAX_CH], par[MAX_CH];
};

// The crossing rule in FP64: straddle iff (a.y > p.y) != (b.y > p.y); with lo
// the end at or below p.y, count iff (hi.x-lo.x)(p.y-lo.y) - (hi.y-lo.y)(p.x-lo.x) > 0.
__device__ __forceinline__ int cross64(double px, double py, double ax, double ay, double bx, double by) {
    bool a_up = ay > py, b_up = by > py;
    if (a_up == b_up) return 0;
    double lx = a_up ? bx : ax, ly = a_up ? by : ay;
    double hx = a_up ? ax : bx, hy = a_up ? ay : by;
    double d = __dsub_rn(__dmul_rn(__dsub_rn(hx, lx), __dsub_rn(py, ly)),
                         __dmul_rn(__dsub_rn(hy, ly), __dsub_rn(px, lx)));
    return d > 0.0;
}

// FP64 re-evaluation of edge i (vertex i -> nxt[i]) for sorted point j.
__device__ __noinline__ int cross64_global(const RefineArgs &a, int i, int j) {
    double2 p = a.spts[j];
    double2 A = a.verts[i], B = a.verts[a.nxt[i]];
    return cross64(p.x, p.y, A.x, A.y, B.x, B.y);
}

// Sign of the orientation d = A*B - C*D on cell-relative FP32 inputs, certified
// against the FP64 rule.  Inputs: point (px, py) rounded once from FP64
// (error <= KP * |coord|), ends (lx, ly), (hx, hy) from the split vertices
// (error <= KV * |coord| + eps).  Returns false when |d| does not exceed the
// bound E = errA + errIn + err64:
//   errA  = 3.0001 u (|AB| + |CD|)          FP32 rounding of d (Shewchuk orient2d)
//   errIn = first-order input perturbation plus cross terms, x (1 + 4u)
//   err64 = 4e-16 (|A||B| + |C||D|)         FP64 rounding of the reference rule
// E is inflated by (1 + 16u) for the FP32 evaluation of the bound itself.
__device__ __forceinline__ bool orient32(float px, float py, float lx, float ly, float hx, float hy, float eps,
                                         bool &pos) {
    const float KV = 2.0001f * U32, KP = 1.0001f * U32;
    float A = __fsub_rn(hx, lx), B = __fsub_rn(py, ly);
    float C = __fsub_rn(hy, ly), Dd = __fsub_rn(px, lx);
    float AB = __fmul_rn(A, B), CD = __fmul_rn(C, Dd);
    float d = __fsub_rn(AB, CD);
    float dhx = fmaf(KV, fabsf(hx), eps), dhy = fmaf(KV, fabsf(hy), eps);
    float dlx = fmaf(KV, fabsf(lx), eps), dly = fmaf(KV, fabsf(ly), eps);
    float dpx = KP * fabsf(px), dpy = KP * fabsf(py);
    float dA = dhx + dlx, dB = dpy + dly, dC = dhy + dly, dD = dpx + dlx;
    float aA = fabsf(A), aB = fabsf(B), aC = fabsf(C), aD = fabsf(Dd);
    float errIn = (dA * aB + aA * dB + dA * dB + dC * aD + aC * dD + dC * dD) * (1.0f + 4.0f * U32);
    float errA = (3.0001f * U32) * (fabsf(AB) + fabsf(CD));
    float err64 = 4e-16f * ((aA + dA) * (aB + dB) + (aC + dC) * (aD + dD));
    float E = (errA + errIn + err64) * (1.0f + 16.0f * U32) + 1e-30f;
    pos = d > 0.0f;
    return fabsf(d) > E;
}

template <bool FP32>
__global__ void __launch_bounds__(PIP_WARPS * 32) k_pip_refine(RefineArgs a) {
    __shared__ PipSmem<FP32> smem[PIP_WARPS];
    const int lane = lane_id(), w = threadIdx.x >> 5;
    PipSmem<FP32> &s = smem[w];
    const int n_items = *a.n_items;
    unsigned long long c_pairs = 0, c_tests = 0, c_fb = 0, c_hits = 0;
    unsigned long long c_items = 0;

    for (int it = blockIdx.x * PIP_WARPS + w; it < n_items; it += gridDim.x * PIP_WARPS) {
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
                s.pyh[q] = __double2float_rn(p.y);
            } else {
                s.px[q] = p.x;
                s.py[q] = p.y;
            }
            s.found[q] = -1;
            s.par[q] = 0;
        }
        __syncwarp();

        const int k1 = a.cand_start[c + 1];
        for (int k = a.cand_start[c]; k < k1; ++k) {
            int pending = 0;
            for (int q = lane; q < np; q += 32) pending += (s.found[q] < 0);
            pending = __reduce_add_sync(FULL, pending);
            if (pending == 0) break;
            const int pid = a.cand_ids[k];
            const int vb = a.obj_voff[pid], ne = a.obj_voff[pid + 1] - vb;
            c_pairs += pending;
            c_tests += (unsigned long long)pending * (unsigned long long)ne;

            for (int e0 = 0; e0 < ne; e0 += PIP_SMAX) {
                const int ns = min(PIP_SMAX, ne - e0);
                for (int t = lane; t < ns; t += 32) {
                    const int i = vb + e0 + t, j = a.nxt[i];
                    if constexpr (FP32) {
                        float4 va = a.vsplit[i], vc = a.vsplit[j];
                        s.yh[t] = make_float2(va.y, vc.y);
                        s.rel[t] = make_float4(__fadd_rn(__fsub_rn(va.x, fox), va.z), __fadd_rn(__fsub_rn(va.y, foy), va.w),
                                               __fadd_rn(__fsub_rn(vc.x, fox), vc.z), __fadd_rn(__fsub_rn(vc.y, foy), vc.w));
                        s.vi[t] = i;
                    } else {
                        double2 A = a.verts[i], B = a.verts[j];
                        s.ax[t] = A.x; s.ay[t] = A.y; s.bx[t] = B.x; s.by[t] = B.y;
                    }
                }
                __syncwarp();
                const int sg = choose_group(np, ns, 0);
                const int lg = __ffs(sg) - 1, pg = 32 >> lg;
                const int sub = lane & (sg - 1), grp = lane >> lg;
                const unsigned gmask = (sg == 32) ? FULL : (((1u << sg) - 1u) << (grp * sg));
                for (int q0 = 0; q0 < np; q0 += pg) {
                    const int q = q0 + grp;
                    const bool act = q < np && s.found[q] < 0;
                    if (!__any_sync(FULL, act)) continue;
                    int odd = 0;
                    if (act) {
                        if constexpr (FP32) {
                            const float px = s.px[q], py = s.py[q], pyh = s.pyh[q];
                            for (int t = sub; t < ns; t += sg) {
                                const float2 yh = s.yh[t];
                                if ((yh.x == pyh) | (yh.y == pyh)) {   // FP32 y tie: decide in FP64
                                    odd ^= cross64_global(a, s.vi[t], j0 + q);
                                    ++c_fb;
                                    continue;
                                }
                                const bool a_up = yh.x > pyh, b_up = yh.y > pyh;
                                if (a_up == b_up) continue;
                                const float4 r = s.rel[t];
                                const float lx = a_up ? r.z : r.x, ly = a_up ? r.w : r.y;
                                const float hx = a_up ? r.x : r.z, hy = a_up ? r.y : r.w;
                                bool pos;
                                if (orient32(px, py, lx, ly, hx, hy, a.eps_abs, pos)) {
                                    odd ^= (int)pos;
                                } else {
                                    odd ^= cross64_global(a, s.vi[t], j0 + q);
                                    ++c_fb;
                                }
                            }
                        } else {
                            const double px = s.px[q], py = s.py[q];
                            for (int t = sub; t < ns; t += sg) odd ^= cross64(px, py, s.ax[t], s.ay[t], s.bx[t], s.by[t]);
                        }
                    }
                    const unsigned bal = __ballot_sync(FULL, odd);
                    if (sub == 0 && act) s.par[q] ^= (__popc(bal & gmask) & 1);
                }
                __syncwarp();
            }
            for (int q = lane; q < np; q += 32) {
                if (s.found[q] < 0 && s.par[q]) s.found[q] = pid;
                s.par[q] = 0;
            }
            __syncwarp();
        }
        for (int q = lane; q < np; q += 32) {
            const int f = s.found[q];
            if (f >= 0) {
                a.out_id[a.perm[j0 + q]] = f;
                ++c_hits;
            }
        }
        __syncwarp();
    }
    if (a.stats) {
        c_fb = __reduce_add_sync(FULL, (unsigned)c_fb);
        c_hits = __reduce_add_sync(FULL, (unsigned)c_hits);
        if (lane == 0) {
            atomicAdd(&a.stats[ST_ITEMS], c_items);
            atomicAdd(&a.stats[ST_PAIRS], c_pairs);
            atomicAdd(&a.stats[ST_TESTS], c_tests);
            atomicAdd(&a.stats[ST_FALLBACK], c_fb);
            atomicAdd(&a.stats[ST_HITS], c_hits);
        }
    }
}

cudaError_t launch_pip_refine(const RefineArgs &a, int form, int warps_per_block, int blocks, cudaStream_t s) {
    (void)warps_per_block;
    if (form == SJ_FP32X)
        k_pip_refine<true><<<blocks, PIP_WARPS * 32, 0, s>>>(a);
    else
        k_pip_refine<false><<<blocks, PIP_WARPS * 32, 0, s>>>(a);
    return cudaGetLastError();
}

int pip_blocks_per_sm(int form) {
    int n = 0;
    if (form == SJ_FP32X)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pip_refine<true>, PIP_WARPS * 32, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pip_refine<false>, PIP_WARPS * 32, 0);
    return n > 0 ? n : 1;
}

}  // namespace sj
