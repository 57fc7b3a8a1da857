// sj_p2p.cu -- P2P refinement (Sec. III.B, Fig. 2): for every point of a work
// item, the candidate polyline at the smallest distance, accepted when the
// distance is within the window D.
//
// Work decomposition: one warp per (cell, point-chunk) item.
//   1. The item's points are converted to cell-relative coordinates and their
//      bounding box is reduced across the warp.
//   2. The cell's segment list -- every segment of the candidate polylines
//      whose box widened by D meets the cell, built with the layer; the others
//      are farther than D from every point of the cell -- is read 32 entries
//      at a time, one per lane, as records prepared with the layer (the
//      segment relative to this cell's FP32 frame, its owner and magnitude).
//   3. Staging: a segment whose bounding box is farther than D (plus a
//      rounding slack) from the points' box cannot be within D of any point of
//      the item and is dropped (exact: it cannot change any result); the others
//      are compacted into shared memory (a, e = b - a, 1 / |e|^2, polyline id)
//      with a ballot.
//   4. Whenever the staging area fills, the warp splits its lanes into point
//      groups of SG lanes (SG chosen so that np points x staged segments fill
//      the warp); each lane strides over the staged segments keeping a running
//      "top-2" -- the best (squared distance, polyline) and the best distance
//      of any other polyline -- and the SG lanes of a group fold their top-2s
//      with shuffles (the cross-lane min of the vertex-per-lane alternative of
//      Sec. III.B); the fold is merged into the point's state in shared memory.
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
//   FP32X  -- cell-relative FP32 coordinates from the (hi, lo) split of the FP64
//             inputs; no FP64 instruction is executed.  Every (point, polyline)
//             distance carries the bound E = 64 u M + 4 eps (u = 2^-24, M the
//             largest |coordinate| of the point and of the item's staged
//             segments).  A point is final only when its best polyline is ahead
//             of the runner-up by more than 2E and its distance differs from D
//             by more than E; otherwise it is queued and redone in FP64
//             (k_p2p_recheck), so ids agree with FP64 up to exact ties.
#include <cuda_runtime.h>

#include <type_traits>

#include "sj_internal.cuh"

namespace sj {

unsigned bounds_take_p2p() { return bounds_take(); }

constexpr int P2P_WARPS = 4;

struct alignas(16) Seg64 {
    double ax, ay, ex, ey;
};

template <bool FP32>
struct P2PSmem;

// FP32X staging holds segments in pairs (2k, 2k + 1), each quantity of the
// pair side by side, so that one lane evaluates both with the packed FP32
// instructions (FADD2 / FMUL2 / FFMA2: two IEEE round-to-nearest operations
// each, the same roundings as the scalar ones).  The stored values are
// negated (-a, -e, -1 / |e|^2), which keeps every packed operation an add or
// a fused multiply-add of the stored operands; the arithmetic is the clamped
// projection below, operation for operation.
template <>
struct P2PSmem<true> {
    static constexpr int SMAX = 128;   // even
    float4 sa[SMAX / 2];     // (-ax, -ax', -ay, -ay') cell-relative
    float4 se[SMAX / 2];     // (-ex, -ex', -ey, -ey')
    float4 si[SMAX / 2];     // (-1 / |e|^2, -1 / |e'|^2, polyline id bits, id' bits)
    float2 pt[MAX_CH];
    float b1[MAX_CH], b2[MAX_CH];
    int i1[MAX_CH];
};

template <>
struct P2PSmem<false> {
    static constexpr int SMAX = 128;
    Seg64 seg[SMAX];
    double inv[SMAX];
    int sid[SMAX];
    double2 pt[MAX_CH];
    double b1[MAX_CH], b2[MAX_CH];
    int i1[MAX_CH];
};

// Squared distance from p to the segment (a, a + e) by the clamped projection:
// d = p - a, t = clamp((e . d) / |e|^2, 0, 1), |d - t e|^2, each operation
// rounded once (FP64 here; the FP32X loop in p2p_compute evaluates the same
// operations in FP32 on segment pairs).
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
        // b1 <= b2 always; the runner-up becomes max(d, b1) when l is another
        // polyline (whichever of the old best and d is not the new best).
        const bool lt = d < s.b1;
        const T nb2 = (l == s.i1) ? s.b2 : fminf(s.b2, fmaxf(d, s.b1));
        s.b1 = fminf(s.b1, d);
        s.i1 = lt ? l : s.i1;
        s.b2 = nb2;
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

// A window w in FP32, rounded down / up with the same 1e-12 relative margin
// the layer's D gets on the host (explicit roundings, no contraction).
__device__ __forceinline__ void window_f32(double w, float &dn, float &up) {
    dn = __double2float_rd(__dmul_rn(w, 1.0 - 1e-12));
    up = __double2float_ru(__dadd_rn(__dmul_rn(w, 1.0 + 1e-12), 1e-300));
}

// Warp-wide min / max of a float (no NaN) in one integer reduction: flipping
// the magnitude bits of negative floats makes signed-integer order equal
// float order (-0 sorts just below +0).
__device__ __forceinline__ int float_key(float v) {
    const int i = __float_as_int(v);
    return i ^ ((i >> 31) & 0x7fffffff);
}
__device__ __forceinline__ float key_float(int k) { return __int_as_float(k ^ ((k >> 31) & 0x7fffffff)); }
__device__ __forceinline__ float warp_min(float v) { return key_float(__reduce_min_sync(FULL, float_key(v))); }
__device__ __forceinline__ float warp_max(float v) { return key_float(__reduce_max_sync(FULL, float_key(v))); }

// Refine the staged segments [0, ns) for the item's np points (FP32X: ns
// counts segment pairs).  Rounds of 32
// points take one lane per point (every lane busy, no merge); the last round,
// of fewer than 32 points, splits each point's segments over a group of sg
// lanes chosen by the cost model (more lanes per point, log2(sg) merges).
template <bool FP32>
__device__ __forceinline__ void p2p_compute(P2PSmem<FP32> &s, int np, int ns, int lane) {
    using T = typename std::conditional<FP32, float, double>::type;
    const T INF = (T)__longlong_as_double(0x7ff0000000000000LL);
    int pg = 32;
    for (int q0 = 0; q0 < np; q0 += pg) {
        const int rem = np - q0;
        const int sg = rem >= 32 ? 1 : choose_group(rem, ns, 2);
        const int lg = __ffs(sg) - 1;
        pg = 32 >> lg;
        const int sub = lane & (sg - 1), grp = lane >> lg;
        const int q = q0 + grp;
        Best<T> st{INF, INF, -1};
        if (q < np) {
            if constexpr (FP32) {
                // the squared distances of the pair by the clamped projection
                // in FP32: dx = px - ax, t = sat(fma(ex, dx, ey * dy) / |e|^2),
                // q = fma(-t, e, d), |q|^2 = fma(qx, qx, qy * qy), written with
                // the negated operands (p + (-a) = p - a, fma(-ex, dx, -ey * dy)
                // * (-1 / |e|^2) = (e . d) / |e|^2, fma(t, -e, d) = d - t e:
                // each rounding the same as the unnegated one)
                const float2 p = s.pt[q];
                const float2 px = make_float2(p.x, p.x), py = make_float2(p.y, p.y);
#pragma unroll 1
                for (int t = sub; t < ns; t += sg) {
                    const float4 A = s.sa[t], E = s.se[t], I = s.si[t];
                    const float2 nex = make_float2(E.x, E.y), ney = make_float2(E.z, E.w);
                    const float2 dx = __fadd2_rn(px, make_float2(A.x, A.y));
                    const float2 dy = __fadd2_rn(py, make_float2(A.z, A.w));
                    const float2 w = __ffma2_rn(nex, dx, __fmul2_rn(ney, dy));
                    const float2 tt = make_float2(__saturatef(__fmul_rn(w.x, I.x)), __saturatef(__fmul_rn(w.y, I.y)));
                    const float2 qx = __ffma2_rn(tt, nex, dx), qy = __ffma2_rn(tt, ney, dy);
                    const float2 d = __ffma2_rn(qx, qx, __fmul2_rn(qy, qy));
                    consider<true>(st, d.x, __float_as_int(I.z));
                    consider<true>(st, d.y, __float_as_int(I.w));
                }
            } else {
                const double2 p = s.pt[q];
                for (int t = sub; t < ns; t += sg) {
                    const Seg64 g = s.seg[t];
                    consider<false>(st, seg_d2(p.x, p.y, g.ax, g.ay, g.ex, g.ey, s.inv[t]), s.sid[t]);
                }
            }
        }
        for (int o = sg >> 1; o > 0; o >>= 1) st = merge<FP32>(st, shfl_best<FP32>(st, o));
        if (sub == 0 && q < np) {
            Best<T> cur{s.b1[q], s.b2[q], s.i1[q]};
            cur = merge<FP32>(cur, st);
            s.b1[q] = cur.b1;
            s.b2[q] = cur.b2;
            s.i1[q] = cur.i1;
        }
    }
}

// PW: per-point windows (a.win_on set; batched rounds).  The direct joins use
// PW = false, whose code has no window load at all.  Eight blocks per SM is
// the shared-memory limit already; saying so keeps the register allocator at
// 64 registers without spills.
template <bool FP32, bool PW, int NW>
__global__ void __launch_bounds__(NW * 32, 32 / NW) k_p2p_refine(RefineArgs a) {
    using T = typename std::conditional<FP32, float, double>::type;
    constexpr int SMAX = P2PSmem<FP32>::SMAX;
    extern __shared__ __align__(16) unsigned char p2p_smem_raw[];
    const int lane = lane_id(), w = threadIdx.x >> 5;
    P2PSmem<FP32> &s = reinterpret_cast<P2PSmem<FP32> *>(p2p_smem_raw)[w];
    const int n_items = *a.n_items;
    const T INF = (T)__longlong_as_double(0x7ff0000000000000LL);
    const float FINF = __int_as_float(0x7f800000);
    const unsigned lt_mask = (1u << lane) - 1u;
    unsigned long long c_pairs = 0, c_tests = 0, c_items = 0, c_algo = 0;
    unsigned c_fb = 0, c_hits = 0;
    const bool pw = PW && *a.win_on;   // per-point windows in this launch (uniform)

    // Items come from a device counter when a.work_next is set (the next index
    // is fetched at the start of an item, so its latency hides behind the
    // item), else in a fixed stride.
    // The next item's record and its cell's point range are loaded while the
    // current item is refined, off the per-item chain of dependent loads.
    // A warp takes a.claim consecutive items per counter update: consecutive
    // items are mostly chunks of one cell, whose segment records are then
    // still in L1 for the second chunk.
    const int claim = a.claim > 1 ? a.claim : 1;
    int it = blockIdx.x * NW + w, it_end = it + 1;
    if (a.work_next) {
        int t0 = 0;
        if (lane == 0) t0 = atomicAdd(a.work_next, claim);
        it = __shfl_sync(FULL, t0, 0);
        it_end = it + claim;
    }
    int2 item = make_int2(0, 0);
    int cs0 = 0, cs1 = 0;
    if (it < n_items) {
        item = a.items[it];
        cs0 = a.cell_start[item.x];
        cs1 = a.cell_start[item.x + 1];
    }
    while (it < n_items) {
        int it_next = it + gridDim.x * NW;
        const bool in_claim = it + 1 < it_end;
        if (a.work_next) {
            if (in_claim) it_next = it + 1;
            else if (lane == 0) it_next = atomicAdd(a.work_next, claim);
        }
        ++c_items;
        const int c = item.x;
        const int j0 = cs0 + item.y;
        const int np = min(cell_chunk(a.ch, a.budget > 0 ? a.cell_work[c] : 0, a.budget), cs1 - j0);
        const int k0 = a.cand_start[c], k1 = a.cand_start[c + 1];
        const float2 fo = cell_frame(a.frame_x, a.frame_y, a.g.nx, c);

        // 1. points: cell-relative FP32 coordinates, their box and magnitude
        float bxlo = FINF, bxhi = -FINF, bylo = FINF, byhi = -FINF;
        // The (up to MAX_CH / 32) point loads of a lane are issued together --
        // every slot index, then every point as an asynchronous copy into the
        // (idle) staging area -- so that their latencies overlap instead of
        // forming one chain per point.
        constexpr int PQ = MAX_CH / 32;
        double2 *pbuf;
        if constexpr (FP32) {
            static_assert(sizeof(P2PSmem<true>::sa) + sizeof(P2PSmem<true>::se) >= MAX_CH * sizeof(double2), "");
            pbuf = reinterpret_cast<double2 *>(&s.sa[0]);   // sa and se, contiguous
        } else {
            static_assert(sizeof(P2PSmem<false>::seg) >= MAX_CH * sizeof(double2), "");
            pbuf = reinterpret_cast<double2 *>(&s.seg[0]);
        }
        {
            int src[PQ];
#pragma unroll
            for (int u = 0; u < PQ; ++u) {
                const int q = lane + 32 * u;
                src[u] = (q < np && SJ_IN_BOUNDS(j0 + q < a.npts, BND_P2P_POINT)) ? (a.spts ? j0 + q : a.perm[j0 + q])
                                                                                 : -1;
            }
#pragma unroll
            for (int u = 0; u < PQ; ++u)
                if (src[u] >= 0 && SJ_IN_BOUNDS(src[u] < a.npts, BND_P2P_POINT))
                    copy16_async(pbuf + lane + 32 * u, a.spts ? a.spts + src[u] : a.pts + src[u]);
            copy_async_wait_all();
        }
        for (int q = lane; q < np; q += 32) {
            const double2 p = pbuf[q];
            float hx, lx, hy, ly;
            split_double(p.x, hx, lx);
            split_double(p.y, hy, ly);
            const float rx = rel_coord(hx, lx, fo.x), ry = rel_coord(hy, ly, fo.y);
            if constexpr (FP32) s.pt[q] = make_float2(rx, ry);
            else s.pt[q] = p;
            s.b1[q] = INF;
            s.b2[q] = INF;
            s.i1[q] = -1;
            bxlo = fminf(bxlo, rx); bxhi = fmaxf(bxhi, rx);
            bylo = fminf(bylo, ry); byhi = fmaxf(byhi, ry);
        }
        __syncwarp();   // every lane is done with the point buffer before staging reuses it
        bxlo = warp_min(bxlo); bylo = warp_min(bylo);
        bxhi = warp_max(bxhi); byhi = warp_max(byhi);
        // largest |coordinate| of the points: the larger magnitude of the box's ends
        const float pmag = fmaxf(fmaxf(fabsf(bxlo), fabsf(bxhi)), fmaxf(fabsf(bylo), fabsf(byhi)));
        if (a.work_next) it_next = __shfl_sync(FULL, it_next, 0);
        const int end_next = in_claim ? it_end : it_next + (a.work_next ? claim : 1);
        int2 item_n = make_int2(0, 0);
        if (it_next < n_items) item_n = a.items[it_next];
        float mag = pmag;   // FP32X: largest |cell-relative coordinate| refined for this item
        c_pairs += (unsigned long long)np * (unsigned long long)(k1 - k0);
        c_algo += (unsigned long long)np * (unsigned long long)a.cell_algo[c];

        // 2. the cell's segment list, 32 segments at a time (one per lane),
        // 3. staging with the exact distance prune, 4. refinement when full
        const int g0 = a.cseg_start[c], g1 = a.cseg_start[c + 1];
        int nst = 0;
        for (int base = g0; base < g1; base += 32) {
            const int g = base + lane;
            bool keep = false;
            int i = 0, sid = 0;
            float ax = 0.0f, ay = 0.0f, ex = 0.0f, ey = 0.0f, inv = 0.0f, smag = 0.0f;
            if (g < g1 && SJ_IN_BOUNDS(g < a.cseg_start[a.g.G], BND_P2P_REC)) {
                const float4 r0 = a.cseg_rec[2 * (size_t)g], r1 = a.cseg_rec[2 * (size_t)g + 1];
                ax = r0.x;
                ay = r0.y;
                ex = r0.z;
                ey = r0.w;
                inv = r1.x;
                sid = __float_as_int(r1.y);
                smag = r1.z;
                i = __float_as_int(r1.w);
                const float bx = ax + ex, by = ay + ey;
                const float gx = fmaxf(0.0f, fmaxf(fminf(ax, bx) - bxhi, bxlo - fmaxf(ax, bx)));
                const float gy = fmaxf(0.0f, fmaxf(fminf(ay, by) - byhi, bylo - fmaxf(ay, by)));
                // rounding slack of the relative coordinates of both boxes (far above it)
                const float lim = a.Df * (1.0f + 1e-6f) + 8.0f * U32 * (smag + pmag) + 8.0f * a.eps_abs;
                keep = gx * gx + gy * gy <= lim * lim * (1.0f + 8.0f * U32);
            }
            const unsigned bal = __ballot_sync(FULL, keep);
            if (keep) {
                const int pos = nst + __popc(bal & lt_mask);
                if constexpr (FP32) {
                    const int k = pos >> 1, h = pos & 1;
                    float *A = reinterpret_cast<float *>(&s.sa[k]);
                    float *E = reinterpret_cast<float *>(&s.se[k]);
                    float *I = reinterpret_cast<float *>(&s.si[k]);
                    A[h] = -ax; A[2 + h] = -ay;
                    E[h] = -ex; E[2 + h] = -ey;
                    I[h] = -inv; I[2 + h] = __int_as_float(sid);
                    mag = fmaxf(mag, smag);
                } else {
                    const double2 v = a.verts[i], e = a.seg_e64[i];
                    s.seg[pos] = Seg64{v.x, v.y, e.x, e.y};
                    s.inv[pos] = a.seg_inv64[i];
                    s.sid[pos] = sid;
                }
            }
            nst += __popc(bal);
            if (nst > SMAX - 32 || base + 32 >= g1) {
                if constexpr (FP32) {
                    // an odd count: the pair's second slot gets a segment at
                    // infinite distance (a far point, zero length), which never
                    // changes a point's top-2
                    if ((nst & 1) && lane == 0) {
                        const int k = nst >> 1;
                        reinterpret_cast<float *>(&s.sa[k])[1] = -3.0e38f;
                        reinterpret_cast<float *>(&s.sa[k])[3] = -3.0e38f;
                        reinterpret_cast<float *>(&s.se[k])[1] = 0.0f;
                        reinterpret_cast<float *>(&s.se[k])[3] = 0.0f;
                        reinterpret_cast<float *>(&s.si[k])[1] = 0.0f;
                        reinterpret_cast<float *>(&s.si[k])[3] = __int_as_float(-2);
                    }
                }
                __syncwarp();
                if (nst > 0) {
                    p2p_compute<FP32>(s, np, FP32 ? (nst + 1) >> 1 : nst, lane);
                    c_tests += (unsigned long long)np * (unsigned long long)nst;
                }
                __syncwarp();
                nst = 0;
            }
        }
        int cs0n = 0, cs1n = 0;
        if (it_next < n_items) {
            cs0n = a.cell_start[item_n.x];
            cs1n = a.cell_start[item_n.x + 1];
        }
        if constexpr (FP32) mag = warp_max(mag);
        for (int q = lane; q < np; q += 32) {
            const int id = s.i1[q];
            int out = -1;
            double dd = __longlong_as_double(0x7ff0000000000000LL);
            float df = FINF;
            if (id >= 0) {
                if constexpr (FP32) {
                    const float d = sqrtf(s.b1[q]), d2 = sqrtf(s.b2[q]);
                    const float2 p = s.pt[q];
                    const float e = fmaf(64.0f * U32, fmaxf(mag, fmaxf(fabsf(p.x), fabsf(p.y))), 4.0f * a.eps_abs) *
                                    (1.0f + 8.0f * U32);
                    float Ddn = a.Ddn, Dup = a.Dup;
                    if (pw) window_f32(a.win[j0 + q], Ddn, Dup);
                    if (!((d - e) * (1.0f - 4.0f * U32) > Dup)) {                    // not certainly outside D
                        const bool in_window = (d + e) * (1.0f + 4.0f * U32) < Ddn;
                        const bool separated = (d2 - d) * (1.0f - 4.0f * U32) > 2.0f * e * (1.0f + 4.0f * U32);
                        if (!(in_window && separated)) {                              // redo in FP64
                            const int slot = atomicAdd(a.n_fb, 1);
                            a.fb[slot] = make_int2(j0 + q, c);
                            ++c_fb;
                            continue;
                        }
                        out = id;
                        dd = widen(d);
                        df = d;
                    }
                } else {
                    const double d = sqrt(s.b1[q]);
                    if (d <= (pw ? a.win[j0 + q] : a.D)) {
                        out = id;
                        dd = d;
                    }
                }
            }
            if (!SJ_IN_BOUNDS(j0 + q < a.npts, BND_P2P_RES)) continue;
            if (a.resf) {
                a.resf[j0 + q] = ResF{out, df};
            } else if (a.resd) {
                a.resd[j0 + q] = ResD{out, 0, dd};
            } else if (a.res_id) {
                a.res_id[j0 + q] = out;
                if (a.res_d) a.res_d[j0 + q] = dd;
            } else if (out >= 0) {
                const int i = a.perm[j0 + q];
                a.out_id[i] = out;
                if (a.out_d) a.out_d[i] = dd;
            }
            if (out >= 0) ++c_hits;
        }
        __syncwarp();
        it = it_next;
        it_end = end_next;
        item = item_n;
        cs0 = cs0n;
        cs1 = cs1n;
    }
    if (a.stats) {
        unsigned long long v[ST_N] = {};
        v[ST_ITEMS] = c_items;
        v[ST_PAIRS] = c_pairs;
        v[ST_TESTS] = c_tests;
        v[ST_ALGO] = c_algo;
        v[ST_FALLBACK] = __reduce_add_sync(FULL, c_fb);
        v[ST_HITS] = __reduce_add_sync(FULL, c_hits);
        flush_stats(a.stats, v);
    }
}

// FP64 recomputation of the points the FP32X pass could not certify: one warp
// per point, lanes over the cell's segment list, each lane keeping the
// smallest (squared distance, polyline id), then a warp fold.
__global__ void __launch_bounds__(256) k_p2p_recheck(RefineArgs a) {
    const int lane = lane_id();
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int n = *a.n_fb;
    const double INF = __longlong_as_double(0x7ff0000000000000LL);
    const bool pw = a.win_on && *a.win_on;
    unsigned c_hits = 0;
    for (int f = warp; f < n; f += nwarps) {
        const int2 e = a.fb[f];
        const int j = e.x, c = e.y;
        const double2 p = slot_point(a, j);
        Best<double> st{INF, INF, -1};
        for (int g = a.cseg_start[c] + lane; g < a.cseg_start[c + 1]; g += 32) {
            const int i = a.cseg_ids[g];
            const double2 v = a.verts[i], ev = a.seg_e64[i];
            consider<false>(st, seg_d2(p.x, p.y, v.x, v.y, ev.x, ev.y, a.seg_inv64[i]), __float_as_int(a.seg32[i].w));
        }
        for (int o = 16; o > 0; o >>= 1) st = merge<false>(st, shfl_best<false>(st, o));
        const double best = sqrt(st.b1);
        const bool hit = st.i1 >= 0 && best <= (pw ? a.win[j] : a.D);
        if (lane == 0) {
            if (a.res_id) {
                a.res_id[j] = hit ? st.i1 : -1;
                if (a.res_d) a.res_d[j] = hit ? best : INF;
            } else {   // final outputs through perm (hits and misses)
                const int i = a.perm[j];
                a.out_id[i] = hit ? st.i1 : -1;
                if (a.out_d) a.out_d[i] = hit ? best : INF;
            }
            if (hit) ++c_hits;
        }
    }
    if (a.stats) {
        c_hits = __reduce_add_sync(FULL, c_hits);
        if (lane == 0 && c_hits) atomicAdd(&a.stats[ST_HITS], (unsigned long long)c_hits);
    }
}

template <bool FP32, int NW>
static size_t p2p_smem_bytes() {
    return sizeof(P2PSmem<FP32>) * NW;
}

template <bool FP32, bool PW, int NW>
static cudaError_t p2p_prepare() {
    static bool done = false;   // per process; the attribute is per function
    if (!done) {
        cudaError_t e = cudaFuncSetAttribute(k_p2p_refine<FP32, PW, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)p2p_smem_bytes<FP32, NW>());
        if (e != cudaSuccess) return e;
        done = true;
    }
    return cudaSuccess;
}

template <bool FP32, bool PW, int NW>
static cudaError_t p2p_launch(const RefineArgs &a, int blocks, cudaStream_t s) {
    cudaError_t e = p2p_prepare<FP32, PW, NW>();
    if (e != cudaSuccess) return e;
    k_p2p_refine<FP32, PW, NW><<<blocks, NW * 32, p2p_smem_bytes<FP32, NW>(), s>>>(a);
    return cudaGetLastError();
}

template <bool FP32, bool PW>
static cudaError_t p2p_launch_nw(const RefineArgs &a, int nw, int blocks, cudaStream_t s) {
    if (nw == 2) return p2p_launch<FP32, PW, 2>(a, blocks, s);
    if (nw == 8) return p2p_launch<FP32, PW, 8>(a, blocks, s);
    return p2p_launch<FP32, PW, P2P_WARPS>(a, blocks, s);
}

// blocks: the grid for blocks of P2P_WARPS warps (resident blocks x SMs); a
// block of warps_per_block (2, 4 or 8) warps gets the same number of warps.
cudaError_t launch_p2p_refine(const RefineArgs &a, int form, int warps_per_block, int blocks, cudaStream_t s) {
    const int nw = (warps_per_block == 2 || warps_per_block == 8) ? warps_per_block : P2P_WARPS;
    blocks = (int)(((long long)blocks * P2P_WARPS + nw - 1) / nw);
    const bool pw = a.win && a.win_on;
    if (form == SJ_FP32X) return pw ? p2p_launch_nw<true, true>(a, nw, blocks, s) : p2p_launch_nw<true, false>(a, nw, blocks, s);
    return pw ? p2p_launch_nw<false, true>(a, nw, blocks, s) : p2p_launch_nw<false, false>(a, nw, blocks, s);
}

cudaError_t launch_p2p_recheck(const RefineArgs &a, int blocks, cudaStream_t s) {
    k_p2p_recheck<<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

int p2p_blocks_per_sm(int form) {
    int n = 0;
    if (form == SJ_FP32X) {
        if (p2p_prepare<true, false, P2P_WARPS>() != cudaSuccess) return 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_p2p_refine<true, false, P2P_WARPS>, P2P_WARPS * 32,
                                                      p2p_smem_bytes<true, P2P_WARPS>());
    } else {
        if (p2p_prepare<false, false, P2P_WARPS>() != cudaSuccess) return 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_p2p_refine<false, false, P2P_WARPS>, P2P_WARPS * 32,
                                                      p2p_smem_bytes<false, P2P_WARPS>());
    }
    return n > 0 ? n : 1;
}

}  // namespace sj
