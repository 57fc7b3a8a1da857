// sj_pip.cu -- PIP refinement (Sec. III.C, Fig. 3): ray-crossing parity of
// each point of a work item against every ring of each candidate polygon of
// its cell; the result is the smallest candidate id with odd parity.
//
// Work decomposition (GB300 design, not the paper's block-per-cell mapping):
// one warp per (cell, point-chunk) item.
//   1. The item's points are loaded; the range [ymin, ymax] of their FP32
//      y roundings is reduced across the warp.
//   2. Candidate polygons are taken 32 at a time (one per lane, in id order):
//      each lane reads its polygon's edge list for the item's grid row (the
//      edges whose y-range spans that row, built with the layer; no other edge
//      can cross the ray of a point in the row), list lengths warp-scanned.
//   3. Staging: the concatenated edges of the group are read 32 at a time; an
//      edge whose y-range lies strictly below ymin or strictly above ymax
//      cannot straddle the horizontal line of any point of the item and is
//      dropped (exact: its crossing count is 0 for every point; the test uses
//      FP32 roundings that are monotone, with strict inequalities); so is an
//      edge lying wholly left of every point of the item by a safe margin (a
//      ray towards +x cannot cross it); the rest is compacted into shared
//      memory with the lane's candidate index k.
//   4. Whenever the staging area fills, the lanes split into point groups of
//      SG lanes; each lane keeps a 32-bit parity mask (bit k = candidate k)
//      over its strided share of the staged edges; the SG lanes XOR-fold their
//      masks with shuffles, and the fold is XORed into the point's mask.
//   After a group, a point's result is the lowest set bit of its mask (ids are
//   sorted, so the smallest id); points with a result skip later groups.
//
// Two arithmetic forms:
//   FP64   -- the crossing rule in FP64, each operation rounded, no FMA.
//   FP32X  -- no FP64 instruction in the common path: the straddle test on the
//             FP32 truncations of y (monotone, so a strict FP32 inequality
//             implies the FP64 one; equal values fall back), the orientation on
//             cell-relative FP32 coordinates (from the (hi, lo) split of the
//             inputs) with a forward error bound (Shewchuk's orient2d bound plus
//             the input-rounding terms); a test whose |d| does not exceed the
//             bound is redone in FP64 from the original vertices, so the result
//             is the FP64 rule's, bit for bit.
#include <cuda_runtime.h>

#include <algorithm>

#include "sj_internal.cuh"

namespace sj {

unsigned bounds_take_pip() { return bounds_take(); }

constexpr int PIP_WARPS = 4;

struct alignas(16) Edge64 {
    double ax, ay, bx, by;
};

template <bool FP32>
struct PipSmem;

template <>
struct PipSmem<true> {
    static constexpr int SMAX = 128;
    float2 yh[SMAX];          // FP32 truncated y of the edge's two ends
    float4 rel[SMAX];         // cell-relative (ax, ay, bx, by)
    int vi[SMAX];             // global index of the edge's first end
    unsigned char kk[SMAX];   // candidate index within the group
    int coff[33], cid[32], cvb[32];
    float2 pt[MAX_CH];
    float pyh[MAX_CH];
    int pin[MAX_CH];          // FP64 source index of the point: sorted slot (spts) or input index (pts)
    int found[MAX_CH];
    unsigned par[MAX_CH];
};

template <>
struct PipSmem<false> {
    static constexpr int SMAX = 128;
    Edge64 e[SMAX];
    unsigned char kk[SMAX];
    int coff[33], cid[32], cvb[32];
    double2 pt[MAX_CH];
    int found[MAX_CH];
    unsigned par[MAX_CH];
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

// FP64 re-evaluation of edge i (vertex i -> nxt[i]) for point k of spts (when
// set) or of pts.
__device__ __noinline__ int cross64_global(const RefineArgs &a, int i, int k) {
    const double2 p = a.spts ? a.spts[k] : a.pts[k];
    const double2 A = a.verts[i], B = a.verts[a.nxt[i]];
    return cross64(p.x, p.y, A.x, A.y, B.x, B.y);
}

// Sign of the orientation d = A*B - C*D on cell-relative FP32 inputs, certified
// against the FP64 rule.  Every input coordinate c carries the rounding bound
// KV |c| + eps of the (hi, lo) split.  Returns false when |d| does not exceed
// E = errA + errIn + err64:
//   errA  = 3.0001 u (|AB| + |CD|)          FP32 rounding of d (Shewchuk orient2d)
//   errIn = first-order input perturbation plus cross terms, x (1 + 4u)
//   err64 = 4e-16 (|A||B| + |C||D|)         FP64 rounding of the reference rule
// E is inflated by (1 + 16u) for the FP32 evaluation of the bound itself.
__device__ __forceinline__ bool orient32(float px, float py, float lx, float ly, float hx, float hy, float eps,
                                         bool &pos) {
    const float KV = 2.0001f * U32;
    float A = __fsub_rn(hx, lx), B = __fsub_rn(py, ly);
    float C = __fsub_rn(hy, ly), Dd = __fsub_rn(px, lx);
    float AB = __fmul_rn(A, B), CD = __fmul_rn(C, Dd);
    float d = __fsub_rn(AB, CD);
    float dhx = fmaf(KV, fabsf(hx), eps), dhy = fmaf(KV, fabsf(hy), eps);
    float dlx = fmaf(KV, fabsf(lx), eps), dly = fmaf(KV, fabsf(ly), eps);
    float dpx = fmaf(KV, fabsf(px), eps), dpy = fmaf(KV, fabsf(py), eps);
    float dA = dhx + dlx, dB = dpy + dly, dC = dhy + dly, dD = dpx + dlx;
    float aA = fabsf(A), aB = fabsf(B), aC = fabsf(C), aD = fabsf(Dd);
    float errIn = (dA * aB + aA * dB + dA * dB + dC * aD + aC * dD + dC * dD) * (1.0f + 4.0f * U32);
    float errA = (3.0001f * U32) * (fabsf(AB) + fabsf(CD));
    float err64 = 4e-16f * ((aA + dA) * (aB + dB) + (aC + dC) * (aD + dD));
    float E = (errA + errIn + err64) * (1.0f + 16.0f * U32) + 1e-30f;
    pos = d > 0.0f;
    return fabsf(d) > E;
}

// Near lists longer than this are not staged: each pending point searches
// the window of the sorted list that can hold its straddling edges.
constexpr int LONG_NEAR = 128;

// Crossing of near edge e (boundary list entry) for point q of the item, the
// arithmetic of pip_compute for one edge: FP32X on the edge's staging record
// (FP32 straddle test on truncations, certified orientation, FP64 rule on a
// tie or an uncertain sign), FP64 on the original vertices.
template <bool FP32>
__device__ __forceinline__ int near_edge_cross(const RefineArgs &a, const PipSmem<FP32> &s, int q, int e, float2 fo,
                                               unsigned &c_fb) {
    if constexpr (FP32) {
        const float pyh = s.pyh[q];
        const float4 va = a.bnear_rec[2 * (size_t)e], vc = a.bnear_rec[2 * (size_t)e + 1];
        if ((va.y == pyh) | (vc.y == pyh)) {   // FP32 y tie: decide in FP64
            ++c_fb;
            return cross64_global(a, a.bnear_ids[e], s.pin[q]);
        }
        const bool a_up = va.y > pyh, b_up = vc.y > pyh;
        if (a_up == b_up) return 0;
        const float ax = rel_coord(va.x, va.z, fo.x), ay = rel_coord(va.y, va.w, fo.y);
        const float bx = rel_coord(vc.x, vc.z, fo.x), by = rel_coord(vc.y, vc.w, fo.y);
        const float lx = a_up ? bx : ax, ly = a_up ? by : ay;
        const float hx = a_up ? ax : bx, hy = a_up ? ay : by;
        const float2 p = s.pt[q];
        bool pos;
        if (orient32(p.x, p.y, lx, ly, hx, hy, a.eps_abs, pos)) return (int)pos;
        ++c_fb;
        return cross64_global(a, a.bnear_ids[e], s.pin[q]);
    } else {
        const int i = a.bnear_ids[e];
        const double2 A = a.verts[i], B = a.verts[a.nxt[i]], p = s.pt[q];
        return cross64(p.x, p.y, A.x, A.y, B.x, B.y);
    }
}

// First index t in [0, n) with keys[t] >= x (upper = false) or > x (upper =
// true), n if none.
__device__ __forceinline__ int key_bound(const float *keys, int n, float x, bool upper) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const float k = keys[mid];
        if (upper ? (k <= x) : (k < x)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Parity masks of the staged edges [0, ns) for the item's pending points.
template <bool FP32>
__device__ __forceinline__ unsigned long long pip_compute(PipSmem<FP32> &s, const RefineArgs &a, int j0, int np,
                                                          int ns, int lane, unsigned &c_fb) {
    unsigned long long tests = 0;
    int pg = 32;
    for (int q0 = 0; q0 < np; q0 += pg) {   // one lane per point while 32 remain, then lane groups
        const int rem = np - q0;
        const int sg = rem >= 32 ? 1 : choose_group(rem, ns, 0);
        const int lg = __ffs(sg) - 1;
        pg = 32 >> lg;
        const int sub = lane & (sg - 1), grp = lane >> lg;
        const int q = q0 + grp;
        const bool act = q < np && s.found[q] < 0;
        const unsigned actb = __ballot_sync(FULL, act && sub == 0);
        if (!actb) continue;
        tests += (unsigned long long)__popc(actb) * (unsigned long long)ns;
        unsigned m = 0;
        if (act) {
            if constexpr (FP32) {
                const float2 p = s.pt[q];
                const float pyh = s.pyh[q];
                for (int t = sub; t < ns; t += sg) {
                    const float2 yh = s.yh[t];
                    if ((yh.x == pyh) | (yh.y == pyh)) {   // FP32 y tie: decide in FP64
                        m ^= (unsigned)cross64_global(a, s.vi[t], s.pin[q]) << s.kk[t];
                        ++c_fb;
                        continue;
                    }
                    const bool a_up = yh.x > pyh, b_up = yh.y > pyh;
                    if (a_up == b_up) continue;
                    const float4 r = s.rel[t];
                    const float lx = a_up ? r.z : r.x, ly = a_up ? r.w : r.y;
                    const float hx = a_up ? r.x : r.z, hy = a_up ? r.y : r.w;
                    bool pos;
                    int cr;
                    if (orient32(p.x, p.y, lx, ly, hx, hy, a.eps_abs, pos)) {
                        cr = (int)pos;
                    } else {
                        cr = cross64_global(a, s.vi[t], s.pin[q]);
                        ++c_fb;
                    }
                    m ^= (unsigned)cr << s.kk[t];
                }
            } else {
                const double2 p = s.pt[q];
                for (int t = sub; t < ns; t += sg) {
                    const Edge64 e = s.e[t];
                    if (cross64(p.x, p.y, e.ax, e.ay, e.bx, e.by)) m ^= 1u << s.kk[t];
                }
            }
        }
        for (int o = sg >> 1; o > 0; o >>= 1) m ^= __shfl_xor_sync(FULL, m, o);
        if (sub == 0 && act) s.par[q] ^= m;
    }
    return tests;
}

template <bool FP32, int NW>
__global__ void __launch_bounds__(NW * 32, 28 / NW) k_pip_refine(RefineArgs a) {
    constexpr int SMAX = PipSmem<FP32>::SMAX;
    extern __shared__ __align__(16) unsigned char pip_smem_raw[];
    const int lane = lane_id(), w = threadIdx.x >> 5;
    PipSmem<FP32> &s = reinterpret_cast<PipSmem<FP32> *>(pip_smem_raw)[w];
    const int n_items = *a.n_items;
    const float FINF = __int_as_float(0x7f800000);
    const unsigned lt_mask = (1u << lane) - 1u;
    unsigned long long c_pairs = 0, c_tests = 0, c_items = 0, c_algo = 0, c_wtests = 0;
    unsigned c_fb = 0, c_hits = 0;

    // Items come from a device counter when a.work_next is set (the next index
    // is fetched at the start of an item, so its latency hides behind the
    // item), else in a fixed stride.
    // a.claim consecutive items per counter update (mostly chunks of one
    // cell, whose staged records are then still in L1).
    // The next item's record and its cell's point range are loaded while the
    // current item is refined, off the per-item chain of dependent loads.
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

        // 1. points, the range of their FP32 y truncations and the smallest x
        // truncation.  Items of more than 32 points: the (up to MAX_CH / 32)
        // point loads of a lane are issued together -- every slot index, then
        // every point as an asynchronous copy into the idle staging area -- so
        // that their latencies overlap instead of forming one chain per point;
        // smaller items (one point per lane) load directly.
        float ylo = FINF, yhi = -FINF, xlo = FINF;
        auto put = [&](int q, double2 p, int src) {
            float hx, lx, hy, ly;
            split_double(p.x, hx, lx);
            split_double(p.y, hy, ly);
            if constexpr (FP32) {
                s.pt[q] = make_float2(rel_coord(hx, lx, fo.x), rel_coord(hy, ly, fo.y));
                s.pyh[q] = hy;
                s.pin[q] = src;
            } else {
                s.pt[q] = p;
            }
            s.found[q] = -1;
            s.par[q] = 0u;
            ylo = fminf(ylo, hy);
            yhi = fmaxf(yhi, hy);
            xlo = fminf(xlo, hx);
        };
        if (np <= 32) {
            if (lane < np) {
                int src = -1;
                double2 p = make_double2(0.0, 0.0);
                if (SJ_IN_BOUNDS(j0 + lane < a.npts, BND_PIP_POINT)) {
                    src = a.spts ? j0 + lane : a.perm[j0 + lane];
                    if (SJ_IN_BOUNDS(src < a.npts, BND_PIP_POINT)) p = a.spts ? __ldcg(a.spts + src) : __ldcg(a.pts + src);
                    else src = -1;
                }
                put(lane, p, src);
            }
        } else {
            constexpr int PQ = MAX_CH / 32;
            double2 *pbuf;
            if constexpr (FP32) {
                static_assert(sizeof(PipSmem<true>::rel) >= MAX_CH * sizeof(double2), "");
                pbuf = reinterpret_cast<double2 *>(&s.rel[0]);
            } else {
                static_assert(sizeof(PipSmem<false>::e) >= MAX_CH * sizeof(double2), "");
                pbuf = reinterpret_cast<double2 *>(&s.e[0]);
            }
            __syncwarp();   // no lane still reads the previous item's staged edges
            int src[PQ];
#pragma unroll
            for (int u = 0; u < PQ; ++u) {
                const int q = lane + 32 * u;
                src[u] = (q < np && SJ_IN_BOUNDS(j0 + q < a.npts, BND_PIP_POINT)) ? (a.spts ? j0 + q : a.perm[j0 + q])
                                                                                 : -1;
                if (src[u] >= 0 && !SJ_IN_BOUNDS(src[u] < a.npts, BND_PIP_POINT)) src[u] = -1;
            }
#pragma unroll
            for (int u = 0; u < PQ; ++u)
                if (src[u] >= 0) copy16_async(pbuf + lane + 32 * u, a.spts ? a.spts + src[u] : a.pts + src[u]);
            copy_async_wait_all();
#pragma unroll
            for (int u = 0; u < PQ; ++u) {
                const int q = lane + 32 * u;
                if (q < np) put(q, src[u] >= 0 ? pbuf[q] : make_double2(0.0, 0.0), src[u]);
            }
        }
        if (a.work_next) it_next = __shfl_sync(FULL, it_next, 0);
        int2 item_n = make_int2(0, 0);
        if (it_next < n_items) item_n = a.items[it_next];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ylo = fminf(ylo, __shfl_xor_sync(FULL, ylo, o));
            yhi = fmaxf(yhi, __shfl_xor_sync(FULL, yhi, o));
            xlo = fminf(xlo, __shfl_xor_sync(FULL, xlo, o));
        }
        __syncwarp();

        for (int kg = k0; kg < k1; kg += 32) {
            int pending = 0;
            for (int q = lane; q < np; q += 32) pending += (s.found[q] < 0);
            pending = __reduce_add_sync(FULL, pending);
            if (pending == 0) break;
            // 2. candidate group: one polygon per lane, its edge list for the
            //    item's grid row, list lengths scanned
            //    (a candidate whose class for this cell is inside / outside
            //    contributes its parity without any edge)
            //    A boundary candidate stages only its near edges; the parity of
            //    its far-right edges comes from the flip keys (k_pip_boundary).
            const int nc = min(32, k1 - kg);
            int pid = 0, vb = 0, ne = 0, nall = 0, cls = 0, fs = 0, fl = 0;
            if (lane < nc) {
                const int k = kg + lane;
                pid = a.cand_ids[k];
                cls = a.cand_cls[k];
                if (cls == 0) {
                    vb = a.bnear_start[k];
                    ne = a.bnear_start[k + 1] - vb;
                    fs = a.bflip_start[k];
                    fl = a.bflip_len[k];
                }
                nall = a.obj_voff[pid + 1] - a.obj_voff[pid];
            }
            const unsigned inside = __ballot_sync(FULL, cls == 1);
            // far-right parity: the number of flip keys at or below the point's y
            for (unsigned far = __ballot_sync(FULL, fl > 0); far; far &= far - 1) {
                const int j = __ffs(far) - 1;
                const int f0 = __shfl_sync(FULL, fs, j), n = __shfl_sync(FULL, fl, j);
                for (int q = lane; q < np; q += 32) {
                    if (s.found[q] >= 0) continue;
                    double py;
                    if constexpr (FP32) py = a.spts ? a.spts[s.pin[q]].y : a.pts[s.pin[q]].y;
                    else py = s.pt[q].y;
                    const unsigned long long ky = y_key(py);
                    int lo = 0, hi = n;   // first key above ky
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (a.bflip_keys[f0 + mid] <= ky) lo = mid + 1;
                        else hi = mid;
                    }
                    if (lo & 1) s.par[q] ^= 1u << j;
                }
            }
            // long near lists: each pending point tests only the edges whose
            // lower truncated y lies in [fl_down(y - h), y] (two binary
            // searches in the sorted list); no other edge of the list can
            // straddle its y (nor tie with it), so the parity is unchanged
            const bool lng = ne > LONG_NEAR;
            for (unsigned lm = __ballot_sync(FULL, lng); lm; lm &= lm - 1) {
                const int j = __ffs(lm) - 1;
                const int b0 = __shfl_sync(FULL, vb, j), n0 = __shfl_sync(FULL, ne, j);
                const float hj = a.bnear_h[kg + j];
                const float *keys = a.bnear_key + b0;
                for (int q = lane; q < np; q += 32) {
                    if (s.found[q] >= 0) continue;
                    float pyh;
                    if constexpr (FP32) pyh = s.pyh[q];
                    else pyh = approx_float(s.pt[q].y);
                    const int lo = key_bound(keys, n0, __fsub_rd(pyh, hj), false);
                    const int hi = key_bound(keys, n0, pyh, true);
                    unsigned par = 0;
                    for (int t = lo; t < hi; ++t)
                        if (SJ_IN_BOUNDS(b0 + t < a.bnear_start[a.cand_start[a.g.G]], BND_PIP_REC))
                            par ^= (unsigned)near_edge_cross<FP32>(a, s, q, b0 + t, fo, c_fb);
                    c_wtests += (unsigned long long)(hi > lo ? hi - lo : 0);
                    if (par & 1u) s.par[q] ^= 1u << j;
                }
            }
            if (lng) ne = 0;   // staged below: the short lists only
            __syncwarp();
            c_pairs += (unsigned long long)pending * (unsigned long long)nc;
            c_algo += (unsigned long long)pending * (unsigned long long)__reduce_add_sync(FULL, (unsigned)nall);
            int incl = ne;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += v;
            }
            const int E = __shfl_sync(FULL, incl, 31);
            __syncwarp();
            if (lane < nc) {
                s.coff[lane] = incl - ne;
                s.cid[lane] = pid;
                s.cvb[lane] = vb;
            }
            if (lane == 0) s.coff[nc] = E;
            __syncwarp();

            // 3. staging with the exact y-range prune, 4. parity when full
            int nst = 0, kw = 0;
            for (int base = 0; base < E; base += 32) {
                const int g = base + lane;
                bool keep = false;
                int i = 0, j = 0, k = 0;
                float4 va = make_float4(0.f, 0.f, 0.f, 0.f), vc = va;
                if (g < E) {
                    while (s.coff[kw + 1] <= g) ++kw;   // candidate of edge g (g grows by 32)
                    k = kw;
                    int e = s.cvb[kw] + (g - s.coff[kw]);
                    if (!SJ_IN_BOUNDS(e < a.bnear_start[a.cand_start[a.g.G]], BND_PIP_REC)) e = 0;
                    i = a.bnear_ids[e];
                    if constexpr (FP32) {
                        va = a.bnear_rec[2 * (size_t)e];
                        vc = a.bnear_rec[2 * (size_t)e + 1];
                    } else {
                        j = a.nxt[i];
                        va = a.vsplit[i];
                        vc = a.vsplit[j];
                    }
                    // y: strictly outside the points' y-range never straddles
                    // (exact compares on monotone truncations).  x: an edge
                    // wholly left of every point cannot cross a ray to +x; the
                    // reference sign is a rounded FP64 orientation, so only
                    // edges clear of the points by far more than its rounding
                    // error (about 1e-10 m here) are dropped: a margin of 8
                    // FP32 ulps plus 1 mm on the truncated coordinates.
                    const float ex = fmaxf(va.x, vc.x);
                    keep = !(fmaxf(va.y, vc.y) < ylo || fminf(va.y, vc.y) > yhi ||
                             ex + fmaf(fabsf(ex) + fabsf(xlo), 9.5367431640625e-07f, 1e-3f) < xlo);
                }
                const unsigned bal = __ballot_sync(FULL, keep);
                if (keep) {
                    const int pos = nst + __popc(bal & lt_mask);
                    if constexpr (FP32) {
                        s.yh[pos] = make_float2(va.y, vc.y);
                        s.rel[pos] = make_float4(rel_coord(va.x, va.z, fo.x), rel_coord(va.y, va.w, fo.y),
                                                 rel_coord(vc.x, vc.z, fo.x), rel_coord(vc.y, vc.w, fo.y));
                        s.vi[pos] = i;
                    } else {
                        const double2 A = a.verts[i], B = a.verts[j];
                        s.e[pos] = Edge64{A.x, A.y, B.x, B.y};
                    }
                    s.kk[pos] = (unsigned char)k;
                }
                nst += __popc(bal);
                if (nst > SMAX - 32 || base + 32 >= E) {
                    __syncwarp();
                    if (nst > 0) c_tests += pip_compute<FP32>(s, a, j0, np, nst, lane, c_fb);
                    __syncwarp();
                    nst = 0;
                }
            }
            // smallest candidate with odd parity
            for (int q = lane; q < np; q += 32) {
                const unsigned m = s.par[q] | inside;
                if (s.found[q] < 0 && m) s.found[q] = s.cid[__ffs(m) - 1];
                s.par[q] = 0u;
            }
            __syncwarp();
        }
        int cs0n = 0, cs1n = 0;
        if (it_next < n_items) {
            cs0n = a.cell_start[item_n.x];
            cs1n = a.cell_start[item_n.x + 1];
        }
        for (int q = lane; q < np; q += 32) {
            const int f = s.found[q];
            if (!SJ_IN_BOUNDS(j0 + q < a.npts, BND_PIP_RES)) continue;
            if (a.res_id) a.res_id[j0 + q] = f;
            else if (f >= 0) a.out_id[a.perm[j0 + q]] = f;
            if (f >= 0) ++c_hits;
        }
        __syncwarp();
        it_end = in_claim ? it_end : it_next + (a.work_next ? claim : 1);
        it = it_next;
        item = item_n;
        cs0 = cs0n;
        cs1 = cs1n;
    }
    if (a.stats) {
        c_fb = __reduce_add_sync(FULL, c_fb);
        c_hits = __reduce_add_sync(FULL, c_hits);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c_wtests += __shfl_xor_sync(FULL, c_wtests, o);
        unsigned long long v[ST_N] = {};
        v[ST_ITEMS] = c_items;
        v[ST_PAIRS] = c_pairs;
        v[ST_TESTS] = c_tests + c_wtests;   // staged tests (warp-uniform) + window tests
        v[ST_ALGO] = c_algo;
        v[ST_FALLBACK] = c_fb;
        v[ST_HITS] = c_hits;
        flush_stats(a.stats, v);
    }
}

// Cell classification (layer build), one warp per cell.  For a candidate P of
// cell c, the only edges that can straddle the horizontal line of a point of c
// are those of P's list for c's row.  If none of them meets the cell box
// widened by delta, every point of the cell lies at least delta from each of
// them, so (i) the straight path from the point to the cell centre crosses no
// edge -- all points of the cell share the centre's inside/outside status --
// and (ii) the FP64 crossing rule evaluates every such edge with the correct
// orientation sign (its rounding error is below 1e-10 m at coordinates of
// 1e5 m, delta is far larger), so the rule gives each point that status.  The
// class is then the FP64 crossing parity of the centre: 1 inside, 2 outside;
// 0 (boundary) when some edge meets the widened box.  The cell box is the
// exact set of doubles the cell rule maps to the cell: [key_value(kx[ix]),
// key_value(kx[ix + 1])) and likewise in y.
__global__ void k_pip_classify(GridDev g, const int *cand_start, const int *cand_ids, const int *prow_base,
                               const int *prow_r0, const int *prow_start, const int *pedge_ids, const int *nxt,
                               const double2 *verts, double delta, unsigned char *cls) {
    const int lane = lane_id();
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int c = warp; c < g.G; c += nwarps) {
        const int k0 = cand_start[c], k1 = cand_start[c + 1];
        if (k0 == k1) continue;
        const int ix = c % g.nx, iy = c / g.nx;
        const double X0 = key_value(g.kx[ix]), X1 = key_value(g.kx[ix + 1]);
        const double Y0 = key_value(g.ky[iy]), Y1 = key_value(g.ky[iy + 1]);
        const double bx0 = X0 - delta, bx1 = X1 + delta, by0 = Y0 - delta, by1 = Y1 + delta;
        const double cx = 0.5 * (X0 + X1), cy = 0.5 * (Y0 + Y1);
        for (int k = k0; k < k1; ++k) {
            const int P = cand_ids[k];
            const int slot = prow_base[P] + (iy - prow_r0[P]);
            const int e0 = prow_start[slot], e1 = prow_start[slot + 1];
            int hit = 0, par = 0;
            for (int e = e0 + lane; e < e1; e += 32) {
                const int i = pedge_ids[e];
                const double2 A = verts[i], B = verts[nxt[i]];
                hit |= !(fmax(A.x, B.x) < bx0 || fmin(A.x, B.x) > bx1 || fmax(A.y, B.y) < by0 ||
                         fmin(A.y, B.y) > by1);
                par ^= cross64(cx, cy, A.x, A.y, B.x, B.y);
            }
            hit = __reduce_or_sync(FULL, (unsigned)hit);
            par = (int)(__reduce_xor_sync(FULL, (unsigned)par) & 1u);
            if (lane == 0) cls[k] = hit ? 0 : (par ? 1 : 2);
        }
    }
}

// Per cell of a polygon layer: the result every point of the cell gets when
// each of its candidates is classified (class 1 inside or 2 outside) -- the
// smallest candidate whose class is inside (candidate ids are sorted), or -1
// -- else CELL_REFINE: some candidate is a boundary candidate and the cell's
// points go through the refinement.  Cells without candidates get -1.
__global__ void k_cell_result(const int *cand_start, const int *cand_ids, const unsigned char *cls, int G, int *res) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < G; c += gridDim.x * blockDim.x) {
        int r = -1;
        for (int k = cand_start[c]; k < cand_start[c + 1]; ++k) {
            if (cls[k] == 0) {
                r = CELL_REFINE;
                break;
            }
            if (cls[k] == 1 && r == -1) r = cand_ids[k];
        }
        res[c] = r;
    }
}

cudaError_t launch_cell_result(const int *cand_start, const int *cand_ids, const unsigned char *cls, int G, int *res,
                               cudaStream_t s) {
    const int nb = (int)std::max<long long>(1, std::min<long long>(((long long)G + 255) / 256, 152LL * 32));
    k_cell_result<<<nb, 256, 0, s>>>(cand_start, cand_ids, cls, G, res);
    return cudaGetLastError();
}

// Per-point edge work of each cell of a polygon layer (the split of work
// items by candidate-edge count): the near edges of its boundary candidates,
// a long list (searched per point) counted as LONG_NEAR.
__global__ void k_cell_work_pip(const int *cand_start, const unsigned char *cls, const int *near_start, int G,
                                int *work) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < G; c += gridDim.x * blockDim.x) {
        long long w = 0;
        for (int k = cand_start[c]; k < cand_start[c + 1]; ++k)
            if (cls[k] == 0) w += min(near_start[k + 1] - near_start[k], LONG_NEAR);
        work[c] = (int)min(w, 2147483647LL);
    }
}

cudaError_t launch_cell_work_pip(const int *cand_start, const unsigned char *cls, const int *near_start, int G,
                                 int *work, cudaStream_t s) {
    const int nb = (int)std::max<long long>(1, std::min<long long>(((long long)G + 255) / 256, 152LL * 32));
    k_cell_work_pip<<<nb, 256, 0, s>>>(cand_start, cls, near_start, G, work);
    return cudaGetLastError();
}

cudaError_t launch_pip_classify(const GridDev &g, const int *cand_start, const int *cand_ids, const int *prow_base,
                                const int *prow_r0, const int *prow_start, const int *pedge_ids, const int *nxt,
                                const double2 *verts, double delta, unsigned char *cls, cudaStream_t s) {
    const long long nb = std::min<long long>(((long long)g.G * 32 + 255) / 256, 152LL * 64);
    k_pip_classify<<<(int)std::max<long long>(nb, 1), 256, 0, s>>>(g, cand_start, cand_ids, prow_base, prow_r0,
                                                                  prow_start, pedge_ids, nxt, verts, delta, cls);
    return cudaGetLastError();
}

// Boundary entries (class 0), one warp per cell.  The candidate's row-list
// edges split three ways against the cell's column [X0, X1) widened by delta:
//   left  (max x < X0 - delta): farther than delta left of every point of the
//         cell, so the FP64 rule never counts a crossing -- dropped;
//   far   (min x > X1 + delta): farther than delta right of every point, so
//         the FP64 rule counts a crossing exactly when the edge straddles the
//         point's y (its orientation sign is far above rounding) -- the parity
//         of those straddles is the parity of the number of end y-values
//         (lower and upper end of each far edge) at or below the point's y,
//         since an edge straddles y iff lower <= y < upper;
//   near  (the rest): tested point by point in the refinement.
// An end shared with the ring's adjacent edge counts twice when that edge is a
// far edge of the same list too (the same vertex, the same y), which leaves
// the parity unchanged: such ends are not emitted, so only the ends of chains
// of far edges remain.
// Count pass: near edges and far end values per entry.  Emit pass: near edge
// ids and far end keys (order keys, -0 folded onto +0).
__device__ __forceinline__ bool far_in_list(const BoundaryArgs &a, int u, int w, double XR, int iy) {
    const double2 U = a.verts[u], W = a.verts[w];
    if (!(fmin(U.x, W.x) > XR)) return false;
    const int ra = clamped_axis(fmin(U.y, W.y), a.g.y0, a.g.ch, a.g.ny);
    const int rb = clamped_axis(fmax(U.y, W.y), a.g.y0, a.g.ch, a.g.ny);
    return ra <= iy && iy <= rb;
}

__global__ void k_pip_boundary(BoundaryArgs a, int emit) {
    const int lane = lane_id();
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int c = warp; c < a.g.G; c += nwarps) {
        const int k0 = a.cand_start[c], k1 = a.cand_start[c + 1];
        if (k0 == k1) continue;
        const int ix = c % a.g.nx, iy = c / a.g.nx;
        const double XL = key_value(a.g.kx[ix]) - a.delta, XR = key_value(a.g.kx[ix + 1]) + a.delta;
        for (int k = k0; k < k1; ++k) {
            if (a.cls[k] != 0) {
                if (!emit && lane == 0) a.near_cnt[k] = a.flip_cnt[k] = 0;
                continue;
            }
            const int P = a.cand_ids[k];
            const int slot = a.prow_base[P] + (iy - a.prow_r0[P]);
            const int e0 = a.prow_start[slot], e1 = a.prow_start[slot + 1];
            int nn = 0, nf = 0;   // running counts (uniform across the warp)
            for (int b = e0; b < e1; b += 32) {
                const int e = b + lane;
                bool is_near = false, ks = false, ke = false;
                int i = 0;
                double ys = 0.0, ye = 0.0;
                if (e < e1) {
                    i = a.pedge_ids[e];
                    const int j = a.nxt[i];
                    const double2 A = a.verts[i], B = a.verts[j];
                    const double xmin = fmin(A.x, B.x), xmax = fmax(A.x, B.x);
                    const bool is_far = xmin > XR;
                    is_near = !is_far && !(xmax < XL);
                    if (is_far) {
                        ks = !far_in_list(a, a.prv[i], i, XR, iy);   // start shared with the previous edge
                        ke = !far_in_list(a, j, a.nxt[j], XR, iy);   // end shared with the next edge
                    }
                    ys = A.y;
                    ye = B.y;
                }
                const unsigned bn = __ballot_sync(FULL, is_near);
                const unsigned bs = __ballot_sync(FULL, ks), be = __ballot_sync(FULL, ke);
                if (emit) {
                    if (is_near) a.near_ids[a.near_start[k] + nn + __popc(bn & lt)] = i;
                    const int f = a.flip_start[k] + nf + __popc(bs & lt) + __popc(be & lt);
                    if (ks) a.flip_keys[f] = y_key(ys);
                    if (ke) a.flip_keys[f + (ks ? 1 : 0)] = y_key(ye);
                }
                nn += __popc(bn);
                nf += __popc(bs) + __popc(be);
            }
            if (!emit && lane == 0) {
                a.near_cnt[k] = nn;
                a.flip_cnt[k] = nf;
            }
        }
    }
}

// Sort each entry's far end keys and drop pairs of equal keys (a value counted
// twice does not change the parity); len[k] = the keys left.  One thread per
// entry, Shell sort (Ciura gaps).
__global__ void k_pip_flips(const int *flip_start, int M, unsigned long long *keys, int *len) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
        const int b = flip_start[k], n = flip_start[k + 1] - b;
        unsigned long long *v = keys + b;
        const int ciura[8] = {1, 4, 10, 23, 57, 132, 301, 701};
        int gaps[32];
        int ng = 0;
        while (ng < 8 && ciura[ng] < n) { gaps[ng] = ciura[ng]; ++ng; }
        if (ng == 8) {
            long long g = 701;
            while (ng < 32 && (g = g * 9 / 4) < n) gaps[ng++] = (int)g;
        }
        for (int u = ng - 1; u >= 0; --u) {
            const int h = gaps[u];
            for (int i = h; i < n; ++i) {
                const unsigned long long x = v[i];
                int j = i;
                while (j >= h && v[j - h] > x) { v[j] = v[j - h]; j -= h; }
                v[j] = x;
            }
        }
        int m = 0;
        for (int i = 0; i < n;) {   // runs of equal keys: keep one key of an odd run
            int j = i + 1;
            while (j < n && v[j] == v[i]) ++j;
            if ((j - i) & 1) v[m++] = v[i];
            i = j;
        }
        len[k] = m;
    }
}

// Near lists sorted by lower y (layer build), one thread per boundary entry:
// key = min(trunc32(a.y), trunc32(b.y)) of each near edge (the FP32 truncations
// the refinement compares, a monotone map of y), ids reordered by key (Shell
// sort, Ciura gaps), and h[k] = the largest max - min of the two truncations
// over the entry's edges, rounded up.  An edge of the list can straddle (or
// tie with) a point's truncated y only if its key lies in
// [fl_down(y - h), y]: the refinement finds that window by binary search.
__global__ void k_pip_near_sort(const int *near_start, int M, int *ids, const int *nxt, const float4 *vsplit,
                                float *keys, float *h) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
        const int b = near_start[k], n = near_start[k + 1] - b;
        float hk = 0.0f;
        for (int t = 0; t < n; ++t) {
            const int i = ids[b + t];
            const float ya = vsplit[i].y, yb = vsplit[nxt[i]].y;
            keys[b + t] = fminf(ya, yb);
            hk = fmaxf(hk, __fsub_ru(fmaxf(ya, yb), fminf(ya, yb)));
        }
        h[k] = hk;
        const int ciura[8] = {1, 4, 10, 23, 57, 132, 301, 701};
        int gaps[32];
        int ng = 0;
        while (ng < 8 && ciura[ng] < n) { gaps[ng] = ciura[ng]; ++ng; }
        if (ng == 8) {
            long long g = 701;
            while (ng < 32 && (g = g * 9 / 4) < n) gaps[ng++] = (int)g;
        }
        float *kv = keys + b;
        int *iv = ids + b;
        for (int u = ng - 1; u >= 0; --u) {
            const int gp = gaps[u];
            for (int i = gp; i < n; ++i) {
                const float x = kv[i];
                const int xi = iv[i];
                int j = i;
                while (j >= gp && kv[j - gp] > x) {
                    kv[j] = kv[j - gp];
                    iv[j] = iv[j - gp];
                    j -= gp;
                }
                kv[j] = x;
                iv[j] = xi;
            }
        }
    }
}

cudaError_t launch_pip_near_sort(const int *near_start, int M, int *ids, const int *nxt, const float4 *vsplit,
                                 float *keys, float *h, cudaStream_t s) {
    const int nb = std::max(1, std::min((M + 127) / 128, 8192));
    k_pip_near_sort<<<nb, 128, 0, s>>>(near_start, M, ids, nxt, vsplit, keys, h);
    return cudaGetLastError();
}

cudaError_t launch_pip_boundary(const BoundaryArgs &a, int emit, cudaStream_t s) {
    const long long nb = std::min<long long>(((long long)a.g.G * 32 + 255) / 256, 152LL * 64);
    k_pip_boundary<<<(int)std::max<long long>(nb, 1), 256, 0, s>>>(a, emit);
    return cudaGetLastError();
}

cudaError_t launch_pip_flips(const int *flip_start, int M, unsigned long long *keys, int *len, cudaStream_t s) {
    const int nb = std::max(1, std::min((M + 127) / 128, 8192));
    k_pip_flips<<<nb, 128, 0, s>>>(flip_start, M, keys, len);
    return cudaGetLastError();
}

// Census of the algorithmic PIP work (a measurement pass, not part of a
// join): for every in-grid point, out[0] += the edges of its cell's candidate
// polygons (every ring), out[1] += how many of them straddle the point's y
// under the crossing rule's straddle test (Sec. III.C).  Only an edge of a
// candidate's list for the point's grid row can straddle it (the row lists are
// exact), so the straddles are counted over those lists.  One thread per point.
__global__ void k_pip_census(RefineArgs a, const double2 *pts, int n, unsigned long long *out) {
    unsigned long long e = 0, st = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double2 p = pts[i];
        const int c = point_cell(a.g, p.x, p.y);
        if (c >= a.g.G) continue;
        const int iy = c / a.g.nx;
        for (int k = a.cand_start[c]; k < a.cand_start[c + 1]; ++k) {
            const int P = a.cand_ids[k];
            e += (unsigned long long)(a.obj_voff[P + 1] - a.obj_voff[P]);
            const int slot = a.prow_base[P] + (iy - a.prow_r0[P]);
            for (int t = a.prow_start[slot]; t < a.prow_start[slot + 1]; ++t) {
                const int v = a.pedge_ids[t];
                st += (unsigned long long)((a.verts[v].y > p.y) != (a.verts[a.nxt[v]].y > p.y));
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(FULL, e, o);
        st += __shfl_xor_sync(FULL, st, o);
    }
    if (lane_id() == 0) {
        atomicAdd(&out[0], e);
        atomicAdd(&out[1], st);
    }
}

cudaError_t launch_pip_census(const RefineArgs &a, const double2 *pts, int n, unsigned long long *out,
                              cudaStream_t s) {
    const int nb = std::max(1, std::min((n + 255) / 256, 152 * 16));
    k_pip_census<<<nb, 256, 0, s>>>(a, pts, n, out);
    return cudaGetLastError();
}

template <bool FP32, int NW>
static size_t pip_smem_bytes() {
    return sizeof(PipSmem<FP32>) * NW;
}

template <bool FP32, int NW>
static cudaError_t pip_prepare() {
    static bool done = false;
    if (!done) {
        cudaError_t e = cudaFuncSetAttribute(k_pip_refine<FP32, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)pip_smem_bytes<FP32, NW>());
        if (e != cudaSuccess) return e;
        done = true;
    }
    return cudaSuccess;
}

template <bool FP32, int NW>
static cudaError_t pip_launch(const RefineArgs &a, int blocks, cudaStream_t s) {
    cudaError_t e = pip_prepare<FP32, NW>();
    if (e != cudaSuccess) return e;
    k_pip_refine<FP32, NW><<<blocks, NW * 32, pip_smem_bytes<FP32, NW>(), s>>>(a);
    return cudaGetLastError();
}

// blocks: the grid for blocks of PIP_WARPS warps; a block of warps_per_block
// (2, 4 or 8) warps gets the same number of warps.
cudaError_t launch_pip_refine(const RefineArgs &a, int form, int warps_per_block, int blocks, cudaStream_t s) {
    const int nw = (warps_per_block == 2 || warps_per_block == 8) ? warps_per_block : PIP_WARPS;
    blocks = (int)(((long long)blocks * PIP_WARPS + nw - 1) / nw);
    if (form == SJ_FP32X) {
        if (nw == 2) return pip_launch<true, 2>(a, blocks, s);
        if (nw == 8) return pip_launch<true, 8>(a, blocks, s);
        return pip_launch<true, PIP_WARPS>(a, blocks, s);
    }
    if (nw == 2) return pip_launch<false, 2>(a, blocks, s);
    if (nw == 8) return pip_launch<false, 8>(a, blocks, s);
    return pip_launch<false, PIP_WARPS>(a, blocks, s);
}

int pip_blocks_per_sm(int form) {
    int n = 0;
    if (form == SJ_FP32X) {
        if (pip_prepare<true, PIP_WARPS>() != cudaSuccess) return 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pip_refine<true, PIP_WARPS>, PIP_WARPS * 32,
                                                      pip_smem_bytes<true, PIP_WARPS>());
    } else {
        if (pip_prepare<false, PIP_WARPS>() != cudaSuccess) return 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pip_refine<false, PIP_WARPS>, PIP_WARPS * 32,
                                                      pip_smem_bytes<false, PIP_WARPS>());
    }
    return n > 0 ? n : 1;
}

}  // namespace sj
