// sj_api.cu -- C ABI of libsj.so (declared in include/sj.h): argument checks,
// layer construction (validation, MBBs, candidate lists) and the join
// pipelines (bucketing -> work items -> refinement), all stream-ordered.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <cmath>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "sj_host.hpp"

namespace sj {
cudaError_t launch_check_offsets(const int64_t *off, int64_t n, int64_t min_size, int64_t first, int64_t last, int *out,
                                 int *bad, cudaStream_t s);
cudaError_t launch_check_finite(const double2 *v, int n, int *bad, cudaStream_t s);
cudaError_t launch_pip_topology(const int *ring_off, int R, const int *poly_ring_off, int P, int *poly_voff, int *nxt,
                                int *prv, cudaStream_t s);
cudaError_t launch_split(const double2 *v, int n, float4 *vs, cudaStream_t s);
cudaError_t launch_seg_table(const double2 *v, const int *line_off, int L, double2 *e64, double *inv64, float4 *seg32,
                             cudaStream_t s);
cudaError_t launch_mbb(const LayerBuildArgs &a, cudaStream_t s);
cudaError_t launch_raster_count(const LayerBuildArgs &a, unsigned long long *total, cudaStream_t s);
cudaError_t launch_raster_emit(const LayerBuildArgs &a, int2 *pairs, int M, int *cand_ids, cudaStream_t s);
cudaError_t launch_segcell_count(const LayerBuildArgs &a, const float4 *seg32, const double2 *e64, int *seg_off,
                                 unsigned long long *total, cudaStream_t s);
cudaError_t launch_segcell_emit(const LayerBuildArgs &a, const float4 *seg32, const double2 *e64, const int *seg_off,
                                int2 *pairs, int MS, const int *cand_ids, int *cseg_start, int *cseg_ids,
                                int *cell_algo, cudaStream_t s);
cudaError_t launch_prow_count(const LayerBuildArgs &a, int *prow_base, int *prow_r0, unsigned long long *total,
                              cudaStream_t s);
cudaError_t launch_prow_edge_count(const LayerBuildArgs &a, const int *nxt, const int *prow_base, const int *prow_r0,
                                   int *cnt, unsigned long long *total, cudaStream_t s);
cudaError_t launch_prow_edge_emit(const LayerBuildArgs &a, const int *nxt, const int *prow_base, const int *prow_r0,
                                  const int *cnt, int slots, int *prow_start, int *cursor, int *pedge_ids,
                                  cudaStream_t s);
cudaError_t launch_cseg_records(const int *cseg_start, const int *cseg_ids, const GridDev &g, const float *frame_x,
                                const float *frame_y, const float4 *vsplit, const float4 *seg32, float4 *rec,
                                cudaStream_t s);
cudaError_t launch_prow_records(const int *pedge_ids, long long ME, const int *nxt, const float4 *vsplit,
                                float4 *rec, cudaStream_t s);
cudaError_t launch_offsets(const int *cnt, int n, int *out, int2 *block_sums, size_t cap, int *totals,
                           cudaStream_t s);
cudaError_t launch_sum64(const int *cnt, int n, unsigned long long *total, cudaStream_t s);
cudaError_t launch_thresholds(const GridDev &g, unsigned long long *kx, unsigned long long *ky, cudaStream_t s);
cudaError_t launch_frames(const GridDev &g, float *fx, float *fy, cudaStream_t s);
int pip_blocks_per_sm(int form);
int p2p_blocks_per_sm(int form);
}  // namespace sj

using namespace sj;


// ------------------------------------------------------------------ errors

static thread_local std::string g_err;

sj_status sj::fail(sj_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

sj_status sj::cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorMemoryAllocation ? SJ_ERR_OOM : SJ_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

// ------------------------------------------------------------------ bounds-checked build

// After a join of a build compiled with SJ_CHECK_BOUNDS: synchronise the
// stream and read the kernels' error words; a guard that fired (an index out
// of range, skipped on the device) makes the call fail with SJ_ERR_CUDA.  In
// normal builds: nothing.
static sj_status check_bounds(cudaStream_t s) {
#ifdef SJ_CHECK_BOUNDS
    CUDA_TRY(cudaStreamSynchronize(s));
    const unsigned v = bounds_take_filter() | bounds_take_p2p() | bounds_take_pip();
    if (v) return fail(SJ_ERR_CUDA, "bounds check: out-of-range device accesses skipped, guard codes " +
                                        std::to_string(v));
#else
    (void)s;
#endif
    return SJ_OK;
}

extern "C" int32_t sj_bounds_checked(void) {
#ifdef SJ_CHECK_BOUNDS
    return 1;
#else
    return 0;
#endif
}

// ------------------------------------------------------------------ fault injection

static std::mutex g_fault_mu;
static int g_fault_kind = SJ_FAULT_NONE, g_fault_after = 0, g_fault_count = 0;

bool sj::fault_fires(int kind) {
    std::lock_guard<std::mutex> lk(g_fault_mu);
    if (g_fault_kind != kind || g_fault_count <= 0) return false;
    if (g_fault_after > 0) {
        --g_fault_after;
        return false;
    }
    if (--g_fault_count == 0) g_fault_kind = SJ_FAULT_NONE;
    return true;
}

cudaError_t sj::dev_malloc(void **p, size_t bytes) {
    if (fault_fires(SJ_FAULT_ALLOC)) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

cudaError_t sj::dev_malloc_async(void **p, size_t bytes, cudaStream_t s) {
    if (fault_fires(SJ_FAULT_ALLOC)) return cudaErrorMemoryAllocation;
    return cudaMallocAsync(p, bytes, s);
}

extern "C" sj_status sj_fault_inject(int32_t kind, int32_t after, int32_t count) {
    if (kind != SJ_FAULT_NONE && kind != SJ_FAULT_ALLOC && kind != SJ_FAULT_ADMIT)
        return fail(SJ_ERR_INVALID, "unknown fault kind");
    if (after < 0 || count < 0) return fail(SJ_ERR_INVALID, "after and count must be >= 0");
    std::lock_guard<std::mutex> lk(g_fault_mu);
    g_fault_kind = count > 0 ? kind : SJ_FAULT_NONE;
    g_fault_after = after;
    g_fault_count = count;
    return SJ_OK;
}

extern "C" int32_t sj_fault_pending(void) {
    std::lock_guard<std::mutex> lk(g_fault_mu);
    return g_fault_kind == SJ_FAULT_NONE ? 0 : g_fault_count;
}

// ------------------------------------------------------------------ device info

static DevInfo g_dev[64];
static std::mutex g_dev_mu;

sj_status sj::device_info(int dev, DevInfo **out) {
    if (dev < 0 || dev >= 64) return fail(SJ_ERR_INVALID, "device index out of range");
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DevInfo &d = g_dev[dev];
    if (!d.init) {
        CUDA_TRY(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
        for (int f = 0; f < 2; ++f) {
            d.pip_bps[f] = pip_blocks_per_sm(f);
            d.p2p_bps[f] = p2p_blocks_per_sm(f);
        }
        // keep freed stream-ordered scratch in the pool for the next call
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        for (cudaStream_t &hs : d.hstream) CUDA_TRY(cudaStreamCreateWithFlags(&hs, cudaStreamNonBlocking));
        d.init = true;
    }
    *out = &d;
    return SJ_OK;
}

static bool grid_ok(const sj_grid *g) {
    if (!g) return false;
    if (!(g->nx >= 1 && g->ny >= 1)) return false;
    if (g->nx > (1 << 20) || g->ny > (1 << 20)) return false;
    if ((int64_t)g->nx * (int64_t)g->ny > MAX_COUNT) return false;
    if (!(std::isfinite(g->x0) && std::isfinite(g->x1) && std::isfinite(g->y0) && std::isfinite(g->y1))) return false;
    return g->x1 > g->x0 && g->y1 > g->y0;
}

static GridDev make_grid(const sj_grid *g) {
    GridDev d;
    d.x0 = g->x0; d.y0 = g->y0; d.x1 = g->x1; d.y1 = g->y1;
    d.nx = g->nx; d.ny = g->ny;
    d.G = g->nx * g->ny;
    volatile double cw = (g->x1 - g->x0) / (double)g->nx;   // one IEEE division each
    volatile double ch = (g->y1 - g->y0) / (double)g->ny;
    d.cw = cw; d.ch = ch;
    d.x0f = (float)g->x0; d.y0f = (float)g->y0;
    d.icwf = (float)(1.0 / cw); d.ichf = (float)(1.0 / ch);
    d.kx = d.ky = nullptr;
    return d;
}

// Threshold tables of point_cell for the grid of layer L (computed on the GPU
// with the FP64 cell rule itself).
static sj_status layer_tables(sj_layer *L, cudaStream_t s) {
    CUDA_TRY(dev_malloc((void **)&L->cell_keys, sizeof(unsigned long long) * ((size_t)L->g.nx + L->g.ny + 2)));
    CUDA_TRY(launch_thresholds(L->g, L->cell_keys, L->cell_keys + L->g.nx + 1, s));
    L->g.kx = L->cell_keys;
    L->g.ky = L->cell_keys + L->g.nx + 1;
    CUDA_TRY(dev_malloc((void **)&L->frames, sizeof(float) * ((size_t)L->g.nx + L->g.ny)));
    CUDA_TRY(launch_frames(L->g, L->frames, L->frames + L->g.nx, s));
    L->xmax = std::max(std::max(std::fabs(L->grid.x0), std::fabs(L->grid.x1)),
                       std::max(std::fabs(L->grid.y0), std::fabs(L->grid.y1)));
    return SJ_OK;
}

// FP32 float at or below (down) / at or above (up) the double x.
static float float_down(double x) {
    float f = (float)x;
    return ((double)f > x) ? std::nextafter(f, -INFINITY) : f;
}
static float float_up(double x) {
    float f = (float)x;
    return ((double)f < x) ? std::nextafter(f, INFINITY) : f;
}

// Layer-dependent fields of the refinement arguments.
void sj::fill_refine(const sj_layer *L, RefineArgs &ra) {
    ra.g = L->g;
    ra.cand_start = L->cand_start;
    ra.cand_ids = L->cand_ids;
    ra.obj_voff = L->obj_voff;
    ra.nxt = L->nxt;
    ra.verts = L->verts;
    ra.vsplit = L->vsplit;
    ra.seg_e64 = L->seg_e64;
    ra.seg_inv64 = L->seg_inv64;
    ra.seg32 = L->seg32;
    ra.cseg_start = L->cseg_start;
    ra.cseg_ids = L->cseg_ids;
    ra.cell_algo = L->cell_algo;
    ra.cseg_rec = L->cseg_rec;
    ra.prow_base = L->prow_base;
    ra.prow_r0 = L->prow_r0;
    ra.prow_start = L->prow_start;
    ra.pedge_ids = L->pedge_ids;
    ra.pedge_rec = L->pedge_rec;
    ra.cand_cls = L->cand_cls;
    ra.bnear_start = L->bnear_start;
    ra.bnear_ids = L->bnear_ids;
    ra.bnear_rec = L->bnear_rec;
    ra.bnear_key = L->bnear_key;
    ra.bnear_h = L->bnear_h;
    ra.bflip_start = L->bflip_start;
    ra.bflip_len = L->bflip_len;
    ra.bflip_keys = L->bflip_keys;
    ra.D = L->D;
    ra.Df = L->Df;
    ra.Ddn = L->Ddn;
    ra.Dup = L->Dup;
    ra.eps_abs = L->eps_abs;
    ra.frame_x = L->frames;
    ra.frame_y = L->frames + L->g.nx;
    ra.stats = L->stats;
}

// ------------------------------------------------------------------ layers

// Sum and destroy the pending timing events (the device must be idle).
static void resolve_events(const sj_layer *L) {
    std::lock_guard<std::mutex> lk(L->ev_mu);
    for (auto &p : L->ev_pending) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, p.first, p.second) == cudaSuccess) {
            L->refine_ms += ms;
            L->refine_launches += 1;
        }
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    L->ev_pending.clear();
}

static void layer_free(sj_layer *L) {
    resolve_events(L);
    void *ptrs[] = {L->verts, L->vsplit, L->obj_voff, L->nxt, L->prv, L->ring_off, L->poly_ring_off, L->seg_e64,
                    L->seg_inv64, L->seg32, L->mbb, L->cand_start, L->cand_ids, L->stats, L->cell_keys,
                    L->frames, L->cseg_start, L->cseg_ids, L->cell_algo, L->cseg_rec, L->prow_base, L->prow_r0,
                    L->prow_start, L->pedge_ids, L->pedge_rec, L->cand_cls, L->cell_res, L->cell_work,
                    L->bnear_start, L->bnear_ids,
                    L->bnear_rec, L->bnear_key, L->bnear_h, L->bflip_start, L->bflip_len, L->bflip_keys};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete L;
}

struct LayerGuard {
    sj_layer *L;
    ~LayerGuard() {
        if (L) layer_free(L);
    }
};

template <class T>
static cudaError_t dalloc(T **p, size_t n) {
    return dev_malloc((void **)p, (n ? n : 1) * sizeof(T));
}

static sj_status read_flag(int *dflag, cudaStream_t s, int *out) {
    CUDA_TRY(cudaMemcpyAsync(out, dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return SJ_OK;
}

// Shared tail of both layer builders: MBB, cover check, rasterisation, CSR.
static sj_status build_candidates(sj_layer *L, int *dbad, cudaStream_t s) {
    LayerBuildArgs a{};
    a.g = L->g;
    a.kind = L->kind;
    a.D = L->D;
    a.nobj = L->nobj;
    a.V = L->V;
    a.verts = L->verts;
    a.obj_voff = L->obj_voff;
    a.bad = dbad;
    CUDA_TRY(dalloc(&L->mbb, (size_t)L->nobj));
    CUDA_TRY(dalloc(&L->cand_start, (size_t)L->g.G + 1));
    a.mbb = L->mbb;
    a.cand_start = L->cand_start;

    int *cell_cnt = nullptr, *cursor = nullptr, *obj_cells = nullptr, *totals = nullptr;
    int2 *block_sums = nullptr, *pairs = nullptr;
    unsigned long long *total = nullptr;
    size_t nbs = bucket_scan_blocks(std::max(L->g.G, L->nobj));
    struct Tmp {
        void *p[7] = {};
        ~Tmp() {
            for (void *q : p)
                if (q) cudaFree(q);
        }
    } tmp;
    CUDA_TRY(dalloc(&cell_cnt, (size_t)L->g.G + 1)); tmp.p[0] = cell_cnt;
    CUDA_TRY(dalloc(&cursor, (size_t)L->g.G)); tmp.p[1] = cursor;
    CUDA_TRY(dalloc(&obj_cells, (size_t)L->nobj + 1)); tmp.p[2] = obj_cells;
    CUDA_TRY(dalloc(&block_sums, nbs)); tmp.p[3] = block_sums;
    CUDA_TRY(dalloc(&totals, 4)); tmp.p[4] = totals;
    CUDA_TRY(dalloc(&total, 1)); tmp.p[5] = total;
    CUDA_TRY(cudaMemsetAsync(cell_cnt, 0, sizeof(int) * ((size_t)L->g.G + 1), s));
    CUDA_TRY(cudaMemsetAsync(cursor, 0, sizeof(int) * (size_t)L->g.G, s));
    CUDA_TRY(cudaMemsetAsync(total, 0, sizeof(unsigned long long), s));
    a.cell_cnt = cell_cnt;
    a.cursor = cursor;
    a.obj_cells = obj_cells;
    a.block_sums = block_sums;
    a.bs_cap = nbs;
    a.totals = totals;

    if (L->nobj > 0) {
        CUDA_TRY(launch_mbb(a, s));
        int bad = 0;
        sj_status st = read_flag(dbad, s, &bad);
        if (st != SJ_OK) return st;
        if (bad & 2) return fail(SJ_ERR_GRID_COVER, "an object's MBB is not inside the closed grid box");
        CUDA_TRY(launch_raster_count(a, total, s));
    }
    unsigned long long M = 0;
    CUDA_TRY(cudaMemcpyAsync(&M, total, sizeof(M), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (M > (unsigned long long)MAX_COUNT) return fail(SJ_ERR_INVALID, "more than 2^31 - 2^22 (cell, object) candidate pairs");
    L->M = (int64_t)M;
    CUDA_TRY(dalloc(&L->cand_ids, (size_t)M));
    if (L->nobj > 0) {
        CUDA_TRY(dalloc(&pairs, (size_t)M)); tmp.p[6] = pairs;
        CUDA_TRY(launch_raster_emit(a, pairs, (int)M, L->cand_ids, s));
    } else {
        CUDA_TRY(cudaMemsetAsync(L->cand_start, 0, sizeof(int) * ((size_t)L->g.G + 1), s));
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    // The cell-relative coordinate rel = fl32(fl32(hi - o) + lo) of any value v
    // in the grid box satisfies |rel - (v - o)| <= 2.0001 u |rel| + eps_abs with
    // eps_abs = 6.0001 u^2 max|coordinate| (the truncation remainder |lo| is
    // below 2u |v|, rounded once more by the conversion); 8 u^2 is used.
    double u = 5.9604644775390625e-08;
    L->eps_abs = (float)(8.0 * u * u * L->xmax * (1.0 + 1e-6)) + 1e-30f;
    L->Df = (float)L->D;
    L->Ddn = float_down(L->D * (1.0 - 1e-12));
    L->Dup = float_up(L->D * (1.0 + 1e-12) + 1e-300);
    return SJ_OK;
}

// P2P per-cell segment lists (after build_candidates): every segment whose box
// widened by D meets a cell is listed under that cell, sorted by segment index.
static sj_status build_seg_lists(sj_layer *L, cudaStream_t s) {
    const int G = L->g.G, V = L->V;
    CUDA_TRY(dalloc(&L->cseg_start, (size_t)G + 1));
    CUDA_TRY(dalloc(&L->cell_algo, (size_t)G));
    if (V == 0) {
        L->MS = 0;
        CUDA_TRY(dalloc(&L->cseg_ids, 0));
        CUDA_TRY(dalloc(&L->cseg_rec, 0));
        CUDA_TRY(dalloc(&L->cell_work, (size_t)G));
        CUDA_TRY(cudaMemsetAsync(L->cseg_start, 0, sizeof(int) * ((size_t)G + 1), s));
        CUDA_TRY(cudaMemsetAsync(L->cell_algo, 0, sizeof(int) * (size_t)G, s));
        CUDA_TRY(cudaMemsetAsync(L->cell_work, 0, sizeof(int) * (size_t)G, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        return SJ_OK;
    }
    LayerBuildArgs a{};
    a.g = L->g;
    a.kind = KIND_P2P;
    a.D = L->D;
    a.nobj = L->nobj;
    a.V = V;
    a.verts = L->verts;
    a.obj_voff = L->obj_voff;
    a.cand_start = L->cand_start;
    struct Tmp {
        void *p[7] = {};
        ~Tmp() {
            for (void *q : p)
                if (q) cudaFree(q);
        }
    } tmp;
    int *seg_off = nullptr;
    int2 *pairs = nullptr;
    unsigned long long *total = nullptr;
    const size_t nbs = bucket_scan_blocks(std::max(G, V));
    CUDA_TRY(dalloc(&a.cell_cnt, (size_t)G + 1)); tmp.p[0] = a.cell_cnt;
    CUDA_TRY(dalloc(&a.cursor, (size_t)G)); tmp.p[1] = a.cursor;
    CUDA_TRY(dalloc(&seg_off, (size_t)V + 1)); tmp.p[2] = seg_off;
    CUDA_TRY(dalloc(&a.block_sums, nbs)); tmp.p[3] = a.block_sums;
    a.bs_cap = nbs;
    CUDA_TRY(dalloc(&a.totals, 4)); tmp.p[4] = a.totals;
    CUDA_TRY(dalloc(&total, 1)); tmp.p[5] = total;
    CUDA_TRY(cudaMemsetAsync(a.cell_cnt, 0, sizeof(int) * ((size_t)G + 1), s));
    CUDA_TRY(cudaMemsetAsync(a.cursor, 0, sizeof(int) * (size_t)G, s));
    CUDA_TRY(cudaMemsetAsync(total, 0, sizeof(unsigned long long), s));
    CUDA_TRY(launch_segcell_count(a, L->seg32, L->seg_e64, seg_off, total, s));
    unsigned long long MS = 0;
    CUDA_TRY(cudaMemcpyAsync(&MS, total, sizeof(MS), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (MS > (unsigned long long)MAX_COUNT) return fail(SJ_ERR_INVALID, "more than 2^31 - 2^22 (cell, segment) pairs");
    L->MS = (int64_t)MS;
    CUDA_TRY(dalloc(&L->cseg_ids, (size_t)MS));
    CUDA_TRY(dalloc(&pairs, (size_t)MS)); tmp.p[6] = pairs;
    CUDA_TRY(launch_segcell_emit(a, L->seg32, L->seg_e64, seg_off, pairs, (int)MS, L->cand_ids, L->cseg_start,
                                 L->cseg_ids, L->cell_algo, s));
    CUDA_TRY(dalloc(&L->cseg_rec, 2 * (size_t)MS));
    CUDA_TRY(launch_cseg_records(L->cseg_start, L->cseg_ids, L->g, L->frames, L->frames + L->g.nx, L->vsplit,
                                 L->seg32, L->cseg_rec, s));
    CUDA_TRY(dalloc(&L->cell_work, (size_t)G));
    CUDA_TRY(launch_cell_work_p2p(L->cseg_start, G, L->cell_work, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return SJ_OK;
}

// PIP boundary entries (after the classes): near edge lists with staging
// records, and the far-right parity flips (see k_pip_boundary).
static sj_status build_boundary_lists(sj_layer *L, double delta, cudaStream_t s) {
    const int M = (int)L->M;
    CUDA_TRY(dalloc(&L->bnear_start, (size_t)M + 1));
    CUDA_TRY(dalloc(&L->bflip_start, (size_t)M + 1));
    CUDA_TRY(dalloc(&L->bflip_len, (size_t)M));
    CUDA_TRY(dalloc(&L->bnear_h, (size_t)M));
    if (M == 0) {
        L->MN = L->MF = 0;
        CUDA_TRY(dalloc(&L->bnear_ids, 0));
        CUDA_TRY(dalloc(&L->bnear_rec, 0));
        CUDA_TRY(dalloc(&L->bnear_key, 0));
        CUDA_TRY(dalloc(&L->cell_work, (size_t)L->g.G));
        CUDA_TRY(cudaMemsetAsync(L->cell_work, 0, sizeof(int) * (size_t)L->g.G, s));
        CUDA_TRY(dalloc(&L->bflip_keys, 0));
        CUDA_TRY(cudaMemsetAsync(L->bnear_start, 0, sizeof(int), s));
        CUDA_TRY(cudaMemsetAsync(L->bflip_start, 0, sizeof(int), s));
        CUDA_TRY(cudaStreamSynchronize(s));
        return SJ_OK;
    }
    struct Tmp {
        void *p[5] = {};
        ~Tmp() {
            for (void *q : p)
                if (q) cudaFree(q);
        }
    } tmp;
    BoundaryArgs a{};
    a.g = L->g;
    a.cand_start = L->cand_start;
    a.cand_ids = L->cand_ids;
    a.cls = L->cand_cls;
    a.prow_base = L->prow_base;
    a.prow_r0 = L->prow_r0;
    a.prow_start = L->prow_start;
    a.pedge_ids = L->pedge_ids;
    a.nxt = L->nxt;
    a.prv = L->prv;
    a.verts = L->verts;
    a.delta = delta;
    int *totals = nullptr;
    int2 *bs = nullptr;
    const size_t cap = bucket_scan_blocks(M);
    CUDA_TRY(dalloc(&a.near_cnt, (size_t)M)); tmp.p[0] = a.near_cnt;
    CUDA_TRY(dalloc(&a.flip_cnt, (size_t)M)); tmp.p[1] = a.flip_cnt;
    CUDA_TRY(dalloc(&totals, 8)); tmp.p[2] = totals;
    CUDA_TRY(dalloc(&bs, cap)); tmp.p[3] = bs;
    CUDA_TRY(launch_pip_boundary(a, 0, s));
    {   // both lists' sizes in 64 bits before their 32-bit offsets
        unsigned long long *sum = nullptr, hs[2] = {0, 0};
        CUDA_TRY(dalloc(&sum, 2)); tmp.p[4] = sum;
        CUDA_TRY(cudaMemsetAsync(sum, 0, 2 * sizeof(unsigned long long), s));
        CUDA_TRY(launch_sum64(a.near_cnt, M, sum, s));
        CUDA_TRY(launch_sum64(a.flip_cnt, M, sum + 1, s));
        CUDA_TRY(cudaMemcpyAsync(hs, sum, sizeof(hs), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        if (hs[0] > (unsigned long long)MAX_COUNT || hs[1] > (unsigned long long)MAX_COUNT)
            return fail(SJ_ERR_INVALID, "boundary lists exceed 2^31 - 2^22 entries");
    }
    CUDA_TRY(launch_offsets(a.near_cnt, M, L->bnear_start, bs, cap, totals, s));
    CUDA_TRY(launch_offsets(a.flip_cnt, M, L->bflip_start, bs, cap, totals + 4, s));
    int tot[8] = {};
    CUDA_TRY(cudaMemcpyAsync(tot, totals, sizeof(tot), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    L->MN = tot[0];
    L->MF = tot[4];
    CUDA_TRY(dalloc(&L->bnear_ids, (size_t)L->MN));
    CUDA_TRY(dalloc(&L->bnear_rec, 2 * (size_t)L->MN));
    CUDA_TRY(dalloc(&L->bnear_key, (size_t)L->MN));
    CUDA_TRY(dalloc(&L->bflip_keys, (size_t)L->MF));
    a.near_start = L->bnear_start;
    a.flip_start = L->bflip_start;
    a.near_ids = L->bnear_ids;
    a.flip_keys = L->bflip_keys;
    CUDA_TRY(launch_pip_boundary(a, 1, s));
    CUDA_TRY(launch_pip_flips(L->bflip_start, M, L->bflip_keys, L->bflip_len, s));
    // near lists ordered by lower y, with their keys and y-extents (the
    // refinement's window search on long lists), then the staging records
    CUDA_TRY(launch_pip_near_sort(L->bnear_start, M, L->bnear_ids, L->nxt, L->vsplit, L->bnear_key, L->bnear_h, s));
    CUDA_TRY(dalloc(&L->cell_work, (size_t)L->g.G));
    CUDA_TRY(launch_cell_work_pip(L->cand_start, L->cand_cls, L->bnear_start, L->g.G, L->cell_work, s));
    if (L->MN > 0) CUDA_TRY(launch_prow_records(L->bnear_ids, (long long)L->MN, L->nxt, L->vsplit, L->bnear_rec, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return SJ_OK;
}

// PIP per-(polygon, row) edge lists (after build_candidates).
static sj_status build_row_lists(sj_layer *L, cudaStream_t s) {
    const int P = L->nobj;
    CUDA_TRY(dalloc(&L->prow_base, (size_t)P + 1));
    CUDA_TRY(dalloc(&L->prow_r0, (size_t)P));
    if (P == 0) {
        L->MR = L->ME = 0;
        CUDA_TRY(dalloc(&L->prow_start, 1));
        CUDA_TRY(dalloc(&L->pedge_ids, 0));
        CUDA_TRY(dalloc(&L->pedge_rec, 0));
        CUDA_TRY(dalloc(&L->cand_cls, 0));
        CUDA_TRY(dalloc(&L->cell_res, (size_t)L->g.G));
        CUDA_TRY(cudaMemsetAsync(L->cell_res, 0xff, sizeof(int) * (size_t)L->g.G, s));   // -1: no candidates
        CUDA_TRY(cudaMemsetAsync(L->prow_base, 0, sizeof(int), s));
        CUDA_TRY(cudaMemsetAsync(L->prow_start, 0, sizeof(int), s));
        CUDA_TRY(cudaStreamSynchronize(s));
        return SJ_OK;
    }
    LayerBuildArgs a{};
    a.g = L->g;
    a.kind = KIND_PIP;
    a.nobj = P;
    a.V = L->V;
    a.verts = L->verts;
    a.obj_voff = L->obj_voff;
    a.mbb = L->mbb;
    struct Tmp {
        void *p[5] = {};
        ~Tmp() {
            for (void *q : p)
                if (q) cudaFree(q);
        }
    } tmp;
    unsigned long long *total = nullptr;
    int *cnt = nullptr, *cursor = nullptr;
    CUDA_TRY(dalloc(&total, 2)); tmp.p[0] = total;
    CUDA_TRY(dalloc(&a.totals, 4)); tmp.p[1] = a.totals;
    CUDA_TRY(cudaMemsetAsync(total, 0, 2 * sizeof(unsigned long long), s));
    {
        const size_t nbs = bucket_scan_blocks(P);
        CUDA_TRY(dalloc(&a.block_sums, nbs)); tmp.p[2] = a.block_sums;
        a.bs_cap = nbs;
    }
    CUDA_TRY(launch_prow_count(a, L->prow_base, L->prow_r0, total, s));
    unsigned long long MR = 0;
    CUDA_TRY(cudaMemcpyAsync(&MR, total, sizeof(MR), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (MR > (unsigned long long)MAX_COUNT) return fail(SJ_ERR_INVALID, "more than 2^31 - 2^22 (polygon, row) slots");
    L->MR = (int64_t)MR;
    CUDA_TRY(dalloc(&cnt, (size_t)MR)); tmp.p[3] = cnt;
    CUDA_TRY(dalloc(&cursor, (size_t)MR)); tmp.p[4] = cursor;
    CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)MR, s));
    CUDA_TRY(cudaMemsetAsync(cursor, 0, sizeof(int) * (size_t)MR, s));
    CUDA_TRY(launch_prow_edge_count(a, L->nxt, L->prow_base, L->prow_r0, cnt, total + 1, s));
    unsigned long long ME = 0;
    CUDA_TRY(cudaMemcpyAsync(&ME, total + 1, sizeof(ME), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (ME > (unsigned long long)MAX_COUNT) return fail(SJ_ERR_INVALID, "more than 2^31 - 2^22 (polygon, row, edge) entries");
    L->ME = (int64_t)ME;
    CUDA_TRY(dalloc(&L->prow_start, (size_t)MR + 1));
    CUDA_TRY(dalloc(&L->pedge_ids, (size_t)ME));
    cudaFree(a.block_sums);
    tmp.p[2] = nullptr;
    {
        const size_t nbs = bucket_scan_blocks((int)MR);
        CUDA_TRY(dalloc(&a.block_sums, nbs)); tmp.p[2] = a.block_sums;
        a.bs_cap = nbs;
    }
    CUDA_TRY(launch_prow_edge_emit(a, L->nxt, L->prow_base, L->prow_r0, cnt, (int)MR, L->prow_start, cursor,
                                   L->pedge_ids, s));
    CUDA_TRY(dalloc(&L->pedge_rec, 2 * (size_t)ME));
    if (ME > 0) CUDA_TRY(launch_prow_records(L->pedge_ids, (long long)ME, L->nxt, L->vsplit, L->pedge_rec, s));
    // cell classes of the candidate entries; delta = 1e-7 of the largest grid
    // coordinate (0.01 m at 1e5 m) is far above FP64 rounding and far below a cell
    CUDA_TRY(dalloc(&L->cand_cls, (size_t)L->M));
    const double delta = 1e-7 * L->xmax + 1e-300;
    if (L->M > 0)
        CUDA_TRY(launch_pip_classify(L->g, L->cand_start, L->cand_ids, L->prow_base, L->prow_r0, L->prow_start,
                                     L->pedge_ids, L->nxt, L->verts, delta, L->cand_cls, s));
    // per cell: the result of its points when every candidate is classified
    CUDA_TRY(dalloc(&L->cell_res, (size_t)L->g.G));
    CUDA_TRY(launch_cell_result(L->cand_start, L->cand_ids, L->cand_cls, L->g.G, L->cell_res, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return build_boundary_lists(L, delta, s);
}

static sj_status layer_common_checks(const double *verts, int64_t V, const sj_grid *g, void *stream,
                                     sj_layer **out, DevInfo **di) {
    if (!out) return fail(SJ_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!grid_ok(g)) return fail(SJ_ERR_INVALID, "invalid grid");
    if (V < 0 || V > MAX_COUNT) return fail(SJ_ERR_INVALID, "vertex count out of range (at most 2^31 - 2^22)");
    if (V > 0 && (!verts || !aligned16(verts))) return fail(SJ_ERR_INVALID, "verts NULL or not 16-byte aligned");
    (void)stream;
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    return device_info(dev, di);
}

extern "C" sj_status sj_pip_layer_create(const double *verts, int64_t V, const int64_t *ring_off, int64_t R,
                                         const int64_t *poly_ring_off, int32_t P, const sj_grid *g, void *stream,
                                         sj_layer **out) {
    DevInfo *di;
    sj_status st = layer_common_checks(verts, V, g, stream, out, &di);
    if (st != SJ_OK) return st;
    if (P < 0 || R < 0 || R > MAX_COUNT) return fail(SJ_ERR_INVALID, "ring or polygon count out of range");
    if (!ring_off || !poly_ring_off) return fail(SJ_ERR_INVALID, "offset array is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    LayerGuard guard{new sj_layer()};
    sj_layer *L = guard.L;
    L->kind = KIND_PIP;
    CUDA_TRY(cudaGetDevice(&L->device));
    L->grid = *g;
    L->g = make_grid(g);
    {
        sj_status ts = layer_tables(L, s);
        if (ts != SJ_OK) return ts;
    }
    L->nobj = P;
    L->V = (int)V;
    L->R = R;
    int *dbad = nullptr;
    CUDA_TRY(dalloc(&dbad, 1));
    struct F { int *p; ~F() { cudaFree(p); } } fbad{dbad};
    CUDA_TRY(cudaMemsetAsync(dbad, 0, sizeof(int), s));
    CUDA_TRY(dalloc(&L->ring_off, (size_t)R + 1));
    CUDA_TRY(dalloc(&L->poly_ring_off, (size_t)P + 1));
    CUDA_TRY(launch_check_offsets(ring_off, R, 3, 0, V, L->ring_off, dbad, s));
    CUDA_TRY(launch_check_offsets(poly_ring_off, P, 1, 0, R, L->poly_ring_off, dbad, s));
    CUDA_TRY(dalloc(&L->verts, (size_t)V));
    if (V > 0) {
        CUDA_TRY(cudaMemcpyAsync(L->verts, verts, sizeof(double2) * (size_t)V, cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(launch_check_finite(L->verts, (int)V, dbad, s));
    }
    int bad = 0;
    st = read_flag(dbad, s, &bad);
    if (st != SJ_OK) return st;
    if (bad) return fail(SJ_ERR_INVALID, "invalid polygon layer (offsets, ring sizes or non-finite vertex)");
    CUDA_TRY(dalloc(&L->obj_voff, (size_t)P + 1));
    CUDA_TRY(dalloc(&L->nxt, (size_t)V));
    CUDA_TRY(dalloc(&L->prv, (size_t)V));
    CUDA_TRY(dalloc(&L->vsplit, (size_t)V));
    CUDA_TRY(launch_pip_topology(L->ring_off, (int)R, L->poly_ring_off, P, L->obj_voff, L->nxt, L->prv, s));
    if (V > 0) CUDA_TRY(launch_split(L->verts, (int)V, L->vsplit, s));
    {   // size of the largest polygon (picks how many items a warp takes at once)
        std::vector<int> voff((size_t)P + 1);
        CUDA_TRY(cudaMemcpyAsync(voff.data(), L->obj_voff, sizeof(int) * ((size_t)P + 1), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        for (int32_t p = 0; p < P; ++p) L->max_obj_verts = std::max<int64_t>(L->max_obj_verts, voff[p + 1] - voff[p]);
    }
    CUDA_TRY(dalloc(&L->stats, ST_N));
    CUDA_TRY(cudaMemsetAsync(L->stats, 0, sizeof(unsigned long long) * ST_N, s));
    st = build_candidates(L, dbad, s);
    if (st != SJ_OK) return st;
    st = build_row_lists(L, s);
    if (st != SJ_OK) return st;
    *out = L;
    guard.L = nullptr;
    return SJ_OK;
}

extern "C" sj_status sj_p2p_layer_create(const double *verts, int64_t V, const int64_t *line_off, int32_t Lc, double D,
                                         const sj_grid *g, void *stream, sj_layer **out) {
    DevInfo *di;
    sj_status st = layer_common_checks(verts, V, g, stream, out, &di);
    if (st != SJ_OK) return st;
    if (Lc < 0) return fail(SJ_ERR_INVALID, "polyline count out of range");
    if (!line_off) return fail(SJ_ERR_INVALID, "line_off is NULL");
    if (!(std::isfinite(D) && D >= 0.0)) return fail(SJ_ERR_INVALID, "D must be finite and >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    LayerGuard guard{new sj_layer()};
    sj_layer *L = guard.L;
    L->kind = KIND_P2P;
    CUDA_TRY(cudaGetDevice(&L->device));
    L->grid = *g;
    L->g = make_grid(g);
    {
        sj_status ts = layer_tables(L, s);
        if (ts != SJ_OK) return ts;
    }
    L->nobj = Lc;
    L->V = (int)V;
    L->R = Lc;
    L->D = D;
    int *dbad = nullptr;
    CUDA_TRY(dalloc(&dbad, 1));
    struct F { int *p; ~F() { cudaFree(p); } } fbad{dbad};
    CUDA_TRY(cudaMemsetAsync(dbad, 0, sizeof(int), s));
    CUDA_TRY(dalloc(&L->obj_voff, (size_t)Lc + 1));
    CUDA_TRY(launch_check_offsets(line_off, Lc, 1, 0, V, L->obj_voff, dbad, s));
    CUDA_TRY(dalloc(&L->verts, (size_t)V));
    if (V > 0) {
        CUDA_TRY(cudaMemcpyAsync(L->verts, verts, sizeof(double2) * (size_t)V, cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(launch_check_finite(L->verts, (int)V, dbad, s));
    }
    int bad = 0;
    st = read_flag(dbad, s, &bad);
    if (st != SJ_OK) return st;
    if (bad) return fail(SJ_ERR_INVALID, "invalid polyline layer (offsets or non-finite vertex)");
    CUDA_TRY(dalloc(&L->vsplit, (size_t)V));
    CUDA_TRY(dalloc(&L->seg_e64, (size_t)V));
    CUDA_TRY(dalloc(&L->seg_inv64, (size_t)V));
    CUDA_TRY(dalloc(&L->seg32, (size_t)V));
    if (V > 0) {
        CUDA_TRY(launch_split(L->verts, (int)V, L->vsplit, s));
        CUDA_TRY(launch_seg_table(L->verts, L->obj_voff, Lc, L->seg_e64, L->seg_inv64, L->seg32, s));
    }
    CUDA_TRY(dalloc(&L->stats, ST_N));
    CUDA_TRY(cudaMemsetAsync(L->stats, 0, sizeof(unsigned long long) * ST_N, s));
    st = build_candidates(L, dbad, s);
    if (st != SJ_OK) return st;
    st = build_seg_lists(L, s);
    if (st != SJ_OK) return st;
    *out = L;
    guard.L = nullptr;
    return SJ_OK;
}

extern "C" sj_status sj_layer_destroy(sj_layer *L) {
    if (!L) return SJ_OK;
    cudaDeviceSynchronize();
    layer_free(L);
    return SJ_OK;
}

extern "C" sj_status sj_layer_get_info(const sj_layer *L, sj_layer_info *out) {
    if (!L || !out) return fail(SJ_ERR_INVALID, "NULL argument");
    out->kind = L->kind;
    out->n_objects = L->nobj;
    out->n_vertices = L->V;
    out->n_rings = L->R;
    out->n_cells = L->g.G;
    out->n_candidates = L->M;
    out->D = L->D;
    return SJ_OK;
}

extern "C" sj_status sj_layer_get_candidates(const sj_layer *L, int32_t *cand_start, int32_t *cand_ids) {
    if (!L || !cand_start || (!cand_ids && L->M > 0)) return fail(SJ_ERR_INVALID, "NULL argument");
    CUDA_TRY(cudaMemcpy(cand_start, L->cand_start, sizeof(int) * ((size_t)L->g.G + 1), cudaMemcpyDeviceToHost));
    if (L->M > 0) CUDA_TRY(cudaMemcpy(cand_ids, L->cand_ids, sizeof(int) * (size_t)L->M, cudaMemcpyDeviceToHost));
    return SJ_OK;
}

extern "C" sj_status sj_layer_get_stats(const sj_layer *L, sj_run_stats *out) {
    if (!L || !out) return fail(SJ_ERR_INVALID, "NULL argument");
    unsigned long long h[ST_N];
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaMemcpy(h, L->stats, sizeof(h), cudaMemcpyDeviceToHost));
    resolve_events(L);
    out->refine_launches = L->refine_launches;
    out->refine_ms = L->refine_ms;
    out->joins = L->joins.load();
    out->points = L->points.load();
    out->items = (int64_t)h[ST_ITEMS];
    out->pairs = (int64_t)h[ST_PAIRS];
    out->edge_tests = (int64_t)h[ST_TESTS];
    out->fallbacks = (int64_t)h[ST_FALLBACK];
    out->hits = (int64_t)h[ST_HITS];
    out->algo_tests = (int64_t)h[ST_ALGO];
    out->resolved = (int64_t)h[ST_RESOLVED];
    out->census_tests = L->census_tests.load();
    out->census_straddles = L->census_straddles.load();
    return SJ_OK;
}

extern "C" sj_status sj_layer_reset_stats(sj_layer *L) {
    if (!L) return fail(SJ_ERR_INVALID, "NULL argument");
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaMemset(L->stats, 0, sizeof(unsigned long long) * ST_N));
    resolve_events(L);
    L->refine_ms = 0.0;
    L->refine_launches = 0;
    L->joins = 0;
    L->points = 0;
    L->census_tests = 0;
    L->census_straddles = 0;
    return SJ_OK;
}

// ------------------------------------------------------------------ joins

struct JoinBufs {
    int *cnt, *cell_start, *perm, *totals, *pos, *res_id, *cell_base, *sub_start;
    int2 *key_rank, *items, *block_sums, *fb;
    double2 *spts;
    ResF *resf;
    ResD *resd;
};

// Result layout of a join: through perm into the outputs (RES_PERM), or
// cell-ordered and gathered back through pos: ids only (RES_IDS, PIP) or packed
// P2P records (RES_F for FP32X, RES_D for FP64).
enum { RES_PERM = 0, RES_IDS, RES_F, RES_D };

// with_spts: also a cell-ordered copy of the points (else the refinement reads
// the input points through perm).
// ch_min: the smallest work item (cell_chunk's floor when items are split by
// edge budget, else ch).
static void carve(Scratch &s, JoinBufs &b, int64_t N, int G, int ch, bool need_fb, bool with_spts = true,
                  int res = RES_PERM, int lS = 0, int ch_min = 0) {
    size_t max_items = (size_t)(N / (ch_min > 0 ? ch_min : ch)) + (size_t)std::min<int64_t>(G, N) + 1;
    b.cnt = s.take<int>(((size_t)G << lS) + 1);
    b.sub_start = lS ? s.take<int>((size_t)G << lS) : nullptr;
    b.cell_start = s.take<int>((size_t)G + 1);
    b.totals = s.take<int>(4);
    b.key_rank = s.take<int2>((size_t)N);
    b.perm = s.take<int>((size_t)N);
    b.spts = with_spts ? s.take<double2>((size_t)N) : nullptr;
    b.items = s.take<int2>(max_items);
    b.block_sums = s.take<int2>(bucket_scan_blocks(G));
    b.fb = need_fb ? s.take<int2>((size_t)N) : nullptr;
    const bool sorted_res = res != RES_PERM;
    b.pos = sorted_res ? s.take<int>((size_t)N) : nullptr;
    b.cell_base = sorted_res ? s.take<int>((size_t)G) : nullptr;
    b.res_id = res == RES_IDS ? s.take<int>((size_t)N) : nullptr;
    b.resf = res == RES_F ? s.take<ResF>((size_t)N) : nullptr;
    b.resd = res == RES_D ? s.take<ResD>((size_t)N) : nullptr;
}

// window < 0: the layer's D; else a P2P window 0 <= window <= D for this call
// alone (the layer's lists, built for D, hold every segment within any smaller
// window, so the same kernels apply with the window's thresholds).
static sj_status join_impl(const sj_layer *L, int kind, const double *pts, int64_t N, int32_t *out_id, double *out_d,
                           const sj_opts *o, void *stream, double window = -1.0) {
    if (!L) return fail(SJ_ERR_INVALID, "layer is NULL");
    if (L->kind != kind) return fail(SJ_ERR_INVALID, kind == KIND_PIP ? "not a polygon layer" : "not a polyline layer");
    if (window >= 0.0 && !(window <= L->D)) return fail(SJ_ERR_INVALID, "window must lie in [0, layer D]");
    if (N < 0 || N > MAX_COUNT) return fail(SJ_ERR_INVALID, "N out of range (at most 2^31 - 2^22)");
    if (N > 0 && (!pts || !out_id)) return fail(SJ_ERR_INVALID, "NULL buffer");
    if (N > 0 && !aligned16(pts)) return fail(SJ_ERR_INVALID, "pts not 16-byte aligned");
    int form = o ? o->form : SJ_FP64;
    if (form != SJ_FP64 && form != SJ_FP32X) return fail(SJ_ERR_INVALID, "unknown form");
    int launch = o ? o->launch : SJ_PER_REQUEST;
    if (launch != SJ_PER_REQUEST && launch != SJ_PERSISTENT) return fail(SJ_ERR_INVALID, "unknown launch form");
    if (form == SJ_FP32X && L->xmax > 1e30)
        return fail(SJ_ERR_INVALID, "SJ_FP32X needs grid coordinates below 1e30 in magnitude; use SJ_FP64");
    int ch = (o && o->pts_per_item) ? o->pts_per_item : 128;
    if (ch < 1 || ch > MAX_CH) return fail(SJ_ERR_INVALID, "pts_per_item must be in 1..128");
    const int nw = (o && o->block) ? o->block : 4;
    if (nw != 2 && nw != 4 && nw != 8) return fail(SJ_ERR_INVALID, "block must be 0, 2, 4 or 8 (warps per block)");
    int budget = o ? o->edges_per_chunk : 0;
    if (budget < 0) return fail(SJ_ERR_INVALID, "edges_per_chunk must be >= 0");
    // default: polygon layers split heavy cells at 64 edges per point (the
    // autotuner's best on both tilings at 100 M points: heavy-tail layer
    // 8.1 -> 6.5 ms, 40,000 tiles 5.2 -> 4.8 ms); polyline layers do not (no
    // setting was faster on the walks)
    if (budget == 0 && kind == KIND_PIP) budget = 64;
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev != L->device) return fail(SJ_ERR_INVALID, "layer belongs to another device");
    DevInfo *di;
    sj_status st = device_info(dev, &di);
    if (st != SJ_OK) return st;
    L->joins++;
    L->points += N;
    if (N == 0) return SJ_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int G = L->g.G;
    const bool need_fb = (kind == KIND_P2P && form == SJ_FP32X);
    // Sub-cell order of the points inside their cells (see BucketArgs), on
    // request (SJ_FLAG_SUBCELL_ON): each work item of a dense cell then covers
    // a compact part of it and the exact per-item prunes (the P2P box
    // distance, the PIP y-range) drop more of the staged segments / edges --
    // 40 % fewer P2P tests at 170 M points, 47 % fewer PIP tests on the
    // heavy-tail tiling -- but the per-sub-cell start table (G x S entries,
    // read at random by the scatter) costs more than that saves on the
    // workloads measured, so arrival order is the default.  P2P: 4 x 4
    // sub-cells in Z-order; PIP: 8 horizontal bands (its prune is in y).
    int sub_lx = 0, sub_ly = 0;
    {
        const int fl = o ? o->flags : 0;
        const bool on = (fl & SJ_FLAG_SUBCELL_ON) && !(fl & SJ_FLAG_SUBCELL_OFF);
        if (on) {
            if (kind == KIND_P2P) sub_lx = sub_ly = 2;
            else sub_ly = 3;
        }
        if (((long long)G << (sub_lx + sub_ly)) > MAX_COUNT) sub_lx = sub_ly = 0;
    }
    const int lS = sub_lx + sub_ly;

    JoinBufs b;
    const int res = kind == KIND_PIP ? RES_IDS : (form == SJ_FP32X ? RES_F : RES_D);
    const bool split = budget > 0 && L->cell_work;   // items sized by the cells' edge work
    const int ch_min = split ? std::min(ch, 8) : ch;
    size_t bytes = measure([&](Scratch &sc) { carve(sc, b, N, G, ch, need_fb, false, res, lS, ch_min); });
    Scratch sc;
    CUDA_TRY(dev_malloc_async((void **)&sc.base, bytes, s));
    carve(sc, b, N, G, ch, need_fb, false, res, lS, ch_min);
    cudaError_t e = cudaMemsetAsync(b.cnt, 0, sizeof(int) * (((size_t)G << lS) + 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.totals, 0, sizeof(int) * 4, s);

    BucketArgs ba{};
    ba.g = L->g;
    ba.pts = (const double2 *)pts;
    ba.n = (int)N;
    ba.cnt = b.cnt;
    ba.key_rank = b.key_rank;
    ba.cell_start = b.cell_start;
    ba.perm = b.perm;
    ba.spts = b.spts;
    ba.cand_start = L->cand_start;
    ba.ch = ch;
    ba.cell_work = split ? L->cell_work : nullptr;
    ba.budget = split ? budget : 0;
    ba.items = b.items;
    ba.block_sums = b.block_sums;
    ba.bs_cap = bucket_scan_blocks(G);
    ba.totals = b.totals;
    ba.pos = b.pos;
    ba.cell_base = b.cell_base;
    ba.sub_lx = sub_lx;
    ba.sub_ly = sub_ly;
    ba.sub_start = b.sub_start;
    if (kind == KIND_PIP) {   // points of fully classified cells: results written by the cell-id pass
        ba.cell_res = L->cell_res;
        ba.out_id = out_id;
        ba.stats = L->stats;
    }
    if (e == cudaSuccess) e = launch_bucket(ba, s);

    RefineArgs ra{};
    fill_refine(L, ra);
    if (window >= 0.0) {
        ra.D = window;
        ra.Df = (float)window;
        ra.Ddn = float_down(window * (1.0 - 1e-12));
        ra.Dup = float_up(window * (1.0 + 1e-12) + 1e-300);
    }
    ra.items = b.items;
    ra.n_items = b.totals + 1;
    ra.work_next = b.totals + 3;   // zeroed with the totals at the start of the join
    // Items a warp takes per counter update.  P2P on dense grids (two or more
    // items per cell on average): two consecutive items, mostly two chunks of
    // one cell, whose second reads the cell's records from L1 and halves the
    // counter traffic (170 M points, 512^2 grid, D = 50 m: refine 5.35 ->
    // 4.21 ms; D = 100 m unchanged); sparse grids keep one (the 10 M point
    // join is 1 % slower with two).  PIP: two when every polygon is small
    // (1 M points on the stars: refine 0.072 -> 0.067 ms); one when some
    // polygon is large, whose boundary items would pair into stragglers
    // (heavy-tail tiling: 5.3 -> 6.9 ms with two).
    if (kind == KIND_P2P) ra.claim = (N >= 2LL * ch * (long long)G) ? 2 : 1;
    else ra.claim = L->max_obj_verts <= 256 ? 2 : 1;
    ra.cell_start = b.cell_start;
    ra.perm = b.perm;
    ra.spts = b.spts;
    ra.pts = (const double2 *)pts;
    ra.ch = ch;
    ra.npts = (int)N;
    ra.cell_work = ba.cell_work;
    ra.budget = ba.budget;
    ra.res_id = b.res_id;   // cell-ordered results, every slot of a refined cell written
    ra.resf = b.resf;
    ra.resd = b.resd;
    ra.out_id = out_id;     // FP32X recheck: final outputs through perm
    ra.out_d = out_d;
    ra.fb = b.fb;
    ra.n_fb = b.totals + 2;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    const bool timed = o && (o->flags & SJ_FLAG_TIME_REFINE);
    if (e == cudaSuccess && timed) {
        e = cudaEventCreate(&ev0);
        if (e == cudaSuccess) e = cudaEventCreate(&ev1);
        if (e == cudaSuccess) e = cudaEventRecord(ev0, s);
    }
    if (e == cudaSuccess) {
        if (kind == KIND_PIP) e = launch_pip_refine(ra, form, nw, di->sms * di->pip_bps[form], s);
        else e = launch_p2p_refine(ra, form, nw, di->sms * di->p2p_bps[form], s);
    }
    if (timed && ev1) {   // the refinement launch alone
        if (e == cudaSuccess) e = cudaEventRecord(ev1, s);
        std::lock_guard<std::mutex> lk(L->ev_mu);
        L->ev_pending.emplace_back(ev0, ev1);
    }
    // a8: results to input order; then the FP32X recheck overwrites the points
    // it redoes in FP64, through perm
    if (e == cudaSuccess) {
        if (res == RES_IDS) e = launch_unsort(b.pos, b.res_id, nullptr, (int)N, out_id, nullptr, s);
        else if (res == RES_F) e = launch_unsort_f(b.pos, b.resf, (int)N, out_id, out_d, s);
        else e = launch_unsort_d(b.pos, b.resd, (int)N, out_id, out_d, s);
    }
    if (e == cudaSuccess && need_fb) e = launch_p2p_recheck(ra, di->sms * 4, s);
    cudaError_t e2 = cudaFreeAsync(sc.base, s);
    if (e != cudaSuccess) return cuda_fail(e, "join launch");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
    return check_bounds(s);
}

extern "C" sj_status sj_pip_join(const sj_layer *L, const double *pts, int64_t N, int32_t *out_id, const sj_opts *o,
                                 void *stream) {
    return join_impl(L, KIND_PIP, pts, N, out_id, nullptr, o, stream);
}

extern "C" sj_status sj_p2p_join(const sj_layer *L, const double *pts, int64_t N, int32_t *out_id, double *out_d,
                                 const sj_opts *o, void *stream) {
    return join_impl(L, KIND_P2P, pts, N, out_id, out_d, o, stream);
}

extern "C" sj_status sj_p2p_join_window(const sj_layer *L, const double *pts, int64_t N, double window,
                                        int32_t *out_id, double *out_d, const sj_opts *o, void *stream) {
    if (!(window >= 0.0)) return fail(SJ_ERR_INVALID, "window must lie in [0, layer D]");   // NaN too
    return join_impl(L, KIND_P2P, pts, N, out_id, out_d, o, stream, window);
}

// Host-buffer join, pipelined in three stages on library streams: chunks of
// the points are copied in on one stream, joined on a second (each waiting for
// its chunk's copy) and their results copied out on a third (each waiting for
// its chunk's join), so that copies in, joins and copies out of different
// chunks overlap (both copy directions and the SMs work at once).  Each chunk
// is an independent join (a point's result does not depend on the other
// points), so the outputs equal those of one join over all N points.  At most
// three chunks: every chunk is a full join with fixed costs (scans over every
// cell, sparser work items), so four quarter joins were measured slower.
static sj_status join_host(const sj_layer *L, int kind, const double *pts, int64_t N, int32_t *out_id, double *out_d,
                           const sj_opts *o, void *stream, double window = -1.0) {
    if (N < 0 || N > MAX_COUNT) return fail(SJ_ERR_INVALID, "N out of range (at most 2^31 - 2^22)");
    if (N > 0 && (!pts || !out_id)) return fail(SJ_ERR_INVALID, "NULL buffer");
    if (!L) return fail(SJ_ERR_INVALID, "layer is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (N == 0) return join_impl(L, kind, nullptr, 0, nullptr, nullptr, o, stream, window);
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    DevInfo *di;
    sj_status st = device_info(dev, &di);
    if (st != SJ_OK) return st;
    cudaStream_t t_in = di->hstream[0], t_cmp = di->hstream[1], t_out = di->hstream[2];
    // chunk bounds: one chunk up to 2 M points, halves up to 8 M, else quarter /
    // half / quarter (a short first chunk starts the joins early, a short last
    // one keeps the final copy out short)
    int64_t bound[4] = {0, N, N, N};
    int nchunks = 1;
    if (N > (int64_t)8 << 20) {
        bound[1] = N / 4;
        bound[2] = N - N / 4;
        nchunks = 3;
    } else if (N > (int64_t)2 << 20) {
        bound[1] = N / 2;
        nchunks = 2;
    }
    char *d = nullptr;
    size_t bp = (size_t)N * 16, bi = ((size_t)N * 4 + 255) & ~(size_t)255, bd = out_d ? (size_t)N * 8 : 0;
    CUDA_TRY(dev_malloc_async((void **)&d, bp + bi + bd, s));
    double *dp = (double *)d;
    int32_t *dI = (int32_t *)(d + bp);
    double *dD = out_d ? (double *)(d + bp + bi) : nullptr;
    std::vector<cudaEvent_t> evs(2 * (size_t)nchunks + 3, nullptr);
    cudaError_t e = cudaSuccess;
    for (auto &ev : evs)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaEvent_t ev_start = evs[0], ev_done = evs[1];
    // every stage starts after the caller's stream (its prior work and the allocation)
    if (e == cudaSuccess) e = cudaEventRecord(ev_start, s);
    for (cudaStream_t t : {t_in, t_cmp, t_out})
        if (e == cudaSuccess) e = cudaStreamWaitEvent(t, ev_start, 0);
    for (int c = 0; c < nchunks && e == cudaSuccess && st == SJ_OK; ++c) {
        cudaEvent_t copied = evs[2 + 2 * c], joined = evs[3 + 2 * c];
        const int64_t off = bound[c], n = bound[c + 1] - off;
        e = cudaMemcpyAsync(dp + 2 * off, pts + 2 * off, (size_t)n * 16, cudaMemcpyHostToDevice, t_in);
        if (e == cudaSuccess) e = cudaEventRecord(copied, t_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(t_cmp, copied, 0);
        if (e != cudaSuccess) break;
        st = join_impl(L, kind, dp + 2 * off, n, dI + off, dD ? dD + off : nullptr, o, t_cmp, window);
        if (st != SJ_OK) break;
        e = cudaEventRecord(joined, t_cmp);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(t_out, joined, 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out_id + off, dI + off, (size_t)n * 4, cudaMemcpyDeviceToHost, t_out);
        if (e == cudaSuccess && out_d)
            e = cudaMemcpyAsync(out_d + off, dD + off, (size_t)n * 8, cudaMemcpyDeviceToHost, t_out);
    }
    // the caller's stream waits for the join and copy-out stages (the copy-in
    // stage is behind both), then frees the buffer
    cudaError_t e2 = cudaEventRecord(ev_done, t_out);
    if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, ev_done, 0);
    if (e2 == cudaSuccess) e2 = cudaEventRecord(evs.back(), t_cmp);
    if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, evs.back(), 0);
    cudaFreeAsync(d, s);
    cudaError_t e3 = cudaStreamSynchronize(s);
    for (cudaEvent_t ev : evs)
        if (ev) cudaEventDestroy(ev);
    if (st != SJ_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "host join copy");
    if (e2 != cudaSuccess) return cuda_fail(e2, "host join streams");
    if (e3 != cudaSuccess) return cuda_fail(e3, "cudaStreamSynchronize");
    return SJ_OK;
}

extern "C" sj_status sj_pip_join_host(const sj_layer *L, const double *pts, int64_t N, int32_t *out_id,
                                      const sj_opts *o, void *stream) {
    return join_host(L, KIND_PIP, pts, N, out_id, nullptr, o, stream);
}

extern "C" sj_status sj_p2p_join_host(const sj_layer *L, const double *pts, int64_t N, int32_t *out_id, double *out_d,
                                      const sj_opts *o, void *stream) {
    return join_host(L, KIND_P2P, pts, N, out_id, out_d, o, stream);
}

extern "C" sj_status sj_p2p_join_window_host(const sj_layer *L, const double *pts, int64_t N, double window,
                                             int32_t *out_id, double *out_d, const sj_opts *o, void *stream) {
    if (!(window >= 0.0)) return fail(SJ_ERR_INVALID, "window must lie in [0, layer D]");   // NaN too
    if (L && L->kind == KIND_P2P && !(window <= L->D)) return fail(SJ_ERR_INVALID, "window must lie in [0, layer D]");
    return join_host(L, KIND_P2P, pts, N, out_id, out_d, o, stream, window);
}

extern "C" sj_status sj_bucket_points(const double *pts, int64_t N, const sj_grid *g, int32_t *cell_start, int32_t *perm,
                                      void *stream) {
    if (!grid_ok(g)) return fail(SJ_ERR_INVALID, "invalid grid");
    if (N < 0 || N > MAX_COUNT) return fail(SJ_ERR_INVALID, "N out of range (at most 2^31 - 2^22)");
    if (!cell_start || (N > 0 && (!pts || !perm))) return fail(SJ_ERR_INVALID, "NULL buffer");
    if (N > 0 && !aligned16(pts)) return fail(SJ_ERR_INVALID, "pts not 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    GridDev gd = make_grid(g);
    Scratch sc;
    auto lay = [&](Scratch &x, int **cnt, int **totals, int2 **kr, int2 **bs, unsigned long long **keys) {
        *cnt = x.take<int>((size_t)gd.G + 1);
        *totals = x.take<int>(4);
        *kr = x.take<int2>((size_t)N);
        *bs = x.take<int2>(bucket_scan_blocks(gd.G));
        *keys = x.take<unsigned long long>((size_t)gd.nx + gd.ny + 2);
    };
    int *cnt, *totals;
    int2 *kr, *bs;
    unsigned long long *keys;
    size_t bytes = measure([&](Scratch &x) { lay(x, &cnt, &totals, &kr, &bs, &keys); });
    CUDA_TRY(dev_malloc_async((void **)&sc.base, bytes, s));
    lay(sc, &cnt, &totals, &kr, &bs, &keys);
    gd.kx = keys;
    gd.ky = keys + gd.nx + 1;
    BucketArgs ba{};
    ba.g = gd;
    ba.pts = (const double2 *)pts;
    ba.n = (int)N;
    ba.cnt = cnt;
    ba.key_rank = kr;
    ba.cell_start = cell_start;
    ba.perm = perm;
    ba.block_sums = bs;
    ba.bs_cap = bucket_scan_blocks(gd.G);
    ba.totals = totals;
    ba.ch = 1;
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * ((size_t)gd.G + 1), s);
    if (e == cudaSuccess) e = launch_thresholds(gd, keys, keys + gd.nx + 1, s);
    if (e == cudaSuccess) e = launch_bucket(ba, s);
    cudaError_t e2 = cudaFreeAsync(sc.base, s);
    if (e != cudaSuccess) return cuda_fail(e, "bucket launch");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
    return SJ_OK;
}

extern "C" sj_status sj_pip_census(const sj_layer *L, const double *pts, int64_t N, int64_t *out, void *stream) {
    if (!L || !out) return fail(SJ_ERR_INVALID, "NULL argument");
    if (L->kind != KIND_PIP) return fail(SJ_ERR_INVALID, "not a polygon layer");
    if (N < 0 || N > MAX_COUNT) return fail(SJ_ERR_INVALID, "N out of range (at most 2^31 - 2^22)");
    if (N > 0 && (!pts || !aligned16(pts))) return fail(SJ_ERR_INVALID, "pts NULL or not 16-byte aligned");
    out[0] = out[1] = 0;
    if (N == 0) return SJ_OK;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *d = nullptr, h[2] = {0, 0};
    CUDA_TRY(dev_malloc_async((void **)&d, sizeof(h), s));
    RefineArgs ra{};
    fill_refine(L, ra);
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(h), s);
    if (e == cudaSuccess) e = launch_pip_census(ra, (const double2 *)pts, (int)N, d, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "census");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
    out[0] = (int64_t)h[0];
    out[1] = (int64_t)h[1];
    L->census_tests += out[0];
    L->census_straddles += out[1];
    return SJ_OK;
}

extern "C" const char *sj_last_error(void) { return g_err.c_str(); }

extern "C" const char *sj_version(void) { return "sj 0.1 (sm_103a)"; }

// ------------------------------------------------------------------ P2P join without allocation
//
// Some callers cannot allocate device memory at the moment they join: code on
// a hard latency budget (a device allocation can stall for milliseconds),
// code that runs inside a pre-sized memory arena or a fixed memory budget, and
// hosts where another component owns the CUDA allocator and forbids
// allocations from libraries.  sj_p2p_join_noalloc runs the same kernels as
// sj_p2p_join but takes all of its scratch from one file-scope device array
// of fixed size, so it calls no allocator at all.
//
// The array is part of this module's device image: every GPU that loads the
// module holds it until the process exits.  All calls share it, so two calls
// whose kernels overlap on the GPU race on it; callers must serialise them
// (one stream, or events between streams).  It keeps the previous call's
// contents, so the counters that must start at zero are cleared on the
// caller's stream at the start of every call.

namespace {

constexpr int64_t NOALLOC_MAX_POINTS = SJ_NOALLOC_MAX_POINTS;
constexpr int64_t NOALLOC_MAX_CELLS = SJ_NOALLOC_MAX_CELLS;
constexpr int NOALLOC_CH = 64;
constexpr size_t NOALLOC_BYTES = 32u << 20;   // holds carve() at the two limits above (about 31.6 MB)

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

void *g_noalloc_ptr[64];
std::mutex g_noalloc_mu;

// Device address of the array on the current device, looked up once per
// device (host code cannot use the symbol itself: on the host it names a
// stand-in, not device memory).
sj_status noalloc_scratch(int dev, char **out) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
        g_noalloc_ptr[dev] = p;
    }
    *out = (char *)g_noalloc_ptr[dev];
    return SJ_OK;
}

}  // namespace

extern "C" sj_status sj_p2p_join_noalloc(const sj_layer *L, const double *pts, int64_t N, int32_t *out_id,
                                         double *out_d, const sj_opts *o, void *stream) {
    if (!L) return fail(SJ_ERR_INVALID, "layer is NULL");
    if (L->kind != KIND_P2P) return fail(SJ_ERR_INVALID, "not a polyline layer");
    if (N < 0 || N > NOALLOC_MAX_POINTS)
        return fail(SJ_ERR_INVALID, "sj_p2p_join_noalloc: N must be in 0.." + std::to_string(NOALLOC_MAX_POINTS) +
                                        " (fixed scratch size); use sj_p2p_join for larger batches");
    if ((int64_t)L->g.G > NOALLOC_MAX_CELLS)
        return fail(SJ_ERR_INVALID, "sj_p2p_join_noalloc: the layer's grid has more than " +
                                        std::to_string(NOALLOC_MAX_CELLS) + " cells (fixed scratch size)");
    if (N > 0 && (!pts || !out_id)) return fail(SJ_ERR_INVALID, "NULL buffer");
    if (N > 0 && !aligned16(pts)) return fail(SJ_ERR_INVALID, "pts not 16-byte aligned");
    const int form = o ? o->form : SJ_FP64;
    if (form != SJ_FP64 && form != SJ_FP32X) return fail(SJ_ERR_INVALID, "unknown form");
    if (form == SJ_FP32X && L->xmax > 1e30)
        return fail(SJ_ERR_INVALID, "SJ_FP32X needs grid coordinates below 1e30 in magnitude; use SJ_FP64");
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev != L->device) return fail(SJ_ERR_INVALID, "layer belongs to another device");
    if (dev < 0 || dev >= 64) return fail(SJ_ERR_INVALID, "device index out of range");
    DevInfo *di;
    sj_status st = device_info(dev, &di);
    if (st != SJ_OK) return st;
    char *base = nullptr;
    st = noalloc_scratch(dev, &base);
    if (st != SJ_OK) return st;
    L->joins++;
    L->points += N;
    if (N == 0) return SJ_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int G = L->g.G;
    const bool need_fb = form == SJ_FP32X;
    JoinBufs b;
    size_t bytes = measure([&](Scratch &sc) { carve(sc, b, N, G, NOALLOC_CH, need_fb); });
    if (bytes > NOALLOC_BYTES) return fail(SJ_ERR_INVALID, "sj_p2p_join_noalloc: scratch does not fit");
    Scratch sc;
    sc.base = base;
    carve(sc, b, N, G, NOALLOC_CH, need_fb);
    CUDA_TRY(cudaMemsetAsync(b.cnt, 0, sizeof(int) * ((size_t)G + 1), s));
    CUDA_TRY(cudaMemsetAsync(b.totals, 0, sizeof(int) * 4, s));

    BucketArgs ba{};
    ba.g = L->g;
    ba.pts = (const double2 *)pts;
    ba.n = (int)N;
    ba.cnt = b.cnt;
    ba.key_rank = b.key_rank;
    ba.cell_start = b.cell_start;
    ba.perm = b.perm;
    ba.spts = b.spts;
    ba.cand_start = L->cand_start;
    ba.ch = NOALLOC_CH;
    ba.items = b.items;
    ba.block_sums = b.block_sums;
    ba.bs_cap = bucket_scan_blocks(G);
    ba.totals = b.totals;
    ba.out_id = out_id;
    ba.out_d = out_d;
    CUDA_TRY(launch_bucket(ba, s));

    RefineArgs ra{};
    fill_refine(L, ra);
    ra.items = b.items;
    ra.n_items = b.totals + 1;
    ra.cell_start = b.cell_start;
    ra.perm = b.perm;
    ra.spts = b.spts;
    ra.ch = NOALLOC_CH;
    ra.npts = (int)N;
    ra.out_id = out_id;
    ra.out_d = out_d;
    ra.fb = b.fb;
    ra.n_fb = b.totals + 2;
    // items from the device counter, as in join_impl (totals[3], zeroed above)
    ra.work_next = b.totals + 3;
    ra.claim = (N >= 2LL * NOALLOC_CH * (long long)G) ? 2 : 1;
    CUDA_TRY(launch_p2p_refine(ra, form, 4, di->sms * di->p2p_bps[form], s));
    if (need_fb) CUDA_TRY(launch_p2p_recheck(ra, di->sms * 4, s));
    return check_bounds(s);
}
