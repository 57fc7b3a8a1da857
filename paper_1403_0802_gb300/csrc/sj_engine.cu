// sj_engine.cu -- batched rounds for continuous batching (sj_engine_*).
//
// A round joins many requests at once.  Requests against the same layer are
// treated as one point set: one cell-id pass over all of them (a request
// table maps the global point index to its request), one scan over the grid,
// one scatter, ONE refinement launch over the merged work items (results in
// cell order), and one coalesced pass that writes every request's outputs.
// The results are those of joining each request alone: a point's result
// depends only on the point and the layer.
//
// All sizes a round needs are read from device memory (the request table and
// the counters the scan writes) and every grid is sized for the engine's
// maximum, so the per-layer kernel sequence has a fixed shape: it is captured
// once into a CUDA graph and replayed every round after the request table is
// copied in.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "sj_host.hpp"

namespace sj {
cudaError_t launch_pip_refine(const RefineArgs &a, int form, int warps_per_block, int blocks, cudaStream_t s);
cudaError_t launch_p2p_refine(const RefineArgs &a, int form, int warps_per_block, int blocks, cudaStream_t s);
cudaError_t launch_p2p_recheck(const RefineArgs &a, int blocks, cudaStream_t s);
size_t bucket_scan_blocks(int G);

namespace {

// One request as the kernels see it.
struct ReqDev {
    const double2 *pts;
    int *out_id;
    double *out_d;
    double window;   // P2P window of this request (the layer's D when none is asked)
    int off;         // first global point index
    int n;
};

struct MultiArgs {
    GridDev g;
    const ReqDev *reqs;
    const int *meta;       // [0] number of requests, [1] total points, [2] per-request windows on
    int *cnt;
    int2 *key_rank;
    int *pos;
    const int *cell_start;
    int *perm;
    double2 *spts;
    int *res_id;           // cell-ordered results (refinement writes the points of work items)
    double *res_d;
    double *win;           // P2P: per-slot window, written when meta[2] != 0
};

// Request owning global point i: the last request whose offset is <= i.
__device__ __forceinline__ int find_req(const ReqDev *r, int nr, int i) {
    int lo = 0, hi = nr;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (r[mid].off <= i) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void k_cell_hist_multi(MultiArgs m) {
    const int nr = m.meta[0], total = m.meta[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const ReqDev &R = m.reqs[find_req(m.reqs, nr, i)];
        const double2 p = R.pts[i - R.off];
        const int c = point_cell(m.g, p.x, p.y);
        int r = 0;
        if (c < m.g.G) r = atomicAdd(&m.cnt[c], 1);
        m.key_rank[i] = make_int2(c, r);
    }
}

// Also initialises every in-grid slot's result to (-1, +inf): points of cells
// without candidates belong to no work item and keep that result.
__global__ void k_scatter_multi(MultiArgs m) {
    const int nr = m.meta[0], total = m.meta[1];
    const bool pw = m.win && m.meta[2];
    const double INF = __longlong_as_double(0x7ff0000000000000LL);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int2 k = m.key_rank[i];
        int q = -1;
        if (k.x < m.g.G) {
            const ReqDev &R = m.reqs[find_req(m.reqs, nr, i)];
            q = m.cell_start[k.x] + k.y;
            m.perm[q] = i;
            m.spts[q] = R.pts[i - R.off];
            m.res_id[q] = -1;
            if (m.res_d) m.res_d[q] = INF;
            if (pw) m.win[q] = R.window;
        }
        m.pos[i] = q;
    }
}

// Every request's outputs in input order: a gather from the cell-ordered
// results, coalesced writes.
__global__ void k_unsort_multi(MultiArgs m) {
    const int nr = m.meta[0], total = m.meta[1];
    const double INF = __longlong_as_double(0x7ff0000000000000LL);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const ReqDev &R = m.reqs[find_req(m.reqs, nr, i)];
        const int q = m.pos[i];
        R.out_id[i - R.off] = q >= 0 ? m.res_id[q] : -1;
        if (R.out_d) R.out_d[i - R.off] = (q >= 0 && m.res_d) ? m.res_d[q] : INF;
    }
}

// Per-layer workspace, request-table staging and the captured round graph.
struct LayerWork {
    const sj_layer *L = nullptr;
    char *base = nullptr;
    ReqDev *d_reqs = nullptr;
    int *d_meta = nullptr;
    BucketArgs ba{};
    RefineArgs ra{};
    MultiArgs ma{};
    // pinned request tables (two, so the host can fill one while the other's
    // copy may still be pending) and the events that mark their copies done
    ReqDev *h_reqs[2] = {nullptr, nullptr};
    int *h_meta[2] = {nullptr, nullptr};
    cudaEvent_t copied[2] = {nullptr, nullptr};
    int slot = 0;
    cudaGraphExec_t exec = nullptr;
};

}  // namespace
}  // namespace sj

using namespace sj;

struct sj_engine {
    int device = 0;
    int64_t max_points = 0;
    int max_requests = 0;
    int form = SJ_FP64;
    int ch = 64;
    bool use_graph = true;
    std::vector<LayerWork *> work;
    std::mutex mu;
};

static void work_free(LayerWork *w) {
    if (!w) return;
    if (w->exec) cudaGraphExecDestroy(w->exec);
    for (int k = 0; k < 2; ++k) {
        if (w->copied[k]) cudaEventDestroy(w->copied[k]);
        if (w->h_reqs[k]) cudaFreeHost(w->h_reqs[k]);
        if (w->h_meta[k]) cudaFreeHost(w->h_meta[k]);
    }
    if (w->base) cudaFree(w->base);
    delete w;
}

// Workspace of one layer, carved like the per-request join's scratch.
static sj_status work_create(sj_engine *E, const sj_layer *L, LayerWork **out) {
    LayerWork *w = new LayerWork();
    struct Guard {
        LayerWork *w;
        ~Guard() { work_free(w); }
    } guard{w};
    w->L = L;
    const int64_t N = E->max_points;
    const int G = L->g.G;
    const bool p2p = L->kind == KIND_P2P;
    int *cnt, *cell_start, *totals, *pos, *perm, *res_id;
    int2 *key_rank, *items, *block_sums, *fb;
    double2 *spts;
    double *res_d, *win;
    auto lay = [&](Scratch &x) {
        cnt = x.take<int>((size_t)G + 1);
        cell_start = x.take<int>((size_t)G + 1);
        totals = x.take<int>(4);
        key_rank = x.take<int2>((size_t)N);
        pos = x.take<int>((size_t)N);
        perm = x.take<int>((size_t)N);
        spts = x.take<double2>((size_t)N);
        items = x.take<int2>((size_t)(N / E->ch) + (size_t)std::min<int64_t>(G, N) + 1);
        block_sums = x.take<int2>(bucket_scan_blocks(G));
        res_id = x.take<int>((size_t)N);
        res_d = p2p ? x.take<double>((size_t)N) : nullptr;
        win = p2p ? x.take<double>((size_t)N) : nullptr;
        fb = (p2p && E->form == SJ_FP32X) ? x.take<int2>((size_t)N) : nullptr;
        w->d_reqs = x.take<ReqDev>((size_t)E->max_requests);
        w->d_meta = x.take<int>(4);
    };
    size_t bytes = measure(lay);
    CUDA_TRY(dev_malloc((void **)&w->base, bytes));
    Scratch sc;
    sc.base = w->base;
    lay(sc);
    for (int k = 0; k < 2; ++k) {
        CUDA_TRY(cudaMallocHost((void **)&w->h_reqs[k], sizeof(ReqDev) * (size_t)E->max_requests));
        CUDA_TRY(cudaMallocHost((void **)&w->h_meta[k], sizeof(int) * 4));
        CUDA_TRY(cudaEventCreateWithFlags(&w->copied[k], cudaEventDisableTiming));
    }

    BucketArgs &ba = w->ba;
    ba.g = L->g;
    ba.cnt = cnt;
    ba.cell_start = cell_start;
    ba.cand_start = L->cand_start;
    ba.ch = E->ch;
    ba.items = items;
    ba.block_sums = block_sums;
    ba.bs_cap = bucket_scan_blocks(G);
    ba.totals = totals;

    RefineArgs &ra = w->ra;
    fill_refine(L, ra);
    ra.items = items;
    ra.n_items = totals + 1;
    ra.work_next = totals + 3;     // zeroed with the totals at the start of each round
    ra.cell_start = cell_start;
    ra.perm = perm;
    ra.spts = spts;
    ra.ch = E->ch;
    ra.npts = (int)E->max_points;   // slots and point indices of a round stay below it
    ra.res_id = res_id;
    ra.res_d = res_d;
    ra.fb = fb;
    ra.n_fb = totals + 2;
    ra.win = win;
    ra.win_on = p2p ? w->d_meta + 2 : nullptr;

    MultiArgs &ma = w->ma;
    ma.g = L->g;
    ma.reqs = w->d_reqs;
    ma.meta = w->d_meta;
    ma.cnt = cnt;
    ma.key_rank = key_rank;
    ma.pos = pos;
    ma.cell_start = cell_start;
    ma.perm = perm;
    ma.spts = spts;
    ma.res_id = res_id;
    ma.res_d = res_d;
    ma.win = win;
    guard.w = nullptr;
    *out = w;
    return SJ_OK;
}

// The round's kernel sequence for one layer (fixed shape).
static cudaError_t enqueue_round(const sj_engine *E, const LayerWork *w, const DevInfo *di, cudaStream_t s) {
    const sj_layer *L = w->L;
    const int blocks = di->sms * 8;
    cudaError_t e = cudaMemsetAsync(w->ba.cnt, 0, sizeof(int) * ((size_t)L->g.G + 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w->ba.totals, 0, sizeof(int) * 4, s);
    if (e != cudaSuccess) return e;
    k_cell_hist_multi<<<blocks, 256, 0, s>>>(w->ma);
    if ((e = launch_bucket_scan(w->ba, s)) != cudaSuccess) return e;
    k_scatter_multi<<<blocks, 256, 0, s>>>(w->ma);
    if (L->kind == KIND_PIP) {
        e = launch_pip_refine(w->ra, E->form, 4, di->sms * di->pip_bps[E->form], s);
    } else {
        e = launch_p2p_refine(w->ra, E->form, 4, di->sms * di->p2p_bps[E->form], s);
        if (e == cudaSuccess && E->form == SJ_FP32X) e = launch_p2p_recheck(w->ra, di->sms * 4, s);
    }
    if (e != cudaSuccess) return e;
    k_unsort_multi<<<blocks, 256, 0, s>>>(w->ma);
    return cudaGetLastError();
}

extern "C" sj_status sj_engine_create(int64_t max_points, int32_t max_requests, const sj_opts *o, sj_engine **out) {
    if (!out) return fail(SJ_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (max_points < 1 || max_points > MAX_COUNT) return fail(SJ_ERR_INVALID, "max_points must be in 1..2^31-2^22");
    if (max_requests < 1 || max_requests > (1 << 20)) return fail(SJ_ERR_INVALID, "max_requests must be in 1..2^20");
    const int form = o ? o->form : SJ_FP64;
    if (form != SJ_FP64 && form != SJ_FP32X) return fail(SJ_ERR_INVALID, "unknown form");
    const int ch = (o && o->pts_per_item) ? o->pts_per_item : 128;
    if (ch < 1 || ch > MAX_CH) return fail(SJ_ERR_INVALID, "pts_per_item must be in 1..128");
    sj_engine *E = new sj_engine();
    cudaError_t e = cudaGetDevice(&E->device);
    if (e != cudaSuccess) {
        delete E;
        return cuda_fail(e, "cudaGetDevice");
    }
    E->max_points = max_points;
    E->max_requests = max_requests;
    E->form = form;
    E->ch = ch;
    E->use_graph = !(o && (o->flags & SJ_FLAG_NO_GRAPH));
    *out = E;
    return SJ_OK;
}

extern "C" sj_status sj_engine_destroy(sj_engine *E) {
    if (!E) return SJ_OK;
    cudaDeviceSynchronize();
    for (LayerWork *w : E->work) work_free(w);
    delete E;
    return SJ_OK;
}

extern "C" sj_status sj_engine_round(sj_engine *E, const sj_request *reqs, int32_t n, void *stream) {
    if (!E) return fail(SJ_ERR_INVALID, "engine is NULL");
    if (n < 0 || (n > 0 && !reqs)) return fail(SJ_ERR_INVALID, "bad request list");
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev != E->device) return fail(SJ_ERR_INVALID, "engine belongs to another device");
    DevInfo *di;
    sj_status st = device_info(dev, &di);
    if (st != SJ_OK) return st;
    // validate everything before touching the device
    std::vector<const sj_layer *> layers;
    for (int k = 0; k < n; ++k) {
        const sj_request &r = reqs[k];
        if (!r.layer) return fail(SJ_ERR_INVALID, "request without a layer");
        if (r.layer->device != dev) return fail(SJ_ERR_INVALID, "layer belongs to another device");
        if (r.N < 0 || r.N > MAX_COUNT) return fail(SJ_ERR_INVALID, "request N out of range");
        if (r.N > 0 && (!r.pts || !r.out_id || !aligned16(r.pts))) return fail(SJ_ERR_INVALID, "bad request buffers");
        if (r.use_window && (r.layer->kind != KIND_P2P || !(r.window >= 0.0 && r.window <= r.layer->D)))
            return fail(SJ_ERR_INVALID, "a request window needs a polyline layer and 0 <= window <= its D");
        if (E->form == SJ_FP32X && r.layer->xmax > 1e30)
            return fail(SJ_ERR_INVALID, "SJ_FP32X needs grid coordinates below 1e30 in magnitude");
        if (std::find(layers.begin(), layers.end(), r.layer) == layers.end()) layers.push_back(r.layer);
    }
    for (const sj_layer *L : layers) {
        int64_t tot = 0;
        int cntr = 0;
        for (int k = 0; k < n; ++k)
            if (reqs[k].layer == L) { tot += reqs[k].N; ++cntr; }
        if (tot > E->max_points) return fail(SJ_ERR_INVALID, "a layer's requests exceed the engine's max_points");
        if (cntr > E->max_requests) return fail(SJ_ERR_INVALID, "more requests than the engine's max_requests");
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(E->mu);
    for (const sj_layer *L : layers) {
        LayerWork *w = nullptr;
        for (LayerWork *x : E->work)
            if (x->L == L) w = x;
        if (!w) {
            st = work_create(E, L, &w);
            if (st != SJ_OK) return st;
            E->work.push_back(w);
        }
        // request table of this layer into the next pinned slot
        const int sl = w->slot;
        w->slot ^= 1;
        CUDA_TRY(cudaEventSynchronize(w->copied[sl]));   // its previous copy has been consumed
        int nr = 0, off = 0, windows = 0;
        for (int k = 0; k < n; ++k) {
            const sj_request &r = reqs[k];
            if (r.layer != L || r.N == 0) continue;
            ReqDev d;
            d.pts = (const double2 *)r.pts;
            d.out_id = r.out_id;
            d.out_d = L->kind == KIND_P2P ? r.out_d : nullptr;
            d.window = r.use_window ? r.window : L->D;
            if (d.window < L->D) windows = 1;
            d.off = off;
            d.n = (int)r.N;
            w->h_reqs[sl][nr++] = d;
            off += (int)r.N;
        }
        L->joins += nr;
        L->points += off;
        if (nr == 0) continue;
        w->h_meta[sl][0] = nr;
        w->h_meta[sl][1] = off;
        w->h_meta[sl][2] = windows;
        CUDA_TRY(cudaMemcpyAsync(w->d_reqs, w->h_reqs[sl], sizeof(ReqDev) * (size_t)nr, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(w->d_meta, w->h_meta[sl], sizeof(int) * 4, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaEventRecord(w->copied[sl], s));
        if (E->use_graph && s != nullptr) {
            if (!w->exec) {
                cudaGraph_t graph = nullptr;
                CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
                cudaError_t e = enqueue_round(E, w, di, s);
                cudaError_t e2 = cudaStreamEndCapture(s, &graph);
                if (e != cudaSuccess) return cuda_fail(e, "round capture");
                if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
                e = cudaGraphInstantiate(&w->exec, graph, 0);
                cudaGraphDestroy(graph);
                if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
            }
            CUDA_TRY(cudaGraphLaunch(w->exec, s));
        } else {
            CUDA_TRY(enqueue_round(E, w, di, s));
        }
    }
    return SJ_OK;
}
