// sj_serve.cu -- the continuous-batching request server of include/sj_serve.h.
//
// One worker thread per server owns every CUDA call of the serving loop:
//   admission  -- queued requests, in submission order, get a block of the
//                 device arena (a ring: blocks are handed out in order and
//                 reclaimed once every older block is free) and an
//                 asynchronous host-to-device copy of their points (stream
//                 copy_in; one event per admitted batch);
//   rounds     -- with fewer than two rounds in flight, the admitted requests
//                 (up to round_points / max_requests; a large request alone,
//                 small ones together) form a round on stream compute, which
//                 first waits for the copies it needs; the round is one
//                 sj_engine_round (SJ_SERVE_BATCHED) or one join call per
//                 request (SJ_SERVE_PER_REQUEST);
//   results    -- stream copy_out waits for the round and copies ids (and
//                 distances) back; when its event completes, the round's
//                 requests are done (completion time taken then) and their
//                 arena blocks are released.
// Client threads only queue requests and wait on a condition variable.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sj_host.hpp"
#include "sj_serve.h"

using namespace sj;

namespace {

using Clock = std::chrono::steady_clock;

constexpr size_t ALIGN = 256;
constexpr int64_t SMALL_ROUND = 1000000;   // points; smaller batched rounds run as direct joins

size_t round_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

// Device bytes of one request: points, ids and (P2P) distances, each aligned.
size_t request_bytes(const sj_serve_request &r) {
    const size_t n = (size_t)r.n;
    return round_up(16 * n) + round_up(4 * n) + (r.kind == SJ_SERVE_P2P ? round_up(8 * n) : 0);
}

struct Block {
    size_t start = 0, size = 0;
    bool freed = false;
};

// Ring allocator over one device buffer.
struct Ring {
    char *base = nullptr;
    size_t cap = 0, head = 0;
    std::deque<Block *> live;   // allocation order

    Block *alloc(size_t size) {
        size = round_up(size);
        if (size > cap) return nullptr;
        size_t start;
        if (live.empty()) {
            head = 0;
            start = 0;
        } else {
            const size_t tail = live.front()->start;
            if (head >= tail) {   // free: [head, cap) and [0, tail)
                if (cap - head >= size) start = head;
                else if (tail >= size) start = 0;
                else return nullptr;
            } else {              // free: [head, tail)
                if (tail - head >= size) start = head;
                else return nullptr;
            }
        }
        Block *b = new Block{start, size, false};
        live.push_back(b);
        head = start + size;
        return b;
    }
    void release(Block *b) {
        b->freed = true;
        while (!live.empty() && live.front()->freed) {
            delete live.front();
            live.pop_front();
        }
    }
};

enum { Q_QUEUED = 0, Q_ADMITTED, Q_RUNNING, Q_DONE };

struct Req {
    int64_t ticket = 0;
    sj_serve_request r{};
    double t_submit = 0.0, t_done = 0.0;
    int state = Q_QUEUED;
    bool cancel = false;     // sj_server_cancel asked; the worker finishes it before admission
    sj_status status = SJ_OK;
    Block *blk = nullptr;
    double *d_pts = nullptr;
    int32_t *d_id = nullptr;
    double *d_d = nullptr;
    struct CopyBatch *batch = nullptr;   // admission batch whose event covers this copy
};

// Requests admitted together share one copy event; it is destroyed once every
// one of them has been placed in a round (whose stream has waited for it).
struct CopyBatch {
    cudaEvent_t ev = nullptr;
    int remaining = 0;
};

struct Round {
    cudaEvent_t done = nullptr;
    std::vector<Req *> reqs;
    double t_issue = 0.0;
};

}  // namespace

struct sj_server {
    sj_layer *layers[2] = {nullptr, nullptr};
    sj_engine *engine = nullptr;
    int form = SJ_FP64;
    int ppi = 0;
    std::atomic<int> mode{SJ_SERVE_BATCHED};
    std::atomic<int> run_form{SJ_FP64};
    int64_t round_points = 0;
    int32_t max_requests = 0;
    int device = 0;
    Clock::time_point epoch = Clock::now();
    double now() const { return std::chrono::duration<double>(Clock::now() - epoch).count(); }
    cudaStream_t copy_in = nullptr, compute = nullptr, copy_out = nullptr;
    Ring ring;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> incoming;                       // submitted, not yet taken by the worker
    std::unordered_map<int64_t, Req *> reqs;          // every request not yet waited for
    std::atomic<bool> cancels{false};                 // a cancel is pending (wakes the worker)
    int64_t next_ticket = 0;
    bool stop = false;
    sj_status fatal = SJ_OK;
    std::string fatal_msg;

    std::atomic<long long> submitted{0}, completed{0}, rounds{0}, points{0};
    std::atomic<double> max_launch{0.0}, max_round{0.0};
    std::thread worker;

    // worker-only state
    std::deque<Req *> arriving;                       // submitted, not_before still ahead
    std::deque<Req *> queue;                          // arrived, waiting for arena space
    std::deque<Req *> ready;                          // admitted, copy issued
    std::deque<Round> in_flight;
    std::deque<CopyBatch *> batches;                  // admission batches, oldest first

    void run();
    void finish_cancelled(std::deque<Req *> &d);
    bool admit();
    bool launch_round();
    bool retire();
    void fail_all(sj_status st, const std::string &msg);
};

void sj_server::fail_all(sj_status st, const std::string &msg) {
    std::lock_guard<std::mutex> lk(mu);
    if (fatal == SJ_OK) {
        fatal = st;
        fatal_msg = msg;
    }
    auto finish = [&](Req *q) {
        if (q->state != Q_DONE) {
            q->state = Q_DONE;
            q->status = st;
            q->t_done = now();
            completed++;
        }
    };
    for (Req *q : arriving) finish(q);
    for (Req *q : queue) finish(q);
    for (Req *q : ready) finish(q);
    for (auto &rd : in_flight) {
        for (Req *q : rd.reqs) finish(q);
        if (rd.done) cudaEventDestroy(rd.done);
    }
    for (Req *q : incoming) finish(q);
    arriving.clear();
    queue.clear();
    ready.clear();
    in_flight.clear();
    incoming.clear();
    cv_done.notify_all();
}

// Requests cancelled before admission leave their queue, done with status
// SJ_ERR_CANCELLED (worker thread).
void sj_server::finish_cancelled(std::deque<Req *> &d) {
    std::lock_guard<std::mutex> lk(mu);
    bool any = false;
    for (auto it = d.begin(); it != d.end();) {
        Req *q = *it;
        if (q->cancel) {
            q->state = Q_DONE;
            q->status = SJ_ERR_CANCELLED;
            q->t_done = now();
            completed++;
            it = d.erase(it);
            any = true;
        } else {
            ++it;
        }
    }
    cancels = false;
    if (any) cv_done.notify_all();
}

// Admission: arena blocks and host-to-device copies, in submission order.
bool sj_server::admit() {
    std::vector<Req *> batch;
    while (!queue.empty()) {
        Req *q = queue.front();
        Block *b = ring.alloc(request_bytes(q->r));
        if (!b) break;
        queue.pop_front();
        q->blk = b;
        char *p = ring.base + b->start;
        const size_t n = (size_t)q->r.n;
        q->d_pts = (double *)p;
        q->d_id = (int32_t *)(p + round_up(16 * n));
        q->d_d = q->r.kind == SJ_SERVE_P2P ? (double *)(p + round_up(16 * n) + round_up(4 * n)) : nullptr;
        cudaError_t e = cudaMemcpyAsync(q->d_pts, q->r.pts, 16 * n, cudaMemcpyHostToDevice, copy_in);
        if (e != cudaSuccess) {
            for (Req *b2 : batch) ready.push_back(b2);   // so that fail_all finishes them
            ready.push_back(q);
            fail_all(SJ_ERR_CUDA, std::string("server copy in: ") + cudaGetErrorString(e));
            return false;
        }
        q->state = Q_ADMITTED;
        batch.push_back(q);
    }
    if (batch.empty()) return false;
    CopyBatch *cb = new CopyBatch();
    batches.push_back(cb);
    cb->remaining = (int)batch.size();
    cudaError_t e = cudaEventCreateWithFlags(&cb->ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(cb->ev, copy_in);
    if (e != cudaSuccess) {
        for (Req *b2 : batch) ready.push_back(b2);
        fail_all(SJ_ERR_CUDA, std::string("server copy event: ") + cudaGetErrorString(e));
        return false;
    }
    for (Req *q : batch) {
        q->batch = cb;
        ready.push_back(q);
    }
    return true;
}

// One round from the admitted requests (submission order).
bool sj_server::launch_round() {
    if (ready.empty() || in_flight.size() >= 2) return false;
    const int m = mode.load();
    Round rd;
    rd.t_issue = now();
    int64_t tot = 0;
    // Batched rounds merge consecutive small requests only: a request of at
    // least `small` points forms a round of its own (a direct join, efficient
    // alone), and a round of small requests stops before the next large one,
    // so that no small request waits for a large one's work inside its round
    // (in submission order, as in the per-request form).
    const int64_t small = std::min<int64_t>(SMALL_ROUND, round_points / 4);
    while (!ready.empty()) {
        Req *q = ready.front();
        if (!rd.reqs.empty() && (m == SJ_SERVE_PER_REQUEST || tot + q->r.n > round_points ||
                                 (int64_t)rd.reqs.size() >= max_requests || q->r.n >= small ||
                                 rd.reqs.front()->r.n >= small))
            break;
        ready.pop_front();
        rd.reqs.push_back(q);
        tot += q->r.n;
    }
    // the copies are in order on copy_in: waiting for the newest event covers all
    cudaError_t e = cudaStreamWaitEvent(compute, rd.reqs.back()->batch->ev, 0);
    if (e != cudaSuccess) {
        fail_all(SJ_ERR_CUDA, std::string("server wait: ") + cudaGetErrorString(e));
        return false;
    }
    for (Req *q : rd.reqs) q->batch->remaining--;
    while (!batches.empty() && batches.front()->remaining == 0) {
        cudaEventDestroy(batches.front()->ev);
        delete batches.front();
        batches.pop_front();
    }
    // A batched round below min(SMALL_ROUND, round_points / 4) points, or of
    // one request, runs as direct joins: the
    // engine's graph is sized for its maximum round, and its fixed cost
    // (scans over every cell, grids for round_points) exceeds a few direct
    // launches when the round is small.
    sj_status st = SJ_OK;
    if (m == SJ_SERVE_BATCHED && tot >= small && rd.reqs.size() > 1) {
        std::vector<sj_request> t(rd.reqs.size());
        for (size_t k = 0; k < rd.reqs.size(); ++k) {
            Req *q = rd.reqs[k];
            t[k].layer = layers[q->r.kind];
            t[k].pts = q->d_pts;
            t[k].N = q->r.n;
            t[k].out_id = q->d_id;
            t[k].out_d = q->d_d;
            t[k].use_window = q->r.use_window;
            t[k].window = q->r.window;
        }
        st = sj_engine_round(engine, t.data(), (int32_t)t.size(), compute);
    } else {
        sj_opts o{};
        o.form = m == SJ_SERVE_BATCHED ? form : run_form.load();
        o.launch = SJ_PER_REQUEST;
        o.pts_per_item = ppi;
        for (Req *q : rd.reqs) {
            if (q->r.kind == SJ_SERVE_PIP)
                st = sj_pip_join(layers[0], q->d_pts, q->r.n, q->d_id, &o, compute);
            else if (q->r.use_window)
                st = sj_p2p_join_window(layers[1], q->d_pts, q->r.n, q->r.window, q->d_id, q->d_d, &o, compute);
            else
                st = sj_p2p_join(layers[1], q->d_pts, q->r.n, q->d_id, q->d_d, &o, compute);
            if (st != SJ_OK) break;
        }
    }
    if (st != SJ_OK) {
        in_flight.push_back(std::move(rd));   // so that fail_all finishes them
        fail_all(st, std::string("server round: ") + sj_last_error());
        return false;
    }
    cudaEvent_t ran = nullptr;
    e = cudaEventCreateWithFlags(&ran, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ran, compute);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(copy_out, ran, 0);
    for (Req *q : rd.reqs) {
        q->state = Q_RUNNING;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(q->r.out_id, q->d_id, 4 * (size_t)q->r.n, cudaMemcpyDeviceToHost, copy_out);
        if (e == cudaSuccess && q->d_d && q->r.out_d)
            e = cudaMemcpyAsync(q->r.out_d, q->d_d, 8 * (size_t)q->r.n, cudaMemcpyDeviceToHost, copy_out);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&rd.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(rd.done, copy_out);
    if (ran) cudaEventDestroy(ran);   // destruction waits for nothing; the dependency stays
    if (e != cudaSuccess) {
        in_flight.push_back(std::move(rd));
        fail_all(SJ_ERR_CUDA, std::string("server results: ") + cudaGetErrorString(e));
        return false;
    }
    const double dt = now() - rd.t_issue;
    if (dt > max_launch.load()) max_launch = dt;
    in_flight.push_back(std::move(rd));
    rounds++;
    return true;
}

// Completed rounds, in order.
bool sj_server::retire() {
    bool any = false;
    while (!in_flight.empty()) {
        cudaError_t e = cudaEventQuery(in_flight.front().done);
        if (e == cudaErrorNotReady) break;
        if (e != cudaSuccess) {
            fail_all(SJ_ERR_CUDA, std::string("server round failed: ") + cudaGetErrorString(e));
            return false;
        }
        Round rd = std::move(in_flight.front());
        in_flight.pop_front();
        cudaEventDestroy(rd.done);
        const double t = now();
        if (t - rd.t_issue > max_round.load()) max_round = t - rd.t_issue;
        {
            std::lock_guard<std::mutex> lk(mu);
            for (Req *q : rd.reqs) {
                q->t_done = t;
                q->state = Q_DONE;
                ring.release(q->blk);
                q->blk = nullptr;
                completed++;
                points += q->r.n;
            }
        }
        cv_done.notify_all();
        any = true;
    }
    return any;
}

void sj_server::run() {
    cudaSetDevice(device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(mu);
            if (incoming.empty() && queue.empty() && ready.empty() && in_flight.empty()) {
                if (arriving.empty()) {
                    if (stop) break;
                    cv_work.wait(lk, [&] { return stop || !incoming.empty(); });
                    if (stop && incoming.empty()) break;
                } else {   // sleep until the next arrival (or a new submission)
                    const double dt = arriving.front()->t_submit - now();
                    if (dt > 2e-4)
                        cv_work.wait_for(lk, std::chrono::duration<double>(dt - 1e-4),
                                         [&] { return stop || cancels || !incoming.empty(); });
                }
            }
            while (!incoming.empty()) {
                arriving.push_back(incoming.front());
                incoming.pop_front();
            }
        }
        if (fatal != SJ_OK) {
            fail_all(fatal, fatal_msg);
            continue;
        }
        if (cancels) {
            finish_cancelled(arriving);
            finish_cancelled(queue);
        }
        const double t = now();
        while (!arriving.empty() && arriving.front()->t_submit <= t) {   // arrivals, in order
            queue.push_back(arriving.front());
            arriving.pop_front();
        }
        bool progress = retire();
        progress |= admit();
        progress |= launch_round();
        if (!progress) std::this_thread::yield();   // GPU work in flight: poll again
    }
    for (CopyBatch *cb : batches) {
        if (cb->ev) cudaEventDestroy(cb->ev);
        delete cb;
    }
    batches.clear();
}

extern "C" sj_status sj_server_create(sj_layer *pip, sj_layer *p2p, const sj_opts *opts, int32_t mode,
                                      int64_t hbm_budget, int64_t round_points, int32_t max_requests,
                                      sj_server **out) {
    if (!out) return fail(SJ_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!pip && !p2p) return fail(SJ_ERR_INVALID, "a server needs at least one layer");
    if (pip && pip->kind != KIND_PIP) return fail(SJ_ERR_INVALID, "pip is not a polygon layer");
    if (p2p && p2p->kind != KIND_P2P) return fail(SJ_ERR_INVALID, "p2p is not a polyline layer");
    if (mode != SJ_SERVE_BATCHED && mode != SJ_SERVE_PER_REQUEST) return fail(SJ_ERR_INVALID, "unknown mode");
    if (hbm_budget < (int64_t)(4 * ALIGN)) return fail(SJ_ERR_INVALID, "hbm_budget too small");
    if (round_points < 1 || round_points > MAX_COUNT) return fail(SJ_ERR_INVALID, "round_points out of range");
    if (max_requests < 1) return fail(SJ_ERR_INVALID, "max_requests must be >= 1");
    const int form = opts ? opts->form : SJ_FP64;
    if (form != SJ_FP64 && form != SJ_FP32X) return fail(SJ_ERR_INVALID, "unknown form");
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if ((pip && pip->device != dev) || (p2p && p2p->device != dev))
        return fail(SJ_ERR_INVALID, "layers belong to another device");

    sj_server *S = new sj_server();
    S->layers[0] = pip;
    S->layers[1] = p2p;
    S->form = form;
    S->ppi = opts ? opts->pts_per_item : 0;
    S->mode = mode;
    S->run_form = form;
    S->round_points = round_points;
    S->max_requests = max_requests;
    S->device = dev;
    auto undo = [&](sj_status st) {
        if (S->engine) sj_engine_destroy(S->engine);
        if (S->ring.base) cudaFree(S->ring.base);
        for (cudaStream_t st_ : {S->copy_in, S->compute, S->copy_out})
            if (st_) cudaStreamDestroy(st_);
        delete S;
        return st;
    };
    cudaError_t e = dev_malloc((void **)&S->ring.base, (size_t)hbm_budget);
    if (e != cudaSuccess) return undo(cuda_fail(e, "server arena"));
    S->ring.cap = (size_t)hbm_budget / ALIGN * ALIGN;
    for (cudaStream_t *st_ : {&S->copy_in, &S->compute, &S->copy_out}) {
        e = cudaStreamCreateWithFlags(st_, cudaStreamNonBlocking);
        if (e != cudaSuccess) return undo(cuda_fail(e, "server stream"));
    }
    sj_opts eo{};
    eo.form = form;
    eo.launch = SJ_PERSISTENT;
    eo.pts_per_item = S->ppi;
    sj_status st = sj_engine_create(round_points, max_requests, &eo, &S->engine);
    if (st != SJ_OK) return undo(st);
    // The engine builds a layer's workspace and captures its graph on the first
    // round that uses the layer (allocations of hundreds of MB): do that now,
    // with a one-point round per layer, so that no served request waits for it.
    {
        char *tmp = nullptr;
        e = cudaMalloc((void **)&tmp, 256 * 3);
        if (e != cudaSuccess) return undo(cuda_fail(e, "server warm-up"));
        const double origin[2] = {0.0, 0.0};
        e = cudaMemcpy(tmp, origin, sizeof(origin), cudaMemcpyHostToDevice);
        for (int k = 0; k < 2 && e == cudaSuccess && st == SJ_OK; ++k) {
            if (!S->layers[k]) continue;
            sj_request r{};
            r.layer = S->layers[k];
            r.pts = (const double *)tmp;
            r.N = 1;
            r.out_id = (int32_t *)(tmp + 256);
            r.out_d = k == 1 ? (double *)(tmp + 512) : nullptr;
            st = sj_engine_round(S->engine, &r, 1, S->compute);
        }
        // Direct joins take their scratch from the device's stream-ordered
        // pool.  By default the pool hands freed memory back at every
        // synchronising call (the engine waits on events), and the next join
        // then grows it again (milliseconds for hundreds of MB).  The server
        // makes the pool keep what it holds (a process-wide attribute of this
        // device's default pool) and reserves the largest join now (a request
        // of round_points points needs under 64 B per point plus per-cell
        // arrays), so that the pool never grows while requests are served.
        cudaMemPool_t pool = nullptr;
        if (e == cudaSuccess) e = cudaDeviceGetDefaultMemPool(&pool, dev);
        if (e == cudaSuccess) {
            unsigned long long keep = ~0ULL;   // the attribute is a 64-bit unsigned value
            e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        void *big = nullptr;
        if (e == cudaSuccess)
            e = cudaMallocAsync(&big, (size_t)round_points * 64 + ((size_t)64 << 20), S->compute);
        if (e == cudaSuccess) e = cudaFreeAsync(big, S->compute);
        if (e == cudaSuccess) e = cudaStreamSynchronize(S->compute);
        cudaFree(tmp);
        if (st != SJ_OK) return undo(st);
        if (e != cudaSuccess) return undo(cuda_fail(e, "server warm-up"));
    }
    S->worker = std::thread([S] { S->run(); });
    *out = S;
    return SJ_OK;
}

extern "C" sj_status sj_server_submit(sj_server *S, const sj_serve_request *req, int64_t *ticket) {
    if (!S || !req || !ticket) return fail(SJ_ERR_INVALID, "NULL argument");
    const sj_serve_request &r = *req;
    if (r.kind != SJ_SERVE_PIP && r.kind != SJ_SERVE_P2P) return fail(SJ_ERR_INVALID, "unknown request kind");
    if (!S->layers[r.kind]) return fail(SJ_ERR_INVALID, "the server has no layer of this kind");
    if (r.n < 1 || r.n > S->round_points) return fail(SJ_ERR_INVALID, "request size out of range");
    if (!r.pts || !r.out_id) return fail(SJ_ERR_INVALID, "NULL buffer");
    if (r.use_window && (r.kind != SJ_SERVE_P2P || !(r.window >= 0.0 && r.window <= S->layers[r.kind]->D)))
        return fail(SJ_ERR_INVALID, "a request window needs a P2P request and 0 <= window <= the layer's D");
    if (request_bytes(r) > S->ring.cap) return fail(SJ_ERR_INVALID, "request larger than the device budget");
    if (fault_fires(SJ_FAULT_ADMIT)) return fail(SJ_ERR_BUSY, "request refused at admission (injected fault)");
    Req *q = new Req();
    q->r = r;
    if (r.kind == SJ_SERVE_PIP) q->r.out_d = nullptr;
    q->t_submit = std::max(S->now(), r.not_before);   // the arrival
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->fatal != SJ_OK) {
            delete q;
            return fail(S->fatal, "server stopped: " + S->fatal_msg);
        }
        q->ticket = S->next_ticket++;
        S->reqs[q->ticket] = q;
        S->incoming.push_back(q);
        S->submitted++;
    }
    S->cv_work.notify_one();
    *ticket = q->ticket;
    return SJ_OK;
}

extern "C" sj_status sj_server_wait(sj_server *S, int64_t ticket, double *latency_s) {
    if (!S) return fail(SJ_ERR_INVALID, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(SJ_ERR_INVALID, "unknown or already waited-for ticket");
    Req *q = it->second;
    S->cv_done.wait(lk, [&] { return q->state == Q_DONE; });
    if (latency_s) *latency_s = q->t_done - q->t_submit;
    const sj_status st = q->status;
    S->reqs.erase(it);
    delete q;
    if (st == SJ_ERR_CANCELLED) return fail(st, "request cancelled");
    if (st != SJ_OK) return fail(st, "request failed: " + S->fatal_msg);
    return SJ_OK;
}

extern "C" sj_status sj_server_wait_for(sj_server *S, int64_t ticket, double timeout_s, double *latency_s) {
    if (!S) return fail(SJ_ERR_INVALID, "NULL server");
    if (!(timeout_s >= 0.0)) return fail(SJ_ERR_INVALID, "timeout must be >= 0");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(SJ_ERR_INVALID, "unknown or already waited-for ticket");
    Req *q = it->second;
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(std::min(timeout_s, 1e9)));
    if (!S->cv_done.wait_until(lk, deadline, [&] { return q->state == Q_DONE; }))
        return fail(SJ_ERR_TIMEOUT, "request not done within the timeout (it keeps running; wait again)");
    if (latency_s) *latency_s = q->t_done - q->t_submit;
    const sj_status st = q->status;
    S->reqs.erase(it);
    delete q;
    if (st == SJ_ERR_CANCELLED) return fail(st, "request cancelled");
    if (st != SJ_OK) return fail(st, "request failed: " + S->fatal_msg);
    return SJ_OK;
}

extern "C" sj_status sj_server_cancel(sj_server *S, int64_t ticket) {
    if (!S) return fail(SJ_ERR_INVALID, "NULL server");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return fail(SJ_ERR_INVALID, "unknown or already waited-for ticket");
        Req *q = it->second;
        if (q->state != Q_QUEUED) return fail(SJ_ERR_BUSY, "request already admitted or done");
        q->cancel = true;
        S->cancels = true;
    }
    S->cv_work.notify_one();
    return SJ_OK;
}

extern "C" sj_status sj_server_poll(sj_server *S, int64_t ticket, int32_t *done) {
    if (!S || !done) return fail(SJ_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(SJ_ERR_INVALID, "unknown or already waited-for ticket");
    *done = it->second->state == Q_DONE ? 1 : 0;
    return SJ_OK;
}

extern "C" sj_status sj_server_drain(sj_server *S) {
    if (!S) return fail(SJ_ERR_INVALID, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_done.wait(lk, [&] { return S->completed.load() >= S->submitted.load(); });
    if (S->fatal != SJ_OK) return fail(S->fatal, "server stopped: " + S->fatal_msg);
    return SJ_OK;
}

extern "C" sj_status sj_server_set_mode(sj_server *S, int32_t mode, int32_t form) {
    if (!S) return fail(SJ_ERR_INVALID, "NULL server");
    if (mode != SJ_SERVE_BATCHED && mode != SJ_SERVE_PER_REQUEST) return fail(SJ_ERR_INVALID, "unknown mode");
    if (form != SJ_FP64 && form != SJ_FP32X) return fail(SJ_ERR_INVALID, "unknown form");
    if (mode == SJ_SERVE_BATCHED && form != S->form)
        return fail(SJ_ERR_INVALID, "batched rounds use the form the server was created with");
    S->run_form = form;
    S->mode = mode;
    return SJ_OK;
}

extern "C" sj_status sj_server_get_stats(sj_server *S, sj_server_stats *out) {
    if (!S || !out) return fail(SJ_ERR_INVALID, "NULL argument");
    out->submitted = S->submitted.load();
    out->completed = S->completed.load();
    out->rounds = S->rounds.load();
    out->points = S->points.load();
    out->max_launch_s = S->max_launch.load();
    out->max_round_s = S->max_round.load();
    return SJ_OK;
}

extern "C" sj_status sj_server_reset_maxima(sj_server *S) {
    if (!S) return fail(SJ_ERR_INVALID, "NULL server");
    S->max_launch = 0.0;
    S->max_round = 0.0;
    return SJ_OK;
}

extern "C" double sj_server_now(const sj_server *S) { return S ? S->now() : 0.0; }

extern "C" sj_status sj_server_destroy(sj_server *S) {
    if (!S) return SJ_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaDeviceSynchronize();
    for (auto &kv : S->reqs) {
        if (kv.second->blk) S->ring.release(kv.second->blk);
        delete kv.second;
    }
    S->reqs.clear();
    for (Block *b : S->ring.live) delete b;
    S->ring.live.clear();
    if (S->engine) sj_engine_destroy(S->engine);
    if (S->ring.base) cudaFree(S->ring.base);
    for (cudaStream_t st_ : {S->copy_in, S->compute, S->copy_out})
        if (st_) cudaStreamDestroy(st_);
    delete S;
    return SJ_OK;
}
