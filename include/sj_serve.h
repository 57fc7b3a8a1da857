/*
 * sj_serve.h -- continuous-batching request server over resident layers,
 * exported by libsj.so.
 *
 * Not in the paper, which joins one point set at a time (Sec. III).  A server
 * keeps one polygon layer and one polyline layer resident and serves a stream
 * of point batches ("requests") that arrive over time.  A worker thread owned
 * by the server
 *   - admits queued requests in submission order while their device memory
 *     (points, ids, distances) fits a fixed device budget, and copies their
 *     points to the device on a copy stream;
 *   - whenever fewer than two rounds are in flight, forms a round from the
 *     admitted requests in submission order and runs it through the batched
 *     engine (sj_engine_round: one graph replay per layer, however many
 *     requests), so that requests arriving while a round runs join the next
 *     one (SJ_SERVE_BATCHED).  A request of at least
 *     small = min(10^6, round_points / 4) points forms a round of its own, and
 *     a round of smaller ones stops before the next large one (and at
 *     round_points points or max_requests requests), so that no small request
 *     waits for a large one's work inside its round; a round of one request,
 *     or of fewer than `small` points, runs as direct join calls, which cost
 *     less than the graph sized for the largest round.  Or the server runs one
 *     join call per request in submission order (SJ_SERVE_PER_REQUEST, the
 *     baseline the batched form is measured against);
 *   - copies each round's results back on a second copy stream and marks its
 *     requests done with their completion time.
 * Every result is what sj_pip_join / sj_p2p_join computes for the request
 * alone, in the server's form.
 */
#ifndef SJ_SERVE_H
#define SJ_SERVE_H

#include <stdint.h>

#include "sj.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sj_server sj_server;

enum { SJ_SERVE_BATCHED = 0, SJ_SERVE_PER_REQUEST = 1 };
enum { SJ_SERVE_PIP = 0, SJ_SERVE_P2P = 1 };

/* One request.  All three buffers are host memory owned by the caller, and
 * must stay valid (and unread / unwritten by the caller) until the request is
 * done; page-locked memory (cudaHostAlloc, torch pin_memory) lets the copies
 * run asynchronously.  pts: [n, 2] float64, x and y interleaved; out_id: [n]
 * int32; out_d: [n] float64 for P2P (may be NULL; ignored for PIP). */
typedef struct {
    int32_t kind;         /* SJ_SERVE_PIP or SJ_SERVE_P2P                        */
    int32_t use_window;   /* P2P: nonzero = join within `window` instead of the
                             layer's D (as sj_p2p_join_window)                    */
    const double *pts;
    int64_t n;            /* 1 .. round_points                                    */
    int32_t *out_id;
    double *out_d;
    double not_before;    /* server clock (sj_server_now), seconds: the request
                             arrives then and is not admitted earlier; 0 = now.
                             Requests must be submitted in not_before order.      */
    double window;        /* 0 <= window <= the P2P layer's D when use_window     */
} sj_serve_request;

typedef struct {
    int64_t submitted;    /* requests accepted by sj_server_submit                */
    int64_t completed;
    int64_t rounds;       /* rounds (batched) or join calls (per request) issued  */
    int64_t points;       /* points of the completed requests                     */
    double max_launch_s;  /* longest host time spent issuing one round            */
    double max_round_s;   /* longest time from issuing a round to its completion  */
} sj_server_stats;

/* Create a server on the current device (this also builds the engine's
 * workspace and graph for each layer, and grows the device's default
 * stream-ordered memory pool to the largest direct join, so that no request
 * waits for them; the server sets that pool's release threshold to keep its
 * memory, an attribute of this process's pool that stays after destroy).
 * pip / p2p: resident layers (either
 * may be NULL if no request of that kind is submitted; they must outlive the
 * server).  opts: form and points per work item of every round (NULL = FP64,
 * defaults).  mode: SJ_SERVE_BATCHED or SJ_SERVE_PER_REQUEST.  hbm_budget:
 * bytes of device memory for admitted requests (one allocation; a request
 * needs 16 n + 4 n (+ 8 n for P2P) bytes plus alignment).  round_points /
 * max_requests: limits of one batched round.  Errors: SJ_ERR_INVALID,
 * SJ_ERR_OOM, SJ_ERR_CUDA. */
sj_status sj_server_create(sj_layer *pip, sj_layer *p2p, const sj_opts *opts, int32_t mode, int64_t hbm_budget,
                           int64_t round_points, int32_t max_requests, sj_server **out);

/* Queue a request (thread-safe, does not block on the GPU).  *ticket receives
 * its id for sj_server_wait / sj_server_poll.  Errors: SJ_ERR_INVALID (bad
 * kind, missing layer, n out of range, NULL buffers, a request larger than
 * the device budget, a window outside [0, D] or on a PIP request),
 * SJ_ERR_BUSY (refused at admission; the server keeps serving), or the error
 * that stopped the worker. */
sj_status sj_server_submit(sj_server *s, const sj_serve_request *req, int64_t *ticket);

/* Block until request `ticket` is done; *latency_s (may be NULL) receives
 * (results in host memory) - (arrival), in seconds, where arrival is the later
 * of submission and not_before.  Returns the status of the request (SJ_OK,
 * SJ_ERR_CANCELLED, or the CUDA / engine error that failed it). */
sj_status sj_server_wait(sj_server *s, int64_t ticket, double *latency_s);

/* sj_server_wait with a deadline: SJ_ERR_TIMEOUT when the request is not done
 * within timeout_s seconds (it keeps its place; wait for it again), else as
 * sj_server_wait.  Errors: SJ_ERR_INVALID (unknown ticket, negative or NaN
 * timeout), SJ_ERR_TIMEOUT, SJ_ERR_CANCELLED, the request's own error. */
sj_status sj_server_wait_for(sj_server *s, int64_t ticket, double timeout_s, double *latency_s);

/* Cancel a request that has not been admitted yet (it is queued, or its
 * not_before lies ahead): the worker drops it before any device work, and its
 * wait returns SJ_ERR_CANCELLED (its outputs untouched).  SJ_ERR_BUSY when the
 * request is already admitted, running or done; SJ_ERR_INVALID for an unknown
 * ticket. */
sj_status sj_server_cancel(sj_server *s, int64_t ticket);

/* Non-blocking: *done = 1 when request `ticket` is done, else 0. */
sj_status sj_server_poll(sj_server *s, int64_t ticket, int32_t *done);

/* Block until every submitted request is done. */
sj_status sj_server_drain(sj_server *s);

/* Switch between SJ_SERVE_BATCHED and SJ_SERVE_PER_REQUEST for rounds formed
 * from now on; form (SJ_FP64 / SJ_FP32X) applies to per-request joins, and
 * must equal the server's form for batched rounds (the engine's form is fixed
 * at creation).  Errors: SJ_ERR_INVALID. */
sj_status sj_server_set_mode(sj_server *s, int32_t mode, int32_t form);

sj_status sj_server_get_stats(sj_server *s, sj_server_stats *out);

/* Restart the max_launch_s / max_round_s maxima (the counters keep running). */
sj_status sj_server_reset_maxima(sj_server *s);

/* The server's clock: seconds since the server was created (steady clock). */
double sj_server_now(const sj_server *s);

/* Stop the worker after the requests in flight are done, free everything.
 * NULL is a no-op. */
sj_status sj_server_destroy(sj_server *s);

#ifdef __cplusplus
}
#endif

#endif /* SJ_SERVE_H */
