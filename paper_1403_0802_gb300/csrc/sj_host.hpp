// sj_host.hpp -- host-side internals shared by the C ABI translation units
// (sj_api.cu, sj_engine.cu): the layer object, error reporting, device info
// and the scratch carver.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "sj.h"
#include "sj_internal.cuh"

struct sj_layer {
    int kind = 0;
    int device = 0;
    sj_grid grid{};
    sj::GridDev g{};
    int nobj = 0;
    int V = 0;
    int64_t R = 0;
    double D = 0.0;
    int64_t M = 0;
    float eps_abs = 0.0f;
    double2 *verts = nullptr;
    float4 *vsplit = nullptr;
    int *obj_voff = nullptr;
    int *nxt = nullptr;
    int *prv = nullptr;        // PIP: previous vertex of the same ring
    int *ring_off = nullptr;
    int *poly_ring_off = nullptr;
    double2 *seg_e64 = nullptr;
    double *seg_inv64 = nullptr;
    float4 *seg32 = nullptr;   // (fl32(ex), fl32(ey), fl32(1 / |e|^2), owner polyline id as bits or -1)
    sj::Box *mbb = nullptr;
    int *cand_start = nullptr;
    int *cand_ids = nullptr;
    // P2P: per-cell segment lists (segments whose box widened by D meets the
    // cell) and, per cell, the segment count of its candidate polylines.
    int64_t MS = 0;
    int *cseg_start = nullptr;
    int *cseg_ids = nullptr;
    int *cell_algo = nullptr;
    float4 *cseg_rec = nullptr;   // [2 MS] per list entry: cell-relative (ax, ay, ex, ey) and
                                  // (1 / |e|^2, owner id bits, magnitude bound, segment index bits)
    // PIP: per-(polygon, grid row) edge lists (edges whose y-range rows include
    // the row), polygon-major; see sj_filter.cu.
    int64_t MR = 0, ME = 0;
    int *prow_base = nullptr;    // [nobj + 1] first (polygon, row) slot of each polygon
    int *prow_r0 = nullptr;      // [nobj] first row of each polygon's MBB
    int *prow_start = nullptr;   // [MR + 1] list ranges in pedge_ids
    int *pedge_ids = nullptr;    // [ME] edge (= first vertex) indices
    float4 *pedge_rec = nullptr; // [2 ME] FP32X staging records: vsplit of the edge's two ends
    unsigned char *cand_cls = nullptr;   // [M] per candidate entry: 0 boundary, 1 inside, 2 outside
    int *cell_res = nullptr;             // [G] result of every point of a fully classified cell, or CELL_REFINE
    int *cell_work = nullptr;            // [G] per-point edge / segment work of each cell (item sizes)
    // PIP boundary entries (class 0): near edges (x-range meets the cell's column
    // widened by delta) and the flip keys of the far-right edges' parity in y
    int64_t MN = 0, MF = 0;
    int *bnear_start = nullptr;              // [M + 1]
    int *bnear_ids = nullptr;                // [MN]
    float4 *bnear_rec = nullptr;             // [2 MN] vsplit of both ends
    float *bnear_key = nullptr;              // [MN] lower truncated y of each near edge, ascending per entry
    float *bnear_h = nullptr;                // [M] largest truncated y-extent of an entry's near edges
    int *bflip_start = nullptr;              // [M + 1]
    int *bflip_len = nullptr;                // [M] keys left after cancelling equal pairs
    unsigned long long *bflip_keys = nullptr;   // [MF] order keys, ascending within an entry
    unsigned long long *stats = nullptr;
    unsigned long long *cell_keys = nullptr;   // [nx + 1 + ny + 1] threshold tables of point_cell
    float *frames = nullptr;                   // [nx + ny] FP32 cell frame origins
    double xmax = 0.0;                         // largest |coordinate| of the grid box
    int64_t max_obj_verts = 0;                 // vertices of the largest polygon / polyline
    float Df = 0.0f, Ddn = 0.0f, Dup = 0.0f;   // FP32 forms of D (nearest, rounded down, rounded up)
    mutable std::atomic<long long> joins{0};
    mutable std::atomic<long long> points{0};
    mutable std::atomic<long long> census_tests{0};       // sj_pip_census totals since the last reset
    mutable std::atomic<long long> census_straddles{0};
    // SJ_FLAG_TIME_REFINE: event pairs recorded around refinement launches,
    // resolved (and destroyed) by sj_layer_get_stats.
    mutable std::mutex ev_mu;
    mutable std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
    mutable double refine_ms = 0.0;
    mutable long long refine_launches = 0;
};

namespace sj {

// Per-device launch facts, filled on first use.
struct DevInfo {
    int sms = 0;
    int pip_bps[2] = {0, 0};
    int p2p_bps[2] = {0, 0};
    cudaStream_t hstream[3] = {nullptr, nullptr, nullptr};   // host joins: copy in, join, copy out
    bool init = false;
};

sj_status fail(sj_status st, const std::string &msg);
sj_status cuda_fail(cudaError_t e, const char *what);

// Host-side fault injection (sj_fault_inject): true when an armed fault of
// this kind fires now.
bool fault_fires(int kind);
// Device allocations of the library, which an armed SJ_FAULT_ALLOC makes fail
// as out of memory.
cudaError_t dev_malloc(void **p, size_t bytes);
cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t s);
sj_status device_info(int dev, DevInfo **out);
void fill_refine(const sj_layer *L, RefineArgs &ra);

inline bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Scratch carved from one allocation, 256-byte aligned pieces.
struct Scratch {
    char *base = nullptr;
    size_t off = 0;
    template <class T>
    T *take(size_t n) {
        off = (off + 255) & ~(size_t)255;
        T *p = (T *)(base + off);
        off += n * sizeof(T);
        return p;
    }
};

template <class F>
size_t measure(F f) {
    Scratch s;
    f(s);
    return s.off + 256;
}

// Launchers shared across files.
cudaError_t launch_bucket_scan(const BucketArgs &a, cudaStream_t s);

}  // namespace sj

#define CUDA_TRY(x)                                          \
    do {                                                     \
        cudaError_t e_ = (x);                                \
        if (e_ != cudaSuccess) return sj::cuda_fail(e_, #x); \
    } while (0)
