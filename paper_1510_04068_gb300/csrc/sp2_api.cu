// sp2_api.cu -- host side of the C ABI declared in include/sapporo_gb.h:
// context and device memory, argument validation, host<->device staging,
// launch-shape selection (heuristic + autotuner cache), CUDA-graph capture and
// per-stage timing.  All arithmetic of the method runs in the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "sapporo_gb.h"
#include "sp2_internal.h"

using namespace sp2;

namespace {

enum Stage { ST_PREDICT = 0, ST_FORCE, ST_REDUCE, ST_BATCHED, ST_VJP, ST_OTHER, ST_COUNT };
constexpr int kEventRing = 4096;
constexpr int kStagesDevice = 3;       // must equal sp2::kStages of sp2_device.cuh
constexpr int kFusedStagesDevice = 2;  // must equal sp2::kFusedStages of sp2_device.cuh
// largest (sinks of one i-block) x (slices) reduced inside the pass kernel
constexpr int64_t kFusedReduceMaxValues = 16384;

}  // namespace

struct sp2_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

struct sp2_batch_plan {
    sp2_ctx *ctx = nullptr;
    int4 *items = nullptr;  // device
    int64_t n_items = 0;
    int64_t out_base = 0;
    int64_t n_rows = 0;
    int64_t max_size = 0;
};

struct sp2_ctx {
    sp2_config cfg{};
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool broken = false;
    bool capturing = false;
    std::string err;

    int rb = 0;       // predicted-record bytes
    JStore js{};
    int64_t n_loaded = 0;
    unsigned char *rec = nullptr;   // predicted records
    bool rec_valid = false;         // sp2_predict has been called since the last sp2_set_j
    bool pred_pending = false;      // mixed: records not yet written for t_pred (written on demand)
    double t_pred = 0.0;
    unsigned char *rec2 = nullptr;  // records of the all-pairs / VJP entry points
    int32_t *iota = nullptr;
    double *tmp = nullptr;          // 4 x (n_max x 3) doubles: a1, j1, xpbar, vpbar
    unsigned int *dev_words = nullptr;  // [0] batched work queue, [1] error flag, [2] finite flag,
                                        // [4] pass work queue, [5] pass exit count (both self-resetting)
    double *part = nullptr;
    int32_t *part_id = nullptr;
    size_t part_cap = 0, part_id_cap = 0;   // bytes
    unsigned int *done = nullptr;           // per-i-block arrival counters of the fused reduction
    size_t done_cap = 0;                    // bytes
    unsigned char *sinkrec = nullptr;       // records of explicit sinks
    int32_t *noslot = nullptr;              // -1 per explicit sink (no self pair)
    size_t sinkrec_cap = 0, noslot_cap = 0;
    double *blk_dt = nullptr;               // block time-steps: per-slot step
    BlockDev *blk_dev = nullptr;            // block time-steps: device-driven run state
    double *blk_cr = nullptr, *blk_s1 = nullptr;  // 6th-order block steps: crackles, new snaps
    size_t blk_cr_cap = 0, blk_s1_cap = 0;
    int32_t *blk_active = nullptr;          // block time-steps: active slots
    size_t blk_dt_cap = 0, blk_active_cap = 0;
    bool blk_ready = false;                 // sp2_block_init has run since the last set_j
    unsigned char *stage = nullptr;  // staging for host-pointer calls
    size_t stage_cap = 0;
    std::vector<void *> owned;       // everything allocated (for close)

    std::map<int64_t, sp2_launch> tuned;  // key: tune_key(n_i, n_j)
    // profiling: per stage a ring of (start, stop) event pairs
    std::vector<cudaEvent_t> ev[ST_COUNT];
    int64_t ev_count[ST_COUNT] = {};
    int64_t launches = 0;
};

namespace {

sp2_status fail(sp2_ctx *c, sp2_status s, const char *fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

sp2_status cuda_fail(sp2_ctx *c, cudaError_t e, const char *what) {
    if (c) c->broken = true;
    return fail(c, SP2_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define SP2_CK(ctx, expr)                                        \
    do {                                                         \
        cudaError_t e_ = (expr);                                 \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #expr); \
    } while (0)

#define SP2_CKS(expr)                \
    do {                             \
        sp2_status s_ = (expr);      \
        if (s_ != SP2_OK) return s_; \
    } while (0)

void *dalloc(sp2_ctx *c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (c->cfg.alloc) {
        p = c->cfg.alloc(bytes, c->cfg.alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) c->owned.push_back(p);
    return p;
}

void dfree(sp2_ctx *c, void *p) {
    if (!p) return;
    auto it = std::find(c->owned.begin(), c->owned.end(), p);
    if (it != c->owned.end()) c->owned.erase(it);
    if (c->cfg.free) c->cfg.free(p, c->cfg.alloc_user);
    else cudaFree(p);
}

sp2_status usable(sp2_ctx *c) {
    if (!c) return SP2_ERR_ARG;
    if (c->broken) return fail(c, SP2_ERR_CUDA, "context unusable after an earlier CUDA error");
    return SP2_OK;
}

void ev_begin(sp2_ctx *c, int st) {
    if (!c->cfg.profile || c->capturing) return;
    std::vector<cudaEvent_t> &r = c->ev[st];
    const size_t k = static_cast<size_t>(c->ev_count[st] % kEventRing);
    while (r.size() < 2 * (k + 1)) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return;
        r.push_back(e0);
        r.push_back(e1);
    }
    cudaEventRecord(r[2 * k], c->stream);
}
void ev_end(sp2_ctx *c, int st) {
    if (!c->cfg.profile || c->capturing) return;
    std::vector<cudaEvent_t> &r = c->ev[st];
    const size_t k = static_cast<size_t>(c->ev_count[st] % kEventRing);
    if (r.size() < 2 * (k + 1)) return;
    cudaEventRecord(r[2 * k + 1], c->stream);
    c->ev_count[st] += 1;
}

// Write the predicted records of a deferred sp2_predict (mixed contexts).
sp2_status materialize(sp2_ctx *c) {
    if (!c->pred_pending) return SP2_OK;
    ev_begin(c, ST_PREDICT);
    SP2_CK(c, launch_predict(c->cfg.order, 1, c->js, c->n_loaded, c->t_pred, c->rec, c->stream));
    ev_end(c, ST_PREDICT);
    c->launches += 1;
    c->pred_pending = false;
    return SP2_OK;
}

// Grow-only device buffer; refused while a graph is being captured.
sp2_status ensure(sp2_ctx *c, void **buf, size_t *cap, size_t need, const char *what) {
    if (need <= *cap) return SP2_OK;
    if (c->capturing)
        return fail(c, SP2_ERR_STATE, "%s scratch (%zu bytes) must be sized by one call before graph capture", what, need);
    size_t n = std::max(need, *cap + *cap / 2);
    SP2_CK(c, cudaStreamSynchronize(c->stream));
    dfree(c, *buf);
    *buf = nullptr;
    *cap = 0;
    void *p = dalloc(c, n);
    if (!p) return fail(c, SP2_ERR_NOMEM, "cannot allocate %zu bytes of %s scratch", n, what);
    *buf = p;
    *cap = n;
    return SP2_OK;
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
int64_t bucket_of(int64_t n_i) {
    int64_t b = 0;
    while ((int64_t(1) << (b + 1)) <= n_i) ++b;
    return b;
}
bool pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }
// autotuner cache key: the power-of-two buckets of the sink and source counts
int64_t tune_key(int64_t n_i, int64_t n_j) { return bucket_of(n_i) * 64 + bucket_of(std::max<int64_t>(n_j, 1)); }

sp2_status check_launch(sp2_ctx *c, const sp2_launch &L) {
    if (!(L.threads == 32 || L.threads == 64 || L.threads == 128 || L.threads == 256))
        return fail(c, SP2_ERR_ARG, "threads must be 32, 64, 128 or 256");
    if (!(L.i_per_thread == 1 || L.i_per_thread == 2 || L.i_per_thread == 4))
        return fail(c, SP2_ERR_ARG, "i_per_thread must be 1, 2 or 4");
    if (!pow2(L.j_lanes) || L.j_lanes > L.threads)
        return fail(c, SP2_ERR_ARG, "j_lanes must be a power of two <= threads");
    if (L.j_tile < 16 || L.j_tile > 1024 || !pow2(L.j_tile) || L.j_tile < 8 * L.j_lanes)
        return fail(c, SP2_ERR_ARG, "j_tile must be a power of two in [16, 1024] and >= 8 * j_lanes");
    if (L.split_j < 1 || L.split_j > 65536) return fail(c, SP2_ERR_ARG, "split_j must be in [1, 65536]");
    if (L.ctas_per_sm < 0 || L.ctas_per_sm > 32) return fail(c, SP2_ERR_ARG, "ctas_per_sm must be in [0, 32]");
    return SP2_OK;
}

// Default launch shape.  Sinks first: when they do not fill one CTA, several
// threads share a sink (j_lanes, the paper's 2D thread blocks) and the CTA
// shrinks; then source slices (the source split) until there are ~4 work
// items per resident CTA, so the dynamic queue balances the SMs.
sp2_launch heuristic(const sp2_ctx *c, int kind, int mixed, int64_t n_i, int64_t n_j) {
    sp2_launch L{};
    L.threads = 256;
    L.i_per_thread = (kind == K_FORCE && mixed) ? 2 : 1;
    L.j_tile = 128;
    L.j_lanes = 1;
    L.ctas_per_sm = 0;
    while (L.j_lanes < 32 && static_cast<int64_t>(L.threads / L.j_lanes) * L.i_per_thread > n_i) {
        L.j_lanes *= 2;
        L.i_per_thread = 1;
    }
    while (L.threads > 32 && L.threads / 2 >= L.j_lanes &&
           static_cast<int64_t>(L.threads / 2 / L.j_lanes) * L.i_per_thread >= n_i)
        L.threads /= 2;
    L.j_tile = std::max(L.j_tile, 8 * L.j_lanes);
    const int64_t sinks_per_cta = static_cast<int64_t>(L.threads / L.j_lanes) * L.i_per_thread;
    const int64_t n_iblk = ceil_div(n_i, sinks_per_cta);
    const int64_t cta_slots = static_cast<int64_t>(c->sm_count) * std::max(1, 512 / L.threads);
    int64_t split = ceil_div(4 * cta_slots, n_iblk);
    const int64_t max_split = std::max<int64_t>(1, n_j / (2 * L.j_tile));
    split = std::max<int64_t>(1, std::min(split, max_split));
    if (n_iblk >= 4 * cta_slots) split = 1;
    L.split_j = static_cast<int>(std::min<int64_t>(split, 65536));
    return L;
}

// Launch one persistent pass (force or VJP policy) plus its reduction.
struct PassOut {
    double *acc = nullptr, *jerk = nullptr, *snap = nullptr, *pot = nullptr;
    int32_t *nn_id = nullptr;
    double *nn_r2 = nullptr;
    double *xbar = nullptr, *vbar = nullptr, *mbar = nullptr;
    int accumulate = 0;
    // explicit sinks (optional): sink i is sink_rec[i]; i_idx then names slots for the self pair
    const unsigned char *sink_rec = nullptr;
    // neighbour lists (optional): squared radii per sink, capacity, counts, lists
    const double *nb_h2 = nullptr;
    int nb_max = 0;
    int32_t *nb_count = nullptr, *nb_list = nullptr;
};

// Dynamic shared memory of a pass launch (the kernel side computes the same):
// the kStages-deep record ring (of double-single cache words when the
// prediction is fused: the pass predicts each tile in shared memory), for the mixed force passes one tile of
// pair records, and for the mixed policies the 8-byte running totals of every
// (thread, sink, field).
size_t pass_smem_bytes(int kind, int order, int mixed, int tile, int rb, int threads, int ipt, int fused = 0,
                       int fused_stages = kFusedStagesDevice) {
    const size_t ring = fused ? static_cast<size_t>(fused_stages) * tile * 16 * dscache_words(order)
                              : static_cast<size_t>(kStagesDevice) * tile * rb;
    const size_t pairs = mixed ? static_cast<size_t>(tile) * rb : 0;  // both mixed policies evaluate source pairs
    const int ns = (kind == K_VJP) ? 7 : (order == 6 ? 10 : (order == 2 ? 4 : 7));
    return ring + pairs + (mixed ? static_cast<size_t>(threads) * ipt * ns * 8 : 0);
}

// rec holds n_valid records; sink slots must lie in [0, n_valid).  With
// allow_fused (the context's own records, mixed precision) a launch whose sinks
// fit one i-block predicts its sources from the double-single cache inside the
// pass (each source is predicted once); otherwise deferred records are written
// first.
sp2_status run_pass(sp2_ctx *c, int kind, int order, int mixed, int nn, const unsigned char *rec, int rb,
                    int64_t n_valid, const int32_t *i_idx, int64_t n_i, int64_t j_begin, int64_t j_end,
                    const PassOut &o, const sp2_launch *forced, int stage_force, float *ms_out = nullptr,
                    bool allow_fused = false, const unsigned int *n_i_dev = nullptr) {
    if (n_i <= 0) return SP2_OK;
    sp2_launch L;
    if (forced) {
        L = *forced;
    } else {
        auto it = (kind == K_FORCE) ? c->tuned.find(tune_key(n_i, j_end - j_begin)) : c->tuned.end();
        L = (it != c->tuned.end()) ? it->second : heuristic(c, kind, mixed, n_i, j_end - j_begin);
    }
    const int nb = (kind == K_FORCE && nn && o.nb_count) ? 1 : 0;
    if (nb) L.i_per_thread = 1;  // neighbour-list kernels take one sink per thread
    const int64_t n_j = j_end - j_begin;
    const int jl = L.j_lanes;
    int tile = L.j_tile;
    const int64_t sinks_per_cta = static_cast<int64_t>(L.threads / jl) * L.i_per_thread;
    const int64_t n_iblk = ceil_div(n_i, sinks_per_cta);
    // n_i_dev: the sink count is chosen on the device (n_i is its bound); the
    // caller has written the records
    const int fused = (!n_i_dev && allow_fused && kind == K_FORCE && mixed && c->js.dsc && n_iblk == 1) ? 1 : 0;
    if (!fused && allow_fused && !n_i_dev) SP2_CKS(materialize(c));
    const int devn = n_i_dev ? 1 : 0;
    if (devn && (kind != K_FORCE || (order != 4 && order != 6) || nn || nb || L.i_per_thread != 1))
        return fail(c, SP2_ERR_UNSUPPORTED, "device-count passes are order-4/6 forces without neighbours");
    KernelKey key{kind, order, mixed, nn, L.i_per_thread, fused, nb, devn};
    int64_t split = std::max<int64_t>(1, std::min<int64_t>(L.split_j, ceil_div(n_j, tile)));
    int64_t slice_len = ceil_div(ceil_div(n_j, split), tile) * tile;
    split = ceil_div(n_j, slice_len);
    const int ns_fields = (kind == K_VJP) ? 7 : (order == 6 ? 10 : (order == 2 ? 4 : 7));
    // fused: two bulk-copy stages when they fit and a slice spans several
    // tiles, else one (the next tile's copy then starts after this one's
    // prediction)
    const bool two_fit = pass_smem_bytes(kind, order, mixed, tile, rb, L.threads, L.i_per_thread, 1, 2) <=
                         static_cast<size_t>(kMaxPassSmem);
    const int fused_stages = (fused && (slice_len <= tile || !two_fit)) ? 1 : kFusedStagesDevice;
    key.fused_stages = fused ? fused_stages : 0;
    key.mw = jl > 32 ? 1 : 0;
    const size_t smem_total = pass_smem_bytes(kind, order, mixed, tile, rb, L.threads, L.i_per_thread, fused,
                                              fused_stages);
    if (smem_total > static_cast<size_t>(kMaxPassSmem))
        return fail(c, SP2_ERR_UNSUPPORTED, "launch shape needs %zu bytes of shared memory (max %d)", smem_total,
                    kMaxPassSmem);
    if ((tile / jl) % 8 != 0) return fail(c, SP2_ERR_ARG, "j_tile / j_lanes must be a multiple of 8");
    if (jl > 32 && (!mixed || L.i_per_thread != 1 || kind != K_FORCE))
        return fail(c, SP2_ERR_UNSUPPORTED,
                    "j_lanes above 32 (several warps per sink) need a mixed-precision force pass and i_per_thread 1");
    int per_sm = L.ctas_per_sm;
    if (per_sm <= 0) {
        SP2_CK(c, force_kernel_occupancy(key, L.threads, tile, &per_sm));
        if (per_sm <= 0) return fail(c, SP2_ERR_UNSUPPORTED, "launch shape does not fit on an SM");
    }
    // a device-count pass may make more work items than the host's bound
    // shows: it takes every resident CTA
    const int64_t resident = static_cast<int64_t>(c->sm_count) * per_sm;
    // Four or more waves of i-blocks: whole waves of them run unsplit (one
    // item over all sources each, outputs written directly; the work queue
    // balances them across the SMs) and only the last, partial wave is split,
    // into as many slices as fill one wave, so partial sums exist for its
    // sinks only.  With fewer waves every i-block is split: a CTA that runs
    // slower than the others (a far L2 partition, a busier SM) then delays
    // the pass by one slice instead of by one whole i-block (measured: 6.8 %
    // at 1.1 waves).
    int64_t n_whole = 0;
    if (!devn && split > 1 && n_iblk >= 4 * resident) {
        n_whole = n_iblk / resident * resident;
        const int64_t rest = n_iblk - n_whole;
        int64_t tail_split = rest > 0 ? std::min<int64_t>(resident / rest, ceil_div(n_j, tile)) : 1;
        if (tail_split > 1 && sinks_per_cta * tail_split <= kFusedReduceMaxValues) {
            slice_len = ceil_div(ceil_div(n_j, tail_split), tile) * tile;
            split = ceil_div(n_j, slice_len);
        } else {
            n_whole = n_iblk;
            split = 1;
            slice_len = n_j;
        }
    }
    const int64_t tail_sink0 = n_whole * sinks_per_cta;
    const int64_t n_part = n_i - tail_sink0;  // sinks with partial rows
    const int64_t n_items = n_whole + (n_iblk - n_whole) * split;
    const int grid = static_cast<int>(devn ? resident : std::min<int64_t>(n_items, resident));
    const int static_items = (!n_i_dev && grid == n_items) ? 1 : 0;  // one wave: CTA b takes item b

    ForceParams p{};
    p.rec = rec;
    p.i_idx = i_idx;
    p.n_i_dev = n_i_dev;
    p.n_i = n_i;
    p.j_begin = j_begin;
    p.j_end = j_end;
    p.slice_len = slice_len;
    p.split = static_cast<int>(split);
    p.jl = jl;
    p.tile = tile;
    p.sinks_per_cta = static_cast<int>(sinks_per_cta);
    p.n_iblk = n_iblk;
    p.n_items = n_items;
    p.n_whole = n_whole;
    p.tail_sink0 = tail_sink0;
    p.queue = c->dev_words + 4;       // self-resetting work counter of the pass kernel
    p.exit_count = c->dev_words + 5;
    p.static_items = static_items;
    p.err = c->dev_words + 1;
    p.n_loaded = n_valid;
    p.eps2 = c->cfg.eps2;
    p.acc = o.acc; p.jerk = o.jerk; p.snap = o.snap; p.pot = o.pot; p.nn_id = o.nn_id; p.nn_r2 = o.nn_r2;
    p.xbar = o.xbar; p.vbar = o.vbar; p.mbar = o.mbar; p.accumulate = o.accumulate;
    p.sink_rec = o.sink_rec;
    if (nb) {
        p.nb_h2 = o.nb_h2;
        p.nb_count = o.nb_count;
        p.nb_list = o.nb_list;
        p.nb_max = o.nb_max;
        SP2_CK(c, cudaMemsetAsync(o.nb_count, 0, static_cast<size_t>(n_i) * sizeof(int32_t), c->stream));
    }
    if (fused) {
        p.fused_stages = fused_stages;
        p.dsc = c->js.dsc;
        p.t_hi = static_cast<float>(c->t_pred);
        p.t_lo = static_cast<float>(c->t_pred - static_cast<double>(p.t_hi));
    }
    const int ns = ns_fields;
    if (split > 1) {
        const size_t need = static_cast<size_t>(ns + (nn ? 1 : 0)) * split * n_part * sizeof(double);
        SP2_CKS(ensure(c, reinterpret_cast<void **>(&c->part), &c->part_cap, need, "partial-sum"));
        if (nn) SP2_CKS(ensure(c, reinterpret_cast<void **>(&c->part_id), &c->part_id_cap,
                               static_cast<size_t>(split) * n_part * sizeof(int32_t), "partial-id"));
        p.part = c->part;
        p.part_id = c->part_id;
        p.sink_major = split >= kWarpReduceMinSplit ? 1 : 0;
        // fuse the reduction into the pass when one CTA's share of it is small
        // (a device-count pass always does; its i-blocks may be as small as
        // threads / 32 sinks)
        if (devn && sinks_per_cta * split > kFusedReduceMaxValues)
            return fail(c, SP2_ERR_UNSUPPORTED, "device-count pass: split too large for the in-pass reduction");
        if (std::min<int64_t>(sinks_per_cta, n_i) * split <= kFusedReduceMaxValues) {
            const int64_t blocks = devn ? ceil_div(n_i, std::max(1, L.threads / 32)) : n_iblk;
            const size_t old_cap = c->done_cap;
            SP2_CKS(ensure(c, reinterpret_cast<void **>(&c->done), &c->done_cap,
                           static_cast<size_t>(blocks) * sizeof(unsigned int), "reduction-counter"));
            if (c->done_cap != old_cap) SP2_CK(c, cudaMemsetAsync(c->done, 0, c->done_cap, c->stream));
            p.fused_reduce = 1;
            p.done = c->done;
        }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms_out) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, c->stream);
    }
    ev_begin(c, stage_force);
    SP2_CK(c, launch_force_kernel(key, p, grid, L.threads, tile, c->stream));
    ev_end(c, stage_force);
    c->launches += 1;
    if (split > 1 && !p.fused_reduce) {
        ReduceParams r{};
        r.part = c->part;
        r.part_id = c->part_id;
        r.n_i = n_i;
        r.split = static_cast<int>(split);
        r.acc = o.acc; r.jerk = o.jerk; r.snap = o.snap; r.pot = o.pot; r.nn_id = o.nn_id; r.nn_r2 = o.nn_r2;
        r.xbar = o.xbar; r.vbar = o.vbar; r.mbar = o.mbar; r.accumulate = o.accumulate;
        ev_begin(c, ST_REDUCE);
        SP2_CK(c, launch_reduce_kernel(key, r, c->stream));
        ev_end(c, ST_REDUCE);
        c->launches += 1;
    }
    if (nb) {
        // slots -> ids, each list sorted by id
        SP2_CK(c, launch_nb_finish(c->js.id, n_i, o.nb_max, o.nb_count, o.nb_list, c->stream));
        c->launches += 1;
    }
    if (ms_out) {
        cudaEventRecord(e1, c->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        SP2_CK(c, e);
        *ms_out = ms;
    }
    return SP2_OK;
}

// Host-pointer staging helpers.
struct Staging {
    sp2_ctx *c;
    size_t off = 0;
    std::vector<std::pair<void *, const void *>> in;     // (device, host)
    std::vector<size_t> in_bytes;
    std::vector<std::pair<void *, void *>> out;          // (host, device)
    std::vector<size_t> out_bytes;
    size_t total = 0;
    void plan(size_t bytes) { total += (bytes + 255) / 256 * 256; }
    template <class T>
    T *slot(size_t bytes) {
        T *p = reinterpret_cast<T *>(c->stage + off);
        off += (bytes + 255) / 256 * 256;
        return p;
    }
};

template <class T>
T *stage_in(Staging &s, const T *host, size_t count) {
    if (!host) return nullptr;
    T *d = s.template slot<T>(count * sizeof(T));
    s.in.push_back({d, host});
    s.in_bytes.push_back(count * sizeof(T));
    return d;
}
template <class T>
T *stage_out(Staging &s, T *host, size_t count) {
    if (!host) return nullptr;
    T *d = s.template slot<T>(count * sizeof(T));
    s.out.push_back({host, d});
    s.out_bytes.push_back(count * sizeof(T));
    return d;
}

sp2_status stage_copy_in(Staging &s) {
    for (size_t k = 0; k < s.in.size(); ++k)
        SP2_CK(s.c, cudaMemcpyAsync(s.in[k].first, s.in[k].second, s.in_bytes[k], cudaMemcpyHostToDevice, s.c->stream));
    return SP2_OK;
}
sp2_status stage_copy_out(Staging &s) {
    for (size_t k = 0; k < s.out.size(); ++k)
        SP2_CK(s.c, cudaMemcpyAsync(s.out[k].first, s.out[k].second, s.out_bytes[k], cudaMemcpyDeviceToHost, s.c->stream));
    SP2_CK(s.c, cudaStreamSynchronize(s.c->stream));
    return SP2_OK;
}

sp2_status check_ptr_kind(sp2_ctx *c, int kind) {
    if (kind != SP2_HOST && kind != SP2_DEVICE) return fail(c, SP2_ERR_ARG, "ptr_kind must be SP2_HOST or SP2_DEVICE");
    if (kind == SP2_HOST && c->capturing) return fail(c, SP2_ERR_STATE, "host pointers are not allowed during graph capture");
    return SP2_OK;
}

sp2_status finite_check(sp2_ctx *c, const double *const *arrs, const int64_t *lens, int n) {
    if (!c->cfg.check_finite || c->capturing) return SP2_OK;
    SP2_CK(c, cudaMemsetAsync(c->dev_words + 2, 0, sizeof(unsigned int), c->stream));
    for (int k = 0; k < n; ++k)
        if (arrs[k]) {
            SP2_CK(c, launch_scan_finite(arrs[k], lens[k], c->dev_words + 2, c->stream));
            c->launches += 1;
        }
    unsigned int flag = 0;
    SP2_CK(c, cudaMemcpyAsync(&flag, c->dev_words + 2, sizeof flag, cudaMemcpyDeviceToHost, c->stream));
    SP2_CK(c, cudaStreamSynchronize(c->stream));
    if (flag) return fail(c, SP2_ERR_NONFINITE, "NaN or Inf in the outputs (coincident particles with eps2 = 0?)");
    return SP2_OK;
}

}  // namespace

namespace sp2 {

cudaError_t launch_force_kernel(const KernelKey &k, const ForceParams &p, int grid, int threads, size_t tile,
                                cudaStream_t s) {
    if (k.kind == K_VJP) return k.mixed ? launch_force_vjpm(k, p, grid, threads, tile, s)
                                        : launch_force_vjpd(k, p, grid, threads, tile, s);
    if (k.order == 6) return k.mixed ? launch_force_h6m(k, p, grid, threads, tile, s)
                                     : launch_force_h6d(k, p, grid, threads, tile, s);
    if (k.order == 2) return k.mixed ? launch_force_h2m(k, p, grid, threads, tile, s)
                                     : launch_force_h2d(k, p, grid, threads, tile, s);
    return k.mixed ? launch_force_h4m(k, p, grid, threads, tile, s) : launch_force_h4d(k, p, grid, threads, tile, s);
}

cudaError_t force_kernel_occupancy(const KernelKey &k, int threads, size_t tile, int *b) {
    if (k.kind == K_VJP) return k.mixed ? occupancy_force_vjpm(k, threads, tile, b) : occupancy_force_vjpd(k, threads, tile, b);
    if (k.order == 6) return k.mixed ? occupancy_force_h6m(k, threads, tile, b) : occupancy_force_h6d(k, threads, tile, b);
    if (k.order == 2) return k.mixed ? occupancy_force_h2m(k, threads, tile, b) : occupancy_force_h2d(k, threads, tile, b);
    return k.mixed ? occupancy_force_h4m(k, threads, tile, b) : occupancy_force_h4d(k, threads, tile, b);
}

cudaError_t launch_reduce_kernel(const KernelKey &k, const ReduceParams &r, cudaStream_t s) {
    if (k.kind == K_VJP) return k.mixed ? launch_reduce_vjpm(k, r, s) : launch_reduce_vjpd(k, r, s);
    if (k.order == 6) return k.mixed ? launch_reduce_h6m(k, r, s) : launch_reduce_h6d(k, r, s);
    if (k.order == 2) return k.mixed ? launch_reduce_h2m(k, r, s) : launch_reduce_h2d(k, r, s);
    return k.mixed ? launch_reduce_h4m(k, r, s) : launch_reduce_h4d(k, r, s);
}

cudaError_t launch_batched_kernel(int order, int mixed, int nn, const BatchParams &b, int grid, int threads,
                                  cudaStream_t s) {
    if (order == 6) return mixed ? launch_batched_h6m(nn, b, grid, threads, s) : launch_batched_h6d(nn, b, grid, threads, s);
    if (order == 2) return mixed ? launch_batched_h2m(nn, b, grid, threads, s) : launch_batched_h2d(nn, b, grid, threads, s);
    return mixed ? launch_batched_h4m(nn, b, grid, threads, s) : launch_batched_h4d(nn, b, grid, threads, s);
}

cudaError_t batched_kernel_occupancy(int order, int mixed, int nn, int threads, int *b) {
    if (order == 6) return mixed ? occupancy_batched_h6m(nn, threads, b) : occupancy_batched_h6d(nn, threads, b);
    if (order == 2) return mixed ? occupancy_batched_h2m(nn, threads, b) : occupancy_batched_h2d(nn, threads, b);
    return mixed ? occupancy_batched_h4m(nn, threads, b) : occupancy_batched_h4d(nn, threads, b);
}

}  // namespace sp2

extern "C" {

void sp2_config_default(sp2_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->order = 4;
    cfg->precision = SP2_MIXED;
    cfg->with_nn = 1;
}

const char *sp2_strerror(sp2_status s) {
    switch (s) {
        case SP2_OK: return "ok";
        case SP2_ERR_ARG: return "invalid argument";
        case SP2_ERR_RANGE: return "size or index out of range";
        case SP2_ERR_NOMEM: return "device allocation failed";
        case SP2_ERR_CUDA: return "CUDA error";
        case SP2_ERR_STATE: return "call out of order";
        case SP2_ERR_TIMEOUT: return "device-side wait timed out";
        case SP2_ERR_NONFINITE: return "non-finite output";
        case SP2_ERR_UNSUPPORTED: return "unsupported option";
    }
    return "unknown status";
}

sp2_status sp2_last_error(const sp2_ctx *ctx, char *buf, size_t len) {
    if (!ctx || !buf || len == 0) return SP2_ERR_ARG;
    std::snprintf(buf, len, "%s", ctx->err.c_str());
    return SP2_OK;
}

sp2_status sp2_open(sp2_ctx **out, const sp2_config *cfg) {
    if (!out || !cfg) return SP2_ERR_ARG;
    *out = nullptr;
    if (cfg->order != 2 && cfg->order != 4 && cfg->order != 6) return SP2_ERR_ARG;
    if (cfg->precision != SP2_FP64 && cfg->precision != SP2_MIXED) return SP2_ERR_ARG;
    if (cfg->n_max <= 0 || cfg->n_max > (int64_t(1) << 30)) return SP2_ERR_ARG;
    if (!(cfg->eps2 >= 0.0) || !std::isfinite(cfg->eps2)) return SP2_ERR_ARG;
    if ((cfg->alloc == nullptr) != (cfg->free == nullptr)) return SP2_ERR_ARG;
    if (cfg->with_nn != 0 && cfg->with_nn != 1) return SP2_ERR_ARG;

    sp2_ctx *c = new sp2_ctx();
    c->cfg = *cfg;
    const int mixed = cfg->precision == SP2_MIXED;
    c->rb = record_bytes(cfg->order, mixed);
    const size_t n = static_cast<size_t>(cfg->n_max);
    const size_t n3 = 3 * n * sizeof(double);
    // every allocation goes through the (optional) allocator before any other CUDA call
    c->js.id = static_cast<int32_t *>(dalloc(c, n * sizeof(int32_t)));
    c->js.m = static_cast<double *>(dalloc(c, n * sizeof(double)));
    c->js.t = static_cast<double *>(dalloc(c, n * sizeof(double)));
    c->js.x = static_cast<double *>(dalloc(c, n3));
    c->js.v = static_cast<double *>(dalloc(c, n3));
    c->js.a = static_cast<double *>(dalloc(c, n3));
    c->js.jk = static_cast<double *>(dalloc(c, n3));
    c->js.sn = cfg->order == 6 ? static_cast<double *>(dalloc(c, n3)) : nullptr;
    c->js.dsc = mixed ? static_cast<float4 *>(dalloc(c, n * dscache_words(cfg->order) * sizeof(float4))) : nullptr;
    c->rec = static_cast<unsigned char *>(dalloc(c, n * c->rb));
    c->rec2 = static_cast<unsigned char *>(dalloc(c, n * std::max(vjp_record_bytes(0), vjp_record_bytes(1))));
    c->iota = static_cast<int32_t *>(dalloc(c, n * sizeof(int32_t)));
    c->tmp = static_cast<double *>(dalloc(c, 4 * n3));
    c->dev_words = static_cast<unsigned int *>(dalloc(c, 64));
    const bool ok = c->js.id && c->js.m && c->js.t && c->js.x && c->js.v && c->js.a && c->js.jk &&
                    (cfg->order != 6 || c->js.sn) && (!mixed || c->js.dsc) && c->rec && c->rec2 && c->iota &&
                    c->tmp && c->dev_words;
    if (!ok) {
        while (!c->owned.empty()) dfree(c, c->owned.back());
        delete c;
        return SP2_ERR_NOMEM;
    }
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) {
        if (cfg->cuda_stream) {
            c->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
        } else {
            e = cudaStreamCreate(&c->stream);
            c->own_stream = (e == cudaSuccess);
        }
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(c->dev_words, 0, 64, c->stream);
    if (cfg->order == 2) {  // velocities, accelerations, jerks and times are optional inputs
        for (double *q : {c->js.v, c->js.a, c->js.jk})
            if (e == cudaSuccess) e = cudaMemsetAsync(q, 0, n3, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->js.t, 0, n * sizeof(double), c->stream);
    }
    if (e == cudaSuccess) e = launch_iota(c->iota, cfg->n_max, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        sp2_close(c);
        return SP2_ERR_CUDA;
    }
    c->launches = 1;
    *out = c;
    return SP2_OK;
}

sp2_status sp2_close(sp2_ctx *c) {
    if (!c) return SP2_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    while (!c->owned.empty()) dfree(c, c->owned.back());
    for (int s = 0; s < ST_COUNT; ++s)
        for (cudaEvent_t e : c->ev[s]) cudaEventDestroy(e);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return SP2_OK;
}

sp2_status sp2_info(const sp2_ctx *c, int64_t *n_loaded, int64_t *n_max, int *sm_count) {
    if (!c) return SP2_ERR_ARG;
    if (n_loaded) *n_loaded = c->n_loaded;
    if (n_max) *n_max = c->cfg.n_max;
    if (sm_count) *sm_count = c->sm_count;
    return SP2_OK;
}

int64_t sp2_kernel_launches(const sp2_ctx *c) { return c ? c->launches : -1; }

sp2_status sp2_set_j(sp2_ctx *c, int64_t first, int64_t n, const int32_t *slots, const int32_t *id, const double *m,
                     const double *x, const double *v, const double *a, const double *jerk, const double *snap,
                     const double *t, int ptr_kind) {
    SP2_CKS(usable(c));
    SP2_CKS(check_ptr_kind(c, ptr_kind));
    if (n < 0) return fail(c, SP2_ERR_ARG, "n < 0");
    if (n == 0) return SP2_OK;
    if (!id || !m || !x) return fail(c, SP2_ERR_ARG, "null input array");
    c->blk_ready = false;
    if (c->cfg.order != 2 && (!v || !a || !jerk || !t)) return fail(c, SP2_ERR_ARG, "null input array");
    if (c->cfg.order == 6 && !snap) return fail(c, SP2_ERR_ARG, "order 6 needs snap");
    if (c->cfg.order != 6 && snap) return fail(c, SP2_ERR_ARG, "snap must be NULL below order 6");
    if (!slots) {
        if (first < 0 || first + n > c->cfg.n_max) return fail(c, SP2_ERR_RANGE, "slots [%lld, %lld) exceed n_max %lld",
                                                                 (long long)first, (long long)(first + n), (long long)c->cfg.n_max);
        if (first > c->n_loaded)
            return fail(c, SP2_ERR_RANGE, "first slot %lld would leave slots [%lld, %lld) unloaded", (long long)first,
                        (long long)c->n_loaded, (long long)first);
    } else {
        if (n > c->n_loaded) return fail(c, SP2_ERR_RANGE, "more slots than loaded particles");
        if (ptr_kind == SP2_HOST)
            for (int64_t k = 0; k < n; ++k)
                if (slots[k] < 0 || slots[k] >= c->n_loaded)
                    return fail(c, SP2_ERR_RANGE, "slot %d outside the loaded set [0, %lld)", slots[k], (long long)c->n_loaded);
    }
    const size_t n3 = 3 * static_cast<size_t>(n) * sizeof(double);
    if (ptr_kind == SP2_HOST) {
        if (!slots) {
            const size_t o = static_cast<size_t>(first);
            SP2_CK(c, cudaMemcpyAsync(c->js.id + o, id, n * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
            SP2_CK(c, cudaMemcpyAsync(c->js.m + o, m, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
            if (t) SP2_CK(c, cudaMemcpyAsync(c->js.t + o, t, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
            SP2_CK(c, cudaMemcpyAsync(c->js.x + 3 * o, x, n3, cudaMemcpyHostToDevice, c->stream));
            if (v) SP2_CK(c, cudaMemcpyAsync(c->js.v + 3 * o, v, n3, cudaMemcpyHostToDevice, c->stream));
            if (a) SP2_CK(c, cudaMemcpyAsync(c->js.a + 3 * o, a, n3, cudaMemcpyHostToDevice, c->stream));
            if (jerk) SP2_CK(c, cudaMemcpyAsync(c->js.jk + 3 * o, jerk, n3, cudaMemcpyHostToDevice, c->stream));
            if (snap) SP2_CK(c, cudaMemcpyAsync(c->js.sn + 3 * o, snap, n3, cudaMemcpyHostToDevice, c->stream));
            if (c->js.dsc) {
                ev_begin(c, ST_OTHER);
                SP2_CK(c, launch_dscache(c->cfg.order, c->js, first, n, c->stream));
                ev_end(c, ST_OTHER);
                c->launches += 1;
            }
            SP2_CK(c, cudaStreamSynchronize(c->stream));
        } else {
            Staging s{c};
            s.plan(n * sizeof(int32_t)); s.plan(n * sizeof(int32_t)); s.plan(2 * n * sizeof(double));
            s.plan(n3); s.plan(n3); s.plan(n3); s.plan(n3); if (snap) s.plan(n3);
            SP2_CKS(ensure(c, reinterpret_cast<void **>(&c->stage), &c->stage_cap, s.total, "staging"));
            const int32_t *dsl = stage_in(s, slots, n);
            const int32_t *did = stage_in(s, id, n);
            const double *dm = stage_in(s, m, n), *dt = stage_in(s, t, n);
            const double *dx = stage_in(s, x, 3 * n), *dv = stage_in(s, v, 3 * n), *da = stage_in(s, a, 3 * n);
            const double *dj = stage_in(s, jerk, 3 * n), *ds = stage_in(s, snap, 3 * n);
            SP2_CKS(stage_copy_in(s));
            ev_begin(c, ST_OTHER);
            SP2_CK(c, launch_scatter_j(c->js, dsl, n, c->n_loaded, c->dev_words + 1, did, dm, dx, dv, da, dj, ds, dt, c->stream));
            ev_end(c, ST_OTHER);
            c->launches += 1;
            SP2_CK(c, cudaStreamSynchronize(c->stream));
        }
    } else {
        if (!slots) {
            const size_t o = static_cast<size_t>(first);
            SP2_CK(c, cudaMemcpyAsync(c->js.id + o, id, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream));
            SP2_CK(c, cudaMemcpyAsync(c->js.m + o, m, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
            if (t) SP2_CK(c, cudaMemcpyAsync(c->js.t + o, t, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
            SP2_CK(c, cudaMemcpyAsync(c->js.x + 3 * o, x, n3, cudaMemcpyDeviceToDevice, c->stream));
            if (v) SP2_CK(c, cudaMemcpyAsync(c->js.v + 3 * o, v, n3, cudaMemcpyDeviceToDevice, c->stream));
            if (a) SP2_CK(c, cudaMemcpyAsync(c->js.a + 3 * o, a, n3, cudaMemcpyDeviceToDevice, c->stream));
            if (jerk) SP2_CK(c, cudaMemcpyAsync(c->js.jk + 3 * o, jerk, n3, cudaMemcpyDeviceToDevice, c->stream));
            if (snap) SP2_CK(c, cudaMemcpyAsync(c->js.sn + 3 * o, snap, n3, cudaMemcpyDeviceToDevice, c->stream));
            if (c->js.dsc) {
                ev_begin(c, ST_OTHER);
                SP2_CK(c, launch_dscache(c->cfg.order, c->js, first, n, c->stream));
                ev_end(c, ST_OTHER);
                c->launches += 1;
            }
        } else {
            ev_begin(c, ST_OTHER);
            SP2_CK(c, launch_scatter_j(c->js, slots, n, c->n_loaded, c->dev_words + 1, id, m, x, v, a, jerk, snap, t, c->stream));
            ev_end(c, ST_OTHER);
            c->launches += 1;
        }
    }
    if (!slots) c->n_loaded = std::max(c->n_loaded, first + n);
    c->rec_valid = false;
    c->pred_pending = false;
    return SP2_OK;
}

sp2_status sp2_predict(sp2_ctx *c, double t) {
    SP2_CKS(usable(c));
    if (!std::isfinite(t)) return fail(c, SP2_ERR_ARG, "t is not finite");
    if (c->n_loaded == 0) return fail(c, SP2_ERR_STATE, "no j-particles loaded");
    c->t_pred = t;
    if (c->js.dsc) {  // mixed: records are written on demand, or predicted inside the pass
        c->pred_pending = true;
        c->rec_valid = true;
        return SP2_OK;
    }
    ev_begin(c, ST_PREDICT);
    SP2_CK(c, launch_predict(c->cfg.order, c->cfg.precision == SP2_MIXED, c->js, c->n_loaded, t, c->rec, c->stream));
    ev_end(c, ST_PREDICT);
    c->launches += 1;
    c->rec_valid = true;
    return SP2_OK;
}

// sp2_compute_range / sp2_compute_nb: the force pass over sources [j_begin, j_end),
// with neighbour lists when h2 is given.
static sp2_status compute_impl(sp2_ctx *c, int64_t j_begin, int64_t j_end, int64_t n_i, const int32_t *i_idx,
                               double *acc, double *jerk, double *snap, double *pot, int32_t *nn_id, double *nn_r2,
                               const double *h2, int32_t nb_max, int32_t *nb_count, int32_t *nb_ids, int ptr_kind) {
    SP2_CKS(usable(c));
    SP2_CKS(check_ptr_kind(c, ptr_kind));
    if (n_i < 0) return fail(c, SP2_ERR_ARG, "n_i < 0");
    if (n_i == 0) return SP2_OK;
    if (!i_idx) return fail(c, SP2_ERR_ARG, "i_idx is NULL");
    if (!c->rec_valid) return fail(c, SP2_ERR_STATE, "predicted records are stale: call sp2_predict first");
    if (j_begin < 0 || j_end > c->n_loaded || j_begin >= j_end)
        return fail(c, SP2_ERR_RANGE, "source range [%lld, %lld) outside the loaded set [0, %lld)", (long long)j_begin,
                    (long long)j_end, (long long)c->n_loaded);
    if (n_i > (int64_t(1) << 30)) return fail(c, SP2_ERR_RANGE, "n_i too large");
    if (snap && c->cfg.order != 6) return fail(c, SP2_ERR_ARG, "snap requested from a context below order 6");
    if (jerk && c->cfg.order == 2) return fail(c, SP2_ERR_ARG, "jerk requested from an order-2 (leap-frog) context");
    if ((nn_id || nn_r2) && !c->cfg.with_nn) return fail(c, SP2_ERR_UNSUPPORTED, "context opened without nearest neighbour");
    const bool want_nb = h2 || nb_count || nb_ids;
    if (want_nb) {
        if (!h2 || !nb_count || !nb_ids) return fail(c, SP2_ERR_ARG, "neighbour lists need h2, nb_count and nb_ids");
        if (nb_max <= 0 || nb_max > 4096) return fail(c, SP2_ERR_ARG, "nb_max must be in [1, 4096]");
        if (!c->cfg.with_nn) return fail(c, SP2_ERR_UNSUPPORTED, "neighbour lists need a context with nearest neighbour");
        if (static_cast<double>(n_i) * nb_max > 2e9) return fail(c, SP2_ERR_RANGE, "n_i * nb_max too large");
    }
    const int mixed = c->cfg.precision == SP2_MIXED;
    PassOut o;
    Staging s{c};
    const int32_t *d_idx = i_idx;
    if (ptr_kind == SP2_HOST) {
        for (int64_t k = 0; k < n_i; ++k)
            if (i_idx[k] < 0 || i_idx[k] >= c->n_loaded)
                return fail(c, SP2_ERR_RANGE, "sink slot %d outside the loaded set", i_idx[k]);
        const size_t v3 = 3 * n_i * sizeof(double), v1 = n_i * sizeof(double);
        s.plan(n_i * 4); s.plan(v3); s.plan(v3); s.plan(v3); s.plan(v1); s.plan(n_i * 4); s.plan(v1);
        if (want_nb) { s.plan(v1); s.plan(n_i * 4); s.plan(static_cast<size_t>(n_i) * nb_max * 4); }
        SP2_CKS(ensure(c, reinterpret_cast<void **>(&c->stage), &c->stage_cap, s.total, "staging"));
        d_idx = stage_in(s, i_idx, n_i);
        o.acc = stage_out(s, acc, 3 * n_i);
        o.jerk = stage_out(s, jerk, 3 * n_i);
        o.snap = stage_out(s, snap, 3 * n_i);
        o.pot = stage_out(s, pot, n_i);
        o.nn_id = stage_out(s, nn_id, n_i);
        o.nn_r2 = stage_out(s, nn_r2, n_i);
        if (want_nb) {
            o.nb_h2 = stage_in(s, h2, n_i);
            o.nb_count = stage_out(s, nb_count, n_i);
            o.nb_list = stage_out(s, nb_ids, static_cast<size_t>(n_i) * nb_max);
        }
        SP2_CKS(stage_copy_in(s));
    } else {
        o.acc = acc; o.jerk = jerk; o.snap = snap; o.pot = pot; o.nn_id = nn_id; o.nn_r2 = nn_r2;
        o.nb_h2 = h2; o.nb_count = nb_count; o.nb_list = nb_ids;
    }
    o.nb_max = nb_max;
    // the neighbour-list kernels are the nearest-neighbour kernels with lists
    const int nn = c->cfg.with_nn && (o.nn_id || o.nn_r2 || want_nb);
    SP2_CKS(run_pass(c, K_FORCE, c->cfg.order, mixed, nn, c->rec, c->rb, c->n_loaded, d_idx, n_i, j_begin, j_end, o,
                     nullptr, ST_FORCE, nullptr, true));
    const double *arrs[4] = {o.acc, o.jerk, o.snap, o.pot};
    const int64_t lens[4] = {3 * n_i, 3 * n_i, 3 * n_i, n_i};
    SP2_CKS(finite_check(c, arrs, lens, 4));
    if (ptr_kind == SP2_HOST) SP2_CKS(stage_copy_out(s));
    return SP2_OK;
}

sp2_status sp2_compute_range(sp2_ctx *c, int64_t j_begin, int64_t j_end, int64_t n_i, const int32_t *i_idx,
                             double *acc, double *jerk, double *snap, double *pot, int32_t *nn_id, double *nn_r2,
                             int ptr_kind) {
    return compute_impl(c, j_begin, j_end, n_i, i_idx, acc, jerk, snap, pot, nn_id, nn_r2, nullptr, 0, nullptr,
                        nullptr, ptr_kind);
}

sp2_status sp2_compute(sp2_ctx *c, int64_t n_i, const int32_t *i_idx, double *acc, double *jerk, double *snap,
                       double *pot, int32_t *nn_id, double *nn_r2, int ptr_kind) {
    SP2_CKS(usable(c));
    if (c->n_loaded == 0) return fail(c, SP2_ERR_STATE, "no j-particles loaded");
    return sp2_compute_range(c, 0, c->n_loaded, n_i, i_idx, acc, jerk, snap, pot, nn_id, nn_r2, ptr_kind);
}

sp2_status sp2_compute_ext(sp2_ctx *c, int64_t n_i, const int32_t *i_slot, const double *xi, const double *vi,
                           const double *ai, double *acc, double *jerk, double *snap, double *pot, int32_t *nn_id,
                           double *nn_r2, int ptr_kind) {
    SP2_CKS(usable(c));
    SP2_CKS(check_ptr_kind(c, ptr_kind));
    if (n_i < 0) return fail(c, SP2_ERR_ARG, "n_i < 0");
    if (n_i == 0) return SP2_OK;
    if (c->n_loaded == 0) return fail(c, SP2_ERR_STATE, "no j-particles loaded");
    if (!c->rec_valid) return fail(c, SP2_ERR_STATE, "predicted records are stale: call sp2_predict first");
    if (n_i > (int64_t(1) << 30)) return fail(c, SP2_ERR_RANGE, "n_i too large");
    const int order = c->cfg.order;
    if (!xi || (order != 2 && !vi) || (order == 6 && !ai))
        return fail(c, SP2_ERR_ARG, "explicit sinks need x, v (orders 4, 6) and a (order 6)");
    if (snap && order != 6) return fail(c, SP2_ERR_ARG, "snap requested from a context below order 6");
    if (jerk && order == 2) return fail(c, SP2_ERR_ARG, "jerk requested from an order-2 (leap-frog) context");
    if ((nn_id || nn_r2) && !c->cfg.with_nn) return fail(c, SP2_ERR_UNSUPPORTED, "context opened without nearest neighbour");
    const int mixed = c->cfg.precision == SP2_MIXED;
    PassOut o;
    Staging s{c};
    const int32_t *d_slot = i_slot;
    if (ptr_kind == SP2_HOST) {
        if (i_slot)
            for (int64_t k = 0; k < n_i; ++k)
                if (i_slot[k] >= c->n_loaded) return fail(c, SP2_ERR_RANGE, "slot %d outside the loaded set", i_slot[k]);
        const size_t v3 = 3 * n_i * sizeof(double), v1 = n_i * sizeof(double);
        s.plan(n_i * 4); s.plan(v3); s.plan(v3); s.plan(v3);
        s.plan(v3); s.plan(v3); s.plan(v3); s.plan(v1); s.plan(n_i * 4); s.plan(v1);
        SP2_CKS(ensure(c, reinterpret_cast<void **>(&c->stage), &c->stage_cap, s.total, "staging"));
        d_slot = stage_in(s, i_slot, n_i);
        xi = stage_in(s, xi, 3 * n_i);
        vi = stage_in(s, vi, 3 * n_i);
        ai = stage_in(s, ai, 3 * n_i);
        o.acc = stage_out(s, acc, 3 * n_i);
        o.jerk = stage_out(s, jerk, 3 * n_i);
        o.snap = stage_out(s, snap, 3 * n_i);
        o.pot = stage_out(s, pot, n_i);
        o.nn_id = stage_out(s, nn_id, n_i);
        o.nn_r2 = stage_out(s, nn_r2, n_i);
        SP2_CKS(stage_copy_in(s));
    } else {
        o.acc = acc; o.jerk = jerk; o.snap = snap; o.pot = pot; o.nn_id = nn_id; o.nn_r2 = nn_r2;
    }
    if (!d_slot) {
        SP2_CKS(ensure(c, reinterpret_cast<void **>(&c->noslot), &c->noslot_cap, n_i * sizeof(int32_t), "sink-slot"));
        SP2_CK(c, cudaMemsetAsync(c->noslot, 0xff, n_i * sizeof(int32_t), c->stream));
        d_slot = c->noslot;
    }
    SP2_CKS(ensure(c, reinterpret_cast<void **>(&c->sinkrec), &c->sinkrec_cap, n_i * c->rb, "sink-record"));
    SP2_CK(c, launch_pack_sinks(order, mixed, n_i, xi, vi, ai, c->sinkrec, c->stream));
    c->launches += 1;
    o.sink_rec = c->sinkrec;
    const int nn = c->cfg.with_nn && (o.nn_id || o.nn_r2);
    SP2_CKS(run_pass(c, K_FORCE, order, mixed, nn, c->rec, c->rb, c->n_loaded, d_slot, n_i, 0, c->n_loaded, o,
                     nullptr, ST_FORCE, nullptr, true));
    const double *arrs[4] = {o.acc, o.jerk, o.snap, o.pot};
    const int64_t lens[4] = {3 * n_i, 3 * n_i, 3 * n_i, n_i};
    SP2_CKS(finite_check(c, arrs, lens, 4));
    if (ptr_kind == SP2_HOST) SP2_CKS(stage_copy_out(s));
    return SP2_OK;
}

sp2_status sp2_compute_nb(sp2_ctx *c, int64_t n_i, const int32_t *i_idx, double *acc, double *jerk, double *snap,
                          double *pot, int32_t *nn_id, double *nn_r2, const double *h2, int32_t nb_max,
                          int32_t *nb_count, int32_t *nb_ids, int ptr_kind) {
    SP2_CKS(usable(c));
    if (c->n_loaded == 0) return fail(c, SP2_ERR_STATE, "no j-particles loaded");
    if (!h2 || !nb_count || !nb_ids) return fail(c, SP2_ERR_ARG, "neighbour lists need h2, nb_count and nb_ids");
    return compute_impl(c, 0, c->n_loaded, n_i, i_idx, acc, jerk, snap, pot, nn_id, nn_r2, h2, nb_max, nb_count,
                        nb_ids, ptr_kind);
}

sp2_status sp2_batch_plan_create(sp2_ctx *c, int64_t n_sys, const int64_t *offsets, sp2_batch_plan **plan) {
    SP2_CKS(usable(c));
    if (!plan || !offsets || n_sys <= 0) return fail(c, SP2_ERR_ARG, "bad batch plan arguments");
    *plan = nullptr;
    if (c->capturing) return fail(c, SP2_ERR_STATE, "cannot build a plan during graph capture");
    struct Item { int4 v; int64_t cost; };
    std::vector<Item> items;
    int64_t max_size = 0;
    for (int64_t s = 0; s < n_sys; ++s) {
        const int64_t a = offsets[s], b = offsets[s + 1];
        if (a < 0 || b < a || b > c->n_loaded) return fail(c, SP2_ERR_RANGE, "system %lld outside the loaded set", (long long)s);
        const int64_t sz = b - a;
        if (sz > 4096) return fail(c, SP2_ERR_RANGE, "system %lld has %lld > 4096 particles", (long long)s, (long long)sz);
        max_size = std::max(max_size, sz);
        for (int64_t q = a; q < b; q += 32) {
            const int64_t cn = std::min<int64_t>(32, b - q);
            items.push_back({make_int4(int(a), int(sz), int(q), int(cn)), sz * 32});
        }
    }
    // largest items first (longest-processing-time order for the dynamic queue)
    std::stable_sort(items.begin(), items.end(), [](const Item &x, const Item &y) { return x.cost > y.cost; });
    std::vector<int4> host(items.size());
    for (size_t k = 0; k < items.size(); ++k) host[k] = items[k].v;
    sp2_batch_plan *p = new sp2_batch_plan();
    p->ctx = c;
    p->n_items = static_cast<int64_t>(host.size());
    p->out_base = offsets[0];
    p->n_rows = offsets[n_sys] - offsets[0];
    p->max_size = max_size;
    if (!host.empty()) {
        p->items = static_cast<int4 *>(dalloc(c, host.size() * sizeof(int4)));
        if (!p->items) {
            delete p;
            return fail(c, SP2_ERR_NOMEM, "cannot allocate the batch plan");
        }
        cudaError_t e = cudaMemcpyAsync(p->items, host.data(), host.size() * sizeof(int4), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            dfree(c, p->items);
            delete p;
            return cuda_fail(c, e, "batch plan upload");
        }
    }
    *plan = p;
    return SP2_OK;
}

sp2_status sp2_batch_plan_destroy(sp2_batch_plan *p) {
    if (!p) return SP2_OK;
    if (p->items) {
        cudaStreamSynchronize(p->ctx->stream);
        dfree(p->ctx, p->items);
    }
    delete p;
    return SP2_OK;
}

sp2_status sp2_compute_batched(sp2_ctx *c, const sp2_batch_plan *plan, double *acc, double *jerk, double *snap,
                               double *pot, int32_t *nn_id, double *nn_r2, int ptr_kind) {
    SP2_CKS(usable(c));
    SP2_CKS(check_ptr_kind(c, ptr_kind));
    if (!plan || plan->ctx != c) return fail(c, SP2_ERR_ARG, "plan does not belong to this context");
    if (!c->rec_valid) return fail(c, SP2_ERR_STATE, "predicted records are stale: call sp2_predict first");
    if (snap && c->cfg.order != 6) return fail(c, SP2_ERR_ARG, "snap requested from a context below order 6");
    if (jerk && c->cfg.order == 2) return fail(c, SP2_ERR_ARG, "jerk requested from an order-2 (leap-frog) context");
    if ((nn_id || nn_r2) && !c->cfg.with_nn) return fail(c, SP2_ERR_UNSUPPORTED, "context opened without nearest neighbour");
    if (plan->n_items == 0) return SP2_OK;
    if (plan->out_base + plan->n_rows > c->n_loaded) return fail(c, SP2_ERR_RANGE, "plan exceeds the loaded set");
    const int64_t n = plan->n_rows;
    Staging s{c};
    BatchParams b{};
    if (ptr_kind == SP2_HOST) {
        const size_t v3 = 3 * n * sizeof(double), v1 = n * sizeof(double);
        s.plan(v3); s.plan(v3); s.plan(v3); s.plan(v1); s.plan(n * 4); s.plan(v1);
        SP2_CKS(ensure(c, reinterpret_cast<void **>(&c->stage), &c->stage_cap, s.total, "staging"));
        b.acc = stage_out(s, acc, 3 * n); b.jerk = stage_out(s, jerk, 3 * n); b.snap = stage_out(s, snap, 3 * n);
        b.pot = stage_out(s, pot, n); b.nn_id = stage_out(s, nn_id, n); b.nn_r2 = stage_out(s, nn_r2, n);
    } else {
        b.acc = acc; b.jerk = jerk; b.snap = snap; b.pot = pot; b.nn_id = nn_id; b.nn_r2 = nn_r2;
    }
    const int mixed = c->cfg.precision == SP2_MIXED;
    const int nn = c->cfg.with_nn && (b.nn_id || b.nn_r2);
    SP2_CKS(materialize(c));
    b.rec = c->rec;
    b.items = plan->items;
    b.n_items = plan->n_items;
    b.out_base = plan->out_base;
    b.queue = c->dev_words;
    b.eps2 = c->cfg.eps2;
    const int threads = 256;
    int per_sm = 0;
    SP2_CK(c, batched_kernel_occupancy(c->cfg.order, mixed, nn, threads, &per_sm));
    const int64_t warps_needed = plan->n_items;
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ceil_div(warps_needed, threads / 32),
                                                                             static_cast<int64_t>(c->sm_count) * std::max(per_sm, 1))));
    SP2_CK(c, cudaMemsetAsync(c->dev_words, 0, sizeof(unsigned int), c->stream));
    ev_begin(c, ST_BATCHED);
    SP2_CK(c, launch_batched_kernel(c->cfg.order, mixed, nn, b, grid, threads, c->stream));
    ev_end(c, ST_BATCHED);
    c->launches += 1;
    const double *arrs[4] = {b.acc, b.jerk, b.snap, b.pot};
    const int64_t lens[4] = {3 * n, 3 * n, 3 * n, n};
    SP2_CKS(finite_check(c, arrs, lens, 4));
    if (ptr_kind == SP2_HOST) SP2_CKS(stage_copy_out(s));
    return SP2_OK;
}

sp2_status sp2_forces(sp2_ctx *c, int64_t n, const double *m, const double *x, const double *v, double *acc,
                      double *jerk, double *pot, int ptr_kind) {
    SP2_CKS(usable(c));
    SP2_CKS(check_ptr_kind(c, ptr_kind));
    if (n < 0) return fail(c, SP2_ERR_ARG, "n < 0");
    if (n == 0) return SP2_OK;
    if (n > c->cfg.n_max) return fail(c, SP2_ERR_RANGE, "n > n_max");
    if (!m || !x || !v) return fail(c, SP2_ERR_ARG, "null input");
    const int mixed = c->cfg.precision == SP2_MIXED;
    Staging s{c};
    PassOut o;
    if (ptr_kind == SP2_HOST) {
        const size_t v3 = 3 * n * sizeof(double), v1 = n * sizeof(double);
        s.plan(v1); s.plan(v3); s.plan(v3); s.plan(v3); s.plan(v3); s.plan(v1);
        SP2_CKS(ensure(c, reinterpret_cast<void **>(&c->stage), &c->stage_cap, s.total, "staging"));
        m = stage_in(s, m, n); x = stage_in(s, x, 3 * n); v = stage_in(s, v, 3 * n);
        o.acc = stage_out(s, acc, 3 * n); o.jerk = stage_out(s, jerk, 3 * n); o.pot = stage_out(s, pot, n);
        SP2_CKS(stage_copy_in(s));
    } else {
        o.acc = acc; o.jerk = jerk; o.pot = pot;
    }
    SP2_CK(c, launch_pack_state(mixed, n, m, x, v, c->rec2, c->stream));
    c->launches += 1;
    SP2_CKS(run_pass(c, K_FORCE, 4, mixed, 0, c->rec2, record_bytes(4, mixed), n, c->iota, n, 0, n, o, nullptr, ST_FORCE));
    if (ptr_kind == SP2_HOST) SP2_CKS(stage_copy_out(s));
    return SP2_OK;
}

sp2_status sp2_force_vjp(sp2_ctx *c, int64_t n, const double *m, const double *x, const double *v,
                         const double *abar, const double *jbar, const double *pbar, double *xbar, double *vbar,
                         double *mbar, int accumulate, int ptr_kind) {
    SP2_CKS(usable(c));
    SP2_CKS(check_ptr_kind(c, ptr_kind));
    if (n < 0) return fail(c, SP2_ERR_ARG, "n < 0");
    if (n == 0) return SP2_OK;
    if (n > c->cfg.n_max) return fail(c, SP2_ERR_RANGE, "n > n_max");
    if (!m || !x || !v || !xbar || !vbar || !mbar) return fail(c, SP2_ERR_ARG, "null argument");
    const int mixed = c->cfg.precision == SP2_MIXED;
    Staging s{c};
    PassOut o;
    o.accumulate = accumulate ? 1 : 0;
    if (ptr_kind == SP2_HOST) {
        const size_t v3 = 3 * n * sizeof(double), v1 = n * sizeof(double);
        for (int k = 0; k < 4; ++k) s.plan(v3);
        s.plan(v1); s.plan(v1); s.plan(v3); s.plan(v3); s.plan(v1);
        SP2_CKS(ensure(c, reinterpret_cast<void **>(&c->stage), &c->stage_cap, s.total, "staging"));
        m = stage_in(s, m, n); x = stage_in(s, x, 3 * n); v = stage_in(s, v, 3 * n);
        abar = stage_in(s, abar, 3 * n); jbar = stage_in(s, jbar, 3 * n); pbar = stage_in(s, pbar, n);
        // accumulate needs the caller's current values on the device
        o.xbar = accumulate ? const_cast<double *>(stage_in(s, static_cast<const double *>(xbar), 3 * n)) : s.slot<double>(3 * n * 8);
        o.vbar = accumulate ? const_cast<double *>(stage_in(s, static_cast<const double *>(vbar), 3 * n)) : s.slot<double>(3 * n * 8);
        o.mbar = accumulate ? const_cast<double *>(stage_in(s, static_cast<const double *>(mbar), n)) : s.slot<double>(n * 8);
        s.out.push_back({xbar, o.xbar}); s.out_bytes.push_back(3 * n * 8);
        s.out.push_back({vbar, o.vbar}); s.out_bytes.push_back(3 * n * 8);
        s.out.push_back({mbar, o.mbar}); s.out_bytes.push_back(n * 8);
        SP2_CKS(stage_copy_in(s));
    } else {
        o.xbar = xbar; o.vbar = vbar; o.mbar = mbar;
    }
    SP2_CK(c, launch_pack_vjp(mixed, n, m, x, v, abar, jbar, pbar, c->rec2, c->stream));
    c->launches += 1;
    SP2_CKS(run_pass(c, K_VJP, 4, mixed, 0, c->rec2, vjp_record_bytes(mixed), n, c->iota, n, 0, n, o, nullptr, ST_VJP));
    if (ptr_kind == SP2_HOST) SP2_CKS(stage_copy_out(s));
    return SP2_OK;
}

sp2_status sp2_get_j(sp2_ctx *c, int64_t first, int64_t n, double *x, double *v, double *a, double *jerk, double *t,
                     int ptr_kind) {
    SP2_CKS(usable(c));
    SP2_CKS(check_ptr_kind(c, ptr_kind));
    if (n < 0 || first < 0 || first + n > c->n_loaded) return fail(c, SP2_ERR_RANGE, "slots outside the loaded set");
    if (n == 0) return SP2_OK;
    const cudaMemcpyKind k = ptr_kind == SP2_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const size_t n3 = 3 * static_cast<size_t>(n) * sizeof(double), o = static_cast<size_t>(first);
    if (x) SP2_CK(c, cudaMemcpyAsync(x, c->js.x + 3 * o, n3, k, c->stream));
    if (v) SP2_CK(c, cudaMemcpyAsync(v, c->js.v + 3 * o, n3, k, c->stream));
    if (a) SP2_CK(c, cudaMemcpyAsync(a, c->js.a + 3 * o, n3, k, c->stream));
    if (jerk) SP2_CK(c, cudaMemcpyAsync(jerk, c->js.jk + 3 * o, n3, k, c->stream));
    if (t) SP2_CK(c, cudaMemcpyAsync(t, c->js.t + o, n * sizeof(double), k, c->stream));
    if (ptr_kind == SP2_HOST) SP2_CK(c, cudaStreamSynchronize(c->stream));
    return SP2_OK;
}

sp2_status sp2_block_init(sp2_ctx *c, double t0, double eta_s, double dt_max) {
    SP2_CKS(usable(c));
    if (c->cfg.order != 4 && c->cfg.order != 6)
        return fail(c, SP2_ERR_UNSUPPORTED, "block time-steps need an order-4 or order-6 context");
    if (c->n_loaded == 0) return fail(c, SP2_ERR_STATE, "no j-particles loaded");
    if (c->capturing) return fail(c, SP2_ERR_STATE, "cannot start block steps during graph capture");
    if (!std::isfinite(t0) || !(eta_s > 0.0) || !(dt_max > 0.0) || !std::isfinite(dt_max))
        return fail(c, SP2_ERR_ARG, "bad t0, eta_s or dt_max");
    const int64_t n = c->n_loaded;
    SP2_CKS(ensure(c, reinterpret_cast<void **>(&c->blk_dt), &c->blk_dt_cap, n * sizeof(double), "block-step"));
    SP2_CKS(ensure(c, reinterpret_cast<void **>(&c->blk_active), &c->blk_active_cap, n * sizeof(int32_t), "block-step"));
    const int order = c->cfg.order;
    // a and jerk (and snap) of every particle at t0 (the stored times are
    // taken to be t0); the snap needs the sources' accelerations, so the
    // 6th-order start takes a second pass with the accelerations of the first
    PassOut o;
    o.acc = c->js.a;  // the pass reads the predicted records, not the store
    o.jerk = c->js.jk;
    o.snap = (order == 6) ? c->js.sn : nullptr;
    for (int pass = 0; pass < (order == 6 ? 2 : 1); ++pass) {
        if (pass > 0) {
            if (c->js.dsc) SP2_CK(c, launch_dscache(order, c->js, 0, n, c->stream));
            c->rec_valid = false;
        }
        SP2_CKS(sp2_predict(c, t0));
        SP2_CKS(materialize(c));
        SP2_CKS(run_pass(c, K_FORCE, order, c->cfg.precision == SP2_MIXED, 0, c->rec, c->rb, n, c->iota, n, 0, n, o,
                         nullptr, ST_FORCE));
    }
    SP2_CK(c, launch_block_init(c->js, c->blk_dt, n, eta_s, dt_max, t0, c->stream));
    if (c->js.dsc) SP2_CK(c, launch_dscache(order, c->js, 0, n, c->stream));
    c->launches += 2;
    if (order == 6) {  // crackles start at zero
        SP2_CKS(ensure(c, reinterpret_cast<void **>(&c->blk_cr), &c->blk_cr_cap, 3 * n * sizeof(double), "block-step"));
        SP2_CKS(ensure(c, reinterpret_cast<void **>(&c->blk_s1), &c->blk_s1_cap, 3 * n * sizeof(double), "block-step"));
        SP2_CK(c, cudaMemsetAsync(c->blk_cr, 0, 3 * n * sizeof(double), c->stream));
    }
    c->rec_valid = false;
    c->blk_ready = true;
    SP2_CK(c, cudaStreamSynchronize(c->stream));
    return SP2_OK;
}

// eta: Aarseth's parameter (4th order) or eta4 of the averaged criterion (6th)
static sp2_status block_run_impl(sp2_ctx *c, double t_end, double eta, double eta6, double dt_max,
                                 sp2_block_stats *st) {
    SP2_CKS(usable(c));
    if (!c->blk_ready) return fail(c, SP2_ERR_STATE, "call sp2_block_init first");
    if (c->capturing) return fail(c, SP2_ERR_STATE, "cannot run block steps during graph capture");
    if (!std::isfinite(t_end) || !(eta > 0.0) || !(dt_max > 0.0)) return fail(c, SP2_ERR_ARG, "bad t_end, eta or dt_max");
    const int64_t n = c->n_loaded;
    const int mixed = c->cfg.precision == SP2_MIXED;
    const int order = c->cfg.order;
    double *a1 = c->tmp, *j1 = c->tmp + 3 * c->cfg.n_max, *s1 = c->blk_s1;
    // 6th order: the predictor adds the crackles (FP64 arithmetic, also for
    // mixed records: the double-single cache holds none); the corrector
    // updates them and keeps the cache in step
    JStore jp = c->js, jc = c->js;
    if (order == 6) {
        jp.cr = jc.cr = c->blk_cr;
        jp.dsc = nullptr;
    }
    if (!c->blk_dev) {
        c->blk_dev = static_cast<BlockDev *>(dalloc(c, sizeof(BlockDev)));
        if (!c->blk_dev) return fail(c, SP2_ERR_NOMEM, "cannot allocate the block-step state");
    }
    BlockDev h{};
    h.min_active = 0xffffffffu;
    h.t_last = -1.0;
    SP2_CK(c, cudaMemcpyAsync(c->blk_dev, &h, sizeof h, cudaMemcpyHostToDevice, c->stream));
    // The active count is only known on the device: the pass kernel derives
    // its sinks per CTA and source split from it.  The host fixes the CTA
    // (256 threads, one sink per thread), the tile (256 sources, room for 32
    // lanes per sink) and the largest split, so that one CTA's share of the
    // in-pass reduction stays bounded and the partial sums of all n sinks fit
    // 256 MB.
    sp2_launch L{};
    L.threads = 256;
    L.i_per_thread = 1;
    L.j_lanes = 1;
    L.j_tile = 256;
    L.split_j = static_cast<int>(kFusedReduceMaxValues / L.threads);
    const double fields = (order == 6) ? 10.0 : 7.0;
    while (L.split_j > 1 && static_cast<double>(n) * fields * 8.0 * L.split_j > 256.0 * (1 << 20)) L.split_j /= 2;
    {
        KernelKey key{K_FORCE, order, mixed, 0, 1, 0, 0, 1};
        int per_sm = 0;
        SP2_CK(c, force_kernel_occupancy(key, L.threads, L.j_tile, &per_sm));
        if (per_sm <= 0) return fail(c, SP2_ERR_UNSUPPORTED, "block-step pass does not fit on an SM");
        L.ctas_per_sm = per_sm;
    }
    PassOut o;
    o.acc = a1;
    o.jerk = j1;
    o.snap = (order == 6) ? s1 : nullptr;
    // Blocks are queued in batches; a block past t_end sets the stop flag on
    // the device and every later kernel of the batch does nothing.  The first
    // batch is launched directly (it sizes the pass buffers); the rest replay
    // one captured batch as a CUDA graph.
    constexpr int kBatch = 32;
    auto enqueue = [&]() -> sp2_status {
        for (int k = 0; k < kBatch; ++k) {
            ev_begin(c, ST_OTHER);
            SP2_CK(c, launch_block_begin(c->blk_dev, c->js.t, c->blk_dt, n, t_end, c->blk_active, c->stream));
            ev_end(c, ST_OTHER);
            ev_begin(c, ST_PREDICT);
            SP2_CK(c, launch_predict(order, mixed, jp, n, 0.0, c->rec, c->stream, c->blk_dev));
            ev_end(c, ST_PREDICT);
            SP2_CKS(run_pass(c, K_FORCE, order, mixed, 0, c->rec, c->rb, n, c->blk_active, n, 0, n, o, &L, ST_FORCE,
                             nullptr, false, &c->blk_dev->count));
            ev_begin(c, ST_OTHER);
            if (order == 6)
                SP2_CK(c, launch_block_correct6_dev(jc, c->blk_dt, c->blk_active, n, c->blk_dev, a1, j1, s1, eta,
                                                    eta6, dt_max, c->stream));
            else
                SP2_CK(c, launch_block_correct_dev(jc, c->blk_dt, c->blk_active, n, c->blk_dev, a1, j1, eta, dt_max,
                                                   c->stream));
            ev_end(c, ST_OTHER);
            c->launches += 5;  // run_pass counts the force kernel
        }
        return SP2_OK;
    };
    auto read_state = [&]() -> sp2_status {
        SP2_CK(c, cudaMemcpyAsync(&h, c->blk_dev, sizeof h, cudaMemcpyDeviceToHost, c->stream));
        SP2_CK(c, cudaStreamSynchronize(c->stream));
        return SP2_OK;
    };
    SP2_CKS(enqueue());
    SP2_CKS(read_state());
    // a stream that cannot be captured (the legacy default stream) keeps
    // direct launches
    if (!h.stop && cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        while (!h.stop) {
            SP2_CKS(enqueue());
            SP2_CKS(read_state());
        }
    }
    if (!h.stop) {
        const int64_t per_batch = c->launches;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        c->capturing = true;
        const sp2_status se = enqueue();
        c->capturing = false;
        cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
        if (se != SP2_OK) {
            if (graph) cudaGraphDestroy(graph);
            return se;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        SP2_CK(c, e);
        const int64_t batch_launches = c->launches - per_batch;
        sp2_status rs = SP2_OK;
        while (!h.stop && rs == SP2_OK) {
            e = cudaGraphLaunch(exec, c->stream);
            if (e != cudaSuccess) break;
            c->launches += batch_launches;
            rs = read_state();
        }
        cudaGraphExecDestroy(exec);
        SP2_CK(c, e);
        if (rs != SP2_OK) return rs;
    }
    c->rec_valid = false;
    if (st) {
        st->block_steps = static_cast<int64_t>(h.steps);
        st->active_sum = static_cast<int64_t>(h.active_sum);
        st->max_active = h.max_active;
        st->min_active = h.steps ? h.min_active : 0;
        st->t = h.t_last;
    }
    if (h.underflow)
        return fail(c, SP2_ERR_RANGE, "block time-step underflow (2^-50) at t = %.17g: the step criterion collapsed",
                    h.t_last);
    return SP2_OK;
}

sp2_status sp2_block_run(sp2_ctx *c, double t_end, double eta, double dt_max, sp2_block_stats *st) {
    SP2_CKS(usable(c));
    if (c->cfg.order != 4) return fail(c, SP2_ERR_UNSUPPORTED, "sp2_block_run takes order-4 contexts (order 6: sp2_block_run_h6)");
    return block_run_impl(c, t_end, eta, 0.0, dt_max, st);
}

sp2_status sp2_block_run_h6(sp2_ctx *c, double t_end, double eta4, double eta6, double dt_max, sp2_block_stats *st) {
    SP2_CKS(usable(c));
    if (c->cfg.order != 6) return fail(c, SP2_ERR_UNSUPPORTED, "sp2_block_run_h6 takes order-6 contexts");
    if (!(eta6 > 0.0)) return fail(c, SP2_ERR_ARG, "bad eta6");
    return block_run_impl(c, t_end, eta4, eta6, dt_max, st);
}

sp2_status sp2_hermite4_step(sp2_ctx *c, int64_t n, double dt, const double *m, double *x, double *v, double *a,
                             double *jerk) {
    SP2_CKS(usable(c));
    if (n <= 0 || n > c->cfg.n_max) return fail(c, SP2_ERR_RANGE, "n outside (0, n_max]");
    if (!m || !x || !v || !a || !jerk) return fail(c, SP2_ERR_ARG, "null argument");
    if (!std::isfinite(dt)) return fail(c, SP2_ERR_ARG, "dt not finite");
    const int mixed = c->cfg.precision == SP2_MIXED;
    double *a1 = c->tmp, *j1 = c->tmp + 3 * c->cfg.n_max;
    SP2_CK(c, launch_h4_predict_pack(mixed, n, dt, m, x, v, a, jerk, c->rec2, c->stream));
    c->launches += 1;
    PassOut o;
    o.acc = a1;
    o.jerk = j1;
    SP2_CKS(run_pass(c, K_FORCE, 4, mixed, 0, c->rec2, record_bytes(4, mixed), n, c->iota, n, 0, n, o, nullptr, ST_FORCE));
    SP2_CK(c, launch_h4_correct(n, dt, x, v, a, jerk, a1, j1, c->stream));
    c->launches += 1;
    return SP2_OK;
}

sp2_status sp2_hermite4_step_vjp(sp2_ctx *c, int64_t n, double dt, const double *m, const double *x, const double *v,
                                 const double *a, const double *jerk, double *gx, double *gv, double *ga, double *gj,
                                 double *gm) {
    SP2_CKS(usable(c));
    if (n <= 0 || n > c->cfg.n_max) return fail(c, SP2_ERR_RANGE, "n outside (0, n_max]");
    if (!m || !x || !v || !a || !jerk || !gx || !gv || !ga || !gj || !gm) return fail(c, SP2_ERR_ARG, "null argument");
    const int mixed = c->cfg.precision == SP2_MIXED;
    double *xpbar = c->tmp + 6 * c->cfg.n_max, *vpbar = c->tmp + 9 * c->cfg.n_max;
    SP2_CK(c, launch_h4_vjp_pre(mixed, n, dt, m, x, v, a, jerk, gx, gv, ga, gj, c->rec2, c->stream));
    c->launches += 1;
    PassOut o;
    o.xbar = xpbar;
    o.vbar = vpbar;
    o.mbar = gm;
    // gm accumulates across steps; xpbar / vpbar start from zero
    SP2_CK(c, cudaMemsetAsync(xpbar, 0, 3 * n * sizeof(double), c->stream));
    SP2_CK(c, cudaMemsetAsync(vpbar, 0, 3 * n * sizeof(double), c->stream));
    o.accumulate = 1;
    SP2_CKS(run_pass(c, K_VJP, 4, mixed, 0, c->rec2, vjp_record_bytes(mixed), n, c->iota, n, 0, n, o, nullptr, ST_VJP));
    SP2_CK(c, launch_h4_vjp_post(n, dt, xpbar, vpbar, gx, gv, ga, gj, c->stream));
    c->launches += 1;
    return SP2_OK;
}

sp2_status sp2_get_launch(sp2_ctx *c, int64_t n_i, sp2_launch *out) {
    SP2_CKS(usable(c));
    if (!out || n_i <= 0) return fail(c, SP2_ERR_ARG, "bad arguments");
    auto it = c->tuned.find(tune_key(n_i, c->n_loaded));
    *out = (it != c->tuned.end()) ? it->second
                                  : heuristic(c, K_FORCE, c->cfg.precision == SP2_MIXED, n_i, std::max<int64_t>(c->n_loaded, 1));
    return SP2_OK;
}

sp2_status sp2_set_launch(sp2_ctx *c, int64_t n_i, const sp2_launch *in) {
    SP2_CKS(usable(c));
    if (!in || n_i <= 0) return fail(c, SP2_ERR_ARG, "bad arguments");
    SP2_CKS(check_launch(c, *in));
    c->tuned[tune_key(n_i, c->n_loaded)] = *in;
    return SP2_OK;
}

sp2_status sp2_autotune(sp2_ctx *c, int64_t n_i, sp2_launch *best) {
    SP2_CKS(usable(c));
    if (c->capturing) return fail(c, SP2_ERR_STATE, "cannot tune during graph capture");
    if (!c->rec_valid) return fail(c, SP2_ERR_STATE, "predicted records are stale: call sp2_predict first");
    if (n_i <= 0 || n_i > c->n_loaded) return fail(c, SP2_ERR_RANGE, "n_i must be in (0, loaded]");
    const int mixed = c->cfg.precision == SP2_MIXED;
    const int order = c->cfg.order;
    const int nn = c->cfg.with_nn;
    const int64_t n_j = c->n_loaded;
    // scratch outputs in tmp (3 n_max doubles each suffice for acc/jerk/snap of n_i <= n_max)
    PassOut o;
    o.acc = c->tmp;
    o.jerk = order == 2 ? nullptr : c->tmp + 3 * c->cfg.n_max;
    o.snap = order == 6 ? c->tmp + 6 * c->cfg.n_max : nullptr;
    o.pot = c->tmp + 9 * c->cfg.n_max;
    o.nn_r2 = nn ? c->tmp + 9 * c->cfg.n_max + n_i : nullptr;
    o.nn_id = nn ? reinterpret_cast<int32_t *>(c->tmp + 9 * c->cfg.n_max + 2 * n_i) : nullptr;
    if (nn && 9 * c->cfg.n_max + 3 * n_i > 12 * c->cfg.n_max) o.nn_r2 = nullptr, o.nn_id = nullptr;

    const sp2_launch h = heuristic(c, K_FORCE, mixed, n_i, n_j);
    // time one launch shape: mean of `reps` runs after one warm-up run
    auto time_shape = [&](const sp2_launch &L, int reps, float *ms_out) -> sp2_status {
        if (check_launch(c, L) != SP2_OK) return SP2_ERR_UNSUPPORTED;
        float ms = 0.f, sum = 0.f;
        sp2_status st = run_pass(c, K_FORCE, order, mixed, nn && o.nn_id, c->rec, c->rb, c->n_loaded, c->iota, n_i,
                                 0, n_j, o, &L, ST_FORCE, &ms, true);
        if (st != SP2_OK) return st;
        for (int r = 0; r < reps; ++r) {
            st = run_pass(c, K_FORCE, order, mixed, nn && o.nn_id, c->rec, c->rb, c->n_loaded, c->iota, n_i, 0, n_j,
                          o, &L, ST_FORCE, &ms, true);
            if (st != SP2_OK) return st;
            sum += ms;
        }
        *ms_out = sum / reps;
        return SP2_OK;
    };
    // resident CTAs per SM of a shape (0 if it does not fit)
    auto occupancy = [&](const sp2_launch &L) -> int {
        int occ = 0;
        // the kernel run_pass will launch: fused prediction when the sinks fit one i-block
        const int fused = (mixed && c->js.dsc && n_i <= int64_t(L.threads / L.j_lanes) * L.i_per_thread) ? 1 : 0;
        KernelKey key{K_FORCE, order, mixed, nn, L.i_per_thread, fused};
        key.mw = L.j_lanes > 32 ? 1 : 0;
        // a fused pass that cannot hold two bulk-copy stages runs with one
        if (fused && pass_smem_bytes(K_FORCE, order, mixed, L.j_tile, c->rb, L.threads, L.i_per_thread, 1, 2) >
                         static_cast<size_t>(kMaxPassSmem))
            key.fused_stages = 1;
        if (pass_smem_bytes(K_FORCE, order, mixed, L.j_tile, c->rb, L.threads, L.i_per_thread, fused,
                            key.fused_stages ? key.fused_stages : 2) > static_cast<size_t>(kMaxPassSmem) ||
            force_kernel_occupancy(key, L.threads, L.j_tile, &occ) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return occ;
    };
    // split counts that give about `rounds` waves of resident CTAs, preferring
    // an exact multiple (a partial last wave leaves SMs idle)
    const int64_t max_split_all = std::max<int64_t>(1, n_j / 32);
    auto split_for = [&](const sp2_launch &L, int rounds, int occ) -> int {
        const int64_t n_iblk = ceil_div(n_i, int64_t(L.threads / L.j_lanes) * L.i_per_thread);
        const int64_t slots = int64_t(c->sm_count) * occ;
        // slices of at least two tiles keep the cp.async ring busy; the fused
        // pass (one i-block, mixed) has no ring, so one tile per slice is fine
        const int64_t min_tiles = (mixed && c->js.dsc && n_iblk == 1) ? 1 : 2;
        const int64_t max_split = std::min<int64_t>(max_split_all, std::max<int64_t>(1, n_j / (min_tiles * L.j_tile)));
        int64_t split = ceil_div(rounds * slots, n_iblk);
        for (int64_t s2 = split; s2 <= split + 2 && s2 <= max_split; ++s2)
            if ((n_iblk * s2) % slots == 0) { split = s2; break; }
        return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(split, max_split)));
    };
    // stage 1: CTA shapes at ~4 waves
    std::vector<std::pair<float, sp2_launch>> shapes;
    for (int threads : {64, 128, 256})
        for (int ipt : {1, 2, 4})
            for (int jl = 1; jl <= ((mixed && ipt == 1) ? threads : 32); jl *= 2) {
                if (jl > threads) continue;
                const int64_t spc = int64_t(threads / jl) * ipt;
                if (spc > 2 * std::max<int64_t>(n_i, 32) && threads > 32) continue;   // mostly empty CTAs
                if (jl > 1 && spc < 8 && n_i > 4096) continue;                       // j-lanes only help few sinks
                for (int tile : {64, 128, 256, 512, 1024}) {
                    if (tile < 8 * jl) continue;
                    sp2_launch L{threads, ipt, jl, tile, 1, 0};
                    const int occ = occupancy(L);
                    if (occ <= 0) continue;
                    L.split_j = split_for(L, 4, occ);
                    float ms = 0.f;
                    const sp2_status st = time_shape(L, 1, &ms);
                    if (st == SP2_ERR_UNSUPPORTED) continue;
                    if (st != SP2_OK) return st;
                    shapes.push_back({ms, L});
                }
            }
    {
        float ms = 0.f;
        if (time_shape(h, 1, &ms) == SP2_OK) shapes.push_back({ms, h});
    }
    if (shapes.empty()) return fail(c, SP2_ERR_UNSUPPORTED, "no launch shape could run");
    std::sort(shapes.begin(), shapes.end(), [](const std::pair<float, sp2_launch> &x, const std::pair<float, sp2_launch> &y) {
        return x.first < y.first;
    });
    // stage 2: the best shapes over 1 .. 16 waves, three timed runs each
    std::vector<sp2_launch> cand;
    for (size_t r = 0; r < std::min<size_t>(4, shapes.size()); ++r) {
        const sp2_launch base = shapes[r].second;
        const int occ = occupancy(base);
        cand.push_back(base);
        for (int rounds : {1, 2, 3, 6, 8, 12, 16}) {
            sp2_launch L = base;
            L.split_j = split_for(L, rounds, occ);
            bool dup = false;
            for (auto &q : cand) dup |= std::memcmp(&q, &L, sizeof L) == 0;
            if (!dup) cand.push_back(L);
        }
    }
    size_t best_k = 0;
    float best_ms = 1e30f;
    for (size_t k = 0; k < cand.size(); ++k) {
        float ms = 0.f;
        const sp2_status st = time_shape(cand[k], 3, &ms);
        if (st == SP2_ERR_UNSUPPORTED) continue;
        if (st != SP2_OK) return st;
        if (ms < best_ms) { best_ms = ms; best_k = k; }
    }
    c->tuned[tune_key(n_i, n_j)] = cand[best_k];
    if (best) *best = cand[best_k];
    return SP2_OK;
}

sp2_status sp2_graph_begin(sp2_ctx *c) {
    SP2_CKS(usable(c));
    if (c->capturing) return fail(c, SP2_ERR_STATE, "already capturing");
    SP2_CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    c->capturing = true;
    return SP2_OK;
}

sp2_status sp2_graph_end(sp2_ctx *c, sp2_graph **out) {
    SP2_CKS(usable(c));
    if (!out) return fail(c, SP2_ERR_ARG, "null output");
    if (!c->capturing) return fail(c, SP2_ERR_STATE, "not capturing");
    c->capturing = false;
    sp2_graph *g = new sp2_graph();
    cudaError_t e = cudaStreamEndCapture(c->stream, &g->graph);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) {
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return cuda_fail(c, e, "graph capture");
    }
    *out = g;
    return SP2_OK;
}

sp2_status sp2_graph_launch(sp2_ctx *c, const sp2_graph *g) {
    SP2_CKS(usable(c));
    if (!g) return fail(c, SP2_ERR_ARG, "null graph");
    SP2_CK(c, cudaGraphLaunch(g->exec, c->stream));
    return SP2_OK;
}

sp2_status sp2_graph_destroy(sp2_graph *g) {
    if (!g) return SP2_OK;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return SP2_OK;
}

sp2_status sp2_sync(sp2_ctx *c) {
    SP2_CKS(usable(c));
    if (c->capturing) return fail(c, SP2_ERR_STATE, "cannot synchronise during graph capture");
    unsigned int flag = 0;
    SP2_CK(c, cudaMemcpyAsync(&flag, c->dev_words + 1, sizeof flag, cudaMemcpyDeviceToHost, c->stream));
    SP2_CK(c, cudaStreamSynchronize(c->stream));
    if (flag) {
        SP2_CK(c, cudaMemsetAsync(c->dev_words + 1, 0, sizeof flag, c->stream));
        SP2_CK(c, cudaStreamSynchronize(c->stream));
        if (flag & 2u)
            return fail(c, SP2_ERR_TIMEOUT, "a bulk copy into shared memory did not complete within the wait limit "
                                            "(outputs undefined)");
        return fail(c, SP2_ERR_RANGE, "a device-side slot index was outside the loaded set (skipped; outputs undefined)");
    }
    return SP2_OK;
}

sp2_status sp2_profile_reset(sp2_ctx *c) {
    SP2_CKS(usable(c));
    for (int s = 0; s < ST_COUNT; ++s) c->ev_count[s] = 0;
    return SP2_OK;
}

sp2_status sp2_profile_read(sp2_ctx *c, int64_t *counts, double *total_ms, int n) {
    SP2_CKS(usable(c));
    if (!counts || !total_ms || n <= 0) return fail(c, SP2_ERR_ARG, "bad arguments");
    if (!c->cfg.profile) return fail(c, SP2_ERR_STATE, "context opened without profile = 1");
    if (c->capturing) return fail(c, SP2_ERR_STATE, "cannot read timings during graph capture");
    SP2_CK(c, cudaStreamSynchronize(c->stream));
    const int k = std::min(n, static_cast<int>(ST_COUNT));
    for (int s = 0; s < k; ++s) {
        const int64_t cnt = std::min<int64_t>(c->ev_count[s], kEventRing);
        double sum = 0.0;
        for (int64_t q = 0; q < cnt; ++q) {
            float ms = 0.f;
            SP2_CK(c, cudaEventElapsedTime(&ms, c->ev[s][2 * q], c->ev[s][2 * q + 1]));
            sum += ms;
        }
        counts[s] = cnt;
        total_ms[s] = sum;
    }
    return SP2_OK;
}

}  // extern "C"
