// sp2_internal.h -- declarations shared by the host API and the kernel
// translation units of the gravity library.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "sapporo_gb.h"

namespace sp2 {

// Device copy of the j-particles, FP64, in the caller's layout (Sec. 2.2.2:
// particle data is always stored in double precision).
struct JStore {
    int32_t *id;
    double *m, *x, *v, *a, *jk, *sn, *t;  // x/v/a/jk/sn: n x 3 row-major
    // Mixed-precision contexts also keep a double-single copy of each particle
    // (null otherwise), written whenever the FP64 store is, so that the
    // per-step predictor needs no FP64 arithmetic:
    //   {xh yh zh m}{xl yl zl th}{vxh vyh vzh tl}{vxl vyl vzl id}
    //   {axh ayh azh 0}{axl ayl azl 0}{jx jy jz 0}[{sx sy sz 0}]   (float4 words)
    float4 *dsc;
    // 6th-order block time-steps only: per-particle crackle (n x 3) from the
    // last correction, added to the predictor when set (null otherwise)
    double *cr;
};
__host__ __device__ constexpr int dscache_words(int order) { return order == 6 ? 8 : 7; }

// Bytes of one predicted record (order 2, leap-frog: the order-4 layout with
// zero velocities).
//   mixed H4: {xh yh zh m}{xl yl zl id}{vx vy vz 0}            48 B
//   mixed H6: + {ax ay az 0}                                   64 B
//   fp64  H4: {x y}{z m}{vx vy}{vz id}                         64 B
//   fp64  H6: + {ax ay}{az 0}                                  96 B
//   mixed VJP: {xh yh zh m}{xl yl zl pbar}{v 0}{abar 0}{jbar 0} 80 B
//   fp64  VJP: {x y}{z m}{vx vy}{vz pbar}{abar x y}{abar z, jbar x}{jbar y z} 112 B
inline int record_bytes(int order, int mixed) {
    if (mixed) return order == 6 ? 64 : 48;
    return order == 6 ? 96 : 64;
}
inline int vjp_record_bytes(int mixed) { return mixed ? 80 : 112; }

// Parameters of one force-kernel launch (persistent grid over work items
// (i-block, j-slice); see sp2_device.cuh).
struct ForceParams {
    const unsigned char *rec;  // predicted records, slot 0
    const int32_t *i_idx;      // sink slots (n_i); with sink_rec: slot for the self pair, or < 0 for none
    const unsigned int *n_i_dev;  // if set: the sink count is read here (n_i is then only its upper bound)
    const unsigned char *sink_rec;  // explicit sinks: record of sink position i (null: sinks are rec[i_idx[i]])
    int64_t n_i;
    int64_t j_begin, j_end;    // source slots [j_begin, j_end)
    int64_t slice_len;         // sources per slice
    int split;                 // slices
    int jl;                    // threads per sink
    int tile;                  // records per shared-memory stage
    int sinks_per_cta;         // threads / jl * ipt
    int64_t n_iblk;            // i-blocks
    int64_t n_items;           // n_whole + (n_iblk - n_whole) * split
    // i-blocks 0 .. n_whole-1 run over all sources as one item each and
    // write their outputs directly; only the remaining i-blocks are split and
    // have partial rows, counted from sink tail_sink0 = n_whole * sinks_per_cta
    int64_t n_whole;
    int64_t tail_sink0;
    unsigned int *queue;       // work-queue counter, zero at launch
    unsigned int *exit_count;  // if set: CTAs count out and the last resets queue and exit_count to zero
    int static_items;          // grid == n_items: CTA b takes item b and the queue is not used
    unsigned int *err;         // bit 1: a sink slot was outside [0, n_loaded); bit 2: a bulk-copy wait gave up
    int64_t n_loaded;
    double eps2;
    // final outputs (split == 1); any may be null
    double *acc, *jerk, *snap, *pot;
    int32_t *nn_id;
    double *nn_r2;
    // partial results (split > 1), NF = summed fields (+1 for the NN r^2),
    // r = i - tail_sink0 the partial row of sink i, pn = n_i - tail_sink0:
    //   field-major (sink_major = 0): part[f * split * pn + slice * pn + r],
    //                                 part_id[slice * pn + r]
    //   sink-major  (sink_major = 1): part[(r * NF + f) * split + slice],
    //                                 part_id[r * split + slice]
    // sink-major is used with the warp-per-sink reduction (split >= 32), so a
    // warp reads its sink's slices contiguously.
    double *part;
    int32_t *part_id;
    int sink_major;
    // fused reduction (split > 1): the last CTA to finish a slice of an
    // i-block (counted in done[iblk], zero between launches and reset by that
    // CTA) sums the i-block's partials in slice order and writes the outputs
    int fused_reduce;
    unsigned int *done;
    // neighbour lists (kernels of the neighbour-list policy only): per sink
    // position i, squared radius nb_h2[i], counter nb_count[i] (zero at launch)
    // and nb_max slots at nb_list + i * nb_max
    const double *nb_h2;
    int32_t *nb_count;
    int32_t *nb_list;
    int nb_max;
    // VJP outputs / flags
    double *xbar, *vbar, *mbar;
    int accumulate;
    // fused prediction (mixed policies): sources and sinks are predicted from
    // the double-single cache to t = t_hi + t_lo inside the pass
    const float4 *dsc;
    float t_hi, t_lo;
    int fused_stages;          // bulk-copy stages of the fused prediction: 1 (a slice fits one tile) or 2
};

struct ReduceParams {
    const double *part;
    const int32_t *part_id;
    int64_t n_i;
    int split;                 // >= 32: warp per sink on the sink-major layout
    double *acc, *jerk, *snap, *pot;
    int32_t *nn_id;
    double *nn_r2;
    double *xbar, *vbar, *mbar;
    int accumulate;
};

struct BatchParams {
    const unsigned char *rec;
    const int4 *items;         // {system first slot, system size, chunk first slot, chunk size}
    int64_t n_items;
    int64_t out_base;          // slot of output row 0
    unsigned int *queue;
    double eps2;
    double *acc, *jerk, *snap, *pot;
    int32_t *nn_id;
    double *nn_r2;
};

enum Kind { K_FORCE = 0, K_VJP = 1 };

// Dynamic shared memory a pass launch may use (the 227 KiB per block of the
// GPU, less room for the kernels' static shared variables, about 2.5 KiB).
constexpr int kMaxPassSmem = 222 * 1024;

// From this many slices on, the split-j reduction runs one warp per sink on
// the sink-major partial layout (ForceParams::sink_major).
constexpr int kWarpReduceMinSplit = 32;
// Up to this many sinks, that reduction uses a whole block per sink.
constexpr int64_t kBlockReduceMaxSinks = 1024;

struct KernelKey {
    int kind;   // K_FORCE / K_VJP
    int order;  // 4 / 6 (VJP: 4)
    int mixed;  // 0 / 1
    int nn;     // 0 / 1
    int ipt;    // 1 / 2 / 4
    int fused;  // 1: predict sources in the pass (mixed force only)
    int nb;     // 1: neighbour lists (force kernels with nearest neighbour, ipt 1)
    int devn;   // 1: sink count read on the device, shape derived from it (order 4 or 6, no NN, ipt 1)
    int fused_stages;  // fused: bulk-copy stages the launch uses (0: the maximum), for the occupancy query
    int mw;     // 1: several warps per sink (j_lanes above 32; one sink per thread, paired force policies)
};

// Each kernel translation unit provides these for its (order, precision).
// They return cudaErrorInvalidValue for a key they do not hold.  tile: the
// sources per shared-memory stage (the kernels size their shared memory).
cudaError_t launch_force_kernel(const KernelKey &k, const ForceParams &p, int grid, int threads,
                                size_t tile, cudaStream_t s);
cudaError_t force_kernel_occupancy(const KernelKey &k, int threads, size_t tile, int *blocks_per_sm);
cudaError_t launch_reduce_kernel(const KernelKey &k, const ReduceParams &p, cudaStream_t s);
cudaError_t launch_batched_kernel(int order, int mixed, int nn, const BatchParams &p, int grid,
                                  int threads, cudaStream_t s);
cudaError_t batched_kernel_occupancy(int order, int mixed, int nn, int threads, int *blocks_per_sm);

// Per-(order, precision) entry points, defined in sp2_kernels_*.cu.
#define SP2_DECLARE_TU(SUFFIX)                                                                     \
    cudaError_t launch_force_##SUFFIX(const KernelKey &, const ForceParams &, int, int, size_t,    \
                                      cudaStream_t);                                               \
    cudaError_t occupancy_force_##SUFFIX(const KernelKey &, int, size_t, int *);                   \
    cudaError_t launch_reduce_##SUFFIX(const KernelKey &, const ReduceParams &, cudaStream_t);     \
    cudaError_t launch_batched_##SUFFIX(int, const BatchParams &, int, int, cudaStream_t);         \
    cudaError_t occupancy_batched_##SUFFIX(int, int, int *);
SP2_DECLARE_TU(h2m)
SP2_DECLARE_TU(h2d)
SP2_DECLARE_TU(h4m)
SP2_DECLARE_TU(h4d)
SP2_DECLARE_TU(h6m)
SP2_DECLARE_TU(h6d)
SP2_DECLARE_TU(vjpm)
SP2_DECLARE_TU(vjpd)
#undef SP2_DECLARE_TU

// Predictor and element-wise kernels (sp2_predict.cu).
// slots outside [0, n_loaded) are skipped and set *err (device word) to 1.
cudaError_t launch_scatter_j(const JStore &dst, const int32_t *slots, int64_t n, int64_t n_loaded,
                             unsigned int *err, const int32_t *id, const double *m, const double *x,
                             const double *v, const double *a, const double *jk, const double *sn,
                             const double *t, cudaStream_t s);
// State of a device-driven block time-step run (one per context).
struct BlockDev {
    unsigned long long t1bits;  // order-preserving key of the current block time
    unsigned int count;         // active particles of the current block (0: none / stopped)
    unsigned int stop;          // set once the next block time passes t_end (or on underflow)
    unsigned int underflow;     // a new step fell to the 2^-50 floor: the run stops there
    unsigned long long steps, active_sum;
    unsigned int max_active, min_active;
    double t_last;              // time of the last block taken
};

// Mixed records come from js.dsc when it is set (double-single arithmetic),
// from the FP64 arrays otherwise.  t_dev: if set, the time is read on the
// device from a BlockDev (the launch does nothing when its count is zero)
cudaError_t launch_predict(int order, int mixed, const JStore &js, int64_t n, double t,
                           unsigned char *rec, cudaStream_t s, const BlockDev *t_dev = nullptr);
// Refresh js.dsc for slots [first, first + n) from the FP64 store.
cudaError_t launch_dscache(int order, const JStore &js, int64_t first, int64_t n, cudaStream_t s);
// (m, x, v) -> order-4 records with no prediction (all-pairs entry points)
cudaError_t launch_pack_state(int mixed, int64_t n, const double *m, const double *x,
                              const double *v, unsigned char *rec, cudaStream_t s);
// explicit sinks in the context's record format (order 2 and 4 share one)
cudaError_t launch_pack_sinks(int order, int mixed, int64_t n, const double *x, const double *v, const double *a,
                              unsigned char *rec, cudaStream_t s);
cudaError_t launch_iota(int32_t *dst, int64_t n, cudaStream_t s);

// Block time-steps (Hermite-4 with individual power-of-two steps).
cudaError_t launch_block_init(const JStore &js, double *dt, int64_t n, double eta_s, double dt_max, double t0,
                              cudaStream_t s);
// bd->t1bits = key of t1 = min(t + dt); active[0 .. bd->count) = slots with
// t + dt == t1, or bd->stop set (count 0) once t1 > t_end
cudaError_t launch_block_begin(BlockDev *bd, const double *t, const double *dt, int64_t n, double t_end,
                               int32_t *active, cudaStream_t s);
// Hermite-4 corrector and new step of the active slots of the current block
cudaError_t launch_block_correct_dev(const JStore &js, double *dt, const int32_t *active, int64_t n_max,
                                     BlockDev *bd, const double *a1, const double *j1, double eta, double dt_max,
                                     cudaStream_t s);
// 6th-order form: s1 the snaps, js.cr the crackles (updated), the averaged
// criterion with eta4 and eta6
cudaError_t launch_block_correct6_dev(const JStore &js, double *dt, const int32_t *active, int64_t n_max,
                                      BlockDev *bd, const double *a1, const double *j1, const double *s1,
                                      double eta4, double eta6, double dt_max, cudaStream_t s);
cudaError_t launch_nb_finish(const int32_t *ids, int64_t n_i, int nb_max, const int32_t *count, int32_t *list,
                             cudaStream_t s);
cudaError_t launch_h4_predict_pack(int mixed, int64_t n, double dt, const double *m,
                                   const double *x, const double *v, const double *a,
                                   const double *jk, unsigned char *rec, cudaStream_t s);
cudaError_t launch_h4_correct(int64_t n, double dt, double *x, double *v, double *a, double *jk,
                              const double *a1, const double *j1, cudaStream_t s);
// Step VJP, part 1: output cotangents -> force cotangents + VJP records of the
// predicted state.  Part 2: combine into input cotangents (in place).
cudaError_t launch_h4_vjp_pre(int mixed, int64_t n, double dt, const double *m, const double *x,
                              const double *v, const double *a, const double *jk,
                              const double *gx, const double *gv, const double *ga,
                              const double *gj, unsigned char *vrec, cudaStream_t s);
cudaError_t launch_h4_vjp_post(int64_t n, double dt, const double *xpbar, const double *vpbar,
                               double *gx, double *gv, double *ga, double *gj, cudaStream_t s);
cudaError_t launch_pack_vjp(int mixed, int64_t n, const double *m, const double *x,
                            const double *v, const double *abar, const double *jbar,
                            const double *pbar, unsigned char *vrec, cudaStream_t s);
cudaError_t launch_scan_finite(const double *p, int64_t n, unsigned int *flag, cudaStream_t s);

}  // namespace sp2
