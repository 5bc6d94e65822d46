// sp2_static.cu -- a block step that allocates nothing: the mixed-precision
// Hermite-4 predict + force pass + source-split reduction, with all of its
// scratch (predicted records, per-slice partial sums, the work-queue counter)
// in one file-scope device array instead of memory from cudaMalloc.
//
// Some callers cannot allocate device memory at the point where they need a
// force evaluation: hosts whose device memory is owned by another allocator or
// a fixed budget they may not bypass (an integrator embedded in a larger code
// that hands out all device memory itself), or real-time / signal-driven loops
// that must not enter the CUDA allocator, whose calls may block or fail under
// memory pressure.  They pass inputs and outputs; everything else lives in
// `sp2_static_scratch`.
//
// The array is kStaticScratchBytes per GPU that loads the library, held until
// the process exits.  Every call shares it and it keeps the previous call's
// contents: the work-queue counter and error word are cleared by each call,
// and calls whose GPU work overlaps (different streams, or different host
// threads on the same device) race on it -- serialise them.
//
// A sink slot outside [0, n_j) is skipped by the force pass; a last small
// kernel then writes NaN into that sink's acc, jerk, pot and nn_r2 and -1 into
// its nn_id, so a bad index shows in the outputs without a host read-back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "sapporo_gb.h"
#include "sp2_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr int64_t kStaticMaxSources = 65536;
constexpr int kMaxDevices = 64;
constexpr int kRecBytes = 48;   // mixed Hermite-4 predicted record
constexpr int kFields = 7;      // acc, jerk, pot

}  // namespace

static __device__ __align__(256) unsigned char sp2_static_scratch[kStaticScratchBytes];

namespace {

// Device address of the array, looked up once per device (with it current).
void *g_scratch[kMaxDevices] = {};

sp2_status scratch_for_current_device(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SP2_ERR_CUDA;
    if (!g_scratch[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, sp2_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SP2_ERR_CUDA;
        }
        g_scratch[dev] = p;
    }
    *out = g_scratch[dev];
    return SP2_OK;
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Outputs of sinks whose slot lies outside [0, n_j): NaN (nn_id -1).
__global__ void mark_bad_sinks_kernel(const int32_t *i_idx, int64_t n_i, int64_t n_j, double *acc, double *jerk,
                                      double *pot, int32_t *nn_id, double *nn_r2) {
    const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n_i) return;
    const int32_t slot = i_idx[k];
    if (slot >= 0 && slot < n_j) return;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    for (int c = 0; c < 3; ++c) {
        acc[3 * k + c] = nan;
        jerk[3 * k + c] = nan;
    }
    pot[k] = nan;
    if (nn_id) nn_id[k] = -1;
    if (nn_r2) nn_r2[k] = nan;
}

}  // namespace

extern "C" sp2_status sp2_step_static(int64_t n_j, const int32_t *id, const double *m, const double *x,
                                      const double *v, const double *a, const double *jerk, const double *t_j,
                                      double t, double eps2, int64_t n_i, const int32_t *i_idx, double *acc,
                                      double *jerk_out, double *pot, int32_t *nn_id, double *nn_r2,
                                      void *cuda_stream) {
    using namespace sp2;
    if (n_j < 0 || n_i < 0) return SP2_ERR_ARG;
    if (n_j > kStaticMaxSources || n_i > kStaticMaxSources) return SP2_ERR_RANGE;
    if (n_i == 0) return SP2_OK;
    if (n_j == 0) return SP2_ERR_STATE;
    if (!id || !m || !x || !v || !a || !jerk || !t_j || !i_idx || !acc || !jerk_out || !pot) return SP2_ERR_ARG;
    if ((nn_id == nullptr) != (nn_r2 == nullptr)) return SP2_ERR_ARG;
    if (!std::isfinite(t) || !(eps2 >= 0.0) || !std::isfinite(eps2)) return SP2_ERR_ARG;
    void *base = nullptr;
    sp2_status st = scratch_for_current_device(&base);
    if (st != SP2_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SP2_ERR_CUDA;

    // scratch layout: [256 B words: queue, error flag][records][partials][partial ids]
    unsigned char *p = static_cast<unsigned char *>(base);
    unsigned int *words = reinterpret_cast<unsigned int *>(p);
    unsigned char *rec = p + 256;
    const size_t rec_bytes = static_cast<size_t>(n_j) * kRecBytes;
    unsigned char *part_base = rec + (rec_bytes + 255) / 256 * 256;
    const size_t room = kStaticScratchBytes - static_cast<size_t>(part_base - p);
    const int nn = (nn_id || nn_r2) ? 1 : 0;
    const size_t per_slice = static_cast<size_t>(n_i) * ((kFields + nn) * sizeof(double) + (nn ? sizeof(int32_t) : 0));

    // launch shape: the library's default form for n_i sinks, with the source
    // split capped by the room left in the array
    sp2_launch L{256, 2, 1, 128, 1, 0};
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
    const int64_t slots = static_cast<int64_t>(sms) * std::max(1, 512 / L.threads);
    int64_t split = ceil_div(4 * slots, n_iblk);
    split = std::max<int64_t>(1, std::min<int64_t>(split, n_j / (2 * L.j_tile)));
    if (n_iblk >= 4 * slots) split = 1;
    const int64_t split_room = static_cast<int64_t>(room / per_slice);
    if (split > 1) split = std::max<int64_t>(1, std::min(split, split_room));
    int64_t slice_len = ceil_div(ceil_div(n_j, split), L.j_tile) * L.j_tile;
    split = ceil_div(n_j, slice_len);
    if (split > 1 && static_cast<size_t>(split) * per_slice > room) return SP2_ERR_RANGE;

    JStore js{};
    js.id = const_cast<int32_t *>(id);
    js.m = const_cast<double *>(m);
    js.x = const_cast<double *>(x);
    js.v = const_cast<double *>(v);
    js.a = const_cast<double *>(a);
    js.jk = const_cast<double *>(jerk);
    js.t = const_cast<double *>(t_j);
    if (cudaMemsetAsync(words, 0, 2 * sizeof(unsigned int), s) != cudaSuccess) return SP2_ERR_CUDA;
    if (launch_predict(4, 1, js, n_j, t, rec, s) != cudaSuccess) return SP2_ERR_CUDA;

    KernelKey key{K_FORCE, 4, 1, nn, L.i_per_thread};
    int per_sm = 0;
    if (force_kernel_occupancy(key, L.threads, L.j_tile, &per_sm) != cudaSuccess || per_sm <= 0) return SP2_ERR_CUDA;
    ForceParams fp{};
    fp.rec = rec;
    fp.i_idx = i_idx;
    fp.n_i = n_i;
    fp.j_begin = 0;
    fp.j_end = n_j;
    fp.slice_len = slice_len;
    fp.split = static_cast<int>(split);
    fp.jl = L.j_lanes;
    fp.tile = L.j_tile;
    fp.sinks_per_cta = static_cast<int>(sinks_per_cta);
    fp.n_iblk = n_iblk;
    fp.n_items = n_iblk * split;
    fp.queue = words;
    fp.err = words + 1;
    fp.n_loaded = n_j;
    fp.eps2 = eps2;
    fp.acc = acc;
    fp.jerk = jerk_out;
    fp.pot = pot;
    fp.nn_id = nn_id;
    fp.nn_r2 = nn_r2;
    double *part = reinterpret_cast<double *>(part_base);
    int32_t *part_id = reinterpret_cast<int32_t *>(part_base + static_cast<size_t>(split) * n_i * (kFields + nn) * sizeof(double));
    fp.part = part;
    fp.part_id = part_id;
    fp.sink_major = split >= kWarpReduceMinSplit ? 1 : 0;
    const int grid = static_cast<int>(std::min<int64_t>(fp.n_items, static_cast<int64_t>(sms) * per_sm));
    if (launch_force_kernel(key, fp, grid, L.threads, L.j_tile, s) != cudaSuccess) return SP2_ERR_CUDA;
    if (split > 1) {
        ReduceParams r{};
        r.part = part;
        r.part_id = part_id;
        r.n_i = n_i;
        r.split = static_cast<int>(split);
        r.acc = acc;
        r.jerk = jerk_out;
        r.pot = pot;
        r.nn_id = nn_id;
        r.nn_r2 = nn_r2;
        if (launch_reduce_kernel(key, r, s) != cudaSuccess) return SP2_ERR_CUDA;
    }
    mark_bad_sinks_kernel<<<static_cast<unsigned>(ceil_div(n_i, 256)), 256, 0, s>>>(i_idx, n_i, n_j, acc, jerk_out,
                                                                                    pot, nn_id, nn_r2);
    if (cudaGetLastError() != cudaSuccess) return SP2_ERR_CUDA;
    return SP2_OK;
}
