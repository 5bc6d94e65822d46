// sp2_predict.cu -- O(N) kernels around the pairwise passes: the copy
// (scatter) kernel and the Taylor predictor of Sec. 2.2.4, the record packing
// for the all-pairs entry points, and the element-wise parts of the shared
// time-step Hermite-4 step and its reverse.
//
// The predictor is memory bound (it reads ~116-140 B and writes 48-96 B per
// particle).  It evaluates each Taylor sum left to right with explicitly
// rounded multiplies and adds (no fused multiply-add), dt^k/k! formed as dt^k
// times the double nearest 1/k!, so the predicted FP64 values are those of a
// plain IEEE evaluation of the polynomial.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sp2_ds.cuh"
#include "sp2_internal.h"

namespace sp2 {
namespace {

constexpr int kThreads = 256;
constexpr double kBlockDtMin = 1.0 / (1ll << 50);  // smallest block step (2^-50)

inline unsigned grid_for(int64_t n) { return static_cast<unsigned>((n + kThreads - 1) / kThreads); }
// FP64-heavy per-particle kernels over a few hundred active particles: one
// warp per CTA spreads them over the SMs (an SM retires 2 FP64 FMAs a clock)
constexpr int kWarpCta = 32;
inline unsigned grid_for_warps(int64_t n) { return static_cast<unsigned>((n + kWarpCta - 1) / kWarpCta); }

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }


__device__ __forceinline__ void store_mixed(unsigned char *rec, int rb, int64_t j, const double *xp,
                                            const double *vp, const double *ap, double m, int id) {
    float xh[3], xl[3];
    for (int c = 0; c < 3; ++c) {
        const ds q = ds_split(xp[c]);  // hi = fl32(x), lo = fl32(x - hi)
        xh[c] = q.h;
        xl[c] = q.l;
    }
    float4 *o = reinterpret_cast<float4 *>(rec + j * rb);
    o[0] = make_float4(xh[0], xh[1], xh[2], __double2float_rn(m));
    o[1] = make_float4(xl[0], xl[1], xl[2], __int_as_float(id));
    o[2] = make_float4(__double2float_rn(vp[0]), __double2float_rn(vp[1]), __double2float_rn(vp[2]), 0.f);
    if (ap) o[3] = make_float4(__double2float_rn(ap[0]), __double2float_rn(ap[1]), __double2float_rn(ap[2]), 0.f);
}

__device__ __forceinline__ void store_fp64(unsigned char *rec, int rb, int64_t j, const double *xp,
                                           const double *vp, const double *ap, double m, int id) {
    double2 *o = reinterpret_cast<double2 *>(rec + j * rb);
    o[0] = make_double2(xp[0], xp[1]);
    o[1] = make_double2(xp[2], m);
    o[2] = make_double2(vp[0], vp[1]);
    o[3] = make_double2(vp[2], __longlong_as_double(static_cast<long long>(id)));
    if (ap) {
        o[4] = make_double2(ap[0], ap[1]);
        o[5] = make_double2(ap[2], 0.0);
    }
}

__device__ __forceinline__ void write_dscache(const JStore &d, int64_t s) {
    float4 *o = d.dsc + s * ((d.sn != nullptr) ? 8 : 7);
    const ds x0 = ds_split(d.x[3 * s]), x1 = ds_split(d.x[3 * s + 1]), x2 = ds_split(d.x[3 * s + 2]);
    const ds v0 = ds_split(d.v[3 * s]), v1 = ds_split(d.v[3 * s + 1]), v2 = ds_split(d.v[3 * s + 2]);
    const ds a0 = ds_split(d.a[3 * s]), a1 = ds_split(d.a[3 * s + 1]), a2 = ds_split(d.a[3 * s + 2]);
    const ds tt = ds_split(d.t[s]);
    o[0] = make_float4(x0.h, x1.h, x2.h, __double2float_rn(d.m[s]));
    o[1] = make_float4(x0.l, x1.l, x2.l, tt.h);
    o[2] = make_float4(v0.h, v1.h, v2.h, tt.l);
    o[3] = make_float4(v0.l, v1.l, v2.l, __int_as_float(d.id[s]));
    o[4] = make_float4(a0.h, a1.h, a2.h, 0.f);
    o[5] = make_float4(a0.l, a1.l, a2.l, 0.f);
    o[6] = make_float4(__double2float_rn(d.jk[3 * s]), __double2float_rn(d.jk[3 * s + 1]),
                       __double2float_rn(d.jk[3 * s + 2]), 0.f);
    if (d.sn)
        o[7] = make_float4(__double2float_rn(d.sn[3 * s]), __double2float_rn(d.sn[3 * s + 1]),
                           __double2float_rn(d.sn[3 * s + 2]), 0.f);
}

__global__ void dscache_kernel(JStore d, int64_t first, int64_t n) {
    const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k < n) write_dscache(d, first + k);
}

// Block times are compared through an unsigned key that orders like the
// doubles (negative times included): the sign bit flipped for t >= 0, every bit
// for t < 0; all ones (the empty minimum) decodes to NaN.
__device__ __forceinline__ unsigned long long time_key(double t) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(t));
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_time(unsigned long long k) {
    const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double(static_cast<long long>(b));
}

// Mixed-precision predictor on the double-single cache (predict_ds_record).
template <int ORDER>
__global__ void predict_ds_kernel(const float4 *dsc, int64_t n, float t_hi, float t_lo, unsigned char *rec,
                                  const BlockDev *bd) {
    const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    if (bd) {  // time of the current block, chosen on the device
        if (bd->count == 0) return;
        const double t = key_time(bd->t1bits);
        t_hi = __double2float_rn(t);
        t_lo = __double2float_rn(t - static_cast<double>(t_hi));
    }
    float4 o[4];
    predict_ds_record<ORDER>(dsc, j, t_hi, t_lo, o);
    float4 *dst = reinterpret_cast<float4 *>(rec + j * (ORDER == 6 ? 64 : 48));
    dst[0] = o[0];
    dst[1] = o[1];
    dst[2] = o[2];
    if (ORDER == 6) dst[3] = o[3];
}

__global__ void scatter_kernel(JStore d, const int32_t *slots, int64_t n, int64_t n_loaded, unsigned int *err,
                               const int32_t *id, const double *m, const double *x, const double *v,
                               const double *a, const double *jk, const double *sn, const double *t) {
    const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t s = slots[k];
    if (s < 0 || s >= n_loaded) {  // reported by sp2_sync; the particle is not stored
        atomicOr(err, 1u);
        return;
    }
    d.id[s] = id[k];
    d.m[s] = m[k];
    d.t[s] = t ? t[k] : 0.0;  // v, a, jk, t may be absent for leap-frog (order 2) sources
    for (int c = 0; c < 3; ++c) {
        d.x[3 * s + c] = x[3 * k + c];
        d.v[3 * s + c] = v ? v[3 * k + c] : 0.0;
        d.a[3 * s + c] = a ? a[3 * k + c] : 0.0;
        d.jk[3 * s + c] = jk ? jk[3 * k + c] : 0.0;
        if (sn) d.sn[3 * s + c] = sn[3 * k + c];
    }
    if (d.dsc) write_dscache(d, s);
}

template <int ORDER, bool MIXED>
__global__ void predict_kernel(JStore js, int64_t n, double t, unsigned char *rec, const BlockDev *bd) {
    const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    if (bd) {
        if (bd->count == 0) return;
        t = key_time(bd->t1bits);
    }
    const double c2 = 0.5, c3 = 1.0 / 6.0, c4 = 1.0 / 24.0;
    const double dt = dadd(t, -js.t[j]);
    const double dt2 = dmul(dt, dt);
    const double dt3 = dmul(dt2, dt);
    const double dt4 = dmul(dt3, dt);
    const double h2 = dmul(dt2, c2), h3 = dmul(dt3, c3), h4 = dmul(dt4, c4);
    double xp[3], vp[3], ap[3];
    // Mixed-precision records: Horner form with fused multiply-adds (the
    // double-single split keeps ~48 bits, far more than the evaluation order
    // changes).  FP64 records: left-to-right sums of explicitly rounded
    // products, exactly the plain IEEE evaluation of the Taylor polynomial.
    const double d2 = 0.5 * dt, d3 = dt * (1.0 / 6.0), d4 = dt * (1.0 / 24.0);
    for (int c = 0; c < 3; ++c) {
        const int64_t q = 3 * j + c;
        const double x = js.x[q], v = js.v[q], a = js.a[q], jk = js.jk[q];
        if (ORDER == 2) {  // leap-frog (GRAPE-5): sources are used where they are
            xp[c] = x;
            vp[c] = 0.0;
        } else if (ORDER == 6 && js.cr) {
            // 6th-order block steps: the crackle term too (x to dt^5, v to
            // dt^4, a to dt^3), Horner form in both precisions
            const double s = js.sn[q], cr = js.cr[q];
            const double d5 = dt * (1.0 / 120.0);
            xp[c] = fma(fma(fma(fma(fma(cr, d5, s * (1.0 / 24.0)), dt, jk * (1.0 / 6.0)), dt, 0.5 * a), dt, v), dt, x);
            vp[c] = fma(fma(fma(fma(cr, d4, s * (1.0 / 6.0)), dt, 0.5 * jk), dt, a), dt, v);
            ap[c] = fma(fma(fma(cr, d3, 0.5 * s), dt, jk), dt, a);
        } else if (MIXED && ORDER == 6) {
            const double s = js.sn[q];
            xp[c] = fma(fma(fma(fma(s, d4, jk * (1.0 / 6.0)), dt, 0.5 * a), dt, v), dt, x);
            vp[c] = fma(fma(fma(s, d3, 0.5 * jk), dt, a), dt, v);
            ap[c] = fma(fma(s, d2, jk), dt, a);
        } else if (MIXED) {
            xp[c] = fma(fma(fma(jk, d3, 0.5 * a), dt, v), dt, x);
            vp[c] = fma(fma(jk, d2, a), dt, v);
        } else if (ORDER == 6) {
            const double s = js.sn[q];
            xp[c] = dadd(dadd(dadd(dadd(x, dmul(v, dt)), dmul(a, h2)), dmul(jk, h3)), dmul(s, h4));
            vp[c] = dadd(dadd(dadd(v, dmul(a, dt)), dmul(jk, h2)), dmul(s, h3));
            ap[c] = dadd(dadd(a, dmul(jk, dt)), dmul(s, h2));
        } else {
            xp[c] = dadd(dadd(dadd(x, dmul(v, dt)), dmul(a, h2)), dmul(jk, h3));
            vp[c] = dadd(dadd(v, dmul(a, dt)), dmul(jk, h2));
        }
    }
    const int rb = MIXED ? (ORDER == 6 ? 64 : 48) : (ORDER == 6 ? 96 : 64);
    if (MIXED) store_mixed(rec, rb, j, xp, vp, ORDER == 6 ? ap : nullptr, js.m[j], js.id[j]);
    else store_fp64(rec, rb, j, xp, vp, ORDER == 6 ? ap : nullptr, js.m[j], js.id[j]);
}

template <bool MIXED>
__global__ void pack_state_kernel(int64_t n, const double *m, const double *x, const double *v, unsigned char *rec) {
    const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double xp[3] = {x[3 * j], x[3 * j + 1], x[3 * j + 2]};
    const double vp[3] = {v[3 * j], v[3 * j + 1], v[3 * j + 2]};
    if (MIXED) store_mixed(rec, 48, j, xp, vp, nullptr, m[j], static_cast<int>(j));
    else store_fp64(rec, 64, j, xp, vp, nullptr, m[j], static_cast<int>(j));
}

// Neighbour lists after the pass: stored slots become ids and each list is
// sorted by id (insertion sort; lists are short), so a list without overflow
// has one defined order.
__global__ void nb_finish_kernel(const int32_t *ids, int64_t n_i, int nb_max, const int32_t *count, int32_t *list) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n_i) return;
    const int c = min(count[i], nb_max);
    int32_t *l = list + i * nb_max;
    for (int k = 0; k < c; ++k) {
        const int32_t v = ids[l[k]];
        int q = k;
        while (q > 0 && l[q - 1] > v) {
            l[q] = l[q - 1];
            --q;
        }
        l[q] = v;
    }
}

// ---- block time-steps (Sec. 3.7: Hermite integration with individual,
// power-of-two time-steps; the integrator around the force pass) ----------
//
// Aarseth's criterion (Aarseth 2003) with the higher derivatives of the
// Hermite interpolation over the last step [t0, t1] (Makino & Aarseth 1992):
//   a2(t0) = (-6 (a0 - a1) - dt (4 j0 + 2 j1)) / dt^2
//   a3     = (12 (a0 - a1) + 6 dt (j0 + j1)) / dt^3
//   a2(t1) = a2(t0) + dt a3
//   dt'    = sqrt(eta (|a1| |a2(t1)| + |j1|^2) / (|j1| |a3| + |a2(t1)|^2))
// quantised to the largest power of two not above dt', at most twice the last
// step and dt_max, and dividing t1 (so the blocks stay synchronised).
__device__ __forceinline__ double norm3(const double *p) { return sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]); }

__device__ __forceinline__ double quantise_dt(double want, double cap, double t1) {
    double d = cap;
    while (d > want && d > kBlockDtMin) d *= 0.5;
    // d = cap 2^-k divides t1 exactly iff fmod(t1, d) == 0.  With r = t1 / cap
    // (one correctly rounded division), a multiple t1 = m d gives r = m 2^-k
    // exactly for m < 2^53, so q = r 2^k (an exact scaling) is the integer m;
    // above 2^53 every double is an integer.  A fractional q therefore rules d
    // out, and the candidate that survives is confirmed exactly: t1 - q d by
    // one fused multiply-add (zero iff t1 = q d) below 2^53, fmod above.
    double q = (t1 / cap) * (cap / d);
    while (d > kBlockDtMin) {
        if (q == trunc(q)) {
            const bool exact = (fabs(q) < 9007199254740992.0) ? (fma(-q, d, t1) == 0.0) : (fmod(t1, d) == 0.0);
            if (exact) break;
        }
        d *= 0.5;
        q *= 2.0;
    }
    return d;
}

// initial steps at t0 from |a| / |j| (the usual start of a Hermite run)
__global__ void block_init_kernel(JStore js, double *dt, int64_t n, double eta_s, double dt_max, double t0) {
    const int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const double an = norm3(js.a + 3 * s), jn = norm3(js.jk + 3 * s);
    const double want = (jn > 0.0) ? eta_s * an / jn : dt_max;
    dt[s] = quantise_dt(want, dt_max, t0);
    js.t[s] = t0;
}

// Hermite-4 corrector and the next step for the active particles (a1, j1 at
// the predicted state, position k of the active list); the double-single
// cache follows the store.
__device__ __forceinline__ void correct_one(const JStore &js, double *dt, int64_t s, int64_t k, double t1,
                                            const double *a1, const double *j1, double eta, double dt_max) {
    const double h = t1 - js.t[s];
    const double h2 = h * h;
    double a2[3], a3[3], an[3], jn[3];
    for (int c = 0; c < 3; ++c) {
        const int64_t q = 3 * s + c;
        const double x0 = js.x[q], v0 = js.v[q], a0 = js.a[q], j0 = js.jk[q];
        const double aa = a1[3 * k + c], jj = j1[3 * k + c];
        const double v1 = v0 + (a0 + aa) * (h / 2) + (j0 - jj) * (h2 / 12);
        const double x1 = x0 + (v0 + v1) * (h / 2) + (a0 - aa) * (h2 / 12);
        const double a2_0 = (-6.0 * (a0 - aa) - h * (4.0 * j0 + 2.0 * jj)) / h2;
        a3[c] = (12.0 * (a0 - aa) + 6.0 * h * (j0 + jj)) / (h2 * h);
        a2[c] = a2_0 + h * a3[c];
        an[c] = aa;
        jn[c] = jj;
        js.x[q] = x1;
        js.v[q] = v1;
        js.a[q] = aa;
        js.jk[q] = jj;
    }
    js.t[s] = t1;
    const double A = norm3(an), J = norm3(jn), A2 = norm3(a2), A3 = norm3(a3);
    const double den = J * A3 + A2 * A2;
    const double want = (den > 0.0) ? sqrt(eta * (A * A2 + J * J) / den) : dt_max;
    dt[s] = quantise_dt(want, fmin(2.0 * h, dt_max), t1);
    if (js.dsc) write_dscache(js, s);
}

// A step at the 2^-50 floor means the criterion has collapsed (Sec. 3.7 notes
// that noisy jerk and snap can drive the step to zero): the run stops after
// this block and the host reports it.
__device__ __forceinline__ void check_underflow(const double *dt, int64_t s, BlockDev *bd) {
    if (dt[s] <= kBlockDtMin) {
        bd->underflow = 1u;
        bd->stop = 1u;
    }
}

// Explicit sinks (sp2_compute_ext): positions / velocities [/ accelerations]
// given by the caller, packed in the context's record format.
template <int ORDER, bool MIXED>
__global__ void pack_sinks_kernel(int64_t n, const double *x, const double *v, const double *a, unsigned char *rec) {
    const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double xp[3], vp[3], ap[3];
    for (int c = 0; c < 3; ++c) {
        xp[c] = x[3 * j + c];
        vp[c] = v ? v[3 * j + c] : 0.0;
        ap[c] = (ORDER == 6) ? a[3 * j + c] : 0.0;
    }
    const int rb = MIXED ? (ORDER == 6 ? 64 : 48) : (ORDER == 6 ? 96 : 64);
    if (MIXED) store_mixed(rec, rb, j, xp, vp, ORDER == 6 ? ap : nullptr, 0.0, -1);
    else store_fp64(rec, rb, j, xp, vp, ORDER == 6 ? ap : nullptr, 0.0, -1);
}

// ---- the same block time-steps driven from the device: the block time,
// the active count and a stop flag live in a BlockDev, so the host can queue
// many blocks without reading anything back.
__global__ void block_begin_kernel(BlockDev *bd) {
    bd->count = 0u;
    if (!bd->stop) bd->t1bits = ~0ull;
}

__global__ void block_next_dev_kernel(const double *t, const double *dt, int64_t n, BlockDev *bd) {
    if (bd->stop) return;
    const int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    unsigned long long v = ~0ull;
    if (s < n) v = static_cast<unsigned long long>(time_key(t[s] + dt[s]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, off));
    if ((threadIdx.x & 31) == 0 && v != ~0ull) atomicMin(&bd->t1bits, v);
}

// active set of the block, unless the block time has passed t_end (then the
// run stops: count stays 0 and every later kernel of the run does nothing)
__global__ void block_active_dev_kernel(const double *t, const double *dt, int64_t n, double t_end, BlockDev *bd,
                                        int32_t *active) {
    if (bd->stop) return;
    const double t1 = key_time(bd->t1bits);
    if (!(t1 <= t_end)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) bd->stop = 1u;
        return;
    }
    const int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s < n && t[s] + dt[s] == t1) active[atomicAdd(&bd->count, 1u)] = static_cast<int32_t>(s);
}

__global__ void block_correct_dev_kernel(JStore js, double *dt, const int32_t *active, BlockDev *bd, const double *a1,
                                         const double *j1, double eta, double dt_max) {
    const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const unsigned int n_act = bd->count;
    const double t1 = key_time(bd->t1bits);
    if (k == 0 && n_act > 0) {
        bd->steps += 1;
        bd->active_sum += n_act;
        bd->max_active = max(bd->max_active, n_act);
        bd->min_active = min(bd->min_active, n_act);
        bd->t_last = t1;
    }
    if (k >= n_act) return;
    correct_one(js, dt, active[k], k, t1, a1, j1, eta, dt_max);
    check_underflow(dt, active[k], bd);
}

// 6th-order Hermite corrector (Nitadori & Makino 2008) for slot s, position k
// of the active list: the quintic Hermite interpolant of the acceleration
// through (a, j, s) at both ends, integrated once for v and, with (v, a, j),
// for x; its 3rd to 5th derivatives at t1 (crackle, pop, and the constant
// fifth derivative q) follow from the three matching conditions at t1:
//   c1 h^3 = 60 (a1 - a0) - 24 h j0 - 36 h j1 - 3 h^2 s0 + 9 h^2 s1
//   p1 h^4 = 360 (a1 - a0) - 168 h j0 - 192 h j1 - 24 h^2 s0 + 36 h^2 s1
//   q  h^5 = 720 (a1 - a0) - 360 h (j0 + j1) - 60 h^2 (s0 - s1).
// The next step is the mean of Aarseth's criterion (eta4 inside the root),
// evaluated as the 4th-order scheme does from a and jerk at both ends (the
// 2nd and 3rd derivatives at t1 of their cubic Hermite interpolant), and its
// 6th-order generalisation (eta6 times the sixth root) with the pass's snap
// and the quintic interpolant's crackle, pop and 5th derivative, quantised
// like the 4th-order step.  Only the 6th-order half sees the h^-5
// amplification of force noise in the interpolated derivatives.
__device__ __forceinline__ void correct6_one(const JStore &js, double *dt, int64_t s, int64_t k, double t1,
                                             const double *a1, const double *j1, const double *s1, double eta4,
                                             double eta6, double dt_max) {
    const double h = t1 - js.t[s];
    const double h2 = h * h, h3 = h2 * h;
    const double ih3 = 1.0 / h3, ih4 = ih3 / h, ih5 = ih4 / h;
    double an[3], jn[3], sn[3], cn[3], pn[3], qn[3], a2[3], a3[3];
    for (int c = 0; c < 3; ++c) {
        const int64_t q = 3 * s + c;
        const double x0 = js.x[q], v0 = js.v[q], a0 = js.a[q], j0 = js.jk[q], s0 = js.sn[q];
        const double aa = a1[3 * k + c], jj = j1[3 * k + c], ss = s1[3 * k + c];
        const double v1 = v0 + (a0 + aa) * (h / 2) - (jj - j0) * (h2 / 10) + (s0 + ss) * (h3 / 120);
        const double x1 = x0 + (v0 + v1) * (h / 2) - (aa - a0) * (h2 / 10) + (j0 + jj) * (h3 / 120);
        const double da = aa - a0;
        cn[c] = (60.0 * da - h * (24.0 * j0 + 36.0 * jj) + h2 * (9.0 * ss - 3.0 * s0)) * ih3;
        pn[c] = (360.0 * da - h * (168.0 * j0 + 192.0 * jj) + h2 * (36.0 * ss - 24.0 * s0)) * ih4;
        qn[c] = (720.0 * da - 360.0 * h * (j0 + jj) - 60.0 * h2 * (s0 - ss)) * ih5;
        a3[c] = (12.0 * (a0 - aa) + 6.0 * h * (j0 + jj)) / h3;
        a2[c] = (-6.0 * (a0 - aa) - h * (4.0 * j0 + 2.0 * jj)) / h2 + h * a3[c];
        an[c] = aa;
        jn[c] = jj;
        sn[c] = ss;
        js.x[q] = x1;
        js.v[q] = v1;
        js.a[q] = aa;
        js.jk[q] = jj;
        js.sn[q] = ss;
        js.cr[q] = cn[c];
    }
    js.t[s] = t1;
    const double A = norm3(an), J = norm3(jn), S = norm3(sn), C = norm3(cn), P = norm3(pn), Q = norm3(qn);
    const double A2 = norm3(a2), A3 = norm3(a3);
    const double d4 = J * A3 + A2 * A2, d6 = C * Q + P * P;
    const double want = (d4 > 0.0 && d6 > 0.0)
                            ? 0.5 * (sqrt(eta4 * (A * A2 + J * J) / d4) + eta6 * pow((A * S + J * J) / d6, 1.0 / 6.0))
                            : dt_max;
    dt[s] = quantise_dt(want, fmin(2.0 * h, dt_max), t1);
    if (js.dsc) write_dscache(js, s);
}

__global__ void block_correct6_dev_kernel(JStore js, double *dt, const int32_t *active, BlockDev *bd,
                                          const double *a1, const double *j1, const double *s1, double eta4,
                                          double eta6, double dt_max) {
    const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const unsigned int n_act = bd->count;
    const double t1 = key_time(bd->t1bits);
    if (k == 0 && n_act > 0) {
        bd->steps += 1;
        bd->active_sum += n_act;
        bd->max_active = max(bd->max_active, n_act);
        bd->min_active = min(bd->min_active, n_act);
        bd->t_last = t1;
    }
    if (k >= n_act) return;
    correct6_one(js, dt, active[k], k, t1, a1, j1, s1, eta4, eta6, dt_max);
    check_underflow(dt, active[k], bd);
}

__global__ void iota_kernel(int32_t *dst, int64_t n) {
    const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j < n) dst[j] = static_cast<int32_t>(j);
}

// Hermite-4 predictor of the shared-step scheme (to t + dt), packed as records.
template <bool MIXED>
__global__ void h4_predict_pack_kernel(int64_t n, double dt, const double *m, const double *x, const double *v,
                                       const double *a, const double *jk, unsigned char *rec) {
    const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double h2 = dt * dt * 0.5, h3 = dt * dt * dt * (1.0 / 6.0);
    double xp[3], vp[3];
    for (int c = 0; c < 3; ++c) {
        const int64_t q = 3 * j + c;
        xp[c] = x[q] + v[q] * dt + a[q] * h2 + jk[q] * h3;
        vp[c] = v[q] + a[q] * dt + jk[q] * h2;
    }
    if (MIXED) store_mixed(rec, 48, j, xp, vp, nullptr, m[j], static_cast<int>(j));
    else store_fp64(rec, 64, j, xp, vp, nullptr, m[j], static_cast<int>(j));
}

// Hermite-4 corrector (Makino & Aarseth 1992), in place; a1, j1 at the predicted state.
__global__ void h4_correct_kernel(int64_t n3, double dt, double *x, double *v, double *a, double *jk,
                                  const double *a1, const double *j1) {
    const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= n3) return;
    const double h = 0.5 * dt, h12 = dt * dt / 12.0;
    const double v1 = v[q] + (a[q] + a1[q]) * h + (jk[q] - j1[q]) * h12;
    x[q] = x[q] + (v[q] + v1) * h + (a[q] - a1[q]) * h12;
    v[q] = v1;
    a[q] = a1[q];
    jk[q] = j1[q];
}

__device__ __forceinline__ void store_vjp(bool mixed, unsigned char *rec, int64_t j, const double *xp, const double *vp,
                                          const double *ab, const double *jb, double pb, double m) {
    if (mixed) {
        float xh[3], xl[3];
        for (int c = 0; c < 3; ++c) {
        const ds q = ds_split(xp[c]);  // hi = fl32(x), lo = fl32(x - hi)
        xh[c] = q.h;
        xl[c] = q.l;
    }
        float4 *o = reinterpret_cast<float4 *>(rec + j * 80);
        o[0] = make_float4(xh[0], xh[1], xh[2], __double2float_rn(m));
        o[1] = make_float4(xl[0], xl[1], xl[2], __double2float_rn(pb));
        o[2] = make_float4(__double2float_rn(vp[0]), __double2float_rn(vp[1]), __double2float_rn(vp[2]), 0.f);
        o[3] = make_float4(__double2float_rn(ab[0]), __double2float_rn(ab[1]), __double2float_rn(ab[2]), 0.f);
        o[4] = make_float4(__double2float_rn(jb[0]), __double2float_rn(jb[1]), __double2float_rn(jb[2]), 0.f);
    } else {
        double2 *o = reinterpret_cast<double2 *>(rec + j * 112);
        o[0] = make_double2(xp[0], xp[1]);
        o[1] = make_double2(xp[2], m);
        o[2] = make_double2(vp[0], vp[1]);
        o[3] = make_double2(vp[2], pb);
        o[4] = make_double2(ab[0], ab[1]);
        o[5] = make_double2(ab[2], jb[0]);
        o[6] = make_double2(jb[1], jb[2]);
    }
}

template <bool MIXED>
__global__ void pack_vjp_kernel(int64_t n, const double *m, const double *x, const double *v, const double *abar,
                                const double *jbar, const double *pbar, unsigned char *rec) {
    const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double zero[3] = {0.0, 0.0, 0.0};
    const double *ab = abar ? abar + 3 * j : zero;
    const double *jb = jbar ? jbar + 3 * j : zero;
    store_vjp(MIXED, rec, j, x + 3 * j, v + 3 * j, ab, jb, pbar ? pbar[j] : 0.0, m[j]);
}

// Reverse of the corrector for the output cotangents (gx, gv, ga, gj):
//   gv1 = gv + gx dt/2,  ga1 = ga + gv1 dt/2 - gx dt^2/12,  gj1 = gj - gv1 dt^2/12
// are the cotangents of the force outputs (a1, j1) at the predicted state,
// which is recomputed here and packed with them into VJP records.
template <bool MIXED>
__global__ void h4_vjp_pre_kernel(int64_t n, double dt, const double *m, const double *x, const double *v,
                                  const double *a, const double *jk, const double *gx, const double *gv,
                                  const double *ga, const double *gj, unsigned char *rec) {
    const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double h2 = dt * dt * 0.5, h3 = dt * dt * dt * (1.0 / 6.0), h12 = dt * dt / 12.0;
    double xp[3], vp[3], ab[3], jb[3];
    for (int c = 0; c < 3; ++c) {
        const int64_t q = 3 * j + c;
        xp[c] = x[q] + v[q] * dt + a[q] * h2 + jk[q] * h3;
        vp[c] = v[q] + a[q] * dt + jk[q] * h2;
        const double gv1 = gv[q] + gx[q] * (0.5 * dt);
        ab[c] = ga[q] + gv1 * (0.5 * dt) - gx[q] * h12;
        jb[c] = gj[q] - gv1 * h12;
    }
    store_vjp(MIXED, rec, j, xp, vp, ab, jb, 0.0, m[j]);
}

// Combine: cotangents of the step inputs from the output cotangents and the
// force VJP (xpbar, vpbar) at the predicted state.
__global__ void h4_vjp_post_kernel(int64_t n3, double dt, const double *xpbar, const double *vpbar, double *gx,
                                   double *gv, double *ga, double *gj) {
    const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= n3) return;
    const double h = 0.5 * dt, h2 = dt * dt * 0.5, h3 = dt * dt * dt * (1.0 / 6.0), h12 = dt * dt / 12.0;
    const double gx1 = gx[q];
    const double gv1 = gv[q] + gx1 * h;
    const double xb = xpbar[q], vb = vpbar[q];
    gx[q] = gx1 + xb;
    gv[q] = gx1 * h + gv1 + xb * dt + vb;
    ga[q] = gx1 * h12 + gv1 * h + xb * h2 + vb * dt;
    gj[q] = gv1 * h12 + xb * h3 + vb * h2;
}

__global__ void scan_finite_kernel(const double *p, int64_t n, unsigned int *flag) {
    const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q < n && !isfinite(p[q])) atomicOr(flag, 1u);
}

}  // namespace

cudaError_t launch_scatter_j(const JStore &dst, const int32_t *slots, int64_t n, int64_t n_loaded, unsigned int *err,
                             const int32_t *id, const double *m, const double *x, const double *v, const double *a,
                             const double *jk, const double *sn, const double *t, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    scatter_kernel<<<grid_for(n), kThreads, 0, s>>>(dst, slots, n, n_loaded, err, id, m, x, v, a, jk, sn, t);
    return cudaGetLastError();
}

cudaError_t launch_dscache(int order, const JStore &js, int64_t first, int64_t n, cudaStream_t s) {
    if (n <= 0 || !js.dsc) return cudaSuccess;
    (void)order;
    dscache_kernel<<<grid_for(n), kThreads, 0, s>>>(js, first, n);
    return cudaGetLastError();
}

cudaError_t launch_predict(int order, int mixed, const JStore &js, int64_t n, double t, unsigned char *rec,
                           cudaStream_t s, const BlockDev *bd) {
    if (n <= 0) return cudaSuccess;
    const unsigned g = grid_for(n);
    if (mixed && js.dsc) {
        const float th = static_cast<float>(t);
        const float tl = static_cast<float>(t - static_cast<double>(th));
        if (order == 6) predict_ds_kernel<6><<<g, kThreads, 0, s>>>(js.dsc, n, th, tl, rec, bd);
        else if (order == 2) predict_ds_kernel<2><<<g, kThreads, 0, s>>>(js.dsc, n, th, tl, rec, bd);
        else predict_ds_kernel<4><<<g, kThreads, 0, s>>>(js.dsc, n, th, tl, rec, bd);
        return cudaGetLastError();
    }
    // the FP64 predictor is FP64-bound: 64-thread CTAs spread it over the SMs
    const unsigned g64 = static_cast<unsigned>((n + 63) / 64);
    if (order == 6) {
        if (mixed) predict_kernel<6, true><<<g64, 64, 0, s>>>(js, n, t, rec, bd);
        else predict_kernel<6, false><<<g64, 64, 0, s>>>(js, n, t, rec, bd);
    } else if (order == 2) {
        if (mixed) predict_kernel<2, true><<<g64, 64, 0, s>>>(js, n, t, rec, bd);
        else predict_kernel<2, false><<<g64, 64, 0, s>>>(js, n, t, rec, bd);
    } else {
        if (mixed) predict_kernel<4, true><<<g64, 64, 0, s>>>(js, n, t, rec, bd);
        else predict_kernel<4, false><<<g64, 64, 0, s>>>(js, n, t, rec, bd);
    }
    return cudaGetLastError();
}

cudaError_t launch_pack_state(int mixed, int64_t n, const double *m, const double *x, const double *v,
                              unsigned char *rec, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (mixed) pack_state_kernel<true><<<grid_for(n), kThreads, 0, s>>>(n, m, x, v, rec);
    else pack_state_kernel<false><<<grid_for(n), kThreads, 0, s>>>(n, m, x, v, rec);
    return cudaGetLastError();
}

cudaError_t launch_pack_sinks(int order, int mixed, int64_t n, const double *x, const double *v, const double *a,
                              unsigned char *rec, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const unsigned g = grid_for(n);
    if (order == 6) {
        if (mixed) pack_sinks_kernel<6, true><<<g, kThreads, 0, s>>>(n, x, v, a, rec);
        else pack_sinks_kernel<6, false><<<g, kThreads, 0, s>>>(n, x, v, a, rec);
    } else {
        if (mixed) pack_sinks_kernel<4, true><<<g, kThreads, 0, s>>>(n, x, v, a, rec);
        else pack_sinks_kernel<4, false><<<g, kThreads, 0, s>>>(n, x, v, a, rec);
    }
    return cudaGetLastError();
}

cudaError_t launch_iota(int32_t *dst, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    iota_kernel<<<grid_for(n), kThreads, 0, s>>>(dst, n);
    return cudaGetLastError();
}

cudaError_t launch_block_begin(BlockDev *bd, const double *t, const double *dt, int64_t n, double t_end,
                               int32_t *active, cudaStream_t s) {
    block_begin_kernel<<<1, 1, 0, s>>>(bd);
    block_next_dev_kernel<<<grid_for(n), kThreads, 0, s>>>(t, dt, n, bd);
    block_active_dev_kernel<<<grid_for(n), kThreads, 0, s>>>(t, dt, n, t_end, bd, active);
    return cudaGetLastError();
}

cudaError_t launch_block_correct_dev(const JStore &js, double *dt, const int32_t *active, int64_t n_max,
                                     BlockDev *bd, const double *a1, const double *j1, double eta, double dt_max,
                                     cudaStream_t s) {
    if (n_max <= 0) return cudaSuccess;
    block_correct_dev_kernel<<<grid_for_warps(n_max), kWarpCta, 0, s>>>(js, dt, active, bd, a1, j1, eta, dt_max);
    return cudaGetLastError();
}

cudaError_t launch_block_correct6_dev(const JStore &js, double *dt, const int32_t *active, int64_t n_max,
                                      BlockDev *bd, const double *a1, const double *j1, const double *s1,
                                      double eta4, double eta6, double dt_max, cudaStream_t s) {
    if (n_max <= 0) return cudaSuccess;
    block_correct6_dev_kernel<<<grid_for_warps(n_max), kWarpCta, 0, s>>>(js, dt, active, bd, a1, j1, s1, eta4, eta6,
                                                                       dt_max);
    return cudaGetLastError();
}

cudaError_t launch_block_init(const JStore &js, double *dt, int64_t n, double eta_s, double dt_max, double t0,
                              cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    block_init_kernel<<<grid_for(n), kThreads, 0, s>>>(js, dt, n, eta_s, dt_max, t0);
    return cudaGetLastError();
}

cudaError_t launch_nb_finish(const int32_t *ids, int64_t n_i, int nb_max, const int32_t *count, int32_t *list,
                             cudaStream_t s) {
    if (n_i <= 0) return cudaSuccess;
    nb_finish_kernel<<<grid_for(n_i), kThreads, 0, s>>>(ids, n_i, nb_max, count, list);
    return cudaGetLastError();
}

cudaError_t launch_h4_predict_pack(int mixed, int64_t n, double dt, const double *m, const double *x,
                                   const double *v, const double *a, const double *jk, unsigned char *rec,
                                   cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (mixed) h4_predict_pack_kernel<true><<<grid_for(n), kThreads, 0, s>>>(n, dt, m, x, v, a, jk, rec);
    else h4_predict_pack_kernel<false><<<grid_for(n), kThreads, 0, s>>>(n, dt, m, x, v, a, jk, rec);
    return cudaGetLastError();
}

cudaError_t launch_h4_correct(int64_t n, double dt, double *x, double *v, double *a, double *jk, const double *a1,
                              const double *j1, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    h4_correct_kernel<<<grid_for(3 * n), kThreads, 0, s>>>(3 * n, dt, x, v, a, jk, a1, j1);
    return cudaGetLastError();
}

cudaError_t launch_h4_vjp_pre(int mixed, int64_t n, double dt, const double *m, const double *x, const double *v,
                              const double *a, const double *jk, const double *gx, const double *gv,
                              const double *ga, const double *gj, unsigned char *vrec, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (mixed) h4_vjp_pre_kernel<true><<<grid_for(n), kThreads, 0, s>>>(n, dt, m, x, v, a, jk, gx, gv, ga, gj, vrec);
    else h4_vjp_pre_kernel<false><<<grid_for(n), kThreads, 0, s>>>(n, dt, m, x, v, a, jk, gx, gv, ga, gj, vrec);
    return cudaGetLastError();
}

cudaError_t launch_h4_vjp_post(int64_t n, double dt, const double *xpbar, const double *vpbar, double *gx,
                               double *gv, double *ga, double *gj, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    h4_vjp_post_kernel<<<grid_for(3 * n), kThreads, 0, s>>>(3 * n, dt, xpbar, vpbar, gx, gv, ga, gj);
    return cudaGetLastError();
}

cudaError_t launch_pack_vjp(int mixed, int64_t n, const double *m, const double *x, const double *v,
                            const double *abar, const double *jbar, const double *pbar, unsigned char *vrec,
                            cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (mixed) pack_vjp_kernel<true><<<grid_for(n), kThreads, 0, s>>>(n, m, x, v, abar, jbar, pbar, vrec);
    else pack_vjp_kernel<false><<<grid_for(n), kThreads, 0, s>>>(n, m, x, v, abar, jbar, pbar, vrec);
    return cudaGetLastError();
}

cudaError_t launch_scan_finite(const double *p, int64_t n, unsigned int *flag, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    scan_finite_kernel<<<grid_for(n), kThreads, 0, s>>>(p, n, flag);
    return cudaGetLastError();
}

}  // namespace sp2
