// sp2_ds.cuh -- double-single arithmetic and the mixed-precision predictor
// of one particle from the double-single cache (shared by the predictor
// kernel and the force pass that predicts its sources in place).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sp2 {

// ---- double-single arithmetic (Dekker 1971; Knuth's TwoSum; TwoProd by FMA).
// Every step is explicitly rounded so no multiply-add is fused behind our back.
struct ds {
    float h, l;
};
__device__ __forceinline__ ds two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ ds fast_two_sum(float a, float b) {  // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ds ds_add(ds a, ds b) {
    ds s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ ds ds_add_f(ds a, float b) {
    ds s = two_sum(a.h, b);
    return fast_two_sum(s.h, __fadd_rn(s.l, a.l));
}
__device__ __forceinline__ ds ds_mul(ds a, ds b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
    return fast_two_sum(p, e);
}
__device__ __forceinline__ ds ds_split(double x) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - static_cast<double>(h))};
}


// The FP64 value of an FP32 number, formed from its bits with integer
// operations (every FP32 value is exactly a double, so this equals the
// conversion instruction, subnormals and infinities included) -- GB300 runs
// FP64 and its conversions at 1/64 of the FP32 rate, and the kernels'
// epilogues convert many double-single totals.
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned long long sign = static_cast<unsigned long long>(u & 0x80000000u) << 32;
    const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    unsigned long long bits;
    if (e == 0xffu) {  // inf / nan
        bits = sign | 0x7ff0000000000000ull | (static_cast<unsigned long long>(m) << 29);
    } else if (e != 0u) {  // normal: rebias the exponent (127 -> 1023)
        bits = sign | (static_cast<unsigned long long>(e + 896u) << 52) | (static_cast<unsigned long long>(m) << 29);
    } else if (m == 0u) {  // signed zero
        bits = sign;
    } else {  // subnormal m 2^-149 with its leading one at bit p
        const unsigned p = 31u - static_cast<unsigned>(__clz(m));
        bits = sign | (static_cast<unsigned long long>(p + 874u) << 52) |
               ((static_cast<unsigned long long>(m) << (52u - p)) & 0xfffffffffffffull);
    }
    return __longlong_as_double(static_cast<long long>(bits));
}

// Words of particle j's double-single cache entry (layout in sp2_internal.h)
// that the predictor uses, loaded into w[0 .. dscache_words) (order 2: words
// 0, 1 and 3 only).
template <int ORDER>
__device__ __forceinline__ void ds_fetch(const float4 *dsc, int64_t j, float4 *w) {
    constexpr int W = (ORDER == 6) ? 8 : 7;
    const float4 *q = dsc + j * W;
    if (ORDER == 2) {
        w[0] = __ldg(q);
        w[1] = __ldg(q + 1);
        w[3] = __ldg(q + 3);
        return;
    }
#pragma unroll
    for (int k = 0; k < W; ++k) w[k] = __ldg(q + k);
}

// Mixed-precision prediction of a particle from the cache words ds_fetch
// loaded: positions
//   x_p = x + dt (v + dt (a/2 + dt (j/6 [+ dt s/24])))
// with x, v, a/2 and dt double-single and the jerk / snap terms in FP32 (they
// enter multiplied by dt^3, far below the double-single resolution of x);
// velocities and accelerations leave as FP32.  Writes the predicted record's
// 16-byte words {xh yh zh m}{xl yl zl id}{v 0}[{a 0}] to o[0..3].
template <int ORDER>
__device__ __forceinline__ void predict_ds_words(const float4 *w, float t_hi, float t_lo, float4 *o) {
    if (ORDER == 2) {  // leap-frog (GRAPE-5) sources are used where they are
        o[0] = w[0];
        o[1] = make_float4(w[1].x, w[1].y, w[1].z, w[3].w);
        o[2] = o[3] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const float4 w0 = w[0], w1 = w[1], w2 = w[2], w3 = w[3], w4 = w[4], w5 = w[5], w6 = w[6];
    float4 w7 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ORDER == 6) w7 = w[7];
    const ds dt = ds_add({t_hi, t_lo}, {-w1.w, -w2.w});
    const float xh[3] = {w0.x, w0.y, w0.z}, xl[3] = {w1.x, w1.y, w1.z};
    const float vh[3] = {w2.x, w2.y, w2.z}, vl[3] = {w3.x, w3.y, w3.z};
    const float ah[3] = {w4.x, w4.y, w4.z}, al[3] = {w5.x, w5.y, w5.z};
    const float jk[3] = {w6.x, w6.y, w6.z}, sn[3] = {w7.x, w7.y, w7.z};
    float oh[3], ol[3], ov[3], oa[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float jx = (ORDER == 6) ? fmaf(dt.h * (1.f / 24.f), sn[c], jk[c] * (1.f / 6.f)) : jk[c] * (1.f / 6.f);
        const ds cx = ds_add_f({0.5f * ah[c], 0.5f * al[c]}, dt.h * jx);
        const ds bx = ds_add({vh[c], vl[c]}, ds_mul(dt, cx));
        const ds px = ds_add({xh[c], xl[c]}, ds_mul(dt, bx));
        oh[c] = px.h;
        ol[c] = px.l;
        const float jv = (ORDER == 6) ? fmaf(dt.h * (1.f / 6.f), sn[c], 0.5f * jk[c]) : 0.5f * jk[c];
        ov[c] = vh[c] + fmaf(dt.h, fmaf(dt.h, jv, ah[c] + al[c]), vl[c]);
        oa[c] = (ORDER == 6) ? ah[c] + fmaf(dt.h, fmaf(dt.h, 0.5f * sn[c], jk[c]), al[c]) : 0.f;
    }
    o[0] = make_float4(oh[0], oh[1], oh[2], w0.w);
    o[1] = make_float4(ol[0], ol[1], ol[2], w3.w);
    o[2] = make_float4(ov[0], ov[1], ov[2], 0.f);
    o[3] = make_float4(oa[0], oa[1], oa[2], 0.f);
}

// Both steps for particle j of the cache.
template <int ORDER>
__device__ __forceinline__ void predict_ds_record(const float4 *dsc, int64_t j, float t_hi, float t_lo, float4 *o) {
    float4 w[8];
    ds_fetch<ORDER>(dsc, j, w);
    predict_ds_words<ORDER>(w, t_hi, t_lo, o);
}

}  // namespace sp2
