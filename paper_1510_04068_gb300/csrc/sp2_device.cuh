// sp2_device.cuh -- device code of the pairwise passes: predicted-record
// layouts, the two precision policies (double-single "mixed" and FP64), the
// adjoint policies, and the persistent kernel skeleton with its work queue,
// the split-j reduction and the batched few-body kernel.
//
// Method (Sec. 2.1 of the paper): one thread (or j_lanes threads, the paper's
// 2D thread blocks) per sink, the sources of a slice streamed through shared
// memory; when the sinks are few the sources are split into slices (the
// source-split method) so that every SM has work, and the slices are combined
// in a fixed order, either by the last CTA of each block of sinks to finish
// (found with an atomic counter) or by a second kernel (Sec. 2.2.4 describes
// a two-kernel form and an atomic form); either way the result does not
// depend on scheduling.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sp2_ds.cuh"
#include "sp2_internal.h"

namespace sp2 {

constexpr int kStages = 3;          // shared-memory pipeline depth (cp.async ring of records)
constexpr int kFusedStages = 2;     // bulk-copy ring of cache words (fused prediction), at most
constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxThreads = 256;

__device__ __forceinline__ float f_inf() { return __int_as_float(0x7f800000); }
__device__ __forceinline__ double d_inf() { return __longlong_as_double(0x7ff0000000000000LL); }

// 16-byte asynchronous global->shared copy (L2 only), grouped and awaited per stage.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
// bring the L1 line holding p in ahead of its load
__device__ __forceinline__ void prefetch_l1(const void *p) {
    asm volatile("prefetch.global.L1 [%0];\n" ::"l"(p));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Bulk asynchronous copies (TMA, no tensor map) into shared memory, completed
// on an mbarrier: one thread arms the barrier with the byte count and issues
// the copies; every thread then waits on the barrier's phase.
__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// make the barrier initialisation visible to the copy engine
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// order this thread's earlier shared-memory accesses before later bulk copies into it
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arm(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// bytes and both addresses multiples of 16
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile("{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, q;\n\t}\n"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// Wait for the barrier's phase `parity` to complete, giving up after
// kMbarWaitLimit polls (each poll may suspend the thread for a short while).
constexpr int kMbarWaitLimit = 1 << 20;
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
    for (int it = 0; it < kMbarWaitLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Drop the 128-byte L2 lines that lie wholly inside [lo, hi) without writing
// them back (their contents are not needed again); lines shared with
// neighbouring data are kept.  Called by all threads of a CTA.
__device__ __forceinline__ void discard_l2_range(const void *lo, const void *hi) {
    const uintptr_t a = (reinterpret_cast<uintptr_t>(lo) + 127u) & ~static_cast<uintptr_t>(127u);
    const uintptr_t e = reinterpret_cast<uintptr_t>(hi) & ~static_cast<uintptr_t>(127u);
    for (uintptr_t q = a + static_cast<uintptr_t>(threadIdx.x) * 128u; q < e; q += static_cast<uintptr_t>(blockDim.x) * 128u)
        asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(q) : "memory");
}

__device__ __forceinline__ uint4 f4bits(float a, float b, float c, float d) {
    return make_uint4(__float_as_uint(a), __float_as_uint(b), __float_as_uint(c), __float_as_uint(d));
}
__device__ __forceinline__ uint4 d2bits(double a, double b) {
    const unsigned long long x = static_cast<unsigned long long>(__double_as_longlong(a));
    const unsigned long long y = static_cast<unsigned long long>(__double_as_longlong(b));
    return make_uint4(static_cast<unsigned>(x), static_cast<unsigned>(x >> 32), static_cast<unsigned>(y),
                      static_cast<unsigned>(y >> 32));
}

// Packed FP32 pairs (f32x2): one instruction performs the same IEEE operation
// on both halves, each rounded as the scalar instruction would be.  The FMA
// pipe's lane throughput is unchanged, but a pair costs one issue slot, which
// leaves the others to the SFU, integer and shared-memory instructions.
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    float2 d;
    asm("{.reg .b64 pa, pb, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "add.rn.ftz.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 d;
    asm("{.reg .b64 pa, pb, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "sub.rn.ftz.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    float2 d;
    asm("{.reg .b64 pa, pb, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "mul.rn.ftz.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
// a * b + c with one rounding per half
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{.reg .b64 pa, pb, pc, pd;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "mov.b64 pc, {%6, %7};\n\tfma.rn.ftz.f32x2 pd, pa, pb, pc;\n\tmov.b64 {%0, %1}, pd;}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// Double-single steps on f32x2 pairs: two particles' values side by side,
// each half rounded exactly as the scalar steps of sp2_ds.cuh round it.
// The error-free steps need every product that feeds a sum rounded on its
// own; the code generator has been seen to fuse a packed multiply into a
// following packed add despite the explicit rounding mode (measured: the
// last bits of the low words then differ from the scalar predictor's), so
// such products are formed with scalar multiplies, which it leaves alone.
__device__ __forceinline__ float2 mul2_sep(float2 a, float2 b) {
    return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y));
}
struct ds2 {
    float2 h, l;
};
__device__ __forceinline__ ds2 two_sum2(float2 a, float2 b) {
    const float2 s = add2(a, b);
    const float2 bb = sub2(s, a);
    return {s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}
__device__ __forceinline__ ds2 fast_two_sum2(float2 a, float2 b) {
    const float2 s = add2(a, b);
    return {s, sub2(b, sub2(s, a))};
}
__device__ __forceinline__ ds2 ds_add2(ds2 a, ds2 b) {
    const ds2 s = two_sum2(a.h, b.h);
    return fast_two_sum2(s.h, add2(s.l, add2(a.l, b.l)));
}
__device__ __forceinline__ ds2 ds_add_f2(ds2 a, float2 b) {
    const ds2 s = two_sum2(a.h, b);
    return fast_two_sum2(s.h, add2(s.l, a.l));
}
__device__ __forceinline__ ds2 ds_mul2(ds2 a, ds2 b) {
    const float2 p = mul2_sep(a.h, b.h);
    float2 e = fma2(a.h, b.h, make_float2(-p.x, -p.y));
    e = fma2(a.h, b.l, fma2(a.l, b.h, e));
    return fast_two_sum2(p, e);
}

// predict_ds_words (sp2_ds.cuh) for two particles at once, a in the .x halves
// and b in the .y halves: the same operations in the same order, so each
// record equals the scalar predictor's bit for bit.
template <int ORDER>
__device__ __forceinline__ void predict_ds_words2(const float4 *wa, const float4 *wb, float t_hi, float t_lo,
                                                  float4 *oa, float4 *ob) {
    if (ORDER == 2) {
        predict_ds_words<ORDER>(wa, t_hi, t_lo, oa);
        predict_ds_words<ORDER>(wb, t_hi, t_lo, ob);
        return;
    }
    auto pk = [](const float4 &x, const float4 &y, int c) {
        return c == 0 ? make_float2(x.x, y.x) : (c == 1 ? make_float2(x.y, y.y) : make_float2(x.z, y.z));
    };
    const ds2 dt = ds_add2(ds2{dup2(t_hi), dup2(t_lo)}, ds2{make_float2(-wa[1].w, -wb[1].w), make_float2(-wa[2].w, -wb[2].w)});
    const float2 half = dup2(0.5f), sixth = dup2(1.f / 6.f), c24 = dup2(1.f / 24.f);
    float2 oh[3], ol[3], ov[3], oc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 xh = pk(wa[0], wb[0], c), xl = pk(wa[1], wb[1], c);
        const float2 vh = pk(wa[2], wb[2], c), vl = pk(wa[3], wb[3], c);
        const float2 ah = pk(wa[4], wb[4], c), al = pk(wa[5], wb[5], c);
        const float2 jk = pk(wa[6], wb[6], c);
        float2 sn = dup2(0.f);
        if constexpr (ORDER == 6) sn = pk(wa[7], wb[7], c);
        const float2 jx = (ORDER == 6) ? fma2(mul2(dt.h, c24), sn, mul2(jk, sixth)) : mul2(jk, sixth);
        // (the halvings are exact, so a fused form of them rounds alike)
        const ds2 cx = ds_add_f2(ds2{mul2(half, ah), mul2(half, al)}, mul2_sep(dt.h, jx));
        const ds2 bx = ds_add2(ds2{vh, vl}, ds_mul2(dt, cx));
        const ds2 px = ds_add2(ds2{xh, xl}, ds_mul2(dt, bx));
        oh[c] = px.h;
        ol[c] = px.l;
        const float2 jv = (ORDER == 6) ? fma2(mul2(dt.h, sixth), sn, mul2(half, jk)) : mul2(half, jk);
        ov[c] = add2(vh, fma2(dt.h, fma2(dt.h, jv, add2(ah, al)), vl));
        oc[c] = (ORDER == 6) ? add2(ah, fma2(dt.h, fma2(dt.h, mul2(half, sn), jk), al)) : dup2(0.f);
    }
    oa[0] = make_float4(oh[0].x, oh[1].x, oh[2].x, wa[0].w);
    ob[0] = make_float4(oh[0].y, oh[1].y, oh[2].y, wb[0].w);
    oa[1] = make_float4(ol[0].x, ol[1].x, ol[2].x, wa[3].w);
    ob[1] = make_float4(ol[0].y, ol[1].y, ol[2].y, wb[3].w);
    oa[2] = make_float4(ov[0].x, ov[1].x, ov[2].x, 0.f);
    ob[2] = make_float4(ov[0].y, ov[1].y, ov[2].y, 0.f);
    oa[3] = make_float4(oc[0].x, oc[1].x, oc[2].x, 0.f);
    ob[3] = make_float4(oc[0].y, oc[1].y, oc[2].y, 0.f);
}

// Policies whose chunk fold reads the chunk's records (batched kernel).
template <class P, class = void>
struct has_fold_tile { static constexpr bool value = false; };
template <class P>
struct has_fold_tile<P, decltype(void(&P::fold_tile))> { static constexpr bool value = true; };

// Force policies whose sinks several warps may share define kSharedSinks = true.
template <class P, class = void>
struct shares_sinks { static constexpr bool value = false; };
template <class P>
struct shares_sinks<P, decltype(void(P::kSharedSinks))> { static constexpr bool value = P::kSharedSinks; };

// Policies that evaluate two sources per step define kPaired = true.
template <class P, class = void>
struct is_paired { static constexpr bool value = false; };
template <class P>
struct is_paired<P, decltype(void(P::kPaired))> { static constexpr bool value = P::kPaired; };

// Cache words a policy's fused prediction loads per source (1 for policies
// without fused prediction, as a placeholder size).
template <class P, class = void>
struct raw_words { static constexpr int value = 1; };
template <class P>
struct raw_words<P, decltype(void(P::kRawWords))> { static constexpr int value = P::kRawWords; };

// Lexicographic (r2, id) minimum; id -1 means "none" and only pairs with r2 = +inf.
__device__ __forceinline__ void nn_merge(double &d, int &id, double od, int oid) {
    if (od < d || (od == d && static_cast<unsigned>(oid) < static_cast<unsigned>(id))) {
        d = od;
        id = oid;
    }
}

// ---------------------------------------------------------------------------
// Mixed precision force policy: positions as double-single (hi + lo FP32),
// x_j - x_i formed as (hi_j - hi_i) + (lo_j - lo_i); rsqrt (SFU) and all terms
// in FP32.  Sums are kept in two FP32 levels -- a partial over kChunk sources,
// folded into a second FP32 level -- and the second level is added into
// running totals once at least kFlush sources have passed (at a tile end in
// the pass kernel): double-single totals in registers here (the batched
// kernel), in shared memory in the paired policy.
// Sequential FP32 summation rounds every add at the scale of the running sum,
// so a long FP32 sum dominated by one large term loses ~sqrt(k) ulps; the two
// short levels bound that error by ~(kChunk + sources per flush / kChunk) ulps.
// ---------------------------------------------------------------------------
template <int ORDER, bool NN>
struct MixedForce {
    static constexpr int NW = (ORDER == 6) ? 4 : 3;  // 16-byte words per record
    static constexpr int RB = NW * 16;
    static constexpr int NS = (ORDER == 6) ? 10 : (ORDER == 2 ? 4 : 7);  // summed fields
    static constexpr bool kNN = NN;
    static constexpr bool kSmemTotals = true;
    static constexpr int kChunk = 8;
    static constexpr int kFlush = 64;
    static constexpr unsigned kKeyMask = kChunk - 1;  // low r^2 bits carrying the in-chunk position
    static constexpr bool kCanFuse = true;
    static constexpr int kOrder = ORDER;
    typedef float real;
    struct Rec {
        float4 w[NW];
    };
    struct Sink {
        float xh, yh, zh, xl, yl, zl, vx, vy, vz, ax, ay, az;
        int slot;
    };
    struct Acc {
        float f[NS];     // level 1: current chunk
        float g[NS];     // level 2: chunks since the last flush
        float th[NS];    // running totals, double-single (hi, lo)
        float tl[NS];
        unsigned ck;     // nearest-neighbour key of the current chunk
        unsigned bk;     // best key so far, and the slot of its chunk's first source
        int bbase;
        float bd;        // nearest neighbour so far: exact r^2 and id (-1: none)
        int bid;
    };

    __device__ static __forceinline__ Rec ld_shared(const unsigned char *p) {
        Rec r;
#pragma unroll
        for (int w = 0; w < NW; ++w) r.w[w] = *reinterpret_cast<const float4 *>(p + 16 * w);
        return r;
    }
    __device__ static __forceinline__ Rec ld_global(const unsigned char *p) {
        Rec r;
#pragma unroll
        for (int w = 0; w < NW; ++w) r.w[w] = __ldg(reinterpret_cast<const float4 *>(p) + w);
        return r;
    }
    // Far-away, massless filler for the ragged end of a tile: its terms are
    // exactly zero and its r^2 overflows to +inf (never a neighbour).
    __device__ static __forceinline__ uint4 sentinel(int w) {
        if (w == 0) return f4bits(1e25f, 1e25f, 1e25f, 0.f);
        if (w == 1) return make_uint4(0u, 0u, 0u, 0xffffffffu);
        return make_uint4(0u, 0u, 0u, 0u);
    }
    // the predicted record of source j, straight from the double-single cache
    __device__ static __forceinline__ Rec predict(const float4 *dsc, int64_t j, float t_hi, float t_lo) {
        float4 o[4];
        predict_ds_record<ORDER>(dsc, j, t_hi, t_lo, o);
        Rec r;
#pragma unroll
        for (int w = 0; w < NW; ++w) r.w[w] = o[w];
        return r;
    }
    // the same in two steps: the cache words of source j (kRawWords float4s),
    // then the record from those words
    static constexpr int kRawWords = dscache_words(ORDER);
    __device__ static __forceinline__ void fetch_raw(const float4 *dsc, int64_t j, float4 *w) {
        ds_fetch<ORDER>(dsc, j, w);
    }
    __device__ static __forceinline__ Rec predict_raw(const float4 *w, float t_hi, float t_lo) {
        float4 o[4];
        predict_ds_words<ORDER>(w, t_hi, t_lo, o);
        Rec r;
#pragma unroll
        for (int k = 0; k < NW; ++k) r.w[k] = o[k];
        return r;
    }
    // two sources' records from their words, in packed f32x2 steps
    __device__ static __forceinline__ void predict_raw2(const float4 *wa, const float4 *wb, float t_hi, float t_lo,
                                                        Rec &ra, Rec &rb) {
        float4 oa[4], ob[4];
        predict_ds_words2<ORDER>(wa, wb, t_hi, t_lo, oa, ob);
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            ra.w[k] = oa[k];
            rb.w[k] = ob[k];
        }
    }
    __device__ static __forceinline__ void sink_from(const Rec &r, Sink &s) {
        s.xh = r.w[0].x; s.yh = r.w[0].y; s.zh = r.w[0].z;
        s.xl = r.w[1].x; s.yl = r.w[1].y; s.zl = r.w[1].z;
        s.vx = r.w[2].x; s.vy = r.w[2].y; s.vz = r.w[2].z;
        if (ORDER == 6) { s.ax = r.w[3].x; s.ay = r.w[3].y; s.az = r.w[3].z; }
        else { s.ax = s.ay = s.az = 0.f; }
    }
    __device__ static __forceinline__ void load_sink(const unsigned char *rec, int64_t slot, Sink &s) {
        const Rec r = ld_global(rec + slot * RB);
        s.xh = r.w[0].x; s.yh = r.w[0].y; s.zh = r.w[0].z;
        s.xl = r.w[1].x; s.yl = r.w[1].y; s.zl = r.w[1].z;
        s.vx = r.w[2].x; s.vy = r.w[2].y; s.vz = r.w[2].z;
        if (ORDER == 6) { s.ax = r.w[3].x; s.ay = r.w[3].y; s.az = r.w[3].z; }
        else { s.ax = s.ay = s.az = 0.f; }
    }
    __device__ static __forceinline__ void init(Acc &c) {
#pragma unroll
        for (int f = 0; f < NS; ++f) c.f[f] = c.g[f] = c.th[f] = c.tl[f] = 0.f;
        c.ck = c.bk = 0xffffffffu;
        c.bbase = -1;
        c.bd = f_inf();
        c.bid = -1;
    }
    // Squared distance between a record and the sink, exactly as interact() forms it.
    __device__ static __forceinline__ float dist2(const Rec &r, const Sink &s) {
        const float dx = (r.w[0].x - s.xh) + (r.w[1].x - s.xl);
        const float dy = (r.w[0].y - s.yh) + (r.w[1].y - s.yl);
        const float dz = (r.w[0].z - s.zh) + (r.w[1].z - s.zl);
        return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    }
    // fields: 0-2 acc, 3-5 jerk, [6-8 snap], NS-1 potential (accumulated as +m/r).
    // Nearest neighbour: r^2 >= 0, so its bit pattern orders like the value;
    // the low log2(kChunk) mantissa bits carry the source's position u in the
    // chunk (a 2^-20 relative truncation for 8, far inside the 1e-5 tie band)
    // and one unsigned min per interaction keeps the chunk's best.
    // FIRST: the first source of a chunk starts the level-1 partials (assigns
    // instead of accumulating, so folding needs no zeroing).
    template <bool SELF, bool FIRST>
    __device__ static __forceinline__ void interact(const Rec &r, int j, int u, const Sink &s, Acc &c, float eps2) {
        const float dx = (r.w[0].x - s.xh) + (r.w[1].x - s.xl);
        const float dy = (r.w[0].y - s.yh) + (r.w[1].y - s.yl);
        const float dz = (r.w[0].z - s.zh) + (r.w[1].z - s.zl);
        const float dvx = r.w[2].x - s.vx, dvy = r.w[2].y - s.vy, dvz = r.w[2].z - s.vz;
        const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        float rinv = rsqrtf(d2 + eps2);
        if (SELF && j == s.slot) rinv = 0.f;
        const float rinv2 = rinv * rinv;
        const float mr = r.w[0].w * rinv;
        const float mr3 = mr * rinv2;
        c.f[NS - 1] = FIRST ? mr : c.f[NS - 1] + mr;
        const float rv = fmaf(dz, dvz, fmaf(dy, dvy, dx * dvx));
        const float al3 = 3.f * (rv * rinv2);
        if (ORDER == 2) {
            c.f[0] = FIRST ? mr3 * dx : fmaf(mr3, dx, c.f[0]);
            c.f[1] = FIRST ? mr3 * dy : fmaf(mr3, dy, c.f[1]);
            c.f[2] = FIRST ? mr3 * dz : fmaf(mr3, dz, c.f[2]);
        } else if (ORDER == 4) {
            c.f[0] = FIRST ? mr3 * dx : fmaf(mr3, dx, c.f[0]);
            c.f[1] = FIRST ? mr3 * dy : fmaf(mr3, dy, c.f[1]);
            c.f[2] = FIRST ? mr3 * dz : fmaf(mr3, dz, c.f[2]);
            c.f[3] = FIRST ? mr3 * fmaf(-al3, dx, dvx) : fmaf(mr3, fmaf(-al3, dx, dvx), c.f[3]);
            c.f[4] = FIRST ? mr3 * fmaf(-al3, dy, dvy) : fmaf(mr3, fmaf(-al3, dy, dvy), c.f[4]);
            c.f[5] = FIRST ? mr3 * fmaf(-al3, dz, dvz) : fmaf(mr3, fmaf(-al3, dz, dvz), c.f[5]);
        } else {
            const float dax = r.w[3].x - s.ax, day = r.w[3].y - s.ay, daz = r.w[3].z - s.az;
            const float Ax = mr3 * dx, Ay = mr3 * dy, Az = mr3 * dz;
            const float Jx = fmaf(-al3, Ax, mr3 * dvx);
            const float Jy = fmaf(-al3, Ay, mr3 * dvy);
            const float Jz = fmaf(-al3, Az, mr3 * dvz);
            const float vv = fmaf(dvz, dvz, fmaf(dvy, dvy, dvx * dvx));
            const float ra = fmaf(dz, daz, fmaf(dy, day, dx * dax));
            const float al = rv * rinv2;
            const float b3 = 3.f * fmaf(vv + ra, rinv2, al * al);
            const float a6 = 2.f * al3;
            const float Sx = fmaf(mr3, dax, -fmaf(a6, Jx, b3 * Ax));
            const float Sy = fmaf(mr3, day, -fmaf(a6, Jy, b3 * Ay));
            const float Sz = fmaf(mr3, daz, -fmaf(a6, Jz, b3 * Az));
            if (FIRST) {
                c.f[0] = Ax; c.f[1] = Ay; c.f[2] = Az;
                c.f[3] = Jx; c.f[4] = Jy; c.f[5] = Jz;
                c.f[6] = Sx; c.f[7] = Sy; c.f[8] = Sz;
            } else {
                c.f[0] += Ax; c.f[1] += Ay; c.f[2] += Az;
                c.f[3] += Jx; c.f[4] += Jy; c.f[5] += Jz;
                c.f[6] += Sx; c.f[7] += Sy; c.f[8] += Sz;
            }
        }
        if (NN) {
            const unsigned key = (SELF && j == s.slot) ? 0xffffffffu : ((__float_as_uint(d2) & ~kKeyMask) | unsigned(u));
            c.ck = FIRST ? key : min(c.ck, key);
        }
    }
    // End of a chunk (batched kernel) whose records start at chunk (stride RB)
    // in shared memory: a new nearest neighbour's exact r^2 and id are taken
    // from its record there (filler records never qualify).
    __device__ static __forceinline__ void fold_tile(Acc &c, int base, const unsigned char *chunk, const Sink &s) {
#pragma unroll
        for (int f = 0; f < NS; ++f) c.g[f] += c.f[f];
        if (NN && c.ck < c.bk) {
            c.bk = c.ck;
            c.bbase = base;
            if ((c.ck & ~kKeyMask) < 0x7f800000u) {
                const Rec r = ld_shared(chunk + static_cast<int>(c.ck & kKeyMask) * RB);
                c.bd = dist2(r, s);
                c.bid = __float_as_int(r.w[1].w);
            } else {
                c.bd = f_inf();
                c.bid = -1;
            }
        }
    }
    // Level 2 -> the running totals, double-single (hi, lo) in registers,
    // updated by TwoSum (Knuth): no FP64 arithmetic per flush.  The tot
    // argument is not used.
    __device__ static __forceinline__ void flush(Acc &c, double *, int) {
#pragma unroll
        for (int f = 0; f < NS; ++f) {
            const float v = c.g[f];
            const float h = c.th[f] + v;
            const float bv = h - c.th[f];
            c.tl[f] += (c.th[f] - (h - bv)) + (v - bv);
            c.th[f] = h;
            c.g[f] = 0.f;
        }
    }
    __device__ static __forceinline__ void totals(const Acc &c, const double *, int, double *t) {
#pragma unroll
        for (int f = 0; f < NS; ++f) t[f] = f2d_exact(c.th[f]) + f2d_exact(c.tl[f]);
        t[NS - 1] = f2d_exact(-c.th[NS - 1]) + f2d_exact(-c.tl[NS - 1]);
    }
    __device__ static __forceinline__ void nn_acc(const Acc &c, double &d, int &id) {
        d = (NN && c.bid >= 0) ? f2d_exact(c.bd) : d_inf();
        id = NN ? c.bid : -1;
    }
    template <class Out>
    __device__ static __forceinline__ void write_final(const Out &o, int64_t i, const double *t, double d, int id) {
        if (o.acc) { o.acc[3 * i] = t[0]; o.acc[3 * i + 1] = t[1]; o.acc[3 * i + 2] = t[2]; }
        if (ORDER != 2 && o.jerk) { o.jerk[3 * i] = t[3]; o.jerk[3 * i + 1] = t[4]; o.jerk[3 * i + 2] = t[5]; }
        if (ORDER == 6 && o.snap) { o.snap[3 * i] = t[6]; o.snap[3 * i + 1] = t[7]; o.snap[3 * i + 2] = t[8]; }
        if (o.pot) o.pot[i] = t[NS - 1];
        if (NN) {
            if (o.nn_id) o.nn_id[i] = id;
            if (o.nn_r2) o.nn_r2[i] = (id < 0) ? d_inf() : d;
        }
    }
};

// ---------------------------------------------------------------------------
// The mixed force policy evaluated two sources at a time in packed FP32 pairs
// (f32x2): half .x of every pair belongs to the first source of the pair,
// half .y to the second.  The pass kernel re-lays each staged tile as pair
// records (PRB bytes): natural word w = {e0,e1,e2,e3} of sources a and b
// becomes the two words {e0a,e0b,e1a,e1b} and {e2a,e2b,e3a,e3b}, so every
// operand pair is an aligned register pair straight from shared memory.  The
// sink's values are held duplicated in both halves.  Each half keeps its own
// two-level partial sums; the halves are added when the second level is
// flushed into the running double-single totals (see flush).  The arithmetic
// of each half is that of MixedForce::interact, operation for operation.
// ---------------------------------------------------------------------------
template <int ORDER, bool NN>
struct MixedPairForce : MixedForce<ORDER, NN> {
    typedef MixedForce<ORDER, NN> Base;
    using Base::NS;
    using Base::kKeyMask;
    using typename Base::Rec;
    static constexpr bool kPaired = true;
    static constexpr bool kSharedSinks = true;
    static constexpr int PRB = 2 * Base::RB;  // bytes of one pair record
    struct PRec {
        float4 w0, w1, w2, w4, w6;  // {xh,yh}, {zh,m}, {xl,yl}, {vx,vy}, [{ax,ay}]
        float2 w3, w5, w7;          // {zl}, {vz}, [{az}]
    };
    __device__ static __forceinline__ PRec ld_pair(const unsigned char *q) {
        const float4 *w = reinterpret_cast<const float4 *>(q);
        PRec r;
        r.w0 = w[0]; r.w1 = w[1]; r.w2 = w[2];
        r.w3 = *reinterpret_cast<const float2 *>(w + 3);
        r.w4 = w[4];
        r.w5 = *reinterpret_cast<const float2 *>(w + 5);
        if (ORDER == 6) {
            r.w6 = w[6];
            r.w7 = *reinterpret_cast<const float2 *>(w + 7);
        }
        return r;
    }
    // words 2w and 2w+1 of the pair record q from natural word w of sources a (x) and b (y)
    __device__ static __forceinline__ void store_pair_word(const float4 &x, const float4 &y, int w, unsigned char *q) {
        float4 *d = reinterpret_cast<float4 *>(q) + 2 * w;
        d[0] = make_float4(x.x, y.x, x.y, y.y);
        d[1] = make_float4(x.z, y.z, x.w, y.w);
    }
    __device__ static __forceinline__ void pack_word(const unsigned char *a, const unsigned char *b, int w,
                                                     unsigned char *q) {
        store_pair_word(reinterpret_cast<const float4 *>(a)[w], reinterpret_cast<const float4 *>(b)[w], w, q);
    }
    struct Sink {
        float2 xh, yh, zh, xl, yl, zl, vx, vy, vz, ax, ay, az;
        int slot;
    };
    struct Acc {
        float2 f[NS];
        float2 g[NS];
        unsigned ck, bk;
        int bbase;
        float bd;  // nearest neighbour so far: exact r^2 and id (-1: none)
        int bid;
    };
    __device__ static __forceinline__ void sink_from(const Rec &r, Sink &s) {
        s.xh = dup2(r.w[0].x); s.yh = dup2(r.w[0].y); s.zh = dup2(r.w[0].z);
        s.xl = dup2(r.w[1].x); s.yl = dup2(r.w[1].y); s.zl = dup2(r.w[1].z);
        s.vx = dup2(r.w[2].x); s.vy = dup2(r.w[2].y); s.vz = dup2(r.w[2].z);
        if (ORDER == 6) { s.ax = dup2(r.w[3].x); s.ay = dup2(r.w[3].y); s.az = dup2(r.w[3].z); }
        else { s.ax = s.ay = s.az = dup2(0.f); }
    }
    __device__ static __forceinline__ void load_sink(const unsigned char *rec, int64_t slot, Sink &s) {
        sink_from(Base::ld_global(rec + slot * Base::RB), s);
    }
    __device__ static __forceinline__ void init(Acc &c) {
#pragma unroll
        for (int f = 0; f < NS; ++f) c.f[f] = c.g[f] = dup2(0.f);
        c.ck = c.bk = 0xffffffffu;
        c.bbase = -1;
        c.bd = f_inf();
        c.bid = -1;
    }
    __device__ static __forceinline__ float dist2(const Rec &r, const Sink &s) {
        const float dx = (r.w[0].x - s.xh.x) + (r.w[1].x - s.xl.x);
        const float dy = (r.w[0].y - s.yh.x) + (r.w[1].y - s.yl.x);
        const float dz = (r.w[0].z - s.zh.x) + (r.w[1].z - s.zl.x);
        return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    }
    // Sources a (slot j, chunk position u) and b (slot j + jl, position u + 1).
    // Returns the pair's unsoftened r^2 (used by the neighbour-list policy).
    template <bool SELF, bool FIRST>
    __device__ static __forceinline__ float2 interact2(const PRec &r, int j, int jl, int u, const Sink &s, Acc &c,
                                                       float eps2) {
        const float2 dx = add2(sub2(make_float2(r.w0.x, r.w0.y), s.xh), sub2(make_float2(r.w2.x, r.w2.y), s.xl));
        const float2 dy = add2(sub2(make_float2(r.w0.z, r.w0.w), s.yh), sub2(make_float2(r.w2.z, r.w2.w), s.yl));
        const float2 dz = add2(sub2(make_float2(r.w1.x, r.w1.y), s.zh), sub2(r.w3, s.zl));
        const float2 dvx = sub2(make_float2(r.w4.x, r.w4.y), s.vx);
        const float2 dvy = sub2(make_float2(r.w4.z, r.w4.w), s.vy);
        const float2 dvz = sub2(r.w5, s.vz);
        const float2 d2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
        const float2 d2e = add2(d2, dup2(eps2));
        float2 rinv = make_float2(rsqrtf(d2e.x), rsqrtf(d2e.y));
        if (SELF) {
            if (j == s.slot) rinv.x = 0.f;
            if (j + jl == s.slot) rinv.y = 0.f;
        }
        const float2 rinv2 = mul2(rinv, rinv);
        const float2 mr = mul2(make_float2(r.w1.z, r.w1.w), rinv);
        const float2 mr3 = mul2(mr, rinv2);
        c.f[NS - 1] = FIRST ? mr : add2(c.f[NS - 1], mr);
        const float2 rv = fma2(dz, dvz, fma2(dy, dvy, mul2(dx, dvx)));
        const float2 al = mul2(rv, rinv2);
        const float2 nal3 = mul2(dup2(-3.f), al);  // -alpha * 3 (sign folded into the constant)
        if (ORDER == 2) {
            c.f[0] = FIRST ? mul2(mr3, dx) : fma2(mr3, dx, c.f[0]);
            c.f[1] = FIRST ? mul2(mr3, dy) : fma2(mr3, dy, c.f[1]);
            c.f[2] = FIRST ? mul2(mr3, dz) : fma2(mr3, dz, c.f[2]);
        } else if (ORDER == 4) {
            c.f[0] = FIRST ? mul2(mr3, dx) : fma2(mr3, dx, c.f[0]);
            c.f[1] = FIRST ? mul2(mr3, dy) : fma2(mr3, dy, c.f[1]);
            c.f[2] = FIRST ? mul2(mr3, dz) : fma2(mr3, dz, c.f[2]);
            c.f[3] = FIRST ? mul2(mr3, fma2(nal3, dx, dvx)) : fma2(mr3, fma2(nal3, dx, dvx), c.f[3]);
            c.f[4] = FIRST ? mul2(mr3, fma2(nal3, dy, dvy)) : fma2(mr3, fma2(nal3, dy, dvy), c.f[4]);
            c.f[5] = FIRST ? mul2(mr3, fma2(nal3, dz, dvz)) : fma2(mr3, fma2(nal3, dz, dvz), c.f[5]);
        } else {
            const float2 dax = sub2(make_float2(r.w6.x, r.w6.y), s.ax);
            const float2 day = sub2(make_float2(r.w6.z, r.w6.w), s.ay);
            const float2 daz = sub2(r.w7, s.az);
            const float2 Ax = mul2(mr3, dx), Ay = mul2(mr3, dy), Az = mul2(mr3, dz);
            const float2 Jx = fma2(nal3, Ax, mul2(mr3, dvx));
            const float2 Jy = fma2(nal3, Ay, mul2(mr3, dvy));
            const float2 Jz = fma2(nal3, Az, mul2(mr3, dvz));
            const float2 vv = fma2(dvz, dvz, fma2(dvy, dvy, mul2(dvx, dvx)));
            const float2 ra = fma2(dz, daz, fma2(dy, day, mul2(dx, dax)));
            const float2 nb3 = mul2(dup2(-3.f), fma2(add2(vv, ra), rinv2, mul2(al, al)));
            const float2 na6 = mul2(dup2(2.f), nal3);
            const float2 Sx = fma2(mr3, dax, fma2(na6, Jx, mul2(nb3, Ax)));
            const float2 Sy = fma2(mr3, day, fma2(na6, Jy, mul2(nb3, Ay)));
            const float2 Sz = fma2(mr3, daz, fma2(na6, Jz, mul2(nb3, Az)));
            if (FIRST) {
                c.f[0] = Ax; c.f[1] = Ay; c.f[2] = Az;
                c.f[3] = Jx; c.f[4] = Jy; c.f[5] = Jz;
                c.f[6] = Sx; c.f[7] = Sy; c.f[8] = Sz;
            } else {
                c.f[0] = add2(c.f[0], Ax); c.f[1] = add2(c.f[1], Ay); c.f[2] = add2(c.f[2], Az);
                c.f[3] = add2(c.f[3], Jx); c.f[4] = add2(c.f[4], Jy); c.f[5] = add2(c.f[5], Jz);
                c.f[6] = add2(c.f[6], Sx); c.f[7] = add2(c.f[7], Sy); c.f[8] = add2(c.f[8], Sz);
            }
        }
        if (NN) {
            const unsigned ka = (SELF && j == s.slot) ? 0xffffffffu : ((__float_as_uint(d2.x) & ~kKeyMask) | unsigned(u));
            const unsigned kb =
                (SELF && j + jl == s.slot) ? 0xffffffffu : ((__float_as_uint(d2.y) & ~kKeyMask) | unsigned(u + 1));
            c.ck = FIRST ? min(ka, kb) : min(c.ck, min(ka, kb));
        }
        return d2;
    }
    // End of a chunk whose pair records start at pq (pair stride pstep).  When
    // the chunk holds a new nearest neighbour, its exact r^2 (the operations
    // of interact2 on that half) and id are taken from the chunk's pair record
    // while it is still in shared memory; filler records (r^2 = inf) never
    // qualify.
    __device__ static __forceinline__ void fold(Acc &c, int base, const unsigned char *pq, int pstep, const Sink &s) {
#pragma unroll
        for (int f = 0; f < NS; ++f) c.g[f] = add2(c.g[f], c.f[f]);
        if (NN && c.ck < c.bk) {
            c.bk = c.ck;
            c.bbase = base;
            if ((c.ck & ~kKeyMask) < 0x7f800000u) {
                const int u = static_cast<int>(c.ck & kKeyMask), h = u & 1;
                // floats of a pair record: xh 0,1  yh 2,3  zh 4,5  xl 8,9  yl 10,11  zl 12,13  id 14,15
                const float *q = reinterpret_cast<const float *>(pq + (u >> 1) * pstep);
                const float dx = (q[h] - s.xh.x) + (q[8 + h] - s.xl.x);
                const float dy = (q[2 + h] - s.yh.x) + (q[10 + h] - s.yl.x);
                const float dz = (q[4 + h] - s.zh.x) + (q[12 + h] - s.zl.x);
                c.bd = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                c.bid = __float_as_int(q[14 + h]);
            } else {
                c.bd = f_inf();
                c.bid = -1;
            }
        }
    }
    // Level 2 (both halves added) -> the running totals, held as unevaluated
    // FP32 sums hi + lo (double-single) in the 8-byte slots tot[f * stride]:
    // hi takes the new value by TwoSum (Knuth), whose exact rounding error
    // goes to lo, so the totals keep ~48 bits without touching the FP64 pipe
    // (1/64 of the FP32 rate on this GPU) inside the pass.
    __device__ static __forceinline__ void flush(Acc &c, double *tot, int stride) {
        float2 *t2 = reinterpret_cast<float2 *>(tot);
#pragma unroll
        for (int f = 0; f < NS; ++f) {
            const float v = c.g[f].x + c.g[f].y;
            float2 T = t2[f * stride];
            const float h = T.x + v;
            const float bv = h - T.x;
            const float e = (T.x - (h - bv)) + (v - bv);
            T.x = h;
            T.y += e;
            t2[f * stride] = T;
            c.g[f] = dup2(0.f);
        }
    }
    __device__ static __forceinline__ void zero_totals(double *tot, int stride) {
        float2 *t2 = reinterpret_cast<float2 *>(tot);
#pragma unroll
        for (int f = 0; f < NS; ++f) t2[f * stride] = dup2(0.f);
    }
    __device__ static __forceinline__ void totals(const Acc &, const double *tot, int stride, double *t) {
        const float2 *t2 = reinterpret_cast<const float2 *>(tot);
#pragma unroll
        for (int f = 0; f < NS; ++f) t[f] = f2d_exact(t2[f * stride].x) + f2d_exact(t2[f * stride].y);
        t[NS - 1] = -t[NS - 1];
    }
    // the potential field is summed as +m/r and leaves with its sign changed
    static constexpr bool kNegLast = true;
    // summed field f of sink i into the final outputs: 0-2 acc, 3-5 jerk,
    // 6-8 snap (order 6), NS-1 pot (null outputs are not written)
    __device__ static __forceinline__ void store_final(const ForceParams &o, int64_t i, int f, double v) {
        double *dst;
        if (f == NS - 1) dst = o.pot ? o.pot + i : nullptr;
        else if (f < 3) dst = o.acc ? o.acc + 3 * i + f : nullptr;
        else if (f < 6) dst = o.jerk ? o.jerk + 3 * i + (f - 3) : nullptr;
        else dst = o.snap ? o.snap + 3 * i + (f - 6) : nullptr;
        if (dst) *dst = v;
    }
};

// ---------------------------------------------------------------------------
// The paired policy as the batched kernel runs it: the same interaction and
// chunk fold, with the running double-single totals held in registers (the
// batched kernel's systems are short and its totals per sink few) instead of
// the pass kernel's shared-memory slots.
// ---------------------------------------------------------------------------
template <int ORDER, bool NN>
struct MixedPairBatch : MixedPairForce<ORDER, NN> {
    typedef MixedPairForce<ORDER, NN> Pair;
    using Pair::NS;
    struct Acc : Pair::Acc {
        float th[NS];  // running totals, double-single (hi, lo)
        float tl[NS];
    };
    __device__ static __forceinline__ void init(Acc &c) {
        Pair::init(c);
#pragma unroll
        for (int f = 0; f < NS; ++f) c.th[f] = c.tl[f] = 0.f;
    }
    // level 2 (both halves added) -> the register totals by TwoSum (Knuth)
    __device__ static __forceinline__ void flush(Acc &c, double *, int) {
#pragma unroll
        for (int f = 0; f < NS; ++f) {
            const float v = c.g[f].x + c.g[f].y;
            const float h = c.th[f] + v;
            const float bv = h - c.th[f];
            c.tl[f] += (c.th[f] - (h - bv)) + (v - bv);
            c.th[f] = h;
            c.g[f] = dup2(0.f);
        }
    }
    __device__ static __forceinline__ void totals(const Acc &c, const double *, int, double *t) {
#pragma unroll
        for (int f = 0; f < NS; ++f) t[f] = f2d_exact(c.th[f]) + f2d_exact(c.tl[f]);
        t[NS - 1] = f2d_exact(-c.th[NS - 1]) + f2d_exact(-c.tl[NS - 1]);
    }
    __device__ static __forceinline__ void nn_acc(const Acc &c, double &d, int &id) {
        d = (NN && c.bid >= 0) ? f2d_exact(c.bd) : d_inf();
        id = NN ? c.bid : -1;
    }
};

// ---------------------------------------------------------------------------
// FP64 force policy: every operation in IEEE double.  The unsoftened r^2 is
// formed without fused multiply-adds, so that nearest-neighbour decisions are
// taken on exactly the values a plain FP64 evaluation produces.
// ---------------------------------------------------------------------------
template <int ORDER, bool NN>
struct Fp64Force {
    static constexpr int kOrder = ORDER;
    static constexpr int NW = (ORDER == 6) ? 6 : 4;
    static constexpr bool kCanFuse = false;
    static constexpr int RB = NW * 16;
    static constexpr int NS = (ORDER == 6) ? 10 : (ORDER == 2 ? 4 : 7);
    static constexpr bool kNN = NN;
    static constexpr bool kSmemTotals = false;
    static constexpr int kChunk = 8;
    static constexpr int kFlush = 1 << 30;
    typedef double real;
    struct Rec {
        double2 w[NW];
    };
    struct Sink {
        double x, y, z, vx, vy, vz, ax, ay, az;
        int slot;
    };
    struct Acc {
        double ax, ay, az, jx, jy, jz, sx, sy, sz, pot;
        double nn_d2;
        int nn_id;
    };
    __device__ static __forceinline__ Rec ld_shared(const unsigned char *p) {
        Rec r;
#pragma unroll
        for (int w = 0; w < NW; ++w) r.w[w] = *reinterpret_cast<const double2 *>(p + 16 * w);
        return r;
    }
    __device__ static __forceinline__ Rec ld_global(const unsigned char *p) {
        Rec r;
#pragma unroll
        for (int w = 0; w < NW; ++w) r.w[w] = __ldg(reinterpret_cast<const double2 *>(p) + w);
        return r;
    }
    __device__ static __forceinline__ uint4 sentinel(int w) {
        if (w == 0) return d2bits(1e200, 1e200);
        if (w == 1) return d2bits(1e200, 0.0);
        if (w == 3) return make_uint4(0u, 0u, 0xffffffffu, 0xffffffffu);
        return make_uint4(0u, 0u, 0u, 0u);
    }
    __device__ static __forceinline__ void load_sink(const unsigned char *rec, int64_t slot, Sink &s) {
        const Rec r = ld_global(rec + slot * RB);
        s.x = r.w[0].x; s.y = r.w[0].y; s.z = r.w[1].x;
        s.vx = r.w[2].x; s.vy = r.w[2].y; s.vz = r.w[3].x;
        if (ORDER == 6) { s.ax = r.w[4].x; s.ay = r.w[4].y; s.az = r.w[5].x; }
        else { s.ax = s.ay = s.az = 0.0; }
    }
    __device__ static __forceinline__ void init(Acc &c) {
        c.ax = c.ay = c.az = c.jx = c.jy = c.jz = c.sx = c.sy = c.sz = c.pot = 0.0;
        c.nn_d2 = d_inf();
        c.nn_id = -1;
    }
    // Returns the pair's unsoftened r^2 (used by the neighbour-list policy).
    template <bool SELF, bool FIRST>
    __device__ static __forceinline__ double interact(const Rec &r, int j, int, const Sink &s, Acc &c, double eps2) {
        const double dx = r.w[0].x - s.x, dy = r.w[0].y - s.y, dz = r.w[1].x - s.z;
        const double m = r.w[1].y;
        const double dvx = r.w[2].x - s.vx, dvy = r.w[2].y - s.vy, dvz = r.w[3].x - s.vz;
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        double rinv = rsqrt(d2 + eps2);
        if (SELF && j == s.slot) rinv = 0.0;
        const double rinv2 = rinv * rinv;
        const double mr = m * rinv;
        const double mr3 = mr * rinv2;
        c.pot -= mr;
        const double Ax = mr3 * dx, Ay = mr3 * dy, Az = mr3 * dz;
        const double rv = dx * dvx + dy * dvy + dz * dvz;
        const double al = rv * rinv2;
        const double Jx = mr3 * dvx - 3.0 * al * Ax;
        const double Jy = mr3 * dvy - 3.0 * al * Ay;
        const double Jz = mr3 * dvz - 3.0 * al * Az;
        c.ax += Ax; c.ay += Ay; c.az += Az;
        if (ORDER != 2) { c.jx += Jx; c.jy += Jy; c.jz += Jz; }
        if (ORDER == 6) {
            const double dax = r.w[4].x - s.ax, day = r.w[4].y - s.ay, daz = r.w[5].x - s.az;
            const double vv = dvx * dvx + dvy * dvy + dvz * dvz;
            const double ra = dx * dax + dy * day + dz * daz;
            const double beta = (vv + ra) * rinv2 + al * al;
            c.sx += mr3 * dax - 6.0 * al * Jx - 3.0 * beta * Ax;
            c.sy += mr3 * day - 6.0 * al * Jy - 3.0 * beta * Ay;
            c.sz += mr3 * daz - 6.0 * al * Jz - 3.0 * beta * Az;
        }
        if (NN) {
            const int id = static_cast<int>(__double_as_longlong(r.w[3].y));
            const bool self = SELF && j == s.slot;
            if (!self && (d2 < c.nn_d2 || (d2 == c.nn_d2 && id < c.nn_id))) {
                c.nn_d2 = d2;
                c.nn_id = id;
            }
        }
        return d2;
    }
    __device__ static __forceinline__ void fold(Acc &, int) {}
    __device__ static __forceinline__ void flush(Acc &, double *, int) {}
    __device__ static __forceinline__ void zero_totals(double *, int) {}
    __device__ static __forceinline__ void totals(const Acc &c, const double *, int, double *t) {
        t[0] = c.ax; t[1] = c.ay; t[2] = c.az;
        if (ORDER == 2) { t[3] = c.pot; return; }
        t[3] = c.jx; t[4] = c.jy; t[5] = c.jz;
        if (ORDER == 6) { t[6] = c.sx; t[7] = c.sy; t[8] = c.sz; t[9] = c.pot; }
        else { t[6] = c.pot; }
    }
    __device__ static __forceinline__ void nn(const Acc &c, const Sink &, const unsigned char *, int64_t, int, double &d,
                                              int &id) {
        d = c.nn_d2;
        id = NN ? c.nn_id : -1;
        if (id < 0) d = d_inf();
    }
    template <class Out>
    __device__ static __forceinline__ void write_final(const Out &o, int64_t i, const double *t, double d, int id) {
        MixedForce<ORDER, NN>::write_final(o, i, t, d, id);
    }
};

// ---------------------------------------------------------------------------
// Neighbour lists (Sec. 1 and Sec. 3: the list of all particles within a
// given radius of each sink, for perturber lists).  Wraps a force policy: after
// each interaction, a source whose unsoftened r^2 is below the sink's h^2
// (strictly; the self pair excluded) is appended to the sink's list by slot,
// with one atomic per neighbour; slots beyond the capacity are counted but not
// stored.  r^2 is the policy's own (FP32 double-single difference in mixed
// precision, exact FP64 otherwise).  The lists are mapped to ids and sorted
// after the pass.
// ---------------------------------------------------------------------------
template <class B>
struct WithNeighbours : B {
    static constexpr bool kNB = true;
    typedef typename B::real real;
    struct Sink : B::Sink {
        real h2;       // squared radius; negative for an unused sink slot
        int32_t *cnt;  // this sink's counter and list
        int32_t *lst;
        int cap;
    };
    __device__ static __forceinline__ void set_nb(Sink &s, const ForceParams &p, int64_t i, bool valid) {
        s.h2 = valid ? static_cast<real>(p.nb_h2[i]) : static_cast<real>(-1);
        s.cnt = p.nb_count + (valid ? i : 0);
        s.lst = p.nb_list + (valid ? i : 0) * static_cast<int64_t>(p.nb_max);
        s.cap = p.nb_max;
    }
    __device__ static __forceinline__ void add(const Sink &s, int j) {
        const int k = atomicAdd(s.cnt, 1);
        if (k < s.cap) s.lst[k] = j;
    }
    template <bool SELF, bool FIRST, class R>
    __device__ static __forceinline__ float2 interact2(const R &r, int j, int jl, int u, const Sink &s,
                                                       typename B::Acc &c, float eps2) {
        const float2 d2 = B::template interact2<SELF, FIRST>(r, j, jl, u, s, c, eps2);
        if (d2.x < s.h2 && (!SELF || j != s.slot)) add(s, j);
        if (d2.y < s.h2 && (!SELF || j + jl != s.slot)) add(s, j + jl);
        return d2;
    }
    template <bool SELF, bool FIRST, class R>
    __device__ static __forceinline__ double interact(const R &r, int j, int u, const Sink &s, typename B::Acc &c,
                                                      double eps2) {
        const double d2 = B::template interact<SELF, FIRST>(r, j, u, s, c, eps2);
        if (d2 < s.h2 && (!SELF || j != s.slot)) add(s, j);
        return d2;
    }
};
template <class P, class = void>
struct is_nb { static constexpr bool value = false; };
template <class P>
struct is_nb<P, decltype(void(P::kNB))> { static constexpr bool value = P::kNB; };

// ---------------------------------------------------------------------------
// Adjoint policies.  For a pair (sink k, source l) with r = x_l - x_k,
// v = v_l - v_k, s = (r.r + eps^2)^-1/2, alpha = (r.v) s^2, q = m_l s^3 and
// the sink's cotangents (abar, jbar, pbar) of (acc, jerk, pot), the scalar
//   L = abar.A + jbar.J + pbar.phi = q (abar.r + jbar.v - 3 alpha jbar.r) - pbar m_l s
// has the gradients
//   dL/dr = q abar - 3 q alpha jbar - 3 q s^2 (jbar.r) v
//           + r [ -3 q s^2 B + 6 q alpha s^2 (jbar.r) + pbar m_l s^3 ],  B = abar.r + jbar.v - 3 alpha jbar.r
//   dL/dv = q (jbar - 3 s^2 (jbar.r) r)
//   dL/dm_l = s^3 B - pbar s.
// Particle k collects -dL/dr, -dL/dv of its own sink sums and +dL/dr, +dL/dv,
// +dL/dm of every other sink's sums in which it is the source, in one pass.
// ---------------------------------------------------------------------------
struct MixedVjp {
    static constexpr int NW = 5;
    static constexpr bool kCanFuse = false;
    static constexpr int RB = 80;
    static constexpr int NS = 7;
    static constexpr bool kNN = false;
    static constexpr bool kSmemTotals = true;
    static constexpr int kChunk = 8;
    static constexpr int kFlush = 64;
    typedef float real;
    struct Rec {
        float4 w[NW];
    };
    struct Sink {
        float xh, yh, zh, xl, yl, zl, vx, vy, vz, abx, aby, abz, jbx, jby, jbz, pb, m;
        int slot;
    };
    struct Acc {
        float f[NS];  // level 1: xbar (3), vbar (3), mbar over the current chunk
        float g[NS];  // level 2
    };
    __device__ static __forceinline__ Rec ld_shared(const unsigned char *p) {
        Rec r;
#pragma unroll
        for (int w = 0; w < NW; ++w) r.w[w] = *reinterpret_cast<const float4 *>(p + 16 * w);
        return r;
    }
    __device__ static __forceinline__ Rec ld_global(const unsigned char *p) {
        Rec r;
#pragma unroll
        for (int w = 0; w < NW; ++w) r.w[w] = __ldg(reinterpret_cast<const float4 *>(p) + w);
        return r;
    }
    __device__ static __forceinline__ uint4 sentinel(int w) {
        if (w == 0) return f4bits(1e25f, 1e25f, 1e25f, 0.f);
        return make_uint4(0u, 0u, 0u, 0u);
    }
    __device__ static __forceinline__ void load_sink(const unsigned char *rec, int64_t slot, Sink &s) {
        const Rec r = ld_global(rec + slot * RB);
        s.xh = r.w[0].x; s.yh = r.w[0].y; s.zh = r.w[0].z; s.m = r.w[0].w;
        s.xl = r.w[1].x; s.yl = r.w[1].y; s.zl = r.w[1].z; s.pb = r.w[1].w;
        s.vx = r.w[2].x; s.vy = r.w[2].y; s.vz = r.w[2].z;
        s.abx = r.w[3].x; s.aby = r.w[3].y; s.abz = r.w[3].z;
        s.jbx = r.w[4].x; s.jby = r.w[4].y; s.jbz = r.w[4].z;
    }
    __device__ static __forceinline__ void init(Acc &c) {
#pragma unroll
        for (int f = 0; f < NS; ++f) c.f[f] = c.g[f] = 0.f;
    }
    template <bool SELF, bool FIRST>
    __device__ static __forceinline__ void interact(const Rec &r, int j, int, const Sink &s, Acc &c, float eps2) {
        const float dx = (r.w[0].x - s.xh) + (r.w[1].x - s.xl);
        const float dy = (r.w[0].y - s.yh) + (r.w[1].y - s.yl);
        const float dz = (r.w[0].z - s.zh) + (r.w[1].z - s.zl);
        const float vx = r.w[2].x - s.vx, vy = r.w[2].y - s.vy, vz = r.w[2].z - s.vz;
        const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        float rinv = rsqrtf(d2 + eps2);
        if (SELF && j == s.slot) rinv = 0.f;
        const float s2 = rinv * rinv, s3 = rinv * s2;
        const float al = fmaf(dz, vz, fmaf(dy, vy, dx * vx)) * s2;
        const float ml = r.w[0].w, pl = r.w[1].w;
        const float abx = r.w[3].x, aby = r.w[3].y, abz = r.w[3].z;
        const float jbx = r.w[4].x, jby = r.w[4].y, jbz = r.w[4].z;
        // sink-side sums (cotangents of k) and source-side sums (cotangents of l)
        const float jr1 = fmaf(s.jbz, dz, fmaf(s.jby, dy, s.jbx * dx));
        const float B1 = fmaf(s.abz, dz, fmaf(s.aby, dy, s.abx * dx)) + fmaf(s.jbz, vz, fmaf(s.jby, vy, s.jbx * vx)) - 3.f * al * jr1;
        const float jr2 = fmaf(jbz, dz, fmaf(jby, dy, jbx * dx));
        const float B2 = fmaf(abz, dz, fmaf(aby, dy, abx * dx)) + fmaf(jbz, vz, fmaf(jby, vy, jbx * vx)) - 3.f * al * jr2;
        const float q1 = ml * s3, q2 = s.m * s3;
        const float D = q1 * jr1 - q2 * jr2;
        const float cv = 3.f * s2 * D;
        const float cr = 3.f * s2 * (q1 * B1 - q2 * B2) - 6.f * al * s2 * D - s3 * fmaf(s.pb, ml, pl * s.m);
        const float t1 = 3.f * al * q1, t2 = 3.f * al * q2;
        const float t[NS] = {q2 * abx - q1 * s.abx + t1 * s.jbx - t2 * jbx + cv * vx + cr * dx,
                             q2 * aby - q1 * s.aby + t1 * s.jby - t2 * jby + cv * vy + cr * dy,
                             q2 * abz - q1 * s.abz + t1 * s.jbz - t2 * jbz + cv * vz + cr * dz,
                             q2 * jbx - q1 * s.jbx + cv * dx,
                             q2 * jby - q1 * s.jby + cv * dy,
                             q2 * jbz - q1 * s.jbz + cv * dz,
                             -fmaf(s3, B2, pl * rinv)};
#pragma unroll
        for (int f = 0; f < NS; ++f) c.f[f] = FIRST ? t[f] : c.f[f] + t[f];
    }
    __device__ static __forceinline__ void fold(Acc &c, int) {
#pragma unroll
        for (int f = 0; f < NS; ++f) c.g[f] += c.f[f];
    }
    __device__ static __forceinline__ void flush(Acc &c, double *tot, int stride) {
#pragma unroll
        for (int f = 0; f < NS; ++f) { tot[f * stride] += static_cast<double>(c.g[f]); c.g[f] = 0.f; }
    }
    __device__ static __forceinline__ void zero_totals(double *tot, int stride) {
#pragma unroll
        for (int f = 0; f < NS; ++f) tot[f * stride] = 0.0;
    }
    __device__ static __forceinline__ void totals(const Acc &, const double *tot, int stride, double *t) {
#pragma unroll
        for (int f = 0; f < NS; ++f) t[f] = tot[f * stride];
    }
    __device__ static __forceinline__ void nn(const Acc &, const Sink &, const unsigned char *, int64_t, int, double &d,
                                              int &id) {
        d = d_inf();
        id = -1;
    }
    template <class Out>
    __device__ static __forceinline__ void write_final(const Out &o, int64_t i, const double *t, double, int) {
        if (o.accumulate) {
            o.xbar[3 * i] += t[0]; o.xbar[3 * i + 1] += t[1]; o.xbar[3 * i + 2] += t[2];
            o.vbar[3 * i] += t[3]; o.vbar[3 * i + 1] += t[4]; o.vbar[3 * i + 2] += t[5];
            o.mbar[i] += t[6];
        } else {
            o.xbar[3 * i] = t[0]; o.xbar[3 * i + 1] = t[1]; o.xbar[3 * i + 2] = t[2];
            o.vbar[3 * i] = t[3]; o.vbar[3 * i + 1] = t[4]; o.vbar[3 * i + 2] = t[5];
            o.mbar[i] = t[6];
        }
    }
};

// ---------------------------------------------------------------------------
// The mixed adjoint evaluated two sources at a time in packed FP32 pairs
// (f32x2), as MixedPairForce does for the forces: the staged tile is re-laid
// as pair records (natural word w = {e0,e1,e2,e3} of sources a and b becomes
// {e0a,e0b,e1a,e1b}, {e2a,e2b,e3a,e3b}), the sink's values are held in both
// halves, and each half keeps its own two-level FP32 partial sums; the halves
// are added when the second level goes into the double-single running totals.
// The terms are those of MixedVjp::interact (the gradients listed above).
// ---------------------------------------------------------------------------
struct MixedPairVjp : MixedVjp {
    static constexpr bool kPaired = true;
    static constexpr int PRB = 2 * RB;  // bytes of one pair record
    struct PRec {
        float4 w0, w1, w2, w3, w4, w6, w8;  // {xh}{yh} {zh}{m} {xl}{yl} {zl}{pbar} {vx}{vy} {abx}{aby} {jbx}{jby}
        float2 w5, w7, w9;                  // {vz} {abz} {jbz}
    };
    __device__ static __forceinline__ PRec ld_pair(const unsigned char *q) {
        const float4 *w = reinterpret_cast<const float4 *>(q);
        PRec r;
        r.w0 = w[0]; r.w1 = w[1]; r.w2 = w[2]; r.w3 = w[3]; r.w4 = w[4]; r.w6 = w[6]; r.w8 = w[8];
        r.w5 = *reinterpret_cast<const float2 *>(w + 5);
        r.w7 = *reinterpret_cast<const float2 *>(w + 7);
        r.w9 = *reinterpret_cast<const float2 *>(w + 9);
        return r;
    }
    __device__ static __forceinline__ void store_pair_word(const float4 &x, const float4 &y, int w, unsigned char *q) {
        float4 *d = reinterpret_cast<float4 *>(q) + 2 * w;
        d[0] = make_float4(x.x, y.x, x.y, y.y);
        d[1] = make_float4(x.z, y.z, x.w, y.w);
    }
    __device__ static __forceinline__ void pack_word(const unsigned char *a, const unsigned char *b, int w,
                                                     unsigned char *q) {
        store_pair_word(reinterpret_cast<const float4 *>(a)[w], reinterpret_cast<const float4 *>(b)[w], w, q);
    }
    struct Sink {
        float2 xh, yh, zh, xl, yl, zl, vx, vy, vz, abx, aby, abz, jbx, jby, jbz, pb, m;
        int slot;
    };
    struct Acc {
        float2 f[NS];  // level 1: xbar (3), vbar (3), mbar over the current chunk
        float2 g[NS];  // level 2
    };
    __device__ static __forceinline__ void load_sink(const unsigned char *rec, int64_t slot, Sink &s) {
        const Rec r = ld_global(rec + slot * RB);
        s.xh = dup2(r.w[0].x); s.yh = dup2(r.w[0].y); s.zh = dup2(r.w[0].z); s.m = dup2(r.w[0].w);
        s.xl = dup2(r.w[1].x); s.yl = dup2(r.w[1].y); s.zl = dup2(r.w[1].z); s.pb = dup2(r.w[1].w);
        s.vx = dup2(r.w[2].x); s.vy = dup2(r.w[2].y); s.vz = dup2(r.w[2].z);
        s.abx = dup2(r.w[3].x); s.aby = dup2(r.w[3].y); s.abz = dup2(r.w[3].z);
        s.jbx = dup2(r.w[4].x); s.jby = dup2(r.w[4].y); s.jbz = dup2(r.w[4].z);
    }
    __device__ static __forceinline__ void init(Acc &c) {
#pragma unroll
        for (int f = 0; f < NS; ++f) c.f[f] = c.g[f] = dup2(0.f);
    }
    // Sources a (slot j) and b (slot j + jl) of the pair record r.
    template <bool SELF, bool FIRST>
    __device__ static __forceinline__ float2 interact2(const PRec &r, int j, int jl, int, const Sink &s, Acc &c,
                                                       float eps2) {
        const float2 dx = add2(sub2(make_float2(r.w0.x, r.w0.y), s.xh), sub2(make_float2(r.w2.x, r.w2.y), s.xl));
        const float2 dy = add2(sub2(make_float2(r.w0.z, r.w0.w), s.yh), sub2(make_float2(r.w2.z, r.w2.w), s.yl));
        const float2 dz = add2(sub2(make_float2(r.w1.x, r.w1.y), s.zh), sub2(make_float2(r.w3.x, r.w3.y), s.zl));
        const float2 vx = sub2(make_float2(r.w4.x, r.w4.y), s.vx);
        const float2 vy = sub2(make_float2(r.w4.z, r.w4.w), s.vy);
        const float2 vz = sub2(r.w5, s.vz);
        const float2 d2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
        const float2 d2e = add2(d2, dup2(eps2));
        float2 rinv = make_float2(rsqrtf(d2e.x), rsqrtf(d2e.y));
        if (SELF) {
            if (j == s.slot) rinv.x = 0.f;
            if (j + jl == s.slot) rinv.y = 0.f;
        }
        const float2 s2 = mul2(rinv, rinv), s3 = mul2(rinv, s2);
        const float2 al = mul2(fma2(dz, vz, fma2(dy, vy, mul2(dx, vx))), s2);
        const float2 ml = make_float2(r.w1.z, r.w1.w), pl = make_float2(r.w3.z, r.w3.w);
        const float2 abx = make_float2(r.w6.x, r.w6.y), aby = make_float2(r.w6.z, r.w6.w), abz = r.w7;
        const float2 jbx = make_float2(r.w8.x, r.w8.y), jby = make_float2(r.w8.z, r.w8.w), jbz = r.w9;
        const float2 n3al = mul2(dup2(-3.f), al);
        // sink-side sums (cotangents of the sink) and source-side sums (of the source)
        const float2 jr1 = fma2(s.jbz, dz, fma2(s.jby, dy, mul2(s.jbx, dx)));
        const float2 B1 = fma2(n3al, jr1, fma2(s.abz, dz, fma2(s.aby, dy, fma2(s.abx, dx,
                                  fma2(s.jbz, vz, fma2(s.jby, vy, mul2(s.jbx, vx)))))));
        const float2 jr2 = fma2(jbz, dz, fma2(jby, dy, mul2(jbx, dx)));
        const float2 B2 = fma2(n3al, jr2, fma2(abz, dz, fma2(aby, dy, fma2(abx, dx,
                                  fma2(jbz, vz, fma2(jby, vy, mul2(jbx, vx)))))));
        const float2 q1 = mul2(ml, s3), q2 = mul2(s.m, s3);
        const float2 D = sub2(mul2(q1, jr1), mul2(q2, jr2));
        const float2 s2_3 = mul2(dup2(3.f), s2);
        const float2 cv = mul2(s2_3, D);
        // cr = 3 s^2 (q1 B1 - q2 B2) - 6 alpha s^2 D - s^3 (pbar_k m_l + pbar_l m_k)
        const float2 ns3 = mul2(dup2(-1.f), s3);
        const float2 cr = fma2(ns3, fma2(s.pb, ml, mul2(pl, s.m)),
                               fma2(mul2(dup2(-2.f), al), cv, mul2(s2_3, sub2(mul2(q1, B1), mul2(q2, B2)))));
        const float2 nq1 = mul2(dup2(-1.f), q1);
        const float2 t1 = mul2(mul2(dup2(-1.f), n3al), q1);  // 3 alpha q1
        const float2 nt2 = mul2(n3al, q2);                    // -3 alpha q2
        float2 t[NS];
        t[0] = fma2(cr, dx, fma2(cv, vx, fma2(nt2, jbx, fma2(t1, s.jbx, fma2(nq1, s.abx, mul2(q2, abx))))));
        t[1] = fma2(cr, dy, fma2(cv, vy, fma2(nt2, jby, fma2(t1, s.jby, fma2(nq1, s.aby, mul2(q2, aby))))));
        t[2] = fma2(cr, dz, fma2(cv, vz, fma2(nt2, jbz, fma2(t1, s.jbz, fma2(nq1, s.abz, mul2(q2, abz))))));
        t[3] = fma2(cv, dx, fma2(nq1, s.jbx, mul2(q2, jbx)));
        t[4] = fma2(cv, dy, fma2(nq1, s.jby, mul2(q2, jby)));
        t[5] = fma2(cv, dz, fma2(nq1, s.jbz, mul2(q2, jbz)));
        t[6] = fma2(ns3, B2, mul2(mul2(dup2(-1.f), pl), rinv));  // -(s^3 B2 + pbar_l s)
#pragma unroll
        for (int f = 0; f < NS; ++f) c.f[f] = FIRST ? t[f] : add2(c.f[f], t[f]);
        return d2;
    }
    __device__ static __forceinline__ void fold(Acc &c, int, const unsigned char *, int, const Sink &) {
#pragma unroll
        for (int f = 0; f < NS; ++f) c.g[f] = add2(c.g[f], c.f[f]);
    }
    // level 2 (both halves added) -> double-single running totals, as MixedPairForce::flush
    __device__ static __forceinline__ void flush(Acc &c, double *tot, int stride) {
        float2 *t2 = reinterpret_cast<float2 *>(tot);
#pragma unroll
        for (int f = 0; f < NS; ++f) {
            const float v = c.g[f].x + c.g[f].y;
            float2 T = t2[f * stride];
            const float h = T.x + v;
            const float bv = h - T.x;
            const float e = (T.x - (h - bv)) + (v - bv);
            T.x = h;
            T.y += e;
            t2[f * stride] = T;
            c.g[f] = dup2(0.f);
        }
    }
    __device__ static __forceinline__ void zero_totals(double *tot, int stride) {
        float2 *t2 = reinterpret_cast<float2 *>(tot);
#pragma unroll
        for (int f = 0; f < NS; ++f) t2[f * stride] = dup2(0.f);
    }
    static constexpr bool kNegLast = false;
    // field f of particle i: 0-2 xbar, 3-5 vbar, 6 mbar (added to when accumulating)
    __device__ static __forceinline__ void store_final(const ForceParams &o, int64_t i, int f, double v) {
        double *dst = (f < 3) ? o.xbar + 3 * i + f : (f < 6) ? o.vbar + 3 * i + (f - 3) : o.mbar + i;
        if (o.accumulate) *dst += v;
        else *dst = v;
    }
};

struct Fp64Vjp {
    static constexpr int NW = 7;
    static constexpr bool kCanFuse = false;
    static constexpr int RB = 112;
    static constexpr int NS = 7;
    static constexpr bool kNN = false;
    static constexpr bool kSmemTotals = false;
    static constexpr int kChunk = 8;
    static constexpr int kFlush = 1 << 30;
    typedef double real;
    struct Rec {
        double2 w[NW];
    };
    struct Sink {
        double x, y, z, vx, vy, vz, abx, aby, abz, jbx, jby, jbz, pb, m;
        int slot;
    };
    struct Acc {
        double gx, gy, gz, hx, hy, hz, gm;
    };
    __device__ static __forceinline__ Rec ld_shared(const unsigned char *p) {
        Rec r;
#pragma unroll
        for (int w = 0; w < NW; ++w) r.w[w] = *reinterpret_cast<const double2 *>(p + 16 * w);
        return r;
    }
    __device__ static __forceinline__ Rec ld_global(const unsigned char *p) {
        Rec r;
#pragma unroll
        for (int w = 0; w < NW; ++w) r.w[w] = __ldg(reinterpret_cast<const double2 *>(p) + w);
        return r;
    }
    __device__ static __forceinline__ uint4 sentinel(int w) {
        if (w == 0) return d2bits(1e200, 1e200);
        if (w == 1) return d2bits(1e200, 0.0);
        return make_uint4(0u, 0u, 0u, 0u);
    }
    __device__ static __forceinline__ void load_sink(const unsigned char *rec, int64_t slot, Sink &s) {
        const Rec r = ld_global(rec + slot * RB);
        s.x = r.w[0].x; s.y = r.w[0].y; s.z = r.w[1].x; s.m = r.w[1].y;
        s.vx = r.w[2].x; s.vy = r.w[2].y; s.vz = r.w[3].x; s.pb = r.w[3].y;
        s.abx = r.w[4].x; s.aby = r.w[4].y; s.abz = r.w[5].x;
        s.jbx = r.w[5].y; s.jby = r.w[6].x; s.jbz = r.w[6].y;
    }
    __device__ static __forceinline__ void init(Acc &c) { c.gx = c.gy = c.gz = c.hx = c.hy = c.hz = c.gm = 0.0; }
    template <bool SELF, bool FIRST>
    __device__ static __forceinline__ void interact(const Rec &r, int j, int, const Sink &s, Acc &c, double eps2) {
        const double dx = r.w[0].x - s.x, dy = r.w[0].y - s.y, dz = r.w[1].x - s.z;
        const double vx = r.w[2].x - s.vx, vy = r.w[2].y - s.vy, vz = r.w[3].x - s.vz;
        const double d2 = dx * dx + dy * dy + dz * dz;
        double rinv = rsqrt(d2 + eps2);
        if (SELF && j == s.slot) rinv = 0.0;
        const double s2 = rinv * rinv, s3 = rinv * s2;
        const double al = (dx * vx + dy * vy + dz * vz) * s2;
        const double ml = r.w[1].y, pl = r.w[3].y;
        const double abx = r.w[4].x, aby = r.w[4].y, abz = r.w[5].x;
        const double jbx = r.w[5].y, jby = r.w[6].x, jbz = r.w[6].y;
        const double jr1 = s.jbx * dx + s.jby * dy + s.jbz * dz;
        const double B1 = s.abx * dx + s.aby * dy + s.abz * dz + s.jbx * vx + s.jby * vy + s.jbz * vz - 3.0 * al * jr1;
        const double jr2 = jbx * dx + jby * dy + jbz * dz;
        const double B2 = abx * dx + aby * dy + abz * dz + jbx * vx + jby * vy + jbz * vz - 3.0 * al * jr2;
        const double q1 = ml * s3, q2 = s.m * s3;
        const double D = q1 * jr1 - q2 * jr2;
        const double cv = 3.0 * s2 * D;
        const double cr = 3.0 * s2 * (q1 * B1 - q2 * B2) - 6.0 * al * s2 * D - s3 * (s.pb * ml + pl * s.m);
        const double t1 = 3.0 * al * q1, t2 = 3.0 * al * q2;
        c.gx += q2 * abx - q1 * s.abx + t1 * s.jbx - t2 * jbx + cv * vx + cr * dx;
        c.gy += q2 * aby - q1 * s.aby + t1 * s.jby - t2 * jby + cv * vy + cr * dy;
        c.gz += q2 * abz - q1 * s.abz + t1 * s.jbz - t2 * jbz + cv * vz + cr * dz;
        c.hx += q2 * jbx - q1 * s.jbx + cv * dx;
        c.hy += q2 * jby - q1 * s.jby + cv * dy;
        c.hz += q2 * jbz - q1 * s.jbz + cv * dz;
        c.gm -= s3 * B2 + pl * rinv;
    }
    __device__ static __forceinline__ void fold(Acc &, int) {}
    __device__ static __forceinline__ void flush(Acc &, double *, int) {}
    __device__ static __forceinline__ void zero_totals(double *, int) {}
    __device__ static __forceinline__ void totals(const Acc &c, const double *, int, double *t) {
        t[0] = c.gx; t[1] = c.gy; t[2] = c.gz; t[3] = c.hx; t[4] = c.hy; t[5] = c.hz; t[6] = c.gm;
    }
    __device__ static __forceinline__ void nn(const Acc &, const Sink &, const unsigned char *, int64_t, int, double &d,
                                              int &id) {
        d = d_inf();
        id = -1;
    }
    template <class Out>
    __device__ static __forceinline__ void write_final(const Out &o, int64_t i, const double *t, double d, int id) {
        MixedVjp::write_final(o, i, t, d, id);
    }
};

// ---------------------------------------------------------------------------
// Persistent pass kernel.  Work item = (i-block, j-slice); CTAs fetch items
// from a device counter (atomicAdd, no waiting).  Sources of the slice stream
// through a kStages-deep ring of shared-memory tiles filled with 16-byte
// cp.async copies; the ragged end of the last tile is filled with sentinel
// records so the inner loop has a fixed trip count.  Sinks whose own slot lies
// in the current tile take the variant of the loop that skips the self pair.
// ---------------------------------------------------------------------------
template <class P>
__device__ __forceinline__ void load_tile(const ForceParams &p, unsigned char *smem, int t, int64_t j0, int64_t j1) {
    const int tile = p.tile;
    constexpr int W = P::RB / 16;
    unsigned char *dst = smem + static_cast<size_t>(t % kStages) * tile * P::RB;
    const int64_t tb = j0 + static_cast<int64_t>(t) * tile;
    const int64_t rem = j1 - tb;
    const int cnt = rem < tile ? static_cast<int>(rem) : tile;
    const unsigned char *src = p.rec + tb * P::RB;
    const int n16 = tile * W, v16 = cnt * W;
    for (int c = threadIdx.x; c < n16; c += blockDim.x) {
        if (c < v16) cp_async16(dst + 16 * c, src + 16 * static_cast<size_t>(c));
        else *reinterpret_cast<uint4 *>(dst + 16 * c) = P::sentinel(c % W);
    }
}

template <class P>
__device__ __forceinline__ typename P::Rec filler_rec() {
    constexpr int W = P::RB / 16;
    typename P::Rec r;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const uint4 u = P::sentinel(w);
        r.w[w] = *reinterpret_cast<const float4 *>(&u);
    }
    return r;
}

// Fused prediction of a tile whose double-single cache words (kRawWords
// float4s per source, sources 0 .. cnt-1) a bulk copy has put in shared
// memory at raw: thread t predicts the two sources of pair records t,
// t + blockDim.x, ... together (packed f32x2 steps) and writes each pair
// record whole; positions past cnt become filler records.
template <class P>
__device__ __forceinline__ void predict_staged_tile(const ForceParams &p, const float4 *raw, int cnt,
                                                    unsigned char *q, int jl) {
    constexpr int RW = P::kRawWords;
    constexpr int W = P::RB / 16;
    const int npair = p.tile >> 1;
    const int lg = __ffs(jl) - 1;  // jl is a power of two
#pragma unroll 1
    for (int pr = threadIdx.x; pr < npair; pr += blockDim.x) {
        // pair pr = k * jl + lj holds tile positions a = lj + 2k jl and a + jl
        const int k = pr >> lg, lj = pr & (jl - 1);
        const int a = lj + 2 * k * jl, b = a + jl;
        float4 wa[RW], wb[RW];
#pragma unroll
        for (int w = 0; w < RW; ++w) {
            wa[w] = (a < cnt) ? raw[a * RW + w] : make_float4(0.f, 0.f, 0.f, 0.f);
            wb[w] = (b < cnt) ? raw[b * RW + w] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        typename P::Rec ra, rb;
        P::predict_raw2(wa, wb, p.t_hi, p.t_lo, ra, rb);
        if (a >= cnt) ra = filler_rec<P>();
        if (b >= cnt) rb = filler_rec<P>();
        unsigned char *d = q + static_cast<size_t>(pr) * P::PRB;
#pragma unroll
        for (int w = 0; w < W; ++w) P::store_pair_word(ra.w[w], rb.w[w], w, d);
    }
}

// Re-lay a staged tile of natural records as pair records: lane lj's sources
// m = 2k and 2k+1 (tile positions lj + jl*m) form pair k*jl + lj.
template <class P>
__device__ __forceinline__ void pair_tile(const unsigned char *st, unsigned char *q, int tile, int jl) {
    constexpr int W = P::RB / 16;
    const int items = (tile >> 1) * W;
    for (int i = threadIdx.x; i < items; i += blockDim.x) {
        const int pr = i / W, w = i - pr * W;
        const int k = pr / jl, lj = pr - k * jl;
        const int a = lj + 2 * k * jl;
        P::pack_word(st + a * P::RB, st + (a + jl) * P::RB, w, q + pr * P::PRB);
    }
}

template <class P, int IPT, bool SELF>
__device__ __forceinline__ void tile_loop(const unsigned char *st, int tb, int per, int jl, int lj,
                                          const typename P::Sink *sk, typename P::Acc *ac,
                                          typename P::real eps2) {
    const unsigned char *base = st + lj * P::RB;
    const int step = jl * P::RB;
    if constexpr (is_paired<P>::value) {
        // st holds pair records: lane lj's k-th pair (its sources 2k and 2k+1)
        // sits at pair index k * jl + lj.
        const unsigned char *pbase = st + lj * P::PRB;
        const int pstep = jl * P::PRB;
        for (int q0 = 0; q0 < per; q0 += P::kChunk) {
            const int jb = tb + q0 * jl + lj;
            const unsigned char *pq = pbase + (q0 >> 1) * pstep;
            {
                const typename P::PRec r = P::ld_pair(pq);
#pragma unroll
                for (int k = 0; k < IPT; ++k) P::template interact2<SELF, true>(r, jb, jl, 0, sk[k], ac[k], eps2);
            }
#pragma unroll
            for (int u = 2; u < P::kChunk; u += 2) {
                const typename P::PRec r = P::ld_pair(pq + (u >> 1) * pstep);
#pragma unroll
                for (int k = 0; k < IPT; ++k)
                    P::template interact2<SELF, false>(r, jb + u * jl, jl, u, sk[k], ac[k], eps2);
            }
#pragma unroll
            for (int k = 0; k < IPT; ++k) P::fold(ac[k], jb, pq, pstep, sk[k]);
        }
    } else {
        for (int q0 = 0; q0 < per; q0 += P::kChunk) {
            const int jb = tb + q0 * jl + lj;  // this thread's first source of the chunk
            {
                const typename P::Rec r = P::ld_shared(base + q0 * step);
#pragma unroll
                for (int k = 0; k < IPT; ++k) P::template interact<SELF, true>(r, jb, 0, sk[k], ac[k], eps2);
            }
#pragma unroll
            for (int u = 1; u < P::kChunk; ++u) {
                const typename P::Rec r = P::ld_shared(base + (q0 + u) * step);
#pragma unroll
                for (int k = 0; k < IPT; ++k) P::template interact<SELF, false>(r, jb + u * jl, u, sk[k], ac[k], eps2);
            }
#pragma unroll
            for (int k = 0; k < IPT; ++k) P::fold(ac[k], jb);
        }
    }
}

// Merge the j-lanes of a sink (paired policies): the double-single totals
// are combined with double-single adds and the nearest-neighbour candidates
// (FP32 distances) with FP32 compares, so the xor-butterfly never waits on
// the FP64 pipe; every lane ends with the sink's totals q[] (double-single)
// and its nearest neighbour.
template <class P>
__device__ __forceinline__ void merge_lanes_ds(const double *tot, int stride, int jl, ds *q, double &nd, int &nid) {
    const float2 *t2 = reinterpret_cast<const float2 *>(tot);
#pragma unroll
    for (int f = 0; f < P::NS; ++f) q[f] = ds{t2[f * stride].x, t2[f * stride].y};
    float d = static_cast<float>(nd);  // exact: an FP32 distance or +inf
    for (int off = jl >> 1; off > 0; off >>= 1) {
#pragma unroll
        for (int f = 0; f < P::NS; ++f)
            q[f] = ds_add(q[f], ds{__shfl_xor_sync(kFull, q[f].h, off), __shfl_xor_sync(kFull, q[f].l, off)});
        if (P::kNN) {
            const float od = __shfl_xor_sync(kFull, d, off);
            const int oid = __shfl_xor_sync(kFull, nid, off);
            if (od < d || (od == d && static_cast<unsigned>(oid) < static_cast<unsigned>(nid))) {
                d = od;
                nid = oid;
            }
        }
    }
    nd = f2d_exact(d);
}

// A sink's merged double-single totals leave as FP64 (the exact value of the
// pair) with the fields spread over its jl lanes (lane lj takes fields lj,
// lj + jl, ...): each lane picks its field with FP32 selects, so one
// conversion per round serves up to jl fields -- GB300 runs FP64 at 1/64 of
// the FP32 rate.  Field f goes to the final outputs (split == 1,
// P::store_final) or to the slice's partial-sum slot, which the split-j
// reduction adds in FP64; with P::kNegLast the last field changes sign (the
// force policies sum the potential as +m/r).
// split == 1: final outputs of sink i; else the partial-sum slot of the
// slice for partial row pi of pn (the sinks that have partials).
template <class P>
__device__ __forceinline__ void write_fields_ds(const ForceParams &p, int64_t i, int split, int slice, int64_t pi,
                                                int64_t pn, const ds *q, int jl, int lj) {
    constexpr int NF = P::NS + (P::kNN ? 1 : 0);
    for (int f0 = 0; f0 < P::NS; f0 += jl) {
        const int f = f0 + lj;
        float h = 0.f, l = 0.f;
#pragma unroll
        for (int g = 0; g < P::NS; ++g)
            if (g == f) {
                h = q[g].h;
                l = q[g].l;
            }
        if (f < P::NS) {
            if (P::kNegLast && f == P::NS - 1) {
                h = -h;
                l = -l;
            }
            const double v = f2d_exact(h) + f2d_exact(l);
            if (split == 1) P::store_final(p, i, f, v);
            else if (p.sink_major) p.part[(pi * NF + f) * split + slice] = v;
            else p.part[static_cast<int64_t>(f) * split * pn + static_cast<int64_t>(slice) * pn + pi] = v;
        }
    }
}

// FP64 reduction of one sink's slices (sink-major row: field f's slices are
// contiguous) by the whole CTA, fields spread over the warps (two at a time,
// so that different warps' 1/64-rate FP64 adds run side by side): lane l of
// a warp sums slices l, l+32, ... of a field in order, a fixed xor-butterfly
// combines the lanes, and the field totals meet in shared
// memory, where thread 0 writes the outputs (write(t, d, id)).  The
// nearest-neighbour field (non-negative r^2, FP64) is merged by comparing bit
// patterns as integers, which orders them like the values.  Deterministic:
// the order of every sum is fixed.
template <class P, class Write>
__device__ __forceinline__ void reduce_sink_fields(const double *row, const int32_t *row_id, int split, double *s_f,
                                                   long long &s_nd, int &s_nid, const Write &write) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    // columns 0 .. NS-1 are the summed fields and (with nearest neighbour)
    // column NS the neighbour candidates; warp w takes columns w, w + nw, ...
    // two at a time, so the neighbour's loads travel with a field's
    constexpr int NC = P::NS + (P::kNN ? 1 : 0);
    for (int c0 = warp; c0 < NC; c0 += 2 * nw) {
        const int c1 = c0 + nw;
        const bool two = c1 < NC;  // (warp-uniform)
        const bool nn0 = P::kNN && c0 == P::NS, nn1 = P::kNN && two && c1 == P::NS;
        const double *col0 = row + static_cast<int64_t>(c0) * split;
        const double *col1 = row + static_cast<int64_t>(two ? c1 : c0) * split;
        // lane l takes slices l, l + 32, l + 64, ... in that order; the loads of
        // 256 slices per column are all issued before the first add
        double v0 = 0.0, v1 = 0.0;
        long long d = 0x7ff0000000000000LL;  // neighbour column: best r^2 bits (+inf) and id
        int id = -1;
        for (int s0 = 0; s0 < split; s0 += 8 * 32) {
            double x0[8], x1[8];
            int xi[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int s = s0 + lane + 32 * e;
                x0[e] = (s < split) ? __ldcg(col0 + s) : 0.0;
                x1[e] = (two && s < split) ? __ldcg(col1 + s) : 0.0;
                xi[e] = ((nn0 || nn1) && s < split) ? __ldcg(row_id + s) : -1;
            }
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (s0 + lane + 32 * e < split) {
                    if (nn0 || nn1) {
                        // non-negative r^2: the bit patterns order like the values
                        const long long xd = __double_as_longlong(nn0 ? x0[e] : x1[e]);
                        if (xd < d || (xd == d && static_cast<unsigned>(xi[e]) < static_cast<unsigned>(id))) {
                            d = xd;
                            id = xi[e];
                        }
                    }
                    if (!nn0) v0 += x0[e];
                    if (two && !nn1) v1 += x1[e];
                }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            if (!nn0) v0 += __shfl_xor_sync(kFull, v0, off);
            if (two && !nn1) v1 += __shfl_xor_sync(kFull, v1, off);
            if (nn0 || nn1) {
                const long long od = __shfl_xor_sync(kFull, d, off);
                const int oid = __shfl_xor_sync(kFull, id, off);
                if (od < d || (od == d && static_cast<unsigned>(oid) < static_cast<unsigned>(id))) {
                    d = od;
                    id = oid;
                }
            }
        }
        if (lane == 0) {
            if (!nn0) s_f[c0] = v0;
            if (two && !nn1) s_f[c1] = v1;
            if (nn0 || nn1) {
                s_nd = d;
                s_nid = id;
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        double t[P::NS];
#pragma unroll
        for (int f = 0; f < P::NS; ++f) t[f] = s_f[f];
        write(t, P::kNN ? __longlong_as_double(s_nd) : d_inf(), P::kNN ? s_nid : -1);
    }
    __syncthreads();
}

// One lane's share of a sink-major row: slices lane, lane + 32, ... of every
// field added in that order (FP64) and the lexicographic (r^2, id) minimum of
// their neighbours; beyond two slices per lane the loads of a few slices
// (every field) are issued before their adds, so a row of a few hundred
// slices costs one or two memory round trips instead of one per slice.
template <class P>
__device__ __forceinline__ void lane_sum_slices(const double *row, const int32_t *row_id, int split, int lane,
                                                double *t, double &nd, int &nid) {
    constexpr int E = (P::NS <= 7) ? 4 : 2;  // slices in flight per lane
#pragma unroll
    for (int f = 0; f < P::NS; ++f) t[f] = 0.0;
    nd = d_inf();
    nid = -1;
    if (split <= 64) {
        // one or two slices per lane: the plain loop (the chunks would be
        // mostly empty, their predicated loads and adds pure cost)
        for (int s = lane; s < split; s += 32) {
#pragma unroll
            for (int f = 0; f < P::NS; ++f) t[f] += __ldcg(row + f * split + s);
            if (P::kNN) nn_merge(nd, nid, __ldcg(row + P::NS * split + s), __ldcg(row_id + s));
        }
        return;
    }
    for (int s0 = 0; s0 < split; s0 += E * 32) {
        double x[E][P::NS], xd[E];
        int xi[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int s = s0 + lane + 32 * e;
            const bool in = s < split;
#pragma unroll
            for (int f = 0; f < P::NS; ++f) x[e][f] = in ? __ldcg(row + f * split + s) : 0.0;
            if (P::kNN) {
                xd[e] = in ? __ldcg(row + P::NS * split + s) : d_inf();
                xi[e] = in ? __ldcg(row_id + s) : -1;
            }
        }
#pragma unroll
        for (int e = 0; e < E; ++e)
            if (s0 + lane + 32 * e < split) {
#pragma unroll
                for (int f = 0; f < P::NS; ++f) t[f] += x[e][f];
                if (P::kNN) nn_merge(nd, nid, xd[e], xi[e]);
            }
    }
}

// Fused split-j reduction of one i-block, run by the last CTA to finish one
// of its slices.  Partials are read from L2 (__ldcg: written by other SMs in
// this launch) in slice order, so the result does not depend on which CTA
// arrives last.  Field-major partials (few slices): a thread per sink.
// Sink-major partials (many slices): a warp per sink, or the whole CTA per
// sink (a warp per field) when the i-block has fewer sinks than the CTA has
// warps.
template <class P>
__device__ __noinline__ void reduce_iblock(const ForceParams &p, int64_t iblk) {
    __shared__ double s_f[P::NS];
    __shared__ long long s_nd;
    __shared__ int s_nid;
    constexpr int NF = P::NS + (P::kNN ? 1 : 0);
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int64_t b0 = iblk * p.sinks_per_cta;
    const int64_t b1 = (b0 + p.sinks_per_cta < p.n_i) ? b0 + p.sinks_per_cta : p.n_i;
    const int split = p.split;
    // partial rows are counted from the first sink of the split i-blocks
    const int64_t r0 = p.tail_sink0, pn = p.n_i - p.tail_sink0;
    if (!p.sink_major) {
        const int64_t stride = static_cast<int64_t>(split) * pn;
        for (int64_t i = b0 + tid; i < b1; i += nt) {
            double t[P::NS];
#pragma unroll
            for (int f = 0; f < P::NS; ++f) t[f] = 0.0;
            double nd = d_inf();
            int nid = -1;
            const double *base = p.part + (i - r0);       // slice 0, field 0 of this sink's row
            const int32_t *base_id = p.part_id + (i - r0);
#pragma unroll 2
            for (int s = 0; s < split; ++s, base += pn, base_id += pn) {
#pragma unroll
                for (int f = 0; f < P::NS; ++f) t[f] += __ldcg(base + f * stride);
                if (P::kNN) nn_merge(nd, nid, __ldcg(base + P::NS * stride), __ldcg(base_id));
            }
            P::write_final(p, i, t, nd, nid);
        }
        return;
    }
    if (b1 - b0 < nw) {
        // few sinks: the whole CTA on each, one warp per field
        for (int64_t i = b0; i < b1; ++i)
            reduce_sink_fields<P>(p.part + (i - r0) * NF * split, p.part_id + (i - r0) * split, split, s_f, s_nd, s_nid,
                                  [&](const double *t, double d, int id) { P::write_final(p, i, t, d, id); });
        return;
    }
    // a warp per sink
    for (int64_t i = b0 + warp; i < b1; i += nw) {
        const double *row = p.part + (i - r0) * NF * split;
        const int32_t *row_id = p.part_id + (i - r0) * split;
        double t[P::NS];
        double nd;
        int nid;
        lane_sum_slices<P>(row, row_id, split, lane, t, nd, nid);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
            for (int f = 0; f < P::NS; ++f) t[f] += __shfl_xor_sync(kFull, t[f], off);
            if (P::kNN) {
                const double od = __shfl_xor_sync(kFull, nd, off);
                const int oid = __shfl_xor_sync(kFull, nid, off);
                nn_merge(nd, nid, od, oid);
            }
        }
        if (lane == 0) P::write_final(p, i, t, nd, nid);
    }
}

// The partial-sum rows of one split i-block, dropped from L2 once reduced.
template <class P>
__device__ __forceinline__ void discard_partials(const ForceParams &p, int64_t iblk) {
    constexpr int NF = P::NS + (P::kNN ? 1 : 0);
    const int64_t b0 = iblk * p.sinks_per_cta - p.tail_sink0;
    const int64_t b1 = ((iblk * p.sinks_per_cta + p.sinks_per_cta < p.n_i) ? iblk * p.sinks_per_cta + p.sinks_per_cta
                                                                          : p.n_i) - p.tail_sink0;
    const int64_t pn = p.n_i - p.tail_sink0;
    const int split = p.split;
    if (p.sink_major) {
        discard_l2_range(p.part + b0 * NF * split, p.part + b1 * NF * split);
        if (P::kNN) discard_l2_range(p.part_id + b0 * split, p.part_id + b1 * split);
        return;
    }
    for (int f = 0; f < NF; ++f)
        for (int sl = 0; sl < split; ++sl) {
            const double *row = p.part + (static_cast<int64_t>(f) * split + sl) * pn;
            discard_l2_range(row + b0, row + b1);
        }
    if (P::kNN)
        for (int sl = 0; sl < split; ++sl) discard_l2_range(p.part_id + sl * pn + b0, p.part_id + sl * pn + b1);
}

// Shared memory: kStages tiles of records, (paired policies) one tile of pair
// records, then (mixed policies) the running totals (8 bytes each: FP64, or a
// double-single pair in the paired policy), [sink k][field f][thread]
// so each thread owns its slots.
template <class P, int IPT, bool FUSED, bool MW = false>
__device__ __forceinline__ void pass_body(const ForceParams &p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned int s_item;
    const int tid = threadIdx.x;
    const int nt = blockDim.x;
    // p.jl threads share a sink; beyond a warp (paired policies only) they
    // form ws groups of one warp each, group g taking the g-th contiguous
    // part of every tile: thread = g * (nt / ws) + sink slot * 32 + lane
    // (several warps per sink: a kernel of its own, for the one-sink-per-thread
    // kernels of the paired force policies, so the others keep their registers)
    constexpr bool kMultiWarp = MW && shares_sinks<P>::value && IPT == 1;
    const int jl = (kMultiWarp && p.jl > 32) ? 32 : p.jl;  // lanes of one warp per sink
    const int ws = kMultiWarp ? p.jl / jl : 1;            // warps per sink
    const int nt_g = nt / ws;
    const int grp = kMultiWarp ? tid / nt_g : 0;
    const int lj = tid & (jl - 1);
    const int islot = (tid - grp * nt_g) / jl;
    const int slots = nt_g / jl;
    const typename P::real eps2 = static_cast<typename P::real>(p.eps2);
    const int per = p.tile / p.jl;  // sources per lane and tile, a multiple of P::kChunk (host-checked)
    const int c0 = kMultiWarp ? grp * (p.tile / ws) : 0;  // this group's part of a tile starts at tile position c0
    constexpr bool kPair = is_paired<P>::value;
    static_assert(kPair || !FUSED, "fused prediction needs a paired policy");
    // the ring holds predicted records (cp.async), or with fused prediction
    // the sources' double-single cache words (bulk copies)
    constexpr int kRaw = raw_words<P>::value;
    // fused: one stage when a slice fits one tile, else two
    const int nstage = FUSED ? p.fused_stages : kStages;
    const size_t ring_stride = static_cast<size_t>(p.tile) * (FUSED ? kRaw * 16 : P::RB);
    unsigned char *pbuf = smem + nstage * ring_stride;  // pair records (kPair)
    double *tot = reinterpret_cast<double *>(pbuf + (kPair ? static_cast<size_t>(p.tile) * P::RB : 0)) + tid;

    // fused prediction: one completion barrier per ring stage; bit s of
    // `phase` is the parity of stage s's next completion
    __shared__ __align__(8) unsigned long long s_bar[kFusedStages];
    unsigned phase = 0u;
    if constexpr (FUSED) {
        if (tid == 0) {
#pragma unroll
            for (int s = 0; s < kFusedStages; ++s) mbar_init(&s_bar[s], 1u);  // (unused stages stay idle)
            fence_barrier_init();
        }
        __syncthreads();
    }
    // one thread arms stage t % nstage and copies tile t's cache words into it
    auto issue = [&](int t, int64_t j0_, int64_t j1_) {
        const int64_t tb = j0_ + static_cast<int64_t>(t) * p.tile;
        const int cnt = (tb + p.tile < j1_) ? p.tile : static_cast<int>(j1_ - tb);
        const unsigned bytes = static_cast<unsigned>(cnt) * kRaw * 16u;
        unsigned long long *bar = &s_bar[t % nstage];
        unsigned char *dst = smem + static_cast<size_t>(t % nstage) * ring_stride;
        const unsigned char *src = reinterpret_cast<const unsigned char *>(p.dsc + tb * kRaw);
        fence_proxy_async_smem();
        mbar_arm(bar, bytes);
        for (unsigned off = 0; off < bytes; off += 32768u)
            bulk_copy_g2s(dst + off, src + off, (bytes - off < 32768u) ? bytes - off : 32768u, bar);
    };

    __shared__ int s_last;
    __shared__ float s_gnd[kMaxThreads];  // several warps per sink: the groups' nearest neighbours
    __shared__ int s_gnid[kMaxThreads];
    for (int round = 0;; ++round) {
        int64_t item;
        if (p.static_items) {
            // one work item per CTA (grid == n_items): no counter to contend on
            if (round > 0) break;
            item = blockIdx.x;
        } else {
            __syncthreads();
            if (tid == 0) s_item = atomicAdd(p.queue, 1u);
            __syncthreads();
            item = s_item;
        }
        if (item >= p.n_items) break;
        // items 0 .. n_whole-1: i-blocks over all sources (final outputs);
        // then (i-block, slice) items of the remaining i-blocks (partials)
        // (work items, i-blocks and slices stay below 2^31)
        const bool whole = item < p.n_whole;
        int64_t iblk;
        int slice;
        if (whole) {
            iblk = item;
            slice = 0;
        } else {
            // i-block-major: the slices of one i-block are taken one after the
            // other, so they finish close together and its partial sums are
            // reduced while they are still fresh in L2
            const unsigned k = static_cast<unsigned>(item - p.n_whole);
            const unsigned sp = static_cast<unsigned>(p.split);
            iblk = p.n_whole + static_cast<int64_t>(k / sp);
            slice = static_cast<int>(k % sp);
        }

        // the slice's first tiles are requested before the sinks are read, so
        // the two memory round trips overlap
        const int64_t j0 = whole ? p.j_begin : p.j_begin + static_cast<int64_t>(slice) * p.slice_len;
        const int64_t j1 = (whole || j0 + p.slice_len >= p.j_end) ? p.j_end : j0 + p.slice_len;
        const int n_tiles = static_cast<int>((j1 - j0 + p.tile - 1) / p.tile);
        if constexpr (!FUSED) {
#pragma unroll
            for (int s = 0; s < kStages - 1; ++s) {
                if (s < n_tiles) load_tile<P>(p, smem, s, j0, j1);
                cp_async_commit();
            }
        }

        // fused prediction: the first tiles' cache words are requested before
        // the sinks are read
        if constexpr (FUSED) {
            if (tid == 0)
                for (int s = 0; s < nstage && s < n_tiles; ++s) issue(s, j0, j1);
        }

        typename P::Sink sk[IPT];
        typename P::Acc ac[IPT];
        bool val[IPT];
        int64_t ii[IPT];
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            ii[k] = iblk * p.sinks_per_cta + static_cast<int64_t>(k) * slots + islot;
            val[k] = ii[k] < p.n_i;
            const int raw = val[k] ? __ldg(p.i_idx + ii[k]) : 0;
            if (p.sink_rec) {
                // explicit sink: its own record; raw names its slot for the self pair (< 0: none)
                if (val[k] && raw >= p.n_loaded) {
                    atomicOr(p.err, 1u);
                    val[k] = false;
                }
                P::load_sink(p.sink_rec, val[k] ? ii[k] : 0, sk[k]);
                sk[k].slot = (val[k] && raw >= 0) ? raw : -1;
            } else {
                if (val[k] && (raw < 0 || raw >= p.n_loaded)) {
                    atomicOr(p.err, 1u);  // reported by sp2_sync; this sink is skipped
                    val[k] = false;
                }
                const int slot = val[k] ? raw : static_cast<int>(p.j_begin);
                // fused: the sink's cache words are only prefetched here; it is
                // predicted after the first tile, so the fetch overlaps that
                // tile's copy and prediction (and holds no registers)
                if constexpr (FUSED && P::kCanFuse) {
                    const float4 *w = p.dsc + static_cast<int64_t>(slot) * kRaw;
                    prefetch_l1(w);
                    prefetch_l1(w + kRaw - 1);
                } else {
                    P::load_sink(p.rec, slot, sk[k]);
                }
                sk[k].slot = val[k] ? slot : -1;
            }
            if constexpr (is_nb<P>::value) P::set_nb(sk[k], p, ii[k], val[k]);
            P::init(ac[k]);
            P::zero_totals(tot + k * P::NS * nt, nt);
        }
        bool any_val = false;
#pragma unroll
        for (int k = 0; k < IPT; ++k) any_val |= val[k];
        const bool warp_busy = __any_sync(kFull, any_val);
        int since_flush = 0;
        for (int t = 0; t < n_tiles; ++t) {
            const int tb = static_cast<int>(j0) + t * p.tile;
            const unsigned char *st;
            if constexpr (FUSED) {
                const int stage = t % nstage;
                // the barrier of this wait also means: every thread has left the previous tile
                if (!__syncthreads_and(mbar_wait(&s_bar[stage], (phase >> stage) & 1u))) {
                    // the copy did not complete within the limit: report it and
                    // wait once more (bounded); give up on the pass if that fails too
                    if (tid == 0) atomicOr(p.err, 2u);
                    if (!__syncthreads_and(mbar_wait(&s_bar[stage], (phase >> stage) & 1u))) return;
                }
                phase ^= 1u << stage;
                const int cnt = (tb + p.tile < j1) ? p.tile : static_cast<int>(j1 - tb);
                predict_staged_tile<P>(p, reinterpret_cast<const float4 *>(smem + stage * ring_stride), cnt, pbuf, jl);
                if constexpr (P::kCanFuse) {
                    if (t == 0 && !p.sink_rec) {
#pragma unroll
                        for (int k = 0; k < IPT; ++k) {
                            const int slot = sk[k].slot;
                            P::sink_from(P::predict(p.dsc, val[k] ? slot : static_cast<int>(p.j_begin), p.t_hi, p.t_lo), sk[k]);
                            sk[k].slot = slot;
                        }
                    }
                }
                __syncthreads();  // pair records ready, the stage is free again
                if (tid == 0 && t + nstage < n_tiles) issue(t + nstage, j0, j1);
                st = pbuf;
            } else {
                cp_async_wait<kStages - 2>();
                __syncthreads();
                if (t + kStages - 1 < n_tiles) load_tile<P>(p, smem, t + kStages - 1, j0, j1);
                cp_async_commit();
                st = smem + (t % kStages) * ring_stride;
                if constexpr (kPair) {
                    // every thread has left the previous tile's pair records (barrier above)
                    pair_tile<P>(st, pbuf, p.tile, jl);
                    __syncthreads();
                    st = pbuf;
                }
            }
            const int te = (tb + p.tile < j1) ? tb + p.tile : static_cast<int>(j1);
            bool mine = false;
#pragma unroll
            for (int k = 0; k < IPT; ++k) mine |= (sk[k].slot >= tb) && (sk[k].slot < te);
            // a warp whose sink slots are all empty (fewer sinks than the CTA
            // holds) skips the tile and leaves the issue slots to the others
            if (warp_busy) {
                // the group's part: c0 .. c0 + per * jl, whose (pair) records start c0 records in
                const unsigned char *sg = st + static_cast<size_t>(c0) * P::RB;
                if (__any_sync(kFull, mine)) tile_loop<P, IPT, true>(sg, tb + c0, per, jl, lj, sk, ac, eps2);
                else tile_loop<P, IPT, false>(sg, tb + c0, per, jl, lj, sk, ac, eps2);
            }
            since_flush += per;
            if (since_flush >= P::kFlush) {
#pragma unroll
                for (int k = 0; k < IPT; ++k) P::flush(ac[k], tot + k * P::NS * nt, nt);
                since_flush = 0;
            }
        }
        cp_async_wait<0>();

        const int isplit = whole ? 1 : p.split;
        const int64_t pn = p.n_i - p.tail_sink0;  // sinks with partial rows
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            P::flush(ac[k], tot + k * P::NS * nt, nt);
            double t[P::NS];
            double nd = d_inf();
            int nid = -1;
            if constexpr (kPair) {
                if constexpr (P::kNN) {
                    if (ac[k].bid >= 0) {
                        nd = f2d_exact(ac[k].bd);
                        nid = ac[k].bid;
                    }
                }
                ds q[P::NS];
                if (warp_busy) merge_lanes_ds<P>(tot + k * P::NS * nt, nt, jl, q, nd, nid);
                if (kMultiWarp && ws > 1) {
                    // groups 1 .. ws-1 leave their merged totals and neighbour in
                    // their own slots; group 0 adds them in group order
                    float2 *t2 = reinterpret_cast<float2 *>(tot + k * P::NS * nt);
                    if (grp > 0 && warp_busy) {
#pragma unroll
                        for (int f = 0; f < P::NS; ++f) t2[f * nt] = make_float2(q[f].h, q[f].l);
                        if (P::kNN) {
                            s_gnd[tid] = static_cast<float>(nd);
                            s_gnid[tid] = nid;
                        }
                    }
                    __syncthreads();
                    if (grp == 0 && warp_busy) {
                        for (int g2 = 1; g2 < ws; ++g2) {
                            const int o = g2 * nt_g;
#pragma unroll
                            for (int f = 0; f < P::NS; ++f) q[f] = ds_add(q[f], ds{t2[f * nt + o].x, t2[f * nt + o].y});
                            if (P::kNN) {
                                const float od = s_gnd[tid + o];
                                const int oid = s_gnid[tid + o];
                                const float d = static_cast<float>(nd);
                                if (od < d || (od == d && static_cast<unsigned>(oid) < static_cast<unsigned>(nid))) {
                                    nd = f2d_exact(od);
                                    nid = oid;
                                }
                            }
                        }
                    }
                    __syncthreads();  // the slots are free again
                }
                if (!warp_busy || grp > 0) continue;  // nothing (more) to write from this warp
                const int64_t pi = ii[k] - p.tail_sink0;
                if (val[k]) write_fields_ds<P>(p, ii[k], isplit, slice, pi, pn, q, jl, lj);
                if (P::kNN && lj == 0 && val[k]) {
                    if (isplit == 1) {
                        if (p.nn_id) p.nn_id[ii[k]] = nid;
                        if (p.nn_r2) p.nn_r2[ii[k]] = (nid < 0) ? d_inf() : nd;
                    } else if (p.sink_major) {
                        constexpr int NF = P::NS + (P::kNN ? 1 : 0);
                        p.part[(pi * NF + P::NS) * isplit + slice] = nd;
                        p.part_id[pi * isplit + slice] = nid;
                    } else {
                        const int64_t stride = static_cast<int64_t>(isplit) * pn;
                        p.part[P::NS * stride + static_cast<int64_t>(slice) * pn + pi] = nd;
                        p.part_id[static_cast<int64_t>(slice) * pn + pi] = nid;
                    }
                }
                continue;
            } else {
                P::nn(ac[k], sk[k], p.rec, p.j_end, jl, nd, nid);
                P::totals(ac[k], tot + k * P::NS * nt, nt, t);
                for (int off = jl >> 1; off > 0; off >>= 1) {
#pragma unroll
                    for (int f = 0; f < P::NS; ++f) t[f] += __shfl_xor_sync(kFull, t[f], off);
                    if (P::kNN) {
                        const double od = __shfl_xor_sync(kFull, nd, off);
                        const int oid = __shfl_xor_sync(kFull, nid, off);
                        nn_merge(nd, nid, od, oid);
                    }
                }
            }
            if (lj == 0 && val[k]) {
                const int64_t pi = ii[k] - p.tail_sink0;
                if (isplit == 1) {
                    P::write_final(p, ii[k], t, nd, nid);
                } else if (p.sink_major) {
                    constexpr int NF = P::NS + (P::kNN ? 1 : 0);
                    double *base = p.part + pi * NF * isplit + slice;
#pragma unroll
                    for (int f = 0; f < P::NS; ++f) base[f * isplit] = t[f];
                    if (P::kNN) {
                        base[P::NS * isplit] = nd;
                        p.part_id[pi * isplit + slice] = nid;
                    }
                } else {
                    const int64_t stride = static_cast<int64_t>(isplit) * pn;
                    double *base = p.part + static_cast<int64_t>(slice) * pn + pi;
#pragma unroll
                    for (int f = 0; f < P::NS; ++f) base[f * stride] = t[f];
                    if (P::kNN) {
                        base[P::NS * stride] = nd;
                        p.part_id[static_cast<int64_t>(slice) * pn + pi] = nid;
                    }
                }
            }
        }
        if (isplit > 1 && p.fused_reduce) {
            // every partial of this CTA is written (barrier); thread 0's fence
            // then makes them visible device-wide before the CTA is counted.
            // The last CTA's thread 0 fences again after the count, and the
            // barrier orders every thread's reads of the other CTAs' partials
            // after that fence (one thread fences for the CTA, as in a grid
            // barrier)
            __syncthreads();
            if (tid == 0) {
                __threadfence();
                const bool last = atomicAdd(p.done + iblk, 1u) == static_cast<unsigned>(p.split - 1);
                if (last) __threadfence();
                s_last = last ? 1 : 0;
            }
            __syncthreads();
            if (s_last) {
                reduce_iblock<P>(p, iblk);
                if (tid == 0) p.done[iblk] = 0u;  // ready for the next launch
                // the i-block's partial sums are consumed: their L2 lines need
                // no write-back to DRAM
                __syncthreads();
                discard_partials<P>(p, iblk);
            }
        }
    }
    cp_async_wait<0>();
    if (p.exit_count && !p.static_items && tid == 0) {
        // the last CTA out resets the work counter for the next launch (every
        // CTA has taken its last item before it is counted here)
        __threadfence();
        if (atomicAdd(p.exit_count, 1u) == gridDim.x - 1) {
            *p.queue = 0u;
            *p.exit_count = 0u;
            __threadfence();
        }
    }
}

// Device-count form (block time-steps): the sink count is read from device
// memory, written there by the kernel that chose the active set, and every
// CTA derives the launch shape from it, with the launch's threads and tile,
// and the host's source split as an upper bound (it sized the partial-sum
// buffers and the reduction counters).  Sources are cut into slices of at
// least one tile; lanes share a sink (j_lanes) while the sinks do not fill a
// CTA or the (i-block, slice) items do not cover the grid; then the split
// aims at ~4 items per CTA.
__device__ __forceinline__ void device_shape(ForceParams &q) {
    const int nt = blockDim.x;
    const int64_t n_i = *q.n_i_dev;
    const int64_t n_j = q.j_end - q.j_begin;
    int64_t cap = n_j / q.tile;
    if (cap > q.split) cap = q.split;
    if (cap < 1) cap = 1;
    int jl = 1;
    while (jl < 32 && jl * 8 < q.tile) {
        const int64_t spc = nt / jl;
        if (spc <= n_i && (n_i + spc - 1) / spc * cap >= gridDim.x) break;
        jl *= 2;
    }
    const int spc = nt / jl;
    const int64_t n_iblk = (n_i + spc - 1) / spc;
    int64_t split = n_iblk > 0 ? (4 * static_cast<int64_t>(gridDim.x) + n_iblk - 1) / n_iblk : 1;
    if (split > cap) split = cap;
    if (split < 1) split = 1;
    const int64_t per_slice = (n_j + split - 1) / split;
    q.slice_len = (per_slice + q.tile - 1) / q.tile * q.tile;
    q.split = static_cast<int>((n_j + q.slice_len - 1) / q.slice_len);
    q.n_i = n_i;
    q.n_iblk = n_iblk;
    q.n_items = n_iblk * q.split;
    q.sinks_per_cta = spc;
    q.jl = jl;
    q.sink_major = q.split >= kWarpReduceMinSplit ? 1 : 0;
}

// Resident CTAs of kMaxThreads that a kernel's register budget must allow
// (0: no bound beyond the block size, the compiler's own choice).  The mixed
// Hermite-4 force pass with nearest neighbour and two sinks per thread (the
// large-N_active kernel) is held to 128 registers, which leaves 16 warps per
// SM instead of 12 at its natural 164; ptxas then spills ~80 bytes, and the
// pass runs 1 % faster (measured at N = N_active = 131072 with the autotuned
// shape).  The same bound on the variant without neighbours (96 bytes of
// spills) made the adjoint benchmark's forward passes 16 % slower, so that
// one keeps its registers.
template <class P, int IPT, bool FUSED>
struct pass_min_blocks { static constexpr int value = 0; };
template <>
struct pass_min_blocks<MixedPairForce<4, true>, 2, false> { static constexpr int value = 2; };

// MODE 0: the pass; 1: the device-count form; 2: several warps per sink.
template <class P, int IPT, bool FUSED, int MODE = 0>
__global__ void __launch_bounds__(kMaxThreads, (pass_min_blocks<P, IPT, FUSED>::value)) pass_kernel(const ForceParams p) {
    constexpr bool DEVN = MODE == 1;
    if constexpr (MODE == 2) {
        pass_body<P, IPT, FUSED, true>(p);
    } else if constexpr (DEVN) {
        static_assert(IPT == 1 && !FUSED, "the device-count form takes one sink per thread");
        ForceParams q = p;
        device_shape(q);
        pass_body<P, IPT, FUSED>(q);
    } else {
        pass_body<P, IPT, FUSED>(p);
    }
}

// Second kernel of the source split: sum the slices of each sink in slice
// order (deterministic, FP64) and take the lexicographic (r2, id) minimum.
template <class P>
__global__ void reduce_kernel(const ReduceParams r) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= r.n_i) return;
    const int64_t stride = static_cast<int64_t>(r.split) * r.n_i;
    double t[P::NS];
#pragma unroll
    for (int f = 0; f < P::NS; ++f) t[f] = 0.0;
    double nd = d_inf();
    int nid = -1;
    for (int s = 0; s < r.split; ++s) {
        const double *base = r.part + static_cast<int64_t>(s) * r.n_i + i;
#pragma unroll
        for (int f = 0; f < P::NS; ++f) t[f] += base[f * stride];
        if (P::kNN) nn_merge(nd, nid, base[P::NS * stride], r.part_id[static_cast<int64_t>(s) * r.n_i + i]);
    }
    P::write_final(r, i, t, nd, nid);
}

// The same reduction with one warp per sink, for many slices, on the
// sink-major layout (a warp's loads are contiguous): lane l sums slices l,
// l+32, ... in order, then a fixed xor-butterfly combines the lanes, so the
// result is still independent of scheduling.
template <class P>
__global__ void reduce_warp_kernel(const ReduceParams r) {
    const int64_t i = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= r.n_i) return;  // uniform across the warp
    constexpr int NF = P::NS + (P::kNN ? 1 : 0);
    const double *row = r.part + i * NF * r.split;
    const int32_t *row_id = r.part_id + i * r.split;
    double t[P::NS];
#pragma unroll
    for (int f = 0; f < P::NS; ++f) t[f] = 0.0;
    double nd = d_inf();
    int nid = -1;
    // (many warps in flight hide the loads here; the chunked loads of
    // lane_sum_slices would only cost registers and occupancy)
    for (int s = lane; s < r.split; s += 32) {
#pragma unroll
        for (int f = 0; f < P::NS; ++f) t[f] += row[f * r.split + s];
        if (P::kNN) nn_merge(nd, nid, row[P::NS * r.split + s], row_id[s]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int f = 0; f < P::NS; ++f) t[f] += __shfl_xor_sync(kFull, t[f], off);
        if (P::kNN) {
            const double od = __shfl_xor_sync(kFull, nd, off);
            const int oid = __shfl_xor_sync(kFull, nid, off);
            nn_merge(nd, nid, od, oid);
        }
    }
    if (lane == 0) P::write_final(r, i, t, nd, nid);
}

// Few sinks, many slices: one 256-thread block per sink on the sink-major
// layout, a warp per field (reduce_sink_fields).
template <class P>
__global__ void __launch_bounds__(256) reduce_block_kernel(const ReduceParams r) {
    __shared__ double s_f[P::NS];
    __shared__ long long s_nd;
    __shared__ int s_nid;
    constexpr int NF = P::NS + (P::kNN ? 1 : 0);
    const int64_t i = blockIdx.x;
    reduce_sink_fields<P>(r.part + i * NF * r.split, r.part_id + i * r.split, r.split, s_f, s_nd, s_nid,
                          [&](const double *t, double d, int id) { P::write_final(r, i, t, d, id); });
}

// ---------------------------------------------------------------------------
// Batched kernel for many small independent systems: persistent warps, each
// fetching (system, up-to-32-sink chunk) items from the device work queue in
// the plan's cost order; one sink per lane, the system's sources read with
// warp-uniform (broadcast) loads that stay in L1 while the chunks of one
// system are processed.
// ---------------------------------------------------------------------------
constexpr int kBatchTile = 64;  // sources per warp-private shared-memory tile

template <class P, bool SELF>
__device__ __forceinline__ void batch_tile_loop(const unsigned char *st, int tb, int n, const typename P::Sink &sk,
                                                typename P::Acc &ac, typename P::real eps2) {
    if constexpr (is_paired<P>::value) {
        // st holds pair records of sources (2k, 2k+1)
        for (int q0 = 0; q0 < n; q0 += P::kChunk) {
            const unsigned char *pq = st + (q0 >> 1) * P::PRB;
            P::template interact2<SELF, true>(P::ld_pair(pq), tb + q0, 1, 0, sk, ac, eps2);
#pragma unroll
            for (int u = 2; u < P::kChunk; u += 2)
                P::template interact2<SELF, false>(P::ld_pair(pq + (u >> 1) * P::PRB), tb + q0 + u, 1, u, sk, ac, eps2);
            P::fold(ac, tb + q0, pq, P::PRB, sk);
        }
    } else {
        for (int q0 = 0; q0 < n; q0 += P::kChunk) {
            {
                const typename P::Rec r = P::ld_shared(st + q0 * P::RB);
                P::template interact<SELF, true>(r, tb + q0, 0, sk, ac, eps2);
            }
#pragma unroll
            for (int u = 1; u < P::kChunk; ++u) {
                const typename P::Rec r = P::ld_shared(st + (q0 + u) * P::RB);
                P::template interact<SELF, false>(r, tb + q0 + u, u, sk, ac, eps2);
            }
            if constexpr (has_fold_tile<P>::value) P::fold_tile(ac, tb + q0, st + q0 * P::RB, sk);
            else P::fold(ac, tb + q0);
        }
    }
}

// Warps take (system, up-to-32-sink chunk) items from the device queue in the
// plan's cost order; one sink per lane.  The system's sources pass through a
// warp-private shared-memory tile filled with coalesced 16-byte loads (ragged
// ends padded with filler records), then are read as broadcasts.  The running
// totals stay in registers (systems are short).
template <class P>
__global__ void __launch_bounds__(kMaxThreads) batched_kernel(const BatchParams b) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    unsigned char *wbuf = smem + static_cast<size_t>(threadIdx.x >> 5) * kBatchTile * P::RB;
    const typename P::real eps2 = static_cast<typename P::real>(b.eps2);
    constexpr int W = P::RB / 16;
    for (;;) {
        unsigned int item = 0;
        if (lane == 0) item = atomicAdd(b.queue, 1u);
        item = __shfl_sync(kFull, item, 0);
        if (item >= b.n_items) break;
        const int4 it = __ldg(b.items + item);  // {system first slot, size, chunk first slot, chunk size}
        const bool val = lane < it.w;
        const int slot = it.z + (val ? lane : 0);
        typename P::Sink sk;
        typename P::Acc ac;
        P::load_sink(b.rec, slot, sk);
        sk.slot = val ? slot : -1;
        P::init(ac);
        double tot[P::NS];
#pragma unroll
        for (int f = 0; f < P::NS; ++f) tot[f] = 0.0;
        const unsigned char *src = b.rec + static_cast<int64_t>(it.x) * P::RB;
        int since = 0;
        for (int t0 = 0; t0 < it.y; t0 += kBatchTile) {
            const int cnt = min(kBatchTile, it.y - t0);
            const int padded = (cnt + P::kChunk - 1) / P::kChunk * P::kChunk;
            __syncwarp();
            const uint4 *tsrc = reinterpret_cast<const uint4 *>(src + static_cast<int64_t>(t0) * P::RB);
            if constexpr (is_paired<P>::value) {
                for (int c = lane; c < (padded >> 1) * W; c += 32) {
                    const int pr = c / W, w = c - pr * W;
                    const uint4 x = (2 * pr < cnt) ? __ldg(tsrc + 2 * pr * W + w) : P::sentinel(w);
                    const uint4 y = (2 * pr + 1 < cnt) ? __ldg(tsrc + (2 * pr + 1) * W + w) : P::sentinel(w);
                    P::store_pair_word(*reinterpret_cast<const float4 *>(&x), *reinterpret_cast<const float4 *>(&y), w,
                                       wbuf + pr * P::PRB);
                }
            } else {
                for (int c = lane; c < padded * W; c += 32) {
                    uint4 w4;
                    if (c < cnt * W) w4 = __ldg(tsrc + c);
                    else w4 = P::sentinel(c % W);
                    *reinterpret_cast<uint4 *>(wbuf + 16 * c) = w4;
                }
            }
            __syncwarp();
            const int tb = it.x + t0;
            const bool mine = val && slot >= tb && slot < tb + cnt;
            if (__any_sync(kFull, mine)) batch_tile_loop<P, true>(wbuf, tb, padded, sk, ac, eps2);
            else batch_tile_loop<P, false>(wbuf, tb, padded, sk, ac, eps2);
            since += padded;
            if (since >= P::kFlush) {
                P::flush(ac, tot, 1);
                since = 0;
            }
        }
        P::flush(ac, tot, 1);
        double t[P::NS];
        P::totals(ac, tot, 1, t);
        double nd;
        int nid;
        if constexpr (has_fold_tile<P>::value || is_paired<P>::value) P::nn_acc(ac, nd, nid);
        else P::nn(ac, sk, b.rec, static_cast<int64_t>(it.x) + it.y, 1, nd, nid);
        if (val) P::write_final(b, static_cast<int64_t>(slot) - b.out_base, t, nd, nid);
    }
}

// ---------------------------------------------------------------------------
// Instantiation helpers for one (order, precision) translation unit.
// ---------------------------------------------------------------------------
// Dynamic shared memory of a pass launch with tile records per stage: the
// record ring (cache words with fused prediction), one tile of pair records (paired
// policies) and, for the mixed policies, the totals of every (thread, sink,
// field).  The launch and occupancy helpers take the tile, not bytes.
template <class P, int IPT, bool FUSED>
inline size_t pass_smem(size_t tile, int threads, int fused_stages = kFusedStages) {
    const size_t ring = FUSED ? fused_stages * tile * raw_words<P>::value * 16 : kStages * tile * P::RB;
    const size_t pair_bytes = is_paired<P>::value ? tile * P::RB : 0;
    return ring + pair_bytes + (P::kSmemTotals ? static_cast<size_t>(threads) * IPT * P::NS * sizeof(double) : 0);
}

constexpr int kMaxDynSmem = kMaxPassSmem;

template <class P, int IPT, bool FUSED, int DEVN = 0>
inline cudaError_t launch_pass(const ForceParams &p, int grid, int threads, size_t tile, cudaStream_t s) {
    static bool attr_set = false;
    const size_t smem = pass_smem<P, IPT, FUSED>(tile, threads, p.fused_stages);
    if (smem > static_cast<size_t>(kMaxDynSmem)) return cudaErrorInvalidConfiguration;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(pass_kernel<P, IPT, FUSED, DEVN>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    pass_kernel<P, IPT, FUSED, DEVN><<<grid, threads, smem, s>>>(p);
    return cudaGetLastError();
}

template <class P, int IPT, bool FUSED, int DEVN = 0>
inline cudaError_t occupancy_pass(int threads, size_t tile, int *blocks, int fused_stages = 0) {
    const size_t smem = pass_smem<P, IPT, FUSED>(tile, threads, fused_stages > 0 ? fused_stages : kFusedStages);
    if (smem > static_cast<size_t>(kMaxDynSmem)) {
        *blocks = 0;
        return cudaSuccess;
    }
    cudaError_t e = cudaFuncSetAttribute(pass_kernel<P, IPT, FUSED, DEVN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kMaxDynSmem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, pass_kernel<P, IPT, FUSED, DEVN>, threads, smem);
}

// The device-count pass (block time-steps) exists for the order-4 and
// order-6 force policies without nearest neighbours, one sink per thread.
template <class P>
struct takes_device_count { static constexpr bool value = false; };
template <>
struct takes_device_count<MixedPairForce<4, false>> { static constexpr bool value = true; };
template <>
struct takes_device_count<Fp64Force<4, false>> { static constexpr bool value = true; };
template <>
struct takes_device_count<MixedPairForce<6, false>> { static constexpr bool value = true; };
template <>
struct takes_device_count<Fp64Force<6, false>> { static constexpr bool value = true; };

template <class P, bool FUSED>
inline cudaError_t dispatch_ipt_f(bool occ, int ipt, const ForceParams *p, int grid, int threads, size_t tile,
                                  cudaStream_t s, int *blocks, int fstages = 0, int mw = 0) {
    if (mw) {  // several warps per sink: one sink per thread, paired force policies
        if constexpr (shares_sinks<P>::value) {
            if (ipt != 1) return cudaErrorInvalidValue;
            return occ ? occupancy_pass<P, 1, FUSED, 2>(threads, tile, blocks, fstages)
                       : launch_pass<P, 1, FUSED, 2>(*p, grid, threads, tile, s);
        } else {
            return cudaErrorInvalidValue;
        }
    }
    switch (ipt) {
        case 1: return occ ? occupancy_pass<P, 1, FUSED>(threads, tile, blocks, fstages) : launch_pass<P, 1, FUSED>(*p, grid, threads, tile, s);
        case 2: return occ ? occupancy_pass<P, 2, FUSED>(threads, tile, blocks, fstages) : launch_pass<P, 2, FUSED>(*p, grid, threads, tile, s);
        case 4: return occ ? occupancy_pass<P, 4, FUSED>(threads, tile, blocks, fstages) : launch_pass<P, 4, FUSED>(*p, grid, threads, tile, s);
        default: return cudaErrorInvalidValue;
    }
}

// fused = 1 is available for the mixed force policies only
template <class P>
inline cudaError_t dispatch_ipt(bool occ, int ipt, const ForceParams *p, int grid, int threads, size_t tile,
                                cudaStream_t s, int *blocks, int fused = 0, int devn = 0, int fstages = 0,
                                int mw = 0) {
    if constexpr (takes_device_count<P>::value) {
        if (devn) {
            if (ipt != 1 || fused || mw) return cudaErrorInvalidValue;
            return occ ? occupancy_pass<P, 1, false, 1>(threads, tile, blocks)
                       : launch_pass<P, 1, false, 1>(*p, grid, threads, tile, s);
        }
    } else {
        if (devn) return cudaErrorInvalidValue;
    }
    if constexpr (P::kCanFuse && is_paired<P>::value) {
        if (fused) return dispatch_ipt_f<P, true>(occ, ipt, p, grid, threads, tile, s, blocks, fstages, mw);
    } else {
        if (fused) return cudaErrorInvalidValue;
    }
    return dispatch_ipt_f<P, false>(occ, ipt, p, grid, threads, tile, s, blocks, 0, mw);
}

// Neighbour-list kernels exist for one sink per thread only.
template <class P>
inline cudaError_t dispatch_nb(bool occ, int ipt, const ForceParams *p, int grid, int threads, size_t tile,
                               cudaStream_t s, int *blocks, int fused, int fstages = 0, int mw = 0) {
    if (ipt != 1) return cudaErrorInvalidValue;
    if constexpr (P::kCanFuse && is_paired<P>::value) {
        if (fused && mw)
            return occ ? occupancy_pass<P, 1, true, 2>(threads, tile, blocks, fstages)
                       : launch_pass<P, 1, true, 2>(*p, grid, threads, tile, s);
        if (fused)
            return occ ? occupancy_pass<P, 1, true>(threads, tile, blocks, fstages)
                       : launch_pass<P, 1, true>(*p, grid, threads, tile, s);
    } else {
        if (fused) return cudaErrorInvalidValue;
    }
    if (mw) {
        if constexpr (shares_sinks<P>::value)
            return occ ? occupancy_pass<P, 1, false, 2>(threads, tile, blocks)
                       : launch_pass<P, 1, false, 2>(*p, grid, threads, tile, s);
        else
            return cudaErrorInvalidValue;
    }
    return occ ? occupancy_pass<P, 1, false>(threads, tile, blocks) : launch_pass<P, 1, false>(*p, grid, threads, tile, s);
}

template <class P>
inline cudaError_t launch_reduce(const ReduceParams &r, cudaStream_t s) {
    const int threads = 256;
    if (r.split >= kWarpReduceMinSplit && r.n_i <= kBlockReduceMaxSinks) {
        reduce_block_kernel<P><<<static_cast<unsigned>(r.n_i), 256, 0, s>>>(r);
    } else if (r.split >= kWarpReduceMinSplit) {
        const int64_t grid = (32 * r.n_i + threads - 1) / threads;
        reduce_warp_kernel<P><<<static_cast<unsigned>(grid), threads, 0, s>>>(r);
    } else {
        const int64_t grid = (r.n_i + threads - 1) / threads;
        reduce_kernel<P><<<static_cast<unsigned>(grid), threads, 0, s>>>(r);
    }
    return cudaGetLastError();
}

template <class P>
inline size_t batched_smem(int threads) {
    return static_cast<size_t>(threads / 32) * kBatchTile * P::RB;
}

template <class P>
inline cudaError_t launch_batched(const BatchParams &b, int grid, int threads, cudaStream_t s) {
    batched_kernel<P><<<grid, threads, batched_smem<P>(threads), s>>>(b);
    return cudaGetLastError();
}

template <class P>
inline cudaError_t occupancy_batched(int threads, int *blocks) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, batched_kernel<P>, threads, batched_smem<P>(threads));
}

}  // namespace sp2

// Defines the five per-TU entry points: the pass kernel and its reduction use
// POLICY<ORDER, NN>, the batched kernel BATCH_POLICY<ORDER, NN>.
#define SP2_DEFINE_FORCE_TU(SUFFIX, POLICY, BATCH_POLICY, ORDER)                                           \
    namespace sp2 {                                                                                        \
    cudaError_t launch_force_##SUFFIX(const KernelKey &k, const ForceParams &p, int grid, int threads,     \
                                      size_t tile, cudaStream_t s) {                                       \
        if (k.nb)                                                                                          \
            return k.nn ? dispatch_nb<WithNeighbours<POLICY<ORDER, true>>>(false, k.ipt, &p, grid, threads,  \
                                                                           tile, s, nullptr, k.fused, 0,   \
                                                                           k.mw)                           \
                        : cudaErrorInvalidValue;                                                           \
        return k.nn ? dispatch_ipt<POLICY<ORDER, true>>(false, k.ipt, &p, grid, threads, tile, s, nullptr,  \
                                                        k.fused, k.devn, 0, k.mw)                          \
                    : dispatch_ipt<POLICY<ORDER, false>>(false, k.ipt, &p, grid, threads, tile, s, nullptr, \
                                                         k.fused, k.devn, 0, k.mw);                        \
    }                                                                                                      \
    cudaError_t occupancy_force_##SUFFIX(const KernelKey &k, int threads, size_t tile, int *blocks) {       \
        if (k.nb)                                                                                          \
            return k.nn ? dispatch_nb<WithNeighbours<POLICY<ORDER, true>>>(true, k.ipt, nullptr, 0, threads, \
                                                                           tile, 0, blocks, k.fused,        \
                                                                           k.fused_stages, k.mw)            \
                        : cudaErrorInvalidValue;                                                           \
        return k.nn ? dispatch_ipt<POLICY<ORDER, true>>(true, k.ipt, nullptr, 0, threads, tile, 0, blocks,  \
                                                        k.fused, k.devn, k.fused_stages, k.mw)             \
                    : dispatch_ipt<POLICY<ORDER, false>>(true, k.ipt, nullptr, 0, threads, tile, 0, blocks, \
                                                         k.fused, k.devn, k.fused_stages, k.mw);           \
    }                                                                                                      \
    cudaError_t launch_reduce_##SUFFIX(const KernelKey &k, const ReduceParams &r, cudaStream_t s) {        \
        return k.nn ? launch_reduce<POLICY<ORDER, true>>(r, s) : launch_reduce<POLICY<ORDER, false>>(r, s); \
    }                                                                                                      \
    cudaError_t launch_batched_##SUFFIX(int nn, const BatchParams &b, int grid, int threads,               \
                                        cudaStream_t s) {                                                  \
        return nn ? launch_batched<BATCH_POLICY<ORDER, true>>(b, grid, threads, s)                               \
                  : launch_batched<BATCH_POLICY<ORDER, false>>(b, grid, threads, s);                             \
    }                                                                                                      \
    cudaError_t occupancy_batched_##SUFFIX(int nn, int threads, int *blocks) {                             \
        return nn ? occupancy_batched<BATCH_POLICY<ORDER, true>>(threads, blocks)                                \
                  : occupancy_batched<BATCH_POLICY<ORDER, false>>(threads, blocks);                              \
    }                                                                                                      \
    }
