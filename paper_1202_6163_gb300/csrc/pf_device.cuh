// Device-side building blocks shared by the resampling kernels.
//
// Everything here is written for sm_103a (GB300): 32-wide warps, FP32 per
// element, FP64 only for per-tile carries (FP64 issue rate on this part is a
// small fraction of FP32), integer Philox.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pf_internal.h"

namespace pf {

// ---------------------------------------------------------------------------
// Philox-4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 products
// whose halves are permuted and xored with the other counter words and the
// round key; the key advances by the Weyl increments each round.
// ---------------------------------------------------------------------------
struct u32x4 {
    uint32_t x, y, z, w;
};

// ROUNDS rounds of the same function: 10 is the default stream; 7 (listed in
// SC'11 among the Crush-resistant members) is the opt-in cheaper Metropolis stream.
template <int ROUNDS = 10>
__device__ __forceinline__ u32x4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        // one 32x32->64 product each (both halves used)
        const uint64_t a = (uint64_t)0xD2511F53u * c0;
        const uint64_t b = (uint64_t)0xCD9E8D57u * c2;
        c0 = (uint32_t)(b >> 32) ^ c1 ^ k0;
        c1 = (uint32_t)b;
        c2 = (uint32_t)(a >> 32) ^ c3 ^ k1;
        c3 = (uint32_t)a;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return {c0, c1, c2, c3};
}

__device__ __forceinline__ uint32_t word_of(const u32x4& r, int s) {
    return s == 0 ? r.x : (s == 1 ? r.y : (s == 2 ? r.z : r.w));
}

// u23: odd multiples of 2^-24 in (0,1); exact in float.
__device__ __forceinline__ float u23f(uint32_t x) {
    return __uint2float_rn(((x >> 9) << 1) | 1u) * 0x1p-24f;
}

// u32 = (2x+1) 2^-33 as an exact float pair (hi carries the top 24 bits).
__device__ __forceinline__ void u32_pair(uint32_t x, float& hi, float& lo) {
    hi = __uint2float_rn(x >> 8) * 0x1p-24f;
    lo = __uint2float_rn(((x & 0xFFu) << 1) | 1u) * 0x1p-33f;
}

__device__ __forceinline__ uint32_t draw_index(uint32_t x, uint32_t P) { return __umulhi(x, P); }

// ---------------------------------------------------------------------------
// Error-free transformations (Knuth's TwoSum) and float pairs.  The __f*_rn
// intrinsics keep the compiler from contracting or reordering them.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

struct fpair {
    float hi, lo;
};

__device__ __forceinline__ fpair pair_add(fpair a, fpair b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float hi = __fadd_rn(s, e);
    const float lo = __fsub_rn(e, __fsub_rn(hi, s));
    return {hi, lo};
}

// ---------------------------------------------------------------------------
// Tile reference.  A tile's weights are taken relative to 2^k (k near the
// tile's largest log-weight times log2 e), i.e. w_i = exp(lw_i - k ln 2).
// The reference k ln 2 is held as a float pair so that lw_i - k ln 2 is
// formed without rounding loss, and tiles with different k combine by exact
// binary scaling.
// ---------------------------------------------------------------------------
constexpr double kLn2 = 0.69314718055994530942;
constexpr float kLn2Hi = (float)kLn2;
constexpr float kLn2Lo = (float)(kLn2 - (double)(float)kLn2);
constexpr float kLog2e = 1.44269504088896340736f;

__device__ __forceinline__ int tile_exponent(float m) {
    // m = -inf (every weight zero in the tile): any k works, take 0.
    if (!(m > -INFINITY)) return 0;
    float km = fminf(fmaxf(m * kLog2e, -1.0e9f), 1.0e9f);
    return (int)ceilf(km);
}

__device__ __forceinline__ fpair tile_reference(int k) {
    const float kf = (float)k;  // |k| <= 1e9: exact enough; k below 2^24 is exact
    const float hi = __fmul_rn(kf, kLn2Hi);
    const float err = __fmaf_rn(kf, kLn2Hi, -hi);
    return {hi, __fmaf_rn(kf, kLn2Lo, err)};
}

// exp(lw - R) with R = (R.hi, R.lo): the subtraction is error-free and the
// residual d enters as the factor 1 + d + d^2/2 (for a reference k ln 2 beyond
// ~2^16 in magnitude, R.lo, and so d, reaches 4e-3, where the first-order
// factor alone would leave an error d^2/2 near 8e-6).  Zero for lw = -inf.
__device__ __forceinline__ float weight_rel(float lw, fpair R) {
    float s, e;
    two_sum(lw, -R.hi, s, e);
    const float d_lo = __fsub_rn(e, R.lo);
    const float x = expf(s);
    return x > 0.f ? __fmaf_rn(x, __fmaf_rn(d_lo, 0.5f * d_lo, d_lo), x) : 0.f;
}

// ---------------------------------------------------------------------------
// Status word and bounded waits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_status(uint32_t* status, uint32_t code) {
    atomicCAS(status, 0u, code);
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(uint64_t* p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t tag_slot(uint32_t epoch, uint32_t bits) {
    return ((uint64_t)epoch << 32) | bits;
}

// 16-byte loads and stores of two epoch-tagged words.  Each 8-byte word is
// single-copy atomic and carries its own tag, so a reader that sees both tags
// current has both values whatever the order the halves arrived in.
__device__ __forceinline__ void ld_cg_v2(const uint64_t* p, uint64_t& a, uint64_t& b) {
    asm volatile("ld.global.cg.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}

__device__ __forceinline__ void st_v2(uint64_t* p, uint64_t a, uint64_t b) {
    asm volatile("st.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}

__device__ __forceinline__ void red_release_add_u32(uint32_t* p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_v4_u32(uint32_t* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.global.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

__device__ __forceinline__ uint4 ld_cg_v4_u32(const uint32_t* p) {
    uint4 v;
    asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p)
                 : "memory");
    return v;
}

// Float-pair (double-float) arithmetic for the few per-tile scalars that need
// more than float precision; FP64 issue on this part is far slower.
__device__ __forceinline__ fpair fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ fpair pair_mul(fpair a, fpair b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    return fast_two_sum(p, e);
}

__device__ __forceinline__ fpair pair_div(fpair a, fpair b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    // remainder a - q1 b, exactly enough for the second quotient digit
    const float p = __fmul_rn(q1, b.hi);
    const float pe = __fmaf_rn(q1, b.hi, -p);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), __fsub_rn(a.lo, __fmul_rn(q1, b.lo)));
    return fast_two_sum(q1, __fdiv_rn(r, b.hi));
}

__device__ __forceinline__ fpair pair_sub_f(fpair a, float b) {
    float s, e;
    two_sum(a.hi, -b, s, e);
    return fast_two_sum(s, __fadd_rn(e, a.lo));
}

// ceil and floor of a normalised pair below 2^24 in magnitude, as integers.
__device__ __forceinline__ long long pair_ceil(fpair a) {
    const float c = ceilf(a.hi);
    if (c != a.hi) return (long long)c;
    return (long long)a.hi + (long long)ceilf(a.lo);
}

__device__ __forceinline__ long long pair_floor(fpair a) {
    const float f = floorf(a.hi);
    if (f != a.hi) return (long long)f;
    return (long long)a.hi + (long long)floorf(a.lo);
}

// Spin (bounded) until *p carries epoch in its high word; returns false on timeout.
__device__ __forceinline__ bool wait_slot(const uint64_t* p, uint32_t epoch, uint64_t t_start,
                                          uint64_t limit_ns, uint32_t& bits) {
    for (uint32_t it = 0;; ++it) {
        const uint64_t v = ld_acquire_u64(p);
        if ((uint32_t)(v >> 32) == epoch) {
            bits = (uint32_t)v;
            return true;
        }
        if ((it & 63u) == 63u) {
            if (global_ns() - t_start > limit_ns) return false;
            __nanosleep(64);
        }
    }
}

// ---------------------------------------------------------------------------
// Bulk copies global -> shared memory (the tensor-memory-accelerator path,
// cp.async.bulk) completing on an mbarrier: one thread issues a whole tile, the
// block waits on the barrier's phase.  Source, destination and size must be
// 16-byte aligned / multiples of 16 bytes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes barrier initialisation visible to the asynchronous proxy (before first use).
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Orders this thread's earlier shared-memory accesses before later bulk copies into it.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst_smem)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Completes the barrier's current phase without a copy (count 1 barriers).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits, bounded by limit_ns after t_start, for phase `parity` of bar to
// complete; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t t_start, uint64_t limit_ns) {
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 15u) == 15u && global_ns() - t_start > limit_ns) return false;
    }
}

// ---------------------------------------------------------------------------
// Warp and block collectives.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Maximum that propagates NaN (max.NaN): a NaN operand gives NaN.
__device__ __forceinline__ float fmax_nan(float a, float b) {
    float d;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

// Warp maximum of a float in one integer reduction: the bits of a float map to
// an int of the same order (negative values have their magnitude bits
// flipped), so redux.sync's signed maximum is the float maximum.  -inf stays
// the smallest value; a NaN maps above +inf.
__device__ __forceinline__ float warp_max_redux(float v) {
    int b = __float_as_int(v);
    b ^= (b >> 31) & 0x7fffffff;
    b = __reduce_max_sync(0xffffffffu, b);
    b ^= (b >> 31) & 0x7fffffff;
    return __int_as_float(b);
}

__device__ __forceinline__ int warp_max_i(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Inclusive warp scan of float pairs.
__device__ __forceinline__ fpair warp_scan_pair(fpair v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float h = __shfl_up_sync(0xffffffffu, v.hi, o);
        const float l = __shfl_up_sync(0xffffffffu, v.lo, o);
        if (lane >= o) v = pair_add({h, l}, v);
    }
    return v;
}

__device__ __forceinline__ float warp_scan_max(float v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float h = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v = fmaxf(v, h);
    }
    return v;
}

// Inclusive warp scan of doubles (carries only).
__device__ __forceinline__ double warp_scan_d(double v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double h = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += h;
    }
    return v;
}

}  // namespace pf
