// Exact fixed-point arithmetic for inter-tile sums: a tile's sum S 2^(k-K)
// becomes a 128-bit integer with 2^-90 resolution relative to 2^K, so sums of
// any number of tiles in any order are exact and identical everywhere.  Also
// the conversions back to float pairs and doubles.
#pragma once

#include "pf_device.cuh"

namespace pf {

constexpr int kFixFrac = 90;  // fixed point: value * 2^90

typedef __int128 i128;

// ---------------------------------------------------------------------------
// Exact fixed-point helpers.
// ---------------------------------------------------------------------------
// f * 2^sh * 2^kFixFrac, truncated toward zero (f finite; |f| <= 2^15).
__device__ __forceinline__ i128 fixed_of(float f, int sh) {
    const uint32_t b = __float_as_uint(f);
    const int e = (int)((b >> 23) & 0xffu);
    if (e == 0) return 0;  // zero, or a denormal far below the resolution
    const uint64_t m = (b & 0x7fffffu) | 0x800000u;
    const int s = e - 150 + sh + kFixFrac;  // f = m 2^(e-150)
    i128 v;
    if (s >= 0) v = (s > 100) ? (i128)0 : ((i128)m << s);
    else v = (s <= -24) ? (i128)0 : (i128)(m >> (-s));
    return (b >> 31) ? -v : v;
}

__device__ __forceinline__ i128 shfl_up_i128(i128 v, int o) {
    const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
    const unsigned long long l2 = __shfl_up_sync(0xffffffffu, lo, o);
    const unsigned long long h2 = __shfl_up_sync(0xffffffffu, hi, o);
    return (i128)(((unsigned __int128)h2 << 64) | l2);
}

__device__ __forceinline__ i128 warp_scan_i128(i128 v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const i128 h = shfl_up_i128(v, o);
        if (lane >= o) v += h;
    }
    return v;
}

// 2^e as a float for e in [-149, 127] (exact), +inf above, 0 below.
__device__ __forceinline__ float pow2f(int e) {
    if (e > 127) return INFINITY;
    if (e >= -126) return __int_as_float((127 + e) << 23);
    if (e >= -149) return __int_as_float(1 << (e + 149));
    return 0.f;
}

// 2^e as a double for e in [-1022, 1023].
__device__ __forceinline__ double pow2d(int e) {
    e = max(-1022, min(1023, e));
    return __longlong_as_double((long long)(1023 + e) << 52);
}

// A non-negative fixed-point value as a float pair (top 24 and next 24 bits).
__device__ __forceinline__ fpair fixed_to_pair(i128 v) {
    if (v <= 0) return {0.f, 0.f};
    const unsigned long long hi = (unsigned long long)(v >> 64), lo = (unsigned long long)v;
    const int n = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);  // bit length
    if (n <= 24) return {(float)(uint32_t)lo * pow2f(-kFixFrac), 0.f};
    const int s1 = n - 24;
    const uint32_t top = (uint32_t)(v >> s1);
    const i128 rem = v - ((i128)top << s1);
    const float h = (float)top * pow2f(s1 - kFixFrac);
    float l;
    if (s1 <= 24) {
        l = (float)(uint32_t)rem * pow2f(-kFixFrac);
    } else {
        const uint32_t nxt = (uint32_t)(rem >> (s1 - 24));
        l = (float)nxt * pow2f(s1 - 24 - kFixFrac);
    }
    return {h, l};
}

__device__ __forceinline__ double fixed_to_double(i128 v) {
    const double hi = (double)(long long)(v >> 64);
    const double lo = (double)(unsigned long long)v;
    return __fma_rn(hi, 18446744073709551616.0, lo) * 0x1p-90;
}

}  // namespace pf
