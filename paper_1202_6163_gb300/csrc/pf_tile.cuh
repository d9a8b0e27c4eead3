// Tile scan: the per-tile half of the collective prefix sum of weights
// (Section 2: multinomial, stratified and systematic resamplers need the
// cumulative weights c_i).
//
// One CTA of kThreads threads owns a tile of n <= kTileMax consecutive
// log-weights.  Thread k holds K consecutive elements (K in {4, 8, 16}) in
// registers, loaded with 128-bit accesses.  The tile:
//   1. finds its largest log-weight m_t and exponent k_t ~ m_t log2 e;
//   2. forms w_i = exp(lw_i - k_t ln 2) with an error-free subtraction;
//   3. runs a Kahan-compensated serial scan per thread and an exact block scan
//      of the per-thread totals in 64-bit fixed point;
//   4. leaves in registers the tile-local inclusive cumulative weights v_i
//      (float, monotone across threads) and a bit mask of the elements with
//      positive weight.
#pragma once

#include "pf_device.cuh"

namespace pf {

constexpr int kWarps = kThreads / 32;

struct TileShared {
    long long wtot[kWarps];  // per-warp sums of the thread totals (fixed point)
    float redf[kWarps];
    int i_last;
};

struct TileSummary {
    int k;        // tile exponent
    fpair S;      // tile sum relative to 2^k (compensated pair)
    int i_last;   // tile-local index of the last positive weight, -1 if none
    int bad;      // a NaN or +inf log-weight was seen
};

// This thread's share of the tile.
struct TileThread {
    float v[kMaxPerThread];  // tile-local inclusive cumulative weight of element e0 + i
    uint32_t pos;            // bit i: element e0 + i has positive weight
    int K;                   // elements per thread
    int e0;                  // first tile-local element of this thread
};

__device__ __forceinline__ int per_thread_count(int n) {
    const int q = (n + kThreads - 1) / kThreads;
    return q <= 4 ? 4 : (q <= 8 ? 8 : 16);
}

__device__ __forceinline__ bool zero_flag(float v) { return __float_as_uint(v) >> 31; }

// Loads this thread's KK elements (tile-local e0 .. e0+KK) of base[lo..n);
// base is 16-byte aligned, in global memory or (SMEM) in shared memory.
// Slots outside [lo, n) read as -inf (zero weight).
template <int KK, bool SMEM = false>
__device__ __forceinline__ void tile_load_k(const float* __restrict__ base, int lo, int n, int e0,
                                            float (&x)[kMaxPerThread]) {
#pragma unroll
    for (int q = 0; q < KK / 4; ++q) {
        const int idx = e0 + 4 * q;
        if (idx >= lo && idx + 3 < n) {
            const float4 v = SMEM ? *reinterpret_cast<const float4*>(base + idx)
                                  : __ldg(reinterpret_cast<const float4*>(base + idx));
            x[4 * q + 0] = v.x;
            x[4 * q + 1] = v.y;
            x[4 * q + 2] = v.z;
            x[4 * q + 3] = v.w;
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r)
                x[4 * q + r] = (idx + r >= lo && idx + r < n) ? (SMEM ? base[idx + r] : __ldg(base + idx + r)) : -INFINITY;
        }
    }
}

// Block-wide; every thread of the CTA must call it.  Scans base[0..n) with the
// first `lo` slots taken as zero weights; fills th (this thread's elements) and
// returns the tile summary (identical in every thread).
// KK elements per thread (n <= KK * kThreads); tile_scan picks KK from n.
template <int KK, bool SMEM = false>  // SMEM: base is a copy of the tile in shared memory
__device__ __forceinline__ TileSummary tile_scan_k(const float* __restrict__ base, int lo, int n, TileShared& sm,
                                                   TileThread& th) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int e0 = tid * KK;
    th.K = KK;
    th.e0 = e0;

    if (tid == 0) sm.i_last = -1;

    float* x = th.v;
    tile_load_k<KK, SMEM>(base, lo, n, e0, th.v);

    // 1. tile maximum and domain check: the thread's maximum propagates NaN, so
    // one test of it finds a NaN or +inf element
    float m = -INFINITY;
#pragma unroll
    for (int i = 0; i < KK; ++i) m = fmax_nan(m, x[i]);
    int bad = !(m <= 3.402823466e38f);
    m = warp_max_redux(m);
    if (lane == 0) sm.redf[warp] = m;
    bad = __syncthreads_or(bad);
    const float mt = warp_max_redux(lane < kWarps ? sm.redf[lane] : -INFINITY);
    const int k = tile_exponent(mt);
    const fpair R = tile_reference(k);

    // 2-3. weights and the compensated per-thread scan (x[] becomes the running sum)
    float s = 0.f, c = 0.f;
    int p = -1;
    uint32_t posbits = 0;
#pragma unroll
    for (int i = 0; i < KK; ++i) {
        const float w = weight_rel(x[i], R);
        if (w > 0.f) {
            p = i;
            posbits |= 1u << i;
        }
        const float y = __fsub_rn(w, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
        x[i] = s;
    }
    th.pos = posbits;

    // block exclusive scan of the per-thread totals in exact 64-bit fixed point
    // (resolution 2^-48 relative to 2^k; a tile sum is below 2^14): exact
    // sums are monotone, and every thread knows its own next base
    const long long tot = __float2ll_rn(s * 0x1p48f) + __float2ll_rn(-c * 0x1p48f);
    long long inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long h = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += h;
    }
    if (lane == 31) sm.wtot[warp] = inc;
    const int il = __reduce_max_sync(0xffffffffu, p >= 0 ? e0 + p : -1);
    if (lane == 0 && il >= 0) atomicMax(&sm.i_last, il);
    __syncthreads();
    // every warp scans the kWarps warp totals (lane w holds warp w's)
    long long ws = lane < kWarps ? sm.wtot[lane] : 0;
#pragma unroll
    for (int o = 1; o < kWarps; o <<= 1) {
        const long long h = __shfl_up_sync(0xffffffffu, ws, o);
        if (lane >= o) ws += h;
    }
    const long long total = __shfl_sync(0xffffffffu, ws, kWarps - 1);
    const long long wbase = warp > 0 ? __shfl_sync(0xffffffffu, ws, warp - 1) : 0;
    const long long excl = wbase + inc - tot;
    const float Vk = (float)excl * 0x1p-48f, Vn = (float)(excl + tot) * 0x1p-48f;
    const float S_hi = (float)total;
    const fpair S = {S_hi * 0x1p-48f, (float)(total - (long long)S_hi) * 0x1p-48f};

    // 4. tile-local cumulative weights; elements from the last positive one on
    // take the next base so that no gap is left between threads
#pragma unroll
    for (int i = 0; i < KK; ++i) x[i] = (i >= p) ? Vn : fminf(__fadd_rn(Vk, x[i]), Vn);

    TileSummary ts;
    ts.k = k;
    ts.S = S;
    ts.i_last = sm.i_last;
    ts.bad = bad;
    return ts;
}

// Block-wide; KK from the tile length (4, 8 or 16 elements per thread).
__device__ __forceinline__ TileSummary tile_scan(const float* __restrict__ base, int lo, int n, TileShared& sm,
                                                 TileThread& th) {
    const int K = per_thread_count(n);
    if (K == 4) return tile_scan_k<4>(base, lo, n, sm, th);
    if (K == 8) return tile_scan_k<8>(base, lo, n, sm, th);
    return tile_scan_k<16>(base, lo, n, sm, th);
}

}  // namespace pf
