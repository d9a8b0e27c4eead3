// Whole steps of a batch of bootstrap particle filters on the linear-Gaussian
// test model (Section 1, steps 1-4 of the paper's filter, on the model
//   x_t = a_f x_{t-1} + N(0, q I),   y_t = x_t + N(0, r I),   D dimensions).
//
// One launch of k_lg_step does, for every filter f and particle j,
//   propagate from the resampled ancestor (the ancestor gather is fused into
//   the state read: x_prev[a_j] is loaded directly, no gathered copy exists),
//   weight by the observation density, and accumulate the weight in logw;
// and, per filter, the log-sum-exp of the new weights, the effective sample
// size, the increment of the marginal log-likelihood and the decision to
// resample before the next step.  The per-filter reduction is fused into the
// producing kernel: each CTA reduces its tile of 1024 log-weights to
// (max, sum exp, sum exp^2) relative to its own max, and the last CTA of a
// filter to arrive (a per-filter counter) combines the tile records.
//
// Resampling itself is pf_resample_batched_masked with the decision array as
// mask, so a step is two launches and can be captured in a CUDA graph.
//
// Noise: Philox-4x32-10 with key = seed and counter (j, t*G + g, f, 6),
// G = D/4; its four words give four N(0,1) draws by the Box-Muller transform
// (words 0,1 -> dimensions 4g, 4g+1; words 2,3 -> 4g+2, 4g+3), with
// z = sqrt(-2 ln u23(w0)) cos(2 pi u23(w1)) and the sine for the second.
#include <cmath>
#include <cstdint>

#include "pf_device.cuh"
#include "pf_internal.h"

namespace pf {
namespace {

constexpr int kLgThreads = 256;
constexpr int kLgPerThread = 4;
constexpr int kLgWarps = kLgThreads / 32;
constexpr uint32_t kTagPropagate = 6;

// The angle 2 pi u is taken to (-pi, pi) (u - 1 is exact for u >= 1/2) where
// the hardware sine and cosine have an absolute error below 2^-21.4; with the
// rounding of the product, each normal is within about 6e-7 * sqrt(-2 ln u1)
// of its exact value.  The logarithm stays the accurate one: near u1 = 1 its
// absolute error is divided by the small radius.
__device__ __forceinline__ void box_muller(uint32_t w0, uint32_t w1, float& z0, float& z1) {
    const float rad = sqrtf(-2.0f * logf(u23f(w0)));
    const float u = u23f(w1);
    const float theta = 6.28318530717958647692f * (u < 0.5f ? u : u - 1.0f);
    float s, c;
    __sincosf(theta, &s, &c);
    z0 = rad * c;
    z1 = rad * s;
}

__device__ __forceinline__ float4 normals4(uint32_t j, uint32_t c1, uint32_t f, uint32_t k0, uint32_t k1) {
    const u32x4 w = philox(j, c1, f, kTagPropagate, k0, k1);
    float4 z;
    box_muller(w.x, w.y, z.x, z.y);
    box_muller(w.z, w.w, z.z, z.w);
    return z;
}

__device__ __forceinline__ float block_max(float v, float* red) {
    v = warp_max(v);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float m = red[0];
#pragma unroll
    for (int w = 1; w < kLgWarps; ++w) m = fmaxf(m, red[w]);
    __syncthreads();
    return m;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void block_sum2(float& a, float& b, float* ra, float* rb) {
    a = warp_sum(a);
    b = warp_sum(b);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        ra[warp] = a;
        rb[warp] = b;
    }
    __syncthreads();
    a = 0.0f;
    b = 0.0f;
#pragma unroll
    for (int w = 0; w < kLgWarps; ++w) {
        a += ra[w];
        b += rb[w];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kLgThreads) k_lg_init(LgParams p) {
    const int64_t n = (int64_t)p.F * p.P;
    const int G = p.D >> 2;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int f = (int)(e / p.P);
        const uint32_t j = (uint32_t)(e - (int64_t)f * p.P);
        float4* xo = reinterpret_cast<float4*>(p.x_next + e * p.D);
        for (int g = 0; g < G; ++g) {
            const float4 z = normals4(j, (uint32_t)g, (uint32_t)f, p.key0, p.key1);
            xo[g] = make_float4(p.m0 + p.sigma * z.x, p.m0 + p.sigma * z.y, p.m0 + p.sigma * z.z,
                                p.m0 + p.sigma * z.w);
        }
        p.lw[e] = 0.0f;
        if (j == 0) {
            p.loglik[f] = 0.0;
            p.log_sum[f] = p.log_P;
            p.ess[f] = (float)p.P;
            p.resample[f] = 0;
        }
    }
}

// GS > 0: D = 4 GS known at compile time; GS = 0: D from the parameters.
template <int GS>
__global__ void __launch_bounds__(kLgThreads) k_lg_step(LgParams p) {
    __shared__ float ra[kLgWarps], rb[kLgWarps];
    __shared__ int last;
    const int f = (int)(blockIdx.x / (unsigned)p.n_tiles);
    const int tile = (int)(blockIdx.x - (unsigned)f * (unsigned)p.n_tiles);
    const int tid = threadIdx.x;
    const int G = GS > 0 ? GS : (p.D >> 2);
    const int D = 4 * G;
    const int64_t base = (int64_t)f * p.P;
    const int rf = __ldcg(p.resample + f);
    const float a = __ldg(p.a + f);
    const float* yf = p.y + (int64_t)f * D;
    const uint32_t c1 = p.t * (uint32_t)G;

    // the filter's arrays; particle indices within a filter fit 32 bits (P < 2^31)
    const uint32_t Pu = (uint32_t)p.P;
    float* lw_f = p.lw + base;
    const int32_t* anc_f = p.anc + base;
    const float4* xprev_f = reinterpret_cast<const float4*>(p.x_prev + base * D);
    float4* xnext_f = reinterpret_cast<float4*>(p.x_next + base * D);

    // loads first (ancestors, then the rows they select, then old log-weights)
    uint32_t jj[kLgPerThread], src[kLgPerThread];
    bool bad_anc = false, bad_w = false;
#pragma unroll
    for (int k = 0; k < kLgPerThread; ++k) {
        jj[k] = (uint32_t)tile * (kLgThreads * kLgPerThread) + (uint32_t)(k * kLgThreads + tid);
        src[k] = jj[k];
        if (rf && jj[k] < Pu) {
            const int32_t q = __ldcs(anc_f + jj[k]);
            if (q < 0 || (uint32_t)q >= Pu) bad_anc = true;
            else src[k] = (uint32_t)q;
        }
    }
    float prev[kLgPerThread];
#pragma unroll
    for (int k = 0; k < kLgPerThread; ++k) prev[k] = (!rf && jj[k] < Pu) ? lw_f[jj[k]] : 0.0f;

    float v[kLgPerThread];
    float m = -INFINITY;
#pragma unroll
    for (int k = 0; k < kLgPerThread; ++k) {
        const uint32_t j = jj[k];
        v[k] = -INFINITY;
        if (j >= Pu) continue;
        const float4* xi = xprev_f + (size_t)src[k] * G;
        float4* xo = xnext_f + (size_t)j * G;
        float ss = 0.0f;
#pragma unroll
        for (int g = 0; g < (GS > 0 ? GS : 16); ++g) {
            if (GS == 0 && g >= G) break;
            const float4 x = __ldcs(xi + g);
            const float4 z = normals4(j, c1 + (uint32_t)g, (uint32_t)f, p.key0, p.key1);
            float4 xn;
            xn.x = a * x.x + p.sigma * z.x;
            xn.y = a * x.y + p.sigma * z.y;
            xn.z = a * x.z + p.sigma * z.z;
            xn.w = a * x.w + p.sigma * z.w;
            __stcs(xo + g, xn);
            const float4 y = *reinterpret_cast<const float4*>(yf + 4 * g);
            const float d0 = y.x - xn.x, d1 = y.y - xn.y, d2 = y.z - xn.z, d3 = y.w - xn.w;
            ss += (d0 * d0 + d1 * d1) + (d2 * d2 + d3 * d3);
        }
        const float w = prev[k] + (p.c_obs - p.inv2r * ss);
        lw_f[j] = w;
        if (w != w || w == INFINITY) bad_w = true;
        v[k] = w;
        m = fmaxf(m, w);
    }
    if (bad_anc) set_status(p.status, ST_INVALID);
    if (bad_w) set_status(p.status, ST_DOMAIN);

    // tile record: (max, sum exp(lw - max), sum exp(2 (lw - max)))
    const float M = block_max(m, ra);
    float s = 0.0f, s2 = 0.0f;
    if (M != -INFINITY) {
#pragma unroll
        for (int k = 0; k < kLgPerThread; ++k) {
            // hardware exp2: relative error ~1e-7 near the maximum, where the sums are decided
            const float e = exp2f((v[k] - M) * 1.44269504088896341f);  // 0 for the masked slots
            s += e;
            s2 += e * e;
        }
    }
    block_sum2(s, s2, ra, rb);
    if (tid == 0) {
        __stcg(p.records + (int64_t)f * p.n_tiles + tile, make_float4(M, s, s2, 0.0f));
        __threadfence();
        last = atomicAdd(p.counters + f, 1u) == (unsigned)p.n_tiles - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();

    // the last CTA of filter f combines the tile records
    const float4* rec = p.records + (int64_t)f * p.n_tiles;
    float mm = -INFINITY;
    for (int r = tid; r < p.n_tiles; r += kLgThreads) mm = fmaxf(mm, __ldcg(rec + r).x);
    const float Mf = block_max(mm, ra);
    float S = 0.0f, S2 = 0.0f;
    if (Mf != -INFINITY) {
        for (int r = tid; r < p.n_tiles; r += kLgThreads) {
            const float4 q = __ldcg(rec + r);
            if (q.x == -INFINITY) continue;
            const float sc = expf(q.x - Mf);
            S += q.y * sc;
            S2 += q.z * sc * sc;
        }
    }
    block_sum2(S, S2, ra, rb);
    if (tid == 0) {
        if (Mf == -INFINITY) {
            set_status(p.status, ST_DOMAIN);
        } else {
            const double L = (double)Mf + log((double)S);
            const double L_prev = rf ? p.log_P : p.log_sum[f];
            p.loglik[f] += L - L_prev;
            p.log_sum[f] = L;
            const float e = (S * S) / S2;
            p.ess[f] = e;
            p.resample[f] = (double)e < p.threshold * (double)p.P ? 1 : 0;
        }
        p.counters[f] = 0u;  // ready for the next launch
    }
}

}  // namespace

int lg_tile() { return kLgThreads * kLgPerThread; }

cudaError_t launch_lg_init(const LgParams& p, int num_sms, cudaStream_t s) {
    const int64_t n = (int64_t)p.F * p.P;
    int64_t blocks = (n + kLgThreads - 1) / kLgThreads;
    const int64_t cap = (int64_t)num_sms * 4;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_lg_init<<<(unsigned)blocks, kLgThreads, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_lg_step(const LgParams& p, cudaStream_t s) {
    const unsigned blocks = (unsigned)((int64_t)p.F * p.n_tiles);
    switch (p.D) {
    case 4: k_lg_step<1><<<blocks, kLgThreads, 0, s>>>(p); break;
    case 8: k_lg_step<2><<<blocks, kLgThreads, 0, s>>>(p); break;
    case 16: k_lg_step<4><<<blocks, kLgThreads, 0, s>>>(p); break;
    default: k_lg_step<0><<<blocks, kLgThreads, 0, s>>>(p); break;
    }
    return cudaGetLastError();
}

}  // namespace pf
