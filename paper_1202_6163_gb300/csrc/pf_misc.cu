// Ancestor gather (Section 1, step 4) and the weight reduction behind the
// effective sample size (Section 3) and the device-side choice of the
// Metropolis step count (Section 2, Eqs. 1-5).
#include <climits>

#include "pf_fixed.cuh"

namespace pf {

// ---------------------------------------------------------------------------
// Gather: dst row j <- src row anc[j].  One thread moves one VT-sized chunk;
// each thread handles kUnroll chunks spread a grid apart, issuing all loads
// before the stores so that several random row reads are in flight.
// ---------------------------------------------------------------------------
constexpr int kGatherThreads = 256;
constexpr int kUnroll = 4;

template <typename VT, bool POW2>
__global__ void __launch_bounds__(kGatherThreads) k_gather(const VT* __restrict__ src, int64_t P_src, int64_t vecs,
                                                           int vshift, const int32_t* __restrict__ anc,
                                                           int64_t P_dst, VT* __restrict__ dst, uint32_t* ctl) {
    const int64_t total = P_dst * vecs;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; base < total; base += stride * kUnroll) {
        VT v[kUnroll];
        int64_t idx[kUnroll];
        bool ok[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            idx[u] = base + u * stride;
            ok[u] = false;
            if (idx[u] < total) {
                const int64_t j = POW2 ? (idx[u] >> vshift) : idx[u] / vecs;
                const int64_t c = POW2 ? (idx[u] & (vecs - 1)) : idx[u] - j * vecs;
                const int32_t a = __ldg(anc + j);
                if (a >= 0 && a < P_src) {
                    v[u] = __ldg(src + (int64_t)a * vecs + c);
                    ok[u] = true;
                } else if (c == 0) {
                    set_status(ctl + CTL_STATUS, ST_INVALID);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (ok[u]) __stcs(dst + idx[u], v[u]);
    }
}

template <typename VT>
static cudaError_t gather_vt(const void* src, int64_t P_src, int64_t row_bytes, const int32_t* anc, int64_t P_dst,
                             void* dst, uint32_t* ctl, int num_sms, cudaStream_t s) {
    const int64_t vecs = row_bytes / (int64_t)sizeof(VT);
    const int64_t total = P_dst * vecs;
    int64_t blocks = (total + (int64_t)kGatherThreads * kUnroll - 1) / ((int64_t)kGatherThreads * kUnroll);
    const int64_t cap = (int64_t)num_sms * 8;  // one resident wave (8 CTAs of 256 threads per SM)
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    const bool pow2 = (vecs & (vecs - 1)) == 0;
    int vshift = 0;
    while (pow2 && (1LL << vshift) < vecs) ++vshift;
    if (pow2)
        k_gather<VT, true><<<(unsigned)blocks, kGatherThreads, 0, s>>>(
            (const VT*)src, P_src, vecs, vshift, anc, P_dst, (VT*)dst, ctl);
    else
        k_gather<VT, false><<<(unsigned)blocks, kGatherThreads, 0, s>>>(
            (const VT*)src, P_src, vecs, vshift, anc, P_dst, (VT*)dst, ctl);
    return cudaGetLastError();
}

cudaError_t launch_gather(const void* src, int64_t P_src, int64_t row_bytes, const int32_t* anc, int64_t P_dst,
                          void* dst, uint32_t* ctl, int num_sms, cudaStream_t s) {
    const uintptr_t a = (uintptr_t)src | (uintptr_t)dst | (uintptr_t)row_bytes;
    if ((a & 15) == 0) return gather_vt<uint4>(src, P_src, row_bytes, anc, P_dst, dst, ctl, num_sms, s);
    if ((a & 7) == 0) return gather_vt<uint2>(src, P_src, row_bytes, anc, P_dst, dst, ctl, num_sms, s);
    return gather_vt<uint32_t>(src, P_src, row_bytes, anc, P_dst, dst, ctl, num_sms, s);
}

// ---------------------------------------------------------------------------
// Weight reduction: per tile (k_t, sum w, sum w^2, max lw) with weights taken
// relative to 2^k_t; the last CTA to finish combines the tiles in index order
// in FP64 and writes ESS = (sum w)^2 / sum w^2, log sum exp(lw), and, when
// asked, the Metropolis step bound of Eq. 5 for the actual w_max.
// ---------------------------------------------------------------------------
constexpr int kRedThreads = 256;
constexpr int kRedPerThread = 16;
constexpr int kRedTile = kRedThreads * kRedPerThread;

struct RedRecord {  // 32 bytes, read back as two 16-byte halves
    int32_t k;
    float m;
    float s_hi, s_lo, q_hi, q_lo;
    uint32_t bad, pad;
};
static_assert(sizeof(RedRecord) == 32, "record layout");

__device__ __forceinline__ void kahan_add(float& s, float& c, float w) {
    const float y = __fsub_rn(w, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

__device__ __forceinline__ i128 shfl_xor_i128(i128 v, int o) {
    const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
    const unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    const unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    return (i128)(((unsigned __int128)h2 << 64) | l2);
}

__global__ void __launch_bounds__(kRedThreads) k_reduce(const float* __restrict__ lw, int64_t P, RedRecord* rec,
                                                        uint32_t* ctl, float* ess_out, double* log_sum_out,
                                                        uint32_t* B_out, double eps, uint32_t B_cap) {
    __shared__ float rm[kRedThreads / 32];
    __shared__ fpair rs[kRedThreads / 32], rq[kRedThreads / 32];
    __shared__ int rk[kRedThreads / 32];
    __shared__ i128 rS[kRedThreads / 32], rQ[kRedThreads / 32];
    __shared__ int last;
    const float eps_f = (float)eps;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t t0 = (int64_t)blockIdx.x * kRedTile;
    const int n = (int)min((int64_t)kRedTile, P - t0);
    const float* base = lw + t0;

    float x[kRedPerThread];
#pragma unroll
    for (int q = 0; q < kRedPerThread / 4; ++q) {
        // coalesced: thread tid reads vector q*kRedThreads + tid
        const int e = 4 * (q * kRedThreads + tid);
        if (e + 3 < n) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(base + e));
            x[4 * q] = v.x;
            x[4 * q + 1] = v.y;
            x[4 * q + 2] = v.z;
            x[4 * q + 3] = v.w;
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r) x[4 * q + r] = (e + r < n) ? __ldg(base + e + r) : -INFINITY;
        }
    }
    float m = -INFINITY;
    int bad = 0;
#pragma unroll
    for (int i = 0; i < kRedPerThread; ++i) {
        bad |= !(x[i] <= 3.402823466e38f);
        m = fmaxf(m, x[i]);
    }
    m = warp_max(m);
    if (lane == 0) rm[warp] = m;
    bad = __syncthreads_or(bad);
    float mt = rm[0];
#pragma unroll
    for (int w = 1; w < kRedThreads / 32; ++w) mt = fmaxf(mt, rm[w]);
    const int k = tile_exponent(mt);
    const fpair R = tile_reference(k);
    float s = 0.f, sc = 0.f, q = 0.f, qc = 0.f;
#pragma unroll
    for (int i = 0; i < kRedPerThread; ++i) {
        const float w = weight_rel(x[i], R);
        kahan_add(s, sc, w);
        kahan_add(q, qc, w * w);
    }
    fpair ps = {s, -sc}, pq = {q, -qc};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ps = pair_add(ps, {__shfl_xor_sync(0xffffffffu, ps.hi, o), __shfl_xor_sync(0xffffffffu, ps.lo, o)});
        pq = pair_add(pq, {__shfl_xor_sync(0xffffffffu, pq.hi, o), __shfl_xor_sync(0xffffffffu, pq.lo, o)});
    }
    if (lane == 0) {
        rs[warp] = ps;
        rq[warp] = pq;
    }
    __syncthreads();
    if (tid == 0) {
        fpair S = rs[0], Q = rq[0];
        for (int w = 1; w < kRedThreads / 32; ++w) {
            S = pair_add(S, rs[w]);
            Q = pair_add(Q, rq[w]);
        }
        RedRecord r;
        r.k = k;
        r.m = mt;
        r.s_hi = S.hi;
        r.s_lo = S.lo;
        r.q_hi = Q.hi;
        r.q_lo = Q.lo;
        r.bad = bad;
        r.pad = 0;
        rec[blockIdx.x] = r;
        __threadfence();
        const uint32_t prev = atomicAdd(ctl + CTL_ESS_COUNT, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // last CTA: combine all tiles (exact fixed-point sums, all threads)
    const int T = gridDim.x;
    int kmax = INT_MIN, anybad = 0;
    float mmax = -INFINITY;
    // each record as two 16-byte loads; the first one a thread reads stays in
    // registers for the second pass (the only one when T <= kRedThreads)
    const uint32_t* rw = reinterpret_cast<const uint32_t*>(rec);
    uint4 r0 = make_uint4(0, 0, 0, 0), r1 = make_uint4(0, 0, 0, 0);
    for (int t = tid; t < T; t += kRedThreads) {
        const uint4 a = ld_cg_v4_u32(rw + 8 * t), b = ld_cg_v4_u32(rw + 8 * t + 4);
        if (t == tid) {
            r0 = a;
            r1 = b;
        }
        anybad |= (int)b.z;
        if (__uint_as_float(a.z) > 0.f) kmax = max(kmax, (int)a.x);
        mmax = fmaxf(mmax, __uint_as_float(a.y));
    }
    kmax = warp_max_i(kmax);
    mmax = warp_max(mmax);
    if (lane == 0) {
        rk[warp] = kmax;
        rm[warp] = mmax;
    }
    anybad = __syncthreads_or(anybad);
    int K = rk[0];
    float M = rm[0];
#pragma unroll
    for (int w = 1; w < kRedThreads / 32; ++w) {
        K = max(K, rk[w]);
        M = fmaxf(M, rm[w]);
    }
    if (anybad || K == INT_MIN) {
        if (tid == 0) {
            set_status(ctl + CTL_STATUS, ST_DOMAIN);
            if (ess_out) *ess_out = NAN;
            if (log_sum_out) *log_sum_out = NAN;
            if (B_out) *B_out = 0;
            ctl[CTL_ESS_COUNT] = 0;
        }
        return;
    }
    i128 S = 0, Q = 0;
    for (int t = tid; t < T; t += kRedThreads) {
        uint4 a = r0, b = r1;
        if (t != tid) {
            a = ld_cg_v4_u32(rw + 8 * t);
            b = ld_cg_v4_u32(rw + 8 * t + 4);
        }
        const int sh = (int)a.x - K;
        S += fixed_of(__uint_as_float(a.z), sh) + fixed_of(__uint_as_float(a.w), sh);
        Q += fixed_of(__uint_as_float(b.x), 2 * sh) + fixed_of(__uint_as_float(b.y), 2 * sh);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        S += shfl_xor_i128(S, o);
        Q += shfl_xor_i128(Q, o);
    }
    if (lane == 0) {
        rS[warp] = S;
        rQ[warp] = Q;
    }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < kRedThreads / 32; ++w) {
            S += rS[w];
            Q += rQ[w];
        }
        const fpair Sp = fixed_to_pair(S), Qp = fixed_to_pair(Q);
        // ESS = S^2 / Q in float (first order in the low parts)
        const float ratio = Sp.hi * (Sp.hi / Qp.hi);
        const float corr = 2.f * (Sp.lo / Sp.hi) - Qp.lo / Qp.hi;
        if (ess_out) *ess_out = __fmaf_rn(ratio, corr, ratio);
        // log sum exp(lw) = K ln 2 + log S
        const float logS = logf(Sp.hi) + Sp.lo / Sp.hi;
        const double log_sum = (double)K * kLn2 + (double)logS;
        if (log_sum_out) *log_sum_out = log_sum;
        if (B_out) {
            // Eq. 5 with the actual largest normalised weight
            const float ls = (float)((double)K * kLn2 - (double)M) + logS;  // log W - m
            const float w_max = fminf(1.f, expf(-ls));
            float b;
            if (!(w_max > 0.f)) {
                b = (float)B_cap;
            } else {
                const float beta = 1.f / (float)P;
                const float alpha = (1.f - w_max) / ((float)P * w_max);
                const float target = eps_f * (alpha + beta) / fmaxf(alpha, beta);
                if (target >= 1.f) b = 0.f;
                else b = ceilf(logf(target) / log1pf(-(alpha + beta)));
            }
            if (!(b >= 0.f)) b = (float)B_cap;
            *B_out = (uint32_t)fminf(b, (float)B_cap);
        }
        ctl[CTL_ESS_COUNT] = 0;  // ready for the next reduction on this stream
    }
}

// ---------------------------------------------------------------------------
// Diagnostic: the rate of random 4-byte reads from a buffer held in L2, the
// ceiling of the Metropolis resampler at P of a few million (its chains read
// one random log-weight per step).  Each thread makes `reads` independent
// reads at hashed indices, eight in flight.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t probe_hash(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__global__ void __launch_bounds__(256) k_probe_l2(const float* __restrict__ buf, uint32_t n, int reads, float* sink) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.f;
    for (int l = 0; l < reads; l += 8) {
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = __ldg(buf + __umulhi(probe_hash(t * 977u + (uint32_t)(l + q) * 131071u), n));
#pragma unroll
        for (int q = 0; q < 8; ++q) acc += v[q];
    }
    if (acc == -1.2345e38f) sink[0] = acc;  // keeps the loads; never true for finite data
}

cudaError_t probe_l2_random_reads(const float* buf, int64_t n, int reads, int num_sms, double* rate) {
    if (n < 1 || n > 0xffffffffLL || reads < 8) return cudaErrorInvalidValue;
    const int blocks = num_sms * 16;
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) return e;
    float* sink = const_cast<float*>(buf);
    k_probe_l2<<<blocks, 256>>>(buf, (uint32_t)n, reads, sink);  // warm L2
    cudaEventRecord(a);
    for (int r = 0; r < 5; ++r) k_probe_l2<<<blocks, 256>>>(buf, (uint32_t)n, reads, sink);
    cudaEventRecord(b);
    e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return e;
    *rate = 5.0 * blocks * 256.0 * (reads & ~7) / (ms * 1e-3);
    return cudaGetLastError();
}

// Diagnostic: the tile weights the scans use, out[i] = exp(lw[i] - k ln 2).
__global__ void k_tile_weights(const float* __restrict__ lw, int64_t n, int k, float* __restrict__ out) {
    const fpair R = tile_reference(k);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = weight_rel(lw[i], R);
}

cudaError_t launch_tile_weights(const float* lw, int64_t n, int k, float* out, cudaStream_t s) {
    const int64_t blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    k_tile_weights<<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, s>>>(lw, n, k, out);
    return cudaGetLastError();
}

int reduce_tiles(int64_t P) { return (int)((P + kRedTile - 1) / kRedTile); }
size_t reduce_record_bytes() { return sizeof(RedRecord); }

cudaError_t launch_reduce(const float* lw, int64_t P, void* rec, uint32_t* ctl, float* ess_out, double* log_sum_out,
                          uint32_t* B_out, double eps, uint32_t B_cap, cudaStream_t s) {
    k_reduce<<<reduce_tiles(P), kRedThreads, 0, s>>>(lw, P, (RedRecord*)rec, ctl, ess_out, log_sum_out, B_out, eps,
                                                     B_cap);
    return cudaGetLastError();
}

}  // namespace pf
