// Metropolis resampler (Figure 1d, Section 2).
//
// Thread i runs chain i: k = i, then B steps, each proposing j uniformly over
// all P indices and moving to it when lw_j >= lw_k or when u < exp(lw_j - lw_k).
// No sum of weights is formed, so there is no collective step and one launch
// suffices.  Each Philox-4x32-10 call supplies the (proposal, uniform) pairs of
// two consecutive steps.
//
// When the P weights fit shared memory, each CTA stages them once as
// w_i = exp(lw_i - m) (m the largest log-weight, the subtraction error-free)
// and a step accepts when u w_k < w_j: one product instead of an exponential
// per step.  Each w carries at most 2.5 ulp of error (expf's 2 ulp and one
// rounding), so the decision can differ from the exact rule only where u lies
// within 7e-7 r of r = exp(lw_j - lw_k).  A state whose weight is below 2^-100
// (zero, or too small for the product to stay a normal float) decides in log
// space from the global log-weights instead.  Larger P reads the log-weights
// through L2 (ld.global.nc), where the 4 MiB of P = 2^20 stays resident.
#include "pf_device.cuh"

namespace pf {

constexpr int kMetroThreads = 256;
constexpr int kMetroSmemFloats = 48 * 1024;  // 192 KiB staging limit

// Accept a move from k to j (log-weights lk, lj) with uniform u.
__device__ __forceinline__ bool metropolis_accept(float lj, float lk, float u) {
    if (lj >= lk) return true;  // also covers lk = -inf
    float s, e;
    two_sum(lj, -lk, s, e);
    const float x = expf(s);
    const float r = x > 0.f ? __fmaf_rn(x, e, x) : 0.f;
    return u < r;
}

// B steps of chain i from state (k, lk).  The proposals do not depend on the
// chain's state, so each group of kAhead steps draws its proposals first and
// issues all their log-weight loads before resolving the steps in order.
constexpr int kAhead = 4;

template <int ROUNDS>
__device__ __forceinline__ void run_chain(const float* __restrict__ lw, uint32_t Pu, uint32_t i, int steps,
                                          uint32_t filter, uint32_t key0, uint32_t key1, uint32_t& k, float& lk) {
    for (int b0 = 0; b0 < steps; b0 += kAhead) {
        uint32_t jj[kAhead];
        float uu[kAhead], ll[kAhead];
#pragma unroll
        for (int q = 0; q < kAhead / 2; ++q) {
            const u32x4 r = philox<ROUNDS>(i, (uint32_t)((b0 >> 1) + q), filter, TAG_METRO, key0, key1);
            jj[2 * q] = draw_index(r.x, Pu);
            uu[2 * q] = u23f(r.y);
            jj[2 * q + 1] = draw_index(r.z, Pu);
            uu[2 * q + 1] = u23f(r.w);
        }
#pragma unroll
        for (int s = 0; s < kAhead; ++s) ll[s] = __ldg(lw + jj[s]);
#pragma unroll
        for (int s = 0; s < kAhead; ++s) {
            if (b0 + s < steps && metropolis_accept(ll[s], lk, uu[s])) {
                k = jj[s];
                lk = ll[s];
            }
        }
    }
}

// B steps of chain i from state k over staged weights w (shared memory).
constexpr float kWeightFloor = 0x1p-100f;

template <int ROUNDS>
__device__ __forceinline__ void run_chain_w(const float* __restrict__ lw, const float* w, uint32_t Pu, uint32_t i,
                                            int steps, uint32_t filter, uint32_t key0, uint32_t key1, uint32_t& k) {
    float wk = w[k];
    for (int b0 = 0; b0 < steps; b0 += kAhead) {
        uint32_t jj[kAhead];
        float uu[kAhead], ww[kAhead];
#pragma unroll
        for (int q = 0; q < kAhead / 2; ++q) {
            const u32x4 r = philox<ROUNDS>(i, (uint32_t)((b0 >> 1) + q), filter, TAG_METRO, key0, key1);
            jj[2 * q] = draw_index(r.x, Pu);
            uu[2 * q] = u23f(r.y);
            jj[2 * q + 1] = draw_index(r.z, Pu);
            uu[2 * q + 1] = u23f(r.w);
        }
#pragma unroll
        for (int s = 0; s < kAhead; ++s) ww[s] = w[jj[s]];
#pragma unroll
        for (int s = 0; s < kAhead; ++s) {
            if (b0 + s < steps) {
                const bool acc = wk >= kWeightFloor ? __fmul_rn(uu[s], wk) < ww[s]
                                                    : metropolis_accept(__ldg(lw + jj[s]), __ldg(lw + k), uu[s]);
                if (acc) {
                    k = jj[s];
                    wk = ww[s];
                }
            }
        }
    }
}

// Block-wide: copy lw[0..n) to w[] as weights exp(lw - m), m = max lw (0 when
// every weight is zero); records PF_ERR_DOMAIN for a NaN or +inf log-weight.
template <int THREADS>
__device__ void stage_weights(const float* __restrict__ lw, int64_t n, float* w, float* red, uint32_t* ctl) {
    const int tid = threadIdx.x;
    float m = -INFINITY;
    int bad = 0;
    if ((((uintptr_t)lw) & 15u) == 0) {
        const int64_t n4 = n >> 2;
        for (int64_t q = tid; q < n4; q += THREADS) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(lw) + q);
            reinterpret_cast<float4*>(w)[q] = v;
            m = fmaxf(fmaxf(m, fmaxf(v.x, v.y)), fmaxf(v.z, v.w));
            bad |= !(v.x <= 3.402823466e38f) | !(v.y <= 3.402823466e38f) | !(v.z <= 3.402823466e38f) |
                   !(v.w <= 3.402823466e38f);
        }
        for (int64_t q = 4 * n4 + tid; q < n; q += THREADS) {
            const float x = __ldg(lw + q);
            w[q] = x;
            m = fmaxf(m, x);
            bad |= !(x <= 3.402823466e38f);
        }
    } else {
        for (int64_t q = tid; q < n; q += THREADS) {
            const float x = __ldg(lw + q);
            w[q] = x;
            m = fmaxf(m, x);
            bad |= !(x <= 3.402823466e38f);
        }
    }
    m = warp_max(m);
    if ((tid & 31) == 0) red[tid >> 5] = m;
    bad = __syncthreads_or(bad);
    if (bad && tid == 0) set_status(ctl + CTL_STATUS, ST_DOMAIN);
    float mt = red[0];
#pragma unroll
    for (int q = 1; q < THREADS / 32; ++q) mt = fmaxf(mt, red[q]);
    const fpair R = {mt > -INFINITY ? mt : 0.f, 0.f};
    for (int64_t q = tid; q < n; q += THREADS) w[q] = weight_rel(w[q], R);
    __syncthreads();
}

// Block-wide: the largest normalised weight w_max = max_i w_i / sum_i w_i of
// lw[0..n) (Section 2, Eq. 5's w_max), from the staged weights w (STAGED: w_i =
// exp(lw_i - m), the largest is 1) or from the log-weights in global memory (one
// pass of running (max, sum) pairs, rescaled as the maximum grows).  Returns
// 0 when every weight is zero.  red: THREADS/32 floats of shared memory.
template <int THREADS, bool STAGED>
__device__ float largest_weight(const float* __restrict__ lw, const float* w, int64_t n, float* red) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float m = -INFINITY, sum = 0.f, c = 0.f;
    for (int64_t q = tid; q < n; q += THREADS) {
        if (STAGED) {
            const float y = __fsub_rn(w[q], c);  // compensated sum of the staged weights (max 1)
            const float t = __fadd_rn(sum, y);
            c = __fsub_rn(__fsub_rn(t, sum), y);
            sum = t;
        } else {
            const float x = __ldg(lw + q);
            if (x > m) {
                sum = (m > -INFINITY ? sum * expf(m - x) : 0.f) + 1.f;
                m = x;
            } else if (x > -INFINITY) {
                sum += expf(x - m);
            }
        }
    }
    if (STAGED) {
        sum = __fsub_rn(sum, c);
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) red[warp] = sum;
        __syncthreads();
        float tot = 0.f;
        for (int q = 0; q < THREADS / 32; ++q) tot += red[q];
        __syncthreads();  // red is reused
        return tot > 0.f ? 1.f / tot : 0.f;
    }
    // combine (max, sum) pairs: first the maximum, then every sum rescaled to it
    const float mw = warp_max(m);
    if (lane == 0) red[warp] = mw;
    __syncthreads();
    float M = red[0];
    for (int q = 1; q < THREADS / 32; ++q) M = fmaxf(M, red[q]);
    __syncthreads();
    float s2 = m > -INFINITY ? sum * expf(m - M) : 0.f;
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (lane == 0) red[warp] = s2;
    __syncthreads();
    float tot = 0.f;
    for (int q = 0; q < THREADS / 32; ++q) tot += red[q];
    __syncthreads();
    return (M > -INFINITY && tot > 0.f) ? 1.f / tot : 0.f;
}

// Eq. 5 (Section 2) on the device, in double precision, as pf_metropolis_B
// computes it on the host: the smallest B with lambda^B <= eps (alpha + beta) /
// max(alpha, beta), beta = 1/P, alpha = (1 - w_max)/(P w_max), lambda = 1 -
// alpha - beta; capped at cap (also for w_max = 0).
__device__ uint32_t bound_B(int64_t P, double w_max, double eps, uint32_t cap) {
    if (!(w_max > 0.0)) return cap;
    if (w_max > 1.0) w_max = 1.0;
    const double beta = 1.0 / (double)P;
    const double alpha = (1.0 - w_max) / ((double)P * w_max);
    const double lambda = 1.0 - alpha - beta;
    const double target = eps * (alpha + beta) / (alpha > beta ? alpha : beta);
    if (target >= 1.0) return 0;
    if (lambda <= 0.0) return 1;
    double b = ceil(log(target) / log(lambda));
    if (b >= 1.0 && pow(lambda, b - 1.0) <= target) b -= 1.0;
    if (!(b >= 0.0)) return cap;
    return b < (double)cap ? (uint32_t)b : cap;
}

template <bool STAGED, int ROUNDS>
__global__ void __launch_bounds__(kMetroThreads) k_metropolis(const float* __restrict__ lw, int64_t P, int B,
                                                              const uint32_t* __restrict__ B_dev, uint32_t key0,
                                                              uint32_t key1, uint32_t filter,
                                                              int32_t* __restrict__ anc, uint32_t* ctl) {
    extern __shared__ float wsm[];
    __shared__ float red[kMetroThreads / 32];
    if (STAGED) stage_weights<kMetroThreads>(lw, P, wsm, red, ctl);  // every CTA: the whole vector
    const int steps = B_dev ? (int)__ldg(B_dev) : B;
    const uint32_t Pu = (uint32_t)P;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t k = (uint32_t)i;
        if (STAGED) {
            run_chain_w<ROUNDS>(lw, wsm, Pu, (uint32_t)i, steps, filter, key0, key1, k);
        } else {
            float lk = __ldg(lw + i);
            if (!(lk <= 3.402823466e38f)) set_status(ctl + CTL_STATUS, ST_DOMAIN);  // NaN or +inf
            run_chain<ROUNDS>(lw, Pu, (uint32_t)i, steps, filter, key0, key1, k, lk);
        }
        anc[i] = (int32_t)k;
    }
}

// Once per device: allow the staged variant its full shared-memory copy.
cudaError_t prepare_metropolis() {
    cudaError_t e = cudaFuncSetAttribute(k_metropolis<true, 10>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kMetroSmemFloats * (int)sizeof(float));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_metropolis<true, 7>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kMetroSmemFloats * (int)sizeof(float));
    return e;
}

template <int ROUNDS>
static cudaError_t launch_metropolis_r(const float* lw, int64_t P, int B, const uint32_t* B_dev, uint32_t key0,
                                       uint32_t key1, uint32_t filter, int32_t* anc, uint32_t* ctl, int num_sms,
                                       cudaStream_t s) {
    const bool staged = P <= kMetroSmemFloats;
    const int64_t blocks_needed = (P + kMetroThreads - 1) / kMetroThreads;
    if (staged) {
        // every CTA stages the full vector, so keep the grid to what runs at once
        const size_t smem = (size_t)P * sizeof(float);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_metropolis<true, ROUNDS>, kMetroThreads, smem);
        if (per_sm < 1) per_sm = 1;
        const int64_t grid = blocks_needed < (int64_t)num_sms * per_sm ? blocks_needed : (int64_t)num_sms * per_sm;
        k_metropolis<true, ROUNDS><<<(unsigned)grid, kMetroThreads, smem, s>>>(lw, P, B, B_dev, key0, key1, filter,
                                                                               anc, ctl);
    } else {
        const int64_t cap = (int64_t)num_sms * 64;
        const int64_t grid = blocks_needed < cap ? blocks_needed : cap;
        k_metropolis<false, ROUNDS><<<(unsigned)grid, kMetroThreads, 0, s>>>(lw, P, B, B_dev, key0, key1, filter,
                                                                             anc, ctl);
    }
    return cudaGetLastError();
}

cudaError_t launch_metropolis(const float* lw, int64_t P, int B, const uint32_t* B_dev, uint32_t key0, uint32_t key1,
                              uint32_t filter, int32_t* anc, uint32_t* ctl, int num_sms, cudaStream_t s, int rounds) {
    if (rounds == 7) return launch_metropolis_r<7>(lw, P, B, B_dev, key0, key1, filter, anc, ctl, num_sms, s);
    return launch_metropolis_r<10>(lw, P, B, B_dev, key0, key1, filter, anc, ctl, num_sms, s);
}

// ---------------------------------------------------------------------------
// Batched: each CTA takes whole filters from a ticket counter, copies the
// filter's log-weights to shared memory when they fit, and runs its chains
// (filter-local indices, Philox filter id f, key seeds[f]).  One 1024-thread
// CTA per SM stages up to 56 Ki log-weights (224 KiB): a staged chain step is
// bound by its Philox and acceptance arithmetic, an unstaged one by random
// L2 reads, which sustain fewer steps per second.
// ---------------------------------------------------------------------------
constexpr int kMetroBThreads = 1024;
constexpr int kMetroBStage = 56 * 1024;  // floats staged per CTA (224 KiB)
constexpr uint32_t kBatchedBCap = 1u << 24;  // largest step count chosen for B < 0

// Chain blocks of a filter shared by several CTAs: a filter whose chains
// number more than one block and whose work P_f B_f reaches kHeavyWork steps
// is put on a list after its owner (the CTA that took its ticket) has
// published its step count; CTAs that find the ticket queue empty join the
// listed filters.  Blocks of kMetroBThreads chains are claimed through a 64-bit
// word per filter, (launch epoch, claims): a word from an earlier launch is
// replaced by the first claimer, so no pass clears the words between launches.
// Every chain depends only on (f, i, B_f), so which CTA runs it does not
// change the result.
constexpr long long kHeavyWork = 1LL << 22;

// Claims the next block of the filter's word (thread 0 only).
__device__ __forceinline__ uint32_t claim_block(unsigned long long* w, uint32_t epoch) {
    for (;;) {
        const unsigned long long old = (unsigned long long)ld_relaxed_u64(reinterpret_cast<const uint64_t*>(w));
        if ((uint32_t)(old >> 32) != epoch) {
            if (atomicCAS(w, old, ((unsigned long long)epoch << 32) | 1ull) == old) return 0u;
            continue;
        }
        return (uint32_t)atomicAdd(w, 1ull);
    }
}

// The chains of blocks claimed from filter f (block-wide; the weights are staged).
template <int ROUNDS>
__device__ __forceinline__ void run_claimed_blocks(const BatchParams& bp, const float* lw, const float* wsm, bool staged,
                                                   int64_t Pf, int64_t off0, int steps, int f, uint32_t epoch,
                                                   uint32_t key0, uint32_t key1, int* blk_sm) {
    const int tid = threadIdx.x;
    const uint32_t Pu = (uint32_t)Pf;
    const int64_t nblk = (Pf + kMetroBThreads - 1) / kMetroBThreads;
    for (;;) {
        if (tid == 0) *blk_sm = (int)claim_block(bp.metro + 2 * (int64_t)f, epoch);
        __syncthreads();
        const int64_t blk = *blk_sm;
        __syncthreads();
        if (blk >= nblk) break;
        const int64_t i = blk * kMetroBThreads + tid;
        if (i < Pf) {
            uint32_t k = (uint32_t)i;
            if (staged) {
                run_chain_w<ROUNDS>(lw, wsm, Pu, (uint32_t)i, steps, (uint32_t)f, key0, key1, k);
            } else {
                float lk = __ldg(lw + i);
                if (!(lk <= 3.402823466e38f)) set_status(bp.ctl + CTL_STATUS, ST_DOMAIN);
                run_chain<ROUNDS>(lw, Pu, (uint32_t)i, steps, (uint32_t)f, key0, key1, k, lk);
            }
            bp.anc[off0 + i] = (int32_t)k;
        }
    }
}

template <int ROUNDS>
__global__ void __launch_bounds__(kMetroBThreads) k_batched_metropolis(BatchParams bp) {
    extern __shared__ float wsm[];
    __shared__ int f_sm, f_B, blk_sm;
    __shared__ float red[kMetroBThreads / 32];
    const int tid = threadIdx.x;
    const int n_items = (int)ld_relaxed_u32(bp.ctl + CTL_ITEMS);
    const uint32_t epoch = ld_relaxed_u32(bp.ctl + CTL_METRO_EPOCH);
    for (;;) {
        if (tid == 0) f_sm = (int)atomicAdd(bp.ctl + CTL_QUEUE, 1u);
        __syncthreads();
        const int ticket = f_sm;
        __syncthreads();
        if (ticket >= n_items) break;
        const int f = bp.items[ticket] >> 5;
        const int64_t off0 = bp.offsets[f], off1 = bp.offsets[f + 1];
        const int64_t Pf = off1 - off0;
        if (Pf <= 0 || Pf > 0x7fffffffLL) {
            if (Pf != 0 && tid == 0) set_status(bp.ctl + CTL_STATUS, ST_INVALID);
            continue;
        }
        const float* lw = bp.lw + off0;
        const bool staged = Pf <= kMetroBStage;
        if (bp.trace) {
            trace_stamp(bp.trace, bp.trace_cap, ticket, 0);
            trace_put(bp.trace, bp.trace_cap, ticket, 5, blockIdx.x);
            trace_put(bp.trace, bp.trace_cap, ticket, 6, (uint64_t)f);
            trace_put(bp.trace, bp.trace_cap, ticket, 7, (uint64_t)(bp.items[ticket] & 31));
        }
        if (staged) stage_weights<kMetroBThreads>(lw, Pf, wsm, red, bp.ctl);
        for (int w = 1; w <= 2; ++w) trace_stamp(bp.trace, bp.trace_cap, ticket, w);
        // B < 0: this filter's own step count from Eq. 5 and its largest normalised weight
        int steps = bp.B;
        if (bp.B < 0) {
            const float wmax = staged ? largest_weight<kMetroBThreads, true>(lw, wsm, Pf, red)
                                      : largest_weight<kMetroBThreads, false>(lw, wsm, Pf, red);
            if (tid == 0) {
                f_B = (int)bound_B(Pf, (double)wmax, bp.eps, kBatchedBCap);
                if (bp.B_out) bp.B_out[f] = f_B;
            }
            __syncthreads();
            steps = f_B;
        }
        trace_stamp(bp.trace, bp.trace_cap, ticket, 3);
        const uint64_t seed = bp.seeds[f];
        const uint32_t key0 = (uint32_t)(seed & 0xffffffffu), key1 = (uint32_t)(seed >> 32);
        const uint32_t Pu = (uint32_t)Pf;
        const bool heavy = bp.metro != nullptr && Pf > kMetroBThreads && Pf * (long long)max(steps, 1) >= kHeavyWork;
        if (heavy) {
            // publish the step count, then list the filter for CTAs with nothing left to take
            if (tid == 0) {
                st_release_u64(reinterpret_cast<uint64_t*>(bp.metro + 2 * (int64_t)f + 1),
                               ((uint64_t)epoch << 32) | (uint32_t)steps);
                const uint32_t h = atomicAdd(bp.ctl + CTL_HEAVY, 1u);
                if (h < (uint32_t)kMaxHeavy) {  // the list lives after the items (scratch the plan cleared)
                    int32_t* list = const_cast<int32_t*>(bp.items) + bp.F;
                    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(list + h), "r"(f + 1) : "memory");
                }
            }
            run_claimed_blocks<ROUNDS>(bp, lw, wsm, staged, Pf, off0, steps, f, epoch, key0, key1, &blk_sm);
        } else {
            for (int64_t i = tid; i < Pf; i += kMetroBThreads) {
                uint32_t k = (uint32_t)i;
                if (staged) {
                    run_chain_w<ROUNDS>(lw, wsm, Pu, (uint32_t)i, steps, (uint32_t)f, key0, key1, k);
                } else {
                    float lk = __ldg(lw + i);
                    if (!(lk <= 3.402823466e38f)) set_status(bp.ctl + CTL_STATUS, ST_DOMAIN);
                    run_chain<ROUNDS>(lw, Pu, (uint32_t)i, steps, (uint32_t)f, key0, key1, k, lk);
                }
                bp.anc[off0 + i] = (int32_t)k;
            }
        }
        __syncthreads();  // the staging buffer is reused by the next filter
        trace_stamp(bp.trace, bp.trace_cap, ticket, 4);
    }
    // the queue is empty: join the listed filters that still have unclaimed blocks
    if (bp.metro != nullptr) {
        const uint64_t t_start = global_ns();
        for (int h = 0;; ++h) {
            if (tid == 0) {
                const int H = (int)min(ld_acquire_u32(bp.ctl + CTL_HEAVY), (uint32_t)kMaxHeavy);
                int f = -1;
                if (h < H) {
                    // the owner lists the filter right after counting it: wait (bounded) for the entry
                    for (uint32_t it = 0;; ++it) {
                        const uint32_t e = ld_acquire_u32(reinterpret_cast<const uint32_t*>(bp.items + bp.F + h));
                        if (e != 0u) {
                            f = (int)e - 1;
                            break;
                        }
                        if ((it & 63u) == 63u && global_ns() - t_start > bp.wait_ns) break;
                    }
                }
                f_sm = h < H ? f : -2;
                if (f >= 0) {
                    const uint64_t pw = ld_acquire_u64(reinterpret_cast<const uint64_t*>(bp.metro + 2 * (int64_t)f + 1));
                    const uint64_t cw = ld_relaxed_u64(reinterpret_cast<const uint64_t*>(bp.metro + 2 * (int64_t)f));
                    const int64_t nblk = (bp.offsets[f + 1] - bp.offsets[f] + kMetroBThreads - 1) / kMetroBThreads;
                    const bool done = (uint32_t)(cw >> 32) == epoch && (int64_t)(uint32_t)cw >= nblk;
                    if ((uint32_t)(pw >> 32) != epoch || done) f_sm = -1;  // nothing to join here
                    else f_B = (int)(uint32_t)pw;
                }
            }
            __syncthreads();
            const int f = f_sm;
            const int steps = f_B;
            __syncthreads();
            if (f == -2) break;  // past the end of the list
            if (f < 0) continue;
            const int64_t off0 = bp.offsets[f];
            const int64_t Pf = bp.offsets[f + 1] - off0;
            const float* lw = bp.lw + off0;
            const bool staged = Pf <= kMetroBStage;
            if (staged) stage_weights<kMetroBThreads>(lw, Pf, wsm, red, bp.ctl);
            const uint64_t seed = bp.seeds[f];
            run_claimed_blocks<ROUNDS>(bp, lw, wsm, staged, Pf, off0, steps, f, epoch, (uint32_t)(seed & 0xffffffffu),
                               (uint32_t)(seed >> 32), &blk_sm);
            __syncthreads();  // the staging buffer is reused by the next listed filter
        }
    }
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(bp.ctl + CTL_QUEUE_DONE, 1u) == gridDim.x - 1) {
            atomicExch(bp.ctl + CTL_QUEUE, 0u);
            atomicExch(bp.ctl + CTL_QUEUE_DONE, 0u);
        }
    }
}

int batched_metropolis_blocks_per_sm() {
    const size_t smem = kMetroBStage * sizeof(float);
    int nb10 = 0, nb7 = 0;
    if (cudaFuncSetAttribute(k_batched_metropolis<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_batched_metropolis<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb10, k_batched_metropolis<10>, kMetroBThreads, smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb7, k_batched_metropolis<7>, kMetroBThreads, smem) !=
            cudaSuccess)
        return 0;
    return nb10 < nb7 ? nb10 : nb7;
}

cudaError_t launch_batched_metropolis(const BatchParams& bp, int grid, cudaStream_t s) {
    if (bp.rounds == 7)
        k_batched_metropolis<7><<<grid, kMetroBThreads, kMetroBStage * sizeof(float), s>>>(bp);
    else
        k_batched_metropolis<10><<<grid, kMetroBThreads, kMetroBStage * sizeof(float), s>>>(bp);
    return cudaGetLastError();
}

}  // namespace pf
