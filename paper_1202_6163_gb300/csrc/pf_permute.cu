// Offspring/ancestor conversion for in-place particle moves (Section 2: the
// stratified and systematic schemes give offspring counts, the multinomial
// and Metropolis ones ancestors; converting between the two is direct).
//
// pf_permute rewrites any ancestor vector a into one with the same offspring
// counts o_i in which every particle with offspring keeps one of them in its
// own slot (out[i] = i); the other o_i - 1 copies of each such i (in
// increasing i) fill the slots of the particles without offspring (in
// increasing slot order).  Then out[out[j]] = out[j], so the states can be
// moved in place: row j is overwritten only if particle j has no offspring,
// and every row read belongs to a particle that keeps its slot.
//
// Passes (all bandwidth-light): offspring counts (atomics); per-tile sums of
// the extra copies max(o_i - 1, 0) and of the empty slots [o_i == 0]; their
// exclusive scan; placement (survivors to their own slot, each survivor's run
// start marked in the extras list E, each empty slot listed in DS); a
// max-scan over E that fills the runs (survivor indices increase along E);
// and the fill out[DS[r]] = E[r].
#include <climits>

#include "pf_device.cuh"
#include "pf_internal.h"

namespace pf {
namespace {

constexpr int kPermThreads = 512;
constexpr int kPermPer = 8;
constexpr int kPermTile = kPermThreads * kPermPer;
constexpr int kPermWarps = kPermThreads / 32;
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(256) k_perm_count(const int32_t* __restrict__ anc, int64_t P,
                                                    int32_t* __restrict__ o, uint32_t* ctl) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < P; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = anc[j];
        if (a < 0 || a >= P) set_status(ctl + CTL_STATUS, ST_INVALID);
        else atomicAdd(o + a, 1);
    }
}

// Block exclusive scan of one int per thread (kPermThreads threads); *total gets the sum.
__device__ __forceinline__ int block_excl_scan(int x, int* red, int& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int h = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += h;
    }
    if (lane == 31) red[warp] = inc;
    __syncthreads();
    int base = 0;
    total = 0;
#pragma unroll
    for (int w = 0; w < kPermWarps; ++w) {
        const int v = red[w];
        base += w < warp ? v : 0;
        total += v;
    }
    __syncthreads();
    return base + inc - x;
}

__global__ void __launch_bounds__(kPermThreads) k_perm_tiles(const int32_t* __restrict__ o, int64_t P,
                                                             int32_t* __restrict__ t_extra, int32_t* __restrict__ t_dead) {
    __shared__ int red[kPermWarps];
    const int64_t i0 = (int64_t)blockIdx.x * kPermTile + (int64_t)threadIdx.x * kPermPer;
    int e = 0, d = 0;
#pragma unroll
    for (int k = 0; k < kPermPer; ++k) {
        if (i0 + k < P) {
            const int c = o[i0 + k];
            e += c > 1 ? c - 1 : 0;
            d += c == 0;
        }
    }
    int te, td;
    block_excl_scan(e, red, te);
    block_excl_scan(d, red, td);
    if (threadIdx.x == 0) {
        t_extra[blockIdx.x] = te;
        t_dead[blockIdx.x] = td;
    }
}

// One CTA: exclusive scans (sum) of two arrays of T ints, in place; or, with
// max_mode, an exclusive running maximum of one array (starting at -1).
__global__ void __launch_bounds__(kScanThreads) k_perm_scan(int32_t* a, int32_t* b, int T, int max_mode) {
    __shared__ int red[kScanThreads / 32];
    __shared__ int carry_a, carry_b;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        carry_a = max_mode ? -1 : 0;
        carry_b = 0;
    }
    __syncthreads();
    for (int base = 0; base < T; base += kScanThreads) {
        const int t = base + threadIdx.x;
        for (int which = 0; which < (max_mode ? 1 : 2); ++which) {
            int32_t* arr = which ? b : a;
            const int x = t < T ? arr[t] : (max_mode ? -1 : 0);
            int inc = x;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int h = __shfl_up_sync(0xffffffffu, inc, off);
                if (lane >= off) inc = max_mode ? max(inc, h) : inc + h;
            }
            if (lane == 31) red[warp] = inc;
            __syncthreads();
            int wb = max_mode ? -1 : 0, tot = max_mode ? -1 : 0;
            for (int w = 0; w < kScanThreads / 32; ++w) {
                const int v = red[w];
                if (w < warp) wb = max_mode ? max(wb, v) : wb + v;
                tot = max_mode ? max(tot, v) : tot + v;
            }
            const int c = which ? carry_b : carry_a;
            // exclusive value: carry (+) the block prefix before this thread
            int excl;
            if (max_mode) {
                const int prev = __shfl_up_sync(0xffffffffu, inc, 1);
                excl = max(c, max(wb, lane > 0 ? prev : -1));
            } else {
                excl = c + wb + inc - x;
            }
            __syncthreads();
            if (t < T) arr[t] = excl;
            if (threadIdx.x == 0) {
                if (which) carry_b = c + tot;
                else carry_a = max_mode ? max(c, tot) : c + tot;
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(kPermThreads) k_perm_place(const int32_t* __restrict__ o, int64_t P,
                                                             const int32_t* __restrict__ t_extra,
                                                             const int32_t* __restrict__ t_dead,
                                                             int32_t* __restrict__ out, int32_t* __restrict__ E,
                                                             int32_t* __restrict__ DS) {
    __shared__ int red[kPermWarps];
    const int64_t i0 = (int64_t)blockIdx.x * kPermTile + (int64_t)threadIdx.x * kPermPer;
    int c[kPermPer];
    int e = 0, d = 0;
#pragma unroll
    for (int k = 0; k < kPermPer; ++k) {
        c[k] = i0 + k < P ? o[i0 + k] : 1;  // past the end: neither extra nor empty
        e += c[k] > 1 ? c[k] - 1 : 0;
        d += c[k] == 0;
    }
    int te, td;
    int pe = t_extra[blockIdx.x] + block_excl_scan(e, red, te);
    int pd = t_dead[blockIdx.x] + block_excl_scan(d, red, td);
#pragma unroll
    for (int k = 0; k < kPermPer; ++k) {
        const int64_t i = i0 + k;
        if (i >= P) break;
        if (c[k] > 0) {
            out[i] = (int32_t)i;
            if (c[k] > 1) {
                E[pe] = (int32_t)i;  // start of i's run of extra copies
                pe += c[k] - 1;
            }
        } else {
            DS[pd++] = (int32_t)i;
        }
    }
}

__global__ void __launch_bounds__(kPermThreads) k_perm_tile_max(const int32_t* __restrict__ E, int64_t D,
                                                                int32_t* __restrict__ t_max) {
    __shared__ int red[kPermWarps];
    const int64_t r0 = (int64_t)blockIdx.x * kPermTile + (int64_t)threadIdx.x * kPermPer;
    int m = -1;
#pragma unroll
    for (int k = 0; k < kPermPer; ++k)
        if (r0 + k < D) m = max(m, E[r0 + k]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        int mm = -1;
        for (int w = 0; w < kPermWarps; ++w) mm = max(mm, red[w]);
        t_max[blockIdx.x] = mm;
    }
}

__global__ void __launch_bounds__(kPermThreads) k_perm_fill(const int32_t* __restrict__ E, int64_t D,
                                                            const int32_t* __restrict__ t_carry,
                                                            const int32_t* __restrict__ DS,
                                                            int32_t* __restrict__ out) {
    __shared__ int red[kPermWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * kPermTile + (int64_t)threadIdx.x * kPermPer;
    int v[kPermPer];
    int run = -1;
#pragma unroll
    for (int k = 0; k < kPermPer; ++k) {
        v[k] = r0 + k < D ? E[r0 + k] : -1;
        run = max(run, v[k]);
        v[k] = run;
    }
    // exclusive running maximum of the threads' maxima, then the tile's carry
    int inc = run;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int h = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc = max(inc, h);
    }
    int prev = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) prev = -1;
    if (lane == 31) red[warp] = inc;
    __syncthreads();
    for (int w = 0; w < warp; ++w) prev = max(prev, red[w]);
    prev = max(prev, t_carry[blockIdx.x]);
#pragma unroll
    for (int k = 0; k < kPermPer; ++k) {
        if (r0 + k >= D) break;
        const int32_t slot = DS[r0 + k];  // -1 past the last empty slot
        if (slot >= 0 && slot < D) out[slot] = max(prev, v[k]);
    }
}

// In-place gather: row j <- row perm[j] where they differ; a source must keep
// its own slot (perm[perm[j]] = perm[j]), else the row is left and
// PF_ERR_INVALID recorded.
template <typename VT>
__global__ void __launch_bounds__(256) k_gather_inplace(VT* __restrict__ x, int64_t P, int64_t vecs,
                                                        const int32_t* __restrict__ perm, uint32_t* ctl) {
    const int64_t total = P * vecs;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = idx / vecs, c = idx - j * vecs;
        const int32_t a = perm[j];
        if (a == j) continue;
        if (a < 0 || a >= P || perm[a] != a) {
            if (c == 0) set_status(ctl + CTL_STATUS, ST_INVALID);
            continue;
        }
        x[idx] = x[(int64_t)a * vecs + c];
    }
}

}  // namespace

size_t permute_scratch_bytes(int64_t P) {
    const int64_t T = (P + kPermTile - 1) / kPermTile;
    return ((size_t)3 * P + 4 * (size_t)T + 64) * sizeof(int32_t);
}

cudaError_t launch_permute(const int32_t* anc, int64_t P, int32_t* out, void* scratch, uint32_t* ctl, int num_sms,
                           cudaStream_t s) {
    const int64_t T = (P + kPermTile - 1) / kPermTile;
    int32_t* o = static_cast<int32_t*>(scratch);
    int32_t* E = o + P;
    int32_t* DS = E + P;
    int32_t* t_extra = DS + P;
    int32_t* t_dead = t_extra + T;
    int32_t* t_max = t_dead + T;
    cudaError_t e = cudaMemsetAsync(o, 0, (size_t)P * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(E, 0xff, (size_t)P * sizeof(int32_t), s);  // -1: no mark
    if (e == cudaSuccess) e = cudaMemsetAsync(DS, 0xff, (size_t)P * sizeof(int32_t), s);  // -1: no slot
    if (e != cudaSuccess) return e;
    int64_t blocks = (P + 255) / 256;
    if (blocks > (int64_t)num_sms * 8) blocks = (int64_t)num_sms * 8;
    k_perm_count<<<(unsigned)blocks, 256, 0, s>>>(anc, P, o, ctl);
    k_perm_tiles<<<(unsigned)T, kPermThreads, 0, s>>>(o, P, t_extra, t_dead);
    k_perm_scan<<<1, kScanThreads, 0, s>>>(t_extra, t_dead, (int)T, 0);
    k_perm_place<<<(unsigned)T, kPermThreads, 0, s>>>(o, P, t_extra, t_dead, out, E, DS);
    // the extras list has as many entries as there are empty slots, at most P;
    // entries past that count stay -1 and their DS entries -1, so nothing is written for them
    k_perm_tile_max<<<(unsigned)T, kPermThreads, 0, s>>>(E, P, t_max);
    k_perm_scan<<<1, kScanThreads, 0, s>>>(t_max, nullptr, (int)T, 1);
    k_perm_fill<<<(unsigned)T, kPermThreads, 0, s>>>(E, P, t_max, DS, out);
    return cudaGetLastError();
}

cudaError_t launch_gather_inplace(void* x, int64_t P, int64_t row_bytes, const int32_t* perm, uint32_t* ctl,
                                  int num_sms, cudaStream_t s) {
    const int64_t blocks_cap = (int64_t)num_sms * 8;
    auto go = [&](auto* p, int64_t vecs) {
        int64_t blocks = (P * vecs + 255) / 256;
        if (blocks > blocks_cap) blocks = blocks_cap;
        if (blocks < 1) blocks = 1;
        k_gather_inplace<<<(unsigned)blocks, 256, 0, s>>>(p, P, vecs, perm, ctl);
    };
    const uintptr_t a = (uintptr_t)x | (uintptr_t)row_bytes;
    if ((a & 15) == 0) go(static_cast<uint4*>(x), row_bytes / 16);
    else if ((a & 7) == 0) go(static_cast<uint2*>(x), row_bytes / 8);
    else go(static_cast<uint32_t*>(x), row_bytes / 4);
    return cudaGetLastError();
}

}  // namespace pf
