// Batched resampling of many independent filters in one launch (the many
// filters of particle MCMC, Section 1): cumulative schemes.
//
// A persistent grid takes filters from a ticket counter.  One CTA resamples a
// whole filter -- at most kMaxOwnB tiles -- so no CTA ever waits on another:
// pass 1 scans and records each tile (pf_tile.cuh); warp 0 forms the tiles'
// exact fixed-point carries; pass 2 assigns offsets tile by tile
// (systematic, stratified) or the CTA draws the filter's uniforms and
// searches its tiles (multinomial).  A filter's data may start at any 4-byte
// boundary: tiles are laid out on the aligned window, with the leading slots
// taken as zero weights.  The last CTA to finish resets the ticket.
#include <climits>

#include "pf.h"

#include "pf_assign.cuh"

namespace pf {

constexpr int kMaxOwnB = 16;  // tiles per filter: P_f + lead <= 16 * kTileMax
static_assert(PF_MAX_BATCHED_FILTER == (long long)kMaxOwnB * kTileMax, "batched filter capacity");

struct BatchShared {
    TileShared tile;
    AssignShared as;
    i128 Bown[kMaxOwnB + 1];
    int rk[kMaxOwnB];
    float rsh[kMaxOwnB], rsl[kMaxOwnB];
    int ril[kMaxOwnB];
    TableEntry table[kMaxOwnB];
    int f, skip;
};
// Dynamic shared memory after BatchShared: the staging buffer int32 out[kIoCap]
// (systematic, stratified) or the cumulative weights float v[kTileMax] of a
// one-tile filter (multinomial).

__host__ __device__ constexpr size_t batched_smem_bytes() { return sizeof(BatchShared) + kIoCap * sizeof(int32_t); }


template <int KIND>
__global__ void __launch_bounds__(kThreads, 2) k_batched(BatchParams bp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BatchShared& sm = *reinterpret_cast<BatchShared*>(smem_raw);
    unsigned char* region = smem_raw + sizeof(BatchShared);
    const int tid = threadIdx.x, lane = tid & 31;
    TileThread th;
    for (;;) {
        if (tid == 0) sm.f = (int)atomicAdd(bp.ctl + CTL_QUEUE, 1u);
        __syncthreads();
        const int ticket = sm.f;
        __syncthreads();
        if (ticket >= bp.F) break;
        const int f = bp.order ? bp.order[ticket] : ticket;
        if (bp.mask && bp.mask[f] == 0) continue;
        const int64_t off0 = bp.offsets[f], off1 = bp.offsets[f + 1];
        const int64_t Pf = off1 - off0;
        if (Pf <= 0) {
            if (Pf < 0 && tid == 0) set_status(bp.ctl + CTL_STATUS, ST_INVALID);
            continue;
        }
        const float* lwf = bp.lw + off0;
        const int lead = (int)(((uintptr_t)lwf >> 2) & 3u);
        const int64_t PA = Pf + lead;
        const int Tf = (int)((PA + kTileMax - 1) / kTileMax);
        if (Tf > kMaxOwnB) {
            if (tid == 0) set_status(bp.ctl + CTL_STATUS, ST_INVALID);
            continue;
        }
        SortedParams p;
        p.lw = lwf - lead;
        p.anc = bp.anc + off0;
        p.P = Pf;
        p.Pd = (double)Pf;
        p.tile = kTileMax;
        p.n_tiles = Tf;
        p.tiles_per_cta = Tf;
        const uint64_t seed = bp.seeds[f];
        p.key0 = (uint32_t)(seed & 0xffffffffu);
        p.key1 = (uint32_t)(seed >> 32);
        p.filter = (uint32_t)f;
        p.ctl = bp.ctl;
        p.slots = nullptr;
        p.wait_ns = 0;
        p.skip_tile = -1;
        p.lead = lead;
        // cumulative weights of the filter's tiles: multinomial searches them;
        // systematic and stratified reload them in pass 2 instead of rescanning
        p.v_out = (KIND == KIND_MULTI && Tf == 1) ? reinterpret_cast<float*>(region)
                  : (Tf > 1 ? bp.scratch + (int64_t)blockIdx.x * bp.scratch_per_cta : nullptr);

        // pass 1: scan and record the filter's tiles
        TileSummary ts;
        int bad = 0;
        for (int c = 0; c < Tf; ++c) {
            const int64_t t0 = (int64_t)c * kTileMax;
            const int n = (int)min((int64_t)kTileMax, PA - t0);
            ts = tile_scan(p.lw + t0, c == 0 ? lead : 0, n, sm.tile, th);
            bad |= ts.bad;
            if (tid == 0) {
                sm.rk[c] = ts.k;
                sm.rsh[c] = ts.S.hi;
                sm.rsl[c] = ts.S.lo;
                sm.ril[c] = ts.i_last;
            }
            if (KIND == KIND_MULTI || c < Tf - 1) {
                if (p.v_out) write_tile_v(p, th, t0, n);
            }
            __syncthreads();
        }
        // carries of the filter's tiles (warp 0, one tile per lane)
        if (tid < 32) {
            int kmax = (lane < Tf && sm.rsh[lane] > 0.f) ? sm.rk[lane] : INT_MIN;
            kmax = warp_max_i(kmax);
            const int skip = (kmax == INT_MIN || bad) ? 1 : 0;
            if (lane == 0) {
                sm.skip = skip;
                if (skip) set_status(bp.ctl + CTL_STATUS, ST_DOMAIN);
            }
            if (!skip) {
                const int sh = lane < Tf ? sm.rk[lane] - kmax : 0;
                const i128 a = lane < Tf ? fixed_of(sm.rsh[lane], sh) + fixed_of(sm.rsl[lane], sh) : (i128)0;
                const i128 inc = warp_scan_i128(a, lane);
                const i128 B = inc - a;
                if (lane < Tf) {
                    sm.Bown[lane] = B;
                    if (KIND == KIND_MULTI) {
                        const fpair b = fixed_to_pair(B);
                        sm.table[lane] = {b.hi, b.lo, pow2f(-sh), sm.ril[lane]};
                    }
                }
                if (lane == 31) {
                    sm.Bown[Tf] = inc;
                    sm.as.Wt = inc;
                    sm.as.K = kmax;
                    const fpair Wp = fixed_to_pair(inc);
                    sm.as.W_hi = Wp.hi;
                    sm.as.W_lo = Wp.lo;
                }
            }
        }
        __syncthreads();
        if (sm.skip) continue;

        if (KIND == KIND_MULTI) {
            const int64_t nq = (Pf + 3) >> 2;  // four draws per Philox block
            for (int64_t q = tid; q < nq; q += kThreads) {
                const u32x4 r = philox((uint32_t)q, 0u, p.filter, TAG_MULTI, p.key0, p.key1);
                int32_t a[4];
                if (Tf == 1)
                    multinomial_draws4<true>(r, sm.table, Tf, p.v_out, kTileMax, PA, lead, sm.as.W_hi, sm.as.W_lo, a);
                else
                    multinomial_draws4<false>(r, sm.table, Tf, p.v_out, kTileMax, PA, lead, sm.as.W_hi, sm.as.W_lo,
                                              a);
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    if (4 * q + s < Pf) p.anc[4 * q + s] = a[s];
            }
            __syncthreads();
            continue;
        }
        // pass 2: offsets tile by tile (the last tile's scan is still in registers)
        int32_t* out = reinterpret_cast<int32_t*>(region);
        for (int c = Tf - 1; c >= 0; --c) {
            const int64_t t0 = (int64_t)c * kTileMax;
            if (c != Tf - 1) {
                read_tile_v(p.v_out + t0, (int)min((int64_t)kTileMax, PA - t0), th);
                ts.k = sm.rk[c];
                ts.i_last = sm.ril[c];
            }
            if (tid == 0) tile_offsets<KIND>(p, sm.as, sm.Bown[c], sm.Bown[c + 1], ts.k);
            __syncthreads();
            assign_offspring<KIND>(p, sm.as, out, th, ts, t0 - lead);
        }
    }
    // every CTA has drawn a ticket past the end: the last one to leave resets the queue
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(bp.ctl + CTL_QUEUE_DONE, 1u) == gridDim.x - 1) {
            atomicExch(bp.ctl + CTL_QUEUE, 0u);
            atomicExch(bp.ctl + CTL_QUEUE_DONE, 0u);
        }
    }
}

int batched_blocks_per_sm(int kind) {
    int nb = 0;
    const size_t smem = batched_smem_bytes();
    cudaError_t e = cudaErrorInvalidValue;
    switch (kind) {
    case KIND_MULTI:
        if (cudaFuncSetAttribute(k_batched<KIND_MULTI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
            cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched<KIND_MULTI>, kThreads, smem);
        break;
    case KIND_STRAT:
        if (cudaFuncSetAttribute(k_batched<KIND_STRAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
            cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched<KIND_STRAT>, kThreads, smem);
        break;
    case KIND_SYS:
        if (cudaFuncSetAttribute(k_batched<KIND_SYS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
            cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched<KIND_SYS>, kThreads, smem);
        break;
    }
    return e == cudaSuccess ? nb : 0;
}

size_t batched_scratch_floats_per_cta() { return (size_t)kMaxOwnB * kTileMax; }

// One CTA: a counting sort of the filters by tile count, largest first (the
// order within a class is whatever the shared-memory atomics give; each
// filter's result does not depend on it).
constexpr int kOrderThreads = 1024;
__global__ void __launch_bounds__(kOrderThreads) k_batched_order(const int64_t* __restrict__ offsets, int F,
                                                                 int32_t* __restrict__ order) {
    __shared__ int start[kMaxOwnB + 2];
    const int tid = threadIdx.x;
    if (tid < kMaxOwnB + 2) start[tid] = 0;
    __syncthreads();
    auto cls = [&](int f) {
        const int64_t n = offsets[f + 1] - offsets[f];
        return n <= 0 ? 0 : (int)min((int64_t)kMaxOwnB + 1, (n + kTileMax - 1) / kTileMax);
    };
    for (int f = tid; f < F; f += kOrderThreads) atomicAdd(&start[cls(f)], 1);
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        for (int c = kMaxOwnB + 1; c >= 0; --c) {
            const int n = start[c];
            start[c] = run;
            run += n;
        }
    }
    __syncthreads();
    for (int f = tid; f < F; f += kOrderThreads) order[atomicAdd(&start[cls(f)], 1)] = f;
}

cudaError_t launch_batched_order(const int64_t* offsets, int F, int32_t* order, cudaStream_t s) {
    k_batched_order<<<1, kOrderThreads, 0, s>>>(offsets, F, order);
    return cudaGetLastError();
}

cudaError_t launch_batched(int kind, const BatchParams& bp, int grid, cudaStream_t s) {
    const size_t smem = batched_smem_bytes();
    switch (kind) {
    case KIND_MULTI: k_batched<KIND_MULTI><<<grid, kThreads, smem, s>>>(bp); break;
    case KIND_STRAT: k_batched<KIND_STRAT><<<grid, kThreads, smem, s>>>(bp); break;
    case KIND_SYS: k_batched<KIND_SYS><<<grid, kThreads, smem, s>>>(bp); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pf
