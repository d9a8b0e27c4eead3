// Batched resampling of many independent filters in one launch (the many
// filters of particle MCMC, Section 1): cumulative schemes.
//
// A one-CTA plan pass turns the filters into a list of work items, largest
// filters first (a counting sort by tile count), skipping masked and empty
// filters.  A persistent grid then takes items from a ticket counter:
//   - a filter of one tile (or any multinomial filter) is one item, done by
//     one CTA with no wait on any other: scan and record each tile
//     (pf_tile.cuh), warp 0 forms the tiles' exact fixed-point carries, then
//     offsets are assigned (systematic, stratified) or the filter's uniforms
//     drawn and searched (multinomial);
//   - a systematic or stratified filter of Tf > 1 tiles is Tf items with
//     consecutive tickets, one tile each: every CTA scans its tile in
//     registers, publishes a 16-byte record, waits (bounded) until all Tf
//     records of its filter are in, forms the same carries from them and
//     assigns its own tile's offsets.  Tiles of one filter hold consecutive
//     tickets and a filter has at most kMaxOwnB < grid tiles, so every tile a
//     CTA waits for has been or will be taken by a running CTA (the launch is
//     cooperative, so all CTAs are resident);
//   - unless such filters are at least as many as the resident CTAs: then the
//     plan keeps each one whole, a single item whose CTA scans all its tiles
//     (cumulative weights to the CTA's scratch), forms the carries and every
//     tile's offset map, and assigns the tiles, with no wait on another CTA.
// A filter's data may start at any 4-byte boundary: tiles are laid out on the
// aligned window, with the leading slots taken as zero weights.  The last CTA
// to finish resets the ticket; the last CTA of a split filter resets its
// arrival counters.
#include <climits>

#include "pf.h"

#include "pf_assign.cuh"

namespace pf {

constexpr int kMaxOwnB = 16;  // tiles per filter: P_f + lead <= 16 * kTileMax
static_assert(PF_MAX_BATCHED_FILTER == (long long)kMaxOwnB * kTileMax, "batched filter capacity");
static_assert(kMaxOwnB <= 31, "the carries give one tile to each lane of warp 0; item codes use 5 bits");
static_assert(kMaxOwnB == kMaxItemsPerFilter, "items per filter");
static_assert(kMaxOwnB * (kTileMax / kWin) <= kIoCap, "coarse samples of a multinomial filter fit the staging region");
constexpr int kWhole = 31;  // item code: the whole filter in one CTA

struct BatchShared {
    TileShared tile;
    AssignShared as;
    i128 Bown[kMaxOwnB + 1];
    int rk[kMaxOwnB];
    float rsh[kMaxOwnB], rsl[kMaxOwnB];
    int ril[kMaxOwnB];
    TableEntry table[kMaxOwnB];
    TileMap maps[kMaxOwnB];  // systematic / stratified whole filters: each tile's offset map
    int f, skip;
};
// Dynamic shared memory: BatchShared, then the region -- the two run-length
// staging buffers int32 stage[2 * kIoCap] (systematic, stratified), or the
// cumulative weights float v[kTileMax] of a one-tile filter / the coarse
// samples of a several-tile one (multinomial).
__host__ __device__ constexpr size_t batched_smem_bytes() {
    return sizeof(BatchShared) + 2 * kIoCap * sizeof(int32_t);
}
static_assert(sizeof(BatchShared) % 16 == 0, "the region is 16-byte aligned");


// The filter's geometry and parameters for the tile routines.
__device__ __forceinline__ void filter_params(const BatchParams& bp, int f, int64_t off0, int64_t Pf, int lead, int Tf,
                                              SortedParams& p) {
    p.lw = bp.lw + off0 - lead;
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
    p.v_out = nullptr;
    p.c2_out = nullptr;
    p.c1_out = nullptr;
    p.cpt2 = p.cpt1 = 0;
    p.c1shift = 8;
    p.g_out = nullptr;
    p.M = 0;
    p.guide = 0;
}

// Warp 0: the exact fixed-point carries of a filter's Tf tiles from their
// records (lane t holds tile t's exponent, sum and last positive element)
// into sm.Bown / sm.as (and the multinomial tile table); sm.skip = 1 (and
// PF_ERR_DOMAIN from `report`) when a tile saw NaN/+inf or all weights are zero.
template <int KIND>
__device__ __forceinline__ void filter_carries(BatchShared& sm, const BatchParams& bp, int Tf, int lane, int k,
                                               float shi, float slo, int il, int bad, bool report) {
    int kmax = (lane < Tf && shi > 0.f) ? k : INT_MIN;
    kmax = warp_max_i(kmax);
    bad = __any_sync(0xffffffffu, lane < Tf && bad);
    const int skip = (kmax == INT_MIN || bad) ? 1 : 0;
    if (lane == 0) {
        sm.skip = skip;
        if (skip && report) set_status(bp.ctl + CTL_STATUS, ST_DOMAIN);
    }
    if (skip) return;
    const int sh = lane < Tf ? k - kmax : 0;
    const i128 a = lane < Tf ? fixed_of(shi, sh) + fixed_of(slo, sh) : (i128)0;
    const i128 inc = warp_scan_i128(a, lane);
    const i128 B = inc - a;
    if (lane < Tf) {
        sm.Bown[lane] = B;
        if (KIND == KIND_MULTI) {
            const fpair b = fixed_to_pair(B);
            sm.table[lane] = {b.hi, b.lo, pow2f(-sh), il};
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

template <int KIND>
__global__ void __launch_bounds__(kThreads, 2) k_batched(BatchParams bp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BatchShared& sm = *reinterpret_cast<BatchShared*>(smem_raw);
    unsigned char* region = smem_raw + sizeof(BatchShared);
    const int tid = threadIdx.x, lane = tid & 31;
    const int n_items = (int)ld_relaxed_u32(bp.ctl + CTL_ITEMS);
    TileThread th;
    uint32_t chunks = 0;  // staging chunks decoded by this CTA
    if (KIND != KIND_MULTI) stage_init<kIoCap>(reinterpret_cast<int32_t*>(region));  // before the first ticket's barriers
    for (;;) {
        if (tid == 0) sm.f = (int)atomicAdd(bp.ctl + CTL_QUEUE, 1u);
        __syncthreads();
        const int ticket = sm.f;
        __syncthreads();
        if (ticket >= n_items) break;
        const int item = bp.items[ticket];
        const int f = item >> 5, c_item = item & 31;
        const int64_t off0 = bp.offsets[f];
        const int64_t Pf = bp.offsets[f + 1] - off0;
        const int lead = (int)(((uintptr_t)(bp.lw + off0) >> 2) & 3u);
        const int64_t PA = Pf + lead;
        const int Tf = (int)((PA + kTileMax - 1) / kTileMax);
        SortedParams p;
        filter_params(bp, f, off0, Pf, lead, Tf, p);
        int32_t* stage = reinterpret_cast<int32_t*>(region);
        if (bp.trace) {
            trace_stamp(bp.trace, bp.trace_cap, ticket, 0);
            for (int w = 1; w <= 4; ++w) trace_put(bp.trace, bp.trace_cap, ticket, w, 0);
            trace_put(bp.trace, bp.trace_cap, ticket, 5, blockIdx.x);
            trace_put(bp.trace, bp.trace_cap, ticket, 6, (uint64_t)f);
            trace_put(bp.trace, bp.trace_cap, ticket, 7, (uint64_t)c_item);
        }

        if (KIND != KIND_MULTI && c_item == kWhole && Tf > 1) {
            // ---- systematic / stratified: a whole filter of several tiles in this CTA (the plan
            // gives whole filters when there are enough of them to occupy the grid): every tile is
            // scanned (the cumulative weights of all but the last kept in this CTA's scratch), warp 0
            // forms the carries, two lanes per tile the offset maps, then the tiles are assigned,
            // last first -- no wait on any other CTA ----
            p.v_out = bp.scratch + (int64_t)blockIdx.x * bp.scratch_per_cta;
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
                if (c + 1 < Tf) write_tile_v(p, th, t0, n);  // reloaded for its assignment
                __syncthreads();
            }
            trace_stamp(bp.trace, bp.trace_cap, ticket, 1);
            trace_stamp(bp.trace, bp.trace_cap, ticket, 2);
            if (tid < 32) {
                const bool in = lane < Tf;
                filter_carries<KIND>(sm, bp, Tf, lane, in ? sm.rk[lane] : 0, in ? sm.rsh[lane] : 0.f,
                                     in ? sm.rsl[lane] : 0.f, in ? sm.ril[lane] : -1, bad, true);
            }
            __syncthreads();
            if (!sm.skip) {
                trace_stamp(bp.trace, bp.trace_cap, ticket, 3);
                if (tid < 32) {  // Tf <= 16 pairs of lanes of warp 0
                    const int r = min(tid >> 1, Tf - 1);
                    const TileMap m = tile_map_pair<KIND>(p, sm.as, sm.Bown[r], sm.Bown[r + 1], sm.rk[r], 0xffffffffu);
                    if ((tid & 1) == 0 && (tid >> 1) < Tf) sm.maps[tid >> 1] = m;
                }
                __syncthreads();
                for (int c = Tf - 1; c >= 0; --c) {
                    const int64_t t0 = (int64_t)c * kTileMax;
                    if (c != Tf - 1) read_tile_v(p.v_out + t0, (int)min((int64_t)kTileMax, PA - t0), th);
                    ts.i_last = sm.ril[c];
                    const TileMap map = sm.maps[c];
                    if (th.K == 16)
                        assign_offspring<KIND, 16>(p, sm.as, map, stage, chunks, th, ts, t0 - lead);
                    else if (th.K == 8)
                        assign_offspring<KIND, 8>(p, sm.as, map, stage, chunks, th, ts, t0 - lead);
                    else
                        assign_offspring<KIND, 4>(p, sm.as, map, stage, chunks, th, ts, t0 - lead);
                }
                if (bp.trace) {
                    __syncthreads();
                    trace_stamp(bp.trace, bp.trace_cap, ticket, 4);
                }
            }
            __syncthreads();
            continue;
        }
        if (KIND != KIND_MULTI) {
            // ---- systematic / stratified: one tile (a one-tile filter is its own item) ----
            const int c = c_item == kWhole ? 0 : c_item;
            const int64_t t0 = (int64_t)c * kTileMax;
            TileSummary ts = tile_scan(p.lw + t0, c == 0 ? lead : 0, (int)min((int64_t)kTileMax, PA - t0), sm.tile, th);
            uint32_t* rec = reinterpret_cast<uint32_t*>(bp.records + (ticket - c));  // the filter's Tf records
            uint32_t* arrive = bp.counters + 2 * f;
            if (tid == 0) {
                trace_stamp(bp.trace, bp.trace_cap, ticket, 1);
                int ok = 1;
                if (Tf > 1 && c == bp.skip_tile) {
                    ok = 0;  // test hook: withhold this tile's record; the filter's other tiles time out
                } else if (Tf > 1) {
                    st_v4_u32(rec + 4 * c, (uint32_t)ts.k, __float_as_uint(ts.S.hi), __float_as_uint(ts.S.lo),
                              (uint32_t)(ts.i_last + 1) | (ts.bad ? 0x80000000u : 0u));
                    __threadfence();
                    red_release_add_u32(arrive, 1u);
                    const uint64_t t_start = global_ns();
                    for (uint32_t it = 1; ld_acquire_u32(arrive) < (uint32_t)Tf; ++it) {
                        if ((it & 7u) == 0u && global_ns() - t_start > bp.wait_ns) {
                            ok = 0;
                            break;
                        }
                        __nanosleep(32);
                    }
                    if (!ok) set_status(bp.ctl + CTL_STATUS, ST_TIMEOUT);
                } else {
                    sm.rk[0] = ts.k;
                    sm.rsh[0] = ts.S.hi;
                    sm.rsl[0] = ts.S.lo;
                    sm.ril[0] = ts.i_last;
                }
                sm.skip = !ok;
                trace_stamp(bp.trace, bp.trace_cap, ticket, 2);
            }
            __syncthreads();
            if (!sm.skip) {
                if (tid < 32) {
                    uint4 r = make_uint4(0, 0, 0, 0);
                    if (Tf > 1) {
                        if (lane < Tf) r = ld_cg_v4_u32(rec + 4 * lane);
                    } else if (lane == 0) {
                        r = make_uint4((uint32_t)sm.rk[0], __float_as_uint(sm.rsh[0]), __float_as_uint(sm.rsl[0]),
                                       (uint32_t)(sm.ril[0] + 1) | (ts.bad ? 0x80000000u : 0u));
                    }
                    filter_carries<KIND>(sm, bp, Tf, lane, (int)r.x, __uint_as_float(r.y), __uint_as_float(r.z),
                                         (int)(r.w & 0x7fffffffu) - 1, (int)(r.w >> 31), c == 0);
                }
                __syncthreads();
                if (!sm.skip) {
                    trace_stamp(bp.trace, bp.trace_cap, ticket, 3);
                    if (tid < 2) tile_offsets<KIND>(p, sm.as, sm.Bown[c], sm.Bown[c + 1], ts.k);
                    __syncthreads();
                    const TileMap map = {sm.as.jlo, sm.as.noff, sm.as.tau0, sm.as.inv_rho};
                    // elements per thread as a constant: 16 for full tiles, fewer for small filters
                    if (th.K == 16)
                        assign_offspring<KIND, 16>(p, sm.as, map, stage, chunks, th, ts, t0 - lead);
                    else if (th.K == 8)
                        assign_offspring<KIND, 8>(p, sm.as, map, stage, chunks, th, ts, t0 - lead);
                    else
                        assign_offspring<KIND, 4>(p, sm.as, map, stage, chunks, th, ts, t0 - lead);
                    if (bp.trace) {
                        __syncthreads();
                        trace_stamp(bp.trace, bp.trace_cap, ticket, 4);
                    }
                }
            }
            // the last of a split filter's CTAs to leave resets its counters
            if (Tf > 1 && tid == 0 && atomicAdd(bp.counters + 2 * f + 1, 1u) == (uint32_t)Tf - 1u) {
                atomicExch(arrive, 0u);
                atomicExch(bp.counters + 2 * f + 1, 0u);
            }
            __syncthreads();
            continue;
        }

        // ---- a whole filter in this CTA ----
        // cumulative weights of the filter's tiles: multinomial searches them
        if (KIND == KIND_MULTI)
            p.v_out = Tf == 1 ? reinterpret_cast<float*>(region) : bp.scratch + (int64_t)blockIdx.x * bp.scratch_per_cta;
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
            if (KIND == KIND_MULTI) {
                write_tile_v(p, th, t0, n);
                // several tiles: the coarse samples go to the (otherwise unused) staging region
                if (Tf > 1) write_tile_coarse(th, n, reinterpret_cast<float*>(region) + c * (kTileMax / kWin));
            }
            __syncthreads();
        }
        trace_stamp(bp.trace, bp.trace_cap, ticket, 1);
        trace_stamp(bp.trace, bp.trace_cap, ticket, 2);
        if (tid < 32) {
            const bool in = lane < Tf;
            filter_carries<KIND>(sm, bp, Tf, lane, in ? sm.rk[lane] : 0, in ? sm.rsh[lane] : 0.f,
                                 in ? sm.rsl[lane] : 0.f, in ? sm.ril[lane] : -1, bad, true);
        }
        __syncthreads();
        if (sm.skip) continue;
        trace_stamp(bp.trace, bp.trace_cap, ticket, 3);

        if (KIND == KIND_MULTI) {
            const int64_t nq = (Pf + 3) >> 2;  // four draws per Philox block
            // the same number of passes in every thread (the windowed draws read
            // quad-cooperatively); a lane past the end redraws block 0
            for (int64_t q0 = 0; q0 < nq; q0 += kThreads) {
                const bool mine = q0 + tid < nq;
                if (!__any_sync(0xffffffffu, mine)) continue;  // the whole warp is past the end
                const int64_t q = mine ? q0 + tid : 0;
                const u32x4 r = philox((uint32_t)q, 0u, p.filter, TAG_MULTI, p.key0, p.key1);
                int32_t a[4];
                if (Tf == 1) {
                    multinomial_draws4<true>(r, sm.table, Tf, p.v_out, kTileMax, PA, lead, sm.as.W_hi, sm.as.W_lo, a);
                } else {
                    const float* coarse = reinterpret_cast<const float*>(region);
#pragma unroll
                    for (int s = 0; s < 4; ++s)
                        a[s] = multinomial_draw_windowed(word_of(r, s), sm.table, Tf, p.v_out, coarse, kTileMax / kWin,
                                                         kTileMax, PA, lead, sm.as.W_hi, sm.as.W_lo);
                }
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    if (mine && 4 * q + s < Pf) p.anc[4 * q + s] = a[s];
            }
            __syncthreads();
            trace_stamp(bp.trace, bp.trace_cap, ticket, 4);
            continue;
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

// The plan: one CTA sorts the filters by tile count, largest first (a
// counting sort; the order within a class is whatever the shared-memory
// atomics give, and no filter's result depends on it) and writes the items
// f * 32 + c (tile c of a split filter) or f * 32 + kWhole.  Masked and empty
// filters get no item; a negative size or a filter beyond kMaxOwnB tiles sets
// PF_ERR_INVALID and gets none.  The item count goes to ctl[CTL_ITEMS].
constexpr int kPlanThreads = 1024;
__global__ void __launch_bounds__(kPlanThreads) k_batched_plan(const float* __restrict__ lw,
                                                               const int64_t* __restrict__ offsets, int F,
                                                               const int32_t* __restrict__ mask, int split,
                                                               int32_t* __restrict__ items, uint32_t* ctl, int metro,
                                                               int split_min) {
    __shared__ int count[kMaxOwnB + 1], start[kMaxOwnB + 1], split_sm;
    const int tid = threadIdx.x;
    if (tid <= kMaxOwnB) count[tid] = 0;
    if (metro) {
        // Metropolis: a new launch epoch, and an empty list of shared filters after the items
        if (tid == 0) {
            ctl[CTL_METRO_EPOCH] += 1u;
            ctl[CTL_HEAVY] = 0u;
        }
        for (int i = tid; i < min(F, kMaxHeavy); i += kPlanThreads) items[F + i] = 0;
    }
    __syncthreads();
    auto tiles = [&](int f) -> int {  // 0: no item
        if (mask && mask[f] == 0) return 0;
        const int64_t off0 = offsets[f], n = offsets[f + 1] - off0;
        if (n <= 0) {
            if (n < 0) set_status(ctl + CTL_STATUS, ST_INVALID);
            return 0;
        }
        const int lead = (int)(((uintptr_t)(lw + off0) >> 2) & 3u);
        const int64_t T = (n + lead + kTileMax - 1) / kTileMax;
        if (T > kMaxOwnB) {
            set_status(ctl + CTL_STATUS, ST_INVALID);
            return 0;
        }
        return (int)T;
    };
    for (int f = tid; f < F; f += kPlanThreads) {
        const int T = tiles(f);
        if (T) atomicAdd(&count[T], 1);
    }
    __syncthreads();
    if (tid == 0) {
        // several-tile filters are split over CTAs only while they are too few to occupy the grid
        int multi = 0;
        for (int T = 2; T <= kMaxOwnB; ++T) multi += count[T];
        const int sp = split && multi < split_min;
        split_sm = sp;
        int run = 0;
        for (int T = kMaxOwnB; T >= 1; --T) {
            start[T] = run;
            run += count[T] * (sp && T > 1 ? T : 1);
        }
        ctl[CTL_ITEMS] = (uint32_t)run;
    }
    __syncthreads();
    const int sp = split_sm;
    for (int f = tid; f < F; f += kPlanThreads) {
        const int T = tiles(f);
        if (!T) continue;
        const int per = sp && T > 1 ? T : 1;
        const int at = atomicAdd(&start[T], per);
        if (per == 1) {
            items[at] = f * 32 + kWhole;
        } else {
            for (int c = 0; c < T; ++c) items[at + c] = f * 32 + c;
        }
    }
}

cudaError_t launch_batched_plan(const float* lw, const int64_t* offsets, int F, const int32_t* mask, int split,
                                int32_t* items, uint32_t* ctl, cudaStream_t s, int metro, int split_min) {
    k_batched_plan<<<1, kPlanThreads, 0, s>>>(lw, offsets, F, mask, split, items, ctl, metro, split_min);
    return cudaGetLastError();
}

template <int KIND>
static cudaError_t launch_batched_kind(const BatchParams& bp, int grid, cudaStream_t s) {
    // cooperative: every CTA resident, so a CTA waiting for the other tiles of
    // a split filter never waits on a CTA that cannot run
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = batched_smem_bytes();
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batched<KIND>, bp);
}

cudaError_t launch_batched(int kind, const BatchParams& bp, int grid, cudaStream_t s) {
    switch (kind) {
    case KIND_MULTI: return launch_batched_kind<KIND_MULTI>(bp, grid, s);
    case KIND_STRAT: return launch_batched_kind<KIND_STRAT>(bp, grid, s);
    case KIND_SYS: return launch_batched_kind<KIND_SYS>(bp, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace pf
