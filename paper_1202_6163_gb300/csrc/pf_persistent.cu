// Single-launch resamplers for the cumulative schemes (Figure 1a-c).
//
// One cooperative launch; every CTA is resident and owns R >= 1 consecutive
// tiles of log-weights:
//   1. pass 1, per owned tile: tile scan (pf_tile.cuh) -- the tile's weights,
//      its local cumulative weights v_i, its sum S_t relative to 2^{k_t}.
//      Systematic / stratified: every tile but the last keeps its v_i in
//      global scratch (the last stays in registers), and the CTA publishes one
//      32-byte record of its own mass, S_c = sum_t S_t 2^{k_t - k_c} as an
//      exact 128-bit fixed-point sum relative to its largest tile exponent
//      k_c.  Multinomial: each tile writes v_i and a 16-byte record
//      (k_t, S_t, i_last);
//   2. the CTA arrives on this launch's counter (release) and one thread waits,
//      with a time limit, until every CTA has arrived;
//   3. carries.  Systematic / stratified: the CTA reads the G CTA records
//      (one per thread) and forms the largest exponent K, the mass below this
//      CTA and the total W
//      = sum_c S_c 2^{k_c - K} (exact integer sums, so every CTA holds the
//      same bits and W is the scan's own last prefix), then the boundaries of
//      its own tiles from its own tile sums; two lanes per owned tile then
//      form each tile's offset range and offset map.  Multinomial: every CTA
//      reads all T tile records and forms every tile's carry
//          B_t = sum_{t' < t} S_t' 2^{k_t' - K}
//      (exact 128-bit fixed point, 2^-90 relative to 2^K) for its tile table;
//   4. systematic / stratified (Section 2: these schemes yield offspring
//      counts), per owned tile, last first (the others reload their v_i): the
//      tile owns the offsets j whose position (j + u_j) W / P lies in
//      [B_t, B_{t+1}); each element counts the offsets below its cumulative
//      weight, N_i, and its index fills [N_{i-1}, N_i) by a run-length decode
//      in shared memory (mark run starts, block max-scan), stored with 128-bit
//      writes;
//      multinomial: the CTA draws a balanced slice of the P uniforms; a draw
//      finds its tile from a lookup of the tile boundaries and its element in
//      three levels (every 2^c1shift-th v_i in shared memory, then one
//      16-entry window of the every-16th samples and one of v_i, read from L2).
//      Above one tile per CTA the CTAs first decode a guide table (the first
//      particle above each of P/4 evenly spaced targets) and arrive a second
//      time; a draw then reads its guide entry and one window of v_i, and
//      takes the three-level search only where that window does not settle it.
// Every global write is bounded by [0, P) whatever the data; a NaN/+inf or
// all-zero weight set records PF_ERR_DOMAIN and writes no ancestors.
#include <climits>

#include "pf_assign.cuh"

namespace pf {

constexpr int kMaxOwn = 64;  // tiles per CTA

struct PersistShared {
    TileShared tile;
    AssignShared as;
    i128 wsum[kWarps], wsum2[kWarps];
    i128 Bown[kMaxOwn + 1];  // boundaries of this CTA's tiles
    // the owned tiles' summaries and offset maps (multinomial: exponents, last
    // positive elements and the guide's maps)
    TileMap own_map[kMaxOwn];
    float own_shi[kMaxOwn], own_slo[kMaxOwn];
    int own_k[kMaxOwn], own_il[kMaxOwn];
    int red_k[kWarps];
    int ok;
    uint64_t bar[2];  // completion of the tile copies into the two staging buffers (pass 1)
};
// Dynamic shared memory: PersistShared, then either the two staging buffers
// int32 stage[2 * kIoCap] (systematic, stratified) or, for multinomial, TableEntry
// table[T], the tile lookup int lut[kLut + 1] and the level-1 samples
// float c1[T * cpt1] (sized by the launch).

// Staging entries per buffer for KK elements per thread: tiles of up to 4096
// elements (KK <= 8) need fewer, and the smaller buffers keep more of the SM's
// shared memory as L1.
__host__ __device__ constexpr int stage_cap(int KK) { return KK == 16 ? kIoCap : kIoCapSmall; }

__host__ __device__ constexpr size_t persistent_smem_bytes(int kind, int T, int KK) {
    return sizeof(PersistShared) + (kind == KIND_MULTI ? (size_t)T * sizeof(TableEntry) + (kLut + 1) * sizeof(int)
                                                       : 2 * (size_t)stage_cap(KK) * sizeof(int32_t));
}

// ---------------------------------------------------------------------------
// Arrival and carries.  Block-wide; identical results in every CTA.
// ---------------------------------------------------------------------------
// Arrive on this epoch's counter with release semantics (after the CTA's
// records are written) and wait, one thread, bounded, for every CTA.
// `base` names the pair of counters (CTL_ARRIVE0, or CTL_ARRIVE2 for the
// multinomial kernel's second arrival).
__device__ bool arrive_and_wait(const SortedParams& p, PersistShared& sm, bool skip, uint32_t epoch,
                                uint64_t t_start, int base = CTL_ARRIVE0) {
    const int tid = threadIdx.x;
    uint32_t* arrive = p.ctl + base + (epoch & 1u);
    if (tid == 0) {
        if (!skip) red_release_add_u32(arrive, 1u);
        int ok = 1;
        for (uint32_t it = 1; ld_acquire_u32(arrive) < gridDim.x; ++it) {
            if ((it & 7u) == 0u && global_ns() - t_start > p.wait_ns) {
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        sm.ok = ok;
    }
    __syncthreads();
    return sm.ok != 0;
}

// Block exclusive scan of one int128 per thread; returns the exclusive prefix
// and leaves the block total in sm.as.Wt.
__device__ __forceinline__ i128 block_scan_i128(PersistShared& sm, i128 x) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const i128 inc = warp_scan_i128(x, lane);
    if (lane == 31) sm.wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const i128 v = lane < kWarps ? sm.wsum[lane] : (i128)0;
        const i128 vi = warp_scan_i128(v, lane);
        if (lane < kWarps) sm.wsum[lane] = vi - v;
        if (lane == kWarps - 1) sm.as.Wt = vi;
    }
    __syncthreads();
    return sm.wsum[warp] + (inc - x);
}

template <int KIND>
__device__ bool carries(const SortedParams& p, PersistShared& sm, TableEntry* table, int t_first, int t_count) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = p.n_tiles;
    const uint32_t* rec = reinterpret_cast<const uint32_t*>(p.slots);
    // largest tile exponent among tiles with weight; NaN/+inf check
    int bad = 0, kmax = INT_MIN;
    uint4 mine = make_uint4(0, 0, 0, 0xffffffffu);  // record `tid`, kept for the second pass
    for (int t = tid; t < T; t += kThreads) {
        const uint4 r = ld_cg_v4_u32(rec + 4 * t);
        if (t == tid) mine = r;
        const float sh = __uint_as_float(r.y);
        bad |= !(sh <= 3.402823466e38f);
        if (sh > 0.f) kmax = max(kmax, (int)r.x);
    }
    kmax = warp_max_i(kmax);
    if (lane == 0) sm.red_k[warp] = kmax;
    bad = __syncthreads_or(bad);
    int K = sm.red_k[0];
#pragma unroll
    for (int q = 1; q < kWarps; ++q) K = max(K, sm.red_k[q]);
    if (K == INT_MIN || bad) {  // every weight zero, or a bad tile
        if (tid == 0) set_status(p.ctl + CTL_STATUS, ST_DOMAIN);
        return false;
    }
    // exact prefix sums of the tile masses, kThreads tiles per pass
    i128 running = 0;
    for (int base = 0; base < T; base += kThreads) {
        const int t = base + tid;
        uint4 r = make_uint4(0, 0, 0, 0xffffffffu);
        if (t < T) r = base == 0 ? mine : ld_cg_v4_u32(rec + 4 * t);
        const int sh = (int)r.x - K;
        const i128 a = (t < T) ? fixed_of(__uint_as_float(r.y), sh) + fixed_of(__uint_as_float(r.z), sh) : (i128)0;
        const i128 B = running + block_scan_i128(sm, a);  // carry of tile t
        running += sm.as.Wt;
        __syncthreads();  // sm.wsum / sm.as.Wt are reused by the next pass
        if (t < T) {
            if (KIND == KIND_MULTI) {
                const fpair b = fixed_to_pair(B);
                table[t] = {b.hi, b.lo, pow2f(-sh), (int)r.w};
            }
            if (t >= t_first && t <= t_first + t_count) sm.Bown[t - t_first] = B;  // the owned tiles' boundaries
        }
    }
    if (tid == 0) {
        sm.as.K = K;
        sm.as.Wt = running;
        if (t_first + t_count == T) sm.Bown[t_count] = running;
        const fpair Wp = fixed_to_pair(running);
        sm.as.W_hi = Wp.hi;
        sm.as.W_lo = Wp.lo;
    }
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------------------
// Systematic / stratified: one 32-byte record per CTA, carries by warp 0.
// ---------------------------------------------------------------------------
// Record of CTA c at slots[4c .. 4c+4): (k_c, flags) then S_c as four 32-bit
// words, low first; flags bit 0: a NaN/+inf weight, bit 1: positive mass.
constexpr uint32_t kRecBad = 1u, kRecMass = 2u;

__device__ __forceinline__ i128 i128_of(uint4 w) {
    return (i128)(((unsigned __int128)(((uint64_t)w.w << 32) | w.z) << 64) | (((uint64_t)w.y << 32) | w.x));
}

__device__ __forceinline__ i128 warp_sum_i128(i128 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
        const unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        const unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        v += (i128)(((unsigned __int128)h2 << 64) | l2);
    }
    return v;
}

__device__ __forceinline__ i128 shfl_i128(i128 v, int src) {
    const unsigned long long lo = __shfl_sync(0xffffffffu, (unsigned long long)v, src);
    const unsigned long long hi = __shfl_sync(0xffffffffu, (unsigned long long)(v >> 64), src);
    return (i128)(((unsigned __int128)hi << 64) | lo);
}

// v 2^{-sh} for v >= 0, truncated; sh >= 0.
__device__ __forceinline__ i128 shr_i128(i128 v, int sh) { return sh >= 127 ? (i128)0 : (v >> sh); }

// Warp 0, after pass 1: the fixed-point mass of each owned tile relative to
// the CTA's largest exponent k_c (kept for the boundaries), and the CTA record
// (written by lane 0, before its arrival).  Returns k_c (INT_MIN: no mass).
__device__ int publish_cta_record(const SortedParams& p, PersistShared& sm, int t_count) {
    const int lane = threadIdx.x & 31;
    int kc = INT_MIN;
    uint32_t bad = 0;
    for (int r = lane; r < t_count; r += 32) {
        const float sh = sm.own_shi[r];
        bad |= !(sh <= 3.402823466e38f);
        if (sh > 0.f) kc = max(kc, sm.own_k[r]);
    }
    kc = warp_max_i(kc);
    bad = __any_sync(0xffffffffu, bad);
    i128 a = 0;
    if (kc != INT_MIN && !bad)
        for (int r = lane; r < t_count; r += 32)
            if (sm.own_shi[r] > 0.f) {
                const int sh = sm.own_k[r] - kc;
                a += fixed_of(sm.own_shi[r], sh) + fixed_of(sm.own_slo[r], sh);
            }
    a = warp_sum_i128(a);
    if (lane == 0) {
        uint32_t* rec = reinterpret_cast<uint32_t*>(p.slots) + 8 * blockIdx.x;
        const unsigned __int128 u = (unsigned __int128)a;
        st_v4_u32(rec, (uint32_t)kc, (bad ? kRecBad : 0u) | (kc != INT_MIN ? kRecMass : 0u), 0u, 0u);
        st_v4_u32(rec + 4, (uint32_t)u, (uint32_t)(u >> 32), (uint32_t)(u >> 64), (uint32_t)(u >> 96));
    }
    return kc;
}

// Block-wide, after every CTA arrived: K, W and this CTA's tile boundaries
// sm.Bown[0 .. t_count] (in units of 2^-90 relative to 2^K) from the G CTA
// records (one per thread, all loaded at once) and the owned tiles' sums.
// Tile t's upper boundary is its successor's lower one, also across CTAs
// (both are B_c plus the same truncated sum), and the last tile's is W.
// kc: the CTA's own exponent (needed in warp 0 only).  Returns false (and
// records PF_ERR_DOMAIN) for NaN/+inf or all-zero weights.
__device__ bool carries_agg(const SortedParams& p, PersistShared& sm, int t_count, int kc) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, G = gridDim.x;
    const uint32_t* rec = reinterpret_cast<const uint32_t*>(p.slots);
    uint4 h = make_uint4(0, 0, 0, 0), sw = make_uint4(0, 0, 0, 0);
    if (tid < G) {  // G <= kThreads: one record per thread
        h = __ldcg(reinterpret_cast<const uint4*>(rec + 8 * tid));
        sw = __ldcg(reinterpret_cast<const uint4*>(rec + 8 * tid + 4));
    }
    // largest exponent with mass, and the domain check
    const int bad = __syncthreads_or((int)(h.y & kRecBad));
    const int Kw = __reduce_max_sync(0xffffffffu, (h.y & kRecMass) ? (int)h.x : INT_MIN);
    if (lane == 0) sm.red_k[warp] = Kw;
    __syncthreads();
    const int K = __reduce_max_sync(0xffffffffu, lane < kWarps ? sm.red_k[lane] : INT_MIN);
    if (K == INT_MIN || bad) {
        if (tid == 0) set_status(p.ctl + CTL_STATUS, ST_DOMAIN);
        return false;
    }
    // the masses below this CTA and of all CTAs, relative to 2^K
    const i128 v = (h.y & kRecMass) ? shr_i128(i128_of(sw), K - (int)h.x) : (i128)0;
    const i128 below_w = warp_sum_i128(tid < (int)blockIdx.x ? v : (i128)0);
    const i128 all_w = warp_sum_i128(v);
    if (lane == 0) {
        sm.wsum[warp] = below_w;
        sm.wsum2[warp] = all_w;
    }
    __syncthreads();
    if (warp == 0) {
        const i128 below = warp_sum_i128(lane < kWarps ? sm.wsum[lane] : (i128)0);
        const i128 all = warp_sum_i128(lane < kWarps ? sm.wsum2[lane] : (i128)0);
        // the owned tiles: exclusive prefix of their fixed-point masses, then shifted to 2^K
        const int shc = kc == INT_MIN ? 0 : K - kc;
        i128 run = 0;
        for (int r0 = 0; r0 <= t_count; r0 += 32) {
            const int r = r0 + lane;
            i128 a = 0;
            if (r < t_count && kc != INT_MIN && sm.own_shi[r] > 0.f) {
                const int sh = sm.own_k[r] - kc;
                a = fixed_of(sm.own_shi[r], sh) + fixed_of(sm.own_slo[r], sh);
            }
            const i128 inc = warp_scan_i128(a, lane);
            if (r <= t_count) sm.Bown[r] = below + shr_i128(run + inc - a, shc);
            run += shfl_i128(inc, 31);
        }
        if (lane == 0) {
            sm.as.K = K;
            sm.as.Wt = all;
            const fpair Wp = fixed_to_pair(all);
            sm.as.W_hi = Wp.hi;
            sm.as.W_lo = Wp.lo;
        }
    }
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------------------
// Multinomial draws (Figure 1a): binary searches in global units.
// ---------------------------------------------------------------------------
// GUIDE: draws through the guide table first (p.g_out set), else the
// three-level search alone.
template <bool GUIDE>
__device__ void multinomial_draws(const SortedParams& p, PersistShared& sm, const TableEntry* table) {
    const int tid = threadIdx.x, cta = blockIdx.x, G = gridDim.x;
    const int T = p.n_tiles;
    const float Wh = sm.as.W_hi, Wl = sm.as.W_lo;
    const int64_t nq = (p.P + 3) >> 2;  // four draws per Philox block
    const int64_t q_beg = nq * cta / G, q_end = nq * (cta + 1) / G;
    // the tile lookup, then the level-1 samples of every tile (published before the arrival)
    int* lut = reinterpret_cast<int*>(const_cast<TableEntry*>(table) + T);
    float* c1 = reinterpret_cast<float*>(lut + kLut + 1);
    if (p.c2_out) {
        const int nc = T * p.cpt1;
        for (int i = tid; i < nc; i += kThreads) c1[i] = __ldcg(p.c1_out + i);
        build_tile_lut(table, T, Wh, Wl, lut, sm.red_k);
    }
    // the loop runs the same number of times in every thread: the three-level
    // draws read their windows quad-cooperatively across the warp
    for (int64_t q0 = q_beg; q0 < q_end; q0 += kThreads) {
        const int64_t q = q0 + tid < q_end ? q0 + tid : q_beg;  // a lane past the end redraws block q_beg
        const bool mine = q0 + tid < q_end;
        if (!__any_sync(0xffffffffu, mine)) continue;  // the whole warp is past the end
        const u32x4 r = philox((uint32_t)q, 0u, p.filter, TAG_MULTI, p.key0, p.key1);
        int32_t a[4];
        if (p.c2_out) {
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                if (GUIDE) {
                    bool ok;
                    a[s] = multinomial_draw_guided(word_of(r, s), table, T, p.v_out, p.g_out, p.M, p.tile,
                                                   p.P + p.lead, p.lead, Wh, Wl, ok);
                    if (__any_sync(0xffffffffu, !ok)) {  // the three-level draw, for the lanes the guide did not settle
                        const int32_t f = multinomial_draw_3level(word_of(r, s), table, lut, T, p.v_out, p.c2_out,
                                                                  p.cpt2, c1, p.cpt1, p.c1shift, p.tile, p.P + p.lead,
                                                                  p.lead, Wh, Wl);
                        if (!ok) a[s] = f;
                    }
                } else {
                    a[s] = multinomial_draw_3level(word_of(r, s), table, lut, T, p.v_out, p.c2_out, p.cpt2, c1,
                                                   p.cpt1, p.c1shift, p.tile, p.P + p.lead, p.lead, Wh, Wl);
                }
            }
        } else {
            multinomial_draws4<false>(r, table, T, p.v_out, p.tile, p.P + p.lead, p.lead, Wh, Wl, a);
        }
        const int64_t j = 4 * q;
        if (!mine) continue;
        if (j + 3 < p.P && (((uintptr_t)(p.anc + j)) & 15u) == 0) {
            // streaming store: the ancestors are not read again here, and evicting
            // them first keeps L2 for the cumulative weights the draws read at random
            __stcs(reinterpret_cast<int4*>(p.anc + j), make_int4(a[0], a[1], a[2], a[3]));
        } else {
            for (int s = 0; s < 4; ++s)
                if (j + s < p.P) __stcs(p.anc + j + s, a[s]);
        }
    }
}

// ---------------------------------------------------------------------------
// Multinomial guide table (after the carries): g[b], b < M, the first particle
// whose cumulative weight exceeds the bucket edge (b / M) W.  It is the
// systematic assignment of M offsets at (j / M) W (no uniform shift) over the
// owned tiles, decoded into g with its staging in the tile lookup's area (not
// yet built); then a second grid-wide arrival, so that every entry is written
// before any draw reads one.  Returns false when that wait ran out.
// ---------------------------------------------------------------------------
constexpr int kGuideCap = 2048;  // staging entries per buffer: offsets per chunk + room for the shift
static_assert(2 * kGuideCap <= kLut + 1, "the guide's staging fits the tile lookup's area");

template <int KK>
__device__ bool build_guide(const SortedParams& p, PersistShared& sm, int32_t* stage, TileThread& th, TileSummary ts,
                            int t_first, int t_count, uint32_t epoch, uint64_t t_start, bool skip) {
    const int tid = threadIdx.x;
    SortedParams pg = p;
    pg.anc = p.g_out;
    pg.P = p.M;
    pg.Pd = (double)p.M;
    pg.guide = 1;
    stage_init<kGuideCap>(stage);
    // the guide's offset map of every owned tile, two lanes per tile
    if (tid < 2 * ((t_count + 15) & ~15)) {
        const int r = min(tid >> 1, t_count - 1);
        const TileMap m = tile_map_pair<KIND_SYS>(pg, sm.as, sm.Bown[r], sm.Bown[r + 1], sm.own_k[r], 0xffffffffu);
        if ((tid & 1) == 0 && (tid >> 1) < t_count) sm.own_map[tid >> 1] = m;
    }
    __syncthreads();
    const int64_t PA = p.P + p.lead;
    uint32_t chunks = 0;
    for (int r = t_count - 1; r >= 0; --r) {  // the last tile's scan is still in registers
        const int64_t t0 = (int64_t)(t_first + r) * p.tile;
        if (r != t_count - 1) {
            read_tile_v<KK>(p.v_out + t0, (int)min((int64_t)p.tile, PA - t0), th);
            ts.i_last = sm.own_il[r];
        }
        assign_offspring<KIND_SYS, KK, kGuideCap>(pg, sm.as, sm.own_map[r], stage, chunks, th, ts, t0 - p.lead);
    }
    __threadfence();
    __syncthreads();
    return arrive_and_wait(p, sm, skip, epoch, t_start, CTL_ARRIVE2);
}

// KK: elements per thread of a full tile (4, 8 or 16; the host picks it from p.tile).
// GUIDE (multinomial): draws through the guide table (p.g_out set).
template <int KIND, int KK, bool GUIDE = false>
__global__ void __launch_bounds__(kThreads, 2) k_persistent(SortedParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PersistShared& sm = *reinterpret_cast<PersistShared*>(smem_raw);
    unsigned char* region = smem_raw + sizeof(PersistShared);
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint64_t t_start = global_ns();
    const uint32_t epoch = ld_relaxed_u32(p.ctl + CTL_EPOCH) + 1u;
    const int R = p.tiles_per_cta > 0 ? p.tiles_per_cta : 1;
    const int t_first = blockIdx.x * R;
    const int t_count = max(0, min(R, p.n_tiles - t_first));
    uint32_t* rec = reinterpret_cast<uint32_t*>(p.slots);
    if (p.trace) {
        trace_put(p.trace, p.trace_cap, blockIdx.x, 0, t_start);
        for (int w = 1; w <= 4; ++w) trace_put(p.trace, p.trace_cap, blockIdx.x, w, 0);
        trace_put(p.trace, p.trace_cap, blockIdx.x, 5, blockIdx.x);
        trace_put(p.trace, p.trace_cap, blockIdx.x, 6, 0);
        trace_put(p.trace, p.trace_cap, blockIdx.x, 7, (uint64_t)t_count);
    }

    static_assert(sizeof(PersistShared) % 16 == 0, "the staging buffers are 16-byte aligned");
    // the staging buffers start pass 2 at -1 (below every decode tag); with tile
    // copies in pass 1 they are set after it
    if (KIND != KIND_MULTI && t_count <= 1) stage_init<stage_cap(KK)>(reinterpret_cast<int32_t*>(region));

    // pass 1: scan and record every owned tile.  Systematic / stratified with
    // several tiles per CTA: tile r + 1 is bulk-copied into one of the two
    // staging buffers (idle until pass 2) while tile r is scanned from the other.
    TileThread th;
    TileSummary ts;
    ts.k = 0;
    ts.i_last = -1;
    bool skip = false;
    const int64_t PA = p.P + p.lead;  // length of the aligned window
    constexpr bool kCopies = KIND != KIND_MULTI;
    const bool copies = kCopies && t_count > 1;  // uniform over the CTA
    float* slot = reinterpret_cast<float*>(region);
    constexpr int kSlotFloats = stage_cap(KK);  // floats per staging buffer (>= the tile)
    auto issue = [&](int r) {  // thread 0: the copy of owned tile r (its whole 16-byte pieces)
        const int64_t t0 = (int64_t)(t_first + r) * p.tile;
        const uint32_t bytes = (uint32_t)((int)min((int64_t)p.tile, PA - t0) & ~3) * 4u;
        if (bytes) bulk_load(slot + (r & 1) * kSlotFloats, p.lw + t0, bytes, &sm.bar[r & 1]);
        else mbar_arrive(&sm.bar[r & 1]);
    };
    bool copy_ok = true;
    if (kCopies && copies) {
        if (tid == 0) {
            mbar_init(&sm.bar[0], 1);
            mbar_init(&sm.bar[1], 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (tid == 0) issue(0);
    }
    for (int r = 0; r < t_count; ++r) {
        const int t = t_first + r;
        const int64_t t0 = (int64_t)t * p.tile;
        const int n = (int)min((int64_t)p.tile, PA - t0);
        if (kCopies && copies) {
            if (tid == 0 && r + 1 < t_count) issue(r + 1);
            if (!mbar_wait(&sm.bar[r & 1], (uint32_t)(r >> 1) & 1u, t_start, p.wait_ns)) {
                copy_ok = false;  // a copy that never completed: reported, and this CTA stops after the wait
                if (tid == 0) set_status(p.ctl + CTL_STATUS, ST_TIMEOUT);
            }
            const float* sl = slot + (r & 1) * kSlotFloats;
            if ((n & 3) == 0) {
                ts = tile_scan_k<KK, true>(sl, t == 0 ? p.lead : 0, n, sm.tile, th);
            } else {  // a ragged last tile: its tail is not in the copy; read it from global memory
                ts = tile_scan_k<KK>(p.lw + t0, t == 0 ? p.lead : 0, n, sm.tile, th);
            }
        } else {
            ts = tile_scan_k<KK>(p.lw + t0, t == 0 ? p.lead : 0, n, sm.tile, th);
        }
        if (ts.bad && tid == 0) set_status(p.ctl + CTL_STATUS, ST_DOMAIN);
        skip |= (t == p.skip_tile);
        if (KIND == KIND_MULTI) {
            write_tile_v<KK>(p, th, t0, n);
            if (p.c2_out)
                write_tile_samples<KK>(th, n, p.c2_out + (int64_t)t * p.cpt2, p.c1_out + (int64_t)t * p.cpt1, p.c1shift);
            __threadfence();
            if (tid == 0) {
                st_v4_u32(rec + 4 * t, (uint32_t)ts.k, __float_as_uint(ts.bad ? NAN : ts.S.hi),
                          __float_as_uint(ts.S.lo), (uint32_t)ts.i_last);
                sm.own_k[r] = ts.k;
                sm.own_il[r] = ts.i_last;
            }
        } else {
            if (r + 1 < t_count) write_tile_v<KK>(p, th, t0, n);  // reloaded in pass 2
            if (tid == 0) {
                sm.own_k[r] = ts.k;
                sm.own_il[r] = ts.i_last;
                sm.own_shi[r] = ts.bad ? NAN : ts.S.hi;
                sm.own_slo[r] = ts.S.lo;
            }
            if (kCopies && copies) fence_proxy_async_smem();  // this tile's reads before the buffer's next copy
        }
        __syncthreads();
    }
    copy_ok = __syncthreads_and(copy_ok);
    if (kCopies && copies && copy_ok) stage_init<stage_cap(KK)>(reinterpret_cast<int32_t*>(region));  // pass 2's tags
    int kc = 0;
    if (KIND != KIND_MULTI && warp == 0) kc = publish_cta_record(p, sm, t_count);

    trace_stamp(p.trace, p.trace_cap, blockIdx.x, 1);
    bool ok = arrive_and_wait(p, sm, skip, epoch, t_start);
    trace_stamp(p.trace, p.trace_cap, blockIdx.x, 2);
    if (!ok && tid == 0) set_status(p.ctl + CTL_STATUS, ST_TIMEOUT);
    if (ok) {
        if (KIND == KIND_MULTI) {
            ok = carries<KIND>(p, sm, reinterpret_cast<TableEntry*>(region), t_first, t_count);
        } else {
            ok = carries_agg(p, sm, t_count, kc);
        }
    }
    if (ok) trace_stamp(p.trace, p.trace_cap, blockIdx.x, 3);
    // every CTA read the epoch before arriving, and CTA 0 has seen all arrivals
    // (or waited out its limit): reset the counter the next launch will use and
    // advance the epoch
    if (blockIdx.x == 0 && tid == 0) {
        // every kind resets both pairs: the next launch on this stream, of whatever
        // kind, may be a multinomial one that uses the second pair
        atomicExch(p.ctl + CTL_ARRIVE0 + ((epoch + 1u) & 1u), 0u);
        atomicExch(p.ctl + CTL_ARRIVE2 + ((epoch + 1u) & 1u), 0u);
        atomicExch(p.ctl + CTL_EPOCH, epoch);
    }
    if (!ok || !copy_ok) return;

    if (KIND == KIND_MULTI) {
        if (GUIDE) {
            int32_t* stage = reinterpret_cast<int32_t*>(region + (size_t)p.n_tiles * sizeof(TableEntry));
            if (!build_guide<KK>(p, sm, stage, th, ts, t_first, t_count, epoch, t_start, skip)) {
                if (tid == 0) set_status(p.ctl + CTL_STATUS, ST_TIMEOUT);
                return;
            }
        }
        multinomial_draws<GUIDE>(p, sm, reinterpret_cast<const TableEntry*>(region));
        if (p.trace) {
            __syncthreads();
            trace_stamp(p.trace, p.trace_cap, blockIdx.x, 4);
        }
        return;
    }
    // the offset maps of every owned tile at once, two lanes per tile
    if (tid < 2 * ((t_count + 15) & ~15)) {
        const int r = min(tid >> 1, t_count - 1);
        const TileMap m = tile_map_pair<KIND>(p, sm.as, sm.Bown[r], sm.Bown[r + 1], sm.own_k[r], 0xffffffffu);
        if ((tid & 1) == 0 && (tid >> 1) < t_count) sm.own_map[tid >> 1] = m;
    }
    __syncthreads();
    // pass 2: offsets of every owned tile (the last tile's scan is still in
    // registers; the others reload their cumulative weights)
    int32_t* stage = reinterpret_cast<int32_t*>(region);
    uint32_t chunks = 0;  // staging chunks decoded by this CTA
    for (int r = t_count - 1; r >= 0; --r) {
        const int t = t_first + r;
        const int64_t t0 = (int64_t)t * p.tile;
        if (r != t_count - 1) {
            read_tile_v<KK>(p.v_out + t0, (int)min((int64_t)p.tile, PA - t0), th);
            ts.i_last = sm.own_il[r];
        }
        assign_offspring<KIND, KK, stage_cap(KK)>(p, sm.as, sm.own_map[r], stage, chunks, th, ts, t0 - p.lead);
    }
    if (p.trace) {
        __syncthreads();
        trace_stamp(p.trace, p.trace_cap, blockIdx.x, 4);
    }
}

template <int KIND, int KK, bool GUIDE = false>
static cudaError_t set_smem_attr() {
    return cudaFuncSetAttribute(k_persistent<KIND, KK, GUIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)persistent_smem_bytes(KIND, kMaxTilesTotal, KK));
}

template <int KIND, int KK, bool GUIDE = false>
static cudaError_t launch_kind(const SortedParams& p, int grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes =
        persistent_smem_bytes(KIND, p.n_tiles, KK) + (p.c2_out ? (size_t)p.n_tiles * p.cpt1 * sizeof(float) : 0);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_persistent<KIND, KK, GUIDE>, p);
}

template <int KIND>
static cudaError_t launch_k(const SortedParams& p, int grid, cudaStream_t s) {
    const int q = (p.tile + kThreads - 1) / kThreads;  // elements per thread of a full tile
    if (KIND == KIND_MULTI && p.g_out) {
        if (q <= 4) return launch_kind<KIND, 4, true>(p, grid, s);
        if (q <= 8) return launch_kind<KIND, 8, true>(p, grid, s);
        return launch_kind<KIND, 16, true>(p, grid, s);
    }
    if (q <= 4) return launch_kind<KIND, 4>(p, grid, s);
    if (q <= 8) return launch_kind<KIND, 8>(p, grid, s);
    return launch_kind<KIND, 16>(p, grid, s);
}

cudaError_t launch_sorted_persistent(int kind, const SortedParams& p, int grid, cudaStream_t s) {
    const int R = p.tiles_per_cta > 0 ? p.tiles_per_cta : 1;
    if (p.n_tiles < 1 || p.n_tiles > kMaxTilesTotal || R > kMaxOwn || (int64_t)grid * R < p.n_tiles ||
        p.tile < 4 || p.tile > kTileMax)
        return cudaErrorInvalidValue;
    switch (kind) {
    case KIND_MULTI: return launch_k<KIND_MULTI>(p, grid, s);
    case KIND_STRAT: return launch_k<KIND_STRAT>(p, grid, s);
    case KIND_SYS: return launch_k<KIND_SYS>(p, grid, s);
    }
    return cudaErrorInvalidValue;
}

// Resident CTAs per SM of kind's kernels at the largest shared-memory size a
// launch may ask for (the smallest over the three per-thread widths; raises
// their dynamic shared memory limits on the way).  Called once per device.
template <int KIND, int KK>
static int blocks_per_sm_kk() {
    int nb = 0;
    if (set_smem_attr<KIND, KK>() != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_persistent<KIND, KK>, kThreads,
                                                      persistent_smem_bytes(KIND, kMaxTilesTotal, KK)) != cudaSuccess)
        return 0;
    if (KIND == KIND_MULTI) {  // the guide variant: the same launch shape, so the smaller of the two
        int ng = 0;
        if (set_smem_attr<KIND, KK, true>() != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ng, k_persistent<KIND, KK, true>, kThreads,
                                                          persistent_smem_bytes(KIND, kMaxTilesTotal, KK)) !=
                cudaSuccess)
            return 0;
        nb = min(nb, ng);
    }
    return nb;
}

template <int KIND>
static int blocks_per_sm_kind() {
    return min(blocks_per_sm_kk<KIND, 4>(), min(blocks_per_sm_kk<KIND, 8>(), blocks_per_sm_kk<KIND, 16>()));
}

int persistent_blocks_per_sm(int kind) {
    switch (kind) {
    case KIND_MULTI: return blocks_per_sm_kind<KIND_MULTI>();
    case KIND_STRAT: return blocks_per_sm_kind<KIND_STRAT>();
    case KIND_SYS: return blocks_per_sm_kind<KIND_SYS>();
    }
    return 0;
}

}  // namespace pf
