// Single filters beyond the tiles of one cooperative launch: the cumulative
// schemes (Section 2, Figure 1a-c) for P + lead > PF_MAX_CUMULATIVE, up to
// 2^31 - 1 particles.  Three ordinary launches in stream order, with no wait of
// one CTA on another:
//   1. k_large_scan: tiles of 8192 log-weights, grid-stride, each bulk-copied
//      into shared memory while the CTA's previous tile is scanned: the tile
//      scan (pf_tile.cuh), a 16-byte record (k_t, S_t, i_last) and the tile's
//      cumulative weights v_i (sign bit: zero weight);
//   2. k_large_carries: one CTA: the largest tile exponent K and the exact
//      exclusive prefix B_t = sum_{t' < t} S_t' 2^{k_t' - K} of every tile
//      (128-bit fixed point; each thread a contiguous run of records, then one
//      block scan of the run totals), W = B_T, and the multinomial's tile table;
//   3. k_large_assign (systematic, stratified): grid-stride over tiles: the
//      tile's v_i read back (not rescanned: 6-7% faster at 2^25 - 2^27 for the
//      extra 4 B written and read per particle; bulk-copied into shared memory
//      while the previous tile is assigned), the tile's offset map from B_t and
//      B_{t+1}, the offsets and their run-length decode (pf_assign.cuh).
//      Multinomial: k_large_guide decodes the guide table (the first particle
//      above each of P/4 evenly spaced targets) from the stored v_i, then
//      k_large_draws runs the draws, each through its guide entry and one
//      window of v_i, or, where that does not settle it, by binary searches over
//      the tile table and the tile's v_i.
// The tiles, the exact boundaries and the per-tile arithmetic are those of the
// single-launch kernels, so the results follow the same rules.  A NaN/+inf or
// all-zero weight set records PF_ERR_DOMAIN in launch 1 or 2, and launch 3
// then writes nothing.
#include <cfloat>
#include <climits>

#include "pf_assign.cuh"

namespace pf {

namespace {

// What launch 2 hands to launch 3 (global memory).
struct LargeScalars {
    i128 Wt;  // W in fixed point (units of 2^K)
    int K;    // largest tile exponent with weight
    int ok;   // 0: a domain error was recorded, launch 3 writes nothing
    float W_hi, W_lo;
};

struct LargeShared {
    AssignShared as;
    TileMap map;
    uint64_t bar;  // the assignment's tile copies
};
static_assert(sizeof(LargeShared) % 16 == 0, "the staging buffers are 16-byte aligned");

constexpr int kLargeTile = kTileMax;  // full tiles, 16 log-weights per thread

__device__ __forceinline__ i128 record_mass(uint4 r, int K) {
    const float sh = __uint_as_float(r.y);
    if (!(sh > 0.f)) return (i128)0;
    const int s = (int)r.x - K;
    return fixed_of(sh, s) + fixed_of(__uint_as_float(r.z), s);
}

// ---------------------------------------------------------------------------
// Launch 1: the tile scans.  A CTA's tiles are t = blockIdx.x + r gridDim.x;
// tile r + 1 is bulk-copied into one of two shared-memory buffers while tile r
// is scanned from the other.
// ---------------------------------------------------------------------------
struct ScanShared {
    TileShared tile;
    uint64_t bar[2];
};
constexpr size_t kScanSmem = ((sizeof(ScanShared) + 15) & ~(size_t)15) + 2 * (size_t)kLargeTile * sizeof(float);

// Thread 0: the copy of this CTA's tile r (its whole 16-byte pieces) into buf,
// completing on bar.
__device__ __forceinline__ void issue_tile_copy(const float* src, int64_t PA, int r, float* buf, uint64_t* bar) {
    const int64_t t0 = (int64_t)(blockIdx.x + (int64_t)r * gridDim.x) * kLargeTile;
    const uint32_t bytes = (uint32_t)((int)min((int64_t)kLargeTile, PA - t0) & ~3) * 4u;
    if (bytes) bulk_load(buf, src + t0, bytes, bar);
    else mbar_arrive(bar);
}

template <int KIND>
__global__ void __launch_bounds__(kThreads, 2) k_large_scan(SortedParams p, uint4* rec) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ScanShared& sm = *reinterpret_cast<ScanShared*>(smem_raw);
    float* slot = reinterpret_cast<float*>(smem_raw + ((sizeof(ScanShared) + 15) & ~(size_t)15));
    const int tid = threadIdx.x;
    const int64_t PA = p.P + p.lead;
    const int n_mine = (p.n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;  // grid <= tiles
    if (tid == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) issue_tile_copy(p.lw, PA, 0, slot, &sm.bar[0]);
    TileThread th;
    for (int r = 0; r < n_mine; ++r) {
        const int t = (int)blockIdx.x + r * (int)gridDim.x;
        const int64_t t0 = (int64_t)t * kLargeTile;
        const int n = (int)min((int64_t)kLargeTile, PA - t0);
        if (tid == 0 && r + 1 < n_mine)
            issue_tile_copy(p.lw, PA, r + 1, slot + ((r + 1) & 1) * kLargeTile, &sm.bar[(r + 1) & 1]);
        // a copy not complete within the wait limit (from this wait's start) is
        // reported; the results are then unspecified
        if (!mbar_wait(&sm.bar[r & 1], (uint32_t)(r >> 1) & 1u, global_ns(), p.wait_ns) && tid == 0)
            set_status(p.ctl + CTL_STATUS, ST_TIMEOUT);
        // a ragged last tile: its tail is not in the copy; read it from global memory
        const int lo = t == 0 ? p.lead : 0;
        const TileSummary ts = (n & 3) == 0 ? tile_scan_k<16, true>(slot + (r & 1) * kLargeTile, lo, n, sm.tile, th)
                                            : tile_scan_k<16>(p.lw + t0, lo, n, sm.tile, th);
        if (ts.bad && tid == 0) set_status(p.ctl + CTL_STATUS, ST_DOMAIN);
        write_tile_v<16>(p, th, t0, n);  // read back by launch 3
        if (tid == 0)
            rec[t] = make_uint4((uint32_t)ts.k, __float_as_uint(ts.bad ? NAN : ts.S.hi), __float_as_uint(ts.S.lo),
                                (uint32_t)ts.i_last);
        fence_proxy_async_smem();  // this tile's reads of its buffer before the buffer's next copy
        __syncthreads();           // and the tile scan's shared fields are reused by the next tile
    }
}

// ---------------------------------------------------------------------------
// Launch 2: one CTA forms K, every tile's exact lower boundary B_t (bnd[0..T],
// bnd[T] = W) and, for the multinomial, the tile table the draws search.
// ---------------------------------------------------------------------------
template <int KIND>
__global__ void __launch_bounds__(kThreads) k_large_carries(SortedParams p, const uint4* rec, i128* bnd,
                                                            TableEntry* table, LargeScalars* out) {
    __shared__ int red[kWarps];
    __shared__ i128 wsum[kWarps];
    __shared__ i128 total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = p.n_tiles;
    // the largest exponent among tiles with weight, and the domain check
    int kmax = INT_MIN, bad = 0;
    for (int t = tid; t < T; t += kThreads) {
        const uint4 r = rec[t];
        const float sh = __uint_as_float(r.y);
        bad |= !(sh <= FLT_MAX);
        if (sh > 0.f) kmax = max(kmax, (int)r.x);
    }
    kmax = warp_max_i(kmax);
    if (lane == 0) red[warp] = kmax;
    bad = __syncthreads_or(bad);
    int K = INT_MIN;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) K = max(K, red[w]);
    if (K == INT_MIN || bad) {
        if (tid == 0) {
            set_status(p.ctl + CTL_STATUS, ST_DOMAIN);
            out->ok = 0;
        }
        return;
    }
    // each thread a contiguous run [t_lo, t_hi) of records, read eight at a time
    const int per = (T + kThreads - 1) / kThreads;
    const int t_lo = min(T, tid * per), t_hi = min(T, t_lo + per);
    i128 run = 0;
    for (int t0 = t_lo; t0 < t_hi; t0 += 8) {
        uint4 r[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) r[u] = t0 + u < t_hi ? rec[t0 + u] : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int u = 0; u < 8; ++u) run += record_mass(r[u], K);
    }
    // exclusive block scan of the run totals (integer sums: exact in any order)
    const i128 inc = warp_scan_i128(run, lane);
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const i128 v = lane < kWarps ? wsum[lane] : (i128)0;
        const i128 vi = warp_scan_i128(v, lane);
        if (lane < kWarps) wsum[lane] = vi - v;
        if (lane == kWarps - 1) total = vi;
    }
    __syncthreads();
    i128 B = wsum[warp] + inc - run;  // the boundary of tile t_lo
    for (int t0 = t_lo; t0 < t_hi; t0 += 8) {
        uint4 r[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) r[u] = t0 + u < t_hi ? rec[t0 + u] : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (t0 + u < t_hi) {
                bnd[t0 + u] = B;
                if (KIND == KIND_MULTI) {
                    const fpair b = fixed_to_pair(B);
                    table[t0 + u] = {b.hi, b.lo, pow2f(K - (int)r[u].x), (int)r[u].w};
                }
                B += record_mass(r[u], K);
            }
        }
    }
    if (tid == 0) {
        bnd[T] = total;
        const fpair Wp = fixed_to_pair(total);
        out->Wt = total;
        out->K = K;
        out->W_hi = Wp.hi;
        out->W_lo = Wp.lo;
        out->ok = 1;
    }
}

// ---------------------------------------------------------------------------
// Launch 3, systematic / stratified: each tile's stored cumulative weights and
// record read back, its offset map from its two boundaries (the same function
// of a boundary for both ends, so neighbouring tiles share their end exactly),
// then its offsets decoded.
// ---------------------------------------------------------------------------
template <int KIND>
__global__ void __launch_bounds__(kThreads, 2) k_large_assign(SortedParams p, const uint4* rec, const i128* bnd,
                                                              const LargeScalars* sc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LargeShared& sm = *reinterpret_cast<LargeShared*>(smem_raw);
    int32_t* stage = reinterpret_cast<int32_t*>(smem_raw + sizeof(LargeShared));
    float* vbuf = reinterpret_cast<float*>(stage + 2 * kIoCap);  // one tile's stored cumulative weights
    const int tid = threadIdx.x;
    if (!sc->ok) return;  // launch 2 recorded a domain error
    const int64_t PA = p.P + p.lead;
    const int n_mine = (p.n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;  // grid <= tiles
    if (tid == 0) {
        sm.as.Wt = sc->Wt;
        sm.as.K = sc->K;
        sm.as.W_hi = sc->W_hi;
        sm.as.W_lo = sc->W_lo;
        mbar_init(&sm.bar, 1);
        fence_mbar_init();
    }
    stage_init<kIoCap>(stage);
    __syncthreads();
    // tile r + 1's copy is issued once every thread has taken tile r out of the
    // buffer, and lands while tile r is assigned
    if (tid == 0) issue_tile_copy(p.v_out, PA, 0, vbuf, &sm.bar);
    uint32_t chunks = 0;  // staging chunks decoded by this CTA
    TileThread th;
    for (int r = 0; r < n_mine; ++r) {
        const int t = (int)blockIdx.x + r * (int)gridDim.x;
        const int64_t t0 = (int64_t)t * kLargeTile;
        const int n = (int)min((int64_t)kLargeTile, PA - t0);
        // bounded from this wait's start; the results are then unspecified
        if (!mbar_wait(&sm.bar, (uint32_t)r & 1u, global_ns(), p.wait_ns) && tid == 0)
            set_status(p.ctl + CTL_STATUS, ST_TIMEOUT);
        // a ragged last tile: its tail is not in the copy; read it from global memory
        if ((n & 3) == 0) read_tile_v<16, true>(vbuf, n, th);
        else read_tile_v<16>(p.v_out + t0, n, th);
        const uint4 rc = rec[t];
        TileSummary ts;
        ts.k = (int)rc.x;
        ts.i_last = (int)rc.w;
        ts.bad = 0;
        ts.S = {__uint_as_float(rc.y), __uint_as_float(rc.z)};
        if (tid < 32) {  // lanes 0 and 1 form the map (the other pairs of warp 0 the same one)
            const TileMap m = tile_map_pair<KIND>(p, sm.as, bnd[t], bnd[t + 1], ts.k, 0xffffffffu);
            if (tid == 0) sm.map = m;
        }
        fence_proxy_async_smem();  // this thread's reads of the buffer before its next copy
        __syncthreads();
        if (tid == 0 && r + 1 < n_mine) issue_tile_copy(p.v_out, PA, r + 1, vbuf, &sm.bar);
        assign_offspring<KIND, 16, kIoCap>(p, sm.as, sm.map, stage, chunks, th, ts, t0 - p.lead);
        __syncthreads();  // the map is reused by the next tile
    }
}

// ---------------------------------------------------------------------------
// Multinomial, between launches 2 and 3: the guide table g[b], b < M = P / 4,
// the first particle whose cumulative weight exceeds the bucket edge
// (b / M) W -- the systematic assignment of M offsets with no uniform shift,
// from each tile's stored cumulative weights (pg: the call's parameters with
// anc = g, P = M, guide = 1; PA the call's P + lead).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 2) k_large_guide(SortedParams pg, int64_t PA, const uint4* rec,
                                                             const i128* bnd, const LargeScalars* sc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LargeShared& sm = *reinterpret_cast<LargeShared*>(smem_raw);
    int32_t* stage = reinterpret_cast<int32_t*>(smem_raw + sizeof(LargeShared));
    const int tid = threadIdx.x;
    if (!sc->ok) return;
    if (tid == 0) {
        sm.as.Wt = sc->Wt;
        sm.as.K = sc->K;
        sm.as.W_hi = sc->W_hi;
        sm.as.W_lo = sc->W_lo;
    }
    stage_init<kIoCap>(stage);
    __syncthreads();
    uint32_t chunks = 0;
    TileThread th;
    for (int t = blockIdx.x; t < pg.n_tiles; t += gridDim.x) {
        const int64_t t0 = (int64_t)t * kLargeTile;
        const int n = (int)min((int64_t)kLargeTile, PA - t0);
        read_tile_v<16>(pg.v_out + t0, n, th);
        const uint4 r = rec[t];
        TileSummary ts;
        ts.k = (int)r.x;
        ts.i_last = (int)r.w;
        ts.bad = 0;
        ts.S = {__uint_as_float(r.y), __uint_as_float(r.z)};
        if (tid < 32) {
            const TileMap m = tile_map_pair<KIND_SYS>(pg, sm.as, bnd[t], bnd[t + 1], ts.k, 0xffffffffu);
            if (tid == 0) sm.map = m;
        }
        __syncthreads();
        assign_offspring<KIND_SYS, 16, kIoCap>(pg, sm.as, sm.map, stage, chunks, th, ts, t0 - pg.lead);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Launch 3, multinomial: every draw searches the tile table, then its tile's
// cumulative weights (the plain binary searches of Section 2's description,
// through L2).
// ---------------------------------------------------------------------------
// GUIDE: each draw first reads its guide entry and one 16-element window of v
// (quad-cooperatively, pf_assign.cuh); a lane whose four draws the guide did
// not all settle redoes its Philox block by the plain searches (same results).
template <bool GUIDE>
__global__ void __launch_bounds__(kThreads, 2) k_large_draws(SortedParams p, const TableEntry* table,
                                                             const LargeScalars* sc, const int32_t* g, int64_t M) {
    if (!sc->ok) return;
    const float Wh = sc->W_hi, Wl = sc->W_lo;
    const int64_t PA = p.P + p.lead;
    const int64_t nq = (p.P + 3) >> 2;  // four draws per Philox block
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    // the same number of passes in every thread of a CTA (the guided draws read their
    // windows quad-cooperatively); a lane past the end redraws block 0 and stores nothing
    for (int64_t q0 = (int64_t)blockIdx.x * kThreads; q0 < nq; q0 += stride) {
        const bool mine = q0 + threadIdx.x < nq;
        if (!__any_sync(0xffffffffu, mine)) continue;  // the whole warp is past the end
        const int64_t q = mine ? q0 + threadIdx.x : 0;
        const u32x4 r = philox((uint32_t)q, 0u, p.filter, TAG_MULTI, p.key0, p.key1);
        int32_t a[4];
        bool settled = false;
        if (GUIDE) {
            settled = true;
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                bool ok;
                a[s] = multinomial_draw_guided(word_of(r, s), table, p.n_tiles, p.v_out, g, M, kLargeTile, PA,
                                               p.lead, Wh, Wl, ok);
                settled = settled && ok;
            }
        }
        if (!settled) multinomial_draws4<false>(r, table, p.n_tiles, p.v_out, kLargeTile, PA, p.lead, Wh, Wl, a);
        if (!mine) continue;
        const int64_t j = 4 * q;
        if (j + 3 < p.P && (((uintptr_t)(p.anc + j)) & 15u) == 0) {
            __stcs(reinterpret_cast<int4*>(p.anc + j), make_int4(a[0], a[1], a[2], a[3]));
        } else {
            for (int s = 0; s < 4; ++s)
                if (j + s < p.P) __stcs(p.anc + j + s, a[s]);
        }
    }
}

}  // namespace

namespace {
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct LargeLayout {
    size_t rec, bnd, table, scalars, v, g, total;
};

// Multinomial guide buckets: a quarter of the particles.
int64_t guide_buckets(int64_t P) { return (P + 3) / 4; }

LargeLayout large_layout(int kind, int64_t PA) {
    const size_t T = (size_t)((PA + kLargeTile - 1) / kLargeTile);
    const bool multi = kind == KIND_MULTI;
    LargeLayout l;
    l.rec = 0;
    l.bnd = align256(T * sizeof(uint4));
    l.table = align256(l.bnd + (T + 1) * sizeof(i128));
    l.scalars = align256(l.table + (multi ? T * sizeof(TableEntry) : 0));
    l.v = align256(l.scalars + sizeof(LargeScalars));
    l.g = align256(l.v + (size_t)PA * sizeof(float));
    l.total = l.g + (multi ? (size_t)guide_buckets(PA) * sizeof(int32_t) : 0);
    return l;
}

constexpr size_t kGuideSmem = sizeof(LargeShared) + 2 * (size_t)kIoCap * sizeof(int32_t);
constexpr size_t kAssignSmem = kGuideSmem + (size_t)kLargeTile * sizeof(float);  // and one tile's copy

template <int KIND>
cudaError_t launch_large_kind(SortedParams p, unsigned char* scratch, int num_sms, cudaStream_t s) {
    const int64_t PA = p.P + p.lead;
    const LargeLayout l = large_layout(KIND, PA);
    const int T = p.n_tiles;
    uint4* rec = reinterpret_cast<uint4*>(scratch + l.rec);
    i128* bnd = reinterpret_cast<i128*>(scratch + l.bnd);
    TableEntry* table = reinterpret_cast<TableEntry*>(scratch + l.table);
    LargeScalars* sc = reinterpret_cast<LargeScalars*>(scratch + l.scalars);
    p.v_out = reinterpret_cast<float*>(scratch + l.v);
    const int grid = T < 2 * num_sms ? T : 2 * num_sms;  // two resident CTAs per SM, grid-stride over tiles
    k_large_scan<KIND><<<grid, kThreads, kScanSmem, s>>>(p, rec);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_large_carries<KIND><<<1, kThreads, 0, s>>>(p, rec, bnd, table, sc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if constexpr (KIND == KIND_MULTI) {
        // the guide table, then the draws through it
        int32_t* g = reinterpret_cast<int32_t*>(scratch + l.g);
        const int64_t M = guide_buckets(p.P);
        SortedParams pg = p;
        pg.anc = g;
        pg.P = M;
        pg.Pd = (double)M;
        pg.guide = 1;
        k_large_guide<<<grid, kThreads, kGuideSmem, s>>>(pg, PA, rec, bnd, sc);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const int64_t nq = (p.P + 3) >> 2;
        int64_t gd = (nq + kThreads - 1) / kThreads;
        if (gd > (int64_t)num_sms * 16) gd = (int64_t)num_sms * 16;
        k_large_draws<true><<<(unsigned)gd, kThreads, 0, s>>>(p, table, sc, g, M);
    } else {
        k_large_assign<KIND><<<grid, kThreads, kAssignSmem, s>>>(p, rec, bnd, sc);
    }
    return cudaGetLastError();
}
}  // namespace

// Once per device: the scans' tile buffers and the assignment kernels' staging
// buffers exceed the default dynamic shared-memory limit.
cudaError_t prepare_large() {
    cudaError_t e = cudaFuncSetAttribute(k_large_assign<KIND_SYS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kAssignSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_large_assign<KIND_STRAT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kAssignSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_large_guide, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGuideSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_large_scan<KIND_MULTI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScanSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_large_scan<KIND_STRAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScanSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_large_scan<KIND_SYS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScanSmem);
    return e;
}

size_t large_scratch_bytes(int kind, int64_t PA) { return large_layout(kind, PA).total; }

// p: the call's parameters with lw, anc, P, lead, keys, filter, ctl set; the
// tiles are set here.  scratch: large_scratch_bytes(kind, P + lead) bytes.
cudaError_t launch_large(int kind, SortedParams p, void* scratch, int num_sms, cudaStream_t s) {
    const int64_t PA = p.P + p.lead;
    const int64_t T = (PA + kLargeTile - 1) / kLargeTile;
    if (T < 1 || T > INT_MAX / 2 || num_sms < 1) return cudaErrorInvalidValue;
    p.tile = kLargeTile;
    p.n_tiles = (int)T;
    p.tiles_per_cta = 0;
    p.v_out = nullptr;
    p.c2_out = p.c1_out = nullptr;
    p.g_out = nullptr;
    p.guide = 0;
    unsigned char* sb = static_cast<unsigned char*>(scratch);
    switch (kind) {
    case KIND_MULTI: return launch_large_kind<KIND_MULTI>(p, sb, num_sms, s);
    case KIND_STRAT: return launch_large_kind<KIND_STRAT>(p, sb, num_sms, s);
    case KIND_SYS: return launch_large_kind<KIND_SYS>(p, sb, num_sms, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace pf
