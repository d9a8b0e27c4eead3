// Single-launch resamplers for the cumulative schemes (Figure 1a-c).
//
// One cooperative launch; every CTA is resident and owns R >= 1 consecutive
// tiles of log-weights:
//   1. pass 1, per owned tile: tile scan (pf_tile.cuh) -- the tile's weights,
//      its local cumulative weights v_i, its sum S_t relative to 2^{k_t} --
//      and a 16-byte record (k_t, S_t, i_last) in global memory;
//   2. the CTA arrives on this launch's counter (release) and one thread waits,
//      with a time limit, until every CTA has arrived;
//   3. every CTA reads all T records and forms the inter-tile carries
//          B_t = sum_{t' < t} S_t' 2^{k_t' - K}
//      as exact 128-bit fixed-point sums (2^-90 resolution relative to the
//      largest tile reference 2^K).  Integer sums are exact and associative, so
//      every CTA holds bit-identical boundaries, and W = B_T is the scan's own
//      last prefix;
//   4. systematic / stratified (Section 2: these schemes yield offspring
//      counts), per owned tile (re-scanned when R > 1): the tile owns the
//      offsets j whose position (j + u_j) W / P lies in [B_t, B_{t+1}); each
//      element counts the offsets below its cumulative weight, N_i, and its
//      index fills [N_{i-1}, N_i) by a run-length decode in shared memory (mark
//      run starts, block max-scan), stored with 128-bit writes;
//      multinomial: the tiles' v_i were written to global memory in pass 1;
//      the CTA draws a balanced slice of the P uniforms, finds the tile by a
//      binary search over the boundaries and the element by a binary search in
//      that tile's v_i.
// Every global write is bounded by [0, P) whatever the data; a NaN/+inf or
// all-zero weight set records PF_ERR_DOMAIN and writes no ancestors.
#include <climits>

#include "pf_fixed.cuh"
#include "pf_tile.cuh"

namespace pf {

constexpr int kMaxOwn = 64;    // tiles per CTA
constexpr int kIoCap = 8192;   // staging entries of the run-length decode
enum { KIND_MULTI = 0, KIND_STRAT = 1, KIND_SYS = 2 };

struct TableEntry {  // multinomial: one tile's lower boundary and scale
    float bhi, blo;  // B_t as a float pair (units of 2^K)
    float sc;        // 2^(K - k_t): global units -> tile-local units
    int il;          // last positive element of the tile, -1 if none
};

struct PersistShared {
    TileShared tile;
    i128 wsum[kWarps];
    i128 Wt;
    i128 Bown[kMaxOwn + 1];  // boundaries of this CTA's tiles (systematic, stratified)
    int red_k[kWarps];
    int red_n[kWarps];
    int noff, K, ok, pad;
    long long jlo;
    float tau0, inv_rho, W_hi, W_lo;
};
// Dynamic shared memory: PersistShared, then either the staging buffer
// int32 out[kIoCap] (systematic, stratified) or TableEntry table[T] (multinomial).

__host__ __device__ constexpr size_t persistent_smem_bytes(int kind, int T) {
    return sizeof(PersistShared) + (kind == KIND_MULTI ? (size_t)T * sizeof(TableEntry) : kIoCap * sizeof(int32_t));
}

// ---------------------------------------------------------------------------
// Arrival and carries.  Block-wide; identical results in every CTA.
// ---------------------------------------------------------------------------
// Arrive on this epoch's counter with release semantics (after the CTA's
// records are written) and wait, one thread, bounded, for every CTA.
__device__ bool arrive_and_wait(const SortedParams& p, PersistShared& sm, bool skip, uint32_t epoch,
                                uint64_t t_start) {
    const int tid = threadIdx.x;
    uint32_t* arrive = p.ctl + CTL_ARRIVE0 + (epoch & 1u);
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
// and leaves the block total in sm.Wt.
__device__ __forceinline__ i128 block_scan_i128(PersistShared& sm, i128 x) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const i128 inc = warp_scan_i128(x, lane);
    if (lane == 31) sm.wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const i128 v = lane < kWarps ? sm.wsum[lane] : (i128)0;
        const i128 vi = warp_scan_i128(v, lane);
        if (lane < kWarps) sm.wsum[lane] = vi - v;
        if (lane == kWarps - 1) sm.Wt = vi;
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
    for (int t = tid; t < T; t += kThreads) {
        const uint4 r = ld_cg_v4_u32(rec + 4 * t);
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
        if (t < T) r = ld_cg_v4_u32(rec + 4 * t);
        const int sh = (int)r.x - K;
        const i128 a = (t < T) ? fixed_of(__uint_as_float(r.y), sh) + fixed_of(__uint_as_float(r.z), sh) : (i128)0;
        const i128 B = running + block_scan_i128(sm, a);  // carry of tile t
        running += sm.Wt;
        __syncthreads();  // sm.wsum / sm.Wt are reused by the next pass
        if (t < T) {
            if (KIND == KIND_MULTI) {
                const fpair b = fixed_to_pair(B);
                table[t] = {b.hi, b.lo, pow2f(-sh), (int)r.w};
            } else if (t >= t_first && t <= t_first + t_count) {
                sm.Bown[t - t_first] = B;
            }
        }
    }
    if (tid == 0) {
        sm.K = K;
        sm.Wt = running;
        if (KIND != KIND_MULTI && t_first + t_count == T) sm.Bown[t_count] = running;
        const fpair Wp = fixed_to_pair(running);
        sm.W_hi = Wp.hi;
        sm.W_lo = Wp.lo;
    }
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------------------
// Offspring-count assignment (systematic, stratified).
// ---------------------------------------------------------------------------
// Per-tile scalars (thread 0), in float pairs: the tile's offset range and the
// map from tile-local cumulative weight v to the offset coordinate
// y = v * inv_rho + x0 (offsets counted from jlo).  P <= 2^25 on this path.
template <int KIND>
__device__ void tile_offsets(const SortedParams& p, PersistShared& sm, i128 Bl_i, i128 Bh_i, int k_tile) {
    const fpair W = {sm.W_hi, sm.W_lo};
    const fpair Bl = fixed_to_pair(Bl_i), Bh = fixed_to_pair(Bh_i);
    const fpair Pp = fast_two_sum((float)p.P, (float)(p.P - (int64_t)(float)p.P));  // P exactly
    const fpair PW = pair_div(Pp, W);
    const fpair yl = pair_mul(Bl, PW), yh = pair_mul(Bh, PW);  // B P / W
    const bool last = Bh_i >= sm.Wt;
    long long jl, jh;
    float x0;
    if (KIND == KIND_SYS) {
        const u32x4 r = philox(0u, 0u, p.filter, TAG_SYS, p.key0, p.key1);
        const float u = u23f(r.x);
        const fpair dl = pair_sub_f(yl, u), dh = pair_sub_f(yh, u);
        jl = (Bl_i > 0) ? max(0LL, min((long long)p.P, pair_ceil(dl))) : 0;
        jh = last ? p.P : max(0LL, min((long long)p.P, pair_ceil(dh)));
        x0 = __fadd_rn(__fsub_rn(dl.hi, (float)jl), dl.lo);  // N(v) = ceil(v * inv_rho + x0)
    } else {
        jl = 0;
        if (Bl_i > 0) {
            const long long f = pair_floor(yl);
            if (f >= p.P) {
                jl = p.P;
            } else {
                const float frac = __fadd_rn(__fsub_rn(yl.hi, (float)f), yl.lo);
                const u32x4 r = philox((uint32_t)(f >> 2), 0u, p.filter, TAG_STRAT, p.key0, p.key1);
                jl = f + (u23f(word_of(r, (int)(f & 3))) < frac ? 1 : 0);
            }
        }
        jh = p.P;
        if (!last) {
            const long long f = pair_floor(yh);
            if (f < p.P) {
                const float frac = __fadd_rn(__fsub_rn(yh.hi, (float)f), yh.lo);
                const u32x4 r = philox((uint32_t)(f >> 2), 0u, p.filter, TAG_STRAT, p.key0, p.key1);
                jh = max(0LL, f + (u23f(word_of(r, (int)(f & 3))) < frac ? 1 : 0));
            }
        }
        x0 = __fadd_rn(__fsub_rn(yl.hi, (float)jl), yl.lo);  // y(v) = v * inv_rho + x0
    }
    sm.jlo = jl;
    sm.noff = (int)max(0LL, jh - jl);
    sm.tau0 = x0;
    sm.inv_rho = PW.hi * pow2f(k_tile - sm.K);
}

template <int KIND>
__device__ void assign_offspring(const SortedParams& p, PersistShared& sm, int32_t* out, TileThread& th,
                                 const TileSummary& ts, int64_t t0) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int noff = sm.noff;
    const long long jlo = sm.jlo;
    const float x0 = sm.tau0, ir = sm.inv_rho;
    // N_i: offsets of the tile below the element's cumulative weight (kept in v[] as int bits)
    uint32_t cq = 0xffffffffu;
    u32x4 cw = {0, 0, 0, 0};
    int last_n = -1;
#pragma unroll
    for (int i = 0; i < kMaxPerThread; ++i) {
        if (i < th.K && ((th.pos >> i) & 1u)) {
            int n;
            if (th.e0 + i == ts.i_last) {
                n = noff;
            } else if (KIND == KIND_SYS) {
                const float x = __fmaf_rn(th.v[i], ir, x0);
                n = x <= 0.f ? 0 : (x >= (float)noff ? noff : min(noff, (int)ceilf(x)));
            } else {
                const float y = __fmaf_rn(th.v[i], ir, x0);
                if (y <= 0.f) {
                    n = 0;
                } else {
                    const float fl = floorf(y);
                    if (fl >= (float)noff) {
                        n = noff;
                    } else {
                        const long long j = jlo + (long long)fl;
                        const uint32_t q = (uint32_t)(j >> 2);
                        if (q != cq) {
                            cq = q;
                            cw = philox(q, 0u, p.filter, TAG_STRAT, p.key0, p.key1);
                        }
                        n = min(noff, (int)fl + (u23f(word_of(cw, (int)(j & 3))) < y - fl ? 1 : 0));
                    }
                }
            }
            th.v[i] = __int_as_float(n);
            last_n = n;
        }
    }
    // exclusive running maximum of the threads' last counts: where this thread's first run starts
    int m = last_n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int h = __shfl_up_sync(0xffffffffu, m, o);
        if (lane >= o) m = max(m, h);
    }
    int prev = __shfl_up_sync(0xffffffffu, m, 1);
    if (lane == 0) prev = -1;
    if (lane == 31) sm.red_n[warp] = m;
    __syncthreads();
    for (int w = 0; w < warp; ++w) prev = max(prev, sm.red_n[w]);
    const int start0 = max(prev, 0);
    const int32_t base = (int32_t)(t0 + th.e0);

    // Run-length decode, one staging chunk at a time: each positive element
    // marks the first slot of its run [N_{i-1}, N_i) with its index (runs of
    // later elements start later, so indices increase along the chunk), the
    // element whose run covers the chunk's first slot marks that slot, and an
    // inclusive max-scan over the chunk fills every run.  Chunk slot s sits at
    // out[s + shift] so that out[x] maps to the 16-byte aligned global position
    // gb + x; each thread scans and stores 16 consecutive entries.
    constexpr int kSlots = kIoCap / kThreads;  // entries per thread in the scan
    constexpr int kChunk = kIoCap - 4;         // offsets per chunk (room for the shift)
    for (int c0 = 0; c0 < noff; c0 += kChunk) {
        const int c1 = min(noff, c0 + kChunk);
        const int shift = (int)((jlo + c0) & 3);
#pragma unroll
        for (int q = 0; q < kSlots / 4; ++q)
            *reinterpret_cast<int4*>(&out[tid * kSlots + 4 * q]) = make_int4(-1, -1, -1, -1);
        __syncthreads();
        int a = start0;
#pragma unroll
        for (int i = 0; i < kMaxPerThread; ++i) {
            if (i < th.K && ((th.pos >> i) & 1u)) {
                const int b = __float_as_int(th.v[i]);
                if (b > a) {
                    if (a >= c0 && a < c1) out[a - c0 + shift] = base + i;
                    else if (a < c0 && b > c0) out[shift] = base + i;
                }
                a = b;
            }
        }
        __syncthreads();
        int4 r[kSlots / 4];
        int run = -1;
#pragma unroll
        for (int q = 0; q < kSlots / 4; ++q) {
            r[q] = *reinterpret_cast<const int4*>(&out[tid * kSlots + 4 * q]);
            r[q].x = run = max(run, r[q].x);
            r[q].y = run = max(run, r[q].y);
            r[q].z = run = max(run, r[q].z);
            r[q].w = run = max(run, r[q].w);
        }
        int mm = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int h = __shfl_up_sync(0xffffffffu, mm, o);
            if (lane >= o) mm = max(mm, h);
        }
        int carry = __shfl_up_sync(0xffffffffu, mm, 1);
        if (lane == 0) carry = -1;
        if (lane == 31) sm.red_n[warp] = mm;
        __syncthreads();
        for (int w = 0; w < warp; ++w) carry = max(carry, sm.red_n[w]);
        // entries x in [tid*kSlots, +kSlots) hold chunk slots x - shift
        const int x0i = tid * kSlots;
        const int lo = max(x0i, shift), hi = min(x0i + kSlots, shift + (c1 - c0));
        if (hi > lo) {
            int32_t* g = p.anc + (jlo + c0 - shift) + x0i;  // 16-byte aligned
            int vals[kSlots];
#pragma unroll
            for (int q = 0; q < kSlots / 4; ++q) {
                vals[4 * q + 0] = max(carry, r[q].x);
                vals[4 * q + 1] = max(carry, r[q].y);
                vals[4 * q + 2] = max(carry, r[q].z);
                vals[4 * q + 3] = max(carry, r[q].w);
            }
            if (lo == x0i && hi == x0i + kSlots) {
#pragma unroll
                for (int q = 0; q < kSlots / 4; ++q)
                    *reinterpret_cast<int4*>(g + 4 * q) =
                        make_int4(vals[4 * q], vals[4 * q + 1], vals[4 * q + 2], vals[4 * q + 3]);
            } else {
#pragma unroll
                for (int z = 0; z < kSlots; ++z)
                    if (x0i + z >= lo && x0i + z < hi) g[z] = vals[z];
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Multinomial draws (Figure 1a): binary searches in global units.
// ---------------------------------------------------------------------------
__device__ void multinomial_draws(const SortedParams& p, PersistShared& sm, const TableEntry* table) {
    const int tid = threadIdx.x, cta = blockIdx.x, G = gridDim.x;
    const int T = p.n_tiles;
    const float Wh = sm.W_hi, Wl = sm.W_lo;
    const int64_t nq = (p.P + 3) >> 2;  // four draws per Philox block
    const int64_t q_beg = nq * cta / G, q_end = nq * (cta + 1) / G;
    for (int64_t q = q_beg + tid; q < q_end; q += kThreads) {
        const u32x4 r = philox((uint32_t)q, 0u, p.filter, TAG_MULTI, p.key0, p.key1);
        int32_t a[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            float uh, ul;
            u32_pair(word_of(r, s), uh, ul);
            // target u W as a float pair
            const float th = __fmul_rn(uh, Wh);
            const float tl = __fmaf_rn(uh, Wl, __fmaf_rn(ul, Wh, __fmaf_rn(uh, Wh, -th)));
            // last tile whose carry is <= the target (compared by value)
            int lo = 0, hi = T - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                const float d = __fadd_rn(__fsub_rn(table[mid].bhi, th), __fsub_rn(table[mid].blo, tl));
                if (d <= 0.f) lo = mid;
                else hi = mid - 1;
            }
            int tt = lo;
            while (tt > 0 && table[tt].il < 0) --tt;  // never settle on a tile without weight
            const TableEntry e = table[tt];
            // tile-local target as a pair (exact binary scaling)
            float xh = __fmul_rn(__fsub_rn(th, e.bhi), e.sc);
            float xl = __fmul_rn(__fsub_rn(tl, e.blo), e.sc);
            if (xh + xl < 0.f) {
                xh = 0.f;
                xl = 0.f;
            }
            const int64_t b0 = (int64_t)tt * p.tile;
            const int nt = (int)min((int64_t)p.tile, p.P - b0);
            const float* vt = p.v_out + b0;
            int l2 = 0, h2 = nt;
            while (l2 < h2) {
                const int mid = (l2 + h2) >> 1;
                // |v| > xh + xl, with |v| - xh exact near the decision
                if (__fsub_rn(fabsf(__ldcg(vt + mid)), xh) > xl) h2 = mid;
                else l2 = mid + 1;
            }
            int idx = e.il;
            if (l2 < nt) {
                idx = l2;
                if (zero_flag(__ldcg(vt + idx))) {
                    int f = e.il;
                    for (int z = idx + 1; z < nt; ++z)
                        if (!zero_flag(__ldcg(vt + z))) {
                            f = z;
                            break;
                        }
                    idx = f;
                }
            }
            a[s] = (int32_t)(b0 + idx);
        }
        const int64_t j = 4 * q;
        if (j + 3 < p.P) {
            *reinterpret_cast<int4*>(p.anc + j) = make_int4(a[0], a[1], a[2], a[3]);
        } else {
            for (int s = 0; s < 4; ++s)
                if (j + s < p.P) p.anc[j + s] = a[s];
        }
    }
}

// The tile's cumulative weights to global memory (sign bit: zero weight), for the searches.
__device__ __forceinline__ void write_tile_v(const SortedParams& p, const TileThread& th, int64_t t0, int n) {
    float* vg = p.v_out + t0 + th.e0;
#pragma unroll
    for (int q = 0; q < kMaxPerThread / 4; ++q) {
        if (4 * q < th.K) {
            float o[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int i = 4 * q + r;
                o[r] = ((th.pos >> i) & 1u) ? th.v[i] : -th.v[i];
            }
            if (th.e0 + 4 * q + 3 < n) {
                *reinterpret_cast<float4*>(vg + 4 * q) = make_float4(o[0], o[1], o[2], o[3]);
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (th.e0 + 4 * q + r < n) vg[4 * q + r] = o[r];
            }
        }
    }
}

template <int KIND>
__global__ void __launch_bounds__(kThreads, 2) k_persistent(SortedParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PersistShared& sm = *reinterpret_cast<PersistShared*>(smem_raw);
    unsigned char* region = smem_raw + sizeof(PersistShared);
    const int tid = threadIdx.x;
    const uint64_t t_start = global_ns();
    const uint32_t epoch = ld_relaxed_u32(p.ctl + CTL_EPOCH) + 1u;
    const int R = p.tiles_per_cta > 0 ? p.tiles_per_cta : 1;
    const int t_first = blockIdx.x * R;
    const int t_count = max(0, min(R, p.n_tiles - t_first));
    uint32_t* rec = reinterpret_cast<uint32_t*>(p.slots);

    // pass 1: scan and record every owned tile
    TileThread th;
    TileSummary ts;
    ts.k = 0;
    ts.i_last = -1;
    bool skip = false;
    for (int r = 0; r < t_count; ++r) {
        const int t = t_first + r;
        const int64_t t0 = (int64_t)t * p.tile;
        const int n = (int)min((int64_t)p.tile, p.P - t0);
        ts = tile_scan(p.lw + t0, n, sm.tile, th);
        if (ts.bad && tid == 0) set_status(p.ctl + CTL_STATUS, ST_DOMAIN);
        if (KIND == KIND_MULTI) {
            write_tile_v(p, th, t0, n);
            __threadfence();
        }
        if (tid == 0) {
            skip |= (t == p.skip_tile);
            st_v4_u32(rec + 4 * t, (uint32_t)ts.k, __float_as_uint(ts.bad ? NAN : ts.S.hi), __float_as_uint(ts.S.lo),
                      (uint32_t)ts.i_last);
        }
        __syncthreads();
    }

    bool ok = arrive_and_wait(p, sm, skip, epoch, t_start);
    if (!ok && tid == 0) set_status(p.ctl + CTL_STATUS, ST_TIMEOUT);
    if (ok) ok = carries<KIND>(p, sm, reinterpret_cast<TableEntry*>(region), t_first, t_count);
    // every CTA read the epoch before arriving, and CTA 0 has seen all arrivals
    // (or waited out its limit): reset the counter the next launch will use and
    // advance the epoch
    if (blockIdx.x == 0 && tid == 0) {
        atomicExch(p.ctl + CTL_ARRIVE0 + ((epoch + 1u) & 1u), 0u);
        atomicExch(p.ctl + CTL_EPOCH, epoch);
    }
    if (!ok) return;

    if (KIND == KIND_MULTI) {
        multinomial_draws(p, sm, reinterpret_cast<const TableEntry*>(region));
        return;
    }
    // pass 2: offsets of every owned tile (the last tile's scan is still in registers)
    int32_t* out = reinterpret_cast<int32_t*>(region);
    for (int r = t_count - 1; r >= 0; --r) {
        const int t = t_first + r;
        const int64_t t0 = (int64_t)t * p.tile;
        if (r != t_count - 1) ts = tile_scan(p.lw + t0, (int)min((int64_t)p.tile, p.P - t0), sm.tile, th);
        if (tid == 0) tile_offsets<KIND>(p, sm, sm.Bown[r], sm.Bown[r + 1], ts.k);
        __syncthreads();
        assign_offspring<KIND>(p, sm, out, th, ts, t0);
    }
}

template <int KIND>
static cudaError_t set_smem_attr() {
    return cudaFuncSetAttribute(k_persistent<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)persistent_smem_bytes(KIND, kMaxTilesTotal));
}

template <int KIND>
static cudaError_t launch_kind(const SortedParams& p, int grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = persistent_smem_bytes(KIND, p.n_tiles);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_persistent<KIND>, p);
}

cudaError_t launch_sorted_persistent(int kind, const SortedParams& p, int grid, cudaStream_t s) {
    const int R = p.tiles_per_cta > 0 ? p.tiles_per_cta : 1;
    if (p.n_tiles < 1 || p.n_tiles > kMaxTilesTotal || R > kMaxOwn || (int64_t)grid * R < p.n_tiles)
        return cudaErrorInvalidValue;
    switch (kind) {
    case KIND_MULTI: return launch_kind<KIND_MULTI>(p, grid, s);
    case KIND_STRAT: return launch_kind<KIND_STRAT>(p, grid, s);
    case KIND_SYS: return launch_kind<KIND_SYS>(p, grid, s);
    }
    return cudaErrorInvalidValue;
}

// Called once per device: raises the dynamic shared memory limit and returns
// how many CTAs of the kind fit on one SM (the cooperative grid limit), at the
// largest shared-memory size a launch may ask for.
int persistent_blocks_per_sm(int kind) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    const size_t smem = persistent_smem_bytes(kind, kMaxTilesTotal);
    switch (kind) {
    case KIND_MULTI:
        if (set_smem_attr<KIND_MULTI>() == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_persistent<KIND_MULTI>, kThreads, smem);
        break;
    case KIND_STRAT:
        if (set_smem_attr<KIND_STRAT>() == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_persistent<KIND_STRAT>, kThreads, smem);
        break;
    case KIND_SYS:
        if (set_smem_attr<KIND_SYS>() == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_persistent<KIND_SYS>, kThreads, smem);
        break;
    }
    return e == cudaSuccess ? nb : 0;
}

}  // namespace pf
