// Assignment of offsets to a tile's elements, shared by the single-launch and
// the batched kernels (Section 2: systematic and stratified resampling give
// offspring counts; multinomial resampling a binary search per draw).
#pragma once

#include "pf_fixed.cuh"
#include "pf_tile.cuh"

namespace pf {

enum { KIND_MULTI = 0, KIND_STRAT = 1, KIND_SYS = 2 };
// Staging entries of the run-length decode (per buffer): a chunk holds up to
// CAP - 4 offsets.  kIoCap serves tiles of up to 8192 elements, whose offset
// count varies around the tile length, so such a tile nearly always decodes
// in one chunk; kIoCapSmall serves tiles of up to 4096.
constexpr int kIoCap = 10240;
constexpr int kIoCapSmall = 8192;
static_assert(kIoCap % (4 * 512) == 0 && kIoCapSmall % (4 * 512) == 0, "decode chunks use 4-entry groups per thread");

struct TableEntry {  // multinomial: one tile's lower boundary and scale
    float bhi, blo;  // B_t as a float pair (units of 2^K)
    float sc;        // 2^(K - k_t): global units -> tile-local units
    int il;          // last positive element of the tile, -1 if none
};

// Shared-memory fields of one filter's assignment.
struct AssignShared {
    i128 Wt;       // total mass W (fixed point, units of 2^K)
    int K;         // largest tile exponent
    int noff;      // offsets of the tile being assigned
    long long jlo; // first offset of that tile
    float tau0, inv_rho, W_hi, W_lo;
    int red_n[kWarps];
};

// ---------------------------------------------------------------------------
// Offspring-count assignment (systematic, stratified).
// ---------------------------------------------------------------------------
// Per-tile scalars (lanes 0 and 1 of warp 0), in float pairs: the tile's
// offset range and the map from tile-local cumulative weight v to the offset
// coordinate y = v * inv_rho + x0 (offsets counted from jlo).
// One end of a tile's offset range: the offsets below boundary B (B_t for
// the lower end, B_{t+1} for the upper), the same function of B for both, so
// adjacent tiles share their common end exactly.  A boundary at 0 gives 0 and
// one at the total mass W gives P.  Lower end (SYS, STRAT): x0 of the map.
// (a.hi - j) + a.lo for an integer j near a.hi: the subtraction is exact even
// where j has no float representation (odd j above 2^24, with P up to 2^31),
// as a small integer plus the exact fraction of a.hi.
__device__ __forceinline__ float pair_minus_int(fpair a, long long j) {
    const float fh = floorf(a.hi);
    return __fadd_rn(__fadd_rn((float)((long long)fh - j), __fsub_rn(a.hi, fh)), a.lo);
}

template <int KIND>
__device__ __forceinline__ long long offsets_below(const SortedParams& p, const AssignShared& sm, fpair PW, i128 B_i,
                                                   float& x0) {
    const fpair y = pair_mul(fixed_to_pair(B_i), PW);  // B P / W
    long long j;
    if (KIND == KIND_SYS) {
        // the multinomial guide places its offsets at (j / P) W: no uniform shift
        const float u = p.guide ? 0.f : u23f(philox(0u, 0u, p.filter, TAG_SYS, p.key0, p.key1).x);
        const fpair d = pair_sub_f(y, u);
        j = B_i <= 0 ? 0 : (B_i >= sm.Wt ? p.P : max(0LL, min((long long)p.P, pair_ceil(d))));
        x0 = pair_minus_int(d, j);  // N(v) = ceil(v * inv_rho + x0)
    } else {
        j = 0;
        if (B_i >= sm.Wt) {
            j = p.P;
        } else if (B_i > 0) {
            const long long f = pair_floor(y);
            if (f >= p.P) {
                j = p.P;
            } else {
                const float frac = pair_minus_int(y, f);
                const u32x4 r = philox((uint32_t)(f >> 2), 0u, p.filter, TAG_STRAT, p.key0, p.key1);
                j = max(0LL, f + (u23f(word_of(r, (int)(f & 3))) < frac ? 1 : 0));
            }
        }
        x0 = pair_minus_int(y, j);  // y(v) = v * inv_rho + x0
    }
    return j;
}

// A tile's offset range [jlo, jlo + noff) and the map from its tile-local
// cumulative weight v to offsets: N(v) = ceil(v * ir + x0) (systematic) or the
// stratum test on y(v) = v * ir + x0 (stratified), offsets counted from jlo.
struct TileMap {
    long long jlo;
    int noff;
    float x0, ir;
};

// The map of a tile with boundaries [Bl_i, Bh_i), formed by two lanes of one
// warp together: the even lane forms the lower end, the odd lane the upper;
// `mask` names the participating lanes (both lanes of every pair).  Both lanes
// return the map.
template <int KIND>
__device__ __forceinline__ TileMap tile_map_pair(const SortedParams& p, const AssignShared& sm, i128 Bl_i, i128 Bh_i,
                                                 int k_tile, unsigned mask) {
    const int lane = threadIdx.x & 31;
    const bool upper = lane & 1;
    const fpair W = {sm.W_hi, sm.W_lo};
    const fpair Pp = fast_two_sum((float)p.P, (float)(p.P - (int64_t)(float)p.P));  // P exactly
    const fpair PW = pair_div(Pp, W);
    float x0;
    const long long j = offsets_below<KIND>(p, sm, PW, upper ? Bh_i : Bl_i, x0);
    const long long jl = __shfl_sync(mask, j, lane & ~1);
    const long long jh = __shfl_sync(mask, j, lane | 1);
    const float x0l = __shfl_sync(mask, x0, lane & ~1);
    return {jl, (int)max(0LL, jh - jl), x0l, PW.hi * pow2f(k_tile - sm.K)};
}

// The same for one tile into sm (lanes 0 and 1 of warp 0 together).
template <int KIND>
__device__ void tile_offsets(const SortedParams& p, AssignShared& sm, i128 Bl_i, i128 Bh_i, int k_tile) {
    const TileMap m = tile_map_pair<KIND>(p, sm, Bl_i, Bh_i, k_tile, 0x3u);
    if (threadIdx.x == 0) {
        sm.jlo = m.jlo;
        sm.noff = m.noff;
        sm.tau0 = m.x0;
        sm.inv_rho = m.ir;
    }
}

// Run-length decode staging: two buffers of kIoCap entries, used by
// successive chunks in turn.  A chunk's entries are tagged with the chunk's
// epoch, (epoch << kLocalBits) | element, so entries left by earlier chunks
// are smaller than all of its own and no clearing pass is needed; alternating
// the buffers lets a chunk start before every thread has stored the previous
// one.  stage_init fills both buffers with -1 (below every tag) and must run
// once per launch before the first chunk.
constexpr int kLocalBits = 13;  // tile-local element index
static_assert(kTileMax <= (1 << kLocalBits), "element index must fit the tag's low bits");
constexpr uint32_t kEpochMax = (1u << (31 - kLocalBits)) - 1;  // tags stay positive as int32

template <int CAP>
__device__ __forceinline__ void stage_init(int32_t* stage) {  // stage: 16-byte aligned
    for (int i = threadIdx.x; i < 2 * CAP / 4; i += kThreads)
        reinterpret_cast<int4*>(stage)[i] = make_int4(-1, -1, -1, -1);
}

// One chunk [c0, c1) of the tile's offsets: each positive element marks the
// first slot of its run [N_{i-1}, N_i) with its tagged tile-local index (runs
// of later elements start later, so tags increase along the chunk), the
// element whose run covers the chunk's first slot marks that slot, and an
// inclusive max-scan over the chunk fills every run.  Chunk slot s sits at
// out[s + shift] so that out[x] maps to the 16-byte aligned global position
// gb + x; each thread scans and stores S consecutive entries
// (S * kThreads >= c1 - c0 + shift).  Ancestor = tile_base + element.
template <int S, int KK = 0, bool ONE = false>  // KK: elements per thread when fixed, 0 = th.K;
                                                 // ONE: the chunk is the tile's only one (c0 = 0, c1 = noff)
__device__ __forceinline__ void decode_chunk(const SortedParams& p, AssignShared& sm, int32_t* out,
                                             const TileThread& th, long long jlo, int c0, int c1, int shift,
                                             int start0, int32_t tile_base, int32_t tag) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x0i = tid * S;
    const int32_t mark0 = tag | th.e0;
    int a = start0;
#pragma unroll
    for (int i = 0; i < (KK ? KK : kMaxPerThread); ++i) {
        if ((KK || i < th.K) && ((th.pos >> i) & 1u)) {
            const int b = __float_as_int(th.v[i]);
            if (b > a) {
                if (ONE) out[a + shift] = mark0 + i;  // 0 <= a < b <= noff: inside the only chunk
                else if (a >= c0 && a < c1) out[a - c0 + shift] = mark0 + i;
                else if (a < c0 && b > c0) out[shift] = mark0 + i;
            }
            a = b;
        }
    }
    __syncthreads();
    // pass A: this thread's maximum, then the exclusive maximum over the block
    int run = -1;
#pragma unroll
    for (int q = 0; q < S / 4; ++q) {
        const int4 v = *reinterpret_cast<const int4*>(&out[x0i + 4 * q]);
        run = max(run, max(max(v.x, v.y), max(v.z, v.w)));
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
    carry = max(carry, __reduce_max_sync(0xffffffffu, lane < warp ? sm.red_n[lane] : -1));
    // pass B: the entries again (the buffer is not written again before the
    // chunk after next), as running maxima from the carry, stored.  Entries x in
    // [x0i, x0i + S) hold chunk slots x - shift; every slot of the chunk carries
    // this chunk's tag (its first slot is marked).
    const int lo = max(x0i, shift), hi = min(x0i + S, shift + (c1 - c0));
    if (hi > lo) {
        int32_t* g = p.anc + (jlo + c0 - shift) + x0i;  // 16-byte aligned
        const bool whole = lo == x0i && hi == x0i + S;
        int rr = carry;
        // every filled slot holds tag | element with this chunk's tag, so one
        // add turns it into the ancestor tile_base + element
        const int32_t delta = tile_base - tag;
#pragma unroll
        for (int q = 0; q < S / 4; ++q) {
            const int4 v = *reinterpret_cast<const int4*>(&out[x0i + 4 * q]);
            int4 a4;
            a4.x = delta + (rr = max(rr, v.x));
            a4.y = delta + (rr = max(rr, v.y));
            a4.z = delta + (rr = max(rr, v.z));
            a4.w = delta + (rr = max(rr, v.w));
            if (whole) {
                *reinterpret_cast<int4*>(g + 4 * q) = a4;
            } else {
                const int v4[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
                for (int z = 0; z < 4; ++z)
                    if (x0i + 4 * q + z >= lo && x0i + 4 * q + z < hi) g[4 * q + z] = v4[z];
            }
        }
    }
    // no trailing barrier: the next chunk marks the other buffer, and it reuses
    // sm.red_n only after its own mark barrier, which every thread reaches after
    // finishing this chunk's reads of sm.red_n
}

// stage: the two staging buffers (2 * CAP entries, stage_init<CAP>'ed once per
// launch); epoch: the chunk counter of the launch, identical in every thread.
template <int KIND, int KK = 0, int CAP = kIoCap>  // KK: elements per thread when fixed, 0 = th.K
__device__ void assign_offspring(const SortedParams& p, AssignShared& sm, const TileMap map, int32_t* stage,
                                 uint32_t& epoch, TileThread& th, const TileSummary& ts, int64_t index0) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int noff = map.noff;
    const long long jlo = map.jlo;
    const float x0 = map.x0, ir = map.ir;
    // Stratified: when the tile's strata fit a staging buffer, the block draws
    // their uniforms once, four per Philox block, into the buffer the next
    // decode chunk will use (its last readers finished two chunks ago), stored
    // with the sign bit set so that every entry stays below the decode's tags;
    // otherwise each thread draws the blocks its elements need.
    const bool coop = KIND == KIND_STRAT && noff <= CAP;
    const int32_t* ub = stage + ((epoch + 1u) & 1u) * CAP;
    if (KIND == KIND_STRAT && coop) {
        int32_t* uw = stage + ((epoch + 1u) & 1u) * CAP;
        const long long g0 = jlo >> 2, g1 = (jlo + noff - 1) >> 2;
        for (long long g = g0 + tid; g <= g1; g += kThreads) {
            const u32x4 r = philox((uint32_t)g, 0u, p.filter, TAG_STRAT, p.key0, p.key1);
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const long long j = 4 * g + s;
                if (j >= jlo && j < jlo + noff)
                    uw[j - jlo] = (int32_t)(__float_as_uint(u23f(word_of(r, s))) | 0x80000000u);
            }
        }
        __syncthreads();
    }
    // N_i: offsets of the tile below the element's cumulative weight (kept in v[] as int bits).
    // Systematic: N = min(ceil(y), noff), the conversion rounding up and saturating at 0.
    // Stratified: with k = floor(y) (saturating at 0, at most noff - 1), N = k + [u_k < y - k],
    // capped at noff (y - k is exact).  The tile's last positive element takes noff.
    int last_n = -1;
    const int il = ts.i_last - th.e0;  // this thread's index of the tile's last positive element, if any
    if (KIND == KIND_SYS || coop) {
        const uint32_t kmax = (uint32_t)max(noff - 1, 0);
#pragma unroll
        for (int i = 0; i < (KK ? KK : kMaxPerThread); ++i) {
            if ((KK || i < th.K) && ((th.pos >> i) & 1u)) {
                const float y = __fmaf_rn(th.v[i], ir, x0);
                int n;
                if (KIND == KIND_SYS) {
                    n = (int)min(__float2uint_ru(y), (uint32_t)noff);
                } else {
                    const uint32_t k = min(__float2uint_rd(y), kmax);
                    const float u = __uint_as_float((uint32_t)ub[k] & 0x7fffffffu);
                    n = min(noff, (int)k + (u < __fsub_rn(y, (float)k) ? 1 : 0));
                }
                n = i == il ? noff : n;
                th.v[i] = __int_as_float(n);
                last_n = n;
            }
        }
    } else {
        // stratified, strata beyond the staging buffer: each thread draws the
        // Philox blocks its elements need
        uint32_t cq = 0xffffffffu;
        u32x4 cw = {0, 0, 0, 0};
#pragma unroll
        for (int i = 0; i < (KK ? KK : kMaxPerThread); ++i) {
            if ((KK || i < th.K) && ((th.pos >> i) & 1u)) {
                int n;
                const float y = __fmaf_rn(th.v[i], ir, x0);
                if (th.e0 + i == ts.i_last) {
                    n = noff;
                } else if (y <= 0.f) {
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
                th.v[i] = __int_as_float(n);
                last_n = n;
            }
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
    prev = max(prev, __reduce_max_sync(0xffffffffu, lane < warp ? sm.red_n[lane] : -1));
    const int start0 = max(prev, 0);
    const int32_t tile_base = (int32_t)index0;  // particle index of the tile's element 0

    // Run-length decode, one staging chunk at a time (decode_chunk); chunks
    // of at most 2044 / 4092 / 8188 offsets use 4 / 8 / 16 staging entries per
    // thread, larger ones 20.
    constexpr int kChunk = CAP - 4;  // offsets per chunk (room for the shift)
    for (int c0 = 0; c0 < noff; c0 += kChunk) {
        if (++epoch > kEpochMax) {  // tags exhausted (uniform): clear both buffers and restart
            __syncthreads();
            stage_init<CAP>(stage);
            __syncthreads();
            epoch = 1;
        }
        int32_t* out = stage + (epoch & 1u) * CAP;
        const int32_t tag = (int32_t)(epoch << kLocalBits);
        const int c1 = min(noff, c0 + kChunk);
        const int shift = (int)(((uintptr_t)(p.anc + jlo + c0) >> 2) & 3u);  // to a 16-byte boundary
        const int need = c1 - c0 + shift;
        if constexpr (CAP <= 4 * kThreads) {  // small staging (the multinomial guide): need <= CAP always
            if (noff <= kChunk)
                decode_chunk<4, KK, true>(p, sm, out, th, jlo, c0, c1, shift, start0, tile_base, tag);
            else
                decode_chunk<4, KK>(p, sm, out, th, jlo, c0, c1, shift, start0, tile_base, tag);
        } else if (noff <= kChunk) {  // the tile's only chunk
            if (need <= 4 * kThreads)
                decode_chunk<4, KK, true>(p, sm, out, th, jlo, c0, c1, shift, start0, tile_base, tag);
            else if (need <= 8 * kThreads)
                decode_chunk<8, KK, true>(p, sm, out, th, jlo, c0, c1, shift, start0, tile_base, tag);
            else if (CAP == 16 * kThreads || need <= 16 * kThreads)
                decode_chunk<16, KK, true>(p, sm, out, th, jlo, c0, c1, shift, start0, tile_base, tag);
            else
                decode_chunk<(CAP > 16 * kThreads ? CAP : 16 * kThreads + 4) / kThreads, KK, true>(
                    p, sm, out, th, jlo, c0, c1, shift, start0, tile_base, tag);
        } else if (need <= 4 * kThreads)
            decode_chunk<4, KK>(p, sm, out, th, jlo, c0, c1, shift, start0, tile_base, tag);
        else if (need <= 8 * kThreads)
            decode_chunk<8, KK>(p, sm, out, th, jlo, c0, c1, shift, start0, tile_base, tag);
        else if (CAP == 16 * kThreads || need <= 16 * kThreads)
            decode_chunk<16, KK>(p, sm, out, th, jlo, c0, c1, shift, start0, tile_base, tag);
        else
            decode_chunk<(CAP > 16 * kThreads ? CAP : 16 * kThreads + 4) / kThreads, KK>(
                p, sm, out, th, jlo, c0, c1, shift, start0, tile_base, tag);
    }
}

// Four multinomial draws (the words of one Philox block) of one filter
// (Figure 1a).  Draw s targets u_s W (float pair); a binary search over the
// tile table (shared memory) finds the last tile whose carry is <= the
// target, then a lower-bound search in that tile's cumulative weights finds
// the first element whose weight exceeds the tile-local target.  The four
// in-tile searches advance in lockstep, so their loads overlap.
//   table[T]  tile entries;  v  the filter's cumulative weights by tile
//   (sign bit: zero weight; shared memory if SMEM_V, else global/L2);
//   tile  tile length;  PA = P + lead.  Writes filter-local ancestors to a[].
template <bool SMEM_V>
__device__ __forceinline__ void multinomial_draws4(const u32x4& r, const TableEntry* table, int T,
                                                   const float* v, int tile, int64_t PA, int lead, float Wh,
                                                   float Wl, int32_t (&a)[4]) {
    float xh[4], xl[4];
    int lo[4], n[4], il[4];
    int64_t b0[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        float uh, ul;
        u32_pair(word_of(r, s), uh, ul);
        const float th = __fmul_rn(uh, Wh);
        const float tl = __fmaf_rn(uh, Wl, __fmaf_rn(ul, Wh, __fmaf_rn(uh, Wh, -th)));
        int tlo = 0, thi = T - 1;
        while (tlo < thi) {
            const int mid = (tlo + thi + 1) >> 1;
            const float d = __fadd_rn(__fsub_rn(table[mid].bhi, th), __fsub_rn(table[mid].blo, tl));
            if (d <= 0.f) tlo = mid;
            else thi = mid - 1;
        }
        while (tlo > 0 && table[tlo].il < 0) --tlo;  // never settle on a tile without weight
        const TableEntry e = table[tlo];
        float h = __fmul_rn(__fsub_rn(th, e.bhi), e.sc);
        float l = __fmul_rn(__fsub_rn(tl, e.blo), e.sc);
        if (h + l < 0.f) {
            h = 0.f;
            l = 0.f;
        }
        xh[s] = h;
        xl[s] = l;
        b0[s] = (int64_t)tlo * tile;
        n[s] = (int)min((int64_t)tile, PA - b0[s]);
        lo[s] = 0;
        il[s] = e.il;
    }
    const int nt[4] = {n[0], n[1], n[2], n[3]};
    // lower bound: first i with |v_i| - xh > xl (|v| - xh is exact near the decision)
    for (int it = 0; it < 15 && (n[0] | n[1] | n[2] | n[3]) > 0; ++it) {
        float val[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const float* q = v + b0[s] + lo[s] + (n[s] >> 1);
            val[s] = n[s] > 0 ? (SMEM_V ? *q : __ldcg(q)) : 0.f;
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            if (n[s] > 0) {
                const int half = n[s] >> 1;
                if (__fsub_rn(fabsf(val[s]), xh[s]) > xl[s]) {
                    n[s] = half;
                } else {
                    lo[s] += half + 1;
                    n[s] -= half + 1;
                }
            }
        }
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const float* vt = v + b0[s];
        auto ld = [&](int i) -> float { return SMEM_V ? vt[i] : __ldcg(vt + i); };
        int idx = il[s];
        if (lo[s] < nt[s]) {
            idx = lo[s];
            if (zero_flag(ld(idx))) {  // rounding landed on a zero weight: the next positive one
                int f = il[s];
                for (int z = idx + 1; z < nt[s]; ++z)
                    if (!zero_flag(ld(z))) {
                        f = z;
                        break;
                    }
                idx = f;
            }
        }
        a[s] = (int32_t)(b0[s] + idx - lead);
    }
}

// Quad-cooperative window count.  Every lane of the warp calls it at the same
// point (the shuffles span the full warp).  Each lane brings a window of n <= 16
// monotone entries at base + off (base the same in every lane, base + off
// 16-byte aligned; n = 0: none) and its target (xh, xl); the four lanes of each
// aligned quad read each other's windows, one 16-byte piece per lane, so one
// load instruction touches the lines of 8 windows instead of 32 scattered
// pieces.  Returns the count of this lane's window entries at or below its
// target and (FLAGS) the window's zero-weight flags in zmask (sign bits, bit i
// for entry i).
template <bool FLAGS>
__device__ __forceinline__ int quad_window_below(const float* base, int off, int n, float xh, float xl,
                                                 uint32_t& zmask) {
    const int lane = threadIdx.x & 31, q = lane & 3;
    // all four pieces are requested before any is used, so their latencies overlap
    float t[4][4], hr[4], lr[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int src = (lane & ~3) | r;
        const float* wr = base + __shfl_sync(0xffffffffu, off, src);
        const int nr = __shfl_sync(0xffffffffu, n, src);
        hr[r] = __shfl_sync(0xffffffffu, xh, src);
        lr[r] = __shfl_sync(0xffffffffu, xl, src);
        if (4 * q + 3 < nr) {
            const float4 t4 = __ldcg(reinterpret_cast<const float4*>(wr + 4 * q));
            t[r][0] = t4.x;
            t[r][1] = t4.y;
            t[r][2] = t4.z;
            t[r][3] = t4.w;
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) t[r][i] = 4 * q + i < nr ? __ldcg(wr + 4 * q + i) : INFINITY;
        }
    }
    // this lane's share of each window: count in bits 0-4, flags from bit 5 (the
    // lanes' flag bits are disjoint, so adding shares also merges the flags)
    int part[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        int cnt = 0;
        uint32_t z = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            cnt += __fsub_rn(fabsf(t[r][i]), hr[r]) > lr[r] ? 0 : 1;  // +inf padding counts as above
            if (FLAGS) z |= (__float_as_uint(t[r][i]) >> 31) << (4 * q + i);
        }
        part[r] = cnt + (int)(z << 5);
    }
    // transposed sum over the quad: lane q ends with window q's total
    const bool odd = q & 1, high = q & 2;
    int s0 = odd ? part[1] : part[0], s1 = odd ? part[3] : part[2];  // windows q&1 and 2 + (q&1)
    s0 += __shfl_xor_sync(0xffffffffu, odd ? part[0] : part[1], 1);
    s1 += __shfl_xor_sync(0xffffffffu, odd ? part[2] : part[3], 1);
    int mine = high ? s1 : s0;
    mine += __shfl_xor_sync(0xffffffffu, high ? s0 : s1, 2);
    zmask = FLAGS ? ((uint32_t)mine >> 5) : 0u;
    return mine & 31;
}

// One multinomial draw of a filter whose tiles' cumulative weights v are in
// global memory (L2) and whose every 16th |v| (and each tile's last one) is
// in shared memory: tile search in the table, then a search in the tile's
// coarse samples for the first window of 16 elements whose last sample exceeds
// the tile-local target, then that window read whole (64 bytes, 16-byte
// aligned, quad-cooperatively: every lane of the warp must call it) and the
// first element above the target counted in registers.  Same predicate on the
// same monotone sequence as the plain search, so the same result; one 64-byte
// read from L2 per draw instead of a dozen.
constexpr int kWinShift = 4;
constexpr int kWin = 1 << kWinShift;
__device__ __forceinline__ int32_t multinomial_draw_windowed(uint32_t x, const TableEntry* table, int T,
                                                             const float* v, const float* coarse, int cpt, int tile,
                                                             int64_t PA, int lead, float Wh, float Wl) {
    float uh, ul;
    u32_pair(x, uh, ul);
    const float th = __fmul_rn(uh, Wh);
    const float tl = __fmaf_rn(uh, Wl, __fmaf_rn(ul, Wh, __fmaf_rn(uh, Wh, -th)));
    int lo = 0, hi = T - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const float d = __fadd_rn(__fsub_rn(table[mid].bhi, th), __fsub_rn(table[mid].blo, tl));
        if (d <= 0.f) lo = mid;
        else hi = mid - 1;
    }
    while (lo > 0 && table[lo].il < 0) --lo;
    const TableEntry e = table[lo];
    float xh = __fmul_rn(__fsub_rn(th, e.bhi), e.sc);
    float xl = __fmul_rn(__fsub_rn(tl, e.blo), e.sc);
    if (xh + xl < 0.f) {
        xh = 0.f;
        xl = 0.f;
    }
    const int64_t b0 = (int64_t)lo * tile;
    const int nt = (int)min((int64_t)tile, PA - b0);
    // coarse: first window whose last sample is above the target
    const float* c = coarse + lo * cpt;
    int cl = 0, cn = (nt + kWin - 1) >> kWinShift;
    while (cn > 0) {
        const int half = cn >> 1;
        if (__fsub_rn(c[cl + half], xh) > xl) {
            cn = half;
        } else {
            cl += half + 1;
            cn -= half + 1;
        }
    }
    // the window is read quad-cooperatively: every lane of the warp comes here
    // (wn = 0 where the target lies past the tile's samples)
    const int w0 = cl << kWinShift;
    const int wn = w0 < nt ? min(kWin, nt - w0) : 0;
    uint32_t zmask;
    const int below = quad_window_below<true>(v, (int)(b0 + w0), wn, xh, xl, zmask);  // elements at or below the target
    int idx = e.il;
    if (below < wn) {
        idx = w0 + below;
        if ((zmask >> below) & 1u) {  // rounding landed on a zero weight: the next positive one
            int f = e.il;
            for (int z = idx + 1; z < nt; ++z)
                if (!zero_flag(__ldcg(v + b0 + z))) {
                    f = z;
                    break;
                }
            idx = f;
        }
    }
    return (int32_t)(b0 + idx - lead);
}

// Every 16th |v| of a tile (and its last one), from this thread's elements,
// into the tile's coarse samples (shared memory).
__device__ __forceinline__ void write_tile_coarse(const TileThread& th, int n, float* c) {
#pragma unroll
    for (int i = 0; i < kMaxPerThread; ++i) {
        const int e = th.e0 + i;
        if (i < th.K && e < n && (((e + 1) & (kWin - 1)) == 0 || e == n - 1)) c[e >> kWinShift] = fabsf(th.v[i]);
    }
}

// Tile lookup of the single-launch multinomial draws: lut[k], k = 0..kLut, is
// the last tile t whose boundary B_t is at or below the target (k / kLut) W
// under the draws' own comparison.  A draw whose uniform lies in
// (k / kLut, (k+1) / kLut) then lies in tiles lut[k]..lut[k+1], which narrows
// the search over the table to a tile or two.
constexpr int kLutBits = 12;
constexpr int kLut = 1 << kLutBits;

// The draws' comparison: is tile e's boundary at or below the target (th, tl)?
__device__ __forceinline__ bool boundary_at_or_below(const TableEntry& e, float th, float tl) {
    return __fadd_rn(__fsub_rn(e.bhi, th), __fsub_rn(e.blo, tl)) <= 0.f;
}

// Target u W of a uniform given as an exact pair (uh, ul), W = (Wh, Wl).
__device__ __forceinline__ void draw_target(float uh, float ul, float Wh, float Wl, float& th, float& tl) {
    th = __fmul_rn(uh, Wh);
    tl = __fmaf_rn(uh, Wl, __fmaf_rn(ul, Wh, __fmaf_rn(uh, Wh, -th)));
}

// Block-wide (kThreads): fills lut[0..kLut] from table[0..T); red: kWarps ints.
__device__ inline void build_tile_lut(const TableEntry* table, int T, float Wh, float Wl, int* lut, int* red) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int k = tid; k <= kLut; k += kThreads) lut[k] = 0;
    __syncthreads();
    // each tile t >= 1 marks the first lookup point whose target reaches B_t
    for (int t = 1 + tid; t < T; t += kThreads) {
        const TableEntry e = table[t];
        auto reaches = [&](int k) {
            float th, tl;
            draw_target((float)k * (1.f / kLut), 0.f, Wh, Wl, th, tl);
            return boundary_at_or_below(e, th, tl);
        };
        int k = (int)fminf(fmaxf(ceilf(e.bhi / Wh * (float)kLut), 0.f), (float)kLut);
        while (k > 0 && reaches(k - 1)) --k;
        while (k <= kLut && !reaches(k)) ++k;
        if (k <= kLut) atomicMax(&lut[k], t);
    }
    __syncthreads();
    // running maximum over lut[0..kLut): kLut / kThreads consecutive entries per thread
    constexpr int per = kLut / kThreads;
    int m = 0;
#pragma unroll
    for (int i = 0; i < per; ++i) m = max(m, lut[tid * per + i]);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int h = __shfl_up_sync(0xffffffffu, m, o);
        if (lane >= o) m = max(m, h);
    }
    if (lane == 31) red[warp] = m;
    int prev = __shfl_up_sync(0xffffffffu, m, 1);
    if (lane == 0) prev = 0;
    __syncthreads();
    for (int w = 0; w < warp; ++w) prev = max(prev, red[w]);
    int run = prev;
#pragma unroll
    for (int i = 0; i < per; ++i) {
        run = max(run, lut[tid * per + i]);
        lut[tid * per + i] = run;
    }
    if (tid == kThreads - 1) lut[kLut] = max(lut[kLut], run);
    __syncthreads();
}

// Single-launch multinomial draw over three levels of the tiles' cumulative
// weights: every 2^c1shift-th |v| of each tile (c1, shared memory, c1shift >=
// 8), every 16th (c2, global, cpt2 per tile, each tile's block 64-byte
// aligned) and v itself (global).  Level 1 narrows to 2^(c1shift-4) samples of
// c2; when that is more than 16, a binary search over their 16-entry blocks
// (one 4-byte read a level) picks the block; each remaining level reads one
// 16-entry window whole.  The predicate and the monotone sequence are those of
// the plain search, so the result is the same, with two dependent 64-byte
// reads per draw (plus c1shift - 8 small ones) instead of a dozen 4-byte ones.
__device__ __forceinline__ int last_tile_at_or_below(const TableEntry* table, int lo, int hi, float th, float tl) {
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (boundary_at_or_below(table[mid], th, tl)) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int32_t multinomial_draw_3level(uint32_t x, const TableEntry* table, const int* lut, int T,
                                                           const float* v, const float* c2, int cpt2, const float* c1,
                                                           int cpt1, int c1shift, int tile, int64_t PA, int lead,
                                                           float Wh, float Wl) {
    float uh, ul, th, tl;
    u32_pair(x, uh, ul);
    draw_target(uh, ul, Wh, Wl, th, tl);
    // the last tile whose boundary is at or below the target: searched between
    // the lookup points around u, then confirmed (the predicate is monotone in
    // t, so a confirmed tile is the plain binary search's result over all T)
    const int kq = (int)(x >> (32 - kLutBits));
    int lo = last_tile_at_or_below(table, lut[kq], min(lut[kq + 1], T - 1), th, tl);
    if (!boundary_at_or_below(table[lo], th, tl) || (lo + 1 < T && boundary_at_or_below(table[lo + 1], th, tl)))
        lo = last_tile_at_or_below(table, 0, T - 1, th, tl);
    while (lo > 0 && table[lo].il < 0) --lo;
    const TableEntry e = table[lo];
    float xh = __fmul_rn(__fsub_rn(th, e.bhi), e.sc);
    float xl = __fmul_rn(__fsub_rn(tl, e.blo), e.sc);
    if (xh + xl < 0.f) {
        xh = 0.f;
        xl = 0.f;
    }
    const int64_t b0 = (int64_t)lo * tile;
    const int nt = (int)min((int64_t)tile, PA - b0);
    const int n2 = (nt + 15) >> 4, n1 = (nt + (1 << c1shift) - 1) >> c1shift;
    // level 1: first window whose last sample is above the target
    const float* c = c1 + lo * cpt1;
    int cl = 0, cn = n1;
    while (cn > 0) {
        const int half = cn >> 1;
        if (__fsub_rn(c[cl + half], xh) > xl) {
            cn = half;
        } else {
            cl += half + 1;
            cn -= half + 1;
        }
    }
    // levels 2 and 3 read their 16-entry windows quad-cooperatively, so every
    // lane of the warp takes this path (n = 0 where no window is read)
    const bool has = cl < n1;
    const float* c2t = c2 + (int64_t)lo * cpt2;
    int m2 = cl << (c1shift - 4);  // first c2 sample of the window
    if (has && c1shift > 8) {
        // several 16-sample blocks: the first whose last sample is above the target
        int bl = 0, bn = min(1 << (c1shift - 8), (n2 - m2 + 15) >> 4);
        while (bn > 0) {
            const int half = bn >> 1;
            const int last = min(m2 + ((bl + half + 1) << 4), n2) - 1;
            if (__fsub_rn(__ldcg(c2t + last), xh) > xl) {
                bn = half;
            } else {
                bl += half + 1;
                bn -= half + 1;
            }
        }
        m2 += bl << 4;
    }
    // level 2: the block of 16 samples, then level 3: the 16 elements
    uint32_t zmask;
    m2 += quad_window_below<false>(c2, lo * cpt2 + m2, has ? min(16, n2 - m2) : 0, xh, xl, zmask);
    const int w0 = m2 << 4;
    const int wn = has ? min(16, nt - w0) : 0;
    const int below = quad_window_below<true>(v, (int)(b0 + w0), wn, xh, xl, zmask);
    int idx = e.il;
    if (has) {
        idx = w0 + below;
        if (below >= wn) idx = e.il;  // not reached: the window's last sample is above the target
        else if ((zmask >> below) & 1u) {  // rounding landed on a zero weight: the next positive one
            int f = e.il;
            for (int z = idx + 1; z < nt; ++z)
                if (!zero_flag(__ldcg(v + b0 + z))) {
                    f = z;
                    break;
                }
            idx = f;
        }
    }
    return (int32_t)(b0 + idx - lead);
}

// Single-launch multinomial draw through the guide table g[0..M): g[b] is the
// first particle whose cumulative weight exceeds the bucket edge (b / M) W (the
// systematic assignment's arithmetic with M offsets and no uniform shift).  A
// draw whose uniform lies in bucket b = floor(u M) has its answer at or after
// g[b], up to the rounding that separates the two arithmetics, so the draw
// takes the tile holding particle g[b] - 1, confirms it with its own boundary
// test (the tile's boundary at or below the target, the next one above it),
// reads the 16-element window of v that starts at or just below g[b] - 1 and
// counts the elements at or below its target.  That is the plain search's
// result exactly when the window's first element is at or below the target (or
// is the tile's first), and some element of the window is above it (or the
// window ends the tile): the same predicate on the same monotone sequence.
// Otherwise (a bucket holding more than ~12 particles, or an empty tile) ok is
// false and the caller takes the three-level draw.  Every lane of the warp must
// call it (quad-cooperative window read).
__device__ __forceinline__ int32_t multinomial_draw_guided(uint32_t x, const TableEntry* table, int T,
                                                           const float* v, const int32_t* g, int64_t M, int tile,
                                                           int64_t PA, int lead, float Wh, float Wl, bool& ok) {
    float uh, ul, th, tl;
    u32_pair(x, uh, ul);
    draw_target(uh, ul, Wh, Wl, th, tl);
    // bucket of u = (2x + 1) 2^-33: floor(u M), exact in 64-bit integers
    const int64_t b = (int64_t)(((2ull * x + 1ull) * (unsigned long long)M) >> 33);
    int64_t h = (int64_t)__ldcg(g + b) - 1 + lead;  // aligned-window position of particle g[b] - 1
    h = h < lead ? (int64_t)lead : (h > PA - 1 ? PA - 1 : h);
    static_assert((1 << kLocalBits) == kTileMax, "full tiles are 2^kLocalBits elements");
    const int lo = tile == kTileMax ? (int)((uint64_t)h >> kLocalBits) : (int)(h / tile);
    const bool good = boundary_at_or_below(table[lo], th, tl) &&
                      (lo + 1 >= T || !boundary_at_or_below(table[lo + 1], th, tl)) && table[lo].il >= 0;
    const TableEntry e = table[lo];
    float xh = __fmul_rn(__fsub_rn(th, e.bhi), e.sc);
    float xl = __fmul_rn(__fsub_rn(tl, e.blo), e.sc);
    if (xh + xl < 0.f) {
        xh = 0.f;
        xl = 0.f;
    }
    const int64_t b0 = (int64_t)lo * tile;
    const int nt = (int)min((int64_t)tile, PA - b0);
    const int w0 = (int)(h - b0) & ~3;
    const int wn = good ? min(16, nt - w0) : 0;
    uint32_t zmask;
    const int below = quad_window_below<true>(v, (int)(b0 + w0), wn, xh, xl, zmask);
    ok = good && (w0 == 0 || below >= 1) && (below < wn || w0 + wn >= nt);
    int idx = e.il;
    if (ok && below < wn) {
        idx = w0 + below;
        if ((zmask >> below) & 1u) {  // rounding landed on a zero weight: the next positive one
            int f = e.il;
            for (int z = idx + 1; z < nt; ++z)
                if (!zero_flag(__ldcg(v + b0 + z))) {
                    f = z;
                    break;
                }
            idx = f;
        }
    }
    return (int32_t)(b0 + idx - lead);
}

// This thread's samples of its tile: every 16th |v| (and the tile's last)
// into c2, every 2^c1shift-th (and the last) into c1.
template <int KK = 0>
__device__ __forceinline__ void write_tile_samples(const TileThread& th, int n, float* c2, float* c1, int c1shift) {
    const int m1 = (1 << c1shift) - 1;
#pragma unroll
    for (int i = 0; i < (KK ? KK : kMaxPerThread); ++i) {
        const int e = th.e0 + i;
        if ((KK || i < th.K) && e < n) {
            const bool lastel = e == n - 1;
            if (((e + 1) & 15) == 0 || lastel) c2[e >> 4] = fabsf(th.v[i]);
            if (((e + 1) & m1) == 0 || lastel) c1[e >> c1shift] = fabsf(th.v[i]);
        }
    }
}

// Reloads a tile stored by write_tile_v into th (elements of tile-local
// indices [0, n)): v from the magnitudes, the positive-weight mask from the
// sign bits.  Slots at or beyond n are not read.  SMEM: vg0 is a copy of the
// tile in shared memory.
template <int KK = 0, bool SMEM = false>  // KK: elements per thread when fixed (the tile was scanned with KK), 0 = from n
__device__ __forceinline__ void read_tile_v(const float* vg0, int n, TileThread& th) {
    const int K = KK ? KK : per_thread_count(n);
    th.K = K;
    th.e0 = threadIdx.x * K;
    const float* vg = vg0 + th.e0;
    uint32_t pos = 0;
#pragma unroll
    for (int q = 0; q < kMaxPerThread / 4; ++q) {
        if (4 * q < K) {
            float o[4];
            if (th.e0 + 4 * q + 3 < n) {
                const float4 t = SMEM ? *reinterpret_cast<const float4*>(vg + 4 * q)
                                      : __ldcg(reinterpret_cast<const float4*>(vg + 4 * q));
                o[0] = t.x;
                o[1] = t.y;
                o[2] = t.z;
                o[3] = t.w;
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    o[r] = th.e0 + 4 * q + r < n ? (SMEM ? vg[4 * q + r] : __ldcg(vg + 4 * q + r)) : -0.0f;
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                th.v[4 * q + r] = fabsf(o[r]);
                if (!zero_flag(o[r])) pos |= 1u << (4 * q + r);
            }
        }
    }
    th.pos = pos;
}

// The tile's cumulative weights to global memory (sign bit: zero weight), for the searches.
template <int KK = 0>
__device__ __forceinline__ void write_tile_v(const SortedParams& p, const TileThread& th, int64_t t0, int n) {
    float* vg = p.v_out + t0 + th.e0;
#pragma unroll
    for (int q = 0; q < (KK ? KK : kMaxPerThread) / 4; ++q) {
        if (KK || 4 * q < th.K) {
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

}  // namespace pf
