// Single-launch resamplers for the cumulative schemes (Figure 1a-c).
//
// One cooperative launch, one tile per CTA, every CTA resident:
//   1. tile scan (pf_tile.cuh): the tile's weights, its local cumulative
//      weights v_i in shared memory and its sum S_t relative to 2^{k_t};
//   2. publish (k_t, S_t, i_last) in epoch-tagged 64-bit slots;
//   3. one warp gathers every tile's slots (bounded wait), and forms the
//      inter-tile carries B_t = sum_{t'<t} S_t' 2^{k_t'-K} in FP64 -- the same
//      arithmetic in every CTA, so each tile boundary has one value that both
//      neighbouring tiles see bit for bit, and W = B_T is the scan's own last
//      prefix;
//   4. systematic / stratified: the tile owns the offsets j whose position
//      (j + u_j) W / P lies in [B_t, B_{t+1}) and assigns them to its
//      elements by a merge path over (v_i, offsets), staged through shared
//      memory and stored coalesced;
//      multinomial: the tile's v_i were also written to global memory before
//      publishing; the CTA draws a balanced slice of the P uniforms, finds the
//      tile by binary search over B_t/W in shared memory and the element by
//      binary search in that tile's v_i.
// Every global write is bounded by [0, P) whatever the data; a NaN/+inf or
// all-zero weight set records PF_ERR_DOMAIN and writes nothing.
#include <climits>

#include "pf_tile.cuh"

namespace pf {

constexpr int kMaxTiles = 1024;
constexpr int kIoCap = 4096;  // offsets per merge-path chunk

enum { KIND_MULTI = 0, KIND_STRAT = 1, KIND_SYS = 2 };

struct PersistShared {
    TileShared tile;
    union {
        struct {
            float tau[kIoCap];
            int32_t out[kIoCap + 8];
        } s;
        struct {
            float bhi[kMaxTiles], blo[kMaxTiles], rho[kMaxTiles];
        } m;
    } u;
    double Bs[kMaxTiles + 1];  // carries, units of 2^K
    int kt[kMaxTiles];
    int il[kMaxTiles];
    int jlo, jhi, K, abort;
    float tau0, rho0;
    double W;
};

// ---------------------------------------------------------------------------
// Offset counts N(B) = #{j : position of offset j < B}, in FP64, from the
// canonical boundary values (both neighbouring tiles get the same count).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t n_below_sys(double B, double W, int64_t P, double u) {
    if (!(B > 0.0)) return 0;
    if (B >= W) return P;
    double c = ceil(B / W * (double)P - u);
    c = fmin(fmax(c, 0.0), (double)P);
    return (int64_t)c;
}

__device__ __forceinline__ double u23d(uint32_t x) { return (double)(((x >> 9) << 1) | 1u) * 0x1p-24; }

__device__ __forceinline__ int64_t n_below_strat(double B, double W, int64_t P, uint32_t k0, uint32_t k1,
                                                 uint32_t filter) {
    if (!(B > 0.0)) return 0;
    if (B >= W) return P;
    const double y = B / W * (double)P;
    const double fl = floor(y);
    if (fl >= (double)P) return P;
    if (fl < 0.0) return 0;
    const int64_t j = (int64_t)fl;
    const u32x4 r = philox((uint32_t)(j >> 2), 0u, filter, TAG_STRAT, k0, k1);
    return j + (u23d(word_of(r, (int)(j & 3))) < y - fl ? 1 : 0);
}

// ---------------------------------------------------------------------------
// Gather every tile's slots and form the carries (warp 0; identical in all
// CTAs).  Returns false on timeout or a domain error (status recorded).
// ---------------------------------------------------------------------------
__device__ bool gather_carries(const SortedParams& p, PersistShared& sm, float* tmp_hi, float* tmp_lo,
                               uint32_t epoch, uint64_t t_start) {
    const int lane = threadIdx.x & 31;
    const int T = p.n_tiles;
    bool ok = true;
    int bad = 0;
    int kmax = INT_MIN;
    for (int t = lane; t < T; t += 32) {
        uint32_t kb = 0, hb = 0, lb = 0, ib = 0;
        ok = ok && wait_slot(&p.slots[4 * t + 0], epoch, t_start, p.wait_ns, kb);
        ok = ok && wait_slot(&p.slots[4 * t + 1], epoch, t_start, p.wait_ns, hb);
        ok = ok && wait_slot(&p.slots[4 * t + 2], epoch, t_start, p.wait_ns, lb);
        ok = ok && wait_slot(&p.slots[4 * t + 3], epoch, t_start, p.wait_ns, ib);
        if (!ok) break;
        const float hi = __uint_as_float(hb);
        sm.kt[t] = (int)kb;
        sm.il[t] = (int)ib;
        tmp_hi[t] = hi;
        tmp_lo[t] = __uint_as_float(lb);
        if (hi > 0.f) kmax = max(kmax, (int)kb);
        bad |= !(hi <= 3.402823466e38f);  // a tile saw NaN/+inf
    }
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) {
        if (lane == 0) set_status(p.ctl + CTL_STATUS, ST_TIMEOUT);
        return false;
    }
    kmax = warp_max_i(kmax);
    bad = __any_sync(0xffffffffu, bad);
    if (kmax == INT_MIN || bad) {  // every weight zero, or a bad tile
        if (lane == 0) set_status(p.ctl + CTL_STATUS, ST_DOMAIN);
        return false;
    }
    // contiguous groups of tiles per lane; exclusive FP64 scan
    const int g = (T + 31) / 32;
    const int t_beg = min(T, lane * g), t_end = min(T, t_beg + g);
    double part = 0.0;
    for (int t = t_beg; t < t_end; ++t) {
        const double a = ldexp((double)tmp_hi[t] + (double)tmp_lo[t], sm.kt[t] - kmax);
        sm.Bs[t] = a;  // the tile's own mass, replaced below
        part += a;
    }
    const double inc = warp_scan_d(part, lane);
    double run = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) run = 0.0;
    for (int t = t_beg; t < t_end; ++t) {
        const double a = sm.Bs[t];
        sm.Bs[t] = run;
        run += a;
    }
    const double W = __shfl_sync(0xffffffffu, inc, 31);
    if (lane == 0) {
        sm.Bs[T] = W;
        sm.W = W;
        sm.K = kmax;
    }
    __syncwarp();
    return true;
}

// ---------------------------------------------------------------------------
// Merge path of the tile's elements against a chunk of its offsets.
// ---------------------------------------------------------------------------
template <int KIND>
__device__ __forceinline__ float offset_tau(const PersistShared& sm, int o_tile, int o_chunk) {
    if (KIND == KIND_SYS) return fmaxf(0.f, __fmaf_rn((float)o_tile, sm.rho0, sm.tau0));
    return sm.u.s.tau[o_chunk];
}

// first element in [0, n) with |v| > tau (n if none)
__device__ __forceinline__ int first_above(const float* vs, int n, float tau) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (fabsf(vs[mid]) > tau) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

template <int KIND>
__device__ void assign_chunk(PersistShared& sm, const float* vs, int n, int i_last, int c0, int nc, int shift,
                             int32_t base_index) {
    const int tid = threadIdx.x;
    // element window: every offset of the chunk lands in [e_lo, e_hi]
    const int e_lo = first_above(vs, n, offset_tau<KIND>(sm, c0, 0));
    const int e_hi = first_above(vs, n, offset_tau<KIND>(sm, c0 + nc - 1, nc - 1));
    const int ne = min(n, e_hi + 1) - e_lo;
    const float* v = vs + e_lo;
    const int L = ne + nc;
    const int d0 = (int)((int64_t)tid * L / kThreads);
    const int d1 = (int)((int64_t)(tid + 1) * L / kThreads);
    // partition at diagonal d0: number of window elements consumed
    int lo = max(0, d0 - nc), hi = min(d0, ne);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const int o = d0 - mid - 1;
        if (fabsf(v[mid]) <= offset_tau<KIND>(sm, c0 + o, o)) lo = mid + 1;
        else hi = mid;
    }
    int i = lo, o = d0 - lo;
    for (int d = d0; d < d1; ++d) {
        const bool take = (i < ne) && (o >= nc || fabsf(v[i]) <= offset_tau<KIND>(sm, c0 + o, o));
        if (take) {
            ++i;
        } else {
            int idx = e_lo + i;
            if (idx >= n) idx = i_last;
            else if (zero_flag(vs[idx])) idx = next_positive(vs, n, idx, i_last);
            sm.u.s.out[o + shift] = base_index + idx;
            ++o;
        }
    }
}

// Coalesced store of out[shift .. shift+nc) to anc[g0 .. g0+nc); anc + g0 - shift is 16-byte aligned.
__device__ __forceinline__ void store_chunk(const PersistShared& sm, int32_t* anc, int64_t g0, int nc, int shift) {
    int32_t* a0 = anc + (g0 - shift);
    const int nvec = (shift + nc + 3) >> 2;
    for (int q = threadIdx.x; q < nvec; q += kThreads) {
        const int s0 = 4 * q;
        if (s0 >= shift && s0 + 3 < shift + nc) {
            *reinterpret_cast<int4*>(a0 + s0) = *reinterpret_cast<const int4*>(&sm.u.s.out[s0]);
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int s = s0 + r;
                if (s >= shift && s < shift + nc) a0[s] = sm.u.s.out[s];
            }
        }
    }
}

template <int KIND>
__global__ void __launch_bounds__(kThreads, 2) k_persistent(SortedParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PersistShared& sm = *reinterpret_cast<PersistShared*>(smem_raw);
    const int tid = threadIdx.x;
    const int t = blockIdx.x;
    const uint64_t t_start = global_ns();
    const uint32_t epoch = ld_relaxed_u32(p.ctl + CTL_EPOCH) + 1u;

    const int64_t t0 = (int64_t)t * p.tile;
    const int n = (int)min((int64_t)p.tile, p.P - t0);

    const TileSummary ts = tile_scan(p.lw + t0, n, sm.tile);
    if (ts.bad && tid == 0) set_status(p.ctl + CTL_STATUS, ST_DOMAIN);

    if (KIND == KIND_MULTI) {
        // this tile's cumulative weights go to global memory for the searches
        float* vg = p.v_out + t0;
        for (int i = tid; i < n; i += kThreads) vg[i] = sm.tile.vs[i];
        __threadfence();
        __syncthreads();
    }
    if (tid == 0 && t != p.skip_tile) {
        uint64_t* s = p.slots + 4 * t;
        st_release_u64(s + 0, tag_slot(epoch, (uint32_t)ts.k));
        st_release_u64(s + 1, tag_slot(epoch, __float_as_uint(ts.bad ? NAN : ts.S.hi)));
        st_release_u64(s + 2, tag_slot(epoch, __float_as_uint(ts.S.lo)));
        st_release_u64(s + 3, tag_slot(epoch, (uint32_t)ts.i_last));
    }

    if (tid < 32) {
        const bool ok = gather_carries(p, sm, sm.u.m.bhi, sm.u.m.blo, epoch, t_start);
        if (tid == 0) {
            sm.abort = ok ? 0 : 1;
            if (t == 0) atomicExch(p.ctl + CTL_EPOCH, epoch);
            if (ok && KIND != KIND_MULTI) {
                const double W = sm.W;
                const double Bl = sm.Bs[t], Bh = sm.Bs[t + 1];
                const double scale = ldexp(1.0, sm.K - ts.k);  // global units -> tile-local units
                const double step = W / (double)p.P;
                int64_t jl, jh;
                if (KIND == KIND_SYS) {
                    const u32x4 r = philox(0u, 0u, p.filter, TAG_SYS, p.key0, p.key1);
                    const double u = u23d(r.x);
                    jl = n_below_sys(Bl, W, p.P, u);
                    jh = n_below_sys(Bh, W, p.P, u);
                    sm.tau0 = (float)((((double)jl + u) * step - Bl) * scale);
                } else {
                    jl = n_below_strat(Bl, W, p.P, p.key0, p.key1, p.filter);
                    jh = n_below_strat(Bh, W, p.P, p.key0, p.key1, p.filter);
                    sm.tau0 = (float)(((double)jl * step - Bl) * scale);
                }
                sm.rho0 = (float)(step * scale);
                sm.jlo = (int)jl;
                sm.jhi = (int)max(jl, jh);
            }
        }
    }
    __syncthreads();
    if (sm.abort) return;

    if (KIND != KIND_MULTI) {
        const int jlo = sm.jlo, jhi = sm.jhi;
        for (int c0 = 0; c0 < jhi - jlo; c0 += kIoCap) {
            const int nc = min(kIoCap, jhi - jlo - c0);
            const int shift = (jlo + c0) & 3;
            if (KIND == KIND_STRAT) {
                // position (j + u_j) W/P of each offset of the chunk, tile-local units
                const int64_t j0 = (int64_t)jlo + c0;
                const int64_t q0 = j0 >> 2, q1 = (j0 + nc - 1) >> 2;
                for (int64_t q = q0 + tid; q <= q1; q += kThreads) {
                    const u32x4 r = philox((uint32_t)q, 0u, p.filter, TAG_STRAT, p.key0, p.key1);
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
                        const int64_t j = 4 * q + s;
                        if (j >= j0 && j < j0 + nc) {
                            const float base = __fmaf_rn((float)(j - jlo), sm.rho0, sm.tau0);
                            sm.u.s.tau[(int)(j - j0)] = fmaxf(0.f, __fmaf_rn(u23f(word_of(r, s)), sm.rho0, base));
                        }
                    }
                }
                __syncthreads();
            }
            assign_chunk<KIND>(sm, sm.tile.vs, n, ts.i_last, c0, nc, shift, (int32_t)t0);
            __syncthreads();
            store_chunk(sm, p.anc, (int64_t)jlo + c0, nc, shift);
            __syncthreads();
        }
        return;
    }

    // ---------------- multinomial: table of tile boundaries, then the draws
    const int T = p.n_tiles;
    const double W = sm.W;
    const double invW = 1.0 / W;
    __syncthreads();
    for (int q = tid; q < T; q += kThreads) {
        const double b = sm.Bs[q] * invW;
        const float hi = (float)b;
        sm.u.m.bhi[q] = hi;
        sm.u.m.blo[q] = (float)(b - (double)hi);
        sm.u.m.rho[q] = (float)ldexp(W, sm.K - sm.kt[q]);
    }
    __syncthreads();
    const int64_t nq = (p.P + 3) >> 2;  // four draws per Philox block
    const int64_t q_beg = nq * t / T, q_end = nq * (t + 1) / T;
    for (int64_t q = q_beg + tid; q < q_end; q += kThreads) {
        const u32x4 r = philox((uint32_t)q, 0u, p.filter, TAG_MULTI, p.key0, p.key1);
        int32_t a[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            float uh, ul;
            u32_pair(word_of(r, s), uh, ul);
            // last tile with B_t / W <= u
            int lo = 0, hi = T - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                const float bh = sm.u.m.bhi[mid];
                if (bh < uh || (bh == uh && sm.u.m.blo[mid] <= ul)) lo = mid;
                else hi = mid - 1;
            }
            const int tt = lo;
            const float du = __fadd_rn(__fsub_rn(uh, sm.u.m.bhi[tt]), __fsub_rn(ul, sm.u.m.blo[tt]));
            const float tau = fmaxf(0.f, du * sm.u.m.rho[tt]);
            const int64_t b0 = (int64_t)tt * p.tile;
            const int nt = (int)min((int64_t)p.tile, p.P - b0);
            const float* vt = p.v_out + b0;
            int l2 = 0, h2 = nt;
            while (l2 < h2) {
                const int mid = (l2 + h2) >> 1;
                if (fabsf(__ldcg(vt + mid)) > tau) h2 = mid;
                else l2 = mid + 1;
            }
            int idx = sm.il[tt];
            if (l2 < nt) {
                idx = l2;
                if (zero_flag(__ldcg(vt + idx))) {
                    int f = sm.il[tt];
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

template <int KIND>
static cudaError_t set_smem_attr() {
    return cudaFuncSetAttribute(k_persistent<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(PersistShared));
}

template <int KIND>
static cudaError_t launch_kind(const SortedParams& p, int grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = sizeof(PersistShared);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_persistent<KIND>, p);
}

cudaError_t launch_sorted_persistent(int kind, const SortedParams& p, int grid, cudaStream_t s) {
    switch (kind) {
    case KIND_MULTI: return launch_kind<KIND_MULTI>(p, grid, s);
    case KIND_STRAT: return launch_kind<KIND_STRAT>(p, grid, s);
    case KIND_SYS: return launch_kind<KIND_SYS>(p, grid, s);
    }
    return cudaErrorInvalidValue;
}

// Called once per device: raises the dynamic shared memory limit and returns
// how many CTAs of the kind fit on one SM (the cooperative grid limit).
int persistent_blocks_per_sm(int kind) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    const size_t smem = sizeof(PersistShared);
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
