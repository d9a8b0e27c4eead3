// C ABI of libpf (declared in include/pf.h): argument checks, the per-stream
// workspace, and the choice of launch for each entry point.  All arithmetic
// happens in the kernels; nothing here touches particle data on the host.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>
#include <algorithm>

#include "pf.h"
#include "pf_internal.h"
#include "pf_lg.h"

namespace pf {
cudaError_t launch_metropolis(const float* lw, int64_t P, int B, const uint32_t* B_dev, uint32_t key0, uint32_t key1,
                              uint32_t filter, int32_t* anc, uint32_t* ctl, int num_sms, cudaStream_t s, int rounds);
cudaError_t prepare_metropolis();
cudaError_t prepare_large();
cudaError_t launch_large(int kind, SortedParams p, void* scratch, int num_sms, cudaStream_t s);
size_t large_scratch_bytes(int kind, int64_t PA);
cudaError_t launch_gather(const void* src, int64_t P_src, int64_t row_bytes, const int32_t* anc, int64_t P_dst,
                          void* dst, uint32_t* ctl, int num_sms, cudaStream_t s);
cudaError_t launch_reduce(const float* lw, int64_t P, void* rec, uint32_t* ctl, float* ess_out, double* log_sum_out,
                          uint32_t* B_out, double eps, uint32_t B_cap, cudaStream_t s);
int reduce_tiles(int64_t P);
cudaError_t probe_l2_random_reads(const float* buf, int64_t n, int reads, int num_sms, double* rate);
size_t reduce_record_bytes();
cudaError_t launch_tile_weights(const float* lw, int64_t n, int k, float* out, cudaStream_t s);
}  // namespace pf

using namespace pf;

static_assert(PF_MAX_CUMULATIVE == (long long)kMaxTilesTotal * kTileMax, "single-call tile capacity");

namespace {

constexpr int kMaxDevices = 64;
constexpr int kMaxRecords = kMaxTilesTotal;  // 16-byte tile records per workspace
constexpr uint32_t kMetroBCap = 1u << 24;

struct DeviceInfo {
    bool ready = false;
    int num_sms = 0;
    int persist_per_sm[3] = {0, 0, 0};
    int batched_per_sm[4] = {0, 0, 0, 0};
};

struct Workspace {
    uint32_t* ctl = nullptr;     // CTL_WORDS control words
    uint64_t* slots = nullptr;   // one 16-byte record per tile of the single-launch kernels
    void* scratch = nullptr;     // per-call scratch (multinomial cumulative weights, reduction records)
    size_t scratch_bytes = 0;
    uint32_t* counters = nullptr;  // per-filter arrival counters, zero between launches
    size_t n_counters = 0;
    unsigned long long* metro = nullptr;  // batched Metropolis: two epoch-tagged words per filter
    size_t n_metro = 0;                   // filters they cover
};

std::mutex g_mu;
DeviceInfo g_dev[kMaxDevices];
std::map<std::pair<int, cudaStream_t>, Workspace> g_ws;
uint64_t g_wait_ns = 1000000000ull;
int g_metro_rounds = 10;  // Philox rounds of the Metropolis chains (pf_set_metropolis_philox_rounds)
int64_t g_skip_tile = -1;
static_assert(kTraceWords == PF_TRACE_WORDS, "trace record layout");
uint64_t* g_trace = nullptr;  // phase-trace buffer (pf_set_trace_buffer), or null
int64_t g_trace_cap = 0;

}  // namespace

// The wait limit set by pf_set_wait_limit_ns (read by the allocation-free entry point too).
uint64_t pf::current_wait_ns() {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_wait_ns;
}

namespace {

pf_status cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return PF_OK;
    if (std::getenv("PF_VERBOSE")) std::fprintf(stderr, "libpf: %s: %s\n", what, cudaGetErrorString(e));
    return PF_ERR_CUDA;
}

pf_status device_info(int& dev, DeviceInfo*& info) {
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return PF_ERR_CUDA;
    info = &g_dev[dev];
    if (info->ready) return PF_OK;
    e = cudaDeviceGetAttribute(&info->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    for (int k = 0; k < 3; ++k) info->persist_per_sm[k] = persistent_blocks_per_sm(k);
    for (int k = 0; k < 3; ++k) info->batched_per_sm[k] = batched_blocks_per_sm(k);
    info->batched_per_sm[PF_METROPOLIS] = batched_metropolis_blocks_per_sm();
    e = prepare_metropolis();
    if (e != cudaSuccess) return cuda_fail(e, "prepare_metropolis");
    e = prepare_large();
    if (e != cudaSuccess) return cuda_fail(e, "prepare_large");
    info->ready = true;
    return PF_OK;
}

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
    return st != cudaStreamCaptureStatusNone;
}

// Workspace of (current device, stream) with at least `scratch` bytes.  Caller holds g_mu.
pf_status workspace(cudaStream_t s, size_t scratch, Workspace*& out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    Workspace& w = g_ws[{dev, s}];
    if (!w.ctl) {
        if (capturing(s)) return PF_ERR_NOMEM;
        // stored only once both buffers exist and are cleared, so that a failed
        // first call leaves no half-made workspace behind for the next one
        uint32_t* ctl = nullptr;
        uint64_t* slots = nullptr;
        if (cudaMalloc(&ctl, CTL_WORDS * sizeof(uint32_t)) != cudaSuccess) return PF_ERR_NOMEM;
        if (cudaMalloc(&slots, 2 * kMaxRecords * sizeof(uint64_t)) != cudaSuccess) {
            cudaFree(ctl);
            return PF_ERR_NOMEM;
        }
        e = cudaMemsetAsync(ctl, 0, CTL_WORDS * sizeof(uint32_t), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(slots, 0, 2 * kMaxRecords * sizeof(uint64_t), s);
        if (e != cudaSuccess) {
            cudaFree(slots);
            cudaFree(ctl);
            return cuda_fail(e, "cudaMemsetAsync");
        }
        w.ctl = ctl;
        w.slots = slots;
    }
    if (scratch > w.scratch_bytes) {
        if (capturing(s)) return PF_ERR_NOMEM;
        // the old scratch may still be in use by work queued on this stream
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
        if (w.scratch) cudaFree(w.scratch);
        w.scratch = nullptr;
        w.scratch_bytes = 0;
        size_t sz = scratch < 4096 ? 4096 : scratch;
        void* p = nullptr;
        if (cudaMalloc(&p, sz) != cudaSuccess) return PF_ERR_NOMEM;
        w.scratch = p;
        w.scratch_bytes = sz;
    }
    out = &w;
    return PF_OK;
}

// At least n zeroed per-filter counters in w (allocated and cleared on growth).
pf_status ensure_counters(Workspace& w, size_t n, cudaStream_t s) {
    if (n <= w.n_counters) return PF_OK;
    if (capturing(s)) return PF_ERR_NOMEM;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (w.counters) cudaFree(w.counters);
    w.counters = nullptr;
    w.n_counters = 0;
    uint32_t* c = nullptr;
    if (cudaMalloc(&c, n * sizeof(uint32_t)) != cudaSuccess) return PF_ERR_NOMEM;
    e = cudaMemsetAsync(c, 0, n * sizeof(uint32_t), s);
    if (e != cudaSuccess) {
        cudaFree(c);
        return cuda_fail(e, "cudaMemsetAsync");
    }
    w.counters = c;
    w.n_counters = n;
    return PF_OK;
}

// At least n filters' batched-Metropolis words in w (allocated and zeroed on growth;
// only the batched Metropolis kernel writes them).
pf_status ensure_metro(Workspace& w, size_t n, cudaStream_t s) {
    if (n <= w.n_metro) return PF_OK;
    if (capturing(s)) return PF_ERR_NOMEM;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if (w.metro) cudaFree(w.metro);
    w.metro = nullptr;
    w.n_metro = 0;
    unsigned long long* m = nullptr;
    if (cudaMalloc(&m, 2 * n * sizeof(unsigned long long)) != cudaSuccess) return PF_ERR_NOMEM;
    e = cudaMemsetAsync(m, 0, 2 * n * sizeof(unsigned long long), s);
    if (e != cudaSuccess) {
        cudaFree(m);
        return cuda_fail(e, "cudaMemsetAsync");
    }
    w.metro = m;
    w.n_metro = n;
    return PF_OK;
}

size_t lg_record_bytes(int F, int64_t P) {
    const int64_t tiles = (P + lg_tile() - 1) / lg_tile();
    return (size_t)F * (size_t)tiles * sizeof(float4);
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

size_t reduce_scratch(int64_t P) { return (size_t)reduce_tiles(P) * reduce_record_bytes(); }

// Tile layout of a single-launch call: T tiles of `tile` log-weights (a
// multiple of 4, at most kTileMax), R consecutive tiles per CTA, G <= G_max
// resident CTAs.  While P fits one tile per resident CTA, tiles hold at least
// ~2K log-weights and R = 1; beyond that tiles are full and R grows.
bool persistent_layout(int64_t P, int G_max, int64_t min_tile, int& G, int& tile, int& T, int& R) {
    if (G_max < 1) return false;
    if (P > (int64_t)kMaxTilesTotal * kTileMax) return false;
    if (P <= (int64_t)G_max * kTileMax) {
        if (min_tile < 4) min_tile = 4;
        int64_t g = (P + min_tile - 1) / min_tile;
        if (g > G_max) g = G_max;
        if (g < 1) g = 1;
        int64_t t = (P + g - 1) / g;
        t = (t + 3) & ~int64_t(3);
        if (t > kTileMax) t = kTileMax;
        T = (int)((P + t - 1) / t);
        tile = (int)t;
        G = T;
        R = 1;
        return true;
    }
    tile = kTileMax;
    T = (int)((P + kTileMax - 1) / kTileMax);
    R = (T + G_max - 1) / G_max;
    G = (T + R - 1) / R;
    return R <= 64;
}

// Minimum tile size of the single-launch kernels per (device, kind, size
// class ceil(log2 P)); 0 = the default.  Set by pf_autotune / pf_set_min_tile.
constexpr int kSizeClasses = 32;
constexpr int kDefaultMinTile = 2048;
int g_min_tile[kMaxDevices][3][kSizeClasses] = {};

int size_class(int64_t P) {
    int c = 0;
    while (c < kSizeClasses - 1 && ((int64_t)1 << c) < P) ++c;
    return c;
}

int64_t min_tile_for(int dev, int kind, int64_t P) {
    if (const char* env = std::getenv("PF_MIN_TILE")) return std::atoll(env);
    const int t = g_min_tile[dev][kind][size_class(P)];
    return t > 0 ? t : kDefaultMinTile;
}

pf_status resample_cumulative(int kind, const float* logw, int64_t P, uint64_t seed, int32_t* anc, void* stream) {
    if (!logw || !anc || P < 1 || P > PF_MAX_PARTICLES) return PF_ERR_INVALID;
    if (((uintptr_t)logw & 3u) || ((uintptr_t)anc & 3u)) return PF_ERR_INVALID;
    // tiles are laid out on the 16-byte aligned window that starts `lead` floats before logw
    const int lead = (int)(((uintptr_t)logw >> 2) & 3u);
    const int64_t PA = P + lead;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    DeviceInfo* info;
    pf_status st = device_info(dev, info);
    if (st) return st;
    // beyond one cooperative launch's tiles: ordinary launches in sequence (pf_large.cu)
    auto run_large = [&]() -> pf_status {
        Workspace* w;
        pf_status sl = workspace(s, large_scratch_bytes(kind, PA), w);
        if (sl) return sl;
        SortedParams p;
        std::memset(&p, 0, sizeof(p));
        p.lw = logw - lead;
        p.anc = anc;
        p.lead = lead;
        p.P = P;
        p.Pd = (double)P;
        p.key0 = (uint32_t)(seed & 0xffffffffu);
        p.key1 = (uint32_t)(seed >> 32);
        p.filter = 0;
        p.ctl = w->ctl;
        p.slots = w->slots;
        p.wait_ns = g_wait_ns;
        p.skip_tile = -1;
        return cuda_fail(launch_large(kind, p, w->scratch, info->num_sms, s), "large launch");
    };
    if (PA > PF_MAX_CUMULATIVE) return run_large();
    int G, tile, T, R;
    // at most one CTA per thread of a CTA: the carries read one CTA record per thread
    const int G_max = std::min(info->num_sms * info->persist_per_sm[kind], kThreads);
    if (!persistent_layout(PA, G_max, min_tile_for(dev, kind, P), G, tile, T, R)) {
        return PF_ERR_INVALID;  // P beyond kMaxTilesTotal full tiles
    }
    Workspace* w;
    // multinomial: the tiles' cumulative weights (PA floats), then samples of
    // every 16th (c2) and 256th (c1) for the three-level draws, when the c1
    // samples fit in shared memory beside the tile table
    int cpt2 = 0, cpt1 = 0, c1shift = 8;
    size_t c2_at = 0, c1_at = 0, g_at = 0, mscratch = 0;
    const int64_t M = (P + 3) / 4;  // multinomial guide buckets
    if (kind == PF_MULTINOMIAL) {
        // level-1 stride 2^c1shift >= 256: the smallest whose samples fit beside the table
        cpt2 = ((tile + 15) / 16 + 15) & ~15;
        while ((1 << c1shift) < tile &&
               (size_t)T * sizeof(float4) + (size_t)T * ((tile + (1 << c1shift) - 1) >> c1shift) * sizeof(float) >
                   (size_t)kMaxTilesTotal * sizeof(float4))
            ++c1shift;
        cpt1 = (tile + (1 << c1shift) - 1) >> c1shift;
        // the level-1 samples of this many tiles do not fit beside the table: the
        // ordinary launches' guide table serves such P better than plain searches
        if ((size_t)T * sizeof(float4) + (size_t)T * cpt1 * sizeof(float) > (size_t)kMaxTilesTotal * sizeof(float4))
            return run_large();
        c2_at = ((size_t)PA * sizeof(float) + 255) & ~(size_t)255;
        c1_at = (c2_at + (size_t)T * cpt2 * sizeof(float) + 255) & ~(size_t)255;
        g_at = (c1_at + (size_t)T * cpt1 * sizeof(float) + 255) & ~(size_t)255;
        mscratch = cpt2 > 0 ? g_at + (size_t)M * sizeof(int32_t) : c1_at;
    } else if (R > 1) {
        mscratch = (size_t)PA * sizeof(float);  // cumulative weights of the tiles pass 2 reloads
    }
    st = workspace(s, mscratch, w);
    if (st) return st;
    SortedParams p;
    p.lw = logw - lead;
    p.anc = anc;
    p.lead = lead;
    p.P = P;
    p.Pd = (double)P;
    p.tile = tile;
    p.n_tiles = T;
    p.tiles_per_cta = R;
    p.key0 = (uint32_t)(seed & 0xffffffffu);
    p.key1 = (uint32_t)(seed >> 32);
    p.filter = 0;
    p.ctl = w->ctl;
    p.slots = w->slots;
    p.wait_ns = g_wait_ns;
    p.skip_tile = (int)g_skip_tile;
    g_skip_tile = -1;
    p.v_out = (kind == PF_MULTINOMIAL || R > 1) ? (float*)w->scratch : nullptr;
    p.c2_out = cpt2 > 0 ? reinterpret_cast<float*>((char*)w->scratch + c2_at) : nullptr;
    p.c1_out = cpt2 > 0 ? reinterpret_cast<float*>((char*)w->scratch + c1_at) : nullptr;
    p.cpt2 = cpt2;
    p.cpt1 = cpt1;
    p.c1shift = c1shift;
    p.trace = g_trace;
    p.trace_cap = g_trace_cap;
    // the guide pays for its decode and second grid-wide wait only when each CTA
    // draws for several tiles' worth of particles (P above one tile per resident
    // CTA: 2^22 162 -> 122 us; at 2^20 it took 41.6 -> 45.7 us)
    p.g_out = (cpt2 > 0 && R > 1) ? reinterpret_cast<int32_t*>((char*)w->scratch + g_at) : nullptr;
    p.M = M;
    p.guide = 0;
    return cuda_fail(launch_sorted_persistent(kind, p, G, s), "persistent launch");
}

}  // namespace

extern "C" {

pf_status pf_resample_systematic(const float* logw, int64_t P, int B, uint64_t seed, int32_t* ancestors,
                                 void* stream) {
    (void)B;
    return resample_cumulative(PF_SYSTEMATIC, logw, P, seed, ancestors, stream);
}

pf_status pf_resample_stratified(const float* logw, int64_t P, int B, uint64_t seed, int32_t* ancestors,
                                 void* stream) {
    (void)B;
    return resample_cumulative(PF_STRATIFIED, logw, P, seed, ancestors, stream);
}

pf_status pf_resample_multinomial(const float* logw, int64_t P, int B, uint64_t seed, int32_t* ancestors,
                                  void* stream) {
    (void)B;
    return resample_cumulative(PF_MULTINOMIAL, logw, P, seed, ancestors, stream);
}

pf_status pf_resample_metropolis(const float* logw, int64_t P, int B, uint64_t seed, int32_t* ancestors,
                                 void* stream) {
    if (!logw || !ancestors || P < 1 || P > PF_MAX_PARTICLES) return PF_ERR_INVALID;
    if (((uintptr_t)logw & 3u) || ((uintptr_t)ancestors & 3u)) return PF_ERR_INVALID;
    if (B < 0 && !aligned16(logw)) return PF_ERR_INVALID;  // the w_max reduction reads 16-byte vectors
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    DeviceInfo* info;
    pf_status st = device_info(dev, info);
    if (st) return st;
    Workspace* w;
    st = workspace(s, B < 0 ? reduce_scratch(P) : 0, w);
    if (st) return st;
    const uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
    const uint32_t* B_dev = nullptr;
    if (B < 0) {
        cudaError_t e = launch_reduce(logw, P, w->scratch, w->ctl, nullptr, nullptr, w->ctl + CTL_METRO_B, 0.01,
                                      kMetroBCap, s);
        if (e != cudaSuccess) return cuda_fail(e, "reduce launch");
        B_dev = w->ctl + CTL_METRO_B;
    }
    return cuda_fail(
        launch_metropolis(logw, P, B, B_dev, k0, k1, 0u, ancestors, w->ctl, info->num_sms, s, g_metro_rounds),
        "metropolis launch");
}

pf_status pf_gather(const void* src, int64_t P_src, int64_t row_bytes, const int32_t* ancestors, int64_t P_dst,
                    void* dst, void* stream) {
    if (!src || !dst || !ancestors || P_src < 1 || P_dst < 0 || row_bytes <= 0 || (row_bytes & 3)) {
        return PF_ERR_INVALID;
    }
    if (P_dst == 0) return PF_OK;
    const uintptr_t s0 = (uintptr_t)src, s1 = s0 + (uintptr_t)(P_src * row_bytes);
    const uintptr_t d0 = (uintptr_t)dst, d1 = d0 + (uintptr_t)(P_dst * row_bytes);
    if (s0 < d1 && d0 < s1) return PF_ERR_INVALID;  // overlapping src and dst
    if (((uintptr_t)src & 3) || ((uintptr_t)dst & 3) || ((uintptr_t)ancestors & 3)) return PF_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    DeviceInfo* info;
    pf_status st = device_info(dev, info);
    if (st) return st;
    Workspace* w;
    st = workspace(s, 0, w);
    if (st) return st;
    return cuda_fail(launch_gather(src, P_src, row_bytes, ancestors, P_dst, dst, w->ctl, info->num_sms, s),
                     "gather launch");
}

pf_status pf_ess(const float* logw, int64_t P, float* ess_out, double* log_sum_out, void* stream) {
    if (!logw || !ess_out || P < 1 || P > PF_MAX_PARTICLES || !aligned16(logw)) return PF_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    DeviceInfo* info;
    pf_status st = device_info(dev, info);
    if (st) return st;
    Workspace* w;
    st = workspace(s, reduce_scratch(P), w);
    if (st) return st;
    return cuda_fail(launch_reduce(logw, P, w->scratch, w->ctl, ess_out, log_sum_out, nullptr, 0.0, 0u, s),
                     "reduce launch");
}

namespace {
pf_status resample_batched(int kind, const float* logw, const int64_t* offsets, int F, int B, const uint64_t* seeds,
                           const int32_t* mask, int32_t* ancestors, void* stream, double eps = 0.01,
                           int32_t* B_out = nullptr) {
    if (!logw || !offsets || !seeds || !ancestors || F < 1 || F > (1 << 24)) return PF_ERR_INVALID;
    if (kind < PF_MULTINOMIAL || kind > PF_METROPOLIS) return PF_ERR_INVALID;
    if (!(eps > 0.0) || !(eps < 1.0)) return PF_ERR_INVALID;
    if (((uintptr_t)logw & 3u) || ((uintptr_t)ancestors & 3u) || ((uintptr_t)offsets & 7u) ||
        ((uintptr_t)seeds & 7u) || ((uintptr_t)mask & 3u) || ((uintptr_t)B_out & 3u))
        return PF_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    DeviceInfo* info;
    pf_status st = device_info(dev, info);
    if (st) return st;
    const int per_sm = info->batched_per_sm[kind];
    if (per_sm < 1) return PF_ERR_CUDA;
    const int grid = info->num_sms * per_sm;
    // scratch: per-CTA cumulative weights (multinomial), the plan's items, the
    // split filters' tile records; two counters per filter
    // per-CTA scratch: the cumulative weights of a whole filter's tiles (multinomial, and
    // systematic / stratified filters kept whole in one CTA)
    const int64_t per_cta = kind != PF_METROPOLIS ? (int64_t)batched_scratch_floats_per_cta() : 0;
    const size_t items_at = ((size_t)grid * per_cta * sizeof(float) + 255) & ~(size_t)255;
    const size_t n_items = (size_t)F * kMaxItemsPerFilter;
    const size_t records_at = (items_at + n_items * sizeof(int32_t) + 255) & ~(size_t)255;
    Workspace* w;
    st = workspace(s, records_at + n_items * sizeof(uint4), w);
    if (st) return st;
    st = ensure_counters(*w, 2 * (size_t)F, s);
    if (st) return st;
    if (kind == PF_METROPOLIS) {
        st = ensure_metro(*w, (size_t)F, s);
        if (st) return st;
    }
    int32_t* items = reinterpret_cast<int32_t*>((char*)w->scratch + items_at);
    const int split = kind == PF_STRATIFIED || kind == PF_SYSTEMATIC;
    cudaError_t e = launch_batched_plan(logw, offsets, F, mask, split, items, w->ctl, s, kind == PF_METROPOLIS, grid);
    if (e != cudaSuccess) return cuda_fail(e, "batched plan launch");
    BatchParams bp;
    bp.lw = logw;
    bp.offsets = offsets;
    bp.F = F;
    bp.B = B;
    bp.seeds = seeds;
    bp.anc = ancestors;
    bp.ctl = w->ctl;
    bp.scratch = (float*)w->scratch;
    bp.scratch_per_cta = per_cta;
    bp.items = items;
    bp.records = reinterpret_cast<uint4*>((char*)w->scratch + records_at);
    bp.counters = w->counters;
    bp.wait_ns = g_wait_ns;
    bp.skip_tile = kind == PF_STRATIFIED || kind == PF_SYSTEMATIC ? (int)g_skip_tile : -1;
    if (bp.skip_tile >= 0) g_skip_tile = -1;
    bp.trace = g_trace;
    bp.trace_cap = g_trace_cap;
    bp.B_out = B_out;
    bp.eps = eps;
    bp.metro = kind == PF_METROPOLIS ? w->metro : nullptr;
    bp.rounds = g_metro_rounds;
    if (kind == PF_METROPOLIS) return cuda_fail(launch_batched_metropolis(bp, grid, s), "batched metropolis launch");
    return cuda_fail(launch_batched(kind, bp, grid, s), "batched launch");
}
}  // namespace

pf_status pf_resample_batched(int kind, const float* logw, const int64_t* offsets, int F, int B,
                              const uint64_t* seeds, int32_t* ancestors, void* stream) {
    return resample_batched(kind, logw, offsets, F, B, seeds, nullptr, ancestors, stream);
}

pf_status pf_resample_batched_masked(int kind, const float* logw, const int64_t* offsets, int F, int B,
                                     const uint64_t* seeds, const int32_t* mask, int32_t* ancestors, void* stream) {
    if (!mask) return PF_ERR_INVALID;
    return resample_batched(kind, logw, offsets, F, B, seeds, mask, ancestors, stream);
}

pf_status pf_resample_batched_metropolis_bound(const float* logw, const int64_t* offsets, int F, double eps,
                                               const uint64_t* seeds, const int32_t* mask, int32_t* ancestors,
                                               int32_t* B_out, void* stream) {
    return resample_batched(PF_METROPOLIS, logw, offsets, F, -1, seeds, mask, ancestors, stream, eps, B_out);
}

pf_status pf_reserve(int64_t P_max, int64_t total_max, int F_max, void* stream) {
    if (P_max < 0 || total_max < 0 || F_max < 0) return PF_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    DeviceInfo* info;
    pf_status st = device_info(dev, info);
    if (st) return st;
    // multinomial: P + 3 floats of cumulative weights, their 1/16 and 1/256 samples
    // and the guide table of (P + 3) / 4 entries
    size_t need = (((size_t)(P_max + 3) * sizeof(float) + 255) & ~(size_t)255) +
                  (((size_t)(P_max + 3) / 16 + 16 * (size_t)kMaxTilesTotal) * sizeof(float) + 255) / 256 * 256 +
                  (((size_t)(P_max + 3) / 256 + (size_t)kMaxTilesTotal) * sizeof(float) + 255) / 256 * 256 +
                  ((size_t)(P_max + 3) / 4 + 1) * sizeof(int32_t);
    const size_t red = reduce_scratch(P_max > 0 ? P_max : 1);
    if (red > need) need = red;
    if (P_max + 3 > ((int64_t)1 << 24)) {  // the ordinary-launch path of large single filters
        const size_t large = large_scratch_bytes(PF_MULTINOMIAL, P_max + 3);
        if (large > need) need = large;
    }
    if (F_max > 0) {
        for (int k = PF_MULTINOMIAL; k <= PF_METROPOLIS; ++k) {
            const size_t per_cta = k != PF_METROPOLIS ? batched_scratch_floats_per_cta() : 0;
            const size_t items_at =
                ((size_t)info->num_sms * info->batched_per_sm[k] * per_cta * sizeof(float) + 255) & ~(size_t)255;
            const size_t n_items = (size_t)F_max * kMaxItemsPerFilter;
            const size_t batched = ((items_at + n_items * sizeof(int32_t) + 255) & ~(size_t)255) + n_items * sizeof(uint4);
            if (batched > need) need = batched;
        }
        // bootstrap-filter steps: one record per tile, one counter per filter
        const size_t lg = lg_record_bytes(F_max, (total_max + F_max - 1) / F_max) + (size_t)F_max * sizeof(float4);
        if (lg > need) need = lg;
    }
    Workspace* w;
    st = workspace(s, need, w);
    if (st) return st;
    if (F_max > 0) {
        st = ensure_counters(*w, 2 * (size_t)F_max, s);
        if (st) return st;
        st = ensure_metro(*w, (size_t)F_max, s);
        if (st) return st;
    }
    return cuda_fail(cudaStreamSynchronize(s), "cudaStreamSynchronize");
}

pf_status pf_get_device_status(void* stream, pf_status* out) {
    if (!out) return PF_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_mu);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    auto it = g_ws.find({dev, s});
    if (it == g_ws.end() || !it->second.ctl) {
        e = cudaStreamSynchronize(s);
        *out = PF_OK;
        return cuda_fail(e, "cudaStreamSynchronize");
    }
    uint32_t v = 0;
    e = cudaMemcpyAsync(&v, it->second.ctl + CTL_STATUS, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(it->second.ctl + CTL_STATUS, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    *out = (pf_status)v;
    return PF_OK;
}

int64_t pf_metropolis_B(int64_t P, double w_max, double eps) {
    if (P < 1 || !(w_max > 0.0) || w_max > 1.0 || !(eps > 0.0)) return -1;
    const double beta = 1.0 / (double)P;
    const double alpha = (1.0 - w_max) / ((double)P * w_max);
    const double lambda = 1.0 - alpha - beta;
    const double target = eps * (alpha + beta) / (alpha > beta ? alpha : beta);
    if (target >= 1.0) return 0;
    if (lambda <= 0.0) return 1;
    double b = std::ceil(std::log(target) / std::log(lambda));
    if (b >= 1.0 && std::pow(lambda, b - 1.0) <= target) b -= 1.0;
    return (int64_t)b;
}

double pf_metropolis_bias(int64_t P, double w_max, int64_t B) {
    if (P < 1 || !(w_max > 0.0) || w_max > 1.0 || B < 0) return -1.0;
    const double beta = 1.0 / (double)P;
    const double alpha = (1.0 - w_max) / ((double)P * w_max);
    const double lambda = 1.0 - alpha - beta;
    const double m = (alpha > beta ? alpha : beta) / (alpha + beta);
    return m * std::pow(lambda > 0.0 ? lambda : 0.0, (double)B);
}

const char* pf_status_string(pf_status status) {
    switch (status) {
    case PF_OK: return "ok";
    case PF_ERR_INVALID: return "invalid argument";
    case PF_ERR_DOMAIN: return "domain error (NaN/+inf log-weight or all weights zero)";
    case PF_ERR_TIMEOUT: return "device-side wait ran out";
    case PF_ERR_CUDA: return "CUDA error";
    case PF_ERR_NOMEM: return "workspace allocation failed or needed during capture";
    }
    return "unknown status";
}

pf_status pf_set_wait_limit_ns(uint64_t ns) {
    if (ns == 0) return PF_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_mu);
    g_wait_ns = ns;
    return PF_OK;
}

pf_status pf_debug_tile_weights(const float* logw, int64_t n, int k, float* weights, void* stream) {
    if (!logw || !weights || n < 1 || k < -(1 << 24) || k > (1 << 24) || ((uintptr_t)logw & 3u) ||
        ((uintptr_t)weights & 3u))
        return PF_ERR_INVALID;
    return cuda_fail(launch_tile_weights(logw, n, k, weights, (cudaStream_t)stream), "tile weights launch");
}

pf_status pf_set_metropolis_philox_rounds(int rounds) {
    if (rounds != 10 && rounds != 7) return PF_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_mu);
    g_metro_rounds = rounds;
    return PF_OK;
}

int pf_get_metropolis_philox_rounds(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_metro_rounds;
}

pf_status pf_set_trace_buffer(uint64_t* buf, int64_t capacity) {
    if (capacity < 0 || (((uintptr_t)buf) & 7u) != 0 || (buf != nullptr && capacity == 0)) return PF_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_mu);
    g_trace = buf;
    g_trace_cap = buf ? capacity : 0;
    return PF_OK;
}

pf_status pf_debug_skip_publish(int64_t tile) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_skip_tile = tile < 0 ? -1 : tile;
    return PF_OK;
}

pf_status pf_probe_l2_random_reads(const float* buf, int64_t n, int reads_per_thread, double* reads_per_second) {
    if (!buf || !reads_per_second || n < 1 || reads_per_thread < 8) return PF_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    DeviceInfo* info;
    pf_status st = device_info(dev, info);
    if (st) return st;
    return cuda_fail(probe_l2_random_reads(buf, n, reads_per_thread, info->num_sms, reads_per_second), "l2 probe");
}

namespace {
bool lg_shape_ok(int F, int64_t P, int D) {
    return F >= 1 && F <= (1 << 24) && P >= 1 && P <= 0x7fffffffLL && D >= 4 && D <= 64 && D % 4 == 0 &&
           (int64_t)F * P <= ((int64_t)1 << 40) && (P + lg_tile() - 1) / lg_tile() * (int64_t)F < 0x7fffffffLL;
}
}  // namespace

pf_status pf_lg_init(int F, int64_t P, int D, float m0, float p0, uint64_t seed, float* x, float* logw,
                     double* loglik, double* log_sum, float* ess, int32_t* resample, void* stream) {
    if (!lg_shape_ok(F, P, D) || !(p0 >= 0.0f) || !std::isfinite(m0) || !std::isfinite(p0)) return PF_ERR_INVALID;
    if (!x || !logw || !loglik || !log_sum || !ess || !resample) return PF_ERR_INVALID;
    if (!aligned16(x) || ((uintptr_t)logw & 3u) || ((uintptr_t)loglik & 7u) || ((uintptr_t)log_sum & 7u) ||
        ((uintptr_t)ess & 3u) || ((uintptr_t)resample & 3u))
        return PF_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    DeviceInfo* info;
    pf_status st = device_info(dev, info);
    if (st) return st;
    LgParams p{};
    p.F = F;
    p.P = P;
    p.D = D;
    p.sigma = (float)std::sqrt((double)p0);
    p.m0 = m0;
    p.log_P = std::log((double)P);
    p.key0 = (uint32_t)(seed & 0xffffffffu);
    p.key1 = (uint32_t)(seed >> 32);
    p.x_next = x;
    p.lw = logw;
    p.loglik = loglik;
    p.log_sum = log_sum;
    p.ess = ess;
    p.resample = resample;
    return cuda_fail(launch_lg_init(p, info->num_sms, s), "lg init launch");
}

pf_status pf_lg_step(int F, int64_t P, int D, const float* a, double q, double r, double threshold,
                     const float* y, int t, uint64_t seed, const int32_t* ancestors, const float* x_prev,
                     float* x_next, float* logw, double* loglik, double* log_sum, float* ess, int32_t* resample,
                     void* stream) {
    if (!lg_shape_ok(F, P, D) || t < 1) return PF_ERR_INVALID;
    if (!(q >= 0.0) || !(r > 0.0) || !std::isfinite(q) || !std::isfinite(r) || !(threshold >= 0.0) ||
        !std::isfinite(threshold))
        return PF_ERR_INVALID;
    if (!a || !y || !ancestors || !x_prev || !x_next || !logw || !loglik || !log_sum || !ess || !resample)
        return PF_ERR_INVALID;
    if (x_prev == x_next) return PF_ERR_INVALID;
    if (!aligned16(x_prev) || !aligned16(x_next) || !aligned16(y) || ((uintptr_t)a & 3u) ||
        ((uintptr_t)ancestors & 3u) || ((uintptr_t)logw & 3u) || ((uintptr_t)loglik & 7u) ||
        ((uintptr_t)log_sum & 7u) || ((uintptr_t)ess & 3u) || ((uintptr_t)resample & 3u))
        return PF_ERR_INVALID;
    // the two state buffers must not overlap
    const uintptr_t bytes = (uintptr_t)F * (uintptr_t)P * (uintptr_t)D * sizeof(float);
    const uintptr_t xp = (uintptr_t)x_prev, xn = (uintptr_t)x_next;
    if (xp < xn + bytes && xn < xp + bytes) return PF_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    DeviceInfo* info;
    pf_status st = device_info(dev, info);
    if (st) return st;
    Workspace* w;
    st = workspace(s, lg_record_bytes(F, P), w);
    if (st) return st;
    st = ensure_counters(*w, (size_t)F, s);
    if (st) return st;
    LgParams p{};
    p.F = F;
    p.P = P;
    p.D = D;
    p.n_tiles = (int)((P + lg_tile() - 1) / lg_tile());
    p.a = a;
    p.sigma = (float)std::sqrt(q);
    p.inv2r = (float)(0.5 / r);
    p.c_obs = (float)(-0.5 * D * std::log(6.283185307179586477 * r));
    p.threshold = threshold;
    p.log_P = std::log((double)P);
    p.y = y;
    p.t = (uint32_t)t;
    p.key0 = (uint32_t)(seed & 0xffffffffu);
    p.key1 = (uint32_t)(seed >> 32);
    p.anc = ancestors;
    p.x_prev = x_prev;
    p.x_next = x_next;
    p.lw = logw;
    p.loglik = loglik;
    p.log_sum = log_sum;
    p.ess = ess;
    p.resample = resample;
    p.records = (float4*)w->scratch;
    p.counters = w->counters;
    p.status = w->ctl + CTL_STATUS;
    return cuda_fail(launch_lg_step(p, s), "lg step launch");
}

pf_status pf_set_min_tile(int kind, int64_t P, int min_tile) {
    if (kind < PF_MULTINOMIAL || kind > PF_SYSTEMATIC || P < 1 || min_tile < 0 || min_tile > kTileMax)
        return PF_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_mu);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return PF_ERR_CUDA;
    g_min_tile[dev][kind][size_class(P)] = min_tile;
    return PF_OK;
}

int pf_get_min_tile(int kind, int64_t P) {
    if (kind < PF_MULTINOMIAL || kind > PF_SYSTEMATIC || P < 1) return -1;
    std::lock_guard<std::mutex> lk(g_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return -1;
    return (int)min_tile_for(dev, kind, P);
}

pf_status pf_autotune(int kind, const float* logw, int64_t P, int32_t* ancestors, int reps, void* stream,
                      int* min_tile_out, float* us_out) {
    static const int kCandidates[] = {1024, 1536, 2048, 3072, 4096, 6144, 8192};
    if (kind < PF_MULTINOMIAL || kind > PF_SYSTEMATIC || reps < 1 || reps > 1000) return PF_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    if (capturing(s)) return PF_ERR_INVALID;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return PF_ERR_CUDA;
    const int cls = size_class(P);
    int saved;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        saved = g_min_tile[dev][kind][cls];
    }
    cudaEvent_t ev[2];
    if (cudaEventCreate(&ev[0]) != cudaSuccess) return PF_ERR_CUDA;
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return PF_ERR_CUDA;
    }
    std::vector<float> times;
    int best = 0;
    float best_us = 0.0f;
    pf_status st = PF_OK;
    for (int c : kCandidates) {
        {
            std::lock_guard<std::mutex> lk(g_mu);
            g_min_tile[dev][kind][cls] = c;
        }
        // two warm-up calls, then three batches of `reps` back-to-back calls
        // between one event pair: the device clock behind events ticks in
        // microsecond steps, too coarse to time one call
        times.clear();
        for (int r = 0; r < 2 && st == PF_OK; ++r) st = resample_cumulative(kind, logw, P, (uint64_t)r, ancestors, stream);
        for (int b = 0; b < 3 && st == PF_OK; ++b) {
            e = cudaEventRecord(ev[0], s);
            for (int r = 0; r < reps && e == cudaSuccess && st == PF_OK; ++r)
                st = resample_cumulative(kind, logw, P, (uint64_t)(b * reps + r), ancestors, stream);
            if (st) break;
            if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
            if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
            if (e != cudaSuccess) st = cuda_fail(e, "autotune timing");
            times.push_back(ms * 1e3f / (float)reps);
        }
        if (st) break;
        std::sort(times.begin(), times.end());
        const float med = times[times.size() / 2];
        if (best == 0 || med < best_us) {
            best = c;
            best_us = med;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    std::lock_guard<std::mutex> lk(g_mu);
    g_min_tile[dev][kind][cls] = st == PF_OK ? best : saved;
    if (st) return st;
    if (min_tile_out) *min_tile_out = best;
    if (us_out) *us_out = best_us;
    return PF_OK;
}

pf_status pf_permute(const int32_t* ancestors, int64_t P, int32_t* permuted, void* stream) {
    if (!ancestors || !permuted || P < 1 || P > PF_MAX_PARTICLES) return PF_ERR_INVALID;
    if (((uintptr_t)ancestors & 3u) || ((uintptr_t)permuted & 3u)) return PF_ERR_INVALID;
    const uintptr_t a0 = (uintptr_t)ancestors, p0 = (uintptr_t)permuted, n = (uintptr_t)P * 4;
    if (a0 < p0 + n && p0 < a0 + n) return PF_ERR_INVALID;  // must not overlap
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    DeviceInfo* info;
    pf_status st = device_info(dev, info);
    if (st) return st;
    Workspace* w;
    st = workspace(s, permute_scratch_bytes(P), w);
    if (st) return st;
    return cuda_fail(launch_permute(ancestors, P, permuted, w->scratch, w->ctl, info->num_sms, s), "permute launch");
}

pf_status pf_gather_inplace(void* x, int64_t P, int64_t row_bytes, const int32_t* permuted, void* stream) {
    if (!x || !permuted || P < 1 || P > PF_MAX_PARTICLES || row_bytes < 4 || (row_bytes & 3)) return PF_ERR_INVALID;
    if (((uintptr_t)x & 3u) || ((uintptr_t)permuted & 3u)) return PF_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_mu);
    int dev;
    DeviceInfo* info;
    pf_status st = device_info(dev, info);
    if (st) return st;
    Workspace* w;
    st = workspace(s, 0, w);
    if (st) return st;
    return cuda_fail(launch_gather_inplace(x, P, row_bytes, permuted, w->ctl, info->num_sms, s), "gather launch");
}

int pf_is_device_accessible(const void* ptr) {
    if (!ptr) return 0;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();  // clear the error an unknown pointer leaves
        return 0;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return 1;
    return a.type == cudaMemoryTypeHost && a.devicePointer == ptr ? 1 : 0;
}

int pf_version(void) { return 100; }

}  // extern "C"
