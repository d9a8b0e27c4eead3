// Internal declarations shared by the host API and the kernels of libpf.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pf {

// Status codes (mirror pf_status in include/pf.h).
enum : uint32_t {
    ST_OK = 0,
    ST_INVALID = 1,
    ST_DOMAIN = 2,
    ST_TIMEOUT = 3,
};

// Philox stream tags (counter word 3).
enum : uint32_t { TAG_SYS = 1, TAG_STRAT = 2, TAG_MULTI = 3, TAG_METRO = 4 };

// Control words kept in the per-stream workspace.
enum : int {
    CTL_STATUS = 0,       // first device-side error (pf_status code)
    CTL_EPOCH = 1,        // launch epoch of the single-launch kernels
    CTL_ESS_COUNT = 2,    // arrival counter of the ESS reduction
    CTL_TILE_TICKET = 3,  // tile ticket of the lookback scan
    CTL_QUEUE = 4,        // work-queue ticket of the batched kernels
    CTL_QUEUE_DONE = 5,   // completion counter of the batched kernels
    CTL_METRO_B = 6,      // Metropolis step count chosen on the device
    CTL_METRO_EPOCH = 7,  // launch epoch of the batched Metropolis (tags its per-filter words)
    CTL_ARRIVE0 = 8,      // arrival counters of the single-launch kernels,
    CTL_ARRIVE1 = 9,      //   used by alternate epochs (one is reset while the other counts)
    CTL_ITEMS = 10,       // work items of the current batched call (written by its plan pass)
    CTL_HEAVY = 11,       // batched Metropolis: filters on the list of shared (heavy) filters
    CTL_ARRIVE2 = 12,     // second arrival counters of the single-launch multinomial kernel
    CTL_ARRIVE3 = 13,     //   (after its guide table), alternating like CTL_ARRIVE0 / 1
    CTL_WORDS = 16
};

constexpr int kThreads = 512;     // threads per CTA of the tile kernels
constexpr int kMaxPerThread = 16; // elements per thread (multiple of 4)
constexpr int kTileMax = kThreads * kMaxPerThread;
constexpr int kMaxTilesTotal = 4096;  // tiles of one single-launch call (P <= 2^25)

// Per-tile record of the multi-pass scan (decoupled lookback).
struct TileRecord {
    int32_t k;        // tile exponent: weights are relative to 2^k
    int32_t i_last;   // last positive-weight element of the tile (tile-local), -1 if none
    float s_hi, s_lo; // tile sum (compensated pair), relative to 2^k
    double excl;      // exclusive prefix of the tile, relative to 2^excl_k
    int32_t excl_k;
    uint32_t flags;   // bit 0: aggregate ready, bit 1: inclusive ready (per epoch, see kernels)
};

struct SortedParams {
    const float* lw;   // 16-byte aligned base; element 0 of the filter is lw[lead]
    int32_t* anc;      // ancestors (4-byte aligned)
    int64_t P;
    double Pd;     // P as a double
    int tile;      // elements per tile (multiple of 4, <= kTileMax)
    int n_tiles;   // tiles of the launch (T)
    int tiles_per_cta;  // consecutive tiles owned by each CTA (R >= 1; 0 means 1)
    uint32_t key0, key1, filter;
    uint32_t* ctl;
    uint64_t* slots;  // one 16-byte record per tile
    uint64_t wait_ns;
    int skip_tile;
    float* v_out;     // tile-local cumulative weights (P + lead floats): multinomial, and the tiles
                      // pass 2 reloads (systematic / stratified with several tiles per CTA), else null
    int lead;         // elements of the aligned window before element 0 (0..3)
    float* c2_out;    // multinomial: every 16th |v| of each tile (cpt2 per tile), or null
    float* c1_out;    // multinomial: every 2^c1shift-th |v| of each tile (cpt1 per tile)
    int cpt2, cpt1, c1shift;
    uint64_t* trace;     // phase records (kTraceWords words each), or null
    int64_t trace_cap;   // records the trace buffer holds
    int32_t* g_out;      // multinomial: the guide table g[M] (first particle above each bucket edge), or null
    int64_t M;           // guide buckets
    int guide;           // offsets at (j / P) W with no uniform shift (the guide's decode), else 0
};

// Batched call: F filters, filter f owns lw[offsets[f] .. offsets[f+1]).
struct BatchParams {
    const float* lw;
    const int64_t* offsets;
    int F;
    int B;  // Metropolis steps
    const uint64_t* seeds;
    int32_t* anc;
    uint32_t* ctl;
    float* scratch;           // multinomial: per-CTA cumulative weights of multi-tile filters
    int64_t scratch_per_cta;  // floats per CTA
    const int32_t* items;     // work items from the plan pass: f * 32 + tile, or f * 32 + 31 (whole filter)
    uint4* records;           // one 16-byte tile record per item (split filters)
    uint32_t* counters;       // two per filter (arrivals, departures), zero between launches
    uint64_t wait_ns;         // limit of the wait for a split filter's records
    int skip_tile;            // test hook: tile skip_tile of every split filter withholds its record (-1: off)
    uint64_t* trace;     // phase records per work item (kTraceWords words each), or null
    int64_t trace_cap;
    int32_t* B_out;      // Metropolis with B < 0: each filter's chosen step count, or null
    double eps;          // Metropolis with B < 0: the eps of Eq. 4
    unsigned long long* metro;  // Metropolis: two epoch-tagged words per filter (chain-block claims,
                                // published step count), in a buffer no other kernel writes
    int rounds;                 // Metropolis: Philox rounds of the chains' stream (10 or 7)
};

// Phase record of a traced CTA or work item: global-timer stamps at the start,
// after the scans, after the wait, after the carries and at the end, then the
// CTA, the filter and a tile code.
constexpr int kTraceWords = 8;

// Thread 0 writes word w of record i (a global-timer stamp, or `value`).
__device__ __forceinline__ void trace_put(uint64_t* trace, int64_t cap, int64_t i, int w, uint64_t value) {
    if (trace != nullptr && threadIdx.x == 0 && i < cap) trace[i * kTraceWords + w] = value;
}
__device__ __forceinline__ void trace_stamp(uint64_t* trace, int64_t cap, int64_t i, int w) {
    if (trace != nullptr && threadIdx.x == 0 && i < cap) {
        uint64_t t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        trace[i * kTraceWords + w] = t;
    }
}

// One step of F bootstrap filters on the linear-Gaussian test model.
struct LgParams {
    int F;
    int64_t P;
    int D;        // multiple of 4
    int n_tiles;  // tiles of lg_tile() particles per filter
    const float* a;
    float sigma;   // sqrt(q); sqrt(p0) for the initial draw
    float m0;      // initial mean
    float inv2r;   // 1 / (2 r)
    float c_obs;   // -(D/2) log(2 pi r)
    double threshold;
    double log_P;
    const float* y;  // [F][D] observation of this step
    uint32_t t;
    uint32_t key0, key1;
    const int32_t* anc;
    const float* x_prev;
    float* x_next;
    float* lw;
    double* loglik;
    double* log_sum;
    float* ess;
    int32_t* resample;
    float4* records;     // [F][n_tiles]
    uint32_t* counters;  // [F], zero between launches
    uint32_t* status;
};

// The limit of device-side waits set by pf_set_wait_limit_ns (host).
uint64_t current_wait_ns();

// Kernel launchers (defined in the .cu files; return the launch error).
cudaError_t launch_sorted_persistent(int kind, const SortedParams& p, int grid, cudaStream_t s);
int lg_tile();
cudaError_t launch_lg_init(const LgParams& p, int num_sms, cudaStream_t s);
cudaError_t launch_lg_step(const LgParams& p, cudaStream_t s);
size_t permute_scratch_bytes(int64_t P);
cudaError_t launch_permute(const int32_t* anc, int64_t P, int32_t* out, void* scratch, uint32_t* ctl, int num_sms,
                           cudaStream_t s);
cudaError_t launch_gather_inplace(void* x, int64_t P, int64_t row_bytes, const int32_t* perm, uint32_t* ctl,
                                  int num_sms, cudaStream_t s);
int persistent_blocks_per_sm(int kind);
cudaError_t launch_batched(int kind, const BatchParams& bp, int grid, cudaStream_t s);
cudaError_t launch_batched_plan(const float* lw, const int64_t* offsets, int F, const int32_t* mask, int split,
                                int32_t* items, uint32_t* ctl, cudaStream_t s, int metro = 0, int split_min = 0);
constexpr int kMaxHeavy = 4096;  // batched Metropolis: length of the list of shared filters
constexpr int kMaxItemsPerFilter = 16;  // tiles of a batched filter (kMaxOwnB)
int batched_blocks_per_sm(int kind);
size_t batched_scratch_floats_per_cta();
cudaError_t launch_batched_metropolis(const BatchParams& bp, int grid, cudaStream_t s);
int batched_metropolis_blocks_per_sm();

}  // namespace pf
