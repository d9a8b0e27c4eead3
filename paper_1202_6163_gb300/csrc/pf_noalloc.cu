// Multinomial resampling without any allocation, for callers that must not
// allocate device memory.
//
// pf_resample_multinomial keeps its scratch (control words, per-tile records
// and a P-float array of cumulative weights) in a per-stream workspace that the
// library grows with cudaMalloc on first use.  Some callers cannot let a
// library do that: code running under a custom or pool allocator that owns all
// device memory, real-time loops where a first-call cudaMalloc (which also
// synchronises the device) would stall a deadline, or builds that forbid
// allocations once the application has started.  pf_resample_multinomial_static
// runs the single-launch multinomial kernel with the plain binary search per
// draw (not the windowed draws of pf_resample_multinomial, whose tile lookup and
// strided samples of the cumulative weights would need more scratch; both give
// the same ancestors) with its scratch in the fixed array below.  The array belongs to the library's device code: CUDA
// loads that module on a device lazily, at the first call that needs it, so the
// first call on each device (which also looks up the array's address) is the
// one that may allocate or synchronise inside the driver, and should be made at
// start-up, outside any deadline and before any stream capture.
#include <cstring>
#include <mutex>

#include "pf.h"
#include "pf_internal.h"

namespace pf {

namespace {

// Layout of the fixed scratch array: control words, tile records, cumulative weights.
constexpr int kStaticTiles = 1024;
constexpr size_t kCtlBytes = 256;
constexpr size_t kSlotBytes = (size_t)kStaticTiles * 16;  // one 16-byte record per tile
constexpr size_t kVBytes = (size_t)PF_STATIC_MAX_PARTICLES * sizeof(float);
constexpr size_t kScratchBytes = kCtlBytes + kSlotBytes + kVBytes;

// Zero-initialised when the module is loaded on a device.  Host code must not
// use this name as an address: it is only a host-side stand-in for the device
// symbol, whose device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

struct StaticDevice {
    bool ready = false;
    unsigned char* scratch = nullptr;  // device address of g_static_scratch
    int num_sms = 0;
    int per_sm = 0;
};

constexpr int kMaxDevices = 64;
StaticDevice g_static[kMaxDevices];
std::mutex g_static_mu;  // host threads making their first call at once set up one device once

// Once per device, with that device current.
pf_status static_setup(StaticDevice*& out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PF_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_static_mu);
    StaticDevice& d = g_static[dev];
    if (!d.ready) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || ptr == nullptr) return PF_ERR_CUDA;
        if (cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PF_ERR_CUDA;
        d.per_sm = persistent_blocks_per_sm(PF_MULTINOMIAL);
        if (d.per_sm < 1) return PF_ERR_CUDA;
        d.scratch = static_cast<unsigned char*>(ptr);
        d.ready = true;
    }
    out = &d;
    return PF_OK;
}

}  // namespace
}  // namespace pf

extern "C" pf_status pf_resample_multinomial_static(const float* logw, int64_t P, uint64_t seed, int32_t* ancestors,
                                                    uint32_t* device_status, void* stream) {
    using namespace pf;
    if (!logw || !ancestors || P < 1) return PF_ERR_INVALID;
    if (P > PF_STATIC_MAX_PARTICLES) return PF_ERR_INVALID;  // beyond the fixed scratch
    if (((uintptr_t)logw & 15u) || ((uintptr_t)ancestors & 15u)) return PF_ERR_INVALID;
    StaticDevice* d = nullptr;
    pf_status st = static_setup(d);
    if (st != PF_OK) return st;

    // tile layout: as many tiles as fit at once, at least ~2K log-weights each
    int64_t G_max = (int64_t)d->num_sms * d->per_sm;
    if (G_max > kStaticTiles) G_max = kStaticTiles;
    int64_t g = (P + 2047) / 2048;
    if (g > G_max) g = G_max;
    if (g < 1) g = 1;
    int64_t tile = ((P + g - 1) / g + 3) & ~int64_t(3);
    if (tile > kTileMax) return PF_ERR_INVALID;
    g = (P + tile - 1) / tile;

    cudaStream_t s = (cudaStream_t)stream;
    uint32_t* ctl = reinterpret_cast<uint32_t*>(d->scratch);
    // the status word starts each call at zero; the epoch and arrival counters
    // carry over from call to call by design
    if (cudaMemsetAsync(ctl + CTL_STATUS, 0, sizeof(uint32_t), s) != cudaSuccess) return PF_ERR_CUDA;

    SortedParams p;
    std::memset(&p, 0, sizeof(p));
    p.lw = logw;
    p.anc = ancestors;
    p.P = P;
    p.Pd = (double)P;
    p.tile = (int)tile;
    p.n_tiles = (int)g;
    p.key0 = (uint32_t)(seed & 0xffffffffu);
    p.key1 = (uint32_t)(seed >> 32);
    p.filter = 0;
    p.ctl = ctl;
    p.slots = reinterpret_cast<uint64_t*>(d->scratch + kCtlBytes);
    p.wait_ns = current_wait_ns();
    p.skip_tile = -1;
    p.v_out = reinterpret_cast<float*>(d->scratch + kCtlBytes + kSlotBytes);
    if (launch_sorted_persistent(PF_MULTINOMIAL, p, (int)g, s) != cudaSuccess) return PF_ERR_CUDA;
    if (device_status) {
        if (cudaMemcpyAsync(device_status, ctl + CTL_STATUS, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
            return PF_ERR_CUDA;
    }
    return PF_OK;
}
