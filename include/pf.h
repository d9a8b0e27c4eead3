/*
 * pf.h -- C ABI of the GB300 resampling library (libpf.so).
 *
 * Resampling stage of the bootstrap particle filter as defined in Murray,
 * "GPU acceleration of the particle filter: the Metropolis resampler":
 * given P unnormalised weights, redraw P particles with replacement, using
 * the weights as unnormalised probabilities (Section 1, step 4), by one of
 * the four schemes of Figure 1 -- multinomial, stratified, systematic,
 * Metropolis -- and copy the chosen particles' states (the ancestor gather).
 *
 * Conventions for every entry point
 * ---------------------------------
 *  - Weights are given as FP32 log-weights lw[i]; w_i = exp(lw_i) up to a
 *    common factor.  -inf is a legal log-weight (a zero weight, never
 *    selected by the cumulative schemes).  NaN or +inf is a domain error.
 *  - Outputs are ANCESTORS a_j in [0, P), 0-based (Section 2: offspring and
 *    ancestors are interchangeable; o_i = #{j : a_j = i}).
 *  - Cumulative schemes select, for a position t in [0, W), the smallest i
 *    with c_i > t, where c_i = w_0 + ... + w_i and W = c_{P-1}.
 *  - All array arguments are DEVICE pointers on the current CUDA device,
 *    owned by the caller, and must stay valid until the stream reaches the
 *    call.  `stream` is a cudaStream_t (NULL = legacy default stream).
 *  - Every call is asynchronous and stream-ordered.  Argument errors are
 *    returned synchronously and nothing is enqueued.  Errors found on the
 *    device (NaN/+inf log-weight, all weights zero, a bounded wait that ran
 *    out) are recorded in a per-stream device status word, read and cleared
 *    by pf_get_device_status(); the outputs of that call are then
 *    unspecified.
 *  - The library keeps one workspace per (device, stream), grown on demand
 *    (a synchronous allocation); pf_reserve() pre-sizes it so that later
 *    calls allocate nothing (required before capturing calls into a CUDA
 *    graph).  Calls on the same stream share that workspace; calls on
 *    different streams may run concurrently.
 *  - Randomness: Philox-4x32-10 (Salmon et al., SC'11) with key = (seed mod
 *    2^32, seed div 2^32) and counter (c0, c1, filter, tag); filter = 0 for
 *    the single-filter calls and f for filter f of a batched call; tag 1
 *    systematic, 2 stratified, 3 multinomial, 4 Metropolis.  Draw j of an
 *    element stream is word j%4 of counter (j/4, 0, filter, tag).  Metropolis
 *    chain i, steps b and b+1 (b even), uses counter (i, b/2, filter, 4) whose
 *    words are (proposal_b, uniform_b, proposal_{b+1}, uniform_{b+1}).
 *    The Metropolis chains may instead draw from Philox-4x32-7 (seven rounds
 *    of the same function, with the same counters), a stream that costs 30%
 *    fewer Philox rounds per step: see pf_set_metropolis_philox_rounds.
 *    Uniforms: u23(x) = (2*(x>>9)+1)*2^-24 (systematic, stratified,
 *    Metropolis), u32(x) = (2x+1)*2^-33 (multinomial); proposals
 *    j = floor(x*P/2^32).  Every call is therefore a pure function of its
 *    inputs and seed.
 *  - Arithmetic: FP32 log-weights and per-element work; each tile's weights
 *    are taken relative to a power of two near its maximum, so tiles combine
 *    by exact binary scaling.  Within a tile each thread keeps a compensated
 *    FP32 running sum and the block combines the thread totals exactly in
 *    64-bit fixed point (2^-48); the carries between tiles are exact 128-bit
 *    fixed-point sums (2^-90), and per-tile scalars are FP32 pairs (about 48
 *    significant bits).  Results agree with an FP64 evaluation of the same
 *    definitions except at decisions whose uniform lies within ~1e-6
 *    (relative) of a cumulative-weight or weight-ratio threshold.
 *  - Alignment: log-weight and ancestor arrays need 4-byte alignment (the
 *    kernels read the 16-byte aligned window around them); pf_ess and the
 *    autotuned Metropolis (B < 0) need 16-byte aligned log-weights.
 */
#ifndef PF_H_
#define PF_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pf_status {
    PF_OK = 0,
    PF_ERR_INVALID = 1, /* bad argument (null pointer, size out of range, misalignment) */
    PF_ERR_DOMAIN = 2,  /* NaN or +inf log-weight, or every weight zero */
    PF_ERR_TIMEOUT = 3, /* a bounded device-side wait ran out (see pf_set_wait_limit_ns) */
    PF_ERR_CUDA = 4,    /* a CUDA runtime call failed */
    PF_ERR_NOMEM = 5    /* workspace allocation failed, or growth needed during graph capture */
} pf_status;

/* Resampler kinds for pf_resample_batched. */
enum {
    PF_MULTINOMIAL = 0,
    PF_STRATIFIED = 1,
    PF_SYSTEMATIC = 2,
    PF_METROPOLIS = 3
};

/* Largest P of every single-filter call (int32 ancestors).  A filter of a
 * batched cumulative call stops at PF_MAX_BATCHED_FILTER. */
#define PF_MAX_PARTICLES 2147483647LL

/* Largest P (plus the alignment lead of logw) that a single-filter
 * systematic, stratified or multinomial call resamples in one cooperative
 * launch (4096 tiles of 8192 log-weights).  Beyond it the call runs three
 * ordinary launches on the stream -- the tile scans, one CTA forming every
 * tile's exact carry, then the assignment (systematic, stratified: from the
 * tiles' stored cumulative weights) or, for the multinomial, a guide table
 * and the draws (each through its guide entry and one window of the stored
 * cumulative weights, else binary searches over the tile table and the tile)
 * -- with the same tiles, boundaries and per-tile arithmetic, and workspace
 * scratch of 4 bytes per particle plus about 48 bytes per 8192 (multinomial:
 * 1 byte per particle more, its guide table).  A
 * multinomial call also takes these launches from about 3300 tiles on, where
 * its tile table and samples no longer fit shared memory. */
#define PF_MAX_CUMULATIVE (1LL << 25)

/* Largest P_f (plus the alignment lead) of one filter in a batched
 * systematic, stratified or multinomial call: 16 tiles of 8192. */
#define PF_MAX_BATCHED_FILTER (1LL << 17)

/*
 * Systematic resampler (Figure 1c; Kitagawa 1996; Section 2).
 * One uniform u (stream tag 1, draw 0); a_j = smallest i with
 * c_i > (j + u) W / P, j = 0..P-1.  Output is non-decreasing and every
 * particle gets floor(P w_i/W) or ceil(P w_i/W) offspring.
 *   logw      [P] float, 4-byte aligned       (in)
 *   P         1 <= P <= PF_MAX_PARTICLES
 *   B         ignored
 *   seed      Philox key
 *   ancestors [P] int32, 4-byte aligned       (out)
 * One cooperative launch while P + ((logw mod 16) / 4) <= PF_MAX_CUMULATIVE:
 * every CTA scans its tiles, publishes one record for them, waits (bounded)
 * for all records, forms its carries and assigns its ancestors; larger P as
 * PF_MAX_CUMULATIVE describes.  Errors: PF_ERR_INVALID for null or misaligned
 * pointers or P out of range; device status PF_ERR_DOMAIN for NaN/+inf or all
 * -inf log-weights, PF_ERR_TIMEOUT if the wait for the other CTAs' records ran
 * out.
 */
pf_status pf_resample_systematic(const float* logw, int64_t P, int B, uint64_t seed,
                                 int32_t* ancestors, void* stream);

/*
 * Stratified resampler (Figure 1b, Section 2).  Stratum j draws its own
 * uniform u_j (stream tag 2, draw j); a_j = smallest i with
 * c_i > (j + u_j) W / P.  Output is non-decreasing.  Arguments and errors as
 * pf_resample_systematic.
 */
pf_status pf_resample_stratified(const float* logw, int64_t P, int B, uint64_t seed,
                                 int32_t* ancestors, void* stream);

/*
 * Multinomial resampler (Figure 1a; binary search, Section 3).  P i.i.d.
 * uniforms u_j (stream tag 3, draw j, u32 conversion); a_j = smallest i with
 * c_i > u_j W.  Output is in draw order (not sorted).  Arguments and errors as
 * pf_resample_systematic; the workspace holds a P-float cumulative array.
 */
pf_status pf_resample_multinomial(const float* logw, int64_t P, int B, uint64_t seed,
                                  int32_t* ancestors, void* stream);

/*
 * Metropolis resampler (Figure 1d; Section 2).  Chain i starts at k = i and
 * takes B steps; step b proposes j uniformly over all P indices (a proposal of
 * k itself changes nothing) and moves to it when lw_j >= lw_k or when
 * u_b < exp(lw_j - lw_k).  a_i is the chain's final state.  No sum of weights
 * is formed.  For P <= 49152 (a batched filter: P_f <= 57344) the weights
 * w = exp(lw - max lw) are staged in shared memory and a step moves when
 * u_b w_k < w_j, which differs from the rule above only where u_b lies within
 * 7e-7 (relative) of exp(lw_j - lw_k); larger P uses the rule as written.
 *   B > 0   number of steps;  B == 0 gives a_i = i;
 *   B < 0   B is chosen on the device from the bound of Eqs. 1-5 with
 *           eps = 0.01 and the actual w_max (see pf_metropolis_B), capped at
 *           2^24 steps; this adds one reduction pass over logw.
 * Arguments otherwise as pf_resample_systematic.  Zero weights everywhere are
 * not an error here (the chains simply move to their proposals); NaN/+inf is.
 */
pf_status pf_resample_metropolis(const float* logw, int64_t P, int B, uint64_t seed,
                                 int32_t* ancestors, void* stream);

/*
 * Ancestor gather (Section 1, step 4: the redrawn sample set).
 *   dst row j  <-  src row ancestors[j],   j = 0..P_dst-1
 *   src       [P_src][row_bytes] bytes, row-major   (in)
 *   ancestors [P_dst] int32                         (in)
 *   dst       [P_dst][row_bytes] bytes, row-major   (out; must not overlap src)
 * row_bytes must be a positive multiple of 4.  16-byte alignment of src, dst
 * and row_bytes selects 128-bit accesses; otherwise narrower ones are used.
 * An ancestor outside [0, P_src) leaves that row untouched and sets device
 * status PF_ERR_INVALID.
 */
pf_status pf_gather(const void* src, int64_t P_src, int64_t row_bytes, const int32_t* ancestors,
                    int64_t P_dst, void* dst, void* stream);

/*
 * Ancestors in the form for in-place moves (Section 2: offspring and
 * ancestors are interchangeable).  From any ancestor vector a (offspring
 * counts o_i = #{j : a_j = i}), writes the vector with the same counts in
 * which every particle with offspring keeps one of them in its own slot
 * (permuted[i] = i) and the other o_i - 1 copies of each such i, in
 * increasing i, fill the slots of the particles without offspring, in
 * increasing slot order.  Then permuted[permuted[j]] = permuted[j], and
 * pf_gather_inplace moves the states without a second buffer.  Deterministic.
 *   ancestors [P] int32 (in), permuted [P] int32 (out), 4-byte aligned, not
 *   overlapping.  Uses 3P + P/1024 ints of workspace.
 * Errors: PF_ERR_INVALID for bad arguments (returned) or an ancestor outside
 * [0, P) (device status; the output is then unspecified).
 */
pf_status pf_permute(const int32_t* ancestors, int64_t P, int32_t* permuted, void* stream);

/*
 * In-place ancestor gather: row j of x <- row permuted[j] wherever they
 * differ, for a vector in the form pf_permute gives (a source row keeps its
 * slot, so no row is read after it is written).  Only the rows of particles
 * without offspring are written.
 *   x [P][row_bytes] (in/out), row_bytes a positive multiple of 4
 * A permuted[j] outside [0, P) or whose own entry is not itself leaves row j
 * untouched and sets device status PF_ERR_INVALID.
 */
pf_status pf_gather_inplace(void* x, int64_t P, int64_t row_bytes, const int32_t* permuted, void* stream);

/*
 * 1 if `ptr` can be passed as a device pointer to the calls above at the same
 * address: device memory, managed memory, or page-locked host memory mapped
 * into the device's address space (as cudaHostAlloc gives under unified
 * addressing); 0 otherwise.  With host memory the kernels read and write it
 * over the CPU-GPU link (NVLink-C2C on GB300), e.g. a gather whose states
 * live in host memory.  Host-only.
 */
int pf_is_device_accessible(const void* ptr);

/*
 * Effective sample size (Section 3 quotes ESS/P for its weight sets; the
 * standard form is used): ess_out[0] = (sum w)^2 / sum w^2, and, if
 * log_sum_out is not NULL, log_sum_out[0] = log sum_i exp(lw_i).
 *   logw        [P] float, 16-byte aligned      (in)
 *   ess_out     [1] float  (device)             (out)
 *   log_sum_out [1] double (device) or NULL     (out)
 * Device status PF_ERR_DOMAIN for NaN/+inf or all -inf log-weights.
 */
pf_status pf_ess(const float* logw, int64_t P, float* ess_out, double* log_sum_out, void* stream);

/*
 * Batched resampling of F independent filters (the many filters of particle
 * MCMC, Section 1) in one persistent launch over a work queue.
 *   kind      PF_MULTINOMIAL, PF_STRATIFIED, PF_SYSTEMATIC or PF_METROPOLIS
 *   logw      concatenated log-weights; filter f owns logw[offsets[f] .. offsets[f+1])
 *   offsets   [F+1] int64, device, non-decreasing, offsets[0] = 0
 *   F         1 <= F <= 2^24
 *   B         Metropolis steps: B >= 0 steps for every filter; B < 0: each
 *             filter takes its own B from the bound of Eqs. 1-5 with eps = 0.01
 *             and its own largest normalised weight (as
 *             pf_resample_batched_metropolis_bound, which also returns the B
 *             chosen per filter); ignored by the other kinds
 *   seeds     [F] uint64, device: filter f uses key seeds[f] and filter id f
 *   ancestors concatenated like logw; filter-local indices in [0, P_f)
 * logw and ancestors need 4-byte alignment, offsets and seeds 8-byte.  A
 * cumulative filter needs P_f + ((logw + offsets[f]) mod 16)/4 <=
 * PF_MAX_BATCHED_FILTER, a Metropolis filter P_f <= 2^31 - 1; a larger one
 * sets device status PF_ERR_INVALID and is skipped.  An empty filter is
 * skipped.  A filter with NaN/+inf or all -inf log-weights sets device status
 * PF_ERR_DOMAIN (its ancestors are unspecified; other filters are unaffected).
 */
pf_status pf_resample_batched(int kind, const float* logw, const int64_t* offsets, int F, int B,
                              const uint64_t* seeds, int32_t* ancestors, void* stream);

/*
 * pf_resample_batched restricted to the filters with mask[f] != 0; the
 * ancestors of the other filters are left untouched.  This is the
 * resampling step of a batch of bootstrap filters that resample only when
 * their effective sample size falls below a threshold (Section 1, steps 3-4):
 * the mask is the per-filter decision, written on the device by the step
 * that computed the weights, so the call can sit in a CUDA graph.
 *   mask [F] int32, device (in)
 * Other arguments and errors as pf_resample_batched; PF_ERR_INVALID for a
 * NULL or misaligned mask.
 */
pf_status pf_resample_batched_masked(int kind, const float* logw, const int64_t* offsets, int F, int B,
                                     const uint64_t* seeds, const int32_t* mask, int32_t* ancestors,
                                     void* stream);

/*
 * Batched Metropolis resampling in which every filter takes its own step count
 * from the bias bound (Section 2, last paragraph of the analysis of B: compute
 * an appropriate B from Eq. 5 and use it throughout the filter).  For filter f
 * the CTA that resamples it forms w_max = max_i w_i / sum_i w_i from its
 * log-weights (FP32, compensated sum), then B_f = the smallest B with
 * lambda^B <= eps (alpha + beta) / max(alpha, beta) exactly as pf_metropolis_B
 * computes it (FP64 on the device), capped at 2^24; B_f = 2^24 when every
 * weight of the filter is zero.  The chains then take B_f steps (Philox filter
 * id f, key seeds[f], as pf_resample_batched).
 *   eps       0 < eps < 1
 *   mask      [F] int32, device, or NULL (as pf_resample_batched_masked)
 *   B_out     [F] int32, device, or NULL: B_f of every resampled filter (out;
 *             entries of skipped filters are left untouched)
 * Other arguments and errors as pf_resample_batched with kind PF_METROPOLIS.
 * Because B_f follows from w_max in FP32, it can differ from the bound of the
 * exact w_max by one step where the bound lies within ~1e-6 (relative) of an
 * integer.
 */
pf_status pf_resample_batched_metropolis_bound(const float* logw, const int64_t* offsets, int F, double eps,
                                               const uint64_t* seeds, const int32_t* mask, int32_t* ancestors,
                                               int32_t* B_out, void* stream);

/*
 * Pre-size the workspace of `stream` for single-filter calls with up to P_max
 * particles and batched calls with up to total_max particles in up to F_max
 * filters, so that later calls allocate nothing.  Synchronous.
 */
pf_status pf_reserve(int64_t P_max, int64_t total_max, int F_max, void* stream);

/*
 * Tile-size autotuner for the single-launch systematic, stratified and
 * multinomial calls (the paper has no counterpart: its kernels were tuned by
 * hand for one GPU).  While P fits one tile per resident CTA, a call splits
 * the log-weights into tiles of at least `min_tile` (fewer, larger tiles mean
 * fewer records to combine but less parallel work per element); the choice is
 * kept per (device, kind, size class ceil(log2 P)) in this process.
 *
 * pf_autotune times `kind` on the caller's log-weights for each candidate
 * min_tile in {1024, 1536, 2048, 3072, 4096, 6144, 8192} (2 warm-up calls,
 * then three batches of `reps` back-to-back calls each timed by one pair of
 * CUDA events on `stream`; the median batch mean per call), keeps the fastest
 * for P's size class and returns it in *min_tile_out (and its time per call in
 * microseconds in *us_out; either may be NULL).  Candidates that give the same
 * tiling (P / resident CTAs above them) time alike.  Synchronous; overwrites
 * `ancestors`; arguments as pf_resample_systematic, 1 <= reps <= 1000.
 * PF_ERR_INVALID while `stream` is capturing a graph.  While it runs, other
 * calls of the same kind and size class on the device use the candidate being
 * timed (their results stay correct; only their tiling differs).
 *
 * pf_set_min_tile stores a choice (e.g. one tuned in an earlier process;
 * 0 restores the default of 2048); pf_get_min_tile returns the value in
 * effect (-1 for bad arguments).  The environment variable PF_MIN_TILE, when
 * set, overrides both.
 */
pf_status pf_autotune(int kind, const float* logw, int64_t P, int32_t* ancestors, int reps, void* stream,
                      int* min_tile_out, float* us_out);
pf_status pf_set_min_tile(int kind, int64_t P, int min_tile);
int pf_get_min_tile(int kind, int64_t P);

/*
 * Synchronise `stream`, return in *out the first device-side error recorded
 * by calls on it since the last read (PF_OK if none), and clear it.
 */
pf_status pf_get_device_status(void* stream, pf_status* out);

/*
 * Bound on the number of Metropolis steps (Section 2, Eqs. 1-5): the
 * smallest B with lambda^B <= eps (alpha + beta) / max(alpha, beta), where
 * beta = 1/P, alpha = (1 - w_max)/(P w_max) and lambda = 1 - alpha - beta;
 * w_max is the largest normalised weight.  Returns -1 for invalid arguments
 * (P < 1, w_max outside (0, 1], eps <= 0).  Host-only, pure.
 */
int64_t pf_metropolis_B(int64_t P, double w_max, double eps);

/*
 * Bias of a Metropolis resampling with B steps (Section 2, Eqs. 3-4; for a
 * caller who runs fewer steps than pf_metropolis_B asks, trading bias for
 * time, as the paper's Section 3 suggests): the largest deviation, over the
 * chains' starting particles, of the probability of ending on the heaviest
 * particle from w_max, max(alpha, beta)/(alpha + beta) lambda^B, which equals
 * max(w_max, 1 - w_max) (1 - 1/(P w_max))^B.  The heaviest particle's
 * indicator follows the two-state chain of Eq. 3 exactly, so this is the
 * exact deviation, not only a bound.  Returns -1 for invalid arguments
 * (P < 1, w_max outside (0, 1], B < 0).  Host-only, pure.
 */
double pf_metropolis_bias(int64_t P, double w_max, int64_t B);

/*
 * Random-number stream of the Metropolis chains (Section 3, closing
 * paragraph: the resampler's speed hinges on the rate at which random numbers
 * are generated).  rounds = 10 (the default) draws each chain's proposals and
 * uniforms from Philox-4x32-10; rounds = 7 from Philox-4x32-7, the same round
 * function stopped after seven rounds (Salmon et al., SC'11, list it among
 * the generators that pass the Crush battery), with the same counter layout.
 * The two settings give different, equally valid resamplings.  The setting
 * applies to every later pf_resample_metropolis and batched Metropolis call in
 * the process (all devices and streams).  PF_ERR_INVALID for any other value.
 * pf_get_metropolis_philox_rounds returns the setting in effect.
 */
pf_status pf_set_metropolis_philox_rounds(int rounds);
int pf_get_metropolis_philox_rounds(void);

/* Human-readable name of a status code (static storage). */
const char* pf_status_string(pf_status status);

/*
 * Upper limit, in nanoseconds, on every device-side wait of later calls (the
 * grid-wide gathers of the single-launch kernels and the batched work
 * queue).  A wait that runs out records PF_ERR_TIMEOUT and ends the kernel
 * without writing further outputs.  Default 1e9 (one second).
 */
pf_status pf_set_wait_limit_ns(uint64_t ns);

/*
 * Fault injection for tests of the timeout path (host-side switch, read at
 * launch): when tile >= 0, the next systematic/stratified call -- single
 * launch, or batched, where tile `tile` of every filter split over several
 * CTAs is meant -- has that tile skip publishing its record, so every wait on
 * it runs out and the call records PF_ERR_TIMEOUT.  The switch clears itself
 * after one call.  tile < 0 disarms it.
 */
pf_status pf_debug_skip_publish(int64_t tile);

/*
 * Phase trace of the tile kernels (a diagnostic; off by default).  While a
 * buffer is set, every later single-launch systematic, stratified or
 * multinomial call writes one record per CTA (record index = CTA), and every
 * batched systematic, stratified, multinomial or Metropolis call one record
 * per work item (record index = the item's ticket, items in the order the
 * plan pass issues them), of PF_TRACE_WORDS 64-bit words:
 *   [0] GPU global timer (ns) when the CTA started / took the item
 *   [1] ... when its tile scans and record publication were done
 *   [2] ... when its wait ended: the grid-wide gather of the single-launch
 *       kernel, the filter's other tiles for a batched filter split over
 *       several CTAs ([2] = [1] where nothing is waited for)
 *   [3] ... when its carries (tile boundaries) were formed
 *   [4] ... when its ancestors were written
 *   [5] CTA index   [6] filter (batched; 0 otherwise)
 *   [7] tiles owned (single launch) or the item's tile code (batched)
 * All CTAs read the same timer, so the records of one call share a time base.
 *   buf       device memory of capacity * PF_TRACE_WORDS * 8 bytes, caller
 *             owned and kept alive while set; NULL turns tracing off.
 *   capacity  records; those past it are not written (>= 0).
 * Each call writes from record 0 over what the previous one left; read buf
 * after synchronising the call's stream.  Concurrent calls on several streams
 * share the buffer.  Errors: PF_ERR_INVALID for capacity < 0, a misaligned
 * buf (8 bytes), or a non-NULL buf with capacity 0.
 */
#define PF_TRACE_WORDS 8
pf_status pf_set_trace_buffer(uint64_t* buf, int64_t capacity);

/*
 * Diagnostic (not part of the method): the rate, in reads per second, of
 * random 4-byte reads from buf[0..n) once it is resident in L2.  This is the
 * ceiling of the Metropolis resampler when the log-weights live in L2 (one
 * random read per chain step).  Runs on the legacy default stream and blocks
 * until done; buf (device, 4-byte aligned, n floats, finite values) is only
 * read.  reads_per_thread >= 8.
 */
pf_status pf_probe_l2_random_reads(const float* buf, int64_t n, int reads_per_thread, double* reads_per_second);

/*
 * Diagnostic (the arithmetic of the tile scans, Section 2's weights): the
 * weights the cumulative resamplers and pf_ess form inside a tile whose
 * reference exponent is k, weights[i] = exp(logw[i] - k ln 2): the
 * subtraction of k ln 2 (held as a float pair) is error-free (TwoSum), its
 * remainder enters to first order, and the exponential is expf.  For testing
 * that arithmetic against an exact exp.
 *   logw, weights  [n] float, device, 4-byte aligned;  |k| <= 2^24
 * Asynchronous on `stream`.  PF_ERR_INVALID for bad arguments.
 */
pf_status pf_debug_tile_weights(const float* logw, int64_t n, int k, float* weights, void* stream);

/* Largest P accepted by pf_resample_multinomial_static. */
#define PF_STATIC_MAX_PARTICLES (1LL << 20)

/*
 * Multinomial resampling that allocates nothing.  (The paper has no
 * counterpart; this is a deployment variant of pf_resample_multinomial.)
 *
 * For callers that cannot let a library allocate device memory -- code whose
 * allocator owns all device memory, real-time loops where a first-call
 * cudaMalloc (which also synchronises the device) would stall a deadline, or
 * programs that forbid allocation after start-up.  It gives exactly the
 * ancestors pf_resample_multinomial gives (same random streams, same search
 * predicate), by the single-launch multinomial kernel with a plain binary
 * search per draw rather than the windowed draws of pf_resample_multinomial
 * (tile lookup, then 16-entry window reads of the cumulative weights), and
 * keeps its scratch in a fixed array compiled into the library:
 * PF_STATIC_MAX_PARTICLES floats of cumulative weights (4 MiB) plus 256 bytes of
 * control words and 16 KiB of tile records, present on every GPU that loads
 * the library until the process exits.
 *   logw          [P] float, device, 16-byte aligned               (in)
 *   P             1 <= P <= PF_STATIC_MAX_PARTICLES; larger P returns
 *                 PF_ERR_INVALID without doing anything
 *   seed          Philox key
 *   ancestors     [P] int32, device, 16-byte aligned               (out)
 *   device_status [1] uint32, device, or NULL: receives this call's
 *                 device-side status (0 = ok, else a pf_status code)  (out)
 * No cudaMalloc, cudaFree or other allocating call is made by the library.
 * The first call on each device is a set-up call: it looks up the array's
 * device address (cudaGetSymbolAddress) and the kernel's launch limits, and
 * CUDA may load the library's device code on that device then, which can
 * allocate and synchronise inside the driver; make it at start-up, outside
 * any deadline and before capturing any stream into a CUDA graph.  Every call
 * on every stream shares the one array and it keeps the previous call's
 * contents, so calls that may overlap on the GPU (different streams without
 * ordering between them) race and give wrong results: order them, or use
 * pf_resample_multinomial, whose scratch is per stream.  The device-side wait
 * limit is the one pf_set_wait_limit_ns sets.  pf_get_device_status does not
 * see this call's errors; use device_status.
 */
pf_status pf_resample_multinomial_static(const float* logw, int64_t P, uint64_t seed, int32_t* ancestors,
                                         uint32_t* device_status, void* stream);

/* Library version, major*10000 + minor*100 + patch. */
int pf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PF_H_ */
