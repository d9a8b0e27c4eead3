/*
 * pf_lg.h -- whole steps of a batch of bootstrap particle filters on a
 * linear-Gaussian test model (libpf.so).
 *
 * The bootstrap filter of Section 1 of Murray, "GPU acceleration of the
 * particle filter: the Metropolis resampler": (1) draw the initial particles,
 * then at each time t (2) propagate every particle through the transition
 * density, (3) weight it by the observation density, (4) resample.  The
 * model, in D independent dimensions and for each filter f of a batch
 * (one filter per parameter set, as in particle MCMC):
 *     x_0 ~ N(m0, p0 I),   x_t = a_f x_{t-1} + N(0, q I),   y_t = x_t + N(0, r I).
 * Its exact marginal likelihood log p(y_{1:T}) is given by the Kalman
 * filter, which makes the whole filter checkable.
 *
 * Layout (all DEVICE pointers, caller-owned, F filters of P particles):
 *   x        [F][P][D] float, row-major, 16-byte aligned, D a multiple of 4
 *   logw     [F][P]    float, the accumulated log-weights
 *   loglik   [F] double  running estimate of log p(y_{1:t})
 *   log_sum  [F] double  log sum_j exp(logw[f][j]) after the last step
 *   ess      [F] float   effective sample size (sum w)^2 / sum w^2 of logw
 *   resample [F] int32   1 if filter f resamples before the next step
 * Each step reads the ancestors that pf_resample_batched_masked(kind, logw,
 * offsets = {0, P, 2P, ...}, F, B, seeds, resample, ancestors) wrote for the
 * filters with resample[f] = 1; a step is those two calls, and a run of T
 * steps can be captured in one CUDA graph once pf_reserve(P, F*P, F, stream)
 * has sized the workspace of the capturing stream.
 *
 * Noise: Philox-4x32-10 with key = seed and counter (j, t*(D/4) + g, f, 6)
 * for particle j, dimension group g (t = 0 for the initial draw); the four
 * words give N(0,1) draws for dimensions 4g..4g+3 by the Box-Muller
 * transform: words (0,1) -> sqrt(-2 ln u(w0)) (cos, sin)(2 pi u(w1)), words
 * (2,3) likewise, with u = u23 of pf.h.  The device evaluates the sine and
 * cosine in hardware on the angle reduced to (-pi, pi): each draw is within
 * about 6e-7 sqrt(-2 ln u(w0)) of the exact value.
 *
 * This model is test infrastructure for the resampling library (the paper
 * gives the filter, not this model); the library's resampling calls do not
 * depend on it.
 */
#ifndef PF_LG_H_
#define PF_LG_H_

#include <stdint.h>

#include "pf.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Step 1: x[f][j] = m0 + sqrt(p0) z with z the draws of counter (j, g, f, 6);
 * logw = 0; loglik = 0; log_sum = log P; ess = P; resample = 0.
 *   1 <= F <= 2^24, 1 <= P <= 2^31 - 1, F*P <= 2^40, D in {4, 8, ..., 64}.
 * Errors: PF_ERR_INVALID for shapes out of range, p0 < 0, non-finite m0 or
 * p0, null or misaligned pointers (x 16-byte, the others their element size).
 */
pf_status pf_lg_init(int F, int64_t P, int D, float m0, float p0, uint64_t seed, float* x, float* logw,
                     double* loglik, double* log_sum, float* ess, int32_t* resample, void* stream);

/*
 * Steps 2-3 at time t >= 1, and the resampling decision for step 4.  For
 * every filter f, with R = resample[f] as it is on entry:
 *   src_j        = R ? ancestors[f*P + j] : j
 *   x_next[f][j] = a[f] x_prev[f][src_j] + sqrt(q) z_j            (noise of time t)
 *   logw[f][j]   = (R ? 0 : logw[f][j]) + sum_d log N(y[f][d]; x_next[f][j][d], r)
 *   L            = log sum_j exp(logw[f][j])
 *   loglik[f]   += L - (R ? log P : log_sum[f]);   log_sum[f] = L
 *   ess[f]       = (sum_j w_j)^2 / sum_j w_j^2;      resample[f] = ess[f] < threshold * P
 * The ancestor gather is fused into the state read.  Arithmetic is FP32 per
 * particle; each block of 1024 particles reduces to (max, sum, sum of squares)
 * relative to its max, and the last block of a filter combines them and
 * updates the FP64 scalars.
 *   a        [F] float              y [F][D] float, 16-byte aligned (y_t)
 *   q >= 0, r > 0, threshold >= 0   (finite)
 *   x_prev, x_next  [F][P][D], distinct and not overlapping
 *   ancestors [F*P] int32, filter-local indices (read only where R = 1)
 * Errors: PF_ERR_INVALID for bad shapes, parameters or pointers (returned);
 * device status PF_ERR_INVALID for an ancestor outside [0, P) (that particle
 * then propagates from itself), PF_ERR_DOMAIN for a NaN/+inf log-weight or a
 * filter whose weights are all zero.
 */
pf_status pf_lg_step(int F, int64_t P, int D, const float* a, double q, double r, double threshold,
                     const float* y, int t, uint64_t seed, const int32_t* ancestors, const float* x_prev,
                     float* x_next, float* logw, double* loglik, double* log_sum, float* ess, int32_t* resample,
                     void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PF_LG_H_ */
