/*
 * Reference oracle for the resampling stage of the bootstrap particle filter
 * (Murray, "GPU acceleration of the particle filter: the Metropolis resampler").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded,
 * FP64 statement of what the GPU library computes.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product path never calls it and never falls back to it.  It shares no code,
 * header, table or constant generator with the CUDA sources: its Philox
 * generator is written here, independently, from Salmon et al., "Parallel
 * random numbers: as easy as 1, 2, 3" (SC'11).
 *
 * Conventions (the paper's pseudocode listing is not available, so these are
 * the standard definitions the paper's prose and Figure 1 point to):
 *   lw[i]   FP32 log-weights, widened to double here.
 *   m       max_i lw[i];  w_i = exp(lw_i - m);  c_i = w_0 + ... + w_i;
 *   W       c_{P-1}, the last inclusive prefix (not a separate reduction).
 *   a_j     ancestor of offspring slot j, 0-based; o_i = #{j : a_j = i}.
 * Every cumulative search takes the smallest i with c_i > t, so that particle i
 * owns the half-open interval [c_{i-1}, c_i) and zero-weight particles are
 * never selected.
 *
 * Random streams (shared layout with the GPU library, implemented twice):
 *   key     = (seed mod 2^32, seed div 2^32)
 *   counter = (c0, c1, filter, tag); tags SYS=1, STRAT=2, MULTI=3, METRO=4.
 *   element streams (SYS, STRAT, MULTI): draw j is word j%4 of counter (j/4, 0).
 *   Metropolis chain i, steps b and b+1 (b even): counter (i, b/2) gives the
 *   words (index_b, uniform_b, index_{b+1}, uniform_{b+1}).
 *   u23(x) = (2*(x>>9)+1) * 2^-24   (exact in float and double, in (0,1))
 *   u32(x) = (2*x+1) * 2^-33        (multinomial draws; exact in double)
 *   index(x, P) = floor(x * P / 2^32)
 *
 * Build: gcc -O2 -ffp-contract=off -shared -fPIC pf_oracle.c -lm
 * (-ffp-contract=off keeps every product and sum rounded as written, so the
 * oracle gives the same bits on x86-64 and AArch64.)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_OK = 0, ORC_ERR_INVALID = 1, ORC_ERR_DOMAIN = 2 };
enum { TAG_SYS = 1, TAG_STRAT = 2, TAG_MULTI = 3, TAG_METRO = 4 };

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10 (Salmon et al., SC'11, Section 4): ten rounds of two       */
/* 32x32->64 multiplications whose halves are permuted and xored with the   */
/* counter and round key; the key is bumped by the Weyl constants between   */
/* rounds.                                                                   */
/* ------------------------------------------------------------------------ */
#define PHILOX_MUL_A 0xD2511F53u
#define PHILOX_MUL_B 0xCD9E8D57u
#define PHILOX_WEYL_A 0x9E3779B9u
#define PHILOX_WEYL_B 0xBB67AE85u

/* The same generator with `rounds` rounds (SC'11, Table 2 lists Philox-4x32-7  */
/* among its Crush-resistant members; 10 is the recommended default).          */
void orc_philox4x32_r(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4], int rounds)
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < rounds; ++round) {
        uint64_t pa = (uint64_t)PHILOX_MUL_A * x0;
        uint64_t pb = (uint64_t)PHILOX_MUL_B * x2;
        uint32_t pa_hi = (uint32_t)(pa >> 32), pa_lo = (uint32_t)pa;
        uint32_t pb_hi = (uint32_t)(pb >> 32), pb_lo = (uint32_t)pb;
        uint32_t y0 = pb_hi ^ x1 ^ k0;
        uint32_t y1 = pb_lo;
        uint32_t y2 = pa_hi ^ x3 ^ k1;
        uint32_t y3 = pa_lo;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += PHILOX_WEYL_A;
        k1 += PHILOX_WEYL_B;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    orc_philox4x32_r(ctr, key, out, 10);
}

static void seed_key(uint64_t seed, uint32_t key[2])
{
    key[0] = (uint32_t)(seed & 0xffffffffu);
    key[1] = (uint32_t)(seed >> 32);
}

double orc_u23(uint32_t x) { return (2.0 * (double)(x >> 9) + 1.0) * 0x1p-24; }
double orc_u32(uint32_t x) { return (2.0 * (double)x + 1.0) * 0x1p-33; }
uint32_t orc_index(uint32_t x, uint32_t P) { return (uint32_t)(((uint64_t)x * P) >> 32); }

/* Raw words of an element stream: draw j is word j%4 of counter (j/4, 0, filter, tag). */
void orc_stream_words(uint64_t seed, uint32_t filter, uint32_t tag, int64_t n, uint32_t* out)
{
    uint32_t key[2], ctr[4], r[4];
    seed_key(seed, key);
    for (int64_t q = 0; q * 4 < n; ++q) {
        ctr[0] = (uint32_t)q; ctr[1] = 0; ctr[2] = filter; ctr[3] = tag;
        orc_philox4x32_10(ctr, key, r);
        for (int s = 0; s < 4 && q * 4 + s < n; ++s) out[q * 4 + s] = r[s];
    }
}

/* Uniform draws of an element stream, converted with u23 (kind 0) or u32 (kind 1). */
void orc_stream_uniforms(uint64_t seed, uint32_t filter, uint32_t tag, int64_t n, int kind, double* out)
{
    uint32_t key[2], ctr[4], r[4];
    seed_key(seed, key);
    for (int64_t q = 0; q * 4 < n; ++q) {
        ctr[0] = (uint32_t)q; ctr[1] = 0; ctr[2] = filter; ctr[3] = tag;
        orc_philox4x32_10(ctr, key, r);
        for (int s = 0; s < 4 && q * 4 + s < n; ++s)
            out[q * 4 + s] = kind ? orc_u32(r[s]) : orc_u23(r[s]);
    }
}

/* Proposal indices and acceptance uniforms of Metropolis chain i, steps 0..B-1, */
/* from Philox-4x32 with `rounds` rounds (10: the library's default stream).     */
void orc_metropolis_draws_r(uint64_t seed, uint32_t filter, int64_t P, int64_t i, int B, int rounds,
                            int32_t* prop, double* unif)
{
    uint32_t key[2], ctr[4], r[4];
    seed_key(seed, key);
    for (int b = 0; b < B; b += 2) {
        ctr[0] = (uint32_t)i; ctr[1] = (uint32_t)(b / 2); ctr[2] = filter; ctr[3] = TAG_METRO;
        orc_philox4x32_r(ctr, key, r, rounds);
        prop[b] = (int32_t)orc_index(r[0], (uint32_t)P);
        unif[b] = orc_u23(r[1]);
        if (b + 1 < B) {
            prop[b + 1] = (int32_t)orc_index(r[2], (uint32_t)P);
            unif[b + 1] = orc_u23(r[3]);
        }
    }
}

void orc_metropolis_draws(uint64_t seed, uint32_t filter, int64_t P, int64_t i, int B,
                          int32_t* prop, double* unif)
{
    orc_metropolis_draws_r(seed, filter, P, i, B, 10, prop, unif);
}

/* ------------------------------------------------------------------------ */
/* Weights (Section 1, step 4: weights are unnormalised probabilities).      */
/* ------------------------------------------------------------------------ */
static int check_domain(const float* lw, int64_t P)
{
    for (int64_t i = 0; i < P; ++i) {
        float v = lw[i];
        if (v != v || v == INFINITY) return ORC_ERR_DOMAIN;
    }
    return ORC_OK;
}

static double max_logw(const float* lw, int64_t P)
{
    double m = -INFINITY;
    for (int64_t i = 0; i < P; ++i)
        if ((double)lw[i] > m) m = (double)lw[i];
    return m;
}

/* Inclusive prefix sums c_i of w_i = exp(lw_i - m), left to right. */
static int cumulative_weights(const float* lw, int64_t P, double* c, double* m_out)
{
    if (check_domain(lw, P)) return ORC_ERR_DOMAIN;
    double m = max_logw(lw, P);
    if (m == -INFINITY) return ORC_ERR_DOMAIN; /* every weight is zero */
    double run = 0.0;
    for (int64_t i = 0; i < P; ++i) {
        double w = exp((double)lw[i] - m);
        run += w;
        c[i] = run;
    }
    if (m_out) *m_out = m;
    return ORC_OK;
}

/* theta_i = c_i / W, the normalised inclusive cumulative weights. */
int orc_normalised_cumsum(const float* lw, int64_t P, double* theta)
{
    if (P < 1) return ORC_ERR_INVALID;
    int st = cumulative_weights(lw, P, theta, NULL);
    if (st) return st;
    double W = theta[P - 1];
    for (int64_t i = 0; i < P; ++i) theta[i] /= W;
    return ORC_OK;
}

/* log W + m = log sum_i exp(lw_i), and the effective sample size
 * (sum w)^2 / sum w^2 (the standard ESS; the paper quotes ESS values in
 * Section 3 without the formula). */
int orc_ess(const float* lw, int64_t P, double* ess, double* log_sum)
{
    if (P < 1) return ORC_ERR_INVALID;
    if (check_domain(lw, P)) return ORC_ERR_DOMAIN;
    double m = max_logw(lw, P);
    if (m == -INFINITY) return ORC_ERR_DOMAIN;
    double s = 0.0, q = 0.0;
    for (int64_t i = 0; i < P; ++i) {
        double w = exp((double)lw[i] - m);
        s += w;
        q += w * w;
    }
    if (ess) *ess = s * s / q;
    if (log_sum) *log_sum = m + log(s);
    return ORC_OK;
}

/* Smallest i >= start with c[i] > t; if rounding leaves none, the last index
 * with positive weight (a zero-weight particle is never returned). */
static int64_t walk_to(const double* c, int64_t P, int64_t start, double t)
{
    int64_t i = start;
    while (i < P && c[i] <= t) ++i;
    if (i == P) {
        i = P - 1;
        while (i > 0 && c[i] == c[i - 1]) --i;
    }
    return i;
}

/* Smallest i with c[i] > t, by bisection over the whole range. */
static int64_t search(const double* c, int64_t P, double t)
{
    int64_t lo = 0, hi = P; /* answer in [lo, hi] */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (c[mid] > t) hi = mid; else lo = mid + 1;
    }
    if (lo == P) {
        lo = P - 1;
        while (lo > 0 && c[lo] == c[lo - 1]) --lo;
    }
    return lo;
}

/* ------------------------------------------------------------------------ */
/* Systematic resampler (Figure 1c; Kitagawa 1996): one offset u shared by   */
/* every stratum [j/P, (j+1)/P); offspring slot j takes the particle whose   */
/* cumulative interval holds (j+u) W / P.                                    */
/* ------------------------------------------------------------------------ */
int orc_systematic_u(const float* lw, int64_t P, double u, int32_t* anc)
{
    if (P < 1) return ORC_ERR_INVALID;
    double* c = (double*)malloc(sizeof(double) * (size_t)P);
    if (!c) return ORC_ERR_INVALID;
    int st = cumulative_weights(lw, P, c, NULL);
    if (st) { free(c); return st; }
    double W = c[P - 1];
    int64_t i = 0;
    for (int64_t j = 0; j < P; ++j) {
        double t = ((double)j + u) * W / (double)P;
        i = walk_to(c, P, i, t);
        anc[j] = (int32_t)i;
    }
    free(c);
    return ORC_OK;
}

/* Stratified resampler (Figure 1b): as systematic, but stratum j draws its
 * own offset u_j. */
int orc_stratified_u(const float* lw, int64_t P, const double* u, int32_t* anc)
{
    if (P < 1) return ORC_ERR_INVALID;
    double* c = (double*)malloc(sizeof(double) * (size_t)P);
    if (!c) return ORC_ERR_INVALID;
    int st = cumulative_weights(lw, P, c, NULL);
    if (st) { free(c); return st; }
    double W = c[P - 1];
    int64_t i = 0;
    for (int64_t j = 0; j < P; ++j) {
        double t = ((double)j + u[j]) * W / (double)P;
        i = walk_to(c, P, i, t);
        anc[j] = (int32_t)i;
    }
    free(c);
    return ORC_OK;
}

/* Multinomial resampler (Figure 1a): P independent uniforms, each located by
 * binary search in the cumulative weights (Section 3). Output in draw order. */
int orc_multinomial_u(const float* lw, int64_t P, const double* u, int32_t* anc)
{
    if (P < 1) return ORC_ERR_INVALID;
    double* c = (double*)malloc(sizeof(double) * (size_t)P);
    if (!c) return ORC_ERR_INVALID;
    int st = cumulative_weights(lw, P, c, NULL);
    if (st) { free(c); return st; }
    double W = c[P - 1];
    for (int64_t j = 0; j < P; ++j) anc[j] = (int32_t)search(c, P, u[j] * W);
    free(c);
    return ORC_OK;
}

/* One Metropolis decision (Section 2): move from k to the proposal j when
 * w_j >= w_k, else with probability w_j / w_k, i.e. when u < exp(lw_j - lw_k).
 * Comparing the log-weights first also defines the zero-weight cases
 * (-inf >= -inf moves; a zero-weight proposal from a positive one never does). */
static int metropolis_accept(double lw_j, double lw_k, double u)
{
    if (lw_j >= lw_k) return 1;
    return u < exp(lw_j - lw_k);
}

/* Metropolis resampler (Figure 1d, Section 2): chain i starts at k = i and
 * takes B steps with uniform proposals over all P indices (a proposal of k
 * itself is a no-op); a_i is the final state.  Draws are given explicitly:
 * prop[i*B + b], unif[i*B + b]. */
int orc_metropolis_u(const float* lw, int64_t P, int B, const int32_t* prop, const double* unif,
                     int32_t* anc)
{
    if (P < 1 || B < 0) return ORC_ERR_INVALID;
    if (check_domain(lw, P)) return ORC_ERR_DOMAIN;
    for (int64_t i = 0; i < P; ++i) {
        int64_t k = i;
        for (int b = 0; b < B; ++b) {
            int64_t j = prop[i * (int64_t)B + b];
            if (metropolis_accept((double)lw[j], (double)lw[k], unif[i * (int64_t)B + b])) k = j;
        }
        anc[i] = (int32_t)k;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* The same four resamplers driven by the Philox streams.                    */
/* ------------------------------------------------------------------------ */
int orc_systematic(const float* lw, int64_t P, uint64_t seed, uint32_t filter, int32_t* anc)
{
    if (P < 1) return ORC_ERR_INVALID;
    double u;
    orc_stream_uniforms(seed, filter, TAG_SYS, 1, 0, &u);
    return orc_systematic_u(lw, P, u, anc);
}

int orc_stratified(const float* lw, int64_t P, uint64_t seed, uint32_t filter, int32_t* anc)
{
    if (P < 1) return ORC_ERR_INVALID;
    double* u = (double*)malloc(sizeof(double) * (size_t)P);
    if (!u) return ORC_ERR_INVALID;
    orc_stream_uniforms(seed, filter, TAG_STRAT, P, 0, u);
    int st = orc_stratified_u(lw, P, u, anc);
    free(u);
    return st;
}

int orc_multinomial(const float* lw, int64_t P, uint64_t seed, uint32_t filter, int32_t* anc)
{
    if (P < 1) return ORC_ERR_INVALID;
    double* u = (double*)malloc(sizeof(double) * (size_t)P);
    if (!u) return ORC_ERR_INVALID;
    orc_stream_uniforms(seed, filter, TAG_MULTI, P, 1, u);
    int st = orc_multinomial_u(lw, P, u, anc);
    free(u);
    return st;
}

/* Metropolis chains idx[0..n) only (n = P and idx = NULL runs every chain), */
/* their draws from Philox-4x32 with `rounds` rounds.                        */
int orc_metropolis_chains_r(const float* lw, int64_t P, int B, uint64_t seed, uint32_t filter,
                            const int64_t* idx, int64_t n, int rounds, int32_t* out)
{
    if (P < 1 || B < 0) return ORC_ERR_INVALID;
    if (check_domain(lw, P)) return ORC_ERR_DOMAIN;
    uint32_t key[2], ctr[4], r[4];
    seed_key(seed, key);
    for (int64_t q = 0; q < n; ++q) {
        int64_t i = idx ? idx[q] : q;
        int64_t k = i;
        for (int b = 0; b < B; b += 2) {
            ctr[0] = (uint32_t)i; ctr[1] = (uint32_t)(b / 2); ctr[2] = filter; ctr[3] = TAG_METRO;
            orc_philox4x32_r(ctr, key, r, rounds);
            int64_t j = orc_index(r[0], (uint32_t)P);
            if (metropolis_accept((double)lw[j], (double)lw[k], orc_u23(r[1]))) k = j;
            if (b + 1 < B) {
                j = orc_index(r[2], (uint32_t)P);
                if (metropolis_accept((double)lw[j], (double)lw[k], orc_u23(r[3]))) k = j;
            }
        }
        out[q] = (int32_t)k;
    }
    return ORC_OK;
}

int orc_metropolis_chains(const float* lw, int64_t P, int B, uint64_t seed, uint32_t filter,
                          const int64_t* idx, int64_t n, int32_t* out)
{
    return orc_metropolis_chains_r(lw, P, B, seed, filter, idx, n, 10, out);
}

int orc_metropolis(const float* lw, int64_t P, int B, uint64_t seed, uint32_t filter, int32_t* anc)
{
    return orc_metropolis_chains(lw, P, B, seed, filter, NULL, P, anc);
}

/* ------------------------------------------------------------------------ */
/* Ancestor gather (Section 1, step 4: the redrawn samples).                 */
/* ------------------------------------------------------------------------ */
int orc_gather(const void* src, int64_t P_src, int64_t row_bytes, const int32_t* anc, int64_t P_dst,
               void* dst)
{
    for (int64_t j = 0; j < P_dst; ++j) {
        if (anc[j] < 0 || anc[j] >= P_src) return ORC_ERR_INVALID;
        memcpy((char*)dst + j * row_bytes, (const char*)src + (int64_t)anc[j] * row_bytes,
               (size_t)row_bytes);
    }
    return ORC_OK;
}

/* Offspring counts o_i = #{j : a_j = i} (Section 2). */
void orc_offspring(const int32_t* anc, int64_t n_anc, int64_t P, int64_t* o)
{
    for (int64_t i = 0; i < P; ++i) o[i] = 0;
    for (int64_t j = 0; j < n_anc; ++j) o[anc[j]] += 1;
}

/* ------------------------------------------------------------------------ */
/* Metropolis transition matrix and the bound on B (Section 2, Eqs. 1-5).    */
/* ------------------------------------------------------------------------ */

/* One-step transition matrix of a single chain, row-major P x P:
 * M[k][j] = (1/P) * acceptance(k -> j) for j != k, M[k][k] = 1 - sum. */
int orc_metropolis_matrix(const float* lw, int64_t P, double* M)
{
    if (P < 1) return ORC_ERR_INVALID;
    if (check_domain(lw, P)) return ORC_ERR_DOMAIN;
    for (int64_t k = 0; k < P; ++k) {
        double off = 0.0;
        for (int64_t j = 0; j < P; ++j) {
            if (j == k) continue;
            double a = ((double)lw[j] >= (double)lw[k]) ? 1.0 : exp((double)lw[j] - (double)lw[k]);
            M[k * P + j] = a / (double)P;
            off += M[k * P + j];
        }
        M[k * P + k] = 1.0 - off;
    }
    return ORC_OK;
}

/* Smallest B with lambda^B <= eps (alpha+beta) / max(alpha, beta) for the 0-1
 * process "chain sits on the heaviest particle" (Eqs. 1-5), where
 * beta = 1/P (the heaviest particle is proposed with probability 1/P and
 * always accepted), alpha = (1 - w_max) / (P w_max), lambda = 1 - alpha - beta.
 * The ratio (alpha+beta)/max(alpha,beta) equals 1/max(w_max, 1-w_max), so the
 * bound is symmetric in which state is labelled 1.  Returns 0 when no steps
 * are needed, -1 for invalid arguments. */
int64_t orc_metropolis_B(int64_t P, double w_max, double eps)
{
    if (P < 1 || !(w_max > 0.0) || w_max > 1.0 || !(eps > 0.0)) return -1;
    double beta = 1.0 / (double)P;
    double alpha = (1.0 - w_max) / ((double)P * w_max);
    double lambda = 1.0 - alpha - beta;
    double target = eps * (alpha + beta) / (alpha > beta ? alpha : beta);
    if (target >= 1.0) return 0;      /* already within eps after 0 steps */
    if (lambda <= 0.0) return 1;      /* one step mixes exactly (or overshoots) */
    double B = log(target) / log(lambda);
    double Bc = ceil(B);
    /* guard the ceiling against a rounding of the quotient just above an integer */
    if (Bc - 1.0 >= 0.0 && pow(lambda, Bc - 1.0) <= target) Bc -= 1.0;
    return (int64_t)Bc;
}

/* Batched: F independent filters; filter f owns lw[off[f] .. off[f+1]) and its
 * ancestors are filter-local. kind: 0 multinomial, 1 stratified, 2 systematic,
 * 3 Metropolis (B steps). Filter f uses seed seeds[f] and filter id f. */
int orc_batched(int kind, const float* lw, const int64_t* off, int F, int B, const uint64_t* seeds,
                int32_t* anc)
{
    for (int f = 0; f < F; ++f) {
        int64_t P = off[f + 1] - off[f];
        if (P < 1) continue;
        const float* l = lw + off[f];
        int32_t* a = anc + off[f];
        int st;
        switch (kind) {
        case 0: st = orc_multinomial(l, P, seeds[f], (uint32_t)f, a); break;
        case 1: st = orc_stratified(l, P, seeds[f], (uint32_t)f, a); break;
        case 2: st = orc_systematic(l, P, seeds[f], (uint32_t)f, a); break;
        case 3: st = orc_metropolis(l, P, B, seeds[f], (uint32_t)f, a); break;
        default: return ORC_ERR_INVALID;
        }
        if (st) return st;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Exact log-likelihood of the linear-Gaussian test model used to check a    */
/* whole bootstrap filter (Section 1, steps 1-4): in each of D independent   */
/* dimensions, x_0 ~ N(m0, p0), x_t = a x_{t-1} + N(0, q), y_t = x_t +       */
/* N(0, r).  The Kalman filter gives log p(y_{1:T}) in closed form.          */
/* y is T x D, row-major.                                                    */
/* ------------------------------------------------------------------------ */
double orc_kalman_loglik(double a, double q, double r, double m0, double p0, const double* y, int T, int D)
{
    const double two_pi = 6.283185307179586476925286766559;
    double ll = 0.0;
    for (int d = 0; d < D; ++d) {
        double m = m0, p = p0;
        for (int t = 0; t < T; ++t) {
            /* predict */
            double mp = a * m;
            double pp = a * a * p + q;
            /* observe */
            double s = pp + r;
            double e = y[t * D + d] - mp;
            ll += -0.5 * (log(two_pi * s) + e * e / s);
            /* update */
            double k = pp / s;
            m = mp + k * e;
            p = (1.0 - k) * pp;
        }
    }
    return ll;
}

/* ------------------------------------------------------------------------ */
/* Bootstrap filter on the linear-Gaussian test model (Section 1, steps      */
/* 1-4), one filter per parameter set f:                                     */
/*   x_0 ~ N(m0, p0 I),  x_t = a_f x_{t-1} + N(0, q I),  y_t = x_t + N(0,rI) */
/* in D dimensions (D a multiple of 4).  States are [F][P][D], log-weights   */
/* [F][P], observations of one time [F][D].                                  */
/*                                                                           */
/* Noise of particle j, time t, dimension group g: Philox counter            */
/* (j, t*(D/4) + g, f, TAG_PROPAGATE) with key = seed; its words (w0..w3)    */
/* give four N(0,1) draws by the Box-Muller transform (Box & Muller 1958):   */
/*   z_{4g}   = sqrt(-2 ln u(w0)) cos(2 pi u(w1)),                           */
/*   z_{4g+1} = sqrt(-2 ln u(w0)) sin(2 pi u(w1)),  likewise (w2, w3).       */
/* ------------------------------------------------------------------------ */
#define TAG_PROPAGATE 6u

void orc_lg_normals(uint64_t seed, uint32_t f, uint32_t j, uint32_t c1, double z[4])
{
    const double two_pi = 6.283185307179586476925286766559;
    uint32_t key[2], ctr[4], w[4];
    seed_key(seed, key);
    ctr[0] = j; ctr[1] = c1; ctr[2] = f; ctr[3] = TAG_PROPAGATE;
    orc_philox4x32_10(ctr, key, w);
    for (int h = 0; h < 2; ++h) {
        double rad = sqrt(-2.0 * log(orc_u23(w[2 * h])));
        double ang = two_pi * orc_u23(w[2 * h + 1]);
        z[2 * h] = rad * cos(ang);
        z[2 * h + 1] = rad * sin(ang);
    }
}

/* Step 1: initial particles and filter scalars. */
int orc_lg_init(int F, int64_t P, int D, double m0, double p0, uint64_t seed, double* x, double* lw,
                double* loglik, double* log_sum, double* ess, int32_t* resample)
{
    if (F < 1 || P < 1 || D < 4 || D % 4 || p0 < 0) return ORC_ERR_INVALID;
    double z[4];
    for (int f = 0; f < F; ++f) {
        for (int64_t j = 0; j < P; ++j) {
            for (int g = 0; g < D / 4; ++g) {
                orc_lg_normals(seed, (uint32_t)f, (uint32_t)j, (uint32_t)g, z);
                for (int c = 0; c < 4; ++c)
                    x[((size_t)f * P + j) * D + 4 * g + c] = m0 + sqrt(p0) * z[c];
            }
            lw[(size_t)f * P + j] = 0.0;
        }
        loglik[f] = 0.0;
        log_sum[f] = log((double)P);
        ess[f] = (double)P;
        resample[f] = 0;
    }
    return ORC_OK;
}

/* log sum_j exp(v_j) and (sum w)^2 / sum w^2 of one filter's log-weights. */
static int lse_ess_d(const double* v, int64_t P, double* lse, double* ess)
{
    double m = -INFINITY;
    for (int64_t j = 0; j < P; ++j) {
        if (v[j] != v[j] || v[j] == INFINITY) return ORC_ERR_DOMAIN;
        if (v[j] > m) m = v[j];
    }
    if (m == -INFINITY) return ORC_ERR_DOMAIN;
    double s = 0.0, s2 = 0.0;
    for (int64_t j = 0; j < P; ++j) {
        double w = exp(v[j] - m);
        s += w;
        s2 += w * w;
    }
    *lse = m + log(s);
    *ess = s * s / s2;
    return ORC_OK;
}

/* Steps 2-3 at time t and the resampling decision, for every filter f, with
 * R = resample_in[f]: particle j continues from src_j = R ? anc[f*P+j] : j,
 *   x_next = a_f x_prev[src_j] + sqrt(q) z,
 *   lw_out = (R ? 0 : lw_in) + sum_d log N(y_d; x_next_d, r),
 * then L = log sum exp(lw_out), loglik += L - (R ? log P : log_sum_in),
 * ess = (sum w)^2 / sum w^2 and resample_out = (ess < threshold P).
 * Inputs are the FP32 values a caller holds; everything else is FP64. */
int orc_lg_step(int F, int64_t P, int D, const float* a, double q, double r, double threshold,
                const float* y, int t, uint64_t seed, const int32_t* anc, const float* x_prev,
                const float* lw_in, const int32_t* resample_in, const double* log_sum_in,
                const double* loglik_in, double* x_next, double* lw_out, double* loglik_out,
                double* log_sum_out, double* ess_out, int32_t* resample_out)
{
    const double two_pi = 6.283185307179586476925286766559;
    if (F < 1 || P < 1 || D < 4 || D % 4 || q < 0 || r <= 0 || t < 1) return ORC_ERR_INVALID;
    const int G = D / 4;
    double z[4];
    for (int f = 0; f < F; ++f) {
        const int R = resample_in[f];
        for (int64_t j = 0; j < P; ++j) {
            int64_t src = j;
            if (R) {
                src = anc[(size_t)f * P + j];
                if (src < 0 || src >= P) return ORC_ERR_INVALID;
            }
            double logg = 0.0;
            for (int g = 0; g < G; ++g) {
                orc_lg_normals(seed, (uint32_t)f, (uint32_t)j, (uint32_t)(t * G + g), z);
                for (int c = 0; c < 4; ++c) {
                    const int d = 4 * g + c;
                    double xn = (double)a[f] * (double)x_prev[((size_t)f * P + src) * D + d] + sqrt(q) * z[c];
                    x_next[((size_t)f * P + j) * D + d] = xn;
                    double e = (double)y[(size_t)f * D + d] - xn;
                    logg += -0.5 * log(two_pi * r) - e * e / (2.0 * r);
                }
            }
            double prev = R ? 0.0 : (double)lw_in[(size_t)f * P + j];
            lw_out[(size_t)f * P + j] = prev + logg;
        }
        double L, e;
        int st = lse_ess_d(lw_out + (size_t)f * P, P, &L, &e);
        if (st) return st;
        double L_prev = R ? log((double)P) : log_sum_in[f];
        loglik_out[f] = loglik_in[f] + (L - L_prev);
        log_sum_out[f] = L;
        ess_out[f] = e;
        resample_out[f] = e < threshold * (double)P;
    }
    return ORC_OK;
}

/* Resampling of one filter with FP64 log-weights: kind 2 systematic,
 * 1 stratified, 0 multinomial, same streams and searches as the FP32-input
 * resamplers above. */
static int resample_d(int kind, const double* v, int64_t P, uint64_t seed, uint32_t f, int32_t* anc, double* c,
                      double* u)
{
    double m = -INFINITY;
    for (int64_t i = 0; i < P; ++i) if (v[i] > m) m = v[i];
    if (m == -INFINITY) return ORC_ERR_DOMAIN;
    double run = 0.0;
    for (int64_t i = 0; i < P; ++i) { run += exp(v[i] - m); c[i] = run; }
    const double W = c[P - 1];
    if (kind == 2) {
        orc_stream_uniforms(seed, f, TAG_SYS, 1, 0, u);
        int64_t i = 0;
        for (int64_t j = 0; j < P; ++j) { i = walk_to(c, P, i, ((double)j + u[0]) * W / (double)P); anc[j] = (int32_t)i; }
    } else if (kind == 1) {
        orc_stream_uniforms(seed, f, TAG_STRAT, P, 0, u);
        int64_t i = 0;
        for (int64_t j = 0; j < P; ++j) { i = walk_to(c, P, i, ((double)j + u[j]) * W / (double)P); anc[j] = (int32_t)i; }
    } else if (kind == 0) {
        orc_stream_uniforms(seed, f, TAG_MULTI, P, 1, u);
        for (int64_t j = 0; j < P; ++j) anc[j] = (int32_t)search(c, P, u[j] * W);
    } else {
        return ORC_ERR_INVALID;
    }
    return ORC_OK;
}

/* A whole run: step 1, then T times (step 4 for the filters that asked for
 * it, with key step_seeds[(t-1)*F + f] and filter id f; steps 2-3).  y is
 * [T][F][D]; loglik[f] receives the estimate of log p(y_{1:T}). */
int orc_lg_filter(int kind, int F, int64_t P, int D, const float* a, double q, double r, double m0, double p0,
                  double threshold, const float* y, int T, uint64_t seed, const uint64_t* step_seeds,
                  double* loglik)
{
    if (F < 1 || P < 1 || D < 4 || D % 4 || T < 0) return ORC_ERR_INVALID;
    const size_t n = (size_t)F * P;
    double* x = (double*)malloc(sizeof(double) * n * D);
    double* xn = (double*)malloc(sizeof(double) * n * D);
    double* lw = (double*)malloc(sizeof(double) * n);
    double* c = (double*)malloc(sizeof(double) * P);
    double* u = (double*)malloc(sizeof(double) * P);
    int32_t* anc = (int32_t*)malloc(sizeof(int32_t) * P);
    double* log_sum = (double*)malloc(sizeof(double) * F);
    double* ess = (double*)malloc(sizeof(double) * F);
    int32_t* resample = (int32_t*)malloc(sizeof(int32_t) * F);
    int st = (x && xn && lw && c && u && anc && log_sum && ess && resample) ? ORC_OK : ORC_ERR_INVALID;
    if (!st) st = orc_lg_init(F, P, D, m0, p0, seed, x, lw, loglik, log_sum, ess, resample);
    const int G = D / 4;
    const double two_pi = 6.283185307179586476925286766559;
    double z[4];
    for (int t = 1; t <= T && !st; ++t) {
        for (int f = 0; f < F && !st; ++f) {
            double* lwf = lw + (size_t)f * P;
            const int R = resample[f];
            if (R) st = resample_d(kind, lwf, P, step_seeds[(size_t)(t - 1) * F + f], (uint32_t)f, anc, c, u);
            for (int64_t j = 0; j < P && !st; ++j) {
                const int64_t src = R ? anc[j] : j;
                double logg = 0.0;
                for (int g = 0; g < G; ++g) {
                    orc_lg_normals(seed, (uint32_t)f, (uint32_t)j, (uint32_t)(t * G + g), z);
                    for (int cc = 0; cc < 4; ++cc) {
                        const int d = 4 * g + cc;
                        double v = (double)a[f] * x[((size_t)f * P + src) * D + d] + sqrt(q) * z[cc];
                        xn[((size_t)f * P + j) * D + d] = v;
                        double e = (double)y[((size_t)(t - 1) * F + f) * D + d] - v;
                        logg += -0.5 * log(two_pi * r) - e * e / (2.0 * r);
                    }
                }
                lwf[j] = (R ? 0.0 : lwf[j]) + logg;
            }
            if (st) break;
            double L, e;
            st = lse_ess_d(lwf, P, &L, &e);
            if (st) break;
            loglik[f] += L - (R ? log((double)P) : log_sum[f]);
            log_sum[f] = L;
            ess[f] = e;
            resample[f] = e < threshold * (double)P;
        }
        double* tmp = x; x = xn; xn = tmp;
    }
    free(x); free(xn); free(lw); free(c); free(u); free(anc); free(log_sum); free(ess); free(resample);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Offspring/ancestor conversion (Section 2: the stratified and systematic  */
/* schemes yield offspring counts, the others ancestors; converting is      */
/* direct) in the form that lets particles be moved in place: every        */
/* particle i with offspring keeps one of them in its own slot (out[i] = i), */
/* and the other offspring (o_i - 1 copies of each i, in increasing i) fill  */
/* the slots of the particles without offspring, in increasing slot order.   */
/* out has the same offspring counts as anc, and out[out[j]] = out[j].       */
/* ------------------------------------------------------------------------ */
int orc_permute(const int32_t* anc, int64_t P, int32_t* out)
{
    if (P < 1) return ORC_ERR_INVALID;
    int64_t* o = (int64_t*)calloc((size_t)P, sizeof(int64_t));
    if (!o) return ORC_ERR_INVALID;
    for (int64_t j = 0; j < P; ++j) {
        if (anc[j] < 0 || anc[j] >= P) { free(o); return ORC_ERR_INVALID; }
        o[anc[j]] += 1;
    }
    int64_t next_extra = 0, left = 0; /* the particle whose extra copies are being placed, and how many remain */
    while (next_extra < P && o[next_extra] <= 1) ++next_extra;
    if (next_extra < P) left = o[next_extra] - 1;
    for (int64_t i = 0; i < P; ++i) {
        if (o[i] > 0) {
            out[i] = (int32_t)i;
        } else {
            out[i] = (int32_t)next_extra;
            if (--left == 0) {
                ++next_extra;
                while (next_extra < P && o[next_extra] <= 1) ++next_extra;
                if (next_extra < P) left = o[next_extra] - 1;
            }
        }
    }
    free(o);
    return ORC_OK;
}
