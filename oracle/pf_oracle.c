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

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
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

/* Proposal indices and acceptance uniforms of Metropolis chain i, steps 0..B-1. */
void orc_metropolis_draws(uint64_t seed, uint32_t filter, int64_t P, int64_t i, int B,
                          int32_t* prop, double* unif)
{
    uint32_t key[2], ctr[4], r[4];
    seed_key(seed, key);
    for (int b = 0; b < B; b += 2) {
        ctr[0] = (uint32_t)i; ctr[1] = (uint32_t)(b / 2); ctr[2] = filter; ctr[3] = TAG_METRO;
        orc_philox4x32_10(ctr, key, r);
        prop[b] = (int32_t)orc_index(r[0], (uint32_t)P);
        unif[b] = orc_u23(r[1]);
        if (b + 1 < B) {
            prop[b + 1] = (int32_t)orc_index(r[2], (uint32_t)P);
            unif[b + 1] = orc_u23(r[3]);
        }
    }
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

/* Metropolis chains idx[0..n) only (n = P and idx = NULL runs every chain). */
int orc_metropolis_chains(const float* lw, int64_t P, int B, uint64_t seed, uint32_t filter,
                          const int64_t* idx, int64_t n, int32_t* out)
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
            orc_philox4x32_10(ctr, key, r);
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
