/*
 * oracle.c -- plain, single-threaded CPU oracle for the particle-filter resampling step of
 * Murray, Lee & Jacob, "Parallel resampling in the particle filter".
 *
 * TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the benchmark's CPU
 * baseline may load this file's library. It shares no code, header, table or constant
 * generator with the CUDA library: every definition below is written out from the paper
 * (and, for the random numbers and the exponential, from the published methods named at
 * each function). It is deliberately slow and literal: loops in the paper's order, no
 * blocking, no SIMD, compiled with -ffp-contract=off so that every floating-point
 * operation written here is exactly one IEEE operation.
 *
 * Indexing is 0-based: particles are 0..N-1 and the Prepermute sentinel N+1 of the paper
 * (1-based) becomes N.
 *
 * Parity status: every function is pinned by the CPU test-suite against something other
 * than itself (an independent Philox implementation, libm, closed-form laws, exact rational
 * arithmetic, numpy library routines, invariants stated by the paper). None is unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_NONFINITE (-2)
#define ORC_ERR_ZERO_WEIGHT (-3)
#define ORC_ERR_BOUND_VIOLATED (-4)
#define ORC_ERR_REJECTION_CAP (-5)

/* Purpose tags of the random stream (low 3 bits of counter word 3). */
#define ORC_MULTINOMIAL 0u
#define ORC_STRATIFIED 1u
#define ORC_SYSTEMATIC 2u
#define ORC_METROPOLIS 3u
#define ORC_REJECTION 4u
#define ORC_BOUND_ESTIMATE 5u

/* ------------------------------------------------------------------------------------ */
/* Counter-based random numbers                                                           */
/* ------------------------------------------------------------------------------------ */

/* Philox4x32 with 10 rounds: Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3" (SC'11), Section 4.2. Each round multiplies counter words 0 and 2 by
 * the two round multipliers, and the new words are (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2),
 * hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)); the key is bumped by the two Weyl constants (golden
 * ratio and sqrt(3)-1, as 32-bit fractions) between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The keying of every draw of the method: key = seed, counter = (particle or stratum index,
 * inner step n, SMC time step mod 2^32, filter * 8 + purpose). */
void orc_draw(uint64_t seed, uint32_t index, uint32_t n, uint64_t step, uint32_t filter,
              uint32_t purpose, uint32_t out[4]) {
    uint32_t ctr[4] = {index, n, (uint32_t)step, (filter << 3) | (purpose & 7u)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* U[0,1) in binary32: the top 24 bits of word 0 times 2^-24 (exact). */
float orc_u01_f32(const uint32_t x[4]) { return (float)(x[0] >> 8) * 0x1p-24f; }

/* U[0,1) in binary64: word 0 and the top 21 bits of word 1 (53 bits) times 2^-53 (exact). */
double orc_u01_f64(const uint32_t x[4]) {
    uint64_t m = ((uint64_t)x[0] << 21) | (uint64_t)(x[1] >> 11);
    return (double)m * 0x1p-53;
}

/* The uniform u_k of stratum k (Code 7). One Philox block serves consecutive strata: in
 * binary32 stratum k takes the top 24 bits of word k mod 4 of counter (floor(k/4), 0), times
 * 2^-24; in binary64 words 2 (k mod 2) and 2 (k mod 2) + 1 of counter (floor(k/2), 0), as
 * orc_u01_f64 takes words 0 and 1. */
float orc_stratum_u_f32(uint64_t seed, int64_t k, uint64_t step, uint32_t filter) {
    uint32_t x[4];
    orc_draw(seed, (uint32_t)(k / 4), 0u, step, filter, ORC_STRATIFIED, x);
    return (float)(x[k % 4] >> 8) * 0x1p-24f;
}

double orc_stratum_u_f64(uint64_t seed, int64_t k, uint64_t step, uint32_t filter) {
    uint32_t x[4];
    orc_draw(seed, (uint32_t)(k / 2), 0u, step, filter, ORC_STRATIFIED, x);
    uint32_t pair[4] = {x[2 * (k % 2)], x[2 * (k % 2) + 1], 0u, 0u};
    return orc_u01_f64(pair);
}

/* Uniform index on {0..N-1}: floor(V * N / 2^64) with V = words 2,3 as a 64-bit integer. */
int64_t orc_uniform_index(const uint32_t x[4], int64_t N) {
    uint64_t v = ((uint64_t)x[2] << 32) | (uint64_t)x[3];
    unsigned __int128 p = (unsigned __int128)v * (unsigned __int128)(uint64_t)N;
    return (int64_t)(uint64_t)(p >> 64);
}

/* The binary32 Metropolis chain takes two steps from one block: step half h (0 or 1) uses
 * words 2h and 2h + 1. Its uniform is the top 24 bits of word 2h times 2^-24; its proposal is
 * floor(V * N / 2^40) with V = (the low 8 bits of word 2h) * 2^32 + word 2h + 1, a 40-bit
 * integer (each index has probability within a factor 1 +- N / 2^40 of 1/N). */
float orc_half_u01_f32(const uint32_t x[4], int h) { return (float)(x[2 * h] >> 8) * 0x1p-24f; }

int64_t orc_half_index(const uint32_t x[4], int h, int64_t N) {
    uint64_t v = ((uint64_t)(x[2 * h] & 0xffu) << 32) | (uint64_t)x[2 * h + 1];
    unsigned __int128 p = (unsigned __int128)v * (unsigned __int128)(uint64_t)N;
    return (int64_t)(uint64_t)(p >> 40);
}

/* ------------------------------------------------------------------------------------ */
/* Pinned exponential (both precisions), defined for x <= 0                               */
/* ------------------------------------------------------------------------------------ */

/* Cody & Waite (1980) argument reduction: k = nearest integer to x/ln2, r = x - k ln2 with
 * ln2 split into a head and a tail so that |r| <= ln2/2 is obtained accurately; then the
 * Taylor polynomial of e^r (coefficients 1/n!, degree 7 in binary32, where the truncation
 * error 0.347^8/8! is below 2^-27, and degree 13 in binary64, where 0.347^14/14! is below
 * 2^-57) in Horner form with fused multiply-adds; then the exact scaling by 2^k. Inputs
 * below -86.5 (binary32) or -707 (binary64) return 0 so that every non-zero result is a
 * normal number; NaN propagates. */
static const float EXP32_C[8] = {0x1p+0f, 0x1p+0f, 0x1p-1f, 0x1.555556p-3f, 0x1.555556p-5f,
                                 0x1.111112p-7f, 0x1.6c16c2p-10f, 0x1.a01a02p-13f};
float orc_exp_f32(float x) {
    if (x != x) return x;
    if (x < -86.5f) return 0.0f;
    float k = rintf(x * 0x1.715476p+0f);
    float r = fmaf(-k, 0x1.62e430p-1f, x);
    r = fmaf(-k, -0x1.05c610p-29f, r);
    float p = EXP32_C[7];
    for (int n = 6; n >= 0; --n) p = fmaf(p, r, EXP32_C[n]);
    int32_t ki = (int32_t)k;
    uint32_t bits = (uint32_t)(ki + 127) << 23;
    float scale;
    memcpy(&scale, &bits, sizeof scale);
    return p * scale;
}

static const double EXP64_C[14] = {
    0x1p+0, 0x1p+0, 0x1p-1, 0x1.5555555555555p-3, 0x1.5555555555555p-5,
    0x1.1111111111111p-7, 0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13,
    0x1.a01a01a01a01ap-16, 0x1.71de3a556c734p-19, 0x1.27e4fb7789f5cp-22,
    0x1.ae64567f544e4p-26, 0x1.1eed8eff8d898p-29, 0x1.6124613a86d09p-33};
double orc_exp_f64(double x) {
    if (x != x) return x;
    if (x < -707.0) return 0.0;
    double k = rint(x * 0x1.71547652b82fep+0);
    double r = fma(-k, 0x1.62e42fefa39efp-1, x);
    r = fma(-k, 0x1.abc9e3b39803fp-56, r);
    double p = EXP64_C[13];
    for (int n = 12; n >= 0; --n) p = fma(p, r, EXP64_C[n]);
    int64_t ki = (int64_t)k;
    uint64_t bits = (uint64_t)(ki + 1023) << 52;
    double scale;
    memcpy(&scale, &bits, sizeof scale);
    return p * scale;
}

/* ------------------------------------------------------------------------------------ */
/* Input checks                                                                          */
/* ------------------------------------------------------------------------------------ */

/* Log-weights may be -inf (zero weight) but neither NaN nor +inf. */
static int check_finite_f32(const float* lw, int64_t N) {
    for (int64_t i = 0; i < N; ++i)
        if (lw[i] != lw[i] || lw[i] == INFINITY) return ORC_ERR_NONFINITE;
    return ORC_OK;
}
static int check_finite_f64(const double* lw, int64_t N) {
    for (int64_t i = 0; i < N; ++i)
        if (lw[i] != lw[i] || lw[i] == INFINITY) return ORC_ERR_NONFINITE;
    return ORC_OK;
}
static int check_n(int64_t N) { return (N >= 1 && N <= 2147483647LL) ? ORC_OK : ORC_ERR_ARG; }

/* ------------------------------------------------------------------------------------ */
/* Metropolis resampler (Section 2.1, Code 2)                                            */
/* ------------------------------------------------------------------------------------ */

/* Acceptance of a proposal j from state k: u < w^j / w^k, formed from the difference of
 * log-weights. A ratio >= 1 always accepts; a current state of zero weight accepts any
 * proposal. u is drawn from [0,1), so the strict comparison accepts with probability
 * exactly equal to the ratio on the grid of u and never accepts a zero-weight proposal. */
static int metropolis_accept_f32(float lwk, float lwj, float u) {
    if (lwk == -INFINITY) return 1;
    float delta = lwj - lwk;
    if (delta >= 0.0f) return 1;
    return u < orc_exp_f32(delta);
}
static int metropolis_accept_f64(double lwk, double lwj, double u) {
    if (lwk == -INFINITY) return 1;
    double delta = lwj - lwk;
    if (delta >= 0.0) return 1;
    return u < orc_exp_f64(delta);
}

/* For each particle i: start the chain at k = i; for n = 0..B-1 draw (u, j) and move to j on
 * acceptance; the ancestor is the final state. Binary32: step n takes half n mod 2 of the
 * block of counter (i, floor(n/2)) (orc_half_u01_f32, orc_half_index); binary64: the block of
 * counter (i, n), its 53-bit uniform and 64-bit index. */
int orc_metropolis_f32(const float* lw, int64_t N, int32_t B, uint64_t seed, uint64_t step,
                       uint32_t filter, int32_t* a) {
    if (check_n(N) != ORC_OK || B < 0) return ORC_ERR_ARG;
    if (check_finite_f32(lw, N) != ORC_OK) return ORC_ERR_NONFINITE;
    for (int64_t i = 0; i < N; ++i) {
        int64_t k = i;
        float lwk = lw[i];
        for (int32_t n = 0; n < B; ++n) {
            uint32_t x[4];
            orc_draw(seed, (uint32_t)i, (uint32_t)(n / 2), step, filter, ORC_METROPOLIS, x);
            int64_t j = orc_half_index(x, n % 2, N);
            float u = orc_half_u01_f32(x, n % 2);
            float lwj = lw[j];
            if (metropolis_accept_f32(lwk, lwj, u)) {
                k = j;
                lwk = lwj;
            }
        }
        a[i] = (int32_t)k;
    }
    return ORC_OK;
}

int orc_metropolis_f64(const double* lw, int64_t N, int32_t B, uint64_t seed, uint64_t step,
                       uint32_t filter, int32_t* a) {
    if (check_n(N) != ORC_OK || B < 0) return ORC_ERR_ARG;
    if (check_finite_f64(lw, N) != ORC_OK) return ORC_ERR_NONFINITE;
    for (int64_t i = 0; i < N; ++i) {
        int64_t k = i;
        double lwk = lw[i];
        for (int32_t n = 0; n < B; ++n) {
            uint32_t x[4];
            orc_draw(seed, (uint32_t)i, (uint32_t)n, step, filter, ORC_METROPOLIS, x);
            int64_t j = orc_uniform_index(x, N);
            double u = orc_u01_f64(x);
            double lwj = lw[j];
            if (metropolis_accept_f64(lwk, lwj, u)) {
                k = j;
                lwk = lwj;
            }
        }
        a[i] = (int32_t)k;
    }
    return ORC_OK;
}

/* Number of Metropolis steps B* = log(eps) / log(1 - beta) of Eq. (B), rounded up. */
int32_t orc_metropolis_B(double eps, double beta) {
    if (!(eps > 0.0 && eps < 1.0) || !(beta > 0.0 && beta <= 1.0)) return -1;
    if (beta >= 1.0) return 1;
    double b = ceil(log(eps) / log1p(-beta));
    if (b < 1.0) b = 1.0;
    if (b > 2147483647.0) return -1;
    return (int32_t)b;
}

/* ------------------------------------------------------------------------------------ */
/* Rejection resampler (Section 2.2, Code 3)                                             */
/* ------------------------------------------------------------------------------------ */

/* For each particle i: attempt 0 proposes j = i; attempt n >= 1 proposes j uniformly; both
 * draw from counter (i, n) in binary64, and in binary32 from half n mod 2 of the block of
 * counter (i, floor(n/2)) (orc_half_u01_f32, orc_half_index: two attempts per block, as the
 * binary32 Metropolis steps). Accept when u < w^j / w_max, formed as exp(lw^j - log w_max).
 * A log-weight above the bound is a violated bound: it is flagged and accepted. After
 * max_trials attempts without acceptance the particle keeps a^i = i and the cap is flagged. */
int orc_rejection_f32(const float* lw, int64_t N, double log_wmax, int64_t max_trials,
                      uint64_t seed, uint64_t step, uint32_t filter, int32_t* a,
                      int64_t* trials) {
    if (check_n(N) != ORC_OK || max_trials < 1 || !isfinite(log_wmax)) return ORC_ERR_ARG;
    if (check_finite_f32(lw, N) != ORC_OK) return ORC_ERR_NONFINITE;
    float lwmax = (float)log_wmax;
    int status = ORC_OK;
    for (int64_t i = 0; i < N; ++i) {
        int64_t j = i;
        int64_t n = 0;
        int accepted = 0;
        while (n < max_trials) {
            uint32_t x[4];
            orc_draw(seed, (uint32_t)i, (uint32_t)(n / 2), step, filter, ORC_REJECTION, x);
            if (n > 0) j = orc_half_index(x, (int)(n % 2), N);
            float u = orc_half_u01_f32(x, (int)(n % 2));
            float delta = lw[j] - lwmax;
            n += 1;
            if (delta > 0.0f) {
                status = ORC_ERR_BOUND_VIOLATED;
                accepted = 1;
                break;
            }
            if (delta == 0.0f || u < orc_exp_f32(delta)) {
                accepted = 1;
                break;
            }
        }
        if (!accepted) {
            j = i;
            if (status == ORC_OK) status = ORC_ERR_REJECTION_CAP;
        }
        a[i] = (int32_t)j;
        if (trials) trials[i] = n;
    }
    return status;
}

int orc_rejection_f64(const double* lw, int64_t N, double log_wmax, int64_t max_trials,
                      uint64_t seed, uint64_t step, uint32_t filter, int32_t* a,
                      int64_t* trials) {
    if (check_n(N) != ORC_OK || max_trials < 1 || !isfinite(log_wmax)) return ORC_ERR_ARG;
    if (check_finite_f64(lw, N) != ORC_OK) return ORC_ERR_NONFINITE;
    int status = ORC_OK;
    for (int64_t i = 0; i < N; ++i) {
        int64_t j = i;
        int64_t n = 0;
        int accepted = 0;
        while (n < max_trials) {
            uint32_t x[4];
            orc_draw(seed, (uint32_t)i, (uint32_t)n, step, filter, ORC_REJECTION, x);
            if (n > 0) j = orc_uniform_index(x, N);
            double u = orc_u01_f64(x);
            double delta = lw[j] - log_wmax;
            n += 1;
            if (delta > 0.0) {
                status = ORC_ERR_BOUND_VIOLATED;
                accepted = 1;
                break;
            }
            if (delta == 0.0 || u < orc_exp_f64(delta)) {
                accepted = 1;
                break;
            }
        }
        if (!accepted) {
            j = i;
            if (status == ORC_OK) status = ORC_ERR_REJECTION_CAP;
        }
        a[i] = (int32_t)j;
        if (trials) trials[i] = n;
    }
    return status;
}

/* Partial rejection control (Section 2.2, last paragraph, after Liu et al. 1998): pick
 * v_max below the weight bound, set v^i = min(w^i, v_max) and run the rejection sampler of
 * Code 3 on v with the bound v_max; the outcome stays weighted, particle i carrying
 * w^{a^i} / v^{a^i} (orc_prc_weights_*). In the log domain lv^j = min(lw^j, log v_max), and the
 * attempt accepts when u < exp(lv^j - log v_max); a proposal with w^j >= v_max has ratio 1.
 * No weight can violate the bound, so the only error statuses are the argument checks, a
 * non-finite log-weight and the trial cap. */
int orc_prc_f32(const float* lw, int64_t N, double log_vmax, int64_t max_trials,
                uint64_t seed, uint64_t step, uint32_t filter, int32_t* a, int64_t* trials) {
    if (check_n(N) != ORC_OK || max_trials < 1 || !isfinite(log_vmax)) return ORC_ERR_ARG;
    if (check_finite_f32(lw, N) != ORC_OK) return ORC_ERR_NONFINITE;
    float lvmax = (float)log_vmax;
    int status = ORC_OK;
    for (int64_t i = 0; i < N; ++i) {
        int64_t j = i;
        int64_t n = 0;
        int accepted = 0;
        while (n < max_trials) {
            uint32_t x[4];
            orc_draw(seed, (uint32_t)i, (uint32_t)(n / 2), step, filter, ORC_REJECTION, x);
            if (n > 0) j = orc_half_index(x, (int)(n % 2), N);
            float u = orc_half_u01_f32(x, (int)(n % 2));
            float lv = lw[j] < lvmax ? lw[j] : lvmax;
            float delta = lv - lvmax;
            n += 1;
            if (delta == 0.0f || u < orc_exp_f32(delta)) {
                accepted = 1;
                break;
            }
        }
        if (!accepted) {
            j = i;
            status = ORC_ERR_REJECTION_CAP;
        }
        a[i] = (int32_t)j;
        if (trials) trials[i] = n;
    }
    return status;
}

int orc_prc_f64(const double* lw, int64_t N, double log_vmax, int64_t max_trials,
                uint64_t seed, uint64_t step, uint32_t filter, int32_t* a, int64_t* trials) {
    if (check_n(N) != ORC_OK || max_trials < 1 || !isfinite(log_vmax)) return ORC_ERR_ARG;
    if (check_finite_f64(lw, N) != ORC_OK) return ORC_ERR_NONFINITE;
    int status = ORC_OK;
    for (int64_t i = 0; i < N; ++i) {
        int64_t j = i;
        int64_t n = 0;
        int accepted = 0;
        while (n < max_trials) {
            uint32_t x[4];
            orc_draw(seed, (uint32_t)i, (uint32_t)n, step, filter, ORC_REJECTION, x);
            if (n > 0) j = orc_uniform_index(x, N);
            double u = orc_u01_f64(x);
            double lv = lw[j] < log_vmax ? lw[j] : log_vmax;
            double delta = lv - log_vmax;
            n += 1;
            if (delta == 0.0 || u < orc_exp_f64(delta)) {
                accepted = 1;
                break;
            }
        }
        if (!accepted) {
            j = i;
            status = ORC_ERR_REJECTION_CAP;
        }
        a[i] = (int32_t)j;
        if (trials) trials[i] = n;
    }
    return status;
}

/* A substitute bound for the rejection resampler when no hard bound on the weights is known
 * (Section 2.2: "some reasonable substitute can be made"; the empirical maximum would be a
 * collective over all weights): the largest of `sample` log-weights at indices drawn
 * uniformly, the k-th index from counter (k, 0) with purpose ORC_BOUND_ESTIMATE. NaN
 * log-weights are passed over; the result is -inf when every drawn log-weight is -inf or NaN.
 * Partial rejection control with v_max = this bound then gives a weighted outcome
 * (orc_prc_*, orc_prc_weights_*); the weights above it are its violations. */
double orc_estimate_log_wmax_f32(const float* lw, int64_t N, int64_t sample, uint64_t seed,
                                 uint64_t step, uint32_t filter) {
    double m = -INFINITY;
    for (int64_t k = 0; k < sample; ++k) {
        uint32_t x[4];
        orc_draw(seed, (uint32_t)k, 0u, step, filter, ORC_BOUND_ESTIMATE, x);
        float v = lw[orc_uniform_index(x, N)];
        if (v == v && (double)v > m) m = (double)v;
    }
    return m;
}
double orc_estimate_log_wmax_f64(const double* lw, int64_t N, int64_t sample, uint64_t seed,
                                 uint64_t step, uint32_t filter) {
    double m = -INFINITY;
    for (int64_t k = 0; k < sample; ++k) {
        uint32_t x[4];
        orc_draw(seed, (uint32_t)k, 0u, step, filter, ORC_BOUND_ESTIMATE, x);
        double v = lw[orc_uniform_index(x, N)];
        if (v == v && v > m) m = v;
    }
    return m;
}

/* The log-weights of the outcome of partial rejection control for a delivered ancestry c
 * (the sampler's a, or its permutation by Code 10): out^i = log(w^{c^i} / v^{c^i}) =
 * lw^{c^i} - min(lw^{c^i}, log v_max), which is 0 unless w^{c^i} > v_max. A zero weight has
 * v = w = 0 and is given the ratio 1 (log 0), the limit of w / min(w, v_max) as w -> 0. */
int orc_prc_weights_f32(const float* lw, const int32_t* c, int64_t N, double log_vmax,
                        float* out) {
    if (check_n(N) != ORC_OK || !isfinite(log_vmax)) return ORC_ERR_ARG;
    float lvmax = (float)log_vmax;
    for (int64_t i = 0; i < N; ++i) {
        if (c[i] < 0 || c[i] >= N) return ORC_ERR_ARG;
        float w = lw[c[i]];
        float lv = w < lvmax ? w : lvmax;
        out[i] = (w == -INFINITY) ? 0.0f : w - lv;
    }
    return ORC_OK;
}

int orc_prc_weights_f64(const double* lw, const int32_t* c, int64_t N, double log_vmax,
                        double* out) {
    if (check_n(N) != ORC_OK || !isfinite(log_vmax)) return ORC_ERR_ARG;
    for (int64_t i = 0; i < N; ++i) {
        if (c[i] < 0 || c[i] >= N) return ORC_ERR_ARG;
        double w = lw[c[i]];
        double lv = w < log_vmax ? w : log_vmax;
        out[i] = (w == -INFINITY) ? 0.0 : w - lv;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Weights from log-weights, prefix sums (Appendix A primitives, Appendix E)             */
/* ------------------------------------------------------------------------------------ */

/* w^i = exp(lw^i - max_j lw^j): renormalisation by the maximum log-weight (Appendix E).
 * Returns ORC_ERR_ZERO_WEIGHT when every log-weight is -inf. */
int orc_weights_f32(const float* lw, int64_t N, float* w, float* m_out) {
    if (check_n(N) != ORC_OK) return ORC_ERR_ARG;
    if (check_finite_f32(lw, N) != ORC_OK) return ORC_ERR_NONFINITE;
    float m = -INFINITY;
    for (int64_t i = 0; i < N; ++i) m = lw[i] > m ? lw[i] : m;
    if (m == -INFINITY) return ORC_ERR_ZERO_WEIGHT;
    for (int64_t i = 0; i < N; ++i) w[i] = lw[i] == -INFINITY ? 0.0f : orc_exp_f32(lw[i] - m);
    if (m_out) *m_out = m;
    return ORC_OK;
}
int orc_weights_f64(const double* lw, int64_t N, double* w, double* m_out) {
    if (check_n(N) != ORC_OK) return ORC_ERR_ARG;
    if (check_finite_f64(lw, N) != ORC_OK) return ORC_ERR_NONFINITE;
    double m = -INFINITY;
    for (int64_t i = 0; i < N; ++i) m = lw[i] > m ? lw[i] : m;
    if (m == -INFINITY) return ORC_ERR_ZERO_WEIGHT;
    for (int64_t i = 0; i < N; ++i) w[i] = lw[i] == -INFINITY ? 0.0 : orc_exp_f64(lw[i] - m);
    if (m_out) *m_out = m;
    return ORC_OK;
}

/* Inclusive-Prefix-Sum, sequential, in the working precision. */
void orc_inclusive_prefix_sum_f32(const float* w, int64_t N, float* W) {
    float s = 0.0f;
    for (int64_t i = 0; i < N; ++i) { s = s + w[i]; W[i] = s; }
}
void orc_inclusive_prefix_sum_f64(const double* w, int64_t N, double* W) {
    double s = 0.0;
    for (int64_t i = 0; i < N; ++i) { s = s + w[i]; W[i] = s; }
}

/* Double-double arithmetic (Dekker 1971; Knuth's TwoSum): the "exact" reference prefix. */
static void two_sum(double a, double b, double* s, double* e) {
    double x = a + b;
    double bv = x - a;
    double av = x - bv;
    *s = x;
    *e = (a - av) + (b - bv);
}
static void quick_two_sum(double a, double b, double* s, double* e) {
    double x = a + b;
    *s = x;
    *e = b - (x - a);
}
static void two_prod(double a, double b, double* p, double* e) {
    double x = a * b;
    *p = x;
    *e = fma(a, b, -x);
}
static void dd_add_d(double ah, double al, double b, double* rh, double* rl) {
    double s, e;
    two_sum(ah, b, &s, &e);
    e = e + al;
    quick_two_sum(s, e, rh, rl);
}
static void dd_sub_dd(double ah, double al, double bh, double bl, double* rh, double* rl) {
    double s, e, t, f;
    two_sum(ah, -bh, &s, &e);
    two_sum(al, -bl, &t, &f);
    e = e + t;
    quick_two_sum(s, e, &s, &e);
    e = e + f;
    quick_two_sum(s, e, rh, rl);
}
static void dd_mul_d(double ah, double al, double b, double* rh, double* rl) {
    double p, e;
    two_prod(ah, b, &p, &e);
    e = e + al * b;
    quick_two_sum(p, e, rh, rl);
}
/* a / b in double-double by three steps of long division. */
static void dd_div_dd(double ah, double al, double bh, double bl, double* rh, double* rl) {
    double q1 = ah / bh;
    double ph, pl, rh1, rl1;
    dd_mul_d(bh, bl, q1, &ph, &pl);
    dd_sub_dd(ah, al, ph, pl, &rh1, &rl1);
    double q2 = rh1 / bh;
    dd_mul_d(bh, bl, q2, &ph, &pl);
    dd_sub_dd(rh1, rl1, ph, pl, &rh1, &rl1);
    double q3 = rh1 / bh;
    double s, e;
    quick_two_sum(q1, q2, &s, &e);
    dd_add_d(s, e, q3, rh, rl);
}
static int dd_le(double ah, double al, double bh, double bl) {
    return ah < bh || (ah == bh && al <= bl);
}
/* floor of a normalised double-double (|lo| <= ulp(hi)/2), as an integer. */
static int64_t dd_floor(double h, double l) {
    double f = floor(h);
    if (f != h) return (int64_t)f;
    return (int64_t)f + (int64_t)floor(l);
}

/* Exact-to-about-2^-100 inclusive prefix sum of w (double-double accumulation). */
void orc_dd_prefix_f64(const double* w, int64_t N, double* hi, double* lo) {
    double sh = 0.0, sl = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        dd_add_d(sh, sl, w[i], &sh, &sl);
        hi[i] = sh;
        lo[i] = sl;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Cumulative offspring of the stratified and systematic resamplers (Appendix B.2, B.3)  */
/* ------------------------------------------------------------------------------------ */

/* r^i = N W^i / W^N (Codes 7 and 8) in one pinned evaluation order: the factor
 * c = N / W^N is formed once, as the correctly rounded binary64 quotient rounded once more
 * to the prefix-sum type, and r^i = W^i * c is one rounded product; where W^i equals the
 * total (the last particle and every trailing zero weight) r^i = N exactly, so trailing zero
 * weights receive no offspring. r is non-decreasing in W^i because every rounding is
 * monotone. Systematic (Code 8): O^i = min(N, floor(r^i + u)), the sum rounded in the
 * prefix-sum type. Stratified (Code 7), 0-based: stratum k^i = min(N-1, floor(r^i)),
 * O^i = min(N, k^i + 1, floor(r^i + u^{k^i})); the extra bound k^i + 1 holds in exact
 * arithmetic and keeps O non-decreasing when r^i + u rounds up to the next integer.
 * The double-double forms compute r^i = N (W^i / W^N) to about 2^-100 (the exact value,
 * the reference for the compensated prefix sums). */
static int64_t clamp_n(int64_t v, int64_t N) { return v < N ? v : N; }

/* c = N / W^N: the binary64 quotient, then (binary32) rounded to the prefix-sum type. */
static float scale_f32(int64_t N, float S) { return (float)((double)N / (double)S); }
static double scale_f64(int64_t N, double S) { return (double)N / S; }

void orc_systematic_O_given_u_f32(const float* W, int64_t N, float u, int32_t* O) {
    float S = W[N - 1];
    float c = scale_f32(N, S);
    for (int64_t i = 0; i < N; ++i) {
        if (W[i] == S) { O[i] = (int32_t)N; continue; }
        float r = W[i] * c;
        O[i] = (int32_t)clamp_n((int64_t)floorf(r + u), N);
    }
}
void orc_systematic_O_given_u_f64(const double* W, int64_t N, double u, int32_t* O) {
    double S = W[N - 1];
    double c = scale_f64(N, S);
    for (int64_t i = 0; i < N; ++i) {
        if (W[i] == S) { O[i] = (int32_t)N; continue; }
        double r = W[i] * c;
        O[i] = (int32_t)clamp_n((int64_t)floor(r + u), N);
    }
}
/* Double-double form: W given as (hi, lo) pairs; u given in double (exact for both dtypes). */
void orc_systematic_O_given_u_dd(const double* Wh, const double* Wl, int64_t N, double u,
                                 int32_t* O) {
    double Sh = Wh[N - 1], Sl = Wl[N - 1];
    for (int64_t i = 0; i < N; ++i) {
        double qh, ql, rh, rl;
        dd_div_dd(Wh[i], Wl[i], Sh, Sl, &qh, &ql);
        dd_mul_d(qh, ql, (double)N, &rh, &rl);
        dd_add_d(rh, rl, u, &rh, &rl);
        O[i] = (int32_t)clamp_n(dd_floor(rh, rl), N);
    }
}

/* Stratified with the per-stratum uniforms given explicitly (u has N entries). */
void orc_stratified_O_given_u_f32(const float* W, int64_t N, const float* u, int32_t* O) {
    float S = W[N - 1];
    float c = scale_f32(N, S);
    for (int64_t i = 0; i < N; ++i) {
        if (W[i] == S) { O[i] = (int32_t)N; continue; }
        float r = W[i] * c;
        int64_t k = (int64_t)floorf(r);
        if (k > N - 1) k = N - 1;
        int64_t o = (int64_t)floorf(r + u[k]);
        if (o > k + 1) o = k + 1;
        O[i] = (int32_t)clamp_n(o, N);
    }
}
void orc_stratified_O_given_u_f64(const double* W, int64_t N, const double* u, int32_t* O) {
    double S = W[N - 1];
    double c = scale_f64(N, S);
    for (int64_t i = 0; i < N; ++i) {
        if (W[i] == S) { O[i] = (int32_t)N; continue; }
        double r = W[i] * c;
        int64_t k = (int64_t)floor(r);
        if (k > N - 1) k = N - 1;
        int64_t o = (int64_t)floor(r + u[k]);
        if (o > k + 1) o = k + 1;
        O[i] = (int32_t)clamp_n(o, N);
    }
}
void orc_stratified_O_given_u_dd(const double* Wh, const double* Wl, int64_t N,
                                 const double* u, int32_t* O) {
    double Sh = Wh[N - 1], Sl = Wl[N - 1];
    for (int64_t i = 0; i < N; ++i) {
        double qh, ql, rh, rl, zh, zl;
        dd_div_dd(Wh[i], Wl[i], Sh, Sl, &qh, &ql);
        dd_mul_d(qh, ql, (double)N, &rh, &rl);
        int64_t k = dd_floor(rh, rl);
        if (k > N - 1) k = N - 1;
        dd_add_d(rh, rl, u[k], &zh, &zl);
        int64_t o = dd_floor(zh, zl);
        if (o > k + 1) o = k + 1;
        O[i] = (int32_t)clamp_n(o, N);
    }
}

/* ------------------------------------------------------------------------------------ */
/* Auxiliary functions (Appendix D, Codes 11 and 12; Appendix A primitives)              */
/* ------------------------------------------------------------------------------------ */

/* Code 12: o = 0, then o^{a^i} += 1 for every i. */
int orc_ancestors_to_offspring(const int32_t* a, int64_t N, int32_t* o) {
    for (int64_t i = 0; i < N; ++i) o[i] = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (a[i] < 0 || a[i] >= N) return ORC_ERR_ARG;
        o[a[i]] += 1;
    }
    return ORC_OK;
}

/* Inclusive-Prefix-Sum and Adjacent-Difference on integers (exact). */
void orc_inclusive_prefix_sum_i32(const int32_t* o, int64_t N, int32_t* O) {
    int64_t s = 0;
    for (int64_t i = 0; i < N; ++i) { s += o[i]; O[i] = (int32_t)s; }
}
void orc_adjacent_difference_i32(const int32_t* O, int64_t N, int32_t* o) {
    for (int64_t i = 0; i < N; ++i) o[i] = i == 0 ? O[0] : O[i] - O[i - 1];
}

/* Code 11: particle i fills positions start .. O^i - 1 of a, where start = O^{i-1}
 * (0 for the first particle). Requires O non-decreasing with O^{N-1} = N. */
int orc_cumulative_offspring_to_ancestors(const int32_t* O, int64_t N, int32_t* a) {
    if (O[N - 1] != N) return ORC_ERR_ARG;
    for (int64_t i = 0; i < N; ++i) {
        int64_t start = i == 0 ? 0 : O[i - 1];
        if (O[i] < start) return ORC_ERR_ARG;
        for (int64_t j = start; j < O[i]; ++j) a[j] = (int32_t)i;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Multinomial, stratified and systematic ancestors (Appendix B, Codes 5, 7, 8 with 11)  */
/* ------------------------------------------------------------------------------------ */

/* Lower-Bound of Code 4 taken as the half-open reading: the first j with W^j > u (the
 * particle whose interval [W^{j-1}, W^j) holds u), so a zero-weight particle is never
 * selected; u < W^{N-1} always holds here, so the result is at most N-1. */
static int64_t upper_bound_f32(const float* W, int64_t N, float u) {
    int64_t lo = 0, hi = N;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (W[mid] <= u) lo = mid + 1; else hi = mid;
    }
    return lo < N ? lo : N - 1;
}
static int64_t upper_bound_f64(const double* W, int64_t N, double u) {
    int64_t lo = 0, hi = N;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (W[mid] <= u) lo = mid + 1; else hi = mid;
    }
    return lo < N ? lo : N - 1;
}
static int64_t upper_bound_dd(const double* Wh, const double* Wl, int64_t N, double uh,
                              double ul) {
    int64_t lo = 0, hi = N;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (dd_le(Wh[mid], Wl[mid], uh, ul)) lo = mid + 1; else hi = mid;
    }
    return lo < N ? lo : N - 1;
}

/* prec: 0 = the prefix sum in the dtype's own precision, sequential (the paper's plain
 * algorithm); 1 = the prefix sum of the same weights in double-double (the exact result up
 * to about 2^-100, the reference for compensated scans). */

/* Code 5: W = Inclusive-Prefix-Sum(w); for each i, u^i = U^i W^{N-1} with U^i ~ U[0,1)
 * from counter (i, 0); a^i = the particle whose interval holds u^i. */
int orc_multinomial_f32(const float* lw, int64_t N, int prec, uint64_t seed, uint64_t step,
                        uint32_t filter, int32_t* a) {
    float* w = (float*)malloc((size_t)N * sizeof(float));
    int st = orc_weights_f32(lw, N, w, NULL);
    if (st != ORC_OK) { free(w); return st; }
    if (prec == 0) {
        float* W = (float*)malloc((size_t)N * sizeof(float));
        orc_inclusive_prefix_sum_f32(w, N, W);
        for (int64_t i = 0; i < N; ++i) {
            uint32_t x[4];
            orc_draw(seed, (uint32_t)i, 0u, step, filter, ORC_MULTINOMIAL, x);
            float u = orc_u01_f32(x) * W[N - 1];
            a[i] = (int32_t)upper_bound_f32(W, N, u);
        }
        free(W);
    } else {
        double* wd = (double*)malloc((size_t)N * sizeof(double));
        double* Wh = (double*)malloc((size_t)N * sizeof(double));
        double* Wl = (double*)malloc((size_t)N * sizeof(double));
        for (int64_t i = 0; i < N; ++i) wd[i] = (double)w[i];
        orc_dd_prefix_f64(wd, N, Wh, Wl);
        for (int64_t i = 0; i < N; ++i) {
            uint32_t x[4];
            orc_draw(seed, (uint32_t)i, 0u, step, filter, ORC_MULTINOMIAL, x);
            double uh, ul;
            dd_mul_d(Wh[N - 1], Wl[N - 1], (double)orc_u01_f32(x), &uh, &ul);
            a[i] = (int32_t)upper_bound_dd(Wh, Wl, N, uh, ul);
        }
        free(wd); free(Wh); free(Wl);
    }
    free(w);
    return ORC_OK;
}

int orc_multinomial_f64(const double* lw, int64_t N, int prec, uint64_t seed, uint64_t step,
                        uint32_t filter, int32_t* a) {
    double* w = (double*)malloc((size_t)N * sizeof(double));
    int st = orc_weights_f64(lw, N, w, NULL);
    if (st != ORC_OK) { free(w); return st; }
    if (prec == 0) {
        double* W = (double*)malloc((size_t)N * sizeof(double));
        orc_inclusive_prefix_sum_f64(w, N, W);
        for (int64_t i = 0; i < N; ++i) {
            uint32_t x[4];
            orc_draw(seed, (uint32_t)i, 0u, step, filter, ORC_MULTINOMIAL, x);
            double u = orc_u01_f64(x) * W[N - 1];
            a[i] = (int32_t)upper_bound_f64(W, N, u);
        }
        free(W);
    } else {
        double* Wh = (double*)malloc((size_t)N * sizeof(double));
        double* Wl = (double*)malloc((size_t)N * sizeof(double));
        orc_dd_prefix_f64(w, N, Wh, Wl);
        for (int64_t i = 0; i < N; ++i) {
            uint32_t x[4];
            orc_draw(seed, (uint32_t)i, 0u, step, filter, ORC_MULTINOMIAL, x);
            double uh, ul;
            dd_mul_d(Wh[N - 1], Wl[N - 1], orc_u01_f64(x), &uh, &ul);
            a[i] = (int32_t)upper_bound_dd(Wh, Wl, N, uh, ul);
        }
        free(Wh); free(Wl);
    }
    free(w);
    return ORC_OK;
}

/* Code 8 then Code 11: one u from counter (0, 0); O as above; a from O. */
int orc_systematic_f32(const float* lw, int64_t N, int prec, uint64_t seed, uint64_t step,
                       uint32_t filter, int32_t* O, int32_t* a) {
    float* w = (float*)malloc((size_t)N * sizeof(float));
    int st = orc_weights_f32(lw, N, w, NULL);
    if (st != ORC_OK) { free(w); return st; }
    uint32_t x[4];
    orc_draw(seed, 0u, 0u, step, filter, ORC_SYSTEMATIC, x);
    float u = orc_u01_f32(x);
    if (prec == 0) {
        float* W = (float*)malloc((size_t)N * sizeof(float));
        orc_inclusive_prefix_sum_f32(w, N, W);
        orc_systematic_O_given_u_f32(W, N, u, O);
        free(W);
    } else {
        double* wd = (double*)malloc((size_t)N * sizeof(double));
        double* Wh = (double*)malloc((size_t)N * sizeof(double));
        double* Wl = (double*)malloc((size_t)N * sizeof(double));
        for (int64_t i = 0; i < N; ++i) wd[i] = (double)w[i];
        orc_dd_prefix_f64(wd, N, Wh, Wl);
        orc_systematic_O_given_u_dd(Wh, Wl, N, (double)u, O);
        free(wd); free(Wh); free(Wl);
    }
    free(w);
    return orc_cumulative_offspring_to_ancestors(O, N, a);
}

int orc_systematic_f64(const double* lw, int64_t N, int prec, uint64_t seed, uint64_t step,
                       uint32_t filter, int32_t* O, int32_t* a) {
    double* w = (double*)malloc((size_t)N * sizeof(double));
    int st = orc_weights_f64(lw, N, w, NULL);
    if (st != ORC_OK) { free(w); return st; }
    uint32_t x[4];
    orc_draw(seed, 0u, 0u, step, filter, ORC_SYSTEMATIC, x);
    double u = orc_u01_f64(x);
    if (prec == 0) {
        double* W = (double*)malloc((size_t)N * sizeof(double));
        orc_inclusive_prefix_sum_f64(w, N, W);
        orc_systematic_O_given_u_f64(W, N, u, O);
        free(W);
    } else {
        double* Wh = (double*)malloc((size_t)N * sizeof(double));
        double* Wl = (double*)malloc((size_t)N * sizeof(double));
        orc_dd_prefix_f64(w, N, Wh, Wl);
        orc_systematic_O_given_u_dd(Wh, Wl, N, u, O);
        free(Wh); free(Wl);
    }
    free(w);
    return orc_cumulative_offspring_to_ancestors(O, N, a);
}

/* Code 7 then Code 11: the uniform of stratum k is orc_stratum_u_f32 / orc_stratum_u_f64. */
int orc_stratified_f32(const float* lw, int64_t N, int prec, uint64_t seed, uint64_t step,
                       uint32_t filter, int32_t* O, int32_t* a) {
    float* w = (float*)malloc((size_t)N * sizeof(float));
    int st = orc_weights_f32(lw, N, w, NULL);
    if (st != ORC_OK) { free(w); return st; }
    float* u = (float*)malloc((size_t)N * sizeof(float));
    for (int64_t k = 0; k < N; ++k) u[k] = orc_stratum_u_f32(seed, k, step, filter);
    if (prec == 0) {
        float* W = (float*)malloc((size_t)N * sizeof(float));
        orc_inclusive_prefix_sum_f32(w, N, W);
        orc_stratified_O_given_u_f32(W, N, u, O);
        free(W);
    } else {
        double* wd = (double*)malloc((size_t)N * sizeof(double));
        double* ud = (double*)malloc((size_t)N * sizeof(double));
        double* Wh = (double*)malloc((size_t)N * sizeof(double));
        double* Wl = (double*)malloc((size_t)N * sizeof(double));
        for (int64_t i = 0; i < N; ++i) { wd[i] = (double)w[i]; ud[i] = (double)u[i]; }
        orc_dd_prefix_f64(wd, N, Wh, Wl);
        orc_stratified_O_given_u_dd(Wh, Wl, N, ud, O);
        free(wd); free(ud); free(Wh); free(Wl);
    }
    free(u);
    free(w);
    return orc_cumulative_offspring_to_ancestors(O, N, a);
}

int orc_stratified_f64(const double* lw, int64_t N, int prec, uint64_t seed, uint64_t step,
                       uint32_t filter, int32_t* O, int32_t* a) {
    double* w = (double*)malloc((size_t)N * sizeof(double));
    int st = orc_weights_f64(lw, N, w, NULL);
    if (st != ORC_OK) { free(w); return st; }
    double* u = (double*)malloc((size_t)N * sizeof(double));
    for (int64_t k = 0; k < N; ++k) u[k] = orc_stratum_u_f64(seed, k, step, filter);
    if (prec == 0) {
        double* W = (double*)malloc((size_t)N * sizeof(double));
        orc_inclusive_prefix_sum_f64(w, N, W);
        orc_stratified_O_given_u_f64(W, N, u, O);
        free(W);
    } else {
        double* Wh = (double*)malloc((size_t)N * sizeof(double));
        double* Wl = (double*)malloc((size_t)N * sizeof(double));
        orc_dd_prefix_f64(w, N, Wh, Wl);
        orc_stratified_O_given_u_dd(Wh, Wl, N, u, O);
        free(Wh); free(Wl);
    }
    free(u);
    free(w);
    return orc_cumulative_offspring_to_ancestors(O, N, a);
}

/* ------------------------------------------------------------------------------------ */
/* Ancestor permutation (Appendix C, Codes 9 and 10)                                     */
/* ------------------------------------------------------------------------------------ */

/* Prepermute (Code 10, first procedure): d = N everywhere, then d^{a^i} = min(d^{a^i}, i)
 * for every i; afterwards d^j is the lowest index whose ancestor is j, or N if none. */
int orc_prepermute(const int32_t* a, int64_t N, int32_t* d) {
    for (int64_t i = 0; i < N; ++i) d[i] = (int32_t)N;
    for (int64_t i = 0; i < N; ++i) {
        if (a[i] < 0 || a[i] >= N) return ORC_ERR_ARG;
        if (i < d[a[i]]) d[a[i]] = (int32_t)i;
    }
    return ORC_OK;
}

/* Permute (Code 10, second procedure): for each i whose claim failed (d^{a^i} != i), walk
 * x = i, d^x, d^{d^x}, ... to the first unclaimed slot and claim it for i; then
 * c^i = a^{d^i}. `order` (optional, a permutation of 0..N-1) is the order in which the
 * for-each loop visits i; the result does not depend on it. */
int orc_permute(const int32_t* a, int64_t N, const int64_t* order, int32_t* c) {
    int32_t* d = (int32_t*)malloc((size_t)N * sizeof(int32_t));
    int st = orc_prepermute(a, N, d);
    if (st != ORC_OK) { free(d); return st; }
    for (int64_t t = 0; t < N; ++t) {
        int64_t i = order ? order[t] : t;
        int64_t x = d[a[i]];
        if (x != i) {
            x = i;
            while (d[x] < N) x = d[x];
            d[x] = (int32_t)i;
        }
    }
    for (int64_t i = 0; i < N; ++i) c[i] = a[d[i]];
    free(d);
    return ORC_OK;
}

/* Serial Permute (Code 9), in place: swap a^i with a^{a^i} while a^i != i and
 * a^{a^i} != a^i, then move on. Produces a different (also valid) ordering than Code 10. */
int orc_permute_serial(int32_t* a, int64_t N) {
    for (int64_t i = 0; i < N; ++i) {
        if (a[i] < 0 || a[i] >= N) return ORC_ERR_ARG;
    }
    for (int64_t i = 0; i < N; ++i) {
        while (a[i] != i && a[a[i]] != a[i]) {
            int32_t t = a[a[i]];
            a[a[i]] = a[i];
            a[i] = t;
        }
    }
    return ORC_OK;
}
