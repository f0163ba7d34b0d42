/*
 * resample.h -- C ABI of the GB300 (sm_103a) particle-filter resampling library.
 *
 * The operations follow Murray, Lee & Jacob, "Parallel resampling in the particle filter":
 * the resampling step Ancestors(w) -> a of the SMC loop (Section 1.1, Code 1), done by the
 * multinomial (Appendix B.1, Code 5), stratified (Appendix B.2, Code 7), systematic
 * (Appendix B.3, Code 8), Metropolis (Section 2.1, Code 2) and rejection (Section 2.2,
 * Code 3) resamplers; the ancestor permutation that makes in-place propagation safe
 * (Section 2.3, Eq. predicate; Appendix C, Code 10); and the ancestors <-> offspring
 * conversions (Appendix D, Codes 11 and 12, and the primitives of Code 4).
 *
 * Conventions for every call:
 *  - Indices are 0-based: particles are 0..N-1. 1 <= N <= 2^31 - 1.
 *  - Log-weights are given, not weights (Appendix E). A log-weight may be -inf (a zero
 *    weight) but not NaN or +inf. All schemes are invariant to adding a constant to every
 *    log-weight.
 *  - Pointers named *_dev are device pointers on the handle's device; they are owned by the
 *    caller, must not overlap one another unless stated, and must stay valid until the
 *    stream has executed the call. 16-byte alignment of logw gives the fastest loads; any
 *    alignment of the element type is accepted.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream). Calls are
 *    asynchronous on that stream, make no host synchronisation and allocate no memory, so
 *    they can be captured in a CUDA graph.
 *  - Return value: RS_OK, or a negative status for errors found on the host before any
 *    launch (nothing is launched then). Errors that only the device can see (NaN or +inf
 *    log-weights, all weights zero, a violated rejection bound, the rejection trial cap)
 *    are recorded in the handle and returned by rs_last_error; outputs of such a call are
 *    valid indices but otherwise unspecified.
 *  - Random numbers: draw n of particle (or stratum) i is Philox4x32-10 (Salmon et al.,
 *    SC'11) with key = seed and counter = (i, n, step mod 2^32, filter * 8 + scheme), so any
 *    result is reproducible from (seed, step) on any machine. Some uses take several values
 *    from one 128-bit block: stratum k of the stratified scheme uses word k mod 4 of block
 *    (k / 4, 0) at 24 bits, or words 2 (k mod 2), 2 (k mod 2) + 1 of block (k / 2, 0) at 53
 *    bits; binary32 Metropolis step n and binary32 rejection attempt n use half n mod 2 of
 *    block (i, n / 2) (a 24-bit uniform and a 40-bit proposal index).
 */
#ifndef RS_RESAMPLE_H
#define RS_RESAMPLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------- */
#define RS_OK 0
#define RS_ERR_ARG (-1)            /* invalid argument (host check) or out-of-range index   */
#define RS_ERR_NONFINITE (-2)      /* a log-weight is NaN or +inf                           */
#define RS_ERR_ZERO_WEIGHT (-3)    /* every log-weight is -inf (scan-based schemes)          */
#define RS_ERR_BOUND_VIOLATED (-4) /* rejection: a log-weight exceeds log_wmax (biased)      */
#define RS_ERR_REJECTION_CAP (-5)  /* rejection: a particle hit max_trials; it keeps a^i = i */
#define RS_ERR_TIMEOUT (-6)        /* a bounded device wait gave up                          */
#define RS_ERR_CUDA (-7)           /* a CUDA runtime call failed                             */
#define RS_ERR_CAPACITY (-8)       /* N exceeds the handle's max_n                           */

/* ---- enumerations ------------------------------------------------------------------- */
typedef enum {
    RS_MULTINOMIAL = 0, /* Appendix B.1, Code 5  */
    RS_STRATIFIED = 1,  /* Appendix B.2, Code 7  */
    RS_SYSTEMATIC = 2,  /* Appendix B.3, Code 8  */
    RS_METROPOLIS = 3,  /* Section 2.1, Code 2   */
    RS_REJECTION = 4    /* Section 2.2, Code 3   */
} rs_scheme;

typedef enum { RS_F32 = 0, RS_F64 = 1 } rs_dtype; /* element type of the log-weights */

/* Arithmetic of the weights and prefix sums of the multinomial, stratified and systematic
 * schemes (Section 4.2 and Appendix B.1 discuss the instability of single precision):
 *   RS_F32 + RS_PREC_PLAIN        binary32 weights and sums (the paper's setting).
 *   RS_F32 + RS_PREC_COMPENSATED  binary32 weights, two-float sums (about 48 significand
 *                                 bits), binary64 tile totals.
 *   RS_F64 + RS_PREC_PLAIN or     double-float: weights exp(lw - max) and sums kept as pairs
 *            RS_PREC_COMPENSATED  of binary32 (about 48 bits, relative error of every
 *                                 cumulative weight below 2^-40), binary64 tile totals,
 *                                 computed on the binary32 pipes (GB300 runs binary64 at
 *                                 1/57 of the binary32 rate). Draws keep all 53 bits.
 *   RS_F64 + RS_PREC_BINARY64     IEEE binary64 weights (pinned exp) and sums on the FP64
 *                                 pipe (slow on GB300).
 * The Metropolis and rejection schemes ignore this setting: their decisions are always exactly
 * those of the element type. */
typedef enum {
    RS_PREC_PLAIN = 0,
    RS_PREC_COMPENSATED = 1,
    RS_PREC_BINARY64 = 2
} rs_precision;

/* Optional per-call settings; pass NULL for the defaults shown. */
typedef struct {
    int32_t prec;       /* rs_precision, default RS_PREC_PLAIN                              */
    double log_wmax;    /* rejection: a-priori bound log w_max on every log-weight, finite;
                           default 0                                                       */
    int64_t max_trials; /* rejection: attempts per particle before RS_ERR_REJECTION_CAP;
                           default 1 << 20                                                 */
    uint32_t filter;    /* filter id in the random-number counter (< 2^29), default 0; a
                           single call with filter f reproduces filter f of a batched call  */
} rs_opts;

/* A handle owns the device scratch of the calls that need it (claim vector d, unpermuted
 * ancestors, cumulative weights of the multinomial scheme, per-tile partial sums, the grid
 * barrier counter, the device status word): about 20 bytes per particle of max_n, allocated
 * once here. Calls on one handle share that scratch, so they must execute one after the
 * other: issue them on one stream (or order the streams with events), and from one host
 * thread at a time. Independent work in parallel uses one handle per stream. */
typedef struct rs_handle rs_handle;

/* Creates a handle for problems of up to max_n particles on `device` (made current).
 * Returns RS_OK, RS_ERR_ARG or RS_ERR_CUDA (allocation failure). */
int rs_create(rs_handle** h, int64_t max_n, int device);

/* Frees the handle's device memory. Safe on NULL. */
int rs_destroy(rs_handle* h);

/* Ancestors(w) -> a (Code 1, line "resample"). Reads N log-weights of type `dtype` from
 * logw_dev and writes N ancestor indices to ancestors_dev (int32, values 0..N-1).
 *  scheme  : rs_scheme.
 *  B       : Metropolis steps per particle (Code 2), >= 0; ignored by other schemes. See
 *            rs_metropolis_B for the choice of Eq. (B).
 *  seed    : Philox key; step: SMC time index (counter word 2).
 *  permute : 0 = the scheme's natural order (stratified and systematic give a
 *            non-decreasing a); 1 = the result is permuted by Permute (Code 10) so that
 *            o^i > 0 implies a^i = i (Eq. predicate), ready for in-place propagation.
 *  opts    : NULL or settings above.
 * ancestors_dev must not overlap logw_dev. */
int rs_resample(rs_handle* h, int scheme, int dtype, const void* logw_dev, int64_t N,
                int32_t B, uint64_t seed, uint64_t step, int32_t* ancestors_dev, int permute,
                const rs_opts* opts, void* stream);

/* Partial rejection control (Section 2.2, last paragraph): the rejection resampler of Code 3
 * applied to the clamped weights v^i = min(w^i, v_max) with the bound v_max = exp(log_vmax),
 * for a v_max chosen below the weights' bound (or where no bound is known). The outcome stays
 * weighted: logw_out_dev[i] = log(w^{a^i} / v^{a^i}) = max(lw^{a^i} - log_vmax, 0) for the
 * delivered ancestry a (after Permute when permute = 1), in the dtype of the log-weights
 * (binary32: log_vmax rounded to binary32 first, as the attempts compare against it).
 * The draws are those of RS_REJECTION with opts->log_wmax = log_vmax, so the ancestry equals
 * rs_resample(RS_REJECTION) bit for bit; a weight above v_max is accepted as the clamped
 * weight, not flagged. A smaller v_max raises the acceptance probability E(v)/v_max and
 * lowers the trial count. Statuses via rs_last_error: RS_ERR_NONFINITE, RS_ERR_REJECTION_CAP
 * (max_trials, 1 .. 2^32-1, reached; the particle keeps itself). filter < 2^29 is counter
 * word 3 as in rs_opts. logw_out_dev (N elements of dtype) must not overlap logw_dev or
 * ancestors_dev; the caller owns all three buffers. */
int rs_resample_prc(rs_handle* h, int dtype, const void* logw_dev, int64_t N, double log_vmax,
                    int64_t max_trials, uint64_t seed, uint64_t step, uint32_t filter,
                    int32_t* ancestors_dev, void* logw_out_dev, int permute, void* stream);

/* Rejection resampling with an estimated bound (Section 2.2: when no hard bound on the
 * weights is known, "some reasonable substitute" v_max; the empirical maximum would be a
 * collective over all weights). log v_max is estimated on the device as the largest of
 * `sample` log-weights at indices drawn uniformly (Philox, counter (k, 0, step, filter * 8 +
 * 5) for the k-th; NaN passed over), then partial rejection control runs with it exactly as
 * rs_resample_prc does, so the outcome is weighted: logw_out_dev[i] = lw[c_i] - min(lw[c_i],
 * log v_max), nonzero only for ancestors whose weight exceeds the estimate.
 *   log_wmax_dev   : one binary64 on the device, receives the estimate;
 *   violations_dev : one uint64 on the device, receives the number of particles whose
 *                    log-weight exceeds the estimate (the bound's violations);
 *   sample         : 1 <= sample <= 2^31 - 1 (one CTA draws them: cost ~ sample / 1024);
 *   the rest as rs_resample_prc. When no drawn log-weight is finite the estimate is -inf,
 * every particle keeps itself (logw_out 0) and rs_last_error reports RS_ERR_ZERO_WEIGHT;
 * otherwise the statuses of rs_resample_prc. Asynchronous on `stream`, no host sync. */
int rs_resample_rejection_estimated(rs_handle* h, int dtype, const void* logw_dev, int64_t N,
                                    int64_t sample, int64_t max_trials, uint64_t seed,
                                    uint64_t step, uint32_t filter, int32_t* ancestors_dev,
                                    void* logw_out_dev, double* log_wmax_dev,
                                    unsigned long long* violations_dev, int permute,
                                    void* stream);

/* Many independent filters in one launch. F filters in CSR layout: offsets_dev holds F + 1
 * int64 offsets (device), filter f owning the particles offsets[f] .. offsets[f+1]-1 of
 * logw_dev and ancestors_dev; every filter has at most 2^20 particles (empty filters are
 * skipped) and offsets[F] <= the handle's max_n (violations: RS_ERR_ARG via rs_last_error).
 * ancestors_dev receives, for each filter, local ancestor indices 0..N_f-1. B_dev: NULL
 * (every filter uses B) or F int32 Metropolis step counts. The filter index f is the filter
 * of the random-number counter, so filter f equals rs_resample on its slice with
 * opts->filter = f, bit for bit; opts->filter is ignored. Other arguments as rs_resample.
 * F <= max(1024, max_n / 16) (RS_ERR_CAPACITY otherwise). The work units are the tiles and
 * particles of all filters together, so uneven sizes and per-filter B balance across the GPU. */
int rs_resample_batched(rs_handle* h, int scheme, int dtype, const void* logw_dev,
                        const int64_t* offsets_dev, int32_t F, const int32_t* B_dev, int32_t B,
                        uint64_t seed, uint64_t step, int32_t* ancestors_dev, int permute,
                        const rs_opts* opts, void* stream);

/* Cumulative weights (Code 4 Inclusive-Prefix-Sum of the max-shifted weights, Appendix E):
 * W_dev[i] = sum_{j<=i} exp(logw[j] - max logw) in `dtype` (compensated sums are rounded to
 * binary32 on output), and *log_total_dev (one binary64 on the device) =
 * max logw + log(sum_j exp(logw[j] - max logw)), the log of the sum of weights. */
int rs_cumulative_weights(rs_handle* h, int dtype, int prec, const void* logw_dev, int64_t N,
                          void* W_dev, double* log_total_dev, void* stream);

/* rs_cumulative_weights with W_dev in binary64 whatever the dtype: the accumulator of every
 * mode written out exactly (a binary32 sum, a two-float or double-float pair, or a binary64
 * sum), so that the rounding of the scan itself can be studied (the single-precision
 * instability of Section 4.2). Other arguments as rs_cumulative_weights. */
int rs_cumulative_weights_f64(rs_handle* h, int dtype, int prec, const void* logw_dev,
                              int64_t N, double* W_dev, double* log_total_dev, void* stream);

/* Ancestors-to-Offspring (Code 12): o_dev[j] = #{i : a[i] = j}. Entries of a outside
 * 0..N-1 are skipped and reported as RS_ERR_ARG through rs_last_error. */
int rs_offspring(rs_handle* h, const int32_t* a_dev, int64_t N, int32_t* o_dev, void* stream);

/* Offspring -> cumulative offspring: O = Inclusive-Prefix-Sum(o) on int32 (Appendix D). */
int rs_cumulative_offspring(rs_handle* h, const int32_t* o_dev, int64_t N, int32_t* O_dev,
                            void* stream);

/* Cumulative offspring -> offspring: Adjacent-Difference of Code 4 (Appendix D). */
int rs_adjacent_difference(rs_handle* h, const int32_t* O_dev, int64_t N, int32_t* o_dev,
                           void* stream);

/* Cumulative-Offspring-to-Ancestors (Code 11): particle i fills a[O[i-1] .. O[i]-1].
 * O must be non-decreasing with O[N-1] = N (checked on the device: RS_ERR_ARG). */
int rs_cumulative_offspring_to_ancestors(rs_handle* h, const int32_t* O_dev, int64_t N,
                                         int32_t* a_dev, void* stream);

/* Prepermute (Code 10): d_dev[j] = min{i : a[i] = j}, or N when j has no offspring. */
int rs_prepermute(rs_handle* h, const int32_t* a_dev, int64_t N, int32_t* d_dev, void* stream);

/* Permute (Code 10): c = a permuted so that o^i > 0 implies c^i = i (Eq. predicate). The
 * result is the deterministic one of Code 10 (the lowest claimant keeps its slot).
 * c_dev must not overlap a_dev. */
int rs_permute(rs_handle* h, const int32_t* a_dev, int64_t N, int32_t* c_dev, void* stream);

/* How rs_resample launches the multinomial, stratified and systematic schemes. The result is
 * the same bit for bit in every mode; only the launch structure differs:
 *   RS_LAUNCH_SEPARATE : one kernel per pass (max, tile sums, emission, search, Permute).
 *   RS_LAUNCH_FUSED    : all passes in one cooperative kernel whose CTAs are co-resident and
 *                        meet at grid-wide barriers (bounded waits: RS_ERR_TIMEOUT through
 *                        rs_last_error); used when the device supports cooperative launches,
 *                        else the separate kernels run.
 *   RS_LAUNCH_AUTO     : (default) fused when the device supports cooperative launches.
 * Host-only; RS_ERR_ARG for an unknown mode. The setting belongs to the handle. */
#define RS_LAUNCH_AUTO 0
#define RS_LAUNCH_FUSED 1
#define RS_LAUNCH_SEPARATE 2
int rs_set_launch_mode(rs_handle* h, int mode);

/* The longest a grid-wide barrier of the handle's cooperative kernels waits, in nanoseconds
 * (default 10 s). A wait that runs out records RS_ERR_TIMEOUT and the kernel goes on, so it
 * ends and the context stays usable; rs_last_error reports the status and resets the
 * handle's barrier state, after which the handle works again. Tests set a short limit.
 * Synchronises the handle's device; RS_ERR_ARG for timeout_ns = 0. The paper has no
 * counterpart (its kernels never wait on each other). */
int rs_set_barrier_timeout(rs_handle* h, uint64_t timeout_ns);

/* Effective sample size of N log-weights: *ess_dev (one binary64 on the device) =
 * (sum_i w_i)^2 / sum_i w_i^2 with w_i = exp(logw_i - max logw) (Appendix E), between 1 and N
 * -- the statistic an adaptive particle filter compares with a threshold to decide whether to
 * resample at a step (Section 4.3) -- and, from the same sums, *log_total_dev = max logw +
 * log sum_i w_i, the log of the weight total (the SMC likelihood increment). Either pointer
 * may be NULL, not both. Weights in binary32 (relative error about 2^-23), sums in two-float
 * per CTA and exact across CTAs. NaN/+inf flag RS_ERR_NONFINITE, all weights zero
 * RS_ERR_ZERO_WEIGHT (ess 0, log total -inf). One cooperative launch: RS_ERR_CUDA where the
 * device cannot. */
int rs_ess(rs_handle* h, int dtype, const void* logw_dev, int64_t N, double* ess_dev,
           double* log_total_dev, void* stream);

/* ---- the SMC loop around the resampler (Code 1) ---------------------------------------
 * In-place copy by a permuted ancestry (Section 2.3): x_dev holds N rows of D floats
 * (row-major, device); row i becomes row c_dev[i]. c must satisfy the predicate of Permute
 * (o_j > 0 implies c_j = j, as rs_resample(permute = 1) returns): then every row that is read
 * is one that is not written, and the copy runs in place. Rows i with c_i outside 0..N-1 or
 * c_{c_i} != c_i are left unchanged and reported as RS_ERR_ARG through rs_last_error. */
int rs_copy_ancestors(rs_handle* h, float* x_dev, int32_t D, const int32_t* c_dev, int64_t N,
                      void* stream);

/* Propagate and weight N particles of the 1-D linear-Gaussian state-space model
 *   x_1 ~ N(0, sigma_x^2 / (1 - phi^2)),  x_t = phi x_{t-1} + sigma_x eps_t,
 *   y_t = x_t + sigma_y eta_t
 * (the model of the full SMC loop; Code 1 lines "propagate" and "weight"). init = 1 draws x
 * from the stationary law, init = 0 propagates x in place. With l_i = -(y - x_i)^2 /
 * (2 sigma_y^2) (the constant -log(2 pi sigma_y^2)/2 is dropped, so log w_max = 0 for one
 * step), logw_dev[i] = l_i (accumulate = 0, after resampling) or logw_dev[i] + l_i
 * (accumulate = 1: the weights carried over a step without resampling). The noise of
 * particle i is one Box-Muller normal from the Philox words 0 and 1 of counter
 * (i, 0, step, filter * 8 + 5). |phi| < 1, sigma_x, sigma_y > 0 and y finite (RS_ERR_ARG
 * otherwise). */
int rs_lgssm_step(rs_handle* h, float* x_dev, int64_t N, int init, int accumulate, float phi,
                  float sigma_x, float y, float sigma_y, uint64_t seed, uint64_t step,
                  uint32_t filter, float* logw_dev, void* stream);

/* ---- resampling on demand inside a CUDA graph ------------------------------------------
 * The adaptive filter resamples only when the effective sample size falls below a threshold
 * (Section 4 mentions the practice). To keep that decision on the device -- the whole filter
 * one CUDA graph, no host round trip per step -- these calls build a conditional graph node:
 *
 * rs_capture_if_below: `stream` must be capturing into a CUDA graph (RS_ERR_ARG otherwise).
 * Adds to that graph a one-thread kernel that compares *value_dev (binary64, device) with
 * threshold when the graph runs, and after it an IF node whose body runs only when
 * *value_dev < threshold. Starts capturing that body on a stream owned by the handle and
 * returns it in *body_stream: the calls made on *body_stream (with any handle) until
 * rs_capture_end_if form the body. While the body is captured, this handle's calls use the
 * one-kernel-per-pass launch structure (RS_LAUNCH_SEPARATE) and no launch of this host
 * thread carries a programmatic dependency. Not nestable (RS_ERR_ARG).
 * rs_capture_end_if: ends the body (RS_ERR_ARG unless `stream` is the one given to
 * rs_capture_if_below) and restores the launch structure; work captured on `stream`
 * afterwards follows the conditional node. RS_ERR_CUDA if the runtime rejects a step (the
 * capture is then invalid). */
int rs_capture_if_below(rs_handle* h, const double* value_dev, double threshold, void* stream,
                        void** body_stream);
int rs_capture_end_if(rs_handle* h, void* stream);

/* The adaptive filter's bookkeeping on the device. rs_smc_mark_resampled, after a resampling:
 * logw_dev[0..N) = 0 (equal weights; the next rs_lgssm_step with accumulate = 1 then gives the
 * fresh log-weights exactly), *base_dev = log_n, and *count_dev += 1 (int32; may be NULL).
 * rs_smc_loglik_step, after the log weight total *lse_dev of step t (rs_cumulative_weights):
 * first = 1: *ll_dev = (*lse_dev - log_n) - c and *count_dev = 0; first = 0:
 * *ll_dev += (*lse_dev - *base_dev) - c; then *base_dev = *lse_dev. c is the constant dropped
 * from the log-weights (log(2 pi sigma_y^2)/2 for rs_lgssm_step). All binary64, device. */
int rs_smc_mark_resampled(rs_handle* h, float* logw_dev, int64_t N, double* base_dev,
                          double log_n, int32_t* count_dev, void* stream);
int rs_smc_loglik_step(rs_handle* h, const double* lse_dev, double* base_dev, double* ll_dev,
                       int32_t* count_dev, double c, double log_n, int first, void* stream);

/* ---- many independent filters (the CSR layout of rs_resample_batched) ------------------
 * F filters, filter f owning the particles offsets_dev[f] .. offsets_dev[f+1]-1 (F + 1 int64
 * on the device, non-decreasing, offsets[F] <= the handle's max_n). Filter f of each call
 * below computes exactly what the single-filter call computes on its slice with filter = f
 * (bit for bit), so a batched filter equals F single filters. Particles of a malformed
 * filter are skipped (and RS_ERR_ARG reported where the call checks indices). F >= 1. */

/* rs_copy_ancestors per filter: c_dev holds every filter's local ancestors (0..N_f-1), as
 * rs_resample_batched(permute = 1) returns them; row g of x_dev (D floats) becomes row
 * offsets[f] + c_dev[g] of its filter. */
int rs_copy_ancestors_batched(rs_handle* h, float* x_dev, int32_t D, const int32_t* c_dev,
                              const int64_t* offsets_dev, int32_t F, void* stream);

/* rs_lgssm_step per filter: y_dev holds F floats (device), filter f's observation of this
 * step; particle g of filter f draws its noise from counter (g - offsets[f], 0, step,
 * f * 8 + 5). Other arguments as rs_lgssm_step. */
int rs_lgssm_step_batched(rs_handle* h, float* x_dev, const int64_t* offsets_dev, int32_t F,
                          int init, int accumulate, float phi, float sigma_x,
                          const float* y_dev, float sigma_y, uint64_t seed, uint64_t step,
                          float* logw_dev, void* stream);

/* out_dev[f] = log sum_{g in filter f} exp(logw_dev[g]) (F float64, device): the log of the
 * filter's unnormalised weight total, the ingredient of its marginal-likelihood estimate
 * (Code 1). Computed with the max-shift of Appendix E: m_f + log sum exp(lw - m_f), the
 * exponentials in the dtype and the sum in binary64 (not bit-compatible with
 * rs_cumulative_weights' total). -inf for an empty or all-zero filter; NaN/+inf flag
 * RS_ERR_NONFINITE. */
int rs_log_sum_weights_batched(rs_handle* h, int dtype, const void* logw_dev,
                               const int64_t* offsets_dev, int32_t F, double* out_dev,
                               void* stream);

/* The effective sample size of every filter of a batch (offsets_dev: F+1 int64 CSR bounds,
 * as for rs_resample_batched): ess_dev[f] = (sum_g w_g)^2 / sum_g w_g^2 over the filter's
 * particles g with w_g = exp(logw_g - max logw), the statistic that decides per filter
 * whether an adaptive filter resamples at a step (Section 4.3); log_total_dev[f] = the
 * value rs_log_sum_weights_batched writes (same sums, bit for bit); below_dev[f] (uint8) =
 * 1 where ess < threshold_frac * n_f, the filter's resampling decision, ready for
 * rs_resample_batched_masked and rs_reset_weights_batched. F entries each on the device;
 * any of the three pointers may be NULL, not all. One CTA per filter, the arithmetic of
 * rs_log_sum_weights_batched with the sum of squares beside the sum. An empty or all-zero
 * filter gets ess 0, log total -inf and below 0 (no error); NaN/+inf flag RS_ERR_NONFINITE;
 * offsets outside [0, the handle's max_n] flag RS_ERR_ARG; RS_ERR_ARG on the host for
 * threshold_frac outside [0, 1] when below_dev is given. */
int rs_ess_batched(rs_handle* h, int dtype, const void* logw_dev, const int64_t* offsets_dev,
                   int32_t F, double* ess_dev, double* log_total_dev, double threshold_frac,
                   uint8_t* below_dev, void* stream);

/* rs_resample_batched for the filters f with resample_dev[f] != 0 (F uint8 on the device);
 * every other filter keeps its particles: its ancestors are the identity a_i = i (with
 * permute, c_i = i). The flagged filters' ancestors are those of rs_resample_batched, bit
 * for bit. The resampling on demand of a batch of adaptive filters (Section 4.3), decided on
 * the device (rs_ess_batched's below flags) without a host round trip; the unflagged filters
 * skip every pass of the resampler (their NaN/+inf log-weights may go unchecked). Same
 * arguments and errors as rs_resample_batched otherwise. */
int rs_resample_batched_masked(rs_handle* h, int scheme, int dtype, const void* logw_dev,
                               const int64_t* offsets_dev, int32_t F, const int32_t* B_dev,
                               int32_t B, uint64_t seed, uint64_t step,
                               const uint8_t* resample_dev, int32_t* ancestors_dev,
                               int permute, const rs_opts* opts, void* stream);

/* After a masked resampling: the binary32 log-weights of every flagged filter (flags_dev[f]
 * != 0) set to 0 -- equal weights, the next step's log-likelihood terms are then added to
 * them -- the other filters' left as they are. */
int rs_reset_weights_batched(rs_handle* h, float* logw_dev, const int64_t* offsets_dev,
                             int32_t F, const uint8_t* flags_dev, void* stream);

/* Metropolis B picked per filter from its own weights: beta_dev[f] (may be NULL) = mean w /
 * max w over the filter's particles (the ratio of Eq. beta2, evaluated on the weights rather
 * than from the model) and B_dev[f] = B* of Eq. B (Section 2.1) for eps and that beta, i.e.
 * ceil(log eps / log(1 - beta)), at least 1 (1 for beta = 1, and for an empty or all-zero
 * filter, where beta is 0). F int32 / float64 on the device, ready to pass as B_dev to
 * rs_resample_batched without a host round trip. Same sums as rs_log_sum_weights_batched;
 * beta has the relative accuracy of those sums (about 1e-7 for binary32 weights), so B can
 * differ by one from a binary64 host evaluation where log eps / log(1 - beta) lies that close
 * to an integer. RS_ERR_ARG unless 0 < eps < 1; NaN/+inf flag RS_ERR_NONFINITE. */
int rs_metropolis_B_batched(rs_handle* h, int dtype, const void* logw_dev,
                            const int64_t* offsets_dev, int32_t F, double eps, int32_t* B_dev,
                            double* beta_dev, void* stream);

/* Launch shape of the particle-parallel kernels of rs_resample_batched: kernel
 * RS_BATCHED_METROPOLIS_F32 / _F64 (the per-particle Metropolis chains) or
 * RS_BATCHED_PERMUTE (Code 10 per filter); block = threads per CTA (a multiple of 32, 32 to
 * 512), items_per_thread = particles per thread (1 to 16). The handle starts at 256 x 1. Only
 * the speed depends on the shape: every particle's draws, chain, claim and slot are the same
 * for any shape. RS_ERR_ARG for an unknown kernel or shape. Host-only. */
#define RS_BATCHED_METROPOLIS_F32 0
#define RS_BATCHED_METROPOLIS_F64 1
#define RS_BATCHED_PERMUTE 2
int rs_set_batched_launch(rs_handle* h, int kernel, int block, int items_per_thread);
int rs_get_batched_launch(rs_handle* h, int kernel, int* block, int* items_per_thread);

/* Autotuner of the batched Metropolis path on the caller's own batch (the arguments of
 * rs_resample_batched with scheme RS_METROPOLIS): times every shape block in {128, 256, 512} x
 * items per thread in {1, 2, 4} with CUDA events over `reps` calls (after one untimed call),
 * first for the Metropolis kernel of `dtype` alone, then for Permute with that choice, and
 * keeps the fastest of each in the handle (read them with rs_get_batched_launch). The calls
 * write only the handle's scratch. Synchronises `stream` once per shape; RS_ERR_ARG on a
 * stream being captured or reps outside 1..1000; the argument errors of rs_resample_batched;
 * RS_ERR_CUDA if a timed call fails (the previous shapes are restored). */
int rs_tune_batched(rs_handle* h, int dtype, const void* logw_dev, const int64_t* offsets_dev,
                    int32_t F, const int32_t* B_dev, int32_t B, int reps, void* stream);

/* B* = log(eps) / log(1 - beta) of Eq. (B) (Section 2.1), rounded up: the number of
 * Metropolis steps that bounds the total-variation distance of every chain by eps, for a
 * lower bound beta on min_i(mean(w)/w^i) (Eq. beta), e.g. E(w)/w_max (Eq. beta2).
 * Host-only; writes *B. RS_ERR_ARG unless 0 < eps < 1 and 0 < beta <= 1. */
int rs_metropolis_B(double eps, double beta, int32_t* B);

/* Synchronises `stream`, returns the first (highest-priority) device-side status recorded
 * since the previous rs_last_error on this handle, and clears it. */
int rs_last_error(rs_handle* h, void* stream);

/* Per-kernel timing (an instrumentation aid; the paper times whole calls, Section 4.4).
 * rs_trace(h, events, n) hands the handle n cudaEvent_t (as void*, created by the caller
 * with timing enabled); until the next rs_trace call, every call on h records the next
 * unused event on its stream before each kernel it launches and once after its last
 * kernel. rs_trace(h, NULL, 0) stops tracing. Events are not recorded while the stream is
 * being captured into a CUDA graph (do not trace during capture). rs_trace_count returns
 * how many events were recorded; rs_trace_label(h, i) names the kernel that follows event
 * i ("end" after the last kernel of a call), or NULL for i out of range. */
int rs_trace(rs_handle* h, void* const* events, int n);
int rs_trace_count(const rs_handle* h);
const char* rs_trace_label(const rs_handle* h, int i);

/* ---- systematic resampling without any allocation ------------------------------------
 * The paper has no counterpart to this call: it exists for callers that cannot allocate
 * device memory -- code running under another framework's memory pool or allocator hooks,
 * plugins whose host forbids cudaMalloc after start-up, real-time loops that must never wait
 * on the allocator. It computes exactly what rs_resample(RS_SYSTEMATIC, permute = 0) computes
 * (same kernels, same results) without a handle: its scratch (about 530 KB) is a static
 * device array of the library, which every GPU that loads the library keeps until the
 * process exits. The caller passes only inputs and outputs:
 *   dtype, logw_dev, N : as for rs_resample; 1 <= N <= RS_NOALLOC_MAX_N, larger N returns
 *                        RS_ERR_CAPACITY before anything is launched.
 *   seed, step         : as for rs_resample (filter 0).
 *   ancestors_dev      : N int32 outputs, non-decreasing.
 *   status_dev         : NULL, or one device int32 that receives RS_OK or the device-side
 *                        status (the codes of rs_last_error) when the stream reaches the end
 *                        of the call.
 * logw_dev, ancestors_dev and status_dev must be memory of the current device (or managed
 * memory): a pointer of another device or of host memory returns RS_ERR_ARG before anything
 * is launched. The device address of the static array is looked up once per device
 * (cudaGetSymbolAddress, with that device current) by the first call or by rs_create on
 * that device, and kept for the life of the process. The lookup is not made while `stream`
 * is being captured: a first call inside a capture, with neither an earlier call nor a
 * handle on that device, returns RS_ERR_ARG and launches nothing. Make no call on a device
 * after cudaDeviceReset on it (the kept address would be stale). All calls on a device share
 * the one array and overwrite it: calls that overlap on the GPU (several streams or host
 * threads at once) race and must be serialised by the caller. The call allocates and frees
 * nothing. */
#define RS_NOALLOC_MAX_N (1 << 22)
int rs_systematic_noalloc(int dtype, const void* logw_dev, int64_t N, uint64_t seed,
                          uint64_t step, int32_t* ancestors_dev, int32_t* status_dev,
                          void* stream);

/* Human-readable text of a status code (static storage). */
const char* rs_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* RS_RESAMPLE_H */
