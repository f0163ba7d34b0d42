/*
 * resample_measure.h -- measurement aids and self-checks of the resampling library (C ABI,
 * same conventions as resample.h).
 *
 * The Metropolis (Section 2.1, Code 2) and rejection (Section 2.2, Code 3) resamplers spend
 * their time drawing random numbers: one Philox4x32-10 block (Salmon et al., SC'11) per
 * proposal. Their roofline is the device's Philox throughput, which no vendor figure gives;
 * rs_philox_throughput measures it with the same Philox code the resamplers run.
 *
 * Their acceptance tests u < w^j / w^k (Code 2) and u < w^j / w_max (Code 3) are decided from
 * cheap estimates with an exact fallback; rs_check_acceptance counts, with the device functions
 * the resamplers run, the cases where such a shortcut would decide otherwise than the
 * definition u < exp(delta) with the library's pinned exp.
 */
#ifndef RS_RESAMPLE_MEASURE_H
#define RS_RESAMPLE_MEASURE_H

#include <stdint.h>

#include "resample.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Philox throughput kernel: thread i (0 <= i < threads, 256 per CTA) draws the blocks with
 * counter (i, n, 0, 6) for n < draws_per_thread under key = seed (the resamplers' counter
 * layout with step 0, filter 0 and purpose 6, which no resampler uses) and XORs their four
 * words; *xor_dev (one uint32 on the device, set to 0 by the call) receives the XOR over all
 * threads, which keeps every draw live and lets a test check the draws against a host
 * implementation. Time it with events on `stream`: threads * draws_per_thread blocks per
 * launch. RS_ERR_ARG unless 1 <= threads <= 2^32 and draws_per_thread >= 1. */
int rs_philox_throughput(rs_handle* h, int64_t threads, uint32_t draws_per_thread,
                         uint64_t seed, uint32_t* xor_dev, void* stream);

/* Self-check of the bounded grid barrier (no counterpart in the paper): one cooperative
 * launch on `stream` whose grid barrier expects one arrival more than its CTAs make, so every
 * CTA waits for the handle's barrier timeout (rs_set_barrier_timeout), records RS_ERR_TIMEOUT
 * and ends. rs_last_error then returns RS_ERR_TIMEOUT and resets the barrier state; the
 * handle's next calls run normally. RS_ERR_CUDA without cooperative launches. */
int rs_check_barrier_timeout(rs_handle* h, void* stream);

/* Self-check of the acceptance tests (Codes 2 and 3, the ratio formed from log-weight
 * differences as in Appendix E). Writes to *count_dev (one uint64 on the current device) the
 * number of wrong decisions found:
 *   mode 0: every binary32 delta in [-86.5, 0) (1,118,633,984 values): the binary32 test
 *           compares u with a band of relative half-width 2^-15 around the hardware ex2
 *           estimate of exp(delta) and evaluates the pinned exp only inside it; counted are
 *           the delta whose pinned exp lies outside the band (n is ignored);
 *   mode 1: n log-weight pairs (lw_j < lw_k, lw_k in {0, -2.75, -1234.5678, 30000.5}, lw_j -
 *           lw_k spread over [-90, 0)), each with uniforms on the 53-bit grid at and next to
 *           the boundary exp(lw_j - lw_k) and at relative distances 2^-20, 2^-15 and 2^-10
 *           from it, plus two arbitrary ones: the binary64 decision taken on the binary32
 *           pipes against the binary64 definition.
 * Asynchronous on `stream` (the count is valid after the stream reaches it). RS_ERR_ARG for an
 * unknown mode, n < 1 (mode 1) or a null count_dev; RS_ERR_CUDA if a launch fails. */
int rs_check_acceptance(int mode, int64_t n, unsigned long long* count_dev, void* stream);

/* Self-check of the exponential of the plain binary32 scans (the weights exp(lw - M) that the
 * multinomial, stratified and systematic resamplers of Codes 5, 7 and 8 sum in plain binary32;
 * every other path uses the pinned exponential). Over every binary32 t <= 0 (-0 through -inf,
 * 2,139,095,041 values), with the device function the scans run, against the binary64 pinned
 * exponential: *count_dev (one uint64 on the current device) receives the number of t in
 * [-87, 0] whose relative error exceeds `bound`, plus the number of t < -87 whose result lies
 * outside [0, 2^-125]; *max_rel_dev (one binary64 on the same device) the largest relative
 * error over [-87, 0]. The parity tolerance of the plain binary32 scans assumes the bound
 * 2^-21. Asynchronous on `stream` (the results are valid after the stream reaches them).
 * RS_ERR_ARG for a null pointer or bound <= 0; RS_ERR_CUDA if a launch fails. */
int rs_check_weight_exp(double bound, unsigned long long* count_dev, double* max_rel_dev,
                        void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RS_RESAMPLE_MEASURE_H */
