/*
 * resample_measure.h -- measurement aids of the resampling library (C ABI, same conventions
 * as resample.h).
 *
 * The Metropolis (Section 2.1, Code 2) and rejection (Section 2.2, Code 3) resamplers spend
 * their time drawing random numbers: one Philox4x32-10 block (Salmon et al., SC'11) per
 * proposal. Their roofline is the device's Philox throughput, which no vendor figure gives;
 * this call measures it with the same Philox code the resamplers run.
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

#ifdef __cplusplus
}
#endif

#endif /* RS_RESAMPLE_MEASURE_H */
