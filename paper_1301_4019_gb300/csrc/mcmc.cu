// mcmc.cu -- the collective-free resamplers of Section 2 on sm_103a: Metropolis (Section
// 2.1, Code 2) and rejection (Section 2.2, Code 3), one thread per particle, each with the
// Prepermute claim of Code 10 fused at the end (Appendix E: the claim is appended to every
// procedure that produces an ancestry vector).
//
// Every draw is counter-based (Philox keyed by particle and inner step), so the random
// numbers of step s do not depend on the chain state: the proposals and their log-weight
// gathers of several steps are issued together and only the accept decisions run in
// sequence (mcmc.cuh).
#include "common.cuh"
#include "internal.h"
#include "mcmc.cuh"

namespace rsk {
namespace {

template <typename T>
__global__ void __launch_bounds__(kBlock)
metropolis_kernel(const T* __restrict__ lw, int64_t N, int32_t B, Keys keys,
                  int32_t* __restrict__ a, int32_t* __restrict__ d, int* err) {
  pdl_wait();
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int32_t k = metropolis_one(lw, N, B, keys, i, err);
  a[i] = k;
  if (d) atomicMin(d + k, static_cast<int32_t>(i));
}

// Rejection with warp refill (mcmc.cuh): warp w owns particles [w * kRejRun, ...).
template <typename T>
__global__ void __launch_bounds__(kBlock)
rejection_kernel(const T* __restrict__ lw, int64_t N, double log_wmax, int64_t max_trials,
                 Keys keys, int32_t* __restrict__ a, int32_t* __restrict__ d, int* err) {
  pdl_wait();
  const int lane = threadIdx.x & 31;
  const int64_t run = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t start = run * kRejRun;
  if (start >= N) return;  // uniform across the warp
  const int64_t end = start + kRejRun < N ? start + kRejRun : N;
  const RejBound rb = make_bound(log_wmax);
  int64_t i = start + lane;
  bool active = i < end;
  int64_t head = start + 32;
  uint32_t s = 0;
  T lwi = active ? __ldg(lw + i) : T(0);
  if (active && nonfinite_logw(lwi)) flag_error(err, RS_ERR_NONFINITE);
  for (;;) {
    bool settled = false;
    if (active) {
      int64_t j;
      settled = rejection_attempt(lw, N, rb, keys, i, s, lwi, j, err);
      ++s;
      if (!settled && s >= static_cast<uint64_t>(max_trials)) {
        flag_error(err, RS_ERR_REJECTION_CAP);
        j = i;
        settled = true;
      }
      if (settled) {
        a[i] = static_cast<int32_t>(j);
        if (d) atomicMin(d + j, static_cast<int32_t>(i));
      }
    }
    const unsigned done = __ballot_sync(0xffffffffu, settled);
    if (settled) {
      i = head + __popc(done & ((1u << lane) - 1u));
      active = i < end;
      s = 0;
      if (active) {
        lwi = __ldg(lw + i);
        if (nonfinite_logw(lwi)) flag_error(err, RS_ERR_NONFINITE);
      }
    }
    head += __popc(done);
    if (!__any_sync(0xffffffffu, active)) break;
  }
}

}  // namespace

cudaError_t launch_metropolis(const Scratch& s, bool f64, const void* logw, int64_t N,
                              int32_t B, uint64_t seed, uint64_t step, uint32_t filter,
                              int32_t* a_out, int32_t* d, cudaStream_t st) {
  const Keys keys = make_keys(seed, step, filter, RS_METROPOLIS);
  const int grid = static_cast<int>((N + kBlock - 1) / kBlock);
  trace_mark(s.trace, f64 ? "metropolis_f64" : "metropolis_f32", st);
  if (f64)
    launch_pdl(metropolis_kernel<double>, grid, kBlock, st, static_cast<const double*>(logw), N, B,
                                                       keys, a_out, d, s.err);
  else
    launch_pdl(metropolis_kernel<float>, grid, kBlock, st, static_cast<const float*>(logw), N, B,
                                                      keys, a_out, d, s.err);
  return cudaGetLastError();
}

cudaError_t launch_rejection(const Scratch& s, bool f64, const void* logw, int64_t N,
                             double log_wmax, int64_t max_trials, uint64_t seed,
                             uint64_t step, uint32_t filter, int32_t* a_out, int32_t* d,
                             cudaStream_t st) {
  const Keys keys = make_keys(seed, step, filter, RS_REJECTION);
  const int64_t runs = (N + kRejRun - 1) / kRejRun;
  const int grid = static_cast<int>((runs * 32 + kBlock - 1) / kBlock);
  trace_mark(s.trace, f64 ? "rejection_f64" : "rejection_f32", st);
  if (f64)
    launch_pdl(rejection_kernel<double>, grid, kBlock, st, static_cast<const double*>(logw), N,
                                                      log_wmax, max_trials, keys, a_out, d,
                                                      s.err);
  else
    launch_pdl(rejection_kernel<float>, grid, kBlock, st, static_cast<const float*>(logw), N,
                                                     log_wmax, max_trials, keys, a_out, d,
                                                     s.err);
  return cudaGetLastError();
}

}  // namespace rsk
