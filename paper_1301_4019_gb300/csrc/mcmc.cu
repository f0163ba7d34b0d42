// mcmc.cu -- the collective-free resamplers of Section 2 on sm_103a: Metropolis (Section
// 2.1, Code 2) and rejection (Section 2.2, Code 3), each with the Prepermute claim of Code
// 10 fused at the end (Appendix E: "append Prepermute to any procedure that produces an
// ancestry vector").
//
// One thread per particle. Every draw is counter-based (Philox keyed by particle and inner
// step), so the random numbers of step n do not depend on the chain state: the proposals and
// their log-weight gathers of several steps are issued together and only the accept
// decisions run in sequence.
#include "common.cuh"
#include "internal.h"

namespace rsk {
namespace {

// u < w^j / w^k from log-weights: a ratio >= 1 or a zero-weight current state accepts.
template <typename T>
__device__ __forceinline__ bool metropolis_accept(T lwk, T lwj, T u) {
  if (lwk == neg_inf<T>()) return true;
  const T delta = lwj - lwk;
  if (delta >= T(0)) return true;
  return u < exp_pinned(delta);
}

constexpr int kUnroll = 4;

template <typename T>
__global__ void __launch_bounds__(kBlock)
metropolis_kernel(const T* __restrict__ lw, int64_t N, int32_t B, Keys keys,
                  int32_t* __restrict__ a, int32_t* __restrict__ d, int* err) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  T lwk = __ldg(lw + i);
  if (nonfinite_logw(lwk)) flag_error(err, RS_ERR_NONFINITE);
  int64_t k = i;
  const uint32_t ii = static_cast<uint32_t>(i);
  int32_t n = 0;
  for (; n + kUnroll <= B; n += kUnroll) {
    T u[kUnroll], lwj[kUnroll];
    int64_t j[kUnroll];
#pragma unroll
    for (int s = 0; s < kUnroll; ++s) {
      const uint4 x = draw(keys, ii, static_cast<uint32_t>(n + s));
      j[s] = uniform_index(x, N);
      u[s] = u01<T>(x);
      lwj[s] = __ldg(lw + j[s]);
    }
#pragma unroll
    for (int s = 0; s < kUnroll; ++s) {
      if (metropolis_accept(lwk, lwj[s], u[s])) {
        k = j[s];
        lwk = lwj[s];
      }
    }
  }
  for (; n < B; ++n) {
    const uint4 x = draw(keys, ii, static_cast<uint32_t>(n));
    const int64_t j = uniform_index(x, N);
    const T lwj = __ldg(lw + j);
    if (metropolis_accept(lwk, lwj, u01<T>(x))) {
      k = j;
      lwk = lwj;
    }
  }
  a[i] = static_cast<int32_t>(k);
  if (d) atomicMin(d + k, static_cast<int32_t>(i));
}

// Attempt 0 proposes j = i; attempt n >= 1 a uniform j; both draw u from counter (i, n).
// Accept when u < exp(lw^j - log w_max). A log-weight above the bound is flagged and
// accepted; max_trials attempts without acceptance keep a^i = i and flag the cap.
template <typename T>
__global__ void __launch_bounds__(kBlock)
rejection_kernel(const T* __restrict__ lw, int64_t N, T lwmax, int64_t max_trials, Keys keys,
                 int32_t* __restrict__ a, int32_t* __restrict__ d, int* err) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const T lwi = __ldg(lw + i);
  if (nonfinite_logw(lwi)) flag_error(err, RS_ERR_NONFINITE);
  const uint32_t ii = static_cast<uint32_t>(i);
  int64_t j = i;
  bool accepted = false, bound = false;
  for (int64_t n = 0; n < max_trials; ++n) {
    const uint4 x = draw(keys, ii, static_cast<uint32_t>(n));
    if (n > 0) j = uniform_index(x, N);
    const T u = u01<T>(x);
    const T lwj = (n == 0) ? lwi : __ldg(lw + j);
    const T delta = lwj - lwmax;
    if (delta > T(0)) {
      bound = true;
      accepted = true;
      break;
    }
    if (delta == T(0) || u < exp_pinned(delta)) {
      accepted = true;
      break;
    }
  }
  if (bound) flag_error(err, RS_ERR_BOUND_VIOLATED);
  if (!accepted) {
    j = i;
    flag_error(err, RS_ERR_REJECTION_CAP);
  }
  a[i] = static_cast<int32_t>(j);
  if (d) atomicMin(d + j, static_cast<int32_t>(i));
}

}  // namespace

cudaError_t launch_metropolis(const Scratch& s, bool f64, const void* logw, int64_t N,
                              int32_t B, uint64_t seed, uint64_t step, uint32_t filter,
                              int32_t* a_out, int32_t* d, cudaStream_t st) {
  const Keys keys = make_keys(seed, step, filter, RS_METROPOLIS);
  const int grid = static_cast<int>((N + kBlock - 1) / kBlock);
  trace_mark(s.trace, f64 ? "metropolis_f64" : "metropolis_f32", st);
  if (f64)
    metropolis_kernel<double><<<grid, kBlock, 0, st>>>(static_cast<const double*>(logw), N, B,
                                                       keys, a_out, d, s.err);
  else
    metropolis_kernel<float><<<grid, kBlock, 0, st>>>(static_cast<const float*>(logw), N, B,
                                                      keys, a_out, d, s.err);
  return cudaGetLastError();
}

cudaError_t launch_rejection(const Scratch& s, bool f64, const void* logw, int64_t N,
                             double log_wmax, int64_t max_trials, uint64_t seed,
                             uint64_t step, uint32_t filter, int32_t* a_out, int32_t* d,
                             cudaStream_t st) {
  const Keys keys = make_keys(seed, step, filter, RS_REJECTION);
  const int grid = static_cast<int>((N + kBlock - 1) / kBlock);
  trace_mark(s.trace, f64 ? "rejection_f64" : "rejection_f32", st);
  if (f64)
    rejection_kernel<double><<<grid, kBlock, 0, st>>>(static_cast<const double*>(logw), N,
                                                      log_wmax, max_trials, keys, a_out, d,
                                                      s.err);
  else
    rejection_kernel<float><<<grid, kBlock, 0, st>>>(static_cast<const float*>(logw), N,
                                                     static_cast<float>(log_wmax), max_trials,
                                                     keys, a_out, d, s.err);
  return cudaGetLastError();
}

}  // namespace rsk
