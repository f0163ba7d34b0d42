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

// ---------------------------------------------------------------------------------------
// Binary64 decisions on the binary32 pipes. GB300 runs binary64 arithmetic at 1/57 of the
// binary32 rate, so the binary64 test  u < exp(lw_j - lw_k)  is first decided with binary32
// arithmetic and a rigorous error bound, and evaluated exactly (binary64 subtraction,
// pinned binary64 exp, 53-bit u) only when u falls inside the uncertainty band. The outcome
// is therefore identical to the binary64 definition; the band has relative width about
// 2^-21 + 2^-23 (|lw_j| + |lw_k|), so the exact path runs for a few draws per million.
// ---------------------------------------------------------------------------------------

// Truncation of a finite binary64 to binary32 with integer operations only: |x - f| <
// 2^-23 |x| + 2^-126. Returns false (f unusable) for inf, NaN or |x| >= 2^128.
__device__ __forceinline__ bool f64_to_f32_trunc(double x, float& f) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned int sign = static_cast<unsigned int>(b >> 32) & 0x80000000u;
  const int e = static_cast<int>((b >> 52) & 0x7ffu);
  if (e == 0x7ff) return false;
  const int fe = e - 1023 + 127;
  if (fe >= 255) return false;
  if (fe <= 0) {  // below the binary32 normal range (or zero): 0, absolute error < 2^-126
    f = __uint_as_float(sign);
    return true;
  }
  const unsigned int m = static_cast<unsigned int>((b >> 29) & 0x7fffffu);
  f = __uint_as_float(sign | (static_cast<unsigned int>(fe) << 23) | m);
  return true;
}

// Order-preserving signed key of a binary64 (for exact comparisons without the FP64 pipe).
__device__ __forceinline__ long long f64_key(double x) {
  const long long b = __double_as_longlong(x);
  return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}

// Decides u < exp_pinned(lwj - lwk) for lwj < lwk, lwk > -inf, with u = 53-bit u01 of x.
// lwj_f / lwk_f are binary32 truncations (valid flags as returned above).
__device__ __noinline__ bool exact_f64_less_exp(double lwj, double lwk, uint4 x) {
  return u01_f64(x) < exp_pinned(__dsub_rn(lwj, lwk));
}

__device__ __forceinline__ bool f64_accept_lt(double lwj, float lwj_f, bool okj, double lwk,
                                              float lwk_f, bool okk, uint4 x) {
  if (!(okj && okk)) return exact_f64_less_exp(lwj, lwk, x);
  const float df = __fsub_rn(lwj_f, lwk_f);  // <= 0 up to rounding
  // bound on |df - (lwj - lwk)|: both truncations, the subtraction's rounding, margin
  const float E = __fmaf_ru(fabsf(lwj_f) + fabsf(lwk_f), 0x1p-23f,
                            __fmaf_ru(fabsf(df), 0x1p-24f, 0x1p-124f));
  if (!(E < 0.01f)) return exact_f64_less_exp(lwj, lwk, x);
  // u lies in [x0 2^-32, (x0 + 1) 2^-32)
  const float u_lo = __fmul_rn(__uint2float_rd(x.x), 0x1p-32f);
  const float u_hi = __fmul_rn(__fadd_ru(__uint2float_ru(x.x), 1.0f), 0x1p-32f);
  const float ef = exp_pinned(df);
  if (ef == 0.0f) {  // exp(df) < 2^-124: the binary64 ratio is below e^-86 < 2^-32 <= u
    if (x.x != 0u) return false;
    return exact_f64_less_exp(lwj, lwk, x);
  }
  // exp(lwj - lwk) within ef * exp(+-E) * (1 +- 2^-23) (1 +- 2^-52); m bounds all of it
  const float m = __fmaf_ru(E, 1.02f, 0x1p-21f);
  const float lo = __fmul_rd(ef, __fsub_rd(1.0f, m));
  const float hi = __fmul_ru(ef, __fadd_ru(1.0f, m));
  if (u_hi < lo) return true;
  if (u_lo >= hi) return false;
  return exact_f64_less_exp(lwj, lwk, x);
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

// Binary64 Metropolis with the decisions made on the binary32 pipes (same outcome as
// metropolis_kernel<double>).
__global__ void __launch_bounds__(kBlock)
metropolis_f64_kernel(const double* __restrict__ lw, int64_t N, int32_t B, Keys keys,
                      int32_t* __restrict__ a, int32_t* __restrict__ d, int* err) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  double lwk = __ldg(lw + i);
  if (nonfinite_logw(lwk)) flag_error(err, RS_ERR_NONFINITE);
  float lwk_f;
  bool okk = f64_to_f32_trunc(lwk, lwk_f);
  long long kk = f64_key(lwk);
  const long long kNegInf = f64_key(-INFINITY);
  int64_t k = i;
  const uint32_t ii = static_cast<uint32_t>(i);
  int32_t n = 0;
  for (; n + kUnroll <= B; n += kUnroll) {
    uint4 x[kUnroll];
    double lwj[kUnroll];
    int64_t j[kUnroll];
#pragma unroll
    for (int s = 0; s < kUnroll; ++s) {
      x[s] = draw(keys, ii, static_cast<uint32_t>(n + s));
      j[s] = uniform_index(x[s], N);
      lwj[s] = __ldg(lw + j[s]);
    }
#pragma unroll
    for (int s = 0; s < kUnroll; ++s) {
      const long long kj = f64_key(lwj[s]);
      float lwj_f;
      const bool okj = f64_to_f32_trunc(lwj[s], lwj_f);
      bool acc;
      if (kk == kNegInf || kj >= kk) acc = true;          // zero-weight state, ratio >= 1
      else if (kj == kNegInf) acc = false;                 // zero-weight proposal
      else acc = f64_accept_lt(lwj[s], lwj_f, okj, lwk, lwk_f, okk, x[s]);
      if (acc) {
        k = j[s];
        lwk = lwj[s];
        lwk_f = lwj_f;
        okk = okj;
        kk = kj;
      }
    }
  }
  for (; n < B; ++n) {
    const uint4 x = draw(keys, ii, static_cast<uint32_t>(n));
    const int64_t j = uniform_index(x, N);
    const double lwj = __ldg(lw + j);
    const long long kj = f64_key(lwj);
    float lwj_f;
    const bool okj = f64_to_f32_trunc(lwj, lwj_f);
    bool acc;
    if (kk == kNegInf || kj >= kk) acc = true;
    else if (kj == kNegInf) acc = false;
    else acc = f64_accept_lt(lwj, lwj_f, okj, lwk, lwk_f, okk, x);
    if (acc) {
      k = j;
      lwk = lwj;
      lwk_f = lwj_f;
      okk = okj;
      kk = kj;
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

// Binary64 rejection with the decisions made on the binary32 pipes (same outcome as
// rejection_kernel<double>).
__global__ void __launch_bounds__(kBlock)
rejection_f64_kernel(const double* __restrict__ lw, int64_t N, double lwmax, int64_t max_trials,
                     Keys keys, int32_t* __restrict__ a, int32_t* __restrict__ d, int* err) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double lwi = __ldg(lw + i);
  if (nonfinite_logw(lwi)) flag_error(err, RS_ERR_NONFINITE);
  float lwmax_f;
  const bool okm = f64_to_f32_trunc(lwmax, lwmax_f);
  const long long km = f64_key(lwmax);
  const long long kNegInf = f64_key(-INFINITY);
  const uint32_t ii = static_cast<uint32_t>(i);
  int64_t j = i;
  bool accepted = false, bound = false;
  for (int64_t n = 0; n < max_trials; ++n) {
    const uint4 x = draw(keys, ii, static_cast<uint32_t>(n));
    if (n > 0) j = uniform_index(x, N);
    const double lwj = (n == 0) ? lwi : __ldg(lw + j);
    const long long kj = f64_key(lwj);
    if (kj > km && lwj == lwj) {  // above the bound (NaN never compares)
      bound = true;
      accepted = true;
      break;
    }
    if (kj == km) {  // ratio exactly 1
      accepted = true;
      break;
    }
    if (kj == kNegInf || lwj != lwj) continue;
    float lwj_f;
    const bool okj = f64_to_f32_trunc(lwj, lwj_f);
    if (f64_accept_lt(lwj, lwj_f, okj, lwmax, lwmax_f, okm, x)) {
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
    metropolis_f64_kernel<<<grid, kBlock, 0, st>>>(static_cast<const double*>(logw), N, B, keys,
                                                   a_out, d, s.err);
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
    rejection_f64_kernel<<<grid, kBlock, 0, st>>>(static_cast<const double*>(logw), N, log_wmax,
                                                  max_trials, keys, a_out, d, s.err);
  else
    rejection_kernel<float><<<grid, kBlock, 0, st>>>(static_cast<const float*>(logw), N,
                                                     static_cast<float>(log_wmax), max_trials,
                                                     keys, a_out, d, s.err);
  return cudaGetLastError();
}

}  // namespace rsk
