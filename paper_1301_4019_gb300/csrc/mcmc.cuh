// mcmc.cuh -- per-particle bodies of the collective-free resamplers of Section 2: the
// Metropolis chain of Code 2 and the rejection loop of Code 3, shared by the single-filter
// and batched kernels. Binary64 decisions are made on the binary32 pipes with an exact
// fallback (same outcome as the binary64 definition).
#pragma once

#include <cstdint>

#include "common.cuh"

namespace rsk {
namespace {

// ---------------------------------------------------------------------------------------
// The acceptance test u < exp_pinned(delta) (delta < 0) without evaluating the pinned
// polynomial in almost every case. e = 2^(delta log2 e) from the hardware approximation
// (PTX ex2.approx) is within a relative 1e-5 of exp(delta) for delta >= -86.5: rounding
// delta * log2 e (relative 2^-24, plus 2^-25.6 for log2 e in binary32) moves the exponent by
// at most 86.5 * 8e-8 = 7e-6 in relative terms of the result, the approximation itself is
// accurate to about 2^-22, and exp_pinned is within 2^-22 of exp. exp_pinned(delta) therefore
// lies in [e (1 - 2^-15), e (1 + 2^-15)] (a margin of about 4x), so u below the lower end
// accepts, u at or above the upper end rejects, and only u inside the band (probability
// about 6e-5 e) evaluates exp_pinned: the decision is that of u < exp_pinned(delta) always.
// Below -86.5 exp_pinned is 0 and NaN compares false, so the test is false there.
// ---------------------------------------------------------------------------------------
constexpr float kExpBand = 0x1p-15f;

__device__ __forceinline__ float exp_band_estimate(float delta) {
  float e;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(__fmul_rn(delta, 0x1.715476p+0f)));
  return e;
}

__device__ __forceinline__ bool u_below_exp(float u, float delta) {
  if (!(delta >= -86.5f)) return false;
  const float e = exp_band_estimate(delta);
  if (u < __fmul_rd(e, 1.0f - kExpBand)) return true;
  if (u >= __fmul_ru(e, 1.0f + kExpBand)) return false;
  return u < exp_pinned(delta);
}

// u < w^j / w^k from log-weights: a ratio >= 1 or a zero-weight current state accepts.
template <typename T>
__device__ __forceinline__ bool metropolis_accept(T lwk, T lwj, T u) {
  if (lwk == neg_inf<T>()) return true;
  const T delta = lwj - lwk;
  if (delta >= T(0)) return true;
  return u < exp_pinned(delta);
}
__device__ __forceinline__ bool metropolis_accept(float lwk, float lwj, float u) {
  if (lwk == neg_inf<float>()) return true;
  const float delta = lwj - lwk;
  if (delta >= 0.0f) return true;
  return u_below_exp(u, delta);
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

// The filter of f64_accept_lt on usable truncations lwj_f, lwk_f: true / false where they
// decide, else exact() -- the binary64 test, which the caller evaluates only then (so its
// binary64 log-weights are read only then).
template <typename Exact>
__device__ __forceinline__ bool f64_filter_lt(float lwj_f, float lwk_f, uint4 x, const Exact& exact) {
  const float df = __fsub_rn(lwj_f, lwk_f);  // <= 0 up to rounding
  // bound on |df - (lwj - lwk)|: both truncations, the subtraction's rounding, margin
  const float E = __fmaf_ru(fabsf(lwj_f) + fabsf(lwk_f), 0x1p-23f,
                            __fmaf_ru(fabsf(df), 0x1p-24f, 0x1p-124f));
  if (!(E < 0.01f)) return exact();
  // u lies in [x0 2^-32, (x0 + 1) 2^-32)
  const float u_lo = __fmul_rn(__uint2float_rd(x.x), 0x1p-32f);
  const float u_hi = __fmul_rn(__fadd_ru(__uint2float_ru(x.x), 1.0f), 0x1p-32f);
  if (!(df >= -86.5f)) {  // exp(df) < 2^-124: the binary64 ratio is below e^-86 < 2^-32 <= u
    if (x.x != 0u) return false;
    return exact();
  }
  // ef = exp(df) within a relative 1e-5 (exp_band_estimate); exp(lwj - lwk) within
  // ef * exp(+-E) * (1 +- 1e-5) (1 +- 2^-52): m bounds all of it
  const float ef = exp_band_estimate(df);
  const float m = __fmaf_ru(E, 1.02f, kExpBand);
  const float lo = __fmul_rd(ef, __fsub_rd(1.0f, m));
  const float hi = __fmul_ru(ef, __fadd_ru(1.0f, m));
  if (u_hi < lo) return true;
  if (u_lo >= hi) return false;
  return exact();
}

__device__ __forceinline__ bool f64_accept_lt(double lwj, float lwj_f, bool okj, double lwk,
                                              float lwk_f, bool okk, uint4 x) {
  if (!(okj && okk)) return exact_f64_less_exp(lwj, lwk, x);
  return f64_filter_lt(lwj_f, lwk_f, x, [&] { return exact_f64_less_exp(lwj, lwk, x); });
}

// ---------------------------------------------------------------------------------------
// Binary32 sidecar of binary64 log-weights. The binary64 chains gather a 4-byte sidecar per
// proposal instead of the 8-byte log-weight: the truncation of lw_j to binary32 when usable,
// -inf for lw_j = -inf, a NaN otherwise (NaN, +inf, or beyond the binary32 range). Truncation
// is monotone, so t_j > t_k implies lw_j > lw_k and t_j < t_k implies lw_j < lw_k; the
// binary64 values are read only when the sidecars are equal or NaN, and for the exact
// fallback of the filter. Every decision equals the one taken from the binary64 values.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float f64_sidecar(double x) {
  float f;
  if (f64_to_f32_trunc(x, f)) return f;
  return is_neg_inf(x) ? -INFINITY : __int_as_float(0x7fffffff);
}

constexpr int kUnroll = 4;    // binary32 chains: proposals issued together
constexpr int kUnroll64 = 4;  // binary64 chains (2 measured slower)

// Metropolis chain of particle i over n binary32 log-weights lw (Code 2): B steps; steps 2m
// and 2m + 1 take the two halves of the block of counter (i, m) (half_u01_f32, half_index),
// so a chain draws ceil(B / 2) blocks. Returns the ancestor.
__device__ __forceinline__ int32_t metropolis_one(const float* __restrict__ lw, int64_t n,
                                                  int32_t B, const Keys& keys, int64_t i,
                                                  int* err) {
  static_assert(kUnroll % 2 == 0, "whole blocks per round");
  float lwk = __ldg(lw + i);
  if (nonfinite_logw(lwk)) flag_error(err, RS_ERR_NONFINITE);
  int64_t k = i;
  const uint32_t ii = static_cast<uint32_t>(i);
  int32_t s = 0;
  for (; s + kUnroll <= B; s += kUnroll) {  // (s even)
    float u[kUnroll], lwj[kUnroll];
    int64_t j[kUnroll];
#pragma unroll
    for (int p = 0; p < kUnroll / 2; ++p) {
      const uint4 x = draw(keys, ii, static_cast<uint32_t>(s / 2 + p));
      j[2 * p] = half_index(x.x, x.y, n);
      u[2 * p] = half_u01_f32(x.x);
      j[2 * p + 1] = half_index(x.z, x.w, n);
      u[2 * p + 1] = half_u01_f32(x.z);
      lwj[2 * p] = __ldg(lw + j[2 * p]);
      lwj[2 * p + 1] = __ldg(lw + j[2 * p + 1]);
    }
#pragma unroll
    for (int q = 0; q < kUnroll; ++q) {
      if (metropolis_accept(lwk, lwj[q], u[q])) {
        k = j[q];
        lwk = lwj[q];
      }
    }
  }
  for (; s < B; s += 2) {  // the last B mod kUnroll steps, a block per two
    const uint4 x = draw(keys, ii, static_cast<uint32_t>(s / 2));
    const int64_t j0 = half_index(x.x, x.y, n);
    const float lwj0 = __ldg(lw + j0);
    if (metropolis_accept(lwk, lwj0, half_u01_f32(x.x))) {
      k = j0;
      lwk = lwj0;
    }
    if (s + 1 < B) {
      const int64_t j1 = half_index(x.z, x.w, n);
      const float lwj1 = __ldg(lw + j1);
      if (metropolis_accept(lwk, lwj1, half_u01_f32(x.z))) {
        k = j1;
        lwk = lwj1;
      }
    }
  }
  return static_cast<int32_t>(k);
}

__device__ __forceinline__ bool f64_step_accept(double lwk, float lwk_f, bool okk, long long kk,
                                                double lwj, float lwj_f, bool okj, long long kj,
                                                uint4 x) {
  const long long kNegInf = f64_key(-INFINITY);
  if (kk == kNegInf || kj >= kk) return true;  // zero-weight state, or ratio >= 1
  if (kj == kNegInf) return false;             // zero-weight proposal
  return f64_accept_lt(lwj, lwj_f, okj, lwk, lwk_f, okk, x);
}

__device__ __forceinline__ int32_t metropolis_one(const double* __restrict__ lw, int64_t n,
                                                  int32_t B, const Keys& keys, int64_t i,
                                                  int* err) {
  double lwk = __ldg(lw + i);
  if (nonfinite_logw(lwk)) flag_error(err, RS_ERR_NONFINITE);
  float lwk_f;
  bool okk = f64_to_f32_trunc(lwk, lwk_f);
  long long kk = f64_key(lwk);
  int64_t k = i;
  const uint32_t ii = static_cast<uint32_t>(i);
  int32_t s = 0;
  for (; s + kUnroll64 <= B; s += kUnroll64) {
    uint4 x[kUnroll64];
    double lwj[kUnroll64];
    int64_t j[kUnroll64];
#pragma unroll
    for (int q = 0; q < kUnroll64; ++q) {
      x[q] = draw(keys, ii, static_cast<uint32_t>(s + q));
      j[q] = uniform_index(x[q], n);
      lwj[q] = __ldg(lw + j[q]);
    }
#pragma unroll
    for (int q = 0; q < kUnroll64; ++q) {
      const long long kj = f64_key(lwj[q]);
      float lwj_f;
      const bool okj = f64_to_f32_trunc(lwj[q], lwj_f);
      if (f64_step_accept(lwk, lwk_f, okk, kk, lwj[q], lwj_f, okj, kj, x[q])) {
        k = j[q];
        lwk = lwj[q];
        lwk_f = lwj_f;
        okk = okj;
        kk = kj;
      }
    }
  }
  for (; s < B; ++s) {
    const uint4 x = draw(keys, ii, static_cast<uint32_t>(s));
    const int64_t j = uniform_index(x, n);
    const double lwj = __ldg(lw + j);
    const long long kj = f64_key(lwj);
    float lwj_f;
    const bool okj = f64_to_f32_trunc(lwj, lwj_f);
    if (f64_step_accept(lwk, lwk_f, okk, kk, lwj, lwj_f, okj, kj, x)) {
      k = j;
      lwk = lwj;
      lwk_f = lwj_f;
      okk = okj;
      kk = kj;
    }
  }
  return static_cast<int32_t>(k);
}

// A Metropolis step of a binary64 chain decided from sidecars (f64_sidecar): state k with
// sidecar tk, proposal j with tj; the binary64 log-weights lw[k], lw[j] are read only when the
// sidecars cannot decide. Same decision as f64_step_accept on the binary64 values.
__device__ __forceinline__ bool sc_step_accept(const double* __restrict__ lw, int64_t k, float tk,
                                               int64_t j, float tj, uint4 x) {
  if (tk == -INFINITY) return true;              // zero-weight state (tk = -inf iff lw_k = -inf)
  if (!(tj == tj) || !(tk == tk) || tj == tk) {  // undecided by the truncations
    const double lwk = __ldg(lw + k), lwj = __ldg(lw + j);
    float fk, fj;
    const bool okk = f64_to_f32_trunc(lwk, fk), okj = f64_to_f32_trunc(lwj, fj);
    return f64_step_accept(lwk, fk, okk, f64_key(lwk), lwj, fj, okj, f64_key(lwj), x);
  }
  if (tj > tk) return true;                      // lw_j > lw_k: ratio above 1
  if (tj == -INFINITY) return false;             // zero-weight proposal
  return f64_filter_lt(tj, tk, x,
                       [&] { return exact_f64_less_exp(__ldg(lw + j), __ldg(lw + k), x); });
}

// metropolis_one for binary64 log-weights with their sidecars lwf: the proposals gather
// 4 bytes (lwf[j]) instead of 8; same ancestor as metropolis_one.
__device__ __forceinline__ int32_t metropolis_one_sc(const double* __restrict__ lw,
                                                     const float* __restrict__ lwf, int64_t n,
                                                     int32_t B, const Keys& keys, int64_t i,
                                                     int* err) {
  const double lwi = __ldg(lw + i);
  if (nonfinite_logw(lwi)) flag_error(err, RS_ERR_NONFINITE);
  int64_t k = i;
  float tk = f64_sidecar(lwi);
  const uint32_t ii = static_cast<uint32_t>(i);
  int32_t s = 0;
  for (; s + kUnroll64 <= B; s += kUnroll64) {
    uint4 x[kUnroll64];
    int64_t j[kUnroll64];
    float tj[kUnroll64];
#pragma unroll
    for (int q = 0; q < kUnroll64; ++q) {
      x[q] = draw(keys, ii, static_cast<uint32_t>(s + q));
      j[q] = uniform_index(x[q], n);
      tj[q] = __ldg(lwf + j[q]);
    }
#pragma unroll
    for (int q = 0; q < kUnroll64; ++q) {
      if (sc_step_accept(lw, k, tk, j[q], tj[q], x[q])) {
        k = j[q];
        tk = tj[q];
      }
    }
  }
  for (; s < B; ++s) {
    const uint4 x = draw(keys, ii, static_cast<uint32_t>(s));
    const int64_t j = uniform_index(x, n);
    const float tj = __ldg(lwf + j);
    if (sc_step_accept(lw, k, tk, j, tj, x)) {
      k = j;
      tk = tj;
    }
  }
  return static_cast<int32_t>(k);
}

// Rejection loop of particle i (Code 3): attempt 0 proposes j = i, attempt s >= 1 a uniform
// j; binary64 attempts draw from counter (i, s), binary32 ones from half s mod 2 of the block
// of counter (i, floor(s/2)) (half_u01_f32, half_index); accept when u < exp(lw^j - log w_max).
// A log-weight above the bound is flagged and accepted; max_trials attempts without
// acceptance keep i and flag the cap.
__device__ __forceinline__ int32_t rejection_one(const float* __restrict__ lw, int64_t n,
                                                 double log_wmax, int64_t max_trials,
                                                 const Keys& keys, int64_t i, int* err) {
  const float lwmax = static_cast<float>(log_wmax);
  const float lwi = __ldg(lw + i);
  if (nonfinite_logw(lwi)) flag_error(err, RS_ERR_NONFINITE);
  const uint32_t ii = static_cast<uint32_t>(i);
  int64_t j = i;
  uint4 x = make_uint4(0u, 0u, 0u, 0u);
  for (int64_t s = 0; s < max_trials; ++s) {
    if ((s & 1) == 0) x = draw(keys, ii, static_cast<uint32_t>(s >> 1));
    const uint32_t w0 = (s & 1) ? x.z : x.x, w1 = (s & 1) ? x.w : x.y;
    if (s > 0) j = half_index(w0, w1, n);
    const float u = half_u01_f32(w0);
    const float lwj = (s == 0) ? lwi : __ldg(lw + j);
    const float delta = lwj - lwmax;
    if (delta > 0.0f) {
      flag_error(err, RS_ERR_BOUND_VIOLATED);
      return static_cast<int32_t>(j);
    }
    if (delta == 0.0f || u < exp_pinned(delta)) return static_cast<int32_t>(j);
  }
  flag_error(err, RS_ERR_REJECTION_CAP);
  return static_cast<int32_t>(i);
}

__device__ __forceinline__ int32_t rejection_one(const double* __restrict__ lw, int64_t n,
                                                 double lwmax, int64_t max_trials,
                                                 const Keys& keys, int64_t i, int* err) {
  const double lwi = __ldg(lw + i);
  if (nonfinite_logw(lwi)) flag_error(err, RS_ERR_NONFINITE);
  float lwmax_f;
  const bool okm = f64_to_f32_trunc(lwmax, lwmax_f);
  const long long km = f64_key(lwmax);
  const long long kNegInf = f64_key(-INFINITY);
  const uint32_t ii = static_cast<uint32_t>(i);
  int64_t j = i;
  for (int64_t s = 0; s < max_trials; ++s) {
    const uint4 x = draw(keys, ii, static_cast<uint32_t>(s));
    if (s > 0) j = uniform_index(x, n);
    const double lwj = (s == 0) ? lwi : __ldg(lw + j);
    const long long kj = f64_key(lwj);
    if (kj > km && !is_nan(lwj)) {  // above the bound (NaN never compares)
      flag_error(err, RS_ERR_BOUND_VIOLATED);
      return static_cast<int32_t>(j);
    }
    if (kj == km) return static_cast<int32_t>(j);  // ratio exactly 1
    if (kj == kNegInf || is_nan(lwj)) continue;
    float lwj_f;
    const bool okj = f64_to_f32_trunc(lwj, lwj_f);
    if (f64_accept_lt(lwj, lwj_f, okj, lwmax, lwmax_f, okm, x)) return static_cast<int32_t>(j);
  }
  flag_error(err, RS_ERR_REJECTION_CAP);
  return static_cast<int32_t>(i);
}

// ---------------------------------------------------------------------------------------
// Rejection with warp refill. Trial counts vary per particle (a geometric tail, Section 2.2),
// and a warp would wait for its slowest lane. Instead every warp owns a run of particles and
// a lane that settles its particle takes the next unstarted one of the run, so all lanes stay
// busy. Attempt s of particle i always uses counter (i, s): the result does not depend on
// the schedule and equals rejection_one.
// ---------------------------------------------------------------------------------------
constexpr int kRejRun = 32 * 8;  // particles per warp run

// The bound log w_max in the forms the attempts compare against. clamp: partial rejection
// control (Section 2.2): the attempts sample v = min(w, v_max) with v_max = the bound, so a
// weight above it is the clamped weight v_max (ratio 1, accepted, not an error).
struct RejBound {
  double lwmax;
  float lwmax_rn;  // RN(log w_max) in binary32 (the binary32 scheme's bound)
  float lwmax_f;   // truncation (the binary64 scheme's filter)
  bool okm;
  long long km;
  bool clamp;
};
__device__ __forceinline__ RejBound make_bound(double log_wmax, bool clamp = false) {
  RejBound r;
  r.clamp = clamp;
  r.lwmax = log_wmax;
  r.lwmax_rn = static_cast<float>(log_wmax);
  r.okm = f64_to_f32_trunc(log_wmax, r.lwmax_f);
  r.km = f64_key(log_wmax);
  return r;
}

// Decision of one rejection attempt with uniform u (binary32) or draw x (binary64) and
// proposal log-weight lwj: accept when u < exp(lw^j - log w_max); a log-weight above the bound
// is flagged (unless clamped) and accepted.
__device__ __forceinline__ bool rejection_accept(const RejBound& rb, float u, float lwj,
                                                 int* err) {
  const float delta = lwj - rb.lwmax_rn;
  if (delta > 0.0f) {
    if (!rb.clamp) flag_error(err, RS_ERR_BOUND_VIOLATED);
    return true;
  }
  return delta == 0.0f || u_below_exp(u, delta);
}

__device__ __forceinline__ bool rejection_accept(const RejBound& rb, uint4 x, double lwj,
                                                 int* err) {
  const long long kj = f64_key(lwj);
  if (kj > rb.km && !is_nan(lwj)) {  // above the bound (NaN never compares)
    if (!rb.clamp) flag_error(err, RS_ERR_BOUND_VIOLATED);
    return true;
  }
  if (kj == rb.km) return true;  // ratio exactly 1
  if (kj == f64_key(-INFINITY) || is_nan(lwj)) return false;
  float lwj_f;
  const bool okj = f64_to_f32_trunc(lwj, lwj_f);
  return f64_accept_lt(lwj, lwj_f, okj, rb.lwmax, rb.lwmax_f, rb.okm, x);
}

// rejection_accept for a binary64 proposal decided from its sidecar tj (f64_sidecar); the
// binary64 log-weight lw[j] is read only when the sidecar cannot decide. Same decision.
__device__ __forceinline__ bool rejection_accept_sc(const RejBound& rb, uint4 x,
                                                    const double* __restrict__ lw, int64_t j,
                                                    float tj, int* err) {
  if (!(tj == tj) || !rb.okm || tj == rb.lwmax_f) return rejection_accept(rb, x, __ldg(lw + j), err);
  if (tj > rb.lwmax_f) {  // lw_j above the bound
    if (!rb.clamp) flag_error(err, RS_ERR_BOUND_VIOLATED);
    return true;
  }
  if (tj == -INFINITY) return false;
  return f64_filter_lt(tj, rb.lwmax_f, x,
                       [&] { return exact_f64_less_exp(__ldg(lw + j), rb.lwmax, x); });
}

// Attempts a lane issues together (rejection_attempts): 2 measured 7-16 % faster than 1 at
// N = 2^20 (y = 2 and 4); 4 is faster still at y = 4 but slower at y = 2, where most particles
// settle within two attempts.
constexpr int kRejBatch = 2;

// Attempts s .. s + K - 1 of particle i (those below max_trials) with their draws and
// proposal gathers issued together -- the draws are counter-based, so they do not depend on
// the outcome of earlier attempts -- then decided in order: the first accepted one is the
// result, exactly as attempting one at a time. Returns true with j when one accepts.
template <int K, typename T>
__device__ __forceinline__ bool rejection_attempts(const T* __restrict__ lw, int64_t n,
                                                   const RejBound& rb, const Keys& keys,
                                                   int64_t i, uint32_t s, T lwi,
                                                   int64_t max_trials, int64_t& j, int* err) {
  uint4 x[K];
  int64_t jq[K];
  T lwj[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const uint32_t sq = s + static_cast<uint32_t>(q);
    x[q] = draw(keys, static_cast<uint32_t>(i), sq);
    jq[q] = (sq > 0) ? uniform_index(x[q], n) : i;
    lwj[q] = (sq > 0) ? __ldg(lw + jq[q]) : lwi;
  }
#pragma unroll
  for (int q = 0; q < K; ++q) {
    if (static_cast<int64_t>(s) + q >= max_trials) return false;
    if (rejection_accept(rb, x[q], lwj[q], err)) {
      j = jq[q];
      return true;
    }
  }
  return false;
}

// The same for binary32 log-weights, whose attempts 2m and 2m + 1 share the block of counter
// (i, m) (s even, K even): K / 2 blocks for K attempts.
template <int K>
__device__ __forceinline__ bool rejection_attempts(const float* __restrict__ lw, int64_t n,
                                                   const RejBound& rb, const Keys& keys,
                                                   int64_t i, uint32_t s, float lwi,
                                                   int64_t max_trials, int64_t& j, int* err) {
  static_assert(K % 2 == 0, "whole blocks");
  float u[K], lwj[K];
  int64_t jq[K];
#pragma unroll
  for (int p = 0; p < K / 2; ++p) {
    const uint4 x = draw(keys, static_cast<uint32_t>(i), s / 2 + static_cast<uint32_t>(p));
    const uint32_t s0 = s + 2 * static_cast<uint32_t>(p);
    jq[2 * p] = (s0 > 0) ? half_index(x.x, x.y, n) : i;
    u[2 * p] = half_u01_f32(x.x);
    jq[2 * p + 1] = half_index(x.z, x.w, n);
    u[2 * p + 1] = half_u01_f32(x.z);
    lwj[2 * p] = (s0 > 0) ? __ldg(lw + jq[2 * p]) : lwi;
    lwj[2 * p + 1] = __ldg(lw + jq[2 * p + 1]);
  }
#pragma unroll
  for (int q = 0; q < K; ++q) {
    if (static_cast<int64_t>(s) + q >= max_trials) return false;
    if (rejection_accept(rb, u[q], lwj[q], err)) {
      j = jq[q];
      return true;
    }
  }
  return false;
}

// rejection_attempts for binary64 log-weights with their sidecars lwf (ti: the sidecar of
// particle i's own log-weight): the proposals gather 4 bytes instead of 8; same outcome.
template <int K>
__device__ __forceinline__ bool rejection_attempts_sc(const double* __restrict__ lw,
                                                      const float* __restrict__ lwf, int64_t n,
                                                      const RejBound& rb, const Keys& keys,
                                                      int64_t i, uint32_t s, float ti,
                                                      int64_t max_trials, int64_t& j, int* err) {
  uint4 x[K];
  int64_t jq[K];
  float tj[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const uint32_t sq = s + static_cast<uint32_t>(q);
    x[q] = draw(keys, static_cast<uint32_t>(i), sq);
    jq[q] = (sq > 0) ? uniform_index(x[q], n) : i;
    tj[q] = (sq > 0) ? __ldg(lwf + jq[q]) : ti;
  }
#pragma unroll
  for (int q = 0; q < K; ++q) {
    if (static_cast<int64_t>(s) + q >= max_trials) return false;
    if (rejection_accept_sc(rb, x[q], lw, jq[q], tj[q], err)) {
      j = jq[q];
      return true;
    }
  }
  return false;
}

}  // namespace
}  // namespace rsk
