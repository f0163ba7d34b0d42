// model.cu -- the pieces of the bootstrap particle filter (Code 1) around the resampler:
//  - the in-place copy that a permuted ancestry makes safe (Section 2.3): x_i <- x_{c_i};
//  - the propagate-and-weight step of the 1-D linear-Gaussian state-space model used to run
//    the full SMC loop: x_t = phi x_{t-1} + sigma_x eps, log w = -(y_t - x_t)^2 / (2 sigma_y^2).
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "measure.h"
#include "values.cuh"

namespace rsk {
namespace {

// After Permute, o_j > 0 implies c_j = j: every row that is read (a parent) is one that no
// thread writes, so the copy can run in place with one thread per particle. A c that breaks
// the predicate (c_{c_i} != c_i) is flagged and that row is left alone.
__global__ void __launch_bounds__(kBlock)
copy_ancestors_kernel(float* __restrict__ x, int D, const int32_t* __restrict__ c, int64_t N,
                      int* err) {
  pdl_wait();
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int32_t ci = c[i];
  if (ci < 0 || ci >= N || c[ci] != ci) {
    flag_error(err, RS_ERR_ARG);
    return;
  }
  if (ci == i) return;
  for (int k = 0; k < D; ++k) x[i * D + k] = x[static_cast<int64_t>(ci) * D + k];
}

// One standard normal per particle by Box-Muller from the Philox words 0 and 1 of counter
// (i, 0, step, filter * 8 + 5): u1 = 1 - U_0 in (0, 1], u2 = U_1 in [0, 1).
__device__ __forceinline__ float normal_draw(const Keys& keys, int64_t i) {
  const uint4 r = draw(keys, static_cast<uint32_t>(i), 0u);
  const float u1 = 1.0f - __fmul_rn(__uint2float_rn(r.x >> 8), 0x1p-24f);
  const float u2 = __fmul_rn(__uint2float_rn(r.y >> 8), 0x1p-24f);
  return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

__global__ void __launch_bounds__(kBlock)
lgssm_step_kernel(float* __restrict__ x, int64_t N, int init, int accumulate, float phi,
                  float sigma_x, float sigma_0, float y, float inv_2vy, Keys keys,
                  float* __restrict__ logw) {
  pdl_wait();
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float z = normal_draw(keys, i);
  const float xi = init ? sigma_0 * z : fmaf(phi, x[i], sigma_x * z);
  x[i] = xi;
  const float e = y - xi;
  const float l = -(e * e) * inv_2vy;
  logw[i] = accumulate ? logw[i] + l : l;
}

// ---------------------------------------------------------------------------------------
// Many independent filters (F filters in CSR layout, filter f owning the particles
// offsets[f] .. offsets[f+1]-1, the layout of rs_resample_batched). Filter f runs the
// single-filter kernels' arithmetic on its slice with f in the random-number counter, so a
// batched step equals the single-filter step on that slice with filter = f, bit for bit.
// ---------------------------------------------------------------------------------------

// Filter holding global position g: the last f with off[f] <= g (off has F + 1 entries).
// Returns -1 past offsets[F] or for a filter whose offsets are out of order or range.
__device__ __forceinline__ int locate(const int64_t* __restrict__ off, int F, int64_t cap,
                                      int64_t g, int64_t& lo, int64_t& n) {
  if (g >= __ldg(off + F) || g < __ldg(off)) return -1;
  int a = 0, b = F;  // invariant: off[a] <= g < off[b]
  while (b - a > 1) {
    const int mid = (a + b) >> 1;
    if (__ldg(off + mid) <= g) a = mid; else b = mid;
  }
  lo = __ldg(off + a);
  const int64_t hi = __ldg(off + a + 1);
  n = hi - lo;
  if (lo < 0 || hi > cap || n <= 0 || n > 0x7fffffffLL) return -1;
  return a;
}

__global__ void __launch_bounds__(kBlock)
copy_ancestors_batched_kernel(float* __restrict__ x, int D, const int32_t* __restrict__ c,
                              const int64_t* __restrict__ off, int F, int64_t cap, int* err) {
  pdl_wait();
  const int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  int64_t lo, n;
  if (g >= cap || locate(off, F, cap, g, lo, n) < 0) return;
  const int32_t ci = c[g];
  if (ci < 0 || ci >= n || c[lo + ci] != ci) {
    flag_error(err, RS_ERR_ARG);
    return;
  }
  const int64_t src = lo + ci;
  if (src == g) return;
  for (int k = 0; k < D; ++k) x[g * D + k] = x[src * D + k];
}

__global__ void __launch_bounds__(kBlock)
lgssm_step_batched_kernel(float* __restrict__ x, const int64_t* __restrict__ off, int F,
                          int64_t cap, int init, int accumulate, float phi, float sigma_x,
                          float sigma_0, const float* __restrict__ y, float inv_2vy, Keys keys,
                          float* __restrict__ logw) {
  pdl_wait();
  const int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  int64_t lo, n;
  const int f = g < cap ? locate(off, F, cap, g, lo, n) : -1;
  if (f < 0) return;
  keys.tag = (static_cast<uint32_t>(f) << 3) | 5u;
  const float z = normal_draw(keys, g - lo);
  const float xi = init ? sigma_0 * z : fmaf(phi, x[g], sigma_x * z);
  x[g] = xi;
  const float e = __ldg(y + f) - xi;
  const float l = -(e * e) * inv_2vy;
  logw[g] = accumulate ? logw[g] + l : l;
}

// Per-thread sums of the max-shifted weights w and of w^2: two-float for binary32
// log-weights (no binary64 arithmetic per particle), binary64 for binary64 ones.
__device__ __forceinline__ void lse_acc(float2& acc, float2& acc2, float x, float m) {
  const float e = expf(x - m);
  acc = add21(acc, e);
  acc2 = add21(acc2, e * e);
}
__device__ __forceinline__ void lse_acc(double& acc, double& acc2, double x, double m) {
  const double e = exp(x - m);
  acc += e;
  acc2 += e * e;
}
__device__ __forceinline__ void lse_acc(float2& acc, float x, float m) {
  acc = add21(acc, expf(x - m));
}
__device__ __forceinline__ void lse_acc(double& acc, double x, double m) { acc += exp(x - m); }
__device__ __forceinline__ double lse_to_double(float2 a) { return vto_double(a); }
__device__ __forceinline__ double lse_to_double(double a) { return a; }

// B* of Eq. B for beta = mean w / max w (Section 2.1): ceil(log eps / log(1 - beta)), at
// least 1; 1 for beta >= 1 (every proposal is accepted) or beta <= 0 (no weight: Metropolis
// accepts any proposal from a zero-weight state); clamped to 2^31 - 1.
__device__ __forceinline__ int32_t metropolis_B_of(double beta, double log_eps) {
  if (!(beta > 0.0) || beta >= 1.0) return 1;
  const double b = ceil(log_eps / log1p(-beta));
  if (!(b <= 2147483647.0)) return 2147483647;
  return b < 1.0 ? 1 : static_cast<int32_t>(b);
}

// Per filter f (one CTA each): the maximum m of its n log-weights, then with w = exp(lw - m)
// (so max w = 1): log_total[f] = m + log sum w (Appendix E's max-shift), ess[f] = (sum w)^2 /
// sum w^2 (the effective sample size of Section 4.3), beta[f] = sum w / n = mean w / max w
// (Eq. beta2 evaluated on the filter's own weights) and B[f] = Eq. B for it; null outputs
// are skipped. The exponentials in the log-weights' type, the per-thread sums in two-float
// (binary32) or binary64, the CTA's sums in binary64. A filter that is empty or whose weights
// are all zero gets -inf, 0, 0 and B = 1; NaN / +inf log-weights are flagged. SQ: the sum of
// squares is formed (only the ESS needs it; the sum of w is the same either way).
template <typename T, bool SQ>
__global__ void __launch_bounds__(kBlock)
log_sum_batched_kernel(const T* __restrict__ lw, const int64_t* __restrict__ off, int F,
                       int64_t cap, WeightStatsOut o, int* err) {
  pdl_wait();
  const int f = blockIdx.x;
  const int64_t lo = __ldg(off + f), hi = __ldg(off + f + 1);
  if (lo < 0 || hi > cap || hi < lo) {
    if (threadIdx.x == 0) flag_error(err, RS_ERR_ARG);
    return;
  }
  __shared__ double sh[kBlock / 32], sh2[kBlock / 32];
  T m = neg_inf<T>();
  bool bad = false;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const T v = __ldg(lw + i);
    bad |= nonfinite_logw(v);
    m = v > m ? v : m;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) flag_error(err, RS_ERR_NONFINITE);
  double md = static_cast<double>(m);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) md = fmax(md, __shfl_xor_sync(0xffffffffu, md, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = md;
  __syncthreads();
  md = sh[0];
  for (int k = 1; k < kBlock / 32; ++k) md = fmax(md, sh[k]);
  __syncthreads();
  if (md == -INFINITY) {
    if (threadIdx.x == 0) {
      if (o.log_total) o.log_total[f] = -INFINITY;
      if (o.ess) o.ess[f] = 0.0;
      if (o.beta) o.beta[f] = 0.0;
      if (o.B) o.B[f] = 1;
      if (o.below) o.below[f] = 0;
    }
    return;
  }
  const T mt = static_cast<T>(md);
  using Acc = typename std::conditional<sizeof(T) == 4, float2, double>::type;
  Acc acc{}, acc2{};
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    if constexpr (SQ)
      lse_acc(acc, acc2, __ldg(lw + i), mt);
    else
      lse_acc(acc, __ldg(lw + i), mt);
  }
  double sum = lse_to_double(acc), sum2 = lse_to_double(acc2);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if constexpr (SQ) sum2 += __shfl_xor_sync(0xffffffffu, sum2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[threadIdx.x >> 5] = sum;
    sh2[threadIdx.x >> 5] = sum2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0, t2 = 0.0;
    for (int k = 0; k < kBlock / 32; ++k) {
      t += sh[k];
      t2 += sh2[k];
    }
    if (o.log_total) o.log_total[f] = md + log(t);
    const double ess = t2 > 0.0 ? (t * t) / t2 : 0.0;
    if (o.ess) o.ess[f] = ess;
    if (o.below) o.below[f] = ess < o.below_frac * static_cast<double>(hi - lo) ? 1 : 0;
    const double beta = t / static_cast<double>(hi - lo);
    if (o.beta) o.beta[f] = beta;
    if (o.B) o.B[f] = metropolis_B_of(beta, o.log_eps);
  }
}

// The log-weights of the flagged filters of a batch set to 0 (equal weights after their
// resampling); the other filters keep theirs.
__global__ void __launch_bounds__(kBlock)
reset_logw_batched_kernel(float* __restrict__ logw, const int64_t* __restrict__ off, int F,
                          int64_t cap, const uint8_t* __restrict__ flags) {
  pdl_wait();
  const int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  int64_t lo, n;
  const int f = g < cap ? locate(off, F, cap, g, lo, n) : -1;
  if (f < 0) return;
  if (__ldg(flags + f) != 0) logw[g] = 0.0f;
}

// Philox throughput: thread i draws the blocks (i, n), n < J, under the given keys and XORs
// all their words; the warps' XORs are folded into *out (zeroed before the launch).
__global__ void __launch_bounds__(kBlock)
philox_xor_kernel(Keys keys, int64_t T, uint32_t J, uint32_t* out) {
  pdl_wait();
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  if (i < T) {
    for (uint32_t n = 0; n < J; ++n) {
      const uint4 x = draw(keys, static_cast<uint32_t>(i), n);
      acc ^= x.x ^ x.y ^ x.z ^ x.w;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc ^= __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0u) atomicXor(out, acc);
}

// ---------------------------------------------------------------------------------------
// Resampling on demand inside a CUDA graph: the decision, and the bookkeeping of the
// adaptive filter's likelihood, on the device.
// ---------------------------------------------------------------------------------------
__global__ void set_if_below_kernel(cudaGraphConditionalHandle hnd, const double* v, double thr) {
  cudaGraphSetConditional(hnd, *v < thr ? 1u : 0u);
}

__global__ void noop_kernel() {}

// After a resampling: equal weights (log w = 0), likelihood base log N, one more resampling.
__global__ void __launch_bounds__(kBlock)
mark_resampled_kernel(float* __restrict__ logw, int64_t N, double* base, double log_n,
                      int32_t* count) {
  pdl_wait();
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < N) logw[i] = 0.0f;
  if (i == 0) {
    *base = log_n;
    if (count) *count += 1;
  }
}

// The adaptive filter's likelihood: ll += (log W_t - base) - c, base = log W_t (first step:
// ll = (log W_0 - log N) - c and the resampling count reset).
__global__ void loglik_step_kernel(const double* lse, double* base, double* ll, int32_t* count,
                                   double c, double log_n, int first) {
  pdl_wait();
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  const double l = *lse;
  if (first) {
    *ll = (l - log_n) - c;
    if (count) *count = 0;
  } else {
    *ll = *ll + ((l - *base) - c);
  }
  *base = l;
}

inline int grid_for(int64_t N) { return static_cast<int>((N + kBlock - 1) / kBlock); }

}  // namespace

cudaError_t launch_set_if_below(cudaGraphConditionalHandle hnd, const double* v, double thr,
                                cudaStream_t st) {
  set_if_below_kernel<<<1, 1, 0, st>>>(hnd, v, thr);
  return cudaGetLastError();
}

cudaError_t launch_noop(cudaStream_t st) {
  noop_kernel<<<1, 1, 0, st>>>();
  return cudaGetLastError();
}

cudaError_t launch_mark_resampled(const Scratch& s, float* logw, int64_t N, double* base,
                                  double log_n, int32_t* count, cudaStream_t st) {
  trace_mark(s.trace, "mark_resampled", st);
  launch_pdl(mark_resampled_kernel, grid_for(N), kBlock, st, logw, N, base, log_n, count);
  return cudaGetLastError();
}

cudaError_t launch_loglik_step(const Scratch& s, const double* lse, double* base, double* ll,
                               int32_t* count, double c, double log_n, int first,
                               cudaStream_t st) {
  trace_mark(s.trace, "loglik_step", st);
  launch_pdl(loglik_step_kernel, 1, 32, st, lse, base, ll, count, c, log_n, first);
  return cudaGetLastError();
}

cudaError_t launch_copy_ancestors(const Scratch& s, float* x, int D, const int32_t* c, int64_t N,
                                  cudaStream_t st) {
  trace_mark(s.trace, "copy_ancestors", st);
  launch_pdl(copy_ancestors_kernel, grid_for(N), kBlock, st, x, D, c, N, s.err);
  return cudaGetLastError();
}

cudaError_t launch_lgssm_step(const Scratch& s, float* x, int64_t N, int init, int accumulate,
                              float phi, float sigma_x, float y, float sigma_y, uint64_t seed,
                              uint64_t step, uint32_t filter, float* logw, cudaStream_t st) {
  const double s0 = static_cast<double>(sigma_x) / std::sqrt(1.0 - static_cast<double>(phi) * phi);
  const float inv_2vy = static_cast<float>(0.5 / (static_cast<double>(sigma_y) * sigma_y));
  trace_mark(s.trace, "lgssm_step", st);
  launch_pdl(lgssm_step_kernel, grid_for(N), kBlock, st, x, N, init, accumulate, phi, sigma_x,
                                                   static_cast<float>(s0), y, inv_2vy,
                                                   make_keys(seed, step, filter, 5u), logw);
  return cudaGetLastError();
}

// Grids of the batched kernels cover the handle's capacity: offsets[F] is on the device.
cudaError_t launch_copy_ancestors_batched(const Scratch& s, float* x, int D, const int32_t* c,
                                          const int64_t* offsets, int F, cudaStream_t st) {
  trace_mark(s.trace, "copy_ancestors_batched", st);
  launch_pdl(copy_ancestors_batched_kernel, grid_for(s.max_n), kBlock, st, x, D, c, offsets, F,
             s.max_n, s.err);
  return cudaGetLastError();
}

cudaError_t launch_lgssm_step_batched(const Scratch& s, float* x, const int64_t* offsets, int F,
                                      int init, int accumulate, float phi, float sigma_x,
                                      const float* y, float sigma_y, uint64_t seed,
                                      uint64_t step, float* logw, cudaStream_t st) {
  const double s0 = static_cast<double>(sigma_x) / std::sqrt(1.0 - static_cast<double>(phi) * phi);
  const float inv_2vy = static_cast<float>(0.5 / (static_cast<double>(sigma_y) * sigma_y));
  trace_mark(s.trace, "lgssm_step_batched", st);
  launch_pdl(lgssm_step_batched_kernel, grid_for(s.max_n), kBlock, st, x, offsets, F, s.max_n,
             init, accumulate, phi, sigma_x, static_cast<float>(s0), y, inv_2vy,
             make_keys(seed, step, 0u, 5u), logw);
  return cudaGetLastError();
}

cudaError_t launch_weight_stats_batched(const Scratch& s, bool f64, const void* logw,
                                        const int64_t* offsets, int F, const WeightStatsOut& o,
                                        cudaStream_t st) {
  trace_mark(s.trace, o.B ? "metropolis_B_batched"
                          : (o.ess || o.below) ? "ess_batched" : "log_sum_batched", st);
  const auto* l32 = static_cast<const float*>(logw);
  const auto* l64 = static_cast<const double*>(logw);
  const bool sq = o.ess != nullptr || o.below != nullptr;
  if (f64 && sq)
    launch_pdl(log_sum_batched_kernel<double, true>, F, kBlock, st, l64, offsets, F, s.max_n, o,
               s.err);
  else if (f64)
    launch_pdl(log_sum_batched_kernel<double, false>, F, kBlock, st, l64, offsets, F, s.max_n, o,
               s.err);
  else if (sq)
    launch_pdl(log_sum_batched_kernel<float, true>, F, kBlock, st, l32, offsets, F, s.max_n, o,
               s.err);
  else
    launch_pdl(log_sum_batched_kernel<float, false>, F, kBlock, st, l32, offsets, F, s.max_n, o,
               s.err);
  return cudaGetLastError();
}

cudaError_t launch_reset_logw_batched(const Scratch& s, float* logw, const int64_t* offsets,
                                      int F, const uint8_t* flags, cudaStream_t st) {
  trace_mark(s.trace, "reset_logw_batched", st);
  launch_pdl(reset_logw_batched_kernel, grid_for(s.max_n), kBlock, st, logw, offsets, F,
             s.max_n, flags);
  return cudaGetLastError();
}

cudaError_t launch_philox_throughput(int64_t threads, uint32_t draws_per_thread, uint64_t seed,
                                     uint32_t* xor_out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(xor_out, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  const Keys keys = make_keys(seed, 0, 0u, 6u);
  launch_pdl(philox_xor_kernel, static_cast<int>((threads + kBlock - 1) / kBlock), kBlock, st,
             keys, threads, draws_per_thread, xor_out);
  return cudaGetLastError();
}

}  // namespace rsk
