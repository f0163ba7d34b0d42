// ess.cu -- effective sample size of a weight vector, ESS = (sum w)^2 / sum w^2 with the
// weights w_i = exp(lw_i - max lw) of Appendix E, the quantity that decides when an adaptive
// particle filter resamples (Section 4.3 discusses resampling every step against on demand).
// One cooperative launch: maximum -> grid barrier -> per-CTA sums of w and w^2 -> grid
// barrier -> CTA 0 adds the per-CTA totals exactly (128-bit fixed point, all its threads) and
// divides; the same sums give the log of the weight total, M + log sum w.
#include <cfloat>

#include "common.cuh"
#include "dfexp.cuh"
#include "grid.cuh"
#include "internal.h"
#include "tile.cuh"
#include "values.cuh"

namespace rsk {
namespace {

__device__ __forceinline__ long long ess_key(float v) {
  const int b = __float_as_int(v);
  return static_cast<long long>(b >= 0 ? b : (b ^ 0x7fffffff));
}
__device__ __forceinline__ long long ess_key(double v) {
  const long long b = __double_as_longlong(v);
  return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double ess_value(long long k, double) {
  return __longlong_as_double(k >= 0 ? k : (k ^ 0x7fffffffffffffffLL));
}
__device__ __forceinline__ double ess_value(long long k, float) {
  const int b = static_cast<int>(k);
  return static_cast<double>(__int_as_float(b >= 0 ? b : (b ^ 0x7fffffff)));
}

// Binary32 weight of one log-weight given the maximum (the ESS needs no more precision).
__device__ __forceinline__ float ess_weight(float x, float Mf, float2) {
  return is_neg_inf(x) ? 0.0f : exp_pinned(__fsub_rn(x, Mf));
}
__device__ __forceinline__ float ess_weight(double x, float, float2 M2) {
  return is_neg_inf(x) ? 0.0f : exp_pinned(add22_accurate(split_f64(x), neg2(M2)).x);
}

template <typename T>
__global__ void __launch_bounds__(kBlock)
ess_kernel(const T* __restrict__ lw, int64_t N, double* blockmax, u128* agg, GridBar* bar,
           double* ess_out, double* log_total_out, int* err) {
  __shared__ long long sh_key[kWarps];
  __shared__ float2 sh_s[kWarps][2];
  __shared__ u128 sh_u[kWarps];
  unsigned int target = 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t t0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  // maximum (NaN skipped and flagged, as +inf)
  // keys of the log-weights' own type (no per-particle conversion to binary64)
  long long m = ess_key(neg_inf<T>());
  bool bad = false;
  for (int64_t i = t0; i < N; i += stride) {
    const T x = lw[i];
    bad |= nonfinite_logw(x);
    if (!is_nan(x)) {
      const long long k = ess_key(x);
      m = k > m ? k : m;
    }
  }
  if (bad) flag_error(err, RS_ERR_NONFINITE);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long y = __shfl_xor_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
  }
  if (lane == 0) sh_key[warp] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long bm = sh_key[0];
    for (int k = 1; k < kWarps; ++k) bm = sh_key[k] > bm ? sh_key[k] : bm;
    blockmax[blockIdx.x] = ess_value(bm, T());
  }
  grid_barrier(bar, target, err);
  long long mk = ess_key(-static_cast<double>(INFINITY));  // binary64 keys of the CTA maxima
  for (int b = threadIdx.x; b < static_cast<int>(gridDim.x); b += kBlock) {
    const long long y = ess_key(__ldcg(blockmax + b));
    mk = y > mk ? y : mk;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long y = __shfl_xor_sync(0xffffffffu, mk, o);
    mk = y > mk ? y : mk;
  }
  __syncthreads();
  if (lane == 0) sh_key[warp] = mk;
  __syncthreads();
  long long bm = sh_key[0];
  for (int k = 1; k < kWarps; ++k) bm = sh_key[k] > bm ? sh_key[k] : bm;
  const double M = ess_value(bm, 0.0);
  const bool zero = !(M > -DBL_MAX);
  // two-float sums of w and w^2 per thread, then per CTA
  float2 s1 = make_float2(0.0f, 0.0f), s2 = make_float2(0.0f, 0.0f);
  if (!zero) {
    const float Mf = static_cast<float>(M);
    const float2 M2 = split_f64(M);
    for (int64_t i = t0; i < N; i += stride) {
      const float w = ess_weight(lw[i], Mf, M2);
      s1 = add21(s1, w);
      s2 = add21(s2, __fmul_rn(w, w));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 = vadd(s1, vshfl_xor(s1, o));
    s2 = vadd(s2, vshfl_xor(s2, o));
  }
  if (lane == 0) {
    sh_s[warp][0] = s1;
    sh_s[warp][1] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    u128 a1 = 0, a2 = 0;
    for (int k = 0; k < kWarps; ++k) {
      a1 += to_fixed(sh_s[k][0]);
      a2 += to_fixed(sh_s[k][1]);
    }
    agg[2 * blockIdx.x] = a1;
    agg[2 * blockIdx.x + 1] = a2;
  }
  grid_barrier(bar, target, err);
  if (blockIdx.x == 0) {  // the per-CTA totals, added by the whole CTA (exact, any order)
    u128 a1 = 0, a2 = 0;
    for (int b = threadIdx.x; b < static_cast<int>(gridDim.x); b += kBlock) {
      a1 += ld_u128_cg(agg + 2 * b);
      a2 += ld_u128_cg(agg + 2 * b + 1);
    }
    a1 = block_sum_u128(a1, sh_u);
    a2 = block_sum_u128(a2, sh_u);
    if (threadIdx.x == 0) {
      const double S1 = fixed_to_double(a1, kFixFrac), S2 = fixed_to_double(a2, kFixFrac);
      if (zero || !(S2 > 0.0)) {
        flag_error(err, RS_ERR_ZERO_WEIGHT);
        if (ess_out) *ess_out = 0.0;
        if (log_total_out) *log_total_out = -static_cast<double>(INFINITY);
      } else {
        if (ess_out) *ess_out = __ddiv_rn(__dmul_rn(S1, S1), S2);
        if (log_total_out) *log_total_out = M + log(S1);
      }
    }
  }
  grid_exit(bar, target);
}

}  // namespace

cudaError_t launch_ess(const Scratch& s, bool f64, const void* logw, int64_t N, double* ess,
                       double* log_total, cudaStream_t st) {
  const void* k = f64 ? reinterpret_cast<const void*>(ess_kernel<double>)
                      : reinterpret_cast<const void*>(ess_kernel<float>);
  int cap = coop_capacity(k);
  if (!s.coop || cap < 1) return cudaErrorNotSupported;
  if (cap > s.max_blocks) cap = s.max_blocks;  // blockmax holds max_blocks entries
  if (cap > s.max_tiles + 2) cap = static_cast<int>(s.max_tiles + 2);  // agg below
  const int64_t want = (N + kBlock - 1) / kBlock;
  const int grid = static_cast<int>(want < cap ? want : cap);
  u128* agg = reinterpret_cast<u128*>(s.rec);  // 2 * grid <= 2 * (max_tiles + 2) entries
  trace_mark(s.trace, f64 ? "ess_f64" : "ess_f32", st);
  if (f64)
    return coop_launch(ess_kernel<double>, grid, st, static_cast<const double*>(logw), N,
                       s.blockmax, agg, &s.glob->bar, ess, log_total, s.err);
  return coop_launch(ess_kernel<float>, grid, st, static_cast<const float*>(logw), N,
                     s.blockmax, agg, &s.glob->bar, ess, log_total, s.err);
}

}  // namespace rsk
