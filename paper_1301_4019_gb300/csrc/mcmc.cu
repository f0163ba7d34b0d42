// mcmc.cu -- the collective-free resamplers of Section 2 on sm_103a: Metropolis (Section
// 2.1, Code 2) and rejection (Section 2.2, Code 3), one thread per particle, each with the
// Prepermute claim of Code 10 fused at the end (Appendix E: the claim is appended to every
// procedure that produces an ancestry vector).
//
// Every draw is counter-based (Philox keyed by particle and inner step), so the random
// numbers of step s do not depend on the chain state: the proposals and their log-weight
// gathers of several steps are issued together and only the accept decisions run in
// sequence (mcmc.cuh).
#include <cfloat>

#include "common.cuh"
#include "grid.cuh"
#include "internal.h"
#include "mcmc.cuh"

namespace rsk {
namespace {

// CTAs per SM the register allocation must allow: 6 for the binary32 chains (38 registers,
// measured 3 % faster than 56); the binary64 chains keep their 62 registers (fewer measured
// slower: their four proposals in flight need them).
template <typename T> constexpr int metropolis_min_ctas() { return sizeof(T) == 4 ? 6 : 1; }

// One thread per particle. COOP: a persistent cooperative grid that first sets the claims to
// the sentinel N (the Prepermute initialisation), meets at a grid barrier, then runs the
// chains over a grid-stride loop -- one launch instead of a fill and the chains.
// Binary64 log-weights come with their sidecars lwf (f64_sidecar; sidecar_kernel), which the
// chains gather instead of the binary64 values.
template <typename T, bool COOP>
__global__ void __launch_bounds__(kBlock, metropolis_min_ctas<T>())
metropolis_kernel(const T* __restrict__ lw, const float* __restrict__ lwf, int64_t N, int32_t B,
                  Keys keys, int32_t* __restrict__ a, int32_t* __restrict__ d, GridBar* bar,
                  int* err) {
  pdl_wait();
  const int64_t t0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t stride = COOP ? static_cast<int64_t>(gridDim.x) * blockDim.x : N;
  unsigned int target = 0;
  if constexpr (COOP) {
    if (d)
      for (int64_t i = t0; i < N; i += stride) d[i] = static_cast<int32_t>(N);
    grid_barrier(bar, target, err);
  }
  for (int64_t i = t0; i < N; i += stride) {
    int32_t k;
    if constexpr (sizeof(T) == 8) k = metropolis_one_sc(lw, lwf, N, B, keys, i, err);
    else k = metropolis_one(lw, N, B, keys, i, err);
    a[i] = k;
    if (d) atomicMin(d + k, static_cast<int32_t>(i));
  }
  if constexpr (COOP) grid_exit(bar, target);
}

// Rejection with warp refill (mcmc.cuh) over the particles [start, end) of one warp run.
template <typename T>
__device__ __forceinline__ void rejection_run(const T* __restrict__ lw,
                                              const float* __restrict__ lwf, int64_t N,
                                              int64_t start, int64_t end, const RejBound& rb,
                                              int64_t max_trials, const Keys& keys,
                                              int32_t* __restrict__ a, int32_t* __restrict__ d,
                                              int* err) {
  const int lane = threadIdx.x & 31;
  int64_t i = start + lane;
  bool active = i < end;
  int64_t head = start + 32;
  uint64_t s = 0;  // attempts made (max_trials < 2^32, but s + kRejBatch may pass 2^32)
  T lwi = active ? __ldg(lw + i) : T(0);
  if (active && nonfinite_logw(lwi)) flag_error(err, RS_ERR_NONFINITE);
  for (;;) {
    bool settled = false;
    if (active) {
      int64_t j;
      if constexpr (sizeof(T) == 8)
        settled = rejection_attempts_sc<kRejBatch>(lw, lwf, N, rb, keys, i,
                                                   static_cast<uint32_t>(s), f64_sidecar(lwi),
                                                   max_trials, j, err);
      else
        settled = rejection_attempts<kRejBatch>(lw, N, rb, keys, i, static_cast<uint32_t>(s),
                                                lwi, max_trials, j, err);
      s += kRejBatch;
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

// Warp w takes the runs w, w + W, ... of run_len particles (W = warps of the grid). The host
// sizes run_len so that every warp gets exactly one run (a warp that took an extra run
// would set the kernel's length).
// Binary64 log-weights come with their sidecars lwf, written by the cooperative grid before
// its barrier, else beforehand by sidecar_kernel.
template <typename T, bool COOP>
__global__ void __launch_bounds__(kBlock)
rejection_kernel(const T* __restrict__ lw, float* __restrict__ lwf, int64_t N, double log_wmax,
                 const double* lwmax_dev, bool clamp, int64_t max_trials, Keys keys,
                 int32_t* __restrict__ a, int32_t* __restrict__ d, int64_t run_len,
                 GridBar* bar, int* err) {
  pdl_wait();
  unsigned int target = 0;
  if constexpr (COOP) {
    if (d || sizeof(T) == 8) {
      const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
      for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < N;
           i += stride) {
        if (d) d[i] = static_cast<int32_t>(N);
        if constexpr (sizeof(T) == 8) lwf[i] = f64_sidecar(__ldg(lw + i));
      }
    }
    grid_barrier(bar, target, err);
  }
  // the bound: the argument, or (lwmax_dev) one estimated on the device; an estimate of -inf
  // (no finite log-weight drawn) leaves every particle its own ancestor, flagged
  const double lwm = lwmax_dev ? __ldcg(lwmax_dev) : log_wmax;
  if (!(lwm > -DBL_MAX)) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < N;
         i += stride) {
      a[i] = static_cast<int32_t>(i);
      if (d) atomicMin(d + i, static_cast<int32_t>(i));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) flag_error(err, RS_ERR_ZERO_WEIGHT);
    if constexpr (COOP) grid_exit(bar, target);
    return;
  }
  const RejBound rb = make_bound(lwm, clamp);
  const int64_t warps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t run = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
       run * run_len < N; run += warps) {  // uniform across the warp
    const int64_t start = run * run_len;
    const int64_t end = start + run_len < N ? start + run_len : N;
    rejection_run(lw, lwf, N, start, end, rb, max_trials, keys, a, d, err);
  }
  if constexpr (COOP) grid_exit(bar, target);
}

// Log-weights of the outcome of partial rejection control for the delivered ancestry c:
// out_i = lw[c_i] - min(lw[c_i], log v_max), in the log-weights' type (0 unless the ancestor's
// weight exceeds v_max; 0 for a zero weight, which only the trial cap can deliver).
// With lvmax_dev the bound is read on the device (rounded to T as the attempts round it), a
// bound of -inf gives 0 everywhere (the identity ancestry), and *viol (set to 0 before) counts
// the particles whose own log-weight exceeds the bound.
template <typename T>
__global__ void __launch_bounds__(kBlock)
prc_weights_kernel(const T* __restrict__ lw, const int32_t* __restrict__ c, int64_t N, T lvmax,
                   const double* lvmax_dev, T* __restrict__ out,
                   unsigned long long* viol, int* err) {
  pdl_wait();
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const T bound = lvmax_dev ? static_cast<T>(__ldcg(lvmax_dev)) : lvmax;
  bool above = false;
  if (i < N) {
    const int32_t ci = c[i];
    if (ci < 0 || ci >= N) {
      flag_error(err, RS_ERR_ARG);
    } else {
      const T w = __ldg(lw + ci);
      out[i] = (w > bound && bound > neg_inf<T>()) ? w - bound : T(0);
    }
    above = viol && __ldg(lw + i) > bound;
  }
  if (viol) {
    const unsigned mask = __ballot_sync(0xffffffffu, above);
    if ((threadIdx.x & 31) == 0 && mask) atomicAdd(viol, static_cast<unsigned long long>(__popc(mask)));
  }
}

// The estimated bound of the rejection resampler (Section 2.2, a substitute for w_max): the
// largest of `sample` log-weights at indices drawn uniformly, the k-th from counter (k, 0)
// under the keys' purpose; NaN is passed over, -inf when nothing finite was drawn. One CTA of
// kEstBlock threads; also sets *viol to 0 for the weights kernel.
constexpr int kEstBlock = 1024;
template <typename T>
__global__ void __launch_bounds__(kEstBlock)
estimate_bound_kernel(const T* __restrict__ lw, int64_t N, int64_t sample, Keys keys,
                      double* est, unsigned long long* viol) {
  pdl_wait();
  __shared__ double sh[kEstBlock / 32];
  double m = -INFINITY;
  for (int64_t k = threadIdx.x; k < sample; k += kEstBlock) {
    const uint4 x = draw(keys, static_cast<uint32_t>(k), 0u);
    const double v = static_cast<double>(__ldg(lw + uniform_index(x, N)));
    if (v > m) m = v;  // (NaN never compares)
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double y = __shfl_xor_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = sh[0];
    for (int w = 1; w < kEstBlock / 32; ++w) b = sh[w] > b ? sh[w] : b;
    *est = b;
    if (viol) *viol = 0ull;
  }
}

// Sidecars of binary64 log-weights (f64_sidecar) and, when d is given, the claims d = N (the
// Prepermute initialisation): one pass that replaces the fill of the claims.
__global__ void __launch_bounds__(kBlock)
sidecar_kernel(const double* __restrict__ lw, int64_t N, float* __restrict__ lwf,
               int32_t* __restrict__ d) {
  pdl_wait();
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x * 4;
  const bool vec = ((reinterpret_cast<uintptr_t>(lw) | reinterpret_cast<uintptr_t>(lwf) |
                     reinterpret_cast<uintptr_t>(d)) & 15u) == 0;
  for (int64_t i = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) * 4; i < N;
       i += stride) {
    if (vec && i + 4 <= N) {  // 128-bit loads and stores
      const double2 u = __ldg(reinterpret_cast<const double2*>(lw + i));
      const double2 v = __ldg(reinterpret_cast<const double2*>(lw + i + 2));
      *reinterpret_cast<float4*>(lwf + i) =
          make_float4(f64_sidecar(u.x), f64_sidecar(u.y), f64_sidecar(v.x), f64_sidecar(v.y));
      if (d) {
        const int32_t n = static_cast<int32_t>(N);
        *reinterpret_cast<int4*>(d + i) = make_int4(n, n, n, n);
      }
    } else {
      for (int64_t k = i; k < i + 4 && k < N; ++k) {
        lwf[k] = f64_sidecar(__ldg(lw + k));
        if (d) d[k] = static_cast<int32_t>(N);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Self-checks of the acceptance tests (rs_check_acceptance): they run the device functions
// the resamplers run and count the cases where a shortcut would decide differently from the
// definition u < exp_pinned(delta).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void count_add(unsigned long long* out, unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, v);
}

// Every binary32 delta with bit pattern first + k (k < count): the binary32 test decides
// from the band [RD(e (1 - 2^-15)), RU(e (1 + 2^-15))] around e = exp_band_estimate(delta),
// which is right exactly when exp_pinned(delta) lies inside it.
__global__ void __launch_bounds__(kBlock)
check_band_f32_kernel(uint32_t first, uint32_t count, unsigned long long* out) {
  unsigned long long bad = 0;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += stride) {
    const float delta = __uint_as_float(first + k);
    const float e = exp_band_estimate(delta);
    const float lo = __fmul_rd(e, 1.0f - kExpBand), hi = __fmul_ru(e, 1.0f + kExpBand);
    const float p = exp_pinned(delta);
    if (!(lo <= p && p <= hi)) ++bad;
  }
  count_add(out, bad);
}

// The 53-bit uniform u = m 2^-53 as the Philox words it is drawn from (u01_f64).
__device__ __forceinline__ uint4 words_of_u(uint64_t m) {
  return make_uint4(static_cast<uint32_t>(m >> 21), static_cast<uint32_t>((m & 0x1fffffu) << 11),
                    0u, 0u);
}

// Binary64 decisions on the binary32 pipes (f64_accept_lt) against the binary64 definition
// u < exp_pinned(lwj - lwk), on n log-weight pairs: lwk from four magnitudes (0, -2.75,
// -1234.5678, 30000.5: the last two push the filter to its exact fallback), lwj = lwk + d with
// d spread over [-90, 0) (plus hashed low bits, so that many bit patterns occur), and per pair
// uniforms on the 53-bit grid at and next to p = exp_pinned(lwj - lwk), next to p (1 +- 2^-20),
// p (1 +- 2^-15) and p (1 +- 2^-10), and two hashed ones.
__global__ void __launch_bounds__(kBlock)
check_f64_decisions_kernel(int64_t n, unsigned long long* out) {
  unsigned long long bad = 0;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const double base[4] = {0.0, -2.75, -1234.5678, 30000.5};
  for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < n;
       k += stride) {
    const uint64_t h = (static_cast<uint64_t>(k) + 1) * 0x9E3779B97F4A7C15ull;
    const double lwk = base[k & 3];
    const double frac = (static_cast<double>(k >> 2) + 0.5) / static_cast<double>(n / 4 + 1);
    const double d = -90.0 * frac * (1.0 + static_cast<double>(h >> 40) * 0x1p-50);
    const double lwj = __dadd_rn(lwk, d);
    if (!(lwj < lwk)) continue;
    const double p = exp_pinned(__dsub_rn(lwj, lwk));
    float lwj_f, lwk_f;
    const bool okj = f64_to_f32_trunc(lwj, lwj_f), okk = f64_to_f32_trunc(lwk, lwk_f);
    const double mid = p * 0x1p53;
    const double targets[9] = {mid, mid * (1.0 - 0x1p-20), mid * (1.0 + 0x1p-20),
                               mid * (1.0 - 0x1p-15), mid * (1.0 + 0x1p-15),
                               mid * (1.0 - 0x1p-10), mid * (1.0 + 0x1p-10),
                               static_cast<double>(h >> 11),
                               static_cast<double>((h * 0xBF58476D1CE4E5B9ull) >> 11)};
#pragma unroll 1
    for (int t = 0; t < 9; ++t) {
      const double tm = targets[t];
      if (!(tm < 0x1p53)) continue;
      const uint64_t m0 = static_cast<uint64_t>(tm);
#pragma unroll 1
      for (int dm = -1; dm <= 1; ++dm) {
        if (dm < 0 && m0 == 0) continue;
        const uint64_t m = m0 + dm;
        if (m >= (1ull << 53)) continue;
        const uint4 x = words_of_u(m);
        const bool got = f64_accept_lt(lwj, lwj_f, okj, lwk, lwk_f, okk, x);
        const bool want = u01_f64(x) < p;
        if (got != want) ++bad;
      }
    }
  }
  count_add(out, bad);
}

}  // namespace

// Grid of the sidecar pass: up to 16 CTAs per SM over a grid-stride loop, four particles per
// thread.
inline int side_grid(int64_t N) {
  const int64_t want = (N + 4 * kBlock - 1) / (4 * kBlock);
  const int64_t cap = static_cast<int64_t>(device_sm_count()) * 16;
  return static_cast<int>(want < cap ? want : cap);
}

// d, when given, is first set to the sentinel N (the Prepermute initialisation): inside the
// cooperative rejection kernel when the device allows it, else by a fill launch.
template <typename T>
cudaError_t launch_metropolis_t(const Scratch& s, const T* lw, int64_t N, int32_t B,
                                const Keys& keys, int32_t* a_out, int32_t* d, bool f64,
                                cudaStream_t st) {
  // (The cooperative form, fill and chains in one launch, measured slower than a fill launch
  // followed by one thread per particle: the chains hide their gathers better in waves.)
  GridBar* bar = &s.glob->bar;
  float* lwf = static_cast<float*>(s.W);  // the sidecars of binary64 log-weights (4 B each)
  if (sizeof(T) == 8) {
    trace_mark(s.trace, "sidecar", st);
    launch_pdl(sidecar_kernel, side_grid(N), kBlock, st, reinterpret_cast<const double*>(lw), N,
               lwf, d);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  } else if (d) {
    trace_mark(s.trace, "fill", st);
    const cudaError_t e = launch_fill(d, N, static_cast<int32_t>(N), st);
    if (e != cudaSuccess) return e;
  }
  trace_mark(s.trace, f64 ? "metropolis_f64" : "metropolis_f32", st);
  launch_pdl(metropolis_kernel<T, false>, static_cast<int>((N + kBlock - 1) / kBlock), kBlock,
             st, lw, lwf, N, B, keys, a_out, d, bar, s.err);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rejection_t(const Scratch& s, const T* lw, int64_t N, double log_wmax,
                               const double* lwmax_dev, bool clamp, int64_t max_trials,
                               const Keys& keys, int32_t* a_out, int32_t* d, bool f64,
                               cudaStream_t st) {
  GridBar* bar = &s.glob->bar;
  float* lwf = static_cast<float*>(s.W);  // the sidecars of binary64 log-weights (4 B each)
  const int64_t runs = (N + kRejRun - 1) / kRejRun;
  const int64_t want = (runs * 32 + kBlock - 1) / kBlock;
  if (s.coop && s.launch_mode != RS_LAUNCH_SEPARATE) {
    const int cap = coop_capacity(reinterpret_cast<const void*>(rejection_kernel<T, true>));
    if (cap > 0) {
      // runs of at least kRejRun particles, one per warp of a grid of at most `cap` CTAs
      // (with more runs than warps some warps take two and the kernel waits for them:
      // measured 7-35 % slower at 2^22)
      const int grid = static_cast<int>(want < cap ? want : cap);
      const int64_t warps = static_cast<int64_t>(grid) * (kBlock / 32);
      int64_t run_len = (N + warps - 1) / warps;
      run_len = run_len > kRejRun ? run_len : kRejRun;
      trace_mark(s.trace, f64 ? "rejection_f64" : "rejection_f32", st);
      return coop_launch(rejection_kernel<T, true>, grid, st, lw, lwf, N, log_wmax, lwmax_dev,
                         clamp, max_trials, keys, a_out, d, run_len, bar, s.err);
    }
  }
  if (sizeof(T) == 8) {
    trace_mark(s.trace, "sidecar", st);
    launch_pdl(sidecar_kernel, side_grid(N), kBlock, st, reinterpret_cast<const double*>(lw), N,
               lwf, d);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  } else if (d) {
    trace_mark(s.trace, "fill", st);
    const cudaError_t e = launch_fill(d, N, static_cast<int32_t>(N), st);
    if (e != cudaSuccess) return e;
  }
  trace_mark(s.trace, f64 ? "rejection_f64" : "rejection_f32", st);
  launch_pdl(rejection_kernel<T, false>, static_cast<int>(want), kBlock, st, lw, lwf, N,
             log_wmax, lwmax_dev, clamp, max_trials, keys, a_out, d,
             static_cast<int64_t>(kRejRun), bar, s.err);
  return cudaGetLastError();
}

cudaError_t launch_metropolis(const Scratch& s, bool f64, const void* logw, int64_t N,
                              int32_t B, uint64_t seed, uint64_t step, uint32_t filter,
                              int32_t* a_out, int32_t* d, cudaStream_t st) {
  const Keys keys = make_keys(seed, step, filter, RS_METROPOLIS);
  if (f64)
    return launch_metropolis_t(s, static_cast<const double*>(logw), N, B, keys, a_out, d, true,
                               st);
  return launch_metropolis_t(s, static_cast<const float*>(logw), N, B, keys, a_out, d, false,
                             st);
}

cudaError_t launch_rejection(const Scratch& s, bool f64, const void* logw, int64_t N,
                             double log_wmax, bool clamp, int64_t max_trials, uint64_t seed,
                             uint64_t step, uint32_t filter, int32_t* a_out, int32_t* d,
                             cudaStream_t st, const double* lwmax_dev) {
  const Keys keys = make_keys(seed, step, filter, RS_REJECTION);
  if (f64)
    return launch_rejection_t(s, static_cast<const double*>(logw), N, log_wmax, lwmax_dev, clamp,
                              max_trials, keys, a_out, d, true, st);
  return launch_rejection_t(s, static_cast<const float*>(logw), N, log_wmax, lwmax_dev, clamp,
                            max_trials, keys, a_out, d, false, st);
}

cudaError_t launch_estimate_bound(const Scratch& s, bool f64, const void* logw, int64_t N,
                                  int64_t sample, uint64_t seed, uint64_t step, uint32_t filter,
                                  double* est, unsigned long long* viol, cudaStream_t st) {
  const Keys keys = make_keys(seed, step, filter, kPurposeBoundEstimate);
  trace_mark(s.trace, "estimate_bound", st);
  if (f64)
    launch_pdl(estimate_bound_kernel<double>, 1, kEstBlock, st, static_cast<const double*>(logw),
               N, sample, keys, est, viol);
  else
    launch_pdl(estimate_bound_kernel<float>, 1, kEstBlock, st, static_cast<const float*>(logw),
               N, sample, keys, est, viol);
  return cudaGetLastError();
}

cudaError_t launch_prc_weights(const Scratch& s, bool f64, const void* logw, const int32_t* c,
                               int64_t N, double log_vmax, void* out, cudaStream_t st,
                               const double* lvmax_dev, unsigned long long* viol) {
  trace_mark(s.trace, "prc_weights", st);
  const int grid = static_cast<int>((N + kBlock - 1) / kBlock);
  if (f64)
    launch_pdl(prc_weights_kernel<double>, grid, kBlock, st, static_cast<const double*>(logw),
               c, N, log_vmax, lvmax_dev, static_cast<double*>(out), viol, s.err);
  else  // the bound in binary32 as the binary32 attempts use it: RN(log v_max)
    launch_pdl(prc_weights_kernel<float>, grid, kBlock, st, static_cast<const float*>(logw), c,
               N, static_cast<float>(log_vmax), lvmax_dev, static_cast<float*>(out), viol,
               s.err);
  return cudaGetLastError();
}

cudaError_t launch_check_acceptance(int mode, int64_t n, unsigned long long* count,
                                    cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    sms = 1;
  const int grid = sms * 8;
  if (mode == 0) {  // every binary32 delta in [-86.5, 0): patterns 0x80000001 .. 0xc2ad0000
    const uint32_t first = 0x80000001u, last = 0xc2ad0000u;
    check_band_f32_kernel<<<grid, kBlock, 0, st>>>(first, last - first + 1, count);
  } else {
    check_f64_decisions_kernel<<<grid, kBlock, 0, st>>>(n, count);
  }
  return cudaGetLastError();
}

}  // namespace rsk
