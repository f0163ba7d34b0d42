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
template <typename T, bool COOP>
__global__ void __launch_bounds__(kBlock, metropolis_min_ctas<T>())
metropolis_kernel(const T* __restrict__ lw, int64_t N, int32_t B, Keys keys,
                  int32_t* __restrict__ a, int32_t* __restrict__ d, unsigned int* bar, int* err) {
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
    const int32_t k = metropolis_one(lw, N, B, keys, i, err);
    a[i] = k;
    if (d) atomicMin(d + k, static_cast<int32_t>(i));
  }
  if constexpr (COOP) grid_exit(bar, target);
}

// Rejection with warp refill (mcmc.cuh) over the particles [start, end) of one warp run.
template <typename T>
__device__ __forceinline__ void rejection_run(const T* __restrict__ lw, int64_t N, int64_t start,
                                              int64_t end, const RejBound& rb,
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
template <typename T, bool COOP>
__global__ void __launch_bounds__(kBlock)
rejection_kernel(const T* __restrict__ lw, int64_t N, double log_wmax, bool clamp,
                 int64_t max_trials, Keys keys, int32_t* __restrict__ a,
                 int32_t* __restrict__ d, int64_t run_len, unsigned int* bar, int* err) {
  pdl_wait();
  unsigned int target = 0;
  if constexpr (COOP) {
    if (d) {
      const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
      for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < N;
           i += stride)
        d[i] = static_cast<int32_t>(N);
    }
    grid_barrier(bar, target, err);
  }
  const RejBound rb = make_bound(log_wmax, clamp);
  const int64_t warps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t run = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
       run * run_len < N; run += warps) {  // uniform across the warp
    const int64_t start = run * run_len;
    const int64_t end = start + run_len < N ? start + run_len : N;
    rejection_run(lw, N, start, end, rb, max_trials, keys, a, d, err);
  }
  if constexpr (COOP) grid_exit(bar, target);
}

// Log-weights of the outcome of partial rejection control for the delivered ancestry c:
// out_i = lw[c_i] - min(lw[c_i], log v_max), in the log-weights' type (0 unless the ancestor's
// weight exceeds v_max; 0 for a zero weight, which only the trial cap can deliver).
template <typename T>
__global__ void __launch_bounds__(kBlock)
prc_weights_kernel(const T* __restrict__ lw, const int32_t* __restrict__ c, int64_t N, T lvmax,
                   T* __restrict__ out, int* err) {
  pdl_wait();
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int32_t ci = c[i];
  if (ci < 0 || ci >= N) {
    flag_error(err, RS_ERR_ARG);
    return;
  }
  const T w = __ldg(lw + ci);
  out[i] = w > lvmax ? w - lvmax : T(0);
}

}  // namespace

// d, when given, is first set to the sentinel N (the Prepermute initialisation): inside the
// cooperative rejection kernel when the device allows it, else by a fill launch.
template <typename T>
cudaError_t launch_metropolis_t(const Scratch& s, const T* lw, int64_t N, int32_t B,
                                const Keys& keys, int32_t* a_out, int32_t* d, bool f64,
                                cudaStream_t st) {
  // (The cooperative form, fill and chains in one launch, measured slower than a fill launch
  // followed by one thread per particle: the chains hide their gathers better in waves.)
  unsigned int* bar = &s.glob->bar_count;
  if (d) {
    trace_mark(s.trace, "fill", st);
    const cudaError_t e = launch_fill(d, N, static_cast<int32_t>(N), st);
    if (e != cudaSuccess) return e;
  }
  trace_mark(s.trace, f64 ? "metropolis_f64" : "metropolis_f32", st);
  launch_pdl(metropolis_kernel<T, false>, static_cast<int>((N + kBlock - 1) / kBlock), kBlock,
             st, lw, N, B, keys, a_out, d, bar, s.err);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rejection_t(const Scratch& s, const T* lw, int64_t N, double log_wmax,
                               bool clamp, int64_t max_trials, const Keys& keys, int32_t* a_out,
                               int32_t* d, bool f64, cudaStream_t st) {
  unsigned int* bar = &s.glob->bar_count;
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
      return coop_launch(rejection_kernel<T, true>, grid, st, lw, N, log_wmax, clamp,
                         max_trials, keys, a_out, d, run_len, bar, s.err);
    }
  }
  if (d) {
    trace_mark(s.trace, "fill", st);
    const cudaError_t e = launch_fill(d, N, static_cast<int32_t>(N), st);
    if (e != cudaSuccess) return e;
  }
  trace_mark(s.trace, f64 ? "rejection_f64" : "rejection_f32", st);
  launch_pdl(rejection_kernel<T, false>, static_cast<int>(want), kBlock, st, lw, N, log_wmax,
             clamp, max_trials, keys, a_out, d, static_cast<int64_t>(kRejRun), bar, s.err);
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
                             cudaStream_t st) {
  const Keys keys = make_keys(seed, step, filter, RS_REJECTION);
  if (f64)
    return launch_rejection_t(s, static_cast<const double*>(logw), N, log_wmax, clamp,
                              max_trials, keys, a_out, d, true, st);
  return launch_rejection_t(s, static_cast<const float*>(logw), N, log_wmax, clamp, max_trials,
                            keys, a_out, d, false, st);
}

cudaError_t launch_prc_weights(const Scratch& s, bool f64, const void* logw, const int32_t* c,
                               int64_t N, double log_vmax, void* out, cudaStream_t st) {
  trace_mark(s.trace, "prc_weights", st);
  const int grid = static_cast<int>((N + kBlock - 1) / kBlock);
  if (f64)
    launch_pdl(prc_weights_kernel<double>, grid, kBlock, st, static_cast<const double*>(logw),
               c, N, log_vmax, static_cast<double*>(out), s.err);
  else  // the bound in binary32 as the binary32 attempts use it: RN(log v_max)
    launch_pdl(prc_weights_kernel<float>, grid, kBlock, st, static_cast<const float*>(logw), c,
               N, static_cast<float>(log_vmax), static_cast<float*>(out), s.err);
  return cudaGetLastError();
}

}  // namespace rsk
