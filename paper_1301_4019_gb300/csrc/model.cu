// model.cu -- the pieces of the bootstrap particle filter (Code 1) around the resampler:
//  - the in-place copy that a permuted ancestry makes safe (Section 2.3): x_i <- x_{c_i};
//  - the propagate-and-weight step of the 1-D linear-Gaussian state-space model used to run
//    the full SMC loop: x_t = phi x_{t-1} + sigma_x eps, log w = -(y_t - x_t)^2 / (2 sigma_y^2).
#include <cmath>

#include "common.cuh"
#include "internal.h"

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

inline int grid_for(int64_t N) { return static_cast<int>((N + kBlock - 1) / kBlock); }

}  // namespace

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

}  // namespace rsk
