// values.cuh -- accumulator types of the prefix sums of the scan-based resamplers.
//
//   float  : binary32 sums (RS_F32, RS_PREC_PLAIN: the paper's single-precision setting)
//   float2 : two-float sums, hi + lo with |lo| <= ulp(hi)/2 (RS_F32, RS_PREC_COMPENSATED),
//            built from Knuth's TwoSum and Dekker's FastTwoSum / fma-based TwoProduct
//   double : binary64 sums (RS_F64)
//
// Every operation is an explicitly rounded IEEE operation (no contraction). All values
// handled here are non-negative, and all comparisons are exact.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rsk {

// ---- float ------------------------------------------------------------------------------
__device__ __forceinline__ float vzero(float) { return 0.0f; }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ bool vle(float a, float b) { return a <= b; }
__device__ __forceinline__ float vfrom_w(float w, float) { return w; }
__device__ __forceinline__ double vto_double(float a) { return static_cast<double>(a); }
__device__ __forceinline__ float vfrom_double(double x, float) { return __double2float_rn(x); }
__device__ __forceinline__ float vshfl_up(float v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ float vshfl(float v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ float vshfl_xor(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ float vhi(float a) { return a; }

// ---- double -----------------------------------------------------------------------------
__device__ __forceinline__ double vzero(double) { return 0.0; }
__device__ __forceinline__ double vadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ bool vle(double a, double b) { return a <= b; }
__device__ __forceinline__ double vfrom_w(double w, double) { return w; }
__device__ __forceinline__ double vto_double(double a) { return a; }
__device__ __forceinline__ double vfrom_double(double x, double) { return x; }
__device__ __forceinline__ double vshfl_up(double v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ double vshfl(double v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ double vshfl_xor(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ double vhi(double a) { return a; }

// ---- two-float --------------------------------------------------------------------------
__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float aa = __fsub_rn(s, bb);
  return make_float2(s, __fadd_rn(__fsub_rn(a, aa), __fsub_rn(b, bb)));
}
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 vzero(float2) { return make_float2(0.0f, 0.0f); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) {
  const float2 t = two_sum(a.x, b.x);
  return fast_two_sum(t.x, __fadd_rn(t.y, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ bool vle(float2 a, float2 b) {
  return a.x < b.x || (a.x == b.x && a.y <= b.y);
}
__device__ __forceinline__ float2 vfrom_w(float w, float2) { return make_float2(w, 0.0f); }
__device__ __forceinline__ float2 vfrom_w(float2 w, float2) { return w; }
__device__ __forceinline__ double vto_double(float2 a) {
  return __dadd_rn(static_cast<double>(a.x), static_cast<double>(a.y));
}
__device__ __forceinline__ float2 vfrom_double(double x, float2) {
  const float hi = __double2float_rn(x);
  return make_float2(hi, __double2float_rn(__dsub_rn(x, static_cast<double>(hi))));
}
__device__ __forceinline__ float2 vshfl_up(float2 v, int d) {
  return make_float2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ float2 vshfl(float2 v, int l) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, l), __shfl_sync(0xffffffffu, v.y, l));
}
__device__ __forceinline__ float2 vshfl_xor(float2 v, int m) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}
__device__ __forceinline__ float vhi(float2 a) { return a.x; }
// two-float products and sums with a float
__device__ __forceinline__ float2 mul22(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ float2 mul21(float2 a, float b) {
  const float p = __fmul_rn(a.x, b);
  float e = __fmaf_rn(a.x, b, -p);
  e = __fmaf_rn(a.y, b, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ float2 add21(float2 a, float b) {
  const float2 t = two_sum(a.x, b);
  return fast_two_sum(t.x, __fadd_rn(t.y, a.y));
}

// ---- generic ----------------------------------------------------------------------------
template <typename V> __device__ __forceinline__ V vmax(V a, V b) { return vle(a, b) ? b : a; }
template <typename V> __device__ __forceinline__ V vmin(V a, V b) { return vle(a, b) ? a : b; }
template <typename V> __device__ __forceinline__ V vclamp(V x, V lo, V hi) {
  return vmin(vmax(x, lo), hi);
}
template <typename V> __device__ __forceinline__ bool veq(V a, V b) { return vle(a, b) && vle(b, a); }

// ---- cumulative offspring from a cumulative weight W --------------------------------------
// r = W * (N / W^N); O = floor(r + u) clamped to N; W equal to the total gives O = N (all
// later weights are zero). floor of a two-float is floor(hi) unless hi is an integer.
__device__ __forceinline__ int64_t floor_to_i64(float x) { return static_cast<int64_t>(floorf(x)); }
__device__ __forceinline__ int64_t floor_to_i64(double x) { return static_cast<int64_t>(floor(x)); }
__device__ __forceinline__ int64_t floor_to_i64(float2 z) {
  const float f = floorf(z.x);
  if (f != z.x) return static_cast<int64_t>(f);
  return static_cast<int64_t>(f) + static_cast<int64_t>(floorf(z.y));
}
__device__ __forceinline__ float vscale(float W, float s) { return __fmul_rn(W, s); }
__device__ __forceinline__ double vscale(double W, double s) { return __dmul_rn(W, s); }
__device__ __forceinline__ float2 vscale(float2 W, float2 s) { return mul22(W, s); }
__device__ __forceinline__ float vplus_u(float r, float u) { return __fadd_rn(r, u); }
__device__ __forceinline__ double vplus_u(double r, double u) { return __dadd_rn(r, u); }
__device__ __forceinline__ float2 vplus_u(float2 r, float u) { return add21(r, u); }
// multinomial: u = U * W^N
__device__ __forceinline__ float vtimes_u(float S, float U) { return __fmul_rn(S, U); }
__device__ __forceinline__ double vtimes_u(double S, double U) { return __dmul_rn(S, U); }
__device__ __forceinline__ float2 vtimes_u(float2 S, float U) { return mul21(S, U); }
// double-float path: the 53-bit uniform as a two-float
__device__ __forceinline__ float2 vplus_u(float2 r, float2 u) { return vadd(r, u); }
__device__ __forceinline__ float2 vtimes_u(float2 S, float2 U) { return mul22(S, U); }

}  // namespace rsk
