// dfexp.cuh -- exp of binary64 arguments evaluated in double-float (two-float) arithmetic on
// the binary32 pipes. On GB300 binary64 runs at 1/57 of the binary32 rate, so the binary64
// scan path keeps its weights and prefix sums in two-float form (about 48 significand bits).
//
// Method: x (two-float) -> y = x log2(e) (two-float product) -> y = n + j/64 + f with
// |f| <= 1/128 (the split is exact) -> 2^f = e^g, g = f ln2, by the Taylor series to g^5
// (|g| <= ln2/128, truncation below 2^-54) -> 2^(j/64) (table, hi + lo from a 300-bit
// evaluation) times (1 + (e^g - 1)) -> times 2^n. Relative error about
// 2^-47 |y| + 2^-46 (the argument's own representation error dominates for large |y|).
// Results below 2^-126 are returned as 0 (a weight that small relative to the largest
// weight is far below the precision of the sums).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "values.cuh"

namespace rsk {

// 2^(j/64) for j = 0..63 as hi + lo.
__constant__ float2 kExp2Frac64[64] = {
    {0x1.0000000000000p+0f, 0.0f},
    {0x1.02c9a40000000p+0f, -0x1.887fa00000000p-28f},
    {0x1.059b0e0000000p+0f, -0x1.9d4f520000000p-25f},
    {0x1.0874520000000p+0f, -0x1.e2990e0000000p-26f},
    {0x1.0b55860000000p+0f, 0x1.9f31220000000p-25f},
    {0x1.0e3ec40000000p+0f, -0x1.a585cc0000000p-25f},
    {0x1.11301e0000000p+0f, -0x1.fdb4960000000p-25f},
    {0x1.1429aa0000000p+0f, 0x1.d525bc0000000p-25f},
    {0x1.172b840000000p+0f, -0x1.c157420000000p-27f},
    {0x1.1a35be0000000p+0f, 0x1.6df96e0000000p-25f},
    {0x1.1d48740000000p+0f, -0x1.d2e8ca0000000p-25f},
    {0x1.2063b80000000p+0f, 0x1.0c519a0000000p-25f},
    {0x1.2387a60000000p+0f, 0x1.ceac480000000p-25f},
    {0x1.26b4560000000p+0f, 0x1.789f380000000p-26f},
    {0x1.29e9e00000000p+0f, -0x1.5c04240000000p-25f},
    {0x1.2d285a0000000p+0f, 0x1.b900c20000000p-26f},
    {0x1.306fe00000000p+0f, 0x1.4636e20000000p-25f},
    {0x1.33c08c0000000p+0f, -0x1.b37d200000000p-25f},
    {0x1.371a740000000p+0f, -0x1.18aac60000000p-25f},
    {0x1.3a7db40000000p+0f, -0x1.634c020000000p-25f},
    {0x1.3dea640000000p+0f, 0x1.8246840000000p-25f},
    {0x1.4160a20000000p+0f, 0x1.f72e2a0000000p-28f},
    {0x1.44e0860000000p+0f, 0x1.8624b40000000p-30f},
    {0x1.486a2c0000000p+0f, -0x1.47d8660000000p-25f},
    {0x1.4bfdae0000000p+0f, -0x1.593abc0000000p-25f},
    {0x1.4f9b280000000p+0f, -0x1.2c5a6c0000000p-25f},
    {0x1.5342b60000000p+0f, -0x1.2c56100000000p-25f},
    {0x1.56f4740000000p+0f, -0x1.295b040000000p-25f},
    {0x1.5ab07e0000000p+0f, -0x1.5bd5ec0000000p-27f},
    {0x1.5e76f20000000p+0f, -0x1.4a5bd60000000p-25f},
    {0x1.6247ec0000000p+0f, -0x1.f8b5500000000p-25f},
    {0x1.6623880000000p+0f, 0x1.2a91120000000p-27f},
    {0x1.6a09e60000000p+0f, 0x1.9fcef40000000p-26f},
    {0x1.6dfb240000000p+0f, -0x1.cd72e80000000p-27f},
    {0x1.71f75e0000000p+0f, 0x1.1d8bee0000000p-25f},
    {0x1.75feb60000000p+0f, -0x1.37b3060000000p-25f},
    {0x1.7a11480000000p+0f, -0x1.829fd00000000p-25f},
    {0x1.7e2f340000000p+0f, -0x1.2616340000000p-25f},
    {0x1.82589a0000000p+0f, -0x1.accc7c0000000p-26f},
    {0x1.868d9a0000000p+0f, -0x1.2edb440000000p-26f},
    {0x1.8ace540000000p+0f, 0x1.15506e0000000p-27f},
    {0x1.8f1aea0000000p+0f, -0x1.baa2320000000p-26f},
    {0x1.93737c0000000p+0f, -0x1.e647440000000p-25f},
    {0x1.97d82a0000000p+0f, -0x1.0d8d840000000p-31f},
    {0x1.9c49180000000p+0f, 0x1.51f8480000000p-27f},
    {0x1.a0c6680000000p+0f, -0x1.2886a60000000p-26f},
    {0x1.a5503c0000000p+0f, -0x1.b83b540000000p-25f},
    {0x1.a9e6b60000000p+0f, -0x1.50c0480000000p-25f},
    {0x1.ae89fa0000000p+0f, -0x1.a94b140000000p-26f},
    {0x1.b33a2c0000000p+0f, -0x1.ec3a820000000p-26f},
    {0x1.b7f7700000000p+0f, -0x1.a094380000000p-25f},
    {0x1.bcc1ea0000000p+0f, -0x1.f687c60000000p-25f},
    {0x1.c199be0000000p+0f, -0x1.3d56b20000000p-27f},
    {0x1.c67f120000000p+0f, 0x1.cafa2a0000000p-25f},
    {0x1.cb720e0000000p+0f, -0x1.8837cc0000000p-27f},
    {0x1.d072d40000000p+0f, 0x1.40f1300000000p-25f},
    {0x1.d5818e0000000p+0f, -0x1.822dbc0000000p-27f},
    {0x1.da9e600000000p+0f, 0x1.ed99420000000p-27f},
    {0x1.dfc9740000000p+0f, -0x1.908c940000000p-25f},
    {0x1.e502ee0000000p+0f, 0x1.e2cffe0000000p-26f},
    {0x1.ea4afa0000000p+0f, 0x1.52486c0000000p-27f},
    {0x1.efa1be0000000p+0f, 0x1.cc2b440000000p-25f},
    {0x1.f507660000000p+0f, -0x1.246eb00000000p-26f},
    {0x1.fa7c180000000p+0f, 0x1.9e90d80000000p-28f}
};

// Split of a binary64 into two binary32 (hi = the top 24 significand bits, truncated; lo =
// the next 29 bits rounded to 24), with integer operations only: |x - (hi + lo)| <= 2^-48 |x|.
// Infinities and NaN give hi = x (as binary32), lo = 0; |x| >= 2^128 gives +-inf.
__device__ __forceinline__ float2 split_f64(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned int sign = static_cast<unsigned int>(b >> 32) & 0x80000000u;
  const int e = static_cast<int>((b >> 52) & 0x7ffu);
  if (e == 0x7ff) {
    const bool nan = (b & 0xfffffffffffffull) != 0ull;
    return make_float2(__uint_as_float(sign | (nan ? 0x7fc00000u : 0x7f800000u)), 0.0f);
  }
  const int fe = e - 1023 + 127;
  if (fe >= 255) return make_float2(__uint_as_float(sign | 0x7f800000u), 0.0f);
  if (fe <= 0) return make_float2(__uint_as_float(sign), 0.0f);  // |x| < 2^-126
  const unsigned long long m = b & 0xfffffffffffffull;
  const float hi = __uint_as_float(sign | (static_cast<unsigned int>(fe) << 23) |
                                   static_cast<unsigned int>(m >> 29));
  const unsigned int rest = static_cast<unsigned int>(m & 0x1fffffffull);  // 29 bits
  const int se = e - 1075 + 127;  // exponent of 2^(e - 1075)
  float lo = 0.0f;
  if (se >= 1 && rest != 0u)
    lo = __fmul_rn(__uint2float_rn(rest), __uint_as_float(static_cast<unsigned int>(se) << 23));
  return make_float2(hi, sign ? -lo : lo);
}

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// Accurate two-float sum (both parts with TwoSum), valid under cancellation.
__device__ __forceinline__ float2 add22_accurate(float2 a, float2 b) {
  const float2 s = two_sum(a.x, b.x);
  const float2 t = two_sum(a.y, b.y);
  float2 r = fast_two_sum(s.x, __fadd_rn(s.y, t.x));
  return fast_two_sum(r.x, __fadd_rn(r.y, t.y));
}

// exp(x) for a two-float x <= 0 (tiny positive rounding is treated as 0); `tab` is the
// 2^(j/64) table (kExp2Frac64, usually staged in shared memory).
__device__ __forceinline__ float2 exp_df(float2 x, const float2* tab) {
  if (x.x != x.x) return x;
  if (x.x >= 0.0f) return make_float2(1.0f, 0.0f);
  const float2 y = mul22(x, make_float2(0x1.715476p+0f, 0x1.4ae0c0p-26f));  // x log2(e)
  if (y.x < -126.0f) return make_float2(0.0f, 0.0f);
  const float k = rintf(__fmul_rn(y.x, 64.0f));
  const float2 f = two_sum(__fsub_rn(y.x, __fmul_rn(k, 0x1p-6f)), y.y);  // exact split
  const float2 g = mul22(f, make_float2(0x1.62e430p-1f, -0x1.05c610p-29f));  // f ln2
  // e^g - 1 = g + g^2/2 + g^3 (1/6 + g/24 + g^2/120) as two-float
  const float p = __fmul_rn(g.x, g.x);
  const float pe = __fmaf_rn(g.x, g.x, -p);
  const float q = __fmul_rn(__fmul_rn(p, g.x),
                            __fmaf_rn(g.x, __fmaf_rn(g.x, 0x1.111112p-7f, 0x1.555556p-5f),
                                      0x1.555556p-3f));
  const float2 s = two_sum(g.x, __fmul_rn(0.5f, p));
  float lo = __fmul_rn(g.x, g.y);
  lo = __fadd_rn(lo, __fmul_rn(0.5f, pe));
  lo = __fadd_rn(lo, g.y);
  lo = __fadd_rn(lo, s.y);
  lo = __fadd_rn(lo, q);
  const float2 em1 = fast_two_sum(s.x, lo);
  const int ki = static_cast<int>(k);
  const float2 T = tab[ki & 63];
  const float2 r = vadd(T, mul22(T, em1));
  const int n = ki >> 6;  // floor(k / 64), in [-127, 0]
  if (n < -126) return make_float2(0.0f, 0.0f);
  const float sc = __int_as_float((n + 127) << 23);
  return make_float2(__fmul_rn(r.x, sc), __fmul_rn(r.y, sc));
}

// Uniform on [0,1) with the 53 random bits of u01_f64, as two floats (hi: top 24 bits,
// lo: the next 29 bits rounded to 24).
__device__ __forceinline__ float2 u01_f2(uint4 x) {
  const float hi = __fmul_rn(__uint2float_rn(x.x >> 8), 0x1p-24f);
  const unsigned int rest = ((x.x & 0xffu) << 21) | (x.y >> 11);  // 29 bits
  return make_float2(hi, __fmul_rn(__uint2float_rn(rest), 0x1p-53f));
}

}  // namespace rsk
