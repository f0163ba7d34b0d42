// tile.cuh -- the tile scan shared by the single-filter and batched scan-based resamplers:
// weights per (input type, accumulator type), the kTile-particle tile prefix sum made
// monotone (tile_cum_weights), the exact tile prefixes, and the cumulative offspring of Codes
// 7 and 8 with the Code-11 scatter.
#pragma once

#include <cfloat>
#include <climits>
#include <cstdint>
#include <type_traits>

#include "common.cuh"
#include "dfexp.cuh"
#include "values.cuh"

namespace rsk {
namespace {

// ---------------------------------------------------------------------------------------
// Weights and uniforms per (input type, accumulator type)
// ---------------------------------------------------------------------------------------
struct WeightCtx {
  double Md;          // maximum log-weight
  float Mf;           // as binary32 (binary32 inputs: exact)
  float2 M2;          // as two-float (double-float path)
  const float2* tab;  // 2^(j/64) table in shared memory (double-float path)
};

// kTileRef: the segment records are formed relative to the segment's own maximum
// (seg_record), in the same pass as the maximum of the whole sequence. Not for the compensated
// binary32 sums: they must add exactly the binary32 weights exp(lw - M) that the emission
// scans, and weights rounded to binary32 relative to another reference are other numbers;
// their records are formed relative to M, after the maximum pass.
//
// Weights: the plain binary32 sums use exp_scan_f32 (relative error below kScanExpRelErr,
// a bound the parity tolerance of these sums includes); every other path uses the pinned
// exponential, so its weights are the oracle's bit for bit.
template <typename T, typename V> struct Path;
template <> struct Path<float, float> {
  using U = float;
  static constexpr int id = 0;
  static constexpr bool kTable = false;
  static constexpr bool kTileRef = true;
  // exp_scan_f32(-inf) = 0, so a zero weight needs no test (M is finite here)
  __device__ static float weight(float x, const WeightCtx& c) {
    return exp_scan_f32(__fsub_rn(x, c.Mf));
  }
  __device__ static U draw_u(uint4 x) { return u01_f32(x); }
};
template <> struct Path<float, float2> {
  using U = float;
  static constexpr int id = 1;
  static constexpr bool kTable = false;
  static constexpr bool kTileRef = false;
  __device__ static float2 weight(float x, const WeightCtx& c) {
    return make_float2(exp_pinned(__fsub_rn(x, c.Mf)), 0.0f);
  }
  __device__ static U draw_u(uint4 x) { return u01_f32(x); }
};
template <> struct Path<double, float2> {
  using U = float2;
  static constexpr int id = 2;
  static constexpr bool kTable = true;
  static constexpr bool kTileRef = true;
  __device__ static float2 weight(double x, const WeightCtx& c) {
    if (is_neg_inf(x)) return make_float2(0.0f, 0.0f);
    return exp_df(add22_accurate(split_f64(x), neg2(c.M2)), c.tab);
  }
  __device__ static U draw_u(uint4 x) { return u01_f2(x); }
};
template <> struct Path<double, double> {
  using U = double;
  static constexpr int id = 3;
  static constexpr bool kTable = false;
  static constexpr bool kTileRef = true;
  __device__ static double weight(double x, const WeightCtx& c) {
    return (x == neg_inf<double>()) ? 0.0 : exp_pinned(__dsub_rn(x, c.Md));
  }
  __device__ static U draw_u(uint4 x) { return u01_f64(x); }
};

// Order-preserving integer keys of the log-weights (exact comparisons on the integer pipe, no
// binary64 arithmetic); binary32 keys are 32-bit patterns widened, binary64 keys 64-bit.
__device__ __forceinline__ long long max_key(float v) {
  const int b = __float_as_int(v);
  return static_cast<long long>(b >= 0 ? b : (b ^ 0x7fffffff));
}
__device__ __forceinline__ long long max_key(double v) {
  const long long b = __double_as_longlong(v);
  return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}
__device__ __forceinline__ float key_to_float(long long k) {
  const int b = static_cast<int>(k);
  return __int_as_float(b >= 0 ? b : (b ^ 0x7fffffff));
}
__device__ __forceinline__ double key_to_double(long long k, float) {
  return static_cast<double>(key_to_float(k));
}
__device__ __forceinline__ double key_to_double(long long k, double) {
  return __longlong_as_double(k >= 0 ? k : (k ^ 0x7fffffffffffffffLL));
}
template <typename T> __device__ __forceinline__ T key_to(long long k);
template <> __device__ __forceinline__ float key_to<float>(long long k) { return key_to_float(k); }
template <> __device__ __forceinline__ double key_to<double>(long long k) {
  return key_to_double(k, 0.0);
}

// The weight context of a reference log-weight given by its key (the fields its path reads,
// from the bit pattern: no binary64 arithmetic).
template <typename T, typename V>
__device__ __forceinline__ WeightCtx ctx_of_key(long long k, const float2* tab) {
  WeightCtx c;
  c.tab = tab;
  if constexpr (sizeof(T) == 4) {
    c.Mf = key_to_float(k);
    c.Md = 0.0;  // (unused by the binary32 paths)
    c.M2 = make_float2(c.Mf, 0.0f);
  } else {
    c.Md = key_to_double(k, 0.0);
    c.M2 = split_f64(c.Md);
    c.Mf = c.M2.x;
  }
  return c;
}

// The weight context for the maximum Md with the exp table already staged at tab.
template <typename T, typename V>
__device__ __forceinline__ WeightCtx ctx_staged(double Md, const float2* tab) {
  WeightCtx c;
  c.Md = Md;
  c.Mf = static_cast<float>(Md);
  c.M2 = split_f64(Md);
  c.tab = tab;
  return c;
}

// Builds the weight context (and stages the exp table in shared memory when needed).
template <typename T, typename V>
__device__ __forceinline__ WeightCtx make_ctx(double Md, float2* sh_tab) {
  WeightCtx c;
  c.Md = Md;
  c.Mf = static_cast<float>(Md);
  c.M2 = split_f64(Md);
  c.tab = sh_tab;
  if constexpr (Path<T, V>::kTable) {
    if (threadIdx.x < 64) sh_tab[threadIdx.x] = kExp2Frac64[threadIdx.x];
    __syncthreads();
  }
  return c;
}

// Reads the 4 consecutive log-weights idx..idx+3; positions outside [lo, N) read as -inf.
// `vec` says the base pointer is 16-byte aligned; the 128-bit path is taken when all four
// positions are inside and the first is 16-byte aligned, else four guarded scalar loads.
template <typename T>
__device__ __forceinline__ void load4(const T* __restrict__ lw, int64_t idx, int64_t lo,
                                      int64_t N, bool vec, T (&x)[4]) {
  constexpr int64_t kAlign = sizeof(T) == 4 ? 3 : 1;  // 16-byte alignment of the first load
  if (vec && idx >= lo && idx + 4 <= N && (idx & kAlign) == 0) {
    if constexpr (sizeof(T) == 4) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(lw + idx));
      x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    } else {
      const double2 v0 = __ldg(reinterpret_cast<const double2*>(lw + idx));
      const double2 v1 = __ldg(reinterpret_cast<const double2*>(lw + idx + 2));
      x[0] = v0.x; x[1] = v0.y; x[2] = v1.x; x[3] = v1.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      x[q] = (idx + q >= lo && idx + q < N) ? lw[idx + q] : neg_inf<T>();
  }
}

// The kPer consecutive log-weights idx .. idx + kPer - 1: 128-bit loads when all are inside
// [lo, N) and the first is 16-byte aligned (one test for the eight), else guarded loads.
template <typename T>
__device__ __forceinline__ void load_per(const T* __restrict__ lw, int64_t idx, int64_t lo,
                                         int64_t N, bool vec, T (&x)[kPer],
                                         L2Hint hint = L2Hint::kNormal) {
  static_assert(kPer == 8, "eight consecutive values");
  constexpr int64_t kAlign = sizeof(T) == 4 ? 3 : 1;
  if (vec && idx >= lo && idx + kPer <= N && (idx & kAlign) == 0) {
    const uint64_t pol = l2_policy(hint);
    if constexpr (sizeof(T) == 4) {
      const float4 v0 = ld_stream(reinterpret_cast<const float4*>(lw + idx), hint, pol);
      const float4 v1 = ld_stream(reinterpret_cast<const float4*>(lw + idx + 4), hint, pol);
      x[0] = v0.x; x[1] = v0.y; x[2] = v0.z; x[3] = v0.w;
      x[4] = v1.x; x[5] = v1.y; x[6] = v1.z; x[7] = v1.w;
    } else {
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const double2 v = ld_stream(reinterpret_cast<const double2*>(lw + idx + 2 * h), hint, pol);
        x[2 * h] = v.x;
        x[2 * h + 1] = v.y;
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < kPer; ++q)
      x[q] = (idx + q >= lo && idx + q < N) ? lw[idx + q] : neg_inf<T>();
  }
}

template <typename V> __device__ __forceinline__ V load_v(const double2* p) {
  return *reinterpret_cast<const V*>(p);
}
template <typename V> __device__ __forceinline__ void store_v(double2* p, V v) {
  *reinterpret_cast<V*>(p) = v;
}
template <typename V> __device__ __forceinline__ V load_v_cg(const double2* p);
template <> __device__ __forceinline__ float load_v_cg<float>(const double2* p) {
  return __ldcg(reinterpret_cast<const float*>(p));
}
template <> __device__ __forceinline__ double load_v_cg<double>(const double2* p) {
  return __ldcg(reinterpret_cast<const double*>(p));
}
template <> __device__ __forceinline__ float2 load_v_cg<float2>(const double2* p) {
  return __ldcg(reinterpret_cast<const float2*>(p));
}

// Particles of a tile: thread t holds the kPer consecutive offsets kPer t .. kPer t + kPer - 1,
// so warp w holds 32 kPer consecutive particles and the tile kTile = kBlock kPer.
// Valid elements of the tile starting at `base` of a sequence ending at N (tiles start at or
// after the sequence start): offsets 0 .. count-1.
__device__ __forceinline__ int tile_count(int64_t base, int64_t N) {
  const int64_t c = N - base;
  return c < kTile ? static_cast<int>(c) : kTile;
}
// The same for a segment: the kSeg = 32 kPer particles of one warp (lane l holds kPer l ..
// kPer l + kPer - 1); zero or negative past the end.
constexpr int kSeg = 32 * kPer;
__device__ __forceinline__ int seg_count(int64_t base, int64_t N) {
  const int64_t c = N - base;
  return c < kSeg ? static_cast<int>(c) : kSeg;
}

// Maximum and minimum of non-negative accumulator values (exact; one instruction for the
// IEEE types, whose values here are never NaN).
__device__ __forceinline__ float tmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float tmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ double tmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float2 tmax(float2 a, float2 b) { return vmax(a, b); }
__device__ __forceinline__ float2 tmin(float2 a, float2 b) { return vmin(a, b); }

// Equality of two accumulator values (non-negative, never NaN here).
__device__ __forceinline__ bool vsame(float a, float b) { return a == b; }
__device__ __forceinline__ bool vsame(double a, double b) { return a == b; }
__device__ __forceinline__ bool vsame(float2 a, float2 b) { return a.x == b.x && a.y == b.y; }

// floor(x) as a 32-bit integer (x >= 0; values of 2^31 and above saturate, and every caller
// clamps to n < 2^31 afterwards). floor of a two-float is floor(hi) unless hi is an integer.
__device__ __forceinline__ int32_t floor_i32(float x) { return __float2int_rd(x); }
__device__ __forceinline__ int32_t floor_i32(double x) { return __double2int_rd(x); }
__device__ __forceinline__ int32_t floor_i32(float2 z) {
  const float f = floorf(z.x);
  if (!(f < 0x1p31f)) return INT32_MAX;
  const int32_t i = __float2int_rz(f);
  return f != z.x ? i : i + __float2int_rd(z.y);  // hi an integer below 2^31: |lo| < 64
}

// Uniforms of the strata (Code 7: one uniform u_k per stratum k). One Philox4x32-10 block
// serves consecutive strata: four at 24 bits (stratum k takes the top 24 bits of word k mod 4
// of counter floor(k / 4)) and two at 53 bits (words 2 (k mod 2) and 2 (k mod 2) + 1 of
// counter floor(k / 2), as u01_f64 takes words 0 and 1).
template <typename U> struct StratumU;
template <> struct StratumU<float> {
  static constexpr int kShift = 2;  // log2 of the strata per block
  __device__ static float from(uint2 w) { return u01_f32(make_uint4(w.x, 0u, 0u, 0u)); }
};
template <> struct StratumU<float2> {
  static constexpr int kShift = 1;
  __device__ static float2 from(uint2 w) { return u01_f2(make_uint4(w.x, w.y, 0u, 0u)); }
};
template <> struct StratumU<double> {
  static constexpr int kShift = 1;
  __device__ static double from(uint2 w) { return u01_f64(make_uint4(w.x, w.y, 0u, 0u)); }
};
// the word(s) of stratum k in its block x
template <typename U>
__device__ __forceinline__ uint2 stratum_words(uint4 x, int32_t k) {
  if constexpr (StratumU<U>::kShift == 2) {
    const int j = k & 3;
    return make_uint2(j == 0 ? x.x : j == 1 ? x.y : j == 2 ? x.z : x.w, 0u);
  } else {
    return (k & 1) ? make_uint2(x.z, x.w) : make_uint2(x.x, x.y);
  }
}
template <typename U>
__device__ __forceinline__ U stratum_u(const Keys& keys, int32_t k) {
  const uint4 x = draw(keys, static_cast<uint32_t>(k) >> StratumU<U>::kShift, 0u);
  return StratumU<U>::from(stratum_words<U>(x, k));
}

// Cumulative offspring of a cumulative weight W (Codes 7 and 8): r = W * c with c = N / W^N
// rounded once (the order the oracle pins), O = floor(r + u) (systematic) or, for the stratum
// k = min(n - 1, floor(r)) with its own uniform, min(k + 1, floor(r + u_k)) (stratified);
// W equal to the total gives O = n (all later weights are zero). r and u are non-negative.
template <typename T, typename V>
__device__ __forceinline__ int32_t stratum_of(V r, int32_t n) {
  const int32_t k = floor_i32(r);
  return k < n - 1 ? k : n - 1;
}
template <typename T, typename V>
__device__ __forceinline__ int32_t strat_count(V r, int32_t k, typename Path<T, V>::U uk,
                                               int32_t n) {
  int32_t o = floor_i32(vplus_u(r, uk));
  o = o < k + 1 ? o : k + 1;
  return o < n ? o : n;
}
template <typename T, typename V, bool STRAT>
__device__ __forceinline__ int32_t cum_offspring(V W, V S, V scale,
                                                 typename Path<T, V>::U u_sys,
                                                 const Keys& keys, int32_t n) {
  if (vsame(W, S)) return n;
  const V r = vscale(W, scale);
  if constexpr (STRAT) {
    const int32_t k = stratum_of<T, V>(r, n);
    return strat_count<T, V>(r, k, stratum_u<typename Path<T, V>::U>(keys, k), n);
  } else {
    const int32_t o = floor_i32(vplus_u(r, u_sys));
    return o < n ? o : n;
  }
}

// Stratified cumulative offspring of a warp's kPer particles per lane (W) and, in lane 0 when
// `has_b`, of the particle before them (Wb -> Ob), with the Philox blocks shared: the strata
// of the warp are non-decreasing in particle order, so each block the warp needs is listed
// once (where it differs from the previous particle's), drawn by one lane (the list dealt
// over the lanes) into the warp's shared table, and read back by every particle of it:
// about span / 4 + 1 blocks for a warp whose strata span `span` (binary32), instead of one
// per particle. A warp needing more than kStratCap blocks draws per particle. The uniforms,
// and so the counts, are those of cum_offspring.
constexpr int kStratCap = 160;

template <typename T, typename V>
__device__ __forceinline__ void strat_offspring_warp(const V (&W)[kPer], V Wb, V S, V scale,
                                                     const Keys& keys, int32_t n, bool has_b,
                                                     int32_t (&O)[kPer], int32_t& Ob) {
  using U = typename Path<T, V>::U;
  constexpr int sh = StratumU<U>::kShift;
  __shared__ uint4 tab[kWarps][kStratCap];
  const int lane = threadIdx.x & 31;
  uint4* const tw = tab[threadIdx.x >> 5];
  V r[kPer];
  int32_t k[kPer];
  uint32_t all = 0;  // W = W^N: O = n, no uniform
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    all |= static_cast<uint32_t>(vsame(W[q], S)) << q;
    r[q] = vscale(W[q], scale);
    k[q] = stratum_of<T, V>(r[q], n);
  }
  const V rb = vscale(Wb, scale);
  const int32_t kb = stratum_of<T, V>(rb, n);
  const bool first_b = lane == 0 && has_b;
  int32_t cprev = __shfl_up_sync(0xffffffffu, k[kPer - 1] >> sh, 1);
  if (lane == 0) cprev = has_b ? (kb >> sh) : -1;
  uint32_t nm = 0;  // particles whose block differs from the one before
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int32_t c = k[q] >> sh;
    nm |= static_cast<uint32_t>(c != cprev) << q;
    cprev = c;
  }
  const int mine = __popc(nm) + (first_b ? 1 : 0);
  int incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  const int ex = incl - mine;  // this lane's first entry
  if (total <= kStratCap) {  // (warp-uniform)
    int pos = ex;
    if (first_b) tw[pos++].x = static_cast<uint32_t>(kb >> sh);
#pragma unroll
    for (int q = 0; q < kPer; ++q)
      if ((nm >> q) & 1u) tw[pos++].x = static_cast<uint32_t>(k[q] >> sh);
    __syncwarp();
    for (int j = lane; j < total; j += 32) tw[j] = draw(keys, tw[j].x, 0u);
    __syncwarp();
    auto u_at = [&](int t, int32_t kk) -> U {
      if constexpr (sh == 2) {
        return StratumU<U>::from(make_uint2(reinterpret_cast<const uint32_t*>(tw + t)[kk & 3], 0u));
      } else {
        return StratumU<U>::from(reinterpret_cast<const uint2*>(tw + t)[kk & 1]);
      }
    };
    if (first_b) Ob = vsame(Wb, S) ? n : strat_count<T, V>(rb, kb, u_at(0, kb), n);
    int t = ex + (first_b ? 1 : 0) - 1;  // the entry before this lane's first particle
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      t += static_cast<int>((nm >> q) & 1u);
      O[q] = ((all >> q) & 1u) ? n : strat_count<T, V>(r[q], k[q], u_at(t, k[q]), n);
    }
    __syncwarp();  // (the table is rewritten by the warp's next segment)
  } else {
    if (first_b) Ob = vsame(Wb, S) ? n : strat_count<T, V>(rb, kb, stratum_u<U>(keys, kb), n);
#pragma unroll
    for (int q = 0; q < kPer; ++q)
      O[q] = ((all >> q) & 1u) ? n : strat_count<T, V>(r[q], k[q], stratum_u<U>(keys, k[q]), n);
  }
}

// ---------------------------------------------------------------------------------------
// Exact tile prefixes. Tile totals are non-negative and below 2^31 (each weight is at most
// 1), so they are summed exactly in 128-bit fixed point with 96 fractional bits (only parts
// below 2^-96 are dropped: at most T * 2^-96 in all, against a total of at least 1) and each
// prefix is rounded once, to nearest, to the accumulator type. Integer arithmetic only: the
// binary64 pipe of GB300 runs at 1/57 of the binary32 rate.
// ---------------------------------------------------------------------------------------
using u128 = unsigned __int128;
constexpr int kFixFrac = 96;

// m * 2^E (m < 2^53) as fixed point, truncated; negative when neg (two's complement).
__device__ __forceinline__ u128 fixed_from_parts(uint64_t m, int E, bool neg) {
  const int sh = E + kFixFrac;
  u128 F = 0;
  if (sh >= 0) F = static_cast<u128>(m) << sh;
  else if (sh > -64) F = static_cast<u128>(m >> (-sh));
  return neg ? static_cast<u128>(0) - F : F;
}
__device__ __forceinline__ u128 to_fixed(float v) {
  const uint32_t b = __float_as_uint(v);
  const int e = static_cast<int>((b >> 23) & 0xffu);
  if (e == 0) return 0;  // zero (subnormals: below 2^-126, dropped)
  return fixed_from_parts((b & 0x7fffffu) | 0x800000u, e - 150, (b >> 31) != 0);
}
__device__ __forceinline__ u128 to_fixed(double v) {
  const uint64_t b = static_cast<uint64_t>(__double_as_longlong(v));
  const int e = static_cast<int>((b >> 52) & 0x7ffu);
  if (e == 0) return 0;
  return fixed_from_parts((b & 0xfffffffffffffull) | 0x10000000000000ull, e - 1075,
                          (b >> 63) != 0);
}
__device__ __forceinline__ u128 to_fixed(float2 v) { return to_fixed(v.x) + to_fixed(v.y); }

// Round a non-negative fixed-point value (frac fractional bits) to nearest, ties to even, with
// `bits` significant bits: returns the IEEE bit pattern for the given exponent bias.
__device__ __forceinline__ uint64_t fixed_round_bits(u128 F, int bits, int bias, int frac) {
  if (F == 0) return 0;
  const uint64_t hi = static_cast<uint64_t>(F >> 64), lo = static_cast<uint64_t>(F);
  const int p = hi ? 127 - __clzll(static_cast<long long>(hi)) : 63 - __clzll(static_cast<long long>(lo));
  const int r = p - (bits - 1);  // bits below the kept significand
  uint64_t mant;
  bool up = false;
  if (r <= 0) {
    mant = static_cast<uint64_t>(F) << (-r);
  } else {
    mant = static_cast<uint64_t>(F >> r);
    const bool half = ((F >> (r - 1)) & 1) != 0;
    const bool sticky = r > 1 && (F & ((static_cast<u128>(1) << (r - 1)) - 1)) != 0;
    up = half && (sticky || (mant & 1));
  }
  const uint64_t frac_mask = (1ull << (bits - 1)) - 1;
  const uint64_t expo = static_cast<uint64_t>(p - frac + bias);
  return ((expo << (bits - 1)) | (mant & frac_mask)) + (up ? 1 : 0);
}
__device__ __forceinline__ float fixed_to_float(u128 F, int frac) {
  return __uint_as_float(static_cast<uint32_t>(fixed_round_bits(F, 24, 127, frac)));
}
__device__ __forceinline__ double fixed_to_double(u128 F, int frac) {
  return __longlong_as_double(static_cast<long long>(fixed_round_bits(F, 53, 1023, frac)));
}
__device__ __forceinline__ float fixed_to_float_signed(u128 F, int frac) {
  const bool neg = static_cast<int64_t>(static_cast<uint64_t>(F >> 64)) < 0;
  const float x = fixed_to_float(neg ? static_cast<u128>(0) - F : F, frac);
  return neg ? -x : x;
}
__device__ __forceinline__ float fixed_to(u128 F, float, int frac) { return fixed_to_float(F, frac); }
__device__ __forceinline__ double fixed_to(u128 F, double, int frac) {
  return fixed_to_double(F, frac);
}
__device__ __forceinline__ float2 fixed_to(u128 F, float2, int frac) {  // hi + lo, hi = RN(F)
  const float hi = fixed_to_float(F, frac);
  // hi as fixed point: its bits are a subset of F's (|hi - F| < ulp(hi)), shifted into place
  const uint32_t b = __float_as_uint(hi);
  const int e = static_cast<int>((b >> 23) & 0xffu);
  u128 H = 0;
  if (e != 0) {
    const int sh = e - 150 + frac;
    const u128 m = (b & 0x7fffffu) | 0x800000u;
    H = sh >= 0 ? (m << sh) : (m >> (-sh));
  }
  return make_float2(hi, fixed_to_float_signed(F - H, frac));
}
__device__ __forceinline__ u128 shfl_up_u128(u128 v, int d) {
  const uint64_t hi = __shfl_up_sync(0xffffffffu, static_cast<uint64_t>(v >> 64), d);
  const uint64_t lo = __shfl_up_sync(0xffffffffu, static_cast<uint64_t>(v), d);
  return (static_cast<u128>(hi) << 64) | lo;
}

// u128 helpers of the cooperative kernels: butterfly shuffle, a load through L2 of a value
// another CTA of the same launch wrote before a grid barrier, a 16-byte store, and the
// block-wide sum (every thread gets the result).
__device__ __forceinline__ u128 shfl_xor_u128(u128 v, int m) {
  const uint64_t hi = __shfl_xor_sync(0xffffffffu, static_cast<uint64_t>(v >> 64), m);
  const uint64_t lo = __shfl_xor_sync(0xffffffffu, static_cast<uint64_t>(v), m);
  return (static_cast<u128>(hi) << 64) | lo;
}
__device__ __forceinline__ u128 ld_u128_cg(const u128* p) {
  const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2*>(p));
  return (static_cast<u128>(v.y) << 64) | v.x;
}
__device__ __forceinline__ void st_u128(u128* p, u128 v) {
  *reinterpret_cast<ulonglong2*>(p) =
      make_ulonglong2(static_cast<uint64_t>(v), static_cast<uint64_t>(v >> 64));
}

__device__ __forceinline__ u128 block_sum_u128(u128 v, u128* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += shfl_xor_u128(v, o);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  u128 t = 0;
  for (int k = 0; k < kWarps; ++k) t += sh[k];
  return t;
}

// Block-wide exclusive scan of u128 values in thread order; `total` gets the block's sum
// (every thread). sh: kWarps entries.
__device__ __forceinline__ u128 block_excl_scan_u128(u128 v, u128* sh, u128& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u128 incl = v;
#pragma unroll
  for (int dd = 1; dd < 32; dd <<= 1) {
    const u128 y = shfl_up_u128(incl, dd);
    if (lane >= dd) incl += y;
  }
  __syncthreads();  // sh may still be read from a previous call
  if (lane == 31) sh[warp] = incl;
  __syncthreads();
  u128 before = 0, tot = 0;
#pragma unroll
  for (int k = 0; k < kWarps; ++k) {
    if (k < warp) before += sh[k];
    tot += sh[k];
  }
  total = tot;
  return before + incl - v;
}

// Block-wide sums of two u128 values (every thread gets both).
__device__ __forceinline__ void block_sum2_u128(u128& a, u128& b, u128* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += shfl_xor_u128(a, o);
    b += shfl_xor_u128(b, o);
  }
  __syncthreads();
  if (lane == 0) {
    sh[warp] = a;
    sh[kWarps + warp] = b;
  }
  __syncthreads();
  a = 0;
  b = 0;
#pragma unroll
  for (int k = 0; k < kWarps; ++k) {
    a += sh[k];
    b += sh[kWarps + k];
  }
}

// A segment's record (seg_record): its largest log-weight m_t, in the input type, in the first
// 4 or 8 bytes of a double2, and s_t = the sum of its weights relative to m_t,
// exp(lw_i - m_t), in the accumulator type, in the last 8 bytes.
template <typename T, typename V>
__device__ __forceinline__ void store_rec(double2* p, T m, V s) {
  *reinterpret_cast<T*>(p) = m;
  *reinterpret_cast<V*>(reinterpret_cast<char*>(p) + 8) = s;
}
__device__ __forceinline__ void from_bits(unsigned long long b, float& v) {
  v = __uint_as_float(static_cast<unsigned int>(b));
}
__device__ __forceinline__ void from_bits(unsigned long long b, double& v) {
  v = __longlong_as_double(static_cast<long long>(b));
}
__device__ __forceinline__ void from_bits(unsigned long long b, float2& v) {
  v = make_float2(__uint_as_float(static_cast<unsigned int>(b)),
                  __uint_as_float(static_cast<unsigned int>(b >> 32)));
}
template <typename T, typename V>
__device__ __forceinline__ void load_rec(const double2* p, T& m, V& s) {
  const double2 r = __ldcg(p);  // (written by another CTA, or earlier, in this launch)
  from_bits(static_cast<unsigned long long>(__double_as_longlong(r.x)), m);
  from_bits(static_cast<unsigned long long>(__double_as_longlong(r.y)), s);
}

// The segment's total relative to the maximum M of the whole sequence: s_t exp(m_t - M),
// rounded in the accumulator type, 0 for a segment of zero weights. The difference m_t - M is taken
// exactly (a two-term sum: with it rounded, the relative error of the factor would grow with
// |m_t - M|); binary32 and binary64 scale by exp_pinned(d_hi) (1 + d_lo), the two-float
// accumulators by the two-float exp of the two-term difference, as their weights are formed.
// M = +inf (flagged non-finite input) gives 0 for finite m_t and NaN for m_t = +inf, as the
// weights exp(lw_i - M) themselves do.
template <typename T, typename V>
__device__ __forceinline__ V rec_scaled_of(const double2 r, T M) {
  T m;
  V sv;
  from_bits(static_cast<unsigned long long>(__double_as_longlong(r.x)), m);
  from_bits(static_cast<unsigned long long>(__double_as_longlong(r.y)), sv);
  if (!(m > neg_inf<T>())) return vzero(V());
  if constexpr (std::is_same_v<V, float>) {
    const float dh = __fsub_rn(m, M);
    float dl = 0.0f;
    if (dh > -INFINITY && dh < INFINITY) {  // TwoSum error of m - M
      const float bb = __fsub_rn(dh, m);
      dl = __fadd_rn(__fsub_rn(m, __fsub_rn(dh, bb)), __fsub_rn(-M, bb));
    }
    const float e = exp_pinned(dh);
    return __fmul_rn(sv, __fmaf_rn(e, dl, e));
  } else if constexpr (std::is_same_v<V, double>) {
    const double dh = __dsub_rn(m, M);
    double dl = 0.0;
    if (dh > -DBL_MAX && dh < DBL_MAX) {
      const double bb = __dsub_rn(dh, m);
      dl = __dadd_rn(__dsub_rn(m, __dsub_rn(dh, bb)), __dsub_rn(-M, bb));
    }
    const double e = exp_pinned(dh);
    return __dmul_rn(sv, __fma_rn(e, dl, e));
  } else {  // two-float accumulators
    float2 d;
    if constexpr (sizeof(T) == 4) d = two_sum(m, -M);
    else d = add22_accurate(split_f64(m), neg2(split_f64(M)));
    return mul22(sv, exp_df(d, kExp2Frac64));
  }
}
template <typename T, typename V>
__device__ __forceinline__ V rec_scaled(const double2* p, T M) {
  return rec_scaled_of<T, V>(__ldcg(p), M);  // (written by another CTA, or earlier, in this launch)
}
template <typename T, typename V>
__device__ __forceinline__ u128 rec_fixed(const double2* p, T M) {
  return to_fixed(rec_scaled<T, V>(p, M));
}
template <typename T, typename V>
__device__ __forceinline__ u128 rec_fixed_of(const double2 r, T M) {
  return to_fixed(rec_scaled_of<T, V>(r, M));
}

// Prefixes of one sequence of nt segment records, M the sequence's maximum log-weight
// (block-level, every thread of the CTA calls it): with T_g = rec_scaled(record g), P_g =
// RN(T_0 + ... + T_{g-1}) for g = 0..nt, the exact sums taken in fixed point (each thread a
// contiguous chunk of records, then a warp scan and a scan over the warps: integer adds, so the
// order does not matter). P is non-decreasing because the exact prefixes are and rounding is
// monotone. The total S is P_nt, the cumulative weight the emission gives the last particle
// (seg_cum_weights), so that particle receives O = N.
// Thread 0 writes S, N / S and S (binary64) to the given pointers, then the CTA synchronises.
template <typename T, typename V>
__device__ void seg_prefix_compute(const double2* s_rec, double2* P_rec, int nt, int64_t N,
                                   T M, V* S_out, V* scale_out, double* Sd_out) {
  __shared__ u128 sh_sum[kWarps];
  constexpr int kGroup = 4;  // tile totals loaded together
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int chunk = (nt + kBlock - 1) / kBlock;
  const int t0 = min(nt, tid * chunk), t1 = min(nt, t0 + chunk);
  u128 cache[kGroup];  // the first group stays in registers
  u128 local = 0;
  for (int g = t0; g < t1; g += kGroup) {
    u128 f[kGroup];
#pragma unroll
    for (int k = 0; k < kGroup; ++k) f[k] = (g + k < t1) ? rec_fixed<T, V>(s_rec + g + k, M) : 0;
#pragma unroll
    for (int k = 0; k < kGroup; ++k) {
      local += f[k];
      if (g == t0) cache[k] = f[k];
    }
  }
  u128 incl = local;
#pragma unroll
  for (int dd = 1; dd < 32; dd <<= 1) {
    const u128 y = shfl_up_u128(incl, dd);
    if (lane >= dd) incl += y;
  }
  if (lane == 31) sh_sum[warp] = incl;
  __syncthreads();
  u128 p = incl - local;
  for (int k = 0; k < warp; ++k) p += sh_sum[k];
  for (int g = t0; g < t1; g += kGroup) {
    u128 f[kGroup];
#pragma unroll
    for (int k = 0; k < kGroup; ++k)
      f[k] = (g == t0) ? cache[k] : ((g + k < t1) ? rec_fixed<T, V>(s_rec + g + k, M) : 0);
#pragma unroll
    for (int k = 0; k < kGroup; ++k) {
      if (g + k < t1) {
        store_v<V>(P_rec + g + k, fixed_to(p, V(), kFixFrac));
        p += f[k];
      }
    }
  }
  if (t1 == nt && t0 < nt) store_v<V>(P_rec + nt, fixed_to(p, V(), kFixFrac));
  __syncthreads();
  if (tid == 0) {
    const V S = load_v_cg<V>(P_rec + nt);
    const double Sd = vto_double(S);
    *S_out = S;
    *scale_out = vfrom_double(__ddiv_rn(static_cast<double>(N), Sd), V());
    *Sd_out = Sd;
  }
  __syncthreads();
}

// Shared scratch of the segment emissions: one warp_runs window per warp.
struct SegSh {
  alignas(16) int32_t win[kWarps][kRunWin];
};

// Code 11 for the particles of one warp: out[j] = the index of the particle whose run
// [O_{i-1}, O_i) holds j, for every j of the warp's range [P0, P1) (P0 = the count before the
// warp's first particle, P1 = after its last). Lane l holds the non-decreasing counts Oe[q] of
// its kPer particles i0 + q and `prev`, the count before them. The range is written in
// rounds of kRunWin positions through the warp's shared window: -1 everywhere, the first
// position of each run receives its particle's index, a running maximum (in-lane, then a
// max-scan over the lanes, then the last value of the previous round, which every lane takes
// into account: a run can cover a whole round) fills the runs, and the window is stored with
// consecutive lanes on consecutive positions. The first position P0 always starts a run, so
// the carry of the first round can be -1. Same result as writing out[j] = i for j in
// [O_{i-1}, O_i) particle by particle, without its divergent loops.
__device__ __forceinline__ void warp_runs(const int32_t (&Oe)[kPer], int32_t prev, int32_t i0,
                                          int32_t* __restrict__ out, int32_t* win) {
  const int lane = threadIdx.x & 31;
  const int32_t P0 = __shfl_sync(0xffffffffu, prev, 0);
  const int32_t P1 = __shfl_sync(0xffffffffu, Oe[kPer - 1], 31);
  int4* const w4 = reinterpret_cast<int4*>(win);
  int32_t carry = -1;
  for (int32_t base = P0; base < P1; base += kRunWin) {  // warp-uniform
    __syncwarp();
    w4[2 * lane] = make_int4(-1, -1, -1, -1);
    w4[2 * lane + 1] = make_int4(-1, -1, -1, -1);
    __syncwarp();
    int32_t p = prev;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int32_t pos = p - base;
      if (Oe[q] > p && pos >= 0 && pos < kRunWin) win[pos] = i0 + q;
      p = Oe[q];
    }
    __syncwarp();
    const int4 u0 = w4[2 * lane], u1 = w4[2 * lane + 1];
    int32_t v[kPer] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
    for (int k = 1; k < kPer; ++k) v[k] = max(v[k], v[k - 1]);
    int32_t m = v[kPer - 1];
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, m, dd);
      if (lane >= dd) m = max(m, y);
    }
    int32_t em = __shfl_up_sync(0xffffffffu, m, 1);  // the earlier lanes of this round
    em = lane == 0 ? carry : max(em, carry);          // and the run carried into the round
#pragma unroll
    for (int k = 0; k < kPer; ++k) v[k] = max(v[k], em);
    carry = __shfl_sync(0xffffffffu, v[kPer - 1], 31);
    __syncwarp();
    w4[2 * lane] = make_int4(v[0], v[1], v[2], v[3]);
    w4[2 * lane + 1] = make_int4(v[4], v[5], v[6], v[7]);
    __syncwarp();
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int32_t j = base + 32 * k + lane;
      if (j < P1) out[j] = win[32 * k + lane];
    }
  }
}

// The record of a segment (warp-level) from this lane's kPer log-weights x of it (-inf outside
// the sequence): m_t = the segment's largest log-weight (NaN skipped; NaN and +inf set `bad`)
// and s_t = the sum of the weights relative to it, exp(x_i - m_t), in the accumulator type
// (sequential over a lane's kPer, then a butterfly over the warp; 0 when m_t = -inf). Lane 0
// stores the record at rec; every lane gets the key of m_t. A record does not depend on the
// sequence's maximum M, so the records are formed in the same pass as M; T_t = s_t
// exp(m_t - M) (rec_scaled) is the segment's total relative to M. With a reference key `ref`
// (the paths without kTileRef pass M's) m_t is that reference instead, and nothing is flagged
// here (their maximum pass flags it): the record of M then scales by exactly 1. The prefixes
// only need an accurate total, because the emission pins every segment's last particle to the
// next prefix (seg_cum_weights). No block-level synchronisation.
constexpr long long kTileMaxRef = LLONG_MIN;  // (no valid reference key: never that of a number)

template <typename T, typename V>
__device__ __forceinline__ long long seg_record(const T (&x)[kPer], const float2* tab,
                                                double2* rec, bool& bad,
                                                long long ref = kTileMaxRef) {
  const int lane = threadIdx.x & 31;
  long long m;
  if (ref != kTileMaxRef) {  // (uniform) a given reference replaces the segment's maximum
    m = ref;
  } else if constexpr (sizeof(T) == 4) {
    float mf = -INFINITY;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      bad |= !(x[q] <= FLT_MAX);  // NaN or +inf (-inf and finite values pass)
      mf = fmaxf(mf, x[q]);       // fmaxf skips NaN
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mf = fmaxf(mf, __shfl_xor_sync(0xffffffffu, mf, o));
    m = max_key(mf);
  } else {
    m = max_key(neg_inf<double>());
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const bool nan = is_nan(x[q]);
      bad |= nan || is_pos_inf(x[q]);
      const long long k = max_key(x[q]);
      if (!nan && k > m) m = k;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long y = __shfl_xor_sync(0xffffffffu, m, o);
      m = y > m ? y : m;
    }
  }
  V t = vzero(V());
  if (m > max_key(neg_inf<T>())) {  // (uniform over the warp)
    const WeightCtx wc = ctx_of_key<T, V>(m, tab);
    t = vfrom_w(Path<T, V>::weight(x[0], wc), V());
#pragma unroll
    for (int q = 1; q < kPer; ++q) t = vadd(t, vfrom_w(Path<T, V>::weight(x[q], wc), V()));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = vadd(t, vshfl_xor(t, o));  // same value in every lane
  }
  if (lane == 0) store_rec<T, V>(rec, key_to<T>(m), t);
  return m;
}

// The same, loading the log-weights of the segment starting at `base` of the sequence [lo, N).
template <typename T, typename V>
__device__ __forceinline__ long long seg_record(const T* __restrict__ lw, int64_t lo, int64_t N,
                                                int64_t base, const float2* tab, bool vec,
                                                double2* rec, bool& bad,
                                                long long ref = kTileMaxRef,
                                                L2Hint hint = L2Hint::kNormal) {
  T x[kPer];
  load_per(lw, base + kPer * static_cast<int64_t>(threadIdx.x & 31), lo, N, vec, x, hint);
  return seg_record<T, V>(x, tab, rec, bad, ref);
}

// Cumulative weights W[q] of this lane's kPer particles of the segment starting at `base` of
// the sequence [lo, N) (warp-level), for the segment prefixes Ps (this segment) and Pn (the
// next), and Wb, the cumulative weight of the particle just before this lane's first one.
//
// Scan (the accumulator type's rounded additions, in a fixed order): l_q = sequential prefix
// of the lane's weights; e = exclusive Hillis-Steele scan of the lane totals over the warp;
// W_q = RN(RN(Ps + e) + l_q) -- at most 7 + 5 + 2 roundings on any path. Tree sums are not
// monotone, so:
//   * inside a lane W_q is non-decreasing by construction;
//   * across the lanes, W_q is raised to the running maximum of the earlier lanes' last values
//     (a max-scan over the lanes, from Ps) and clamped to at most Pn;
//   * the segment's last position, and its last valid particle, are pinned to Pn, so the
//     particle before any segment has exactly that segment's prefix Ps, and segments need
//     nothing from each other's scans.
// Every cumulative weight thus lies in [Ps, Pn] and the whole sequence is non-decreasing, so
// Code 11 writes every ancestor position exactly once. Positions past the sequence end have
// weight 0 and repeat the last valid value; callers do not emit them.
template <typename T, typename V>
__device__ __forceinline__ void seg_cum_weights(const T* __restrict__ lw, int64_t lo, int64_t N,
                                                int64_t base, const WeightCtx& wc, bool vec,
                                                V Ps, V Pn, V (&W)[kPer], V& Wb,
                                                L2Hint hint = L2Hint::kNormal) {
  const int lane = threadIdx.x & 31;
  T x[kPer];
  load_per(lw, base + kPer * static_cast<int64_t>(lane), lo, N, vec, x, hint);
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const V wv = vfrom_w(Path<T, V>::weight(x[q], wc), V());
    W[q] = (q == 0) ? wv : vadd(W[q - 1], wv);
  }
  V incl = W[kPer - 1];
#pragma unroll
  for (int dd = 1; dd < 32; dd <<= 1) {
    const V y = vshfl_up(incl, dd);
    if (lane >= dd) incl = vadd(y, incl);
  }
  V excl = vshfl_up(incl, 1);
  if (lane == 0) excl = vzero(V());
  const V b = vadd(Ps, excl);
#pragma unroll
  for (int q = 0; q < kPer; ++q) W[q] = vadd(b, W[q]);
  V m = W[kPer - 1];
#pragma unroll
  for (int dd = 1; dd < 32; dd <<= 1) {
    const V y = vshfl_up(m, dd);
    if (lane >= dd) m = tmax(y, m);
  }
  V pm = vshfl_up(m, 1);
  if (lane == 0) pm = Ps;
#pragma unroll
  for (int q = 0; q < kPer; ++q) W[q] = tmin(tmax(W[q], pm), Pn);
  if (lane == 31) W[kPer - 1] = Pn;
  const int lq = seg_count(base, N) - 1 - kPer * lane;  // the segment's last valid particle here?
  if (lq >= 0 && lq < kPer) {
#pragma unroll
    for (int q = 0; q < kPer; ++q)
      if (q == lq) W[q] = Pn;
  }
  Wb = vshfl_up(W[kPer - 1], 1);
  if (lane == 0) Wb = Ps;
}

// The systematic uniform u (counter (0, 0)), drawn once per CTA.
template <typename T, typename V>
__device__ __forceinline__ typename Path<T, V>::U cta_uniform0(const Keys& keys) {
  __shared__ typename Path<T, V>::U sh_u;
  __syncthreads();
  if (threadIdx.x == 0) sh_u = Path<T, V>::draw_u(draw(keys, 0u, 0u));
  __syncthreads();
  return sh_u;
}

// kPer int32 values to p[0 .. cnt) (128-bit stores when all are inside and p is aligned).
__device__ __forceinline__ void store_per(int32_t* __restrict__ p, const int32_t (&v)[kPer],
                                          int cnt) {
  if (cnt >= kPer && (reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
    reinterpret_cast<int4*>(p)[0] = make_int4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<int4*>(p)[1] = make_int4(v[4], v[5], v[6], v[7]);
  } else {
#pragma unroll
    for (int q = 0; q < kPer; ++q)
      if (q < cnt) p[q] = v[q];
  }
}

// Systematic / stratified emission of one segment starting at `base` of the sequence [lo, N)
// (warp-level): cumulative offspring O of every particle, the Code-11 scatter of local
// ancestor indices into a[lo + j] through the warp's window `win` and, when d is given, the
// Prepermute claims d[lo + i] = O_{i-1} if particle i has offspring, else n (for a
// non-decreasing ancestry the lowest claimant of slot i is the first position of its run).
// When cl is given (single sequence, lo = 0), one bit per particle instead: bit i % 8 of
// cl[i / 8] is set when particle i has offspring (its slot is claimed), the only part of the
// claims that the Permute of a non-decreasing ancestry cannot read off a itself
// (permute_sorted_bits_kernel).
// Ps, Pn: prefixes of this segment and the next; u_sys: the systematic uniform (cta_uniform0;
// unused when STRAT). Local indices are 32-bit (n < 2^31).
template <typename T, typename V, bool STRAT>
__device__ __forceinline__ void emit_seg_cumoff(const T* __restrict__ lw, int64_t lo, int64_t N,
                                                int64_t base, const WeightCtx& wc, bool vec,
                                                V Ps, V Pn, V S, V scale,
                                                typename Path<T, V>::U u_sys,
                                                const Keys& keys, int32_t* __restrict__ a,
                                                int32_t* __restrict__ d, int32_t* win,
                                                uint8_t* __restrict__ cl = nullptr,
                                                L2Hint hint = L2Hint::kNormal) {
  const int lane = threadIdx.x & 31;
  const int32_t n = static_cast<int32_t>(N - lo);
  const int cnt = seg_count(base, N) - kPer * lane;  // valid here
  const int32_t i0 = static_cast<int32_t>(base - lo) + kPer * lane;
  V W[kPer], Wb;
  seg_cum_weights<T, V>(lw, lo, N, base, wc, vec, Ps, Pn, W, Wb, hint);
  // O of this lane's particles; the last particle of the sequence gets n, and positions
  // past the end repeat the count before them (no offspring). A lane with a position past
  // the end holds the sequence's last particle or none, so its last count is n either way.
  int32_t O[kPer];
  int32_t Ob = n;  // (lane 0: the count before the segment)
  if constexpr (STRAT) {
    strat_offspring_warp<T, V>(W, Wb, S, scale, keys, n, cnt > 0, O, Ob);
  } else {
#pragma unroll
    for (int q = 0; q < kPer; ++q) O[q] = cum_offspring<T, V, STRAT>(W[q], S, scale, u_sys, keys, n);
    if (lane == 0 && cnt > 0) Ob = cum_offspring<T, V, STRAT>(Wb, S, scale, u_sys, keys, n);
  }
  const int32_t last = (cnt >= kPer && i0 + kPer - 1 != n - 1) ? O[kPer - 1] : n;
  int32_t prev = __shfl_up_sync(0xffffffffu, last, 1);
  if (lane == 0)  // (a segment wholly past the end follows the sequence's last particle: n)
    prev = Ob;
  int32_t dv[kPer];
  int32_t p = prev;
  if (base + kSeg < N) {  // (warp-uniform) all kSeg particles valid, none the sequence's last
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      dv[q] = (O[q] > p) ? p : n;
      p = O[q];
    }
  } else {
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int32_t Oc = (q >= cnt) ? p : ((i0 + q == n - 1) ? n : O[q]);
      dv[q] = (Oc > p) ? p : n;
      O[q] = Oc;
      p = Oc;
    }
  }
  warp_runs(O, prev, i0, a + lo, win);
  if (d && cnt > 0) store_per(d + lo + i0, dv, cnt);
  if (cl && cnt > 0) {  // (i0 is a multiple of kPer = 8: one byte per lane)
    uint32_t bits = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) bits |= static_cast<uint32_t>(dv[q] != n) << q;
    cl[i0 >> 3] = static_cast<uint8_t>(bits);
  }
}

// Stored cumulative weights of one segment (warp-level): W[e] for e in [lo, N).
template <typename V, typename OUT> __device__ __forceinline__ OUT convert_out(V v);
template <> __device__ __forceinline__ float convert_out<float, float>(float v) { return v; }
template <> __device__ __forceinline__ double convert_out<float, double>(float v) { return v; }
template <> __device__ __forceinline__ double convert_out<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float2 convert_out<float2, float2>(float2 v) { return v; }
template <> __device__ __forceinline__ float convert_out<float2, float>(float2 v) { return v.x; }
template <> __device__ __forceinline__ double convert_out<float2, double>(float2 v) {
  return vto_double(v);
}

template <typename T, typename V, typename OUT>
__device__ __forceinline__ void emit_seg_W(const T* __restrict__ lw, int64_t lo, int64_t N,
                                           int64_t base, const WeightCtx& wc, bool vec, V Ps,
                                           V Pn, OUT* __restrict__ Wout) {
  const int lane = threadIdx.x & 31;
  const int cnt = seg_count(base, N) - kPer * lane;
  V W[kPer], Wb;
  seg_cum_weights<T, V>(lw, lo, N, base, wc, vec, Ps, Pn, W, Wb);
  OUT* const p = Wout + base + kPer * static_cast<int64_t>(lane);
#pragma unroll
  for (int q = 0; q < kPer; ++q)
    if (q < cnt) p[q] = convert_out<V, OUT>(W[q]);
}

// Multinomial search (Code 5) for output i of a sequence of n cumulative weights W: u =
// U_i * W^N with U_i from counter (i, 0); the first j with W_j > u (the particle whose
// half-open interval holds u).
template <typename T, typename V>
__device__ __forceinline__ int32_t search_one(const V* __restrict__ W, int64_t n,
                                              const Keys& keys, int64_t i) {
  const V S = W[n - 1];
  const auto U = Path<T, V>::draw_u(draw(keys, static_cast<uint32_t>(i), 0u));
  const V u = vtimes_u(S, U);
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (vle(W[mid], u)) lo = mid + 1; else hi = mid;
  }
  return static_cast<int32_t>(lo < n ? lo : n - 1);
}

// ---------------------------------------------------------------------------------------
// Guide table of the multinomial search. Bucket edges e_b = float(b) * step (b = 0..n-1,
// step = W^N / n in binary32, e_n = +inf) are non-decreasing in b; G[b] = the first particle
// j with W_j > e_b, b = 0..n (G[n] = n - 1). Particle j owns the buckets b with
// C_{j-1} <= b < C_j, C_j = the first b with e_b >= W_j, so G is written by a Code-11-style
// scatter in the emit pass. For a draw u with e_b <= u < e_{b+1} the answer (the first j with
// W_j > u) lies in [G[b], G[b+1]], so a binary search of that range returns exactly what a
// binary search of the whole array returns, after about three loads instead of log2 n.
// ---------------------------------------------------------------------------------------
struct Guide {
  float step;      // W^N / n
  float inv_step;  // n / W^N (estimates only)
};
__device__ __forceinline__ Guide make_guide(double Sd, int64_t n) {
  Guide g;
  g.step = __double2float_rn(__ddiv_rn(Sd, static_cast<double>(n)));
  g.inv_step = __double2float_rn(__ddiv_rn(static_cast<double>(n), Sd));
  return g;
}
// (b < n < 2^31: a 32-bit conversion gives the same binary32 value as a 64-bit one; the 32-bit
// conversions here measured 2-5 % faster multinomial calls)
__device__ __forceinline__ float guide_edge(int64_t b, const Guide& g, int64_t n) {
  if (b >= n) return INFINITY;
  return __fmul_rn(__int2float_rn(static_cast<int>(b)), g.step);
}
template <typename V> __device__ __forceinline__ V edge_as(float e);
template <> __device__ __forceinline__ float edge_as<float>(float e) { return e; }
template <> __device__ __forceinline__ double edge_as<double>(float e) { return e; }
template <> __device__ __forceinline__ float2 edge_as<float2>(float e) { return make_float2(e, 0.0f); }

// C(W) = the first b in [0, n] with e_b >= W.
template <typename V>
__device__ __forceinline__ int64_t guide_count(V W, const Guide& g, int64_t n) {
  const float est = ceilf(__fmul_rn(vhi(W), g.inv_step));
  int64_t b = est > 0.0f ? (est < __int2float_rn(static_cast<int>(n)) ? __float2int_rz(est) : n)
                         : 0;
  int steps = 0;
  while (b > 0 && vle(W, edge_as<V>(guide_edge(b - 1, g, n))) && ++steps < 64) --b;
  while (b < n && !vle(W, edge_as<V>(guide_edge(b, g, n))) && ++steps < 64) ++b;
  if (steps >= 64) {  // far from the estimate: bisect the edges
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = lo + ((hi - lo) >> 1);
      if (vle(W, edge_as<V>(guide_edge(mid, g, n)))) hi = mid; else lo = mid + 1;
    }
    b = lo;
  }
  return b;
}

// Stored cumulative weights of one segment plus the guide-table scatter of its particles
// (warp-level; same cumulative-count pattern as emit_seg_cumoff).
template <typename T, typename V>
__device__ __forceinline__ void emit_seg_W_guide(const T* __restrict__ lw, int64_t lo, int64_t N,
                                                 int64_t base, const WeightCtx& wc, bool vec,
                                                 V Ps, V Pn, const Guide& gd,
                                                 V* __restrict__ Wout,
                                                 int32_t* __restrict__ G, int32_t* win,
                                                 L2Hint hint = L2Hint::kNormal) {
  const int lane = threadIdx.x & 31;
  const int32_t n = static_cast<int32_t>(N - lo);
  const int cnt = seg_count(base, N) - kPer * lane;
  const int32_t j0 = static_cast<int32_t>(base - lo) + kPer * lane;
  V W[kPer], Wb;
  seg_cum_weights<T, V>(lw, lo, N, base, wc, vec, Ps, Pn, W, Wb, hint);
  V* const p = Wout + base + kPer * static_cast<int64_t>(lane);
  int32_t C[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    if (q < cnt) p[q] = W[q];
    C[q] = static_cast<int32_t>(guide_count<V>(W[q], gd, n));
  }
  // the guide entries of a particle's buckets form runs like the ancestors of Code 11 (the
  // last particle's run ends at n, positions past the end add none)
  const int32_t last = (cnt >= kPer && j0 + kPer - 1 != n - 1) ? C[kPer - 1] : n;
  int32_t prev = __shfl_up_sync(0xffffffffu, last, 1);
  if (lane == 0) prev = cnt > 0 ? static_cast<int32_t>(guide_count<V>(Wb, gd, n)) : n;
  int32_t pc = prev;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int32_t Cc = (q >= cnt) ? pc : ((j0 + q == n - 1) ? n : C[q]);
    C[q] = Cc;
    pc = Cc;
  }
  int32_t* const Gl = G + lo;
  warp_runs(C, prev, j0, Gl, win);
  if (j0 <= n - 1 && n - 1 < j0 + kPer) Gl[n] = n - 1;
}

// Loads of W and G; kCoherent: written earlier in the same kernel launch, read through L2.
template <bool kCoherent, typename X> __device__ __forceinline__ X ld_val(const X* p) {
  if constexpr (kCoherent) return __ldcg(p); else return __ldg(p);
}

// Multinomial search of output i through the guide table (same result as search_one).
template <typename T, typename V, bool kCoherent = false>
__device__ __forceinline__ int32_t search_one_guided(const V* __restrict__ W,
                                                     const int32_t* __restrict__ G, int64_t n,
                                                     const Guide& gd, const Keys& keys,
                                                     int64_t i) {
  const V S = ld_val<kCoherent>(W + (n - 1));
  const auto U = Path<T, V>::draw_u(draw(keys, static_cast<uint32_t>(i), 0u));
  const V u = vtimes_u(S, U);
  // bucket b with e_b <= u < e_{b+1}
  const float est = floorf(__fmul_rn(vhi(u), gd.inv_step));
  int64_t b = est > 0.0f
                  ? (est < __int2float_rn(static_cast<int>(n - 1)) ? __float2int_rz(est) : n - 1)
                  : 0;
  int steps = 0;
  while (b > 0 && !vle(edge_as<V>(guide_edge(b, gd, n)), u) && ++steps < 64) --b;
  while (b < n - 1 && vle(edge_as<V>(guide_edge(b + 1, gd, n)), u) && ++steps < 64) ++b;
  int64_t lo = 0, hi = n;
  if (steps < 64) {
    lo = ld_val<kCoherent>(G + b);
    hi = static_cast<int64_t>(ld_val<kCoherent>(G + b + 1)) + 1;
  }
  if (hi - lo <= 8) {  // the usual case: count W_j <= u over the range, loads in parallel
    const int64_t len = hi - lo;
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q < len && vle(ld_val<kCoherent>(W + lo + q), u)) ++cnt;
    lo += cnt;
  } else {
    while (lo < hi) {
      const int64_t mid = lo + ((hi - lo) >> 1);
      if (vle(ld_val<kCoherent>(W + mid), u)) lo = mid + 1; else hi = mid;
    }
  }
  return static_cast<int32_t>(lo < n ? lo : n - 1);
}

// The same search for K outputs i0 .. i0 + K - 1 at once (the valid ones: i0 + q < n): the
// bucket of every draw first, then the guide entries of all K issued together, then their
// short W ranges (up to 8 entries each) together, so that K dependent chains of loads are in
// flight per thread. Each result equals search_one_guided's for its output.
template <typename T, typename V, int K>
__device__ __forceinline__ void search_group_guided(const V* __restrict__ W,
                                                    const int32_t* __restrict__ G, int64_t n,
                                                    const Guide& gd, const Keys& keys,
                                                    int64_t i0, int32_t (&res)[K]) {
  const V S = __ldg(W + (n - 1));
  V u[K];
  int64_t lo[K], hi[K];
  bool ok[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    ok[q] = i0 + q < n;
    const auto U = Path<T, V>::draw_u(draw(keys, static_cast<uint32_t>(i0 + q), 0u));
    u[q] = vtimes_u(S, U);
    const float est = floorf(__fmul_rn(vhi(u[q]), gd.inv_step));
    int64_t b = est > 0.0f
                    ? (est < __int2float_rn(static_cast<int>(n - 1)) ? __float2int_rz(est) : n - 1)
                    : 0;
    int steps = 0;
    while (b > 0 && !vle(edge_as<V>(guide_edge(b, gd, n)), u[q]) && ++steps < 64) --b;
    while (b < n - 1 && vle(edge_as<V>(guide_edge(b + 1, gd, n)), u[q]) && ++steps < 64) ++b;
    lo[q] = steps < 64 ? b : -1;  // (-1: search the whole range)
  }
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const int64_t b = lo[q];
    if (ok[q] && b >= 0) {
      lo[q] = __ldg(G + b);
      hi[q] = static_cast<int64_t>(__ldg(G + b + 1)) + 1;
    } else {
      lo[q] = 0;
      hi[q] = ok[q] ? n : 0;  // (no output: an empty range)
    }
  }
  int cnt[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    cnt[q] = 0;
    const int64_t len = hi[q] - lo[q];
    if (ok[q] && len <= 8) {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (k < len && vle(__ldg(W + lo[q] + k), u[q])) ++cnt[q];
    }
  }
#pragma unroll
  for (int q = 0; q < K; ++q) {
    int64_t l = lo[q], h = hi[q];
    if (h - l <= 8) {
      l += cnt[q];
    } else {
      while (l < h) {
        const int64_t mid = l + ((h - l) >> 1);
        if (vle(__ldg(W + mid), u[q])) l = mid + 1; else h = mid;
      }
    }
    res[q] = static_cast<int32_t>(l < n ? l : n - 1);
  }
}

}  // namespace
}  // namespace rsk
