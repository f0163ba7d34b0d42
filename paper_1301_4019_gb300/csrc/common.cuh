// common.cuh -- device building blocks shared by the resampling kernels (sm_103a):
// counter-based Philox draws, exact uniforms, the uniform index map, the pinned
// exponential, the device status word and the value types of the prefix sums.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/resample.h"

namespace rsk {

constexpr int kBlock = 256;          // threads per CTA of the streaming kernels
constexpr int kPer = 8;              // consecutive particles per thread in a scan tile
constexpr int kTile = kBlock * kPer; // particles per CTA tile of the scan kernels (2048)
constexpr int kRunWin = 32 * kPer;  // positions a warp covers per round of Code 11 (warp_runs)
constexpr int kWarps = kBlock / 32;  // 8 warps
// Entries of each of the two record blocks of the scan scratch (records, then prefixes): one
// per warp segment of kRunWin particles (kWarps per tile), plus the total's prefix and a spare.
constexpr int64_t seg_cap(int64_t max_tiles) { return int64_t{kWarps} * max_tiles + 2; }

// ---------------------------------------------------------------------------------------
// Device status word: holds -status of the highest-priority error seen (lowest value),
// or INT_MAX when none. RS_ERR_ARG (1) > NONFINITE (2) > ZERO_WEIGHT (3) > BOUND (4) >
// REJECTION_CAP (5) > TIMEOUT (6).
// ---------------------------------------------------------------------------------------
constexpr int kNoError = 0x7fffffff;
__device__ __forceinline__ void flag_error(int* err, int status) { atomicMin(err, -status); }

// ---------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): 10 rounds of two 32x32->64 products
// on counter words 0 and 2, xor-mixed with the other words and the round key; the key is
// bumped by the golden-ratio and sqrt(3)-1 Weyl constants between rounds. The 10 round keys
// depend on the seed only, so they are computed once per call (on the host) and read from
// the kernel parameters.
// ---------------------------------------------------------------------------------------
// The draw keying of the library: key = seed; counter = (index, n, step, filter*8+purpose),
// purpose = the scheme (0..4), kPurposeBoundEstimate for the estimated rejection bound, 6 for
// the Philox throughput measurement.
constexpr uint32_t kPurposeBoundEstimate = 5;
struct Keys {
  uint32_t rk0[10], rk1[10];  // round keys: seed words plus r times the Weyl constants
  uint32_t step;              // SMC step mod 2^32
  uint32_t tag;               // filter * 8 + scheme
};
__host__ __device__ inline Keys make_keys(uint64_t seed, uint64_t step, uint32_t filter,
                                          uint32_t scheme) {
  Keys k;
  const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  for (uint32_t r = 0; r < 10; ++r) {
    k.rk0[r] = k0 + r * 0x9E3779B9u;
    k.rk1[r] = k1 + r * 0xBB67AE85u;
  }
  k.step = static_cast<uint32_t>(step);
  k.tag = (filter << 3) | (scheme & 7u);
  return k;
}
// The same keys for another filter and scheme (the round keys do not change).
__host__ __device__ inline Keys with_tag(const Keys& base, uint32_t filter, uint32_t scheme) {
  Keys k = base;
  k.tag = (filter << 3) | (scheme & 7u);
  return k;
}
__device__ __forceinline__ uint4 draw(const Keys& k, uint32_t index, uint32_t n) {
  uint4 c = make_uint4(index, n, k.step, k.tag);
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint64_t p0 = static_cast<uint64_t>(0xD2511F53u) * c.x;
    const uint64_t p1 = static_cast<uint64_t>(0xCD9E8D57u) * c.z;
    c = make_uint4(static_cast<uint32_t>(p1 >> 32) ^ c.y ^ k.rk0[round],
                   static_cast<uint32_t>(p1),
                   static_cast<uint32_t>(p0 >> 32) ^ c.w ^ k.rk1[round],
                   static_cast<uint32_t>(p0));
  }
  return c;
}

// U[0,1) with 24 (binary32) or 53 (binary64) random bits; both conversions are exact.
__device__ __forceinline__ float u01_f32(uint4 x) {
  return __fmul_rn(__uint2float_rn(x.x >> 8), 0x1p-24f);
}
__device__ __forceinline__ double u01_f64(uint4 x) {
  const uint64_t m = (static_cast<uint64_t>(x.x) << 21) | static_cast<uint64_t>(x.y >> 11);
  return __dmul_rn(__ull2double_rn(m), 0x1p-53);
}
template <typename T> __device__ __forceinline__ T u01(uint4 x);
template <> __device__ __forceinline__ float u01<float>(uint4 x) { return u01_f32(x); }
template <> __device__ __forceinline__ double u01<double>(uint4 x) { return u01_f64(x); }

// Uniform index on {0..N-1}: the high 64 bits of V * N, V = words 2,3 as a 64-bit integer.
// For N < 2^32 this is (x2 N + floor(x3 N / 2^32)) / 2^32 rounded down (the discarded low
// part cannot carry), two 32x32->64 products with no overflow.
__device__ __forceinline__ int64_t uniform_index(uint4 x, int64_t N) {
  const uint64_t n = static_cast<uint64_t>(N);
  const uint64_t lo = static_cast<uint64_t>(x.w) * n;
  const uint64_t hi = static_cast<uint64_t>(x.z) * n + (lo >> 32);
  return static_cast<int64_t>(hi >> 32);
}

// The two step halves of a binary32 Metropolis block (h = 0: words 0, 1; h = 1: words 2, 3):
// the uniform is the top 24 bits of the first word times 2^-24, the proposal floor(V N / 2^40)
// with V = (the first word's low byte) 2^32 + the second word. With Q = (V >> 32) N and
// P = (V mod 2^32) N, V N = (Q + floor(P / 2^32)) 2^32 + (P mod 2^32) and the last term
// cannot carry past bit 40, so the index is (Q + floor(P / 2^32)) / 2^8 rounded down.
__device__ __forceinline__ float half_u01_f32(uint32_t w0) {
  return __fmul_rn(__uint2float_rn(w0 >> 8), 0x1p-24f);
}
__device__ __forceinline__ int64_t half_index(uint32_t w0, uint32_t w1, int64_t N) {
  const uint64_t n = static_cast<uint64_t>(N);
  const uint64_t P = static_cast<uint64_t>(w1) * n;
  const uint64_t Q = static_cast<uint64_t>(w0 & 0xffu) * n;
  return static_cast<int64_t>((Q + (P >> 32)) >> 8);
}

// ---------------------------------------------------------------------------------------
// Pinned exponential for x <= 0, identical bit for bit on host and device: Cody & Waite
// argument reduction (x = k ln2 + r with ln2 split in head and tail), Taylor polynomial of
// e^r with coefficients 1/n! (degree 7 in binary32, 13 in binary64) in Horner form with
// fused multiply-adds, exact scaling by 2^k. Every operation is an explicitly rounded
// IEEE operation, so no compiler contraction can change a result. Below -86.5 (binary32)
// or -707 (binary64) the result is 0, so that every non-zero result is a normal number.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float exp_pinned(float x) {
  if (x != x) return x;
  if (x < -86.5f) return 0.0f;
  const float k = rintf(__fmul_rn(x, 0x1.715476p+0f));
  float r = __fmaf_rn(-k, 0x1.62e430p-1f, x);
  r = __fmaf_rn(-k, -0x1.05c610p-29f, r);
  float p = 0x1.a01a02p-13f;            // 1/7!
  p = __fmaf_rn(p, r, 0x1.6c16c2p-10f);  // 1/6!
  p = __fmaf_rn(p, r, 0x1.111112p-7f);   // 1/5!
  p = __fmaf_rn(p, r, 0x1.555556p-5f);   // 1/4!
  p = __fmaf_rn(p, r, 0x1.555556p-3f);   // 1/3!
  p = __fmaf_rn(p, r, 0x1p-1f);          // 1/2!
  p = __fmaf_rn(p, r, 1.0f);             // 1/1!
  p = __fmaf_rn(p, r, 1.0f);             // 1/0!
  const int ki = static_cast<int>(k);
  const float scale = __uint_as_float(static_cast<uint32_t>(ki + 127) << 23);
  return __fmul_rn(p, scale);
}

__device__ __forceinline__ double exp_pinned(double x) {
  if (x != x) return x;
  if (x < -707.0) return 0.0;
  const double k = rint(__dmul_rn(x, 0x1.71547652b82fep+0));
  double r = __fma_rn(-k, 0x1.62e42fefa39efp-1, x);
  r = __fma_rn(-k, 0x1.abc9e3b39803fp-56, r);
  double p = 0x1.6124613a86d09p-33;       // 1/13!
  p = __fma_rn(p, r, 0x1.1eed8eff8d898p-29);  // 1/12!
  p = __fma_rn(p, r, 0x1.ae64567f544e4p-26);  // 1/11!
  p = __fma_rn(p, r, 0x1.27e4fb7789f5cp-22);  // 1/10!
  p = __fma_rn(p, r, 0x1.71de3a556c734p-19);  // 1/9!
  p = __fma_rn(p, r, 0x1.a01a01a01a01ap-16);  // 1/8!
  p = __fma_rn(p, r, 0x1.a01a01a01a01ap-13);  // 1/7!
  p = __fma_rn(p, r, 0x1.6c16c16c16c17p-10);  // 1/6!
  p = __fma_rn(p, r, 0x1.1111111111111p-7);   // 1/5!
  p = __fma_rn(p, r, 0x1.5555555555555p-5);   // 1/4!
  p = __fma_rn(p, r, 0x1.5555555555555p-3);   // 1/3!
  p = __fma_rn(p, r, 0x1p-1);                 // 1/2!
  p = __fma_rn(p, r, 1.0);                    // 1/1!
  p = __fma_rn(p, r, 1.0);                    // 1/0!
  const long long ki = static_cast<long long>(k);
  const double scale = __longlong_as_double((ki + 1023LL) << 52);
  return __dmul_rn(p, scale);
}

// ---------------------------------------------------------------------------------------
// Binary32 exponential of the plain binary32 scans (the weights exp(lw - M) that the
// multinomial, stratified and systematic resamplers sum in plain binary32), for t <= 0: the
// hardware base-2 exponential (PTX ex2.approx.ftz.f32) of t log2(e) with the rounding error
// of that product restored. With L1 = RN(log2 e) and L2 = RN(log2 e - L1):
//   a = RN(t L1),  e = fma(t, L1, -a) + t L2
// (fma(t, L1, -a) is the exact error of the product: the error-free product of Dekker in the
// FMA form of Ogita, Rump and Oishi, 2005), so t log2(e) = a + e up to a few 2^-48 relative,
// and exp(t) = 2^a 2^e ~ y (1 + e ln 2) with y = ex2(a), the last step one FMA (|e| < 2^-17:
// the dropped (e ln 2)^2 / 2 is below 2^-35). Its relative error is that of ex2 plus about
// two roundings, whatever |t|; kScanExpRelErr bounds it, and rs_check_weight_exp checks that
// bound for every binary32 t in [-87, 0]. Below -150 the argument is clamped (so -inf gives
// 0, not NaN); every t < -87 gives 0 or a value below 2^-125. NaN stays NaN.
// ---------------------------------------------------------------------------------------
constexpr double kScanExpRelErr = 0x1p-21;
__device__ __forceinline__ float exp_scan_f32(float t) {
  t = (t < -150.0f) ? -150.0f : t;
  const float a = __fmul_rn(t, 0x1.715476p+0f);
  float e = __fmaf_rn(t, 0x1.715476p+0f, -a);
  e = __fmaf_rn(t, 0x1.4ae0c0p-26f, e);
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a));
  return __fmaf_rn(y, __fmul_rn(e, 0x1.62e430p-1f), y);
}

// ---------------------------------------------------------------------------------------
// L2 eviction priority of the streaming loads of the log-weights (a cache hint: the values
// loaded are the same). A pass whose data the same launch reads again marks its loads
// evict_last; the last pass over them marks its loads evict_first, leaving room in L2 for
// what the next kernel reads (the ancestors written by the emission).
// ---------------------------------------------------------------------------------------
enum class L2Hint { kNormal, kEvictLast, kEvictFirst };
__device__ __forceinline__ uint64_t l2_policy(L2Hint h) {
  uint64_t p = 0;
  if (h == L2Hint::kEvictLast)
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  else if (h == L2Hint::kEvictFirst)
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ float4 ld_stream(const float4* p, L2Hint h, uint64_t pol) {
  if (h == L2Hint::kNormal) return __ldg(p);
  float4 v;
  asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double2 ld_stream(const double2* p, L2Hint h, uint64_t pol) {
  if (h == L2Hint::kNormal) return __ldg(p);
  double2 v;
  asm("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
      : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
  return v;
}

// ---------------------------------------------------------------------------------------
// Programmatic dependent launch. Kernels of a call are launched with programmatic stream
// serialization, so a kernel is set up while its predecessor drains; it waits here, before
// touching memory, until the predecessor has completed and its writes are visible. (No
// kernel triggers its dependents early: dependents parked on an SM during a multi-wave
// predecessor measured slower.) A no-op for a kernel launched without the attribute.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Set (per host thread) while a conditional graph body is being captured: launches then go
// without the programmatic-serialization attribute (rs_capture_if_below).
inline bool& pdl_disabled() {
  static thread_local bool off = false;
  return off;
}

// Streaming multiprocessors of the current device (queried once per device).
inline int device_sm_count() {
  static int cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  if (cache[dev] < 1) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms < 1)
      return 1;
    cache[dev] = sms;
  }
  return cache[dev];
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_disabled() ? 0 : 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

// ---------------------------------------------------------------------------------------
// Log-weight classification.
// ---------------------------------------------------------------------------------------
// Binary64 classification by the bit pattern (integer pipe; GB300 runs binary64 compares at
// the 1/57 binary64 rate). Binary32 tests compare directly.
__device__ __forceinline__ bool is_nan(float v) { return v != v; }
__device__ __forceinline__ bool is_nan(double v) {
  return (static_cast<unsigned long long>(__double_as_longlong(v)) << 1) > 0xffe0000000000000ull;
}
__device__ __forceinline__ bool is_pos_inf(float v) { return v == INFINITY; }
__device__ __forceinline__ bool is_pos_inf(double v) {
  return __double_as_longlong(v) == 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool is_neg_inf(float v) { return v == -INFINITY; }
__device__ __forceinline__ bool is_neg_inf(double v) {
  return static_cast<unsigned long long>(__double_as_longlong(v)) == 0xfff0000000000000ull;
}
template <typename T> __device__ __forceinline__ bool nonfinite_logw(T v) {
  return is_nan(v) || is_pos_inf(v);
}
template <typename T> __device__ __forceinline__ T neg_inf() { return -static_cast<T>(INFINITY); }

// Order-preserving maps of floats to unsigned integers (for atomicMax of a maximum).
__device__ __forceinline__ uint32_t ordered_key(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float from_ordered_key(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}
__device__ __forceinline__ unsigned long long ordered_key(double f) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(f));
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double from_ordered_key(unsigned long long k) {
  return __longlong_as_double(static_cast<long long>(
      (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k));
}

}  // namespace rsk
