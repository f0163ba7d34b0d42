// scan.cu -- the multinomial, stratified and systematic resamplers (Appendix B, Codes 5, 7,
// 8, with Code 11 and the Prepermute of Code 10 fused) on sm_103a.
//
// Each call makes three passes over the log-weights (Appendix E renormalisation, Code 4
// primitives):
//   1. max pass      : M = max_i lw_i (last-CTA reduction), NaN/+inf detection.
//   2. tile-sum pass : per tile of 4096 particles, the weights w_i = exp(lw_i - M) are
//                      prefix-summed in the accumulator type; the tile total is written and
//                      the last CTA to finish scans the tile totals (binary64) into tile
//                      prefixes P_t and the total W^N.
//   3. emit pass     : the same tile scan is recomputed bit for bit, offset by P_t, and
//                      turned into cumulative offspring O_i (systematic / stratified) with a
//                      direct Code-11 scatter of the ancestors and the Prepermute claims; or
//                      into stored cumulative weights W_i (multinomial, followed by the
//                      search kernel).
// Reading the weights twice is inherent: the normaliser W^N is needed before any O_i. The
// reduce-then-scan order needs no inter-CTA waiting at all.
//
// Monotonicity: floating-point tree sums are not monotone in general, so every tile value
// is passed through an exact running maximum, and every global cumulative weight is
// clamped into [P_t, P_{t+1}] with P monotone. Cumulative weights are therefore
// non-decreasing, the cumulative offspring too, and Code 11 writes every position of the
// ancestry vector exactly once.
//
// Accumulators (input type T, accumulator V): binary32 (float, float), two-float
// (float, float2), double-float for binary64 inputs on the binary32 pipes (double, float2:
// weights by exp_df, GB300 runs binary64 at 1/57 rate), native binary64 (double, double).
#include <cfloat>
#include <climits>

#include "common.cuh"
#include "dfexp.cuh"
#include "internal.h"
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

template <typename T, typename V> struct Path;
template <> struct Path<float, float> {
  using U = float;
  static constexpr int id = 0;
  static constexpr bool kTable = false;
  __device__ static float weight(float x, const WeightCtx& c) {
    return (x == neg_inf<float>()) ? 0.0f : exp_pinned(__fsub_rn(x, c.Mf));
  }
  __device__ static U draw_u(uint4 x) { return u01_f32(x); }
};
template <> struct Path<float, float2> {
  using U = float;
  static constexpr int id = 1;
  static constexpr bool kTable = false;
  __device__ static float2 weight(float x, const WeightCtx& c) {
    return make_float2((x == neg_inf<float>()) ? 0.0f : exp_pinned(__fsub_rn(x, c.Mf)), 0.0f);
  }
  __device__ static U draw_u(uint4 x) { return u01_f32(x); }
};
template <> struct Path<double, float2> {
  using U = float2;
  static constexpr int id = 2;
  static constexpr bool kTable = true;
  __device__ static float2 weight(double x, const WeightCtx& c) {
    if (x == neg_inf<double>()) return make_float2(0.0f, 0.0f);
    return exp_df(add22_accurate(split_f64(x), neg2(c.M2)), c.tab);
  }
  __device__ static U draw_u(uint4 x) { return u01_f2(x); }
};
template <> struct Path<double, double> {
  using U = double;
  static constexpr int id = 3;
  static constexpr bool kTable = false;
  __device__ static double weight(double x, const WeightCtx& c) {
    return (x == neg_inf<double>()) ? 0.0 : exp_pinned(__dsub_rn(x, c.Md));
  }
  __device__ static U draw_u(uint4 x) { return u01_f64(x); }
};

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

// Reads the 4 consecutive log-weights idx..idx+3 (positions >= N read as -inf).
template <typename T>
__device__ __forceinline__ void load4(const T* __restrict__ lw, int64_t idx, int64_t N, bool vec,
                                      T (&x)[4]) {
  if (vec) {
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
    for (int q = 0; q < 4; ++q) x[q] = (idx + q < N) ? lw[idx + q] : neg_inf<T>();
  }
}

// Element e of the tile owned by (warp, row, lane, q): warp*512 + row*128 + lane*4 + q.
__device__ __forceinline__ int tile_offset(int warp, int r, int lane, int q) {
  return warp * 512 + r * 128 + lane * 4 + q;
}

// The tile scan shared by the tile-sum and emit passes: val[r][q] = sum of the weights of
// the tile up to and including the element (r, q) of this thread, as computed by a fixed
// tree: sequential inside a lane, Hillis-Steele across the 32 lanes of a row, a running
// carry across the 4 rows of a warp, and a sequential prefix over the 8 warps. Elements at
// positions >= N have weight 0. All four rows are loaded before any arithmetic.
template <typename T, typename V>
__device__ __forceinline__ void tile_raw_values(const T* __restrict__ lw, int64_t N, int64_t base,
                                                const WeightCtx& wc, bool vec,
                                                V (&val)[kRows][4], V* sh_tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x[kRows][4];
#pragma unroll
  for (int r = 0; r < kRows; ++r) load4(lw, base + tile_offset(warp, r, lane, 0), N, vec, x[r]);
  V carry = vzero(V());
#pragma unroll
  for (int r = 0; r < kRows; ++r) {
    V loc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const V wv = vfrom_w(Path<T, V>::weight(x[r][q], wc), V());
      loc[q] = (q == 0) ? wv : vadd(loc[q - 1], wv);
    }
    V incl = loc[3];
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
      const V y = vshfl_up(incl, dd);
      if (lane >= dd) incl = vadd(y, incl);
    }
    V excl = vshfl_up(incl, 1);
    if (lane == 0) excl = vzero(V());
    const V rowtot = vshfl(incl, 31);
#pragma unroll
    for (int q = 0; q < 4; ++q) val[r][q] = vadd(carry, vadd(excl, loc[q]));
    carry = vadd(carry, rowtot);
  }
  if (lane == 0) sh_tot[warp] = carry;
  __syncthreads();
  V pw = vzero(V());
  for (int k = 0; k < warp; ++k) pw = vadd(pw, sh_tot[k]);
#pragma unroll
  for (int r = 0; r < kRows; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) val[r][q] = vadd(pw, val[r][q]);
}

// Running maximum of the tile values in element order (exact), restricted to positions < N
// (later positions keep their raw value and are never used). Returns, through sh_max, the
// maximum of each warp's valid values; prevmax = maximum over the previous warps.
template <typename V>
__device__ __forceinline__ void tile_running_max(V (&val)[kRows][4], int64_t base, int64_t N,
                                                 V* sh_max, V& prevmax) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  V cm = vzero(V());
#pragma unroll
  for (int r = 0; r < kRows; ++r) {
    V x[4];
    V m = vzero(V());
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool valid = base + tile_offset(warp, r, lane, q) < N;
      if (valid) m = vmax(m, val[r][q]);
      x[q] = m;
    }
    V im = m;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
      const V y = vshfl_up(im, dd);
      if (lane >= dd) im = vmax(y, im);
    }
    V em = vshfl_up(im, 1);
    if (lane == 0) em = vzero(V());
    const V before = vmax(em, cm);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool valid = base + tile_offset(warp, r, lane, q) < N;
      if (valid) val[r][q] = vmax(x[q], before);
    }
    cm = vmax(cm, vshfl(im, 31));
  }
  if (lane == 0) sh_max[warp] = cm;
  __syncthreads();
  prevmax = vzero(V());
  for (int k = 0; k < warp; ++k) prevmax = vmax(prevmax, sh_max[k]);
#pragma unroll
  for (int r = 0; r < kRows; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool valid = base + tile_offset(warp, r, lane, q) < N;
      if (valid) val[r][q] = vmax(val[r][q], prevmax);
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

// ---------------------------------------------------------------------------------------
// Pass 1: maximum log-weight, compared through order-preserving integer keys (exact, and
// no binary64 arithmetic). NaN is skipped (and flagged, as is +inf).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ long long max_key(float v) {
  const int b = __float_as_int(v);
  return static_cast<long long>(b >= 0 ? b : (b ^ 0x7fffffff));
}
__device__ __forceinline__ long long max_key(double v) {
  const long long b = __double_as_longlong(v);
  return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double key_to_double(long long k, float) {
  const int b = static_cast<int>(k);
  return static_cast<double>(__int_as_float(b >= 0 ? b : (b ^ 0x7fffffff)));
}
__device__ __forceinline__ double key_to_double(long long k, double) {
  return __longlong_as_double(k >= 0 ? k : (k ^ 0x7fffffffffffffffLL));
}

template <typename T>
__global__ void __launch_bounds__(kBlock)
max_kernel(const T* __restrict__ lw, int64_t N, ScanGlob* g, double* blockmax, int* err,
           int32_t* d_init) {
  __shared__ long long sh[kWarps];
  __shared__ bool am_last;
  const long long kMin = max_key(neg_inf<T>());
  long long m = kMin;
  bool bad = false;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x * 4;
  const bool vec = (reinterpret_cast<uintptr_t>(lw) & 15u) == 0;
  for (int64_t i0 = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) * 4; i0 < N;
       i0 += stride) {
    T x[4];
    load4(lw, i0, N, vec && i0 + 4 <= N, x);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool nan = x[q] != x[q];
      bad |= nan || x[q] == static_cast<T>(INFINITY);
      const long long k = max_key(x[q]);
      if (!nan && k > m) m = k;
      if (d_init && i0 + q < N) d_init[i0 + q] = static_cast<int32_t>(N);
    }
  }
  if (bad) flag_error(err, RS_ERR_NONFINITE);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long y = __shfl_xor_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long bm = sh[0];
    for (int k = 1; k < kWarps; ++k) bm = sh[k] > bm ? sh[k] : bm;
    blockmax[blockIdx.x] = key_to_double(bm, T());
    __threadfence();
    const unsigned t = atomicAdd(&g->ticket_max, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  long long mm = max_key(-static_cast<double>(INFINITY));  // binary64 keys from here on
  for (int b = threadIdx.x; b < static_cast<int>(gridDim.x); b += blockDim.x) {
    const long long y = max_key(__ldcg(blockmax + b));
    mm = y > mm ? y : mm;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long y = __shfl_xor_sync(0xffffffffu, mm, o);
    mm = y > mm ? y : mm;
  }
  __syncthreads();
  if (lane == 0) sh[warp] = mm;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long bm = sh[0];
    for (int k = 1; k < kWarps; ++k) bm = sh[k] > bm ? sh[k] : bm;
    const double M = key_to_double(bm, 0.0);
    g->M = M;
    if (M == -INFINITY) flag_error(err, RS_ERR_ZERO_WEIGHT);
    g->ticket_max = 0u;
  }
}

// ---------------------------------------------------------------------------------------
// Tile prefixes (run by the last CTA of the tile-sum pass): P_0 = 0, P_{t+1} = P_t + s_t
// in binary64 with a running maximum, rounded monotonically to the accumulator type. The
// total used by the emit pass is the cumulative weight of the last particle exactly as the
// emit pass computes it, so that the last particle receives O = N.
// ---------------------------------------------------------------------------------------
template <typename V>
__device__ void tile_prefix_scan(const double2* s_rec, double2* P_rec, int T, ScanGlob* g,
                                 int64_t N, int* err, double* log_total_out) {
  __shared__ double sh_sum[kWarps];
  __shared__ double sh_max[kWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int chunk = (T + kBlock - 1) / kBlock;
  const int t0 = min(T, tid * chunk), t1 = min(T, t0 + chunk);
  double local = 0.0;
  for (int t = t0; t < t1; ++t) local = __dadd_rn(local, vto_double(load_v_cg<V>(s_rec + t)));
  double incl = local;
#pragma unroll
  for (int dd = 1; dd < 32; dd <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, incl, dd);
    if (lane >= dd) incl = __dadd_rn(y, incl);
  }
  double excl = __shfl_up_sync(0xffffffffu, incl, 1);
  if (lane == 0) excl = 0.0;
  if (lane == 31) sh_sum[warp] = incl;
  __syncthreads();
  double wp = 0.0;
  for (int k = 0; k < warp; ++k) wp = __dadd_rn(wp, sh_sum[k]);
  const double start = __dadd_rn(wp, excl);
  // end value of this thread's chunk (sequential), for the running maximum across threads
  double endv = start;
  for (int t = t0; t < t1; ++t) endv = __dadd_rn(endv, vto_double(load_v_cg<V>(s_rec + t)));
  double im = endv;
#pragma unroll
  for (int dd = 1; dd < 32; dd <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, im, dd);
    if (lane >= dd) im = y > im ? y : im;
  }
  double em = __shfl_up_sync(0xffffffffu, im, 1);
  if (lane == 0) em = 0.0;
  if (lane == 31) sh_max[warp] = im;
  __syncthreads();
  double prevmax = em;
  for (int k = 0; k < warp; ++k) prevmax = sh_max[k] > prevmax ? sh_max[k] : prevmax;
  double p = start;
  for (int t = t0; t < t1; ++t) {
    store_v<V>(P_rec + t, vfrom_double(p > prevmax ? p : prevmax, V()));
    p = __dadd_rn(p, vto_double(load_v_cg<V>(s_rec + t)));
  }
  if (t1 == T && t0 < T) store_v<V>(P_rec + T, vfrom_double(p > prevmax ? p : prevmax, V()));
  __syncthreads();
  if (tid == 0) {
    // the total is the cumulative weight of the last particle exactly as the emit pass
    // computes it: clamp(P_{T-1} + s_{T-1}, P_{T-1}, P_T)
    const V Pm = load_v_cg<V>(P_rec + (T - 1));
    const V Pn = load_v_cg<V>(P_rec + T);
    const V st = load_v_cg<V>(s_rec + (T - 1));
    const V S = vclamp(vadd(Pm, st), Pm, Pn);
    const double Sd = vto_double(S);
    store_v<V>(&g->S_raw, S);
    store_v<V>(&g->scale_raw, vfrom_double(__ddiv_rn(static_cast<double>(N), Sd), V()));
    g->S_d = Sd;
    if (!(Sd > 0.0)) flag_error(err, RS_ERR_ZERO_WEIGHT);
    if (log_total_out) *log_total_out = __dadd_rn(g->M, log(Sd));
  }
}

// ---------------------------------------------------------------------------------------
// Pass 2: tile sums and, in the last CTA, tile prefixes.
// ---------------------------------------------------------------------------------------
template <typename T, typename V>
__global__ void __launch_bounds__(kBlock)
tile_sum_kernel(const T* __restrict__ lw, int64_t N, ScanGlob* g, double2* s_rec,
                double2* P_rec, int* err, double* log_total_out) {
  __shared__ V sh_tot[kWarps];
  __shared__ V sh_max[kWarps];
  __shared__ float2 sh_tab[64];
  __shared__ bool am_last;
  const double Md = g->M;
  const bool zero = !(Md > -DBL_MAX);
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  V m = vzero(V());
  if (!zero) {
    const WeightCtx wc = make_ctx<T, V>(Md, sh_tab);
    const bool vec = ((reinterpret_cast<uintptr_t>(lw) & 15u) == 0) && (base + kTile <= N);
    V val[kRows][4];
    tile_raw_values<T, V>(lw, N, base, wc, vec, val, sh_tot);
#pragma unroll
    for (int r = 0; r < kRows; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (base + tile_offset(warp, r, lane, q) < N) m = vmax(m, val[r][q]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = vmax(m, vshfl_xor(m, o));
    if (lane == 0) sh_max[warp] = m;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    V tm = vzero(V());
    if (!zero)
      for (int k = 0; k < kWarps; ++k) tm = vmax(tm, sh_max[k]);
    store_v<V>(s_rec + blockIdx.x, tm);
    __threadfence();
    const unsigned t = atomicAdd(&g->ticket_tile, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  tile_prefix_scan<V>(s_rec, P_rec, static_cast<int>(gridDim.x), g, N, err, log_total_out);
  if (threadIdx.x == 0) g->ticket_tile = 0u;
}

// Cumulative offspring of a cumulative weight W (Codes 7 and 8 with r = W * N / W^N).
template <typename T, typename V, bool STRAT>
__device__ __forceinline__ int32_t cum_offspring(V W, V S, V scale,
                                                 typename Path<T, V>::U u_sys,
                                                 const Keys& keys, int64_t N) {
  if (veq(W, S)) return static_cast<int32_t>(N);
  const V r = vscale(W, scale);
  int64_t o;
  if constexpr (STRAT) {
    int64_t k = floor_to_i64(r);
    k = k < N - 1 ? k : N - 1;
    const auto uk = Path<T, V>::draw_u(draw(keys, static_cast<uint32_t>(k), 0u));
    o = floor_to_i64(vplus_u(r, uk));
    o = o < k + 1 ? o : k + 1;
  } else {
    o = floor_to_i64(vplus_u(r, u_sys));
  }
  o = o < N ? o : N;
  o = o > 0 ? o : 0;
  return static_cast<int32_t>(o);
}

// ---------------------------------------------------------------------------------------
// Pass 3a: systematic / stratified emission. Writes a (Code 11) and, when d is given, the
// Prepermute claims d_i = O_{i-1} if particle i has offspring, else N (for a
// non-decreasing ancestry the lowest claimant of slot i is the first position of its run).
// ---------------------------------------------------------------------------------------
template <typename T, typename V, bool STRAT>
__global__ void __launch_bounds__(kBlock)
emit_cumoff_kernel(const T* __restrict__ lw, int64_t N, const ScanGlob* g, const double2* s_rec,
                   const double2* P_rec, Keys keys, int32_t* __restrict__ a,
                   int32_t* __restrict__ d) {
  __shared__ V sh_tot[kWarps];
  __shared__ V sh_max[kWarps];
  __shared__ float2 sh_tab[64];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double Md = g->M;
  const V S = load_v<V>(&g->S_raw);
  if (!(Md > -DBL_MAX) || !(g->S_d > 0.0)) {  // all weights zero: flagged; emit identity
#pragma unroll
    for (int r = 0; r < kRows; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t i = base + tile_offset(warp, r, lane, q);
        if (i < N) {
          a[i] = static_cast<int32_t>(i);
          if (d) d[i] = static_cast<int32_t>(i);
        }
      }
    return;
  }
  const WeightCtx wc = make_ctx<T, V>(Md, sh_tab);
  const V scale = load_v<V>(&g->scale_raw);
  using U = typename Path<T, V>::U;
  const U u_sys = Path<T, V>::draw_u(draw(keys, 0u, 0u));
  const bool vec = ((reinterpret_cast<uintptr_t>(lw) & 15u) == 0) && (base + kTile <= N);
  V val[kRows][4];
  tile_raw_values<T, V>(lw, N, base, wc, vec, val, sh_tot);
  V prevmax;
  tile_running_max<V>(val, base, N, sh_max, prevmax);
  const int t = blockIdx.x;
  const V Pt = load_v<V>(P_rec + t), Pn = load_v<V>(P_rec + t + 1);
  int32_t O[kRows][4];
#pragma unroll
  for (int r = 0; r < kRows; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const V W = vclamp(vadd(Pt, val[r][q]), Pt, Pn);
      O[r][q] = cum_offspring<T, V, STRAT>(W, S, scale, u_sys, keys, N);
    }
  // cumulative offspring just before this warp's first element
  int32_t Obefore = 0;
  if (lane == 0) {
    if (warp > 0) {
      const V W = vclamp(vadd(Pt, prevmax), Pt, Pn);
      Obefore = cum_offspring<T, V, STRAT>(W, S, scale, u_sys, keys, N);
    } else if (t > 0) {
      const V Pm = load_v<V>(P_rec + t - 1), sm = load_v<V>(s_rec + t - 1);
      const V W = vclamp(vadd(Pm, sm), Pm, Pt);
      Obefore = cum_offspring<T, V, STRAT>(W, S, scale, u_sys, keys, N);
    }
  }
#pragma unroll
  for (int r = 0; r < kRows; ++r) {
    int32_t prev = __shfl_up_sync(0xffffffffu, O[r][3], 1);
    if (r > 0) {
      const int32_t rowprev = __shfl_sync(0xffffffffu, O[r - 1][3], 31);
      if (lane == 0) prev = rowprev;
    } else if (lane == 0) {
      prev = Obefore;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t i = base + tile_offset(warp, r, lane, q);
      int32_t Oc = O[r][q];
      if (i == N - 1) Oc = static_cast<int32_t>(N);
      if (i < N) {
        for (int32_t j = prev; j < Oc; ++j) a[j] = static_cast<int32_t>(i);
        if (d) d[i] = (Oc > prev) ? prev : static_cast<int32_t>(N);
      }
      prev = Oc;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Pass 3b: stored cumulative weights (multinomial search input, or rs_cumulative_weights
// output converted to the element type).
// ---------------------------------------------------------------------------------------
template <typename V, typename OUT> __device__ __forceinline__ OUT convert_out(V v);
template <> __device__ __forceinline__ float convert_out<float, float>(float v) { return v; }
template <> __device__ __forceinline__ double convert_out<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float2 convert_out<float2, float2>(float2 v) { return v; }
template <> __device__ __forceinline__ float convert_out<float2, float>(float2 v) { return v.x; }
template <> __device__ __forceinline__ double convert_out<float2, double>(float2 v) {
  return vto_double(v);
}

template <typename T, typename V, typename OUT>
__global__ void __launch_bounds__(kBlock)
emit_W_kernel(const T* __restrict__ lw, int64_t N, const ScanGlob* g, const double2* P_rec,
              OUT* __restrict__ Wout) {
  __shared__ V sh_tot[kWarps];
  __shared__ V sh_max[kWarps];
  __shared__ float2 sh_tab[64];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double Md = g->M;
  if (!(Md > -DBL_MAX) || !(g->S_d > 0.0)) {
    for (int r = 0; r < kRows; ++r)
      for (int q = 0; q < 4; ++q) {
        const int64_t i = base + tile_offset(warp, r, lane, q);
        if (i < N) Wout[i] = convert_out<V, OUT>(vzero(V()));
      }
    return;
  }
  const WeightCtx wc = make_ctx<T, V>(Md, sh_tab);
  const bool vec = ((reinterpret_cast<uintptr_t>(lw) & 15u) == 0) && (base + kTile <= N);
  V val[kRows][4];
  tile_raw_values<T, V>(lw, N, base, wc, vec, val, sh_tot);
  V prevmax;
  tile_running_max<V>(val, base, N, sh_max, prevmax);
  const int t = blockIdx.x;
  const V Pt = load_v<V>(P_rec + t), Pn = load_v<V>(P_rec + t + 1);
#pragma unroll
  for (int r = 0; r < kRows; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t i = base + tile_offset(warp, r, lane, q);
      if (i < N) Wout[i] = convert_out<V, OUT>(vclamp(vadd(Pt, val[r][q]), Pt, Pn));
    }
}

// ---------------------------------------------------------------------------------------
// Multinomial search (Code 5): u_i = U_i * W^N with U_i from counter (i, 0); a_i = the first
// j with W_j > u_i (the particle whose half-open interval holds u_i); then the Prepermute
// claim atomicMin(d[a_i], i) when d is given.
// ---------------------------------------------------------------------------------------
template <typename T, typename V>
__global__ void __launch_bounds__(kBlock)
search_kernel(const V* __restrict__ W, int64_t N, const ScanGlob* g, Keys keys,
              int32_t* __restrict__ a, int32_t* __restrict__ d) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (!(g->M > -DBL_MAX) || !(g->S_d > 0.0)) {
    a[i] = static_cast<int32_t>(i);
    if (d) atomicMin(d + i, static_cast<int32_t>(i));
    return;
  }
  const V S = W[N - 1];
  const auto U = Path<T, V>::draw_u(draw(keys, static_cast<uint32_t>(i), 0u));
  const V u = vtimes_u(S, U);
  int64_t lo = 0, hi = N;
  while (lo < hi) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (vle(W[mid], u)) lo = mid + 1; else hi = mid;
  }
  const int32_t k = static_cast<int32_t>(lo < N ? lo : N - 1);
  a[i] = k;
  if (d) atomicMin(d + k, static_cast<int32_t>(i));
}

int max_grid(int64_t N, int max_blocks) {
  const int64_t want = (N + kTile - 1) / kTile;
  return static_cast<int>(want < max_blocks ? want : max_blocks);
}

const char* const kLblMax[4] = {"max_f32", "max_f32c", "max_f64", "max_f64n"};
const char* const kLblTile[4] = {"tile_sum_f32", "tile_sum_f32c", "tile_sum_f64", "tile_sum_f64n"};
const char* const kLblSys[4] = {"emit_systematic_f32", "emit_systematic_f32c",
                                "emit_systematic_f64", "emit_systematic_f64n"};
const char* const kLblStr[4] = {"emit_stratified_f32", "emit_stratified_f32c",
                                "emit_stratified_f64", "emit_stratified_f64n"};
const char* const kLblW[4] = {"emit_W_f32", "emit_W_f32c", "emit_W_f64", "emit_W_f64n"};
const char* const kLblSearch[4] = {"search_f32", "search_f32c", "search_f64", "search_f64n"};

template <typename T, typename V>
cudaError_t run_scan(const Scratch& s, int scheme, const T* lw, int64_t N, uint64_t seed,
                     uint64_t step, uint32_t filter, int32_t* a_out, int32_t* d,
                     cudaStream_t st) {
  const int tiles = static_cast<int>((N + kTile - 1) / kTile);
  double2* s_rec = s.rec;
  double2* P_rec = s.rec + (s.max_tiles + 2);
  const Keys keys = make_keys(seed, step, filter, static_cast<uint32_t>(scheme));
  constexpr int ai = Path<T, V>::id;
  trace_mark(s.trace, kLblMax[ai], st);
  max_kernel<T><<<max_grid(N, s.max_blocks), kBlock, 0, st>>>(
      lw, N, s.glob, s.blockmax, s.err, scheme == RS_MULTINOMIAL ? d : nullptr);
  trace_mark(s.trace, kLblTile[ai], st);
  tile_sum_kernel<T, V><<<tiles, kBlock, 0, st>>>(lw, N, s.glob, s_rec, P_rec, s.err, nullptr);
  if (scheme == RS_SYSTEMATIC) {
    trace_mark(s.trace, kLblSys[ai], st);
    emit_cumoff_kernel<T, V, false><<<tiles, kBlock, 0, st>>>(lw, N, s.glob, s_rec, P_rec, keys,
                                                             a_out, d);
  } else if (scheme == RS_STRATIFIED) {
    trace_mark(s.trace, kLblStr[ai], st);
    emit_cumoff_kernel<T, V, true><<<tiles, kBlock, 0, st>>>(lw, N, s.glob, s_rec, P_rec, keys,
                                                            a_out, d);
  } else {
    V* W = static_cast<V*>(s.W);
    trace_mark(s.trace, kLblW[ai], st);
    emit_W_kernel<T, V, V><<<tiles, kBlock, 0, st>>>(lw, N, s.glob, P_rec, W);
    const int grid = static_cast<int>((N + kBlock - 1) / kBlock);
    trace_mark(s.trace, kLblSearch[ai], st);
    search_kernel<T, V><<<grid, kBlock, 0, st>>>(W, N, s.glob, keys, a_out, d);
  }
  return cudaGetLastError();
}

template <typename T, typename V, typename OUT>
cudaError_t run_cumw(const Scratch& s, const T* lw, int64_t N, OUT* W_out, double* log_total,
                     cudaStream_t st) {
  const int tiles = static_cast<int>((N + kTile - 1) / kTile);
  double2* s_rec = s.rec;
  double2* P_rec = s.rec + (s.max_tiles + 2);
  constexpr int ai = Path<T, V>::id;
  trace_mark(s.trace, kLblMax[ai], st);
  max_kernel<T><<<max_grid(N, s.max_blocks), kBlock, 0, st>>>(lw, N, s.glob, s.blockmax, s.err,
                                                              nullptr);
  trace_mark(s.trace, kLblTile[ai], st);
  tile_sum_kernel<T, V><<<tiles, kBlock, 0, st>>>(lw, N, s.glob, s_rec, P_rec, s.err,
                                                  log_total);
  trace_mark(s.trace, kLblW[ai], st);
  emit_W_kernel<T, V, OUT><<<tiles, kBlock, 0, st>>>(lw, N, s.glob, P_rec, W_out);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_scan_resample(const Scratch& s, int scheme, Acc acc, const void* logw,
                                 int64_t N, uint64_t seed, uint64_t step, uint32_t filter,
                                 int32_t* a_out, int32_t* d, cudaStream_t st) {
  switch (acc) {
    case Acc::F32:
      return run_scan<float, float>(s, scheme, static_cast<const float*>(logw), N, seed, step,
                                    filter, a_out, d, st);
    case Acc::F32C:
      return run_scan<float, float2>(s, scheme, static_cast<const float*>(logw), N, seed, step,
                                     filter, a_out, d, st);
    case Acc::F64:
      return run_scan<double, float2>(s, scheme, static_cast<const double*>(logw), N, seed,
                                      step, filter, a_out, d, st);
    case Acc::F64N:
      return run_scan<double, double>(s, scheme, static_cast<const double*>(logw), N, seed,
                                      step, filter, a_out, d, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_cumulative_weights(const Scratch& s, Acc acc, const void* logw, int64_t N,
                                      void* W_out, double* log_total, cudaStream_t st) {
  switch (acc) {
    case Acc::F32:
      return run_cumw<float, float, float>(s, static_cast<const float*>(logw), N,
                                           static_cast<float*>(W_out), log_total, st);
    case Acc::F32C:
      return run_cumw<float, float2, float>(s, static_cast<const float*>(logw), N,
                                            static_cast<float*>(W_out), log_total, st);
    case Acc::F64:
      return run_cumw<double, float2, double>(s, static_cast<const double*>(logw), N,
                                              static_cast<double*>(W_out), log_total, st);
    case Acc::F64N:
      return run_cumw<double, double, double>(s, static_cast<const double*>(logw), N,
                                              static_cast<double*>(W_out), log_total, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace rsk
