// batched.cu -- many independent filters of uneven sizes resampled in a handful of launches
// (F filters in CSR layout: filter f holds the particles offsets[f] .. offsets[f+1]-1).
//
// The paper resamples one filter per call; resampling thousands of small filters one call at a
// time is launch-bound, and giving each filter to one CTA serialises its passes and leaves the
// largest (or, for Metropolis, the highest-B) filters as a long tail. Here the work units are
// the tiles and the particles of all filters together:
//   plan    : tiles per filter (kTile particles, starting at the filter's first particle) and
//             their prefix over filters; per-filter maxima reset            (1 CTA)
//   max     : per tile, maximum log-weight, combined per filter by an atomic max of keys
//   sums    : per tile, the tile scan total                               (tile-parallel)
//   prefix  : per filter, tile prefixes, W^N and N / W^N                  (CTA per filter)
//   emit    : per tile, cumulative offspring + Code-11 scatter + claims, or stored W
//   search / Metropolis / rejection / Permute: one thread per particle, its filter found by a
//             binary search of the offsets.
// With cooperative launches (the default), max, sums, prefixes and emission run as one
// persistent launch over the tiles of all filters (batch_coop_kernel) after the plan, so a
// scan-based scheme is plan + one launch (+ the search for the multinomial) + Permute.
// Every unit runs the same device functions as the single-filter kernels on the same tile
// structure (relative to the filter's first particle), with the filter index in the
// random-number counter: filter f of a batched call equals rs_resample on that filter's slice
// with filter = f, bit for bit.
#include <climits>

#include "common.cuh"
#include "grid.cuh"
#include "internal.h"
#include "mcmc.cuh"
#include "permute.cuh"
#include "tile.cuh"
#include "values.cuh"

namespace rsk {
namespace {

// Particle g of the batch -> (filter f, its first particle lo, its size n, local index i).
// Returns false for positions past offsets[F] and for filters the plan rejected.
struct PartLoc {
  int f;
  int64_t lo, n, i;
};
__device__ __forceinline__ int filter_of(const int64_t* __restrict__ off, int F, int64_t g);
__device__ __forceinline__ bool locate_particle(const int64_t* __restrict__ off, int F,
                                                int64_t max_n, int64_t g, PartLoc& P) {
  if (g >= __ldg(off + F)) return false;
  P.f = filter_of(off, F, g);
  P.lo = __ldg(off + P.f);
  const int64_t hi = __ldg(off + P.f + 1);
  P.n = hi - P.lo;
  P.i = g - P.lo;
  return P.lo >= 0 && hi <= max_n && P.n > 0 &&
         P.n <= kBatchMaxN && P.i >= 0 && P.i < P.n;
}

// Filter holding global position g: the last f with off[f] <= g (off has F + 1 entries).
__device__ __forceinline__ int filter_of(const int64_t* __restrict__ off, int F, int64_t g) {
  int lo = 0, hi = F;  // invariant: off[lo] <= g < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= g) lo = mid; else hi = mid;
  }
  return lo;
}

// The filter of position g >= off[f] from the filter f of an earlier position: a few steps
// past the offsets g has crossed, else filter_of. Same filter as filter_of(off, F, g).
__device__ __forceinline__ int advance_filter(const int64_t* __restrict__ off, int F, int64_t g,
                                              int f) {
  for (int st = 0; st < 8; ++st) {
    if (f + 1 >= F || __ldg(off + f + 1) > g) return f;
    ++f;
  }
  return (f + 1 < F && __ldg(off + f + 1) <= g) ? filter_of(off, F, g) : f;
}

// locate_particle for position g < off[F] once its filter f is known.
__device__ __forceinline__ bool locate_in(const int64_t* __restrict__ off, int f, int64_t max_n,
                                          int64_t g, PartLoc& P) {
  P.f = f;
  P.lo = __ldg(off + f);
  const int64_t hi = __ldg(off + f + 1);
  P.n = hi - P.lo;
  P.i = g - P.lo;
  return P.lo >= 0 && hi <= max_n && P.n > 0 &&
         P.n <= kBatchMaxN && P.i >= 0 && P.i < P.n;
}

// Tile t of the batch -> its filter (the last f with tile_start[f] <= t).
__device__ __forceinline__ int filter_of_tile(const int32_t* __restrict__ ts, int F, int t) {
  int lo = 0, hi = F;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(ts + mid) <= t) lo = mid; else hi = mid;
  }
  return lo;
}

struct Batch {
  const int64_t* off;
  int F;
  int64_t max_n;
  int32_t* tile_start;   // F + 1
  long long* fmax;       // F, keys of the per-filter maxima
  double2* fS;           // F: total (accumulator type)
  double2* fscale;       // F: N / total
  double* fSd;           // F: total in binary64
  double2* s_rec;        // tile totals, indexed by batch tile
  double2* P_rec;        // tile prefixes, filter f at tile_start[f] + f
  const uint8_t* resample;  // F flags (0: the filter keeps its particles), or null = all
  int* err;
};

// Filter f is resampled unless a flag array says otherwise (rs_resample_batched_masked).
__device__ __forceinline__ bool resampled(const uint8_t* flags, int f) {
  return flags == nullptr || __ldg(flags + f) != 0;
}

// Plan: tiles per filter and their exclusive prefix; per-filter maxima reset; offsets checked.
__global__ void __launch_bounds__(1024) batch_plan_kernel(Batch b) {
  pdl_wait();
  __shared__ int sh[32];
  const int F = b.F;
  const int chunk = (F + blockDim.x - 1) / blockDim.x;
  const int f0 = min(F, static_cast<int>(threadIdx.x) * chunk), f1 = min(F, f0 + chunk);
  int local = 0;
  for (int f = f0; f < f1; ++f) {
    const int64_t lo = b.off[f], hi = b.off[f + 1], n = hi - lo;
    const bool ok = lo >= 0 && n >= 0 && hi <= b.max_n &&
                    n <= kBatchMaxN;
    if (!ok) flag_error(b.err, RS_ERR_ARG);
    local += ok ? static_cast<int>((n + kTile - 1) / kTile) : 0;
    b.fmax[f] = LLONG_MIN;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = local;
#pragma unroll
  for (int dd = 1; dd < 32; dd <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, dd);
    if (lane >= dd) incl += y;
  }
  if (lane == 31) sh[warp] = incl;
  __syncthreads();
  int p = incl - local;
  for (int k = 0; k < warp; ++k) p += sh[k];
  for (int f = f0; f < f1; ++f) {
    b.tile_start[f] = p;
    const int64_t lo = b.off[f], hi = b.off[f + 1], n = hi - lo;
    const bool ok = lo >= 0 && n >= 0 && hi <= b.max_n &&
                    n <= kBatchMaxN;
    p += ok ? static_cast<int>((n + kTile - 1) / kTile) : 0;
  }
  if (f1 == F && f0 < F) b.tile_start[F] = p;
  if (F == 0 && threadIdx.x == 0) b.tile_start[0] = 0;
}

// Locates batch tile t: its filter f, the filter's bounds and the tile's first particle.
struct TileLoc {
  int f;
  int t;       // tile index inside the filter
  int64_t lo, hi, base;
};
__device__ __forceinline__ bool locate_tile(const Batch& b, int tile, TileLoc& L) {
  if (tile >= __ldg(b.tile_start + b.F)) return false;
  L.f = filter_of_tile(b.tile_start, b.F, tile);
  L.t = tile - __ldg(b.tile_start + L.f);
  L.lo = __ldg(b.off + L.f);
  L.hi = __ldg(b.off + L.f + 1);
  L.base = L.lo + static_cast<int64_t>(L.t) * kTile;
  return true;
}

template <typename T>
__global__ void __launch_bounds__(kBlock) batch_max_kernel(const T* __restrict__ lw, Batch b) {
  pdl_wait();
  __shared__ long long sh[kWarps];
  TileLoc L;
  if (!locate_tile(b, blockIdx.x, L)) return;
  if (!resampled(b.resample, L.f)) return;  // a filter that keeps its particles: no passes
  const bool vec = (reinterpret_cast<uintptr_t>(lw) & 15u) == 0;
  const int64_t end = min(L.hi, L.base + kTile);
  long long m = max_key(neg_inf<T>());
  bool bad = false;
  for (int64_t i0 = L.base + 4 * static_cast<int64_t>(threadIdx.x); i0 < end; i0 += 4 * kBlock) {
    T x[4];
    load4(lw, i0, L.lo, end, vec, x);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool nan = is_nan(x[q]);
      bad |= nan || is_pos_inf(x[q]);
      const long long k = max_key(x[q]);
      if (!nan && k > m) m = k;
    }
  }
  if (bad) flag_error(b.err, RS_ERR_NONFINITE);
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
    // stored as the key of the binary64 value, comparable across both input types
    atomicMax(b.fmax + L.f, max_key(key_to_double(bm, T())));
  }
}

__device__ __forceinline__ double filter_M(const Batch& b, int f) {
  return key_to_double(__ldcg(b.fmax + f), 0.0);
}

template <typename T, typename V>
__global__ void __launch_bounds__(kBlock) batch_sum_kernel(const T* __restrict__ lw, Batch b) {
  pdl_wait();
  __shared__ float2 sh_tab[64];
  TileLoc L;
  if (!locate_tile(b, blockIdx.x, L)) return;
  if (!resampled(b.resample, L.f)) return;
  if (threadIdx.x < 64) sh_tab[threadIdx.x] = kExp2Frac64[threadIdx.x];
  __syncthreads();
  const bool vec = (reinterpret_cast<uintptr_t>(lw) & 15u) == 0;
  const int warp = threadIdx.x >> 5;
  bool bad = false;  // (the max pass flags non-finite input)
  long long ref = kTileMaxRef;
  if constexpr (!Path<T, V>::kTileRef) {
    const double M = filter_M(b, L.f);
    if (M > -DBL_MAX) ref = max_key(static_cast<T>(M));  // (records relative to M)
  }
  seg_record<T, V>(lw, L.lo, L.hi, L.base + kSeg * warp, sh_tab, vec,
                   b.s_rec + kWarps * blockIdx.x + warp, bad, ref);
}

template <typename T, typename V>
__global__ void __launch_bounds__(kBlock) batch_prefix_kernel(Batch b) {
  pdl_wait();
  const int f = blockIdx.x;
  const int64_t lo = b.off[f], hi = b.off[f + 1], n = hi - lo;
  const int t0 = b.tile_start[f], nt = b.tile_start[f + 1] - t0;
  if (nt <= 0 || n <= 0 || !resampled(b.resample, f)) return;
  if (!(filter_M(b, f) > -DBL_MAX)) {
    if (threadIdx.x == 0) {
      b.fSd[f] = 0.0;
      flag_error(b.err, RS_ERR_ZERO_WEIGHT);
    }
    return;
  }
  seg_prefix_compute<T, V>(b.s_rec + kWarps * t0, b.P_rec + kWarps * t0 + f, kWarps * nt, n,
                           static_cast<T>(filter_M(b, f)), reinterpret_cast<V*>(b.fS + f),
                           reinterpret_cast<V*>(b.fscale + f), b.fSd + f);
}

template <typename T, typename V, int SCHEME>
__global__ void __launch_bounds__(kBlock)
batch_emit_kernel(const T* __restrict__ lw, Batch b, Keys base_keys,
                  int32_t* __restrict__ a, int32_t* __restrict__ d, V* __restrict__ W) {
  pdl_wait();
  __shared__ SegSh sh;
  __shared__ float2 sh_tab[64];
  TileLoc L;
  if (!locate_tile(b, blockIdx.x, L)) return;
  const int64_t n = L.hi - L.lo;
  const double M = filter_M(b, L.f);
  const double Sd = __ldcg(b.fSd + L.f);
  // all weights zero (flagged), or a filter that is not resampled: the identity
  if (!resampled(b.resample, L.f) || !(M > -DBL_MAX) || !(Sd > 0.0)) {
    for (int64_t e = L.base + threadIdx.x; e < L.hi && e < L.base + kTile; e += kBlock) {
      a[e] = static_cast<int32_t>(e - L.lo);
      if (d) d[e] = static_cast<int32_t>(e - L.lo);
      if (W) W[e] = vzero(V());
    }
    return;
  }
  const WeightCtx wc = make_ctx<T, V>(M, sh_tab);
  const bool vec = (reinterpret_cast<uintptr_t>(lw) & 15u) == 0;
  const int warp = threadIdx.x >> 5;
  const double2* P = b.P_rec + kWarps * __ldg(b.tile_start + L.f) + L.f;
  const int gl = kWarps * L.t + warp;  // this warp's segment within the filter
  const V Ps = load_v_cg<V>(P + gl), Pn = load_v_cg<V>(P + gl + 1);
  const int64_t base = L.base + kSeg * warp;
  if constexpr (SCHEME == RS_MULTINOMIAL) {
    if (d)  // claims of the search kernel start from the sentinel n
      for (int64_t e = L.base + threadIdx.x; e < L.hi && e < L.base + kTile; e += kBlock)
        d[e] = static_cast<int32_t>(n);
    emit_seg_W<T, V, V>(lw, L.lo, L.hi, base, wc, vec, Ps, Pn, W);
  } else {
    const Keys keys = with_tag(base_keys, static_cast<uint32_t>(L.f), SCHEME);
    const typename Path<T, V>::U u_sys =
        SCHEME == RS_STRATIFIED ? typename Path<T, V>::U() : cta_uniform0<T, V>(keys);
    emit_seg_cumoff<T, V, SCHEME == RS_STRATIFIED>(
        lw, L.lo, L.hi, base, wc, vec, Ps, Pn, load_v_cg<V>(b.fS + L.f),
        load_v_cg<V>(b.fscale + L.f), u_sys, keys, a, d, sh.win[warp]);
  }
}

// ---------------------------------------------------------------------------------------
// The max, sum, prefix and emission passes of all filters in one cooperative launch (after the
// plan kernel): CTA c owns the contiguous batch tiles [c T / G, (c+1) T / G) of the T tiles of
// all filters together, and the CTAs meet at one grid barrier (two for compensated binary32,
// whose records follow the filter maxima):
//   phase 1  per tile, the records of its segments (seg_record, each warp its own: the
//            segment's maximum log-weight and its weights' sum relative to it), the maxima
//            combined per filter by an atomic max of keys;
//   phase 2  per tile, the exact sums of its filter's records scaled to the filter's maximum
//            (those before each of its segments, and all), rounded once to the segment
//            prefixes and W^N as seg_prefix_compute rounds them, then the emission.
// Every segment goes through the same device functions and rounded prefixes as in the separate
// batched kernels and the single-filter kernels, so filter f still equals rs_resample on its
// slice with filter = f, bit for bit.
// ---------------------------------------------------------------------------------------
template <typename T, typename V, int SCHEME>
__global__ void __launch_bounds__(kBlock)
batch_coop_kernel(const T* __restrict__ lw, Batch b, Keys base_keys, int32_t* __restrict__ a,
                  int32_t* __restrict__ d, V* __restrict__ W, GridBar* bar) {
  __shared__ SegSh sh;
  __shared__ float2 sh_tab[64];
  __shared__ u128 sh_sum[2 * kWarps];
  __shared__ u128 sh_f[kWarps];
  __shared__ double2 sh_P[kWarps + 1], sh_S, sh_scale;
  __shared__ double sh_Sd;
  unsigned int target = 0;
  const int T_tiles = __ldcg(b.tile_start + b.F);
  const int G = static_cast<int>(gridDim.x), c = static_cast<int>(blockIdx.x);
  const int t0 = static_cast<int>(static_cast<int64_t>(c) * T_tiles / G);
  const int t1 = static_cast<int>(static_cast<int64_t>(c + 1) * T_tiles / G);
  const bool vec = (reinterpret_cast<uintptr_t>(lw) & 15u) == 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < 64) sh_tab[threadIdx.x] = kExp2Frac64[threadIdx.x];
  __syncthreads();

  // ---- phase 1: segment records -> filter maxima (compensated binary32: the maxima only) ----
  {
    bool bad = false;
    for (int t = t0; t < t1; ++t) {
      TileLoc L;
      if (!locate_tile(b, t, L) || !resampled(b.resample, L.f)) continue;  // uniform per CTA
      const int64_t base = L.base + kSeg * warp;
      long long k;
      if constexpr (Path<T, V>::kTileRef) {
        k = seg_record<T, V>(lw, L.lo, L.hi, base, sh_tab, vec,
                             b.s_rec + kWarps * t + warp, bad);
      } else {
        T x[kPer];
        load_per(lw, base + kPer * static_cast<int64_t>(lane), L.lo, L.hi, vec, x);
        k = max_key(neg_inf<T>());
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
          const bool nan = is_nan(x[q]);
          bad |= nan || is_pos_inf(x[q]);
          const long long kq = max_key(x[q]);
          if (!nan && kq > k) k = kq;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const long long y = __shfl_xor_sync(0xffffffffu, k, o);
          k = y > k ? y : k;
        }
      }
      // stored as the key of the binary64 value, comparable across both input types
      if (lane == 0) atomicMax(b.fmax + L.f, max_key(key_to_double(k, T())));
    }
    if (bad) flag_error(b.err, RS_ERR_NONFINITE);
  }
  grid_barrier(bar, target, b.err);
  if constexpr (!Path<T, V>::kTileRef) {
    bool bad = false;
    for (int t = t0; t < t1; ++t) {
      TileLoc L;
      if (!locate_tile(b, t, L) || !resampled(b.resample, L.f)) continue;
      const double M = filter_M(b, L.f);
      seg_record<T, V>(lw, L.lo, L.hi, L.base + kSeg * warp, sh_tab, vec,
                       b.s_rec + kWarps * t + warp, bad,
                       M > -DBL_MAX ? max_key(static_cast<T>(M)) : kTileMaxRef);
    }
    grid_barrier(bar, target, b.err);
  }

  // ---- phase 2: prefixes of each segment from its filter's exact record sums, emission -------
  for (int t = t0; t < t1; ++t) {
    TileLoc L;
    if (!locate_tile(b, t, L)) continue;
    const int64_t n = L.hi - L.lo;
    const double M = filter_M(b, L.f);
    const bool active = resampled(b.resample, L.f) && M > -DBL_MAX;
    if (resampled(b.resample, L.f) && !(M > -DBL_MAX) && L.t == 0 && threadIdx.x == 0) {
      b.fSd[L.f] = 0.0;
      flag_error(b.err, RS_ERR_ZERO_WEIGHT);
    }
    double Sd = 0.0;
    V Ps = vzero(V()), Pn = vzero(V()), S = vzero(V()), scale = vzero(V());
    if (active) {
      const int first = kWarps * __ldg(b.tile_start + L.f);  // the filter's first segment
      const int nseg = kWarps * __ldg(b.tile_start + L.f + 1) - first;
      const int own = kWarps * L.t;                          // this tile's first, in the filter
      const T Mt = static_cast<T>(M);  // (exact: M is one of the filter's log-weights)
      u128 part = 0, tot = 0;
      for (int k = threadIdx.x; k < nseg; k += kBlock) {
        const u128 v = rec_fixed<T, V>(b.s_rec + first + k, Mt);
        tot += v;
        if (k < own) part += v;
        if (k >= own && k < own + kWarps) sh_f[k - own] = v;
      }
      block_sum2_u128(part, tot, sh_sum);  // (its barriers also publish sh_f)
      if (threadIdx.x <= kWarps) {  // the tile's segment prefixes, one per thread
        u128 p = part;
        for (int w = 0; w < static_cast<int>(threadIdx.x); ++w) p += sh_f[w];
        store_v<V>(&sh_P[threadIdx.x], fixed_to(p, V(), kFixFrac));
      }
      if (threadIdx.x == 0) {
        const V S0 = fixed_to(tot, V(), kFixFrac);
        const double Sd0 = vto_double(S0);
        const V sc0 = vfrom_double(__ddiv_rn(static_cast<double>(n), Sd0), V());
        store_v<V>(&sh_S, S0);
        store_v<V>(&sh_scale, sc0);
        sh_Sd = Sd0;
        if (L.t == 0) {  // the filter's totals, for the search kernel
          store_v<V>(b.fS + L.f, S0);
          store_v<V>(b.fscale + L.f, sc0);
          b.fSd[L.f] = Sd0;
        }
      }
      __syncthreads();
      Ps = load_v<V>(&sh_P[warp]);
      Pn = load_v<V>(&sh_P[warp + 1]);
      S = load_v<V>(&sh_S);
      scale = load_v<V>(&sh_scale);
      Sd = sh_Sd;
      __syncthreads();  // the shared values are rewritten by the next tile
    }
    if (!active || !(Sd > 0.0)) {  // all weights zero (flagged) or not resampled: identity
      for (int64_t e = L.base + threadIdx.x; e < L.hi && e < L.base + kTile; e += kBlock) {
        a[e] = static_cast<int32_t>(e - L.lo);
        if (d) d[e] = static_cast<int32_t>(e - L.lo);
        if (W) W[e] = vzero(V());
      }
      continue;
    }
    const WeightCtx wc = ctx_staged<T, V>(M, sh_tab);  // (the table was staged at the start)
    const int64_t base = L.base + kSeg * warp;
    if constexpr (SCHEME == RS_MULTINOMIAL) {
      if (d)  // claims of the search kernel start from the sentinel n
        for (int64_t e = L.base + threadIdx.x; e < L.hi && e < L.base + kTile; e += kBlock)
          d[e] = static_cast<int32_t>(n);
      emit_seg_W<T, V, V>(lw, L.lo, L.hi, base, wc, vec, Ps, Pn, W);
    } else {
      const Keys keys = with_tag(base_keys, static_cast<uint32_t>(L.f), SCHEME);
      // the filter's systematic uniform, drawn by every thread (no block synchronisation)
      const typename Path<T, V>::U u_sys =
          SCHEME == RS_STRATIFIED ? typename Path<T, V>::U()
                                  : Path<T, V>::draw_u(draw(keys, 0u, 0u));
      emit_seg_cumoff<T, V, SCHEME == RS_STRATIFIED>(lw, L.lo, L.hi, base, wc, vec, Ps, Pn, S,
                                                      scale, u_sys, keys, a, d, sh.win[warp]);
    }
  }
  grid_exit(bar, target);
}

template <typename T, typename V>
__global__ void __launch_bounds__(kBlock)
batch_search_kernel(const V* __restrict__ W, Batch b, int64_t total, Keys base_keys,
                    int32_t* __restrict__ a, int32_t* __restrict__ d) {
  pdl_wait();
  const int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  PartLoc P;
  if (g >= total || !locate_particle(b.off, b.F, b.max_n, g, P)) return;
  if (!resampled(b.resample, P.f) || !(__ldcg(b.fSd + P.f) > 0.0) ||
      !(filter_M(b, P.f) > -DBL_MAX))
    return;  // the identity, written by the emission kernel
  const Keys keys = with_tag(base_keys, static_cast<uint32_t>(P.f), RS_MULTINOMIAL);
  const int32_t k = search_one<T, V>(W + P.lo, P.n, keys, P.i);
  a[g] = k;
  if (d) atomicMin(d + P.lo + k, static_cast<int32_t>(P.i));
}

// Claims start from the sentinel n of each particle's filter. Eight consecutive particles per
// thread: the filter of the first is found by binary search (filter_of) and the others by
// stepping past the offsets they cross; each particle gets what locate_particle gives it
// (nothing when it fails), stored 128 bits at a time where all eight are set.
constexpr int kFillPer = 8;
__global__ void __launch_bounds__(kBlock)
batch_fill_sentinel_kernel(const int64_t* __restrict__ off, int F, int64_t total,
                           int32_t* __restrict__ d) {
  pdl_wait();
  const int64_t g0 = kFillPer * (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x);
  const int64_t offF = __ldg(off + F);
  const int64_t end = offF < total ? offF : total;
  if (g0 >= end) return;
  int f = filter_of(off, F, g0);
  int32_t v[kFillPer];
  unsigned set = 0;
#pragma unroll
  for (int q = 0; q < kFillPer; ++q) {
    const int64_t g = g0 + q;
    v[q] = 0;
    if (g >= end) continue;
    f = advance_filter(off, F, g, f);
    PartLoc P;
    if (locate_in(off, f, total, g, P)) {
      v[q] = static_cast<int32_t>(P.n);
      set |= 1u << q;
    }
  }
  if (set == (1u << kFillPer) - 1u && (reinterpret_cast<uintptr_t>(d + g0) & 15u) == 0) {
    int4* const p4 = reinterpret_cast<int4*>(d + g0);
    p4[0] = make_int4(v[0], v[1], v[2], v[3]);
    p4[1] = make_int4(v[4], v[5], v[6], v[7]);
  } else {
#pragma unroll
    for (int q = 0; q < kFillPer; ++q)
      if ((set >> q) & 1u) d[g0 + q] = v[q];
  }
}

// First particle of item q of this thread when each CTA covers blockDim.x * ipt consecutive
// particles, item q being the q-th blockDim.x-wide slice (coalesced for every q).
__device__ __forceinline__ int64_t item_index(int ipt, int q) {
  return (static_cast<int64_t>(blockIdx.x) * ipt + q) * blockDim.x + threadIdx.x;
}

// Metropolis (or one-particle-per-thread rejection) over the particles of all filters, ipt
// particles per thread (the launch shape is tunable; every particle's chain and claim are the
// same for any shape).
template <typename T>
__global__ void __launch_bounds__(kMaxTunedBlock)
batch_mcmc_kernel(const T* __restrict__ lw, const int64_t* __restrict__ off, int F,
                  int64_t total, int scheme, const int32_t* __restrict__ Bf, int32_t B,
                  Keys base_keys, double log_wmax, int64_t max_trials,
                  const uint8_t* __restrict__ flags, int32_t* __restrict__ a,
                  int32_t* __restrict__ d, int ipt, int* err) {
  pdl_wait();
  for (int q = 0; q < ipt; ++q) {
    const int64_t g = item_index(ipt, q);
    if (g >= total) return;
    PartLoc P;
    if (!locate_particle(off, F, total, g, P)) {
      if (g < __ldg(off + F)) flag_error(err, RS_ERR_ARG);
      continue;
    }
    int32_t k;
    if (!resampled(flags, P.f)) {
      k = static_cast<int32_t>(P.i);  // the filter keeps its particles
    } else if (scheme == RS_METROPOLIS) {
      int32_t Bv = Bf ? __ldg(Bf + P.f) : B;
      if (Bv < 0) {
        flag_error(err, RS_ERR_ARG);
        Bv = 0;
      }
      const Keys keys = with_tag(base_keys, static_cast<uint32_t>(P.f), RS_METROPOLIS);
      k = metropolis_one(lw + P.lo, P.n, Bv, keys, P.i, err);
    } else {
      const Keys keys = with_tag(base_keys, static_cast<uint32_t>(P.f), RS_REJECTION);
      k = rejection_one(lw + P.lo, P.n, log_wmax, max_trials, keys, P.i, err);
    }
    a[g] = k;
    if (d) atomicMin(d + P.lo + k, static_cast<int32_t>(P.i));
  }
}

// Rejection with warp refill over the particles of all filters (mcmc.cuh); a lane looks up
// the filter of every particle it takes.
template <typename T>
__global__ void __launch_bounds__(kBlock)
batch_rejection_kernel(const T* __restrict__ lw, const int64_t* __restrict__ off, int F,
                       int64_t total, Keys base_keys, double log_wmax, int64_t max_trials,
                       const uint8_t* __restrict__ flags, int32_t* __restrict__ a,
                       int32_t* __restrict__ d, int* err) {
  pdl_wait();
  const int lane = threadIdx.x & 31;
  const int64_t run = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t start = run * kRejRun;
  const int64_t limit = __ldg(off + F) < total ? __ldg(off + F) : total;
  if (start >= limit) return;  // uniform across the warp
  const int64_t end = start + kRejRun < limit ? start + kRejRun : limit;
  const RejBound rb = make_bound(log_wmax);
  int64_t g = start + lane;
  bool active = false;
  PartLoc P;
  Keys keys = base_keys;
  T lwi = T(0);
  bool keep = false;  // the particle's filter is not resampled: it settles on itself
  auto take = [&](int64_t gg) {
    g = gg;
    active = false;
    if (gg >= end) return;
    if (!locate_particle(off, F, total, gg, P)) {
      flag_error(err, RS_ERR_ARG);
      return;
    }
    active = true;
    keep = !resampled(flags, P.f);
    keys = with_tag(base_keys, static_cast<uint32_t>(P.f), RS_REJECTION);
    lwi = __ldg(lw + gg);
    if (nonfinite_logw(lwi)) flag_error(err, RS_ERR_NONFINITE);
  };
  take(g);
  int64_t head = start + 32;
  uint64_t s = 0;  // attempts made (max_trials < 2^32, but s + kRejBatch may pass 2^32)
  for (;;) {
    bool settled = false;
    if (active) {
      int64_t j = P.i;
      settled = keep || rejection_attempts<kRejBatch>(lw + P.lo, P.n, rb, keys, P.i,
                                                      static_cast<uint32_t>(s), lwi, max_trials,
                                                      j, err);
      s += kRejBatch;
      if (!settled && s >= static_cast<uint64_t>(max_trials)) {
        flag_error(err, RS_ERR_REJECTION_CAP);
        j = P.i;
        settled = true;
      }
      if (settled) {
        a[g] = static_cast<int32_t>(j);
        if (d) atomicMin(d + P.lo + j, static_cast<int32_t>(P.i));
      }
    }
    const unsigned done = __ballot_sync(0xffffffffu, settled);
    if (settled) {
      take(head + __popc(done & ((1u << lane) - 1u)));
      s = 0;
    }
    head += __popc(done);
    if (!__any_sync(0xffffffffu, active)) break;
  }
}

// Permute of every filter (permute.cuh), ipt slots per thread (tunable launch shape).
__global__ void __launch_bounds__(kMaxTunedBlock)
batch_permute_kernel(const int64_t* __restrict__ off, int F, int64_t total,
                     const int32_t* __restrict__ a, const int32_t* __restrict__ d,
                     int32_t* __restrict__ c, int ipt, int* err) {
  pdl_wait();
  const int64_t offF = __ldg(off + F);
  int f = -1;  // the filter of this thread's previous item (items ascend by blockDim.x)
  for (int q = 0; q < ipt; ++q) {
    const int64_t g = item_index(ipt, q);
    if (g >= total || g >= offF) return;
    f = f < 0 ? filter_of(off, F, g) : advance_filter(off, F, g, f);
    PartLoc P;
    if (!locate_in(off, f, total, g, P)) continue;
    permute_one(a + P.lo, d + P.lo, P.n, c + P.lo, P.i, err);
  }
}

// Total number of particles of the batch (offsets[F]) is not known on the host without a
// synchronisation, so grids are sized for the handle's capacity and surplus CTAs exit at once.
inline int grid_particles(int64_t cap) { return static_cast<int>((cap + kBlock - 1) / kBlock); }
inline int grid_shaped(int64_t cap, const LaunchCfg& c) {
  const int64_t per = static_cast<int64_t>(c.block) * c.ipt;
  return static_cast<int>((cap + per - 1) / per);
}

const char* const kLblSum[4] = {"batch_sum_f32", "batch_sum_f32c", "batch_sum_f64", "batch_sum_f64n"};
const char* const kLblEmit[4] = {"batch_emit_f32", "batch_emit_f32c", "batch_emit_f64",
                                 "batch_emit_f64n"};
const char* const kLblSearch[4] = {"batch_search_f32", "batch_search_f32c", "batch_search_f64",
                                   "batch_search_f64n"};

const char* const kLblCoop[4] = {"batch_coop_f32", "batch_coop_f32c", "batch_coop_f64",
                                 "batch_coop_f64n"};

// The cooperative form of the batched scan passes (batch_coop_kernel), sized to the resident
// grid; false when the device cannot run it (then the separate kernels run).
template <typename T, typename V, int SCHEME>
bool launch_batched_coop(const Scratch& s, const T* lw, const Batch& b, int64_t cap_tiles,
                         const Keys& keys, int32_t* a, int32_t* d, V* W, cudaStream_t st,
                         cudaError_t& e) {
  const int cap = coop_capacity(reinterpret_cast<const void*>(batch_coop_kernel<T, V, SCHEME>));
  if (cap < 1) return false;
  const int grid = static_cast<int64_t>(cap) < cap_tiles ? cap : static_cast<int>(cap_tiles);
  trace_mark(s.trace, kLblCoop[Path<T, V>::id], st);
  e = coop_launch(batch_coop_kernel<T, V, SCHEME>, grid, st, lw, b, keys, a, d, W, &s.glob->bar);
  return true;
}

template <typename T, typename V>
cudaError_t run_batched_scan(const Scratch& s, int scheme, const T* lw, const Batch& b,
                             int64_t cap_tiles, const Keys& keys, int32_t* a, int32_t* d,
                             cudaStream_t st) {
  constexpr int ai = Path<T, V>::id;
  const int tiles = static_cast<int>(cap_tiles);
  if (s.coop && s.launch_mode != RS_LAUNCH_SEPARATE) {
    cudaError_t e = cudaSuccess;
    V* Wc = static_cast<V*>(s.W);
    bool done;
    switch (scheme) {
      case RS_MULTINOMIAL:
        done = launch_batched_coop<T, V, RS_MULTINOMIAL>(s, lw, b, cap_tiles, keys, a, d, Wc, st, e);
        if (done && e == cudaSuccess) {
          trace_mark(s.trace, kLblSearch[ai], st);
          launch_pdl(batch_search_kernel<T, V>, grid_particles(s.max_n), kBlock, st, Wc, b,
                     s.max_n, keys, a, d);
          e = cudaGetLastError();
        }
        break;
      case RS_STRATIFIED:
        done = launch_batched_coop<T, V, RS_STRATIFIED>(s, lw, b, cap_tiles, keys, a, d, nullptr,
                                                        st, e);
        break;
      default:
        done = launch_batched_coop<T, V, RS_SYSTEMATIC>(s, lw, b, cap_tiles, keys, a, d, nullptr,
                                                        st, e);
        break;
    }
    if (done) return e;
  }
  trace_mark(s.trace, "batch_max", st);
  launch_pdl(batch_max_kernel<T>, tiles, kBlock, st, lw, b);
  trace_mark(s.trace, kLblSum[ai], st);
  launch_pdl(batch_sum_kernel<T, V>, tiles, kBlock, st, lw, b);
  trace_mark(s.trace, "batch_prefix", st);
  launch_pdl(batch_prefix_kernel<T, V>, b.F, kBlock, st, b);
  V* W = static_cast<V*>(s.W);
  trace_mark(s.trace, kLblEmit[ai], st);
  switch (scheme) {
    case RS_MULTINOMIAL:
      launch_pdl(batch_emit_kernel<T, V, RS_MULTINOMIAL>, tiles, kBlock, st, lw, b, keys, a, d, W);
      trace_mark(s.trace, kLblSearch[ai], st);
      launch_pdl(batch_search_kernel<T, V>, grid_particles(s.max_n), kBlock, st, W, b, s.max_n, keys,
                                                                            a, d);
      break;
    case RS_STRATIFIED:
      launch_pdl(batch_emit_kernel<T, V, RS_STRATIFIED>, tiles, kBlock, st, lw, b, keys, a, d, nullptr);
      break;
    default:
      launch_pdl(batch_emit_kernel<T, V, RS_SYSTEMATIC>, tiles, kBlock, st, lw, b, keys, a, d, nullptr);
      break;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_batched(const Scratch& s, int scheme, Acc acc, const void* logw,
                           const int64_t* offsets, int F, const int32_t* Bf, int32_t B,
                           uint64_t seed, uint64_t step, double log_wmax, int64_t max_trials,
                           const uint8_t* flags, int32_t* out, int permute, cudaStream_t st) {
  int32_t* a = permute ? s.a_tmp : out;
  int32_t* d = permute ? s.d : nullptr;
  const bool f64 = acc == Acc::F64 || acc == Acc::F64N;
  const Keys keys = make_keys(seed, step, 0u, static_cast<uint32_t>(scheme));
  // particles are bounded by the capacity; the true total is offsets[F] (checked per filter)
  const int64_t total = s.max_n;
  cudaError_t e = cudaSuccess;
  if (scheme == RS_METROPOLIS || scheme == RS_REJECTION) {
    if (d) {
      trace_mark(s.trace, "batch_fill", st);
      launch_pdl(batch_fill_sentinel_kernel,
                 static_cast<int>((total + kFillPer * kBlock - 1) / (kFillPer * kBlock)), kBlock, st,
                 offsets, F, total, d);
    }
    trace_mark(s.trace, scheme == RS_METROPOLIS ? (f64 ? "batch_metropolis_f64" : "batch_metropolis_f32")
                                                : (f64 ? "batch_rejection_f64" : "batch_rejection_f32"),
               st);
    const int grid_runs = static_cast<int>(((total + kRejRun - 1) / kRejRun * 32 + kBlock - 1) /
                                           kBlock);
    if (scheme == RS_REJECTION) {
      if (f64)
        launch_pdl(batch_rejection_kernel<double>, grid_runs, kBlock, st,
            static_cast<const double*>(logw), offsets, F, total, keys, log_wmax, max_trials,
            flags, a, d, s.err);
      else
        launch_pdl(batch_rejection_kernel<float>, grid_runs, kBlock, st,
            static_cast<const float*>(logw), offsets, F, total, keys, log_wmax, max_trials,
            flags, a, d, s.err);
    } else if (f64) {
      const LaunchCfg& c = s.batch_cfg[kCfgMetropolisF64];
      launch_pdl(batch_mcmc_kernel<double>, grid_shaped(total, c), c.block, st,
          static_cast<const double*>(logw), offsets, F, total, scheme, Bf, B, keys, log_wmax,
          max_trials, flags, a, d, c.ipt, s.err);
    } else {
      const LaunchCfg& c = s.batch_cfg[kCfgMetropolisF32];
      launch_pdl(batch_mcmc_kernel<float>, grid_shaped(total, c), c.block, st,
          static_cast<const float*>(logw), offsets, F, total, scheme, Bf, B, keys, log_wmax,
          max_trials, flags, a, d, c.ipt, s.err);
    }
  } else {
    Batch b;
    b.off = offsets;
    b.F = F;
    b.max_n = s.max_n;
    b.tile_start = s.batch_tile_start;
    b.fmax = s.batch_fmax;
    b.fS = s.batch_fS;
    b.fscale = s.batch_fscale;
    b.fSd = s.batch_fSd;
    b.s_rec = s.batch_s_rec;
    b.P_rec = s.batch_P_rec;
    b.resample = flags;
    b.err = s.err;
    trace_mark(s.trace, "batch_plan", st);
    launch_pdl(batch_plan_kernel, 1, 1024, st, b);
    // every filter adds at most one partial tile to the max_n / kTile full ones
    const int64_t cap_tiles = s.max_n / kTile + F + 1;
    switch (acc) {
      case Acc::F32:
        e = run_batched_scan<float, float>(s, scheme, static_cast<const float*>(logw), b,
                                           cap_tiles, keys, a, d, st);
        break;
      case Acc::F32C:
        e = run_batched_scan<float, float2>(s, scheme, static_cast<const float*>(logw), b,
                                            cap_tiles, keys, a, d, st);
        break;
      case Acc::F64:
        e = run_batched_scan<double, float2>(s, scheme, static_cast<const double*>(logw), b,
                                             cap_tiles, keys, a, d, st);
        break;
      case Acc::F64N:
        e = run_batched_scan<double, double>(s, scheme, static_cast<const double*>(logw), b,
                                             cap_tiles, keys, a, d, st);
        break;
    }
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess && permute) {
    trace_mark(s.trace, "batch_permute", st);
    const LaunchCfg& c = s.batch_cfg[kCfgPermute];
    launch_pdl(batch_permute_kernel, grid_shaped(total, c), c.block, st, offsets, F, total,
               s.a_tmp, s.d, out, c.ipt, s.err);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace rsk
