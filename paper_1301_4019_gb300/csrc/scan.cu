// scan.cu -- the multinomial, stratified and systematic resamplers (Appendix B, Codes 5, 7,
// 8, with Code 11 and the Prepermute of Code 10 fused) on sm_103a.
//
// Each call makes three passes over the log-weights (Appendix E renormalisation, Code 4
// primitives):
//   1. max pass      : M = max_i lw_i (last-CTA reduction), NaN/+inf detection.
//   2. tile-sum pass : per tile of kTile particles, its record: the tile's largest log-weight
//                      m_t and the sum of exp(lw_i - m_t) in the accumulator type; the last
//                      CTA to finish scales each record to M (T_t = s_t exp(m_t - M)) and sums
//                      them exactly (128-bit fixed point) into tile prefixes P_t, each rounded
//                      once, and the total W^N. (The records need no M, so the fused kernel
//                      forms them in its first pass together with M.)
//   3. emit pass     : the same tile scan is recomputed bit for bit, offset by P_t, and
//                      turned into cumulative offspring O_i (systematic / stratified) with a
//                      direct Code-11 scatter of the ancestors and, for Permute, the claimed
//                      bit of every particle (its Prepermute claim is the first position of
//                      its run); or into stored cumulative weights W_i (multinomial, followed
//                      by the search kernel).
// Reading the weights twice is inherent: the normaliser W^N is needed before any O_i. The
// reduce-then-scan order needs no inter-CTA waiting at all.
//
// Monotonicity: floating-point tree sums are not monotone in general, so the tile values are
// raised to a running maximum and clamped into bounds that are non-decreasing across warps
// and tiles (tile_cum_weights); every global cumulative weight lies in [P_t, P_{t+1}] with P
// monotone. Cumulative weights are therefore non-decreasing, the cumulative offspring too,
// and Code 11 writes every position of the ancestry vector exactly once.
//
// Accumulators (input type T, accumulator V): binary32 (float, float), two-float
// (float, float2), double-float for binary64 inputs on the binary32 pipes (double, float2:
// weights by exp_df, GB300 runs binary64 at 1/57 rate), native binary64 (double, double).
#include <cfloat>
#include <climits>

#include "common.cuh"
#include "dfexp.cuh"
#include "internal.h"
#include "tile.cuh"
#include "values.cuh"

namespace rsk {
namespace {

// ---------------------------------------------------------------------------------------
// Pass 1: maximum log-weight, compared through order-preserving integer keys (exact, and
// no binary64 arithmetic). NaN is skipped (and flagged, as is +inf).
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kBlock)
max_kernel(const T* __restrict__ lw, int64_t N, ScanGlob* g, double* blockmax, int* err,
           int32_t* d_init) {
  pdl_wait();
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
    load4(lw, i0, 0, N, vec && i0 + 4 <= N, x);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool nan = is_nan(x[q]);
      bad |= nan || is_pos_inf(x[q]);
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
// Pass 2: segment records (each warp its own) and, in the last CTA, the segment prefixes.
// ---------------------------------------------------------------------------------------
// The last CTA's work, kept out of line so that its registers do not limit the occupancy of
// the tile work.
template <typename T, typename V>
__device__ __noinline__ void seg_prefix_last_cta(const double2* s_rec, double2* P_rec, int nseg,
                                                 int64_t N, ScanGlob* g, int* err,
                                                 double* log_total_out) {
  seg_prefix_compute<T, V>(s_rec, P_rec, nseg, N, static_cast<T>(g->M),
                           reinterpret_cast<V*>(&g->S_raw), reinterpret_cast<V*>(&g->scale_raw),
                           &g->S_d);
  if (threadIdx.x == 0) {
    const double Sd = g->S_d;
    if (!(Sd > 0.0)) flag_error(err, RS_ERR_ZERO_WEIGHT);
    if (log_total_out) *log_total_out = __dadd_rn(g->M, log(Sd));
    g->all_zero = !(g->M > -DBL_MAX) || !(Sd > 0.0);
    const Guide gd = make_guide(Sd, N);
    g->guide_step = gd.step;
    g->guide_inv_step = gd.inv_step;
    g->ticket_tile = 0u;
  }
}

template <typename T, typename V>
__global__ void __launch_bounds__(kBlock, 4)
tile_sum_kernel(const T* __restrict__ lw, int64_t N, ScanGlob* g, double2* s_rec,
                double2* P_rec, int* err, double* log_total_out) {
  pdl_wait();
  __shared__ float2 sh_tab[64];
  __shared__ bool am_last;
  const int warp = threadIdx.x >> 5;
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile + kSeg * warp;
  if (threadIdx.x < 64) sh_tab[threadIdx.x] = kExp2Frac64[threadIdx.x];
  __syncthreads();
  const bool vec = (reinterpret_cast<uintptr_t>(lw) & 15u) == 0;
  bool bad = false;  // (the max pass flags non-finite input)
  long long ref = kTileMaxRef;
  if constexpr (!Path<T, V>::kTileRef) {
    const double Md = g->M;
    if (Md > -DBL_MAX) ref = max_key(static_cast<T>(Md));  // (records relative to M)
  }
  seg_record<T, V>(lw, 0, N, base, sh_tab, vec, s_rec + kWarps * blockIdx.x + warp, bad, ref);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(&g->ticket_tile, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  seg_prefix_last_cta<T, V>(s_rec, P_rec, kWarps * static_cast<int>(gridDim.x), N, g, err,
                            log_total_out);
}

// ---------------------------------------------------------------------------------------
// Pass 3a: systematic / stratified emission, one tile per CTA, one segment per warp.
// ---------------------------------------------------------------------------------------
template <typename T, typename V, bool STRAT>
__global__ void __launch_bounds__(kBlock)
emit_cumoff_kernel(const T* __restrict__ lw, int64_t N, const ScanGlob* g, const double2* s_rec,
                   const double2* P_rec, Keys keys, int32_t* __restrict__ a,
                   int32_t* __restrict__ d, uint8_t* __restrict__ cl) {
  pdl_wait();
  __shared__ SegSh sh;
  __shared__ float2 sh_tab[64];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile;
  if (g->all_zero) {  // all weights zero: flagged; emit identity (every slot claimed)
    const int64_t end = N < base + kTile ? N : base + kTile;
    for (int64_t i = base + threadIdx.x; i < end; i += kBlock) {
      a[i] = static_cast<int32_t>(i);
      if (d) d[i] = static_cast<int32_t>(i);
    }
    if (cl)  // (base is a multiple of 8)
      for (int64_t b = (base >> 3) + threadIdx.x; b < ((end + 7) >> 3); b += kBlock) cl[b] = 0xFFu;
    return;
  }
  const WeightCtx wc = make_ctx<T, V>(g->M, sh_tab);
  const typename Path<T, V>::U u_sys = STRAT ? typename Path<T, V>::U() : cta_uniform0<T, V>(keys);
  const bool vec = (reinterpret_cast<uintptr_t>(lw) & 15u) == 0;
  const int warp = threadIdx.x >> 5;
  const int64_t sg = static_cast<int64_t>(kWarps) * blockIdx.x + warp;
  emit_seg_cumoff<T, V, STRAT>(lw, 0, N, base + kSeg * warp, wc, vec, load_v<V>(P_rec + sg),
                               load_v<V>(P_rec + sg + 1), load_v<V>(&g->S_raw),
                               load_v<V>(&g->scale_raw), u_sys, keys, a, d, sh.win[warp], cl);
}

// ---------------------------------------------------------------------------------------
// Pass 3b: stored cumulative weights (multinomial search input, or rs_cumulative_weights
// output converted to the element type), one tile per CTA, one segment per warp.
// ---------------------------------------------------------------------------------------
template <typename T, typename V, typename OUT>
__global__ void __launch_bounds__(kBlock)
emit_W_kernel(const T* __restrict__ lw, int64_t N, const ScanGlob* g, const double2* P_rec,
              OUT* __restrict__ Wout) {
  pdl_wait();
  __shared__ float2 sh_tab[64];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile;
  if (g->all_zero) {
    for (int64_t i = base + threadIdx.x; i < N && i < base + kTile; i += kBlock)
      Wout[i] = convert_out<V, OUT>(vzero(V()));
    return;
  }
  const WeightCtx wc = make_ctx<T, V>(g->M, sh_tab);
  const bool vec = (reinterpret_cast<uintptr_t>(lw) & 15u) == 0;
  const int warp = threadIdx.x >> 5;
  const int64_t sg = static_cast<int64_t>(kWarps) * blockIdx.x + warp;
  emit_seg_W<T, V, OUT>(lw, 0, N, base + kSeg * warp, wc, vec, load_v<V>(P_rec + sg),
                        load_v<V>(P_rec + sg + 1), Wout);
}

// Pass 3b for the multinomial scheme: stored cumulative weights plus the guide table.
template <typename T, typename V>
__global__ void __launch_bounds__(kBlock)
emit_W_guide_kernel(const T* __restrict__ lw, int64_t N, const ScanGlob* g, const double2* s_rec,
                    const double2* P_rec, V* __restrict__ Wout, int32_t* __restrict__ G) {
  pdl_wait();
  __shared__ SegSh sh;
  __shared__ float2 sh_tab[64];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile;
  if (g->all_zero) return;  // the search writes the identity
  const WeightCtx wc = make_ctx<T, V>(g->M, sh_tab);
  const bool vec = (reinterpret_cast<uintptr_t>(lw) & 15u) == 0;
  const int warp = threadIdx.x >> 5;
  const int64_t sg = static_cast<int64_t>(kWarps) * blockIdx.x + warp;
  emit_seg_W_guide<T, V>(lw, 0, N, base + kSeg * warp, wc, vec, load_v<V>(P_rec + sg),
                         load_v<V>(P_rec + sg + 1), Guide{g->guide_step, g->guide_inv_step},
                         Wout, G, sh.win[warp]);
}

// ---------------------------------------------------------------------------------------
// Multinomial search (Code 5), one particle per thread, with the Prepermute claim
// atomicMin(d[a_i], i) when d is given.
// ---------------------------------------------------------------------------------------
template <typename T, typename V>
__global__ void __launch_bounds__(kBlock)
search_kernel(const V* __restrict__ W, const int32_t* __restrict__ G, int64_t N,
              const ScanGlob* g, Keys keys, int32_t* __restrict__ a, int32_t* __restrict__ d) {
  pdl_wait();
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (g->all_zero) {
    a[i] = static_cast<int32_t>(i);
    if (d) atomicMin(d + i, static_cast<int32_t>(i));
    return;
  }
  const Guide gd{g->guide_step, g->guide_inv_step};
  const int32_t k = search_one_guided<T, V>(W, G, N, gd, keys, i);
  a[i] = k;
  if (d) atomicMin(d + k, static_cast<int32_t>(i));
}

// The same search, four consecutive outputs per thread (their loads in flight together) and
// one 128-bit store of the four ancestors; used from kSearch4MinN particles, where W and the
// guide table leave L2 (measured at 2^24: 577 vs 656 us binary32, 668 vs 754 us double-float;
// at 2^20-2^22, with the tables in L2, one output per thread keeps more loads in flight:
// 21 vs 27 us at 2^20).
template <typename T, typename V>
__global__ void __launch_bounds__(kBlock)
search4_kernel(const V* __restrict__ W, const int32_t* __restrict__ G, int64_t N,
               const ScanGlob* g, Keys keys, int32_t* __restrict__ a, int32_t* __restrict__ d) {
  pdl_wait();
  const int64_t i0 = 4 * (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x);
  if (i0 >= N) return;
  int32_t k[4];
  if (g->all_zero) {
#pragma unroll
    for (int q = 0; q < 4; ++q) k[q] = static_cast<int32_t>(i0 + q);
  } else {
    const Guide gd{g->guide_step, g->guide_inv_step};
    search_group_guided<T, V, 4>(W, G, N, gd, keys, i0, k);
  }
  if (i0 + 3 < N && (reinterpret_cast<uintptr_t>(a + i0) & 15u) == 0) {
    *reinterpret_cast<int4*>(a + i0) = make_int4(k[0], k[1], k[2], k[3]);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (i0 + q < N) a[i0 + q] = k[q];
  }
  if (d) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (i0 + q < N) atomicMin(d + k[q], static_cast<int32_t>(i0 + q));
  }
}
constexpr int64_t kSearch4MinN = int64_t{1} << 23;

template <typename T, typename V>
void launch_search(const Scratch& s, const V* W, int64_t N, const Keys& keys, int32_t* a,
                   int32_t* d, cudaStream_t st) {
  if (N >= kSearch4MinN)
    launch_pdl(search4_kernel<T, V>, static_cast<int>((N + 4 * kBlock - 1) / (4 * kBlock)),
               kBlock, st, W, s.guide, N, s.glob, keys, a, d);
  else
    launch_pdl(search_kernel<T, V>, static_cast<int>((N + kBlock - 1) / kBlock), kBlock, st, W,
               s.guide, N, s.glob, keys, a, d);
}

int max_grid(int64_t N, int max_blocks) {
  const int64_t want = (N + 4 * kBlock - 1) / (4 * kBlock);  // one 1024-element slice per CTA
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
cudaError_t run_scan(const Scratch& s, int scheme, Acc acc, const T* lw, int64_t N,
                     uint64_t seed, uint64_t step, uint32_t filter, int32_t* a_out, int32_t* d,
                     bool fused, cudaStream_t st, uint8_t* cl) {
  const int tiles = static_cast<int>((N + kTile - 1) / kTile);
  double2* s_rec = s.rec;
  double2* P_rec = s.rec + seg_cap(s.max_tiles);
  const Keys keys = make_keys(seed, step, filter, static_cast<uint32_t>(scheme));
  constexpr int ai = Path<T, V>::id;
  if (fused) {
    cudaError_t e = launch_fused_passes(s, scheme, acc, lw, N, keys, a_out, d, cl, st);
    if (e != cudaSuccess || scheme != RS_MULTINOMIAL) return e;
    trace_mark(s.trace, kLblSearch[ai], st);
    launch_search<T, V>(s, static_cast<const V*>(s.W), N, keys, a_out, d, st);
    return cudaGetLastError();
  }
  trace_mark(s.trace, kLblMax[ai], st);
  launch_pdl(max_kernel<T>, max_grid(N, s.max_blocks), kBlock, st,
      lw, N, s.glob, s.blockmax, s.err, scheme == RS_MULTINOMIAL ? d : nullptr);
  trace_mark(s.trace, kLblTile[ai], st);
  launch_pdl(tile_sum_kernel<T, V>, tiles, kBlock, st, lw, N, s.glob, s_rec, P_rec, s.err, nullptr);
  if (scheme == RS_SYSTEMATIC) {
    trace_mark(s.trace, kLblSys[ai], st);
    launch_pdl(emit_cumoff_kernel<T, V, false>, tiles, kBlock, st, lw, N, s.glob, s_rec, P_rec, keys,
               a_out, d, cl);
  } else if (scheme == RS_STRATIFIED) {
    trace_mark(s.trace, kLblStr[ai], st);
    launch_pdl(emit_cumoff_kernel<T, V, true>, tiles, kBlock, st, lw, N, s.glob, s_rec, P_rec, keys,
               a_out, d, cl);
  } else {
    V* W = static_cast<V*>(s.W);
    trace_mark(s.trace, kLblW[ai], st);
    launch_pdl(emit_W_guide_kernel<T, V>, tiles, kBlock, st, lw, N, s.glob, s_rec, P_rec, W, s.guide);
    trace_mark(s.trace, kLblSearch[ai], st);
    launch_search<T, V>(s, W, N, keys, a_out, d, st);
  }
  return cudaGetLastError();
}

template <typename T, typename V, typename OUT>
cudaError_t run_cumw(const Scratch& s, const T* lw, int64_t N, OUT* W_out, double* log_total,
                     cudaStream_t st) {
  const int tiles = static_cast<int>((N + kTile - 1) / kTile);
  double2* s_rec = s.rec;
  double2* P_rec = s.rec + seg_cap(s.max_tiles);
  constexpr int ai = Path<T, V>::id;
  trace_mark(s.trace, kLblMax[ai], st);
  launch_pdl(max_kernel<T>, max_grid(N, s.max_blocks), kBlock, st, lw, N, s.glob, s.blockmax, s.err,
                                                              nullptr);
  trace_mark(s.trace, kLblTile[ai], st);
  launch_pdl(tile_sum_kernel<T, V>, tiles, kBlock, st, lw, N, s.glob, s_rec, P_rec, s.err,
                                                  log_total);
  trace_mark(s.trace, kLblW[ai], st);
  launch_pdl(emit_W_kernel<T, V, OUT>, tiles, kBlock, st, lw, N, s.glob, P_rec, W_out);
  return cudaGetLastError();
}

// Self-check of exp_scan_f32 (rs_check_weight_exp): the binary32 values t with bit patterns
// first + k (k < count, all t <= 0), against the binary64 pinned exponential of t (within
// about 2^-52 of exp): for t >= -87 a relative error above `bound` counts, and the largest
// relative error is kept (non-negative binary64 values order like their bit patterns, so an
// integer maximum of the patterns is the maximum); below -87 a result outside [0, 2^-125]
// counts.
__global__ void __launch_bounds__(kBlock)
check_scan_exp_kernel(uint32_t first, uint32_t count, double bound, unsigned long long* bad_out,
                      unsigned long long* maxrel_bits) {
  unsigned long long bad = 0;
  double mx = 0.0;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += stride) {
    const float t = __uint_as_float(first + k);
    const float y = exp_scan_f32(t);
    if (t >= -87.0f) {
      const double e = exp_pinned(static_cast<double>(t));
      const double rel = __ddiv_rn(fabs(__dsub_rn(static_cast<double>(y), e)), e);
      if (!(rel <= bound)) ++bad;
      if (rel > mx) mx = rel;
    } else if (!(y >= 0.0f && y <= 0x1p-125f)) {
      ++bad;
    }
  }
  unsigned long long mb = static_cast<unsigned long long>(__double_as_longlong(mx));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, mb, o);
    mb = y > mb ? y : mb;
  }
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicAdd(bad_out, bad);
    atomicMax(maxrel_bits, mb);
  }
}

}  // namespace

cudaError_t launch_check_weight_exp(double bound, unsigned long long* count, double* max_rel,
                                    cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(max_rel, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    sms = 1;
  // every binary32 t <= 0: -0 (0x80000000) through -inf (0xff800000)
  const uint32_t first = 0x80000000u, last = 0xff800000u;
  check_scan_exp_kernel<<<sms * 8, kBlock, 0, st>>>(
      first, last - first + 1, bound, count, reinterpret_cast<unsigned long long*>(max_rel));
  return cudaGetLastError();
}

cudaError_t launch_scan_resample(const Scratch& s, int scheme, Acc acc, const void* logw,
                                 int64_t N, uint64_t seed, uint64_t step, uint32_t filter,
                                 int32_t* a_out, int32_t* d, bool fused, cudaStream_t st,
                                 uint8_t* cl) {
  switch (acc) {
    case Acc::F32:
      return run_scan<float, float>(s, scheme, acc, static_cast<const float*>(logw), N, seed,
                                    step, filter, a_out, d, fused, st, cl);
    case Acc::F32C:
      return run_scan<float, float2>(s, scheme, acc, static_cast<const float*>(logw), N, seed,
                                     step, filter, a_out, d, fused, st, cl);
    case Acc::F64:
      return run_scan<double, float2>(s, scheme, acc, static_cast<const double*>(logw), N, seed,
                                      step, filter, a_out, d, fused, st, cl);
    case Acc::F64N:
      return run_scan<double, double>(s, scheme, acc, static_cast<const double*>(logw), N, seed,
                                      step, filter, a_out, d, fused, st, cl);
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

// The same cumulative weights, every accumulator written out in binary64 (exactly: a
// binary32 value, or a two-float / double-float pair whose halves are at most 29 bits apart).
cudaError_t launch_cumulative_weights_f64(const Scratch& s, Acc acc, const void* logw, int64_t N,
                                          double* W_out, double* log_total, cudaStream_t st) {
  switch (acc) {
    case Acc::F32:
      return run_cumw<float, float, double>(s, static_cast<const float*>(logw), N, W_out,
                                            log_total, st);
    case Acc::F32C:
      return run_cumw<float, float2, double>(s, static_cast<const float*>(logw), N, W_out,
                                             log_total, st);
    case Acc::F64:
      return run_cumw<double, float2, double>(s, static_cast<const double*>(logw), N, W_out,
                                              log_total, st);
    case Acc::F64N:
      return run_cumw<double, double, double>(s, static_cast<const double*>(logw), N, W_out,
                                              log_total, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace rsk
