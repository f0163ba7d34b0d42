// fused.cu -- the passes of the multinomial, stratified and systematic resamplers of one filter
// (maximum and segment records, segment prefixes, emission) as one persistent cooperative
// kernel.
//
// Each CTA owns a contiguous range of tiles; the CTAs are all resident at once (cooperative
// launch) and meet at grid-wide barriers between the phases (see fused_body). The segment
// prefixes are exact fixed-point sums, so they can be assembled in parallel from per-CTA
// totals instead of by one CTA, and each phase calls the same device functions as the
// separate kernels on the same tiles: the results are identical. The latency-bound
// particle-parallel steps that follow (the multinomial search, Permute) stay separate
// full-occupancy kernels.
// A barrier waits at most the handle's barrier timeout (then it records RS_ERR_TIMEOUT and proceeds;
// every phase stays bounds-checked, so the kernel still ends); the barrier counter returns
// to 0 at the end of every launch.
#include <cfloat>
#include <climits>
#include <type_traits>

#include "common.cuh"
#include "grid.cuh"
#include "internal.h"
#include "tile.cuh"
#include "values.cuh"

namespace rsk {
namespace {

// Block-wide maximum of a key (every thread gets the result).
__device__ __forceinline__ long long block_max_key(long long m, long long* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long y = __shfl_xor_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
  }
  __syncthreads();
  if (lane == 0) sh[warp] = m;
  __syncthreads();
  long long bm = sh[0];
  for (int k = 1; k < kWarps; ++k) bm = sh[k] > bm ? sh[k] : bm;
  return bm;
}

struct FusedArgs {
  int64_t N;
  Keys keys;
  int32_t* a;      // ancestors (systematic / stratified)
  int32_t* d;      // Prepermute claims, or nullptr
  uint8_t* cl;     // claimed bits of the particles (in place of d for the sorted Permute), or nullptr
  void* W;         // multinomial cumulative weights
  int32_t* guide;  // multinomial guide table
  double2* s_rec;  // segment records
  double2* P_rec;  // segment prefixes: exact in-range prefixes (u128), then rounded P_g
  u128* agg;       // per-CTA exact totals (gridDim.x entries)
  ScanGlob* g;
  double* blockmax;  // per-CTA maxima (gridDim.x entries)
  int* err;
};

// CTA c owns the contiguous tiles [c T / G, (c+1) T / G) of the T tiles (G = gridDim.x <= T):
//   phase 1  the records (m_g, s_g) of its tiles' segments (seg_record, each warp its own:
//            the segment's maximum and its weights' sum relative to it), last tile to first,
//            and its largest m_g -> barrier;
//   phase 2  M = maximum over the CTAs; T_g = s_g exp(m_g - M) (rec_scaled) of its segments
//            and their exact running sum in fixed point (the in-range prefix of each segment,
//            and the CTA total) -> barrier;
//            (compensated binary32, whose records must sum the weights exp(lw - M) themselves:
//            phase 1 forms the maximum only and phase 2 the records relative to M, which then
//            scale by exactly 1);
//   phase 3  every CTA sums the exact CTA totals: those before it (CP) and all (the total);
//            P_g = RN(CP + in-range prefix of g) for its segments and P_{g1} = RN(CP + its
//            own total), which is the P_{g1} the next CTA computes; W^N = RN(total), N / W^N;
//   phase 4  emission of its tiles, first to last (it starts on the tiles phase 1 read last,
//            still in L2 when the log-weights exceed half of it), each warp its segments.
// Phases 1 and 4 are warp-level work only: no block barrier per tile. The log-weights are read
// twice (phases 1 and 4; three times for compensated binary32), the least the normaliser
// allows. P_g is the exact sum of the T before g rounded once, as in seg_prefix_compute, so the
// results equal
// those of the separate kernels. Two grid barriers per call.

// kKept: phase 2 takes this thread's first record from a load issued before the first grid
// barrier, and phase 3 its first exact in-range prefix and the CTA total from registers (not
// for the compensated binary32 path, whose records follow the maximum pass, nor for native
// binary64, whose emission runs short of registers with them: both read them back from L2).
template <typename T, typename V>
constexpr bool kKept = Path<T, V>::kTileRef && !std::is_same_v<V, double>;

template <typename T, typename V, int SCHEME>
__device__ __forceinline__ void fused_body(const T* __restrict__ lw, const FusedArgs& A,
                                           unsigned int& target) {
  __shared__ SegSh sh;
  __shared__ float2 sh_tab[64];
  __shared__ long long sh_key[kWarps];
  __shared__ u128 sh_sum[2 * kWarps];
  const int64_t N = A.N;
  const int T_tiles = static_cast<int>((N + kTile - 1) / kTile);
  const int G = static_cast<int>(gridDim.x), c = static_cast<int>(blockIdx.x);
  const int t0 = static_cast<int>(static_cast<int64_t>(c) * T_tiles / G);
  const int t1 = static_cast<int>(static_cast<int64_t>(c + 1) * T_tiles / G);
  const int g0 = kWarps * t0, g1 = kWarps * t1;  // this CTA's segments
  const int warp = threadIdx.x >> 5;
  const int64_t e0 = static_cast<int64_t>(t0) * kTile;
  const int64_t e1 = min(static_cast<int64_t>(t1) * kTile, N);
  const int64_t off = kPer * static_cast<int64_t>(threadIdx.x);  // (= kSeg warp + kPer lane)
  const bool vec = (reinterpret_cast<uintptr_t>(lw) & 15u) == 0;
  if (threadIdx.x < 64) sh_tab[threadIdx.x] = kExp2Frac64[threadIdx.x];
  __syncthreads();

  // ---- phase 1: segment records, last tile to first (and the Prepermute sentinel of the
  // multinomial claims); the next tile's log-weights are loaded while this one is reduced.
  // Without kTileRef, the maximum only (the records follow once M is known) ----------------
  double2 rec0 = make_double2(0.0, 0.0);  // (kKept) the record of segment g0 + threadIdx.x
  {
    long long cm = max_key(neg_inf<T>());
    bool bad = false;
    if constexpr (Path<T, V>::kTileRef) {
      T xn[kPer];
      if (t1 > t0)
        load_per(lw, static_cast<int64_t>(t1 - 1) * kTile + off, 0, N, vec, xn, L2Hint::kEvictLast);
      for (int t = t1 - 1; t >= t0; --t) {
        T x[kPer];
#pragma unroll
        for (int q = 0; q < kPer; ++q) x[q] = xn[q];
        if (t > t0)
          load_per(lw, static_cast<int64_t>(t - 1) * kTile + off, 0, N, vec, xn, L2Hint::kEvictLast);
        const long long k = seg_record<T, V>(x, sh_tab, A.s_rec + kWarps * t + warp, bad);
        cm = k > cm ? k : cm;
      }
    } else {
      float mf = -INFINITY;  // (binary32 inputs)
      for (int t = t0; t < t1; ++t) {
        T x[kPer];
        load_per(lw, static_cast<int64_t>(t) * kTile + off, 0, N, vec, x, L2Hint::kEvictLast);
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
          bad |= !(x[q] <= FLT_MAX);  // NaN or +inf
          mf = fmaxf(mf, static_cast<float>(x[q]));
        }
      }
      cm = max_key(mf);
    }
    if constexpr (SCHEME == RS_MULTINOMIAL) {
      if (A.d) {
        int32_t sv[kPer];
#pragma unroll
        for (int q = 0; q < kPer; ++q) sv[q] = static_cast<int32_t>(N);
        for (int64_t i0 = e0 + off; i0 < e1; i0 += kTile)
          store_per(A.d + i0, sv, e1 - i0 < kPer ? static_cast<int>(e1 - i0) : kPer);
      }
    }
    if (bad) flag_error(A.err, RS_ERR_NONFINITE);
    cm = block_max_key(cm, sh_key);
    if (threadIdx.x == 0) A.blockmax[c] = key_to_double(cm, T());
    // this thread's record for phase 2, loaded before the grid barrier so that the load
    // overlaps the wait (lane 0 of each warp stored the records before block_max_key's
    // block barrier)
    if constexpr (kKept<T, V>) {
      const int g = g0 + static_cast<int>(threadIdx.x);
      if (g < g1) rec0 = __ldcg(A.s_rec + g);
    }
  }
  grid_barrier(&A.g->bar, target, A.err);
  double M;
  {
    long long m = max_key(-static_cast<double>(INFINITY));
    for (int b = threadIdx.x; b < G; b += kBlock) {
      const long long y = max_key(__ldcg(A.blockmax + b));
      m = y > m ? y : m;
    }
    M = key_to_double(block_max_key(m, sh_key), 0.0);
  }
  const bool zero = !(M > -DBL_MAX);
  u128* LP = reinterpret_cast<u128*>(A.P_rec);  // in-range exact prefixes, then rounded P_g

  // ---- phase 2: segment totals relative to M and their exact running sum -------------------
  const WeightCtx wc = make_ctx<T, V>(zero ? 0.0 : M, sh_tab);
  u128 run = 0;  // the running exact total of this CTA's segments (the same in every thread)
  u128 lp0 = 0;  // the exact in-range prefix of segment g0 + threadIdx.x (kept for phase 3)
  if (!zero) {
    const T Mt = static_cast<T>(M);  // (exact: M is one of the log-weights)
    if constexpr (!Path<T, V>::kTileRef) {  // the records, relative to M, last tile to first
      bool bad = false;
      for (int t = t1 - 1; t >= t0; --t)
        seg_record<T, V>(lw, 0, N, static_cast<int64_t>(t) * kTile + kSeg * warp, sh_tab, vec,
                         A.s_rec + kWarps * t + warp, bad, max_key(Mt), L2Hint::kEvictLast);
      __syncthreads();  // (lane 0 of each warp stored them; all threads read them below)
    }
    for (int gb = g0; gb < g1; gb += kBlock) {
      const int g = gb + static_cast<int>(threadIdx.x);
      u128 f = 0;
      if (g < g1) {
        if (kKept<T, V> && gb == g0) f = rec_fixed_of<T, V>(rec0, Mt);
        else f = rec_fixed<T, V>(A.s_rec + g, Mt);
      }
      u128 tot;
      const u128 ex = block_excl_scan_u128(f, sh_sum, tot);
      if (g < g1) st_u128(LP + g, run + ex);
      if (gb == g0) lp0 = ex;
      run += tot;
    }
    if (threadIdx.x == 0) st_u128(A.agg + c, run);
  }
  grid_barrier(&A.g->bar, target, A.err);

  // ---- phase 3: the total and this CTA's segment prefixes ----------------------------------
  if (zero) {  // all weights zero (flagged): every particle keeps itself
    if (c == 0 && threadIdx.x == 0) {
      A.g->S_d = 0.0;
      A.g->M = M;
      A.g->all_zero = 1;
      flag_error(A.err, RS_ERR_ZERO_WEIGHT);
    }
    if constexpr (SCHEME != RS_MULTINOMIAL) {  // (the search kernel writes the identity)
      for (int64_t i = e0 + threadIdx.x; i < e1; i += kBlock) {
        A.a[i] = static_cast<int32_t>(i);
        if (A.d) A.d[i] = static_cast<int32_t>(i);
      }
      if (A.cl)  // every slot claimed (e0 is a multiple of 8)
        for (int64_t b = (e0 >> 3) + threadIdx.x; b < ((e1 + 7) >> 3); b += kBlock) A.cl[b] = 0xFFu;
    }
    return;  // uniform over the grid
  }
  u128 CP = 0, TOT = 0;
  for (int k = threadIdx.x; k < G; k += kBlock) {
    const u128 v = ld_u128_cg(A.agg + k);
    TOT += v;
    if (k < c) CP += v;
  }
  block_sum2_u128(CP, TOT, sh_sum);
  // the total, N / total and the guide step: once per CTA (a binary64 division runs on the
  // 1/57-rate pipe), then shared
  __shared__ double2 sh_S, sh_scale;
  __shared__ double sh_Sd;
  __shared__ Guide sh_gd;
  if (threadIdx.x == 0) {
    const V S0 = fixed_to(TOT, V(), kFixFrac);
    const double Sd0 = vto_double(S0);
    store_v<V>(&sh_S, S0);
    store_v<V>(&sh_scale, vfrom_double(__ddiv_rn(static_cast<double>(N), Sd0), V()));
    sh_Sd = Sd0;
    if constexpr (SCHEME == RS_MULTINOMIAL) sh_gd = make_guide(Sd0, N);
  }
  __syncthreads();
  const V S = load_v<V>(&sh_S), scale = load_v<V>(&sh_scale);
  const double Sd = sh_Sd;
  const bool all_zero = !(Sd > 0.0);
  if (c == 0 && threadIdx.x == 0) {  // read by the search kernel and the host-side callers
    store_v<V>(&A.g->S_raw, S);
    store_v<V>(&A.g->scale_raw, scale);
    A.g->S_d = Sd;
    A.g->M = M;
    A.g->all_zero = all_zero;
    const Guide gd = make_guide(Sd, N);
    A.g->guide_step = gd.step;
    A.g->guide_inv_step = gd.inv_step;
    if (all_zero) flag_error(A.err, RS_ERR_ZERO_WEIGHT);
  }
  // the kernels that follow (search, Permute) may launch now; they wait for this grid's end
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (all_zero) {  // the total rounds to zero: every particle keeps itself
    if constexpr (SCHEME != RS_MULTINOMIAL) {
      for (int64_t i = e0 + threadIdx.x; i < e1; i += kBlock) {
        A.a[i] = static_cast<int32_t>(i);
        if (A.d) A.d[i] = static_cast<int32_t>(i);
      }
      if (A.cl)
        for (int64_t b = (e0 >> 3) + threadIdx.x; b < ((e1 + 7) >> 3); b += kBlock) A.cl[b] = 0xFFu;
    }
    return;
  }
  // rounded prefixes of this CTA's segments, in place of their exact in-range prefixes (each
  // slot is read and then overwritten by the same thread), and of the next CTA's first
  // segment, which that CTA owns: kept in shared memory (the last CTA also writes the total's
  // slot)
  __shared__ double2 sh_pend;
  // (kKept: the exact in-range prefixes of the first kBlock segments and the CTA total are
  // still in registers from phase 2)
  const int gfirst = g0 + static_cast<int>(threadIdx.x);
  for (int g = gfirst; g <= g1; g += kBlock) {
    const u128 lp = (g == g1) ? (kKept<T, V> ? run : ld_u128_cg(A.agg + c))
                              : (kKept<T, V> && g == gfirst) ? lp0 : ld_u128_cg(LP + g);
    const V P = fixed_to(CP + lp, V(), kFixFrac);
    if (g < g1 || c == G - 1) store_v<V>(A.P_rec + g, P);
    if (g == g1) store_v<V>(&sh_pend, P);
  }
  __syncthreads();

  // ---- phase 4: emission of this CTA's tiles, each warp its own segments (no block-level
  // synchronisation) -------------------------------------------------------------------------
  typename Path<T, V>::U u_sys = typename Path<T, V>::U();
  Guide gd;
  if constexpr (SCHEME == RS_MULTINOMIAL) {
    gd = sh_gd;
  } else if constexpr (SCHEME == RS_SYSTEMATIC) {
    u_sys = cta_uniform0<T, V>(A.keys);
  }
  for (int t = t0; t < t1; ++t) {
    const int g = kWarps * t + warp;
    const int64_t base = static_cast<int64_t>(t) * kTile + kSeg * warp;
    const V Ps = load_v_cg<V>(A.P_rec + g);
    const V Pn = (g + 1 < g1) ? load_v_cg<V>(A.P_rec + g + 1) : load_v<V>(&sh_pend);
    if constexpr (SCHEME == RS_MULTINOMIAL) {
      emit_seg_W_guide<T, V>(lw, 0, N, base, wc, vec, Ps, Pn, gd, static_cast<V*>(A.W), A.guide,
                             sh.win[warp], L2Hint::kEvictFirst);
    } else {
      emit_seg_cumoff<T, V, SCHEME == RS_STRATIFIED>(lw, 0, N, base, wc, vec, Ps, Pn, S, scale,
                                                      u_sys, A.keys, A.a, A.d, sh.win[warp], A.cl,
                                                      L2Hint::kEvictFirst);
    }
  }
}

// (at most 64 registers a thread, so that four CTAs of kBlock threads share an SM: the
// cooperative grid is four CTAs per SM)
template <typename T, typename V, int SCHEME>
__global__ void __launch_bounds__(kBlock, 4) fused_scan_kernel(const T* __restrict__ lw, FusedArgs A) {
  unsigned int target = 0;
  fused_body<T, V, SCHEME>(lw, A, target);
  grid_exit(&A.g->bar, target);
}

template <typename T, typename V, int SCHEME>
int fused_capacity() {
  static int cap = -1;  // identical devices assumed
  if (cap < 0) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_scan_kernel<T, V, SCHEME>,
                                                      kBlock, 0) != cudaSuccess)
      return 0;
    cap = per_sm * sms;
  }
  return cap;
}

template <typename T, typename V, int SCHEME>
cudaError_t launch_fused(const Scratch& s, const T* lw, const FusedArgs& A, cudaStream_t st) {
  int64_t grid = fused_capacity<T, V, SCHEME>();
  if (grid > s.max_blocks) grid = s.max_blocks;
  const int64_t tiles = (A.N + kTile - 1) / kTile;
  if (grid > tiles) grid = tiles;
  if (grid < 1) return cudaErrorCooperativeLaunchTooLarge;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(grid));
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fused_scan_kernel<T, V, SCHEME>, lw, A);
}

template <typename T, typename V>
int capacity(int scheme) {
  switch (scheme) {
    case RS_MULTINOMIAL: return fused_capacity<T, V, RS_MULTINOMIAL>();
    case RS_STRATIFIED: return fused_capacity<T, V, RS_STRATIFIED>();
    default: return fused_capacity<T, V, RS_SYSTEMATIC>();
  }
}

template <typename T, typename V>
cudaError_t dispatch(const Scratch& s, int scheme, const T* lw, const FusedArgs& A,
                     cudaStream_t st) {
  switch (scheme) {
    case RS_MULTINOMIAL: return launch_fused<T, V, RS_MULTINOMIAL>(s, lw, A, st);
    case RS_STRATIFIED: return launch_fused<T, V, RS_STRATIFIED>(s, lw, A, st);
    default: return launch_fused<T, V, RS_SYSTEMATIC>(s, lw, A, st);
  }
}

const char* const kLblFused[4][3] = {
    {"fused_multinomial_f32", "fused_stratified_f32", "fused_systematic_f32"},
    {"fused_multinomial_f32c", "fused_stratified_f32c", "fused_systematic_f32c"},
    {"fused_multinomial_f64", "fused_stratified_f64", "fused_systematic_f64"},
    {"fused_multinomial_f64n", "fused_stratified_f64n", "fused_systematic_f64n"}};
}  // namespace

bool fused_available(const Scratch& s, int scheme, Acc acc) {
  if (!s.coop) return false;
  switch (acc) {
    case Acc::F32: return capacity<float, float>(scheme) > 0;
    case Acc::F32C: return capacity<float, float2>(scheme) > 0;
    case Acc::F64: return capacity<double, float2>(scheme) > 0;
    case Acc::F64N: return capacity<double, double>(scheme) > 0;
  }
  return false;
}

cudaError_t launch_fused_passes(const Scratch& s, int scheme, Acc acc, const void* logw,
                                int64_t N, const Keys& keys, int32_t* a_out, int32_t* d,
                                uint8_t* cl, cudaStream_t st) {
  FusedArgs A;
  A.N = N;
  A.keys = keys;
  A.a = a_out;
  A.d = d;
  A.cl = scheme == RS_MULTINOMIAL ? nullptr : cl;
  A.W = s.W;
  A.guide = s.guide;
  A.s_rec = s.rec;
  A.P_rec = s.rec + seg_cap(s.max_tiles);
  A.agg = reinterpret_cast<u128*>(s.irec);  // (max_tiles + 2) entries >= gridDim.x
  A.g = s.glob;
  A.blockmax = s.blockmax;
  A.err = s.err;
  trace_mark(s.trace, kLblFused[static_cast<int>(acc)][scheme], st);
  switch (acc) {
    case Acc::F32:
      return dispatch<float, float>(s, scheme, static_cast<const float*>(logw), A, st);
    case Acc::F32C:
      return dispatch<float, float2>(s, scheme, static_cast<const float*>(logw), A, st);
    case Acc::F64:
      return dispatch<double, float2>(s, scheme, static_cast<const double*>(logw), A, st);
    case Acc::F64N:
      return dispatch<double, double>(s, scheme, static_cast<const double*>(logw), A, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace rsk
