// aux.cu -- ancestry permutation (Appendix C, Code 10) and the auxiliary conversions of
// Appendix D (Codes 11 and 12, Inclusive-Prefix-Sum and Adjacent-Difference of Code 4) on
// sm_103a. Integer work only: every result is exact.
#include "common.cuh"
#include "grid.cuh"
#include "internal.h"
#include "permute.cuh"
#include "tile.cuh"

namespace rsk {
namespace {

// p[0..N) = v with 128-bit stores where p is 16-byte aligned.
__global__ void __launch_bounds__(kBlock) fill_kernel(int32_t* __restrict__ p, int64_t N, int32_t v) {
  pdl_wait();
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t t0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t head = ((16 - (reinterpret_cast<uintptr_t>(p) & 15u)) & 15u) / 4;  // to alignment
  const int64_t h = head < N ? head : N;
  for (int64_t i = t0; i < h; i += stride) p[i] = v;
  int4* q = reinterpret_cast<int4*>(p + h);
  const int64_t nv = (N - h) / 4;
  const int4 vv = make_int4(v, v, v, v);
  for (int64_t i = t0; i < nv; i += stride) q[i] = vv;
  for (int64_t i = h + 4 * nv + t0; i < N; i += stride) p[i] = v;
}

// Prepermute: d[a_i] = min(d[a_i], i) (d initialised to the sentinel N beforehand).
__global__ void __launch_bounds__(kBlock)
prepermute_kernel(const int32_t* __restrict__ a, int64_t N, int32_t* __restrict__ d, int* err) {
  pdl_wait();
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int32_t ai = a[i];
  if (ai < 0 || ai >= N) {
    flag_error(err, RS_ERR_ARG);
    return;
  }
  atomicMin(d + ai, static_cast<int32_t>(i));
}

// Permute (second procedure of Code 10), one slot per thread (permute.cuh).
__global__ void __launch_bounds__(kBlock)
permute_kernel(const int32_t* __restrict__ a, const int32_t* __restrict__ d, int64_t N,
               int32_t* __restrict__ c, int* err) {
  pdl_wait();
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  permute_one(a, d, N, c, i, err);
}

// Permute of a non-decreasing ancestry from a and the claimed bits of its emission (cl: bit
// i % 8 of cl[i / 8] set when particle i has offspring), K consecutive slots per thread. For
// such an ancestry the claims of Prepermute are d_j = the first position of the run of j for
// every claimed j, so Code 10's walks can be followed from their ends instead of their starts:
//  - a claimed slot x keeps its particle: c_x = x;
//  - an unclaimed slot x that is not the first of its run (a_{x-1} = a_x) is a failed claim
//    whose walk ends at once, at x: c_x = a_x;
//  - an unclaimed slot x that is the first of its run was reached from z = a_x (d_z = x);
//    while z is itself the first of its run (z = 0 or a_{z-1} != a_z) it was reached from
//    a_z in turn, and the first z that is not is the walk's start: c_x = a_z.
// d is injective on the claimed slots and the walks end (Appendix C), so each backward chain
// is one walk reversed and c is Code 10's exactly; the claims are never stored. The chains
// that go on past their first step are queued per warp and run one per lane (as walk_queue).
template <int K>
__global__ void __launch_bounds__(kBlock)
permute_sorted_bits_kernel(const int32_t* __restrict__ a, const uint8_t* __restrict__ cl,
                           int64_t N, int32_t* __restrict__ c, int* err) {
  static_assert(K == 1 || K == 4, "one or four slots per thread");
  pdl_wait();
  const int64_t i0 = K * (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x);
  // (no early exit: the chains are finished warp-wide; threads past N have no slots)
  const int lane = threadIdx.x & 31;
  const bool full = i0 + K <= N;
  int32_t A[K];
  if (K == 4 && full && (reinterpret_cast<uintptr_t>(a) & 15u) == 0) {
    const int4 va = *reinterpret_cast<const int4*>(a + i0);
    A[0] = va.x; A[1] = va.y; A[2] = va.z; A[3] = va.w;
  } else {
#pragma unroll
    for (int q = 0; q < K; ++q) A[q] = i0 + q < N ? a[i0 + q] : 0;
  }
  // a_{i0-1}: the previous lane's last slot, loaded by lane 0 only
  int32_t prev = __shfl_up_sync(0xffffffffu, A[K - 1], 1);
  if (lane == 0) prev = (i0 > 0 && i0 - 1 < N) ? a[i0 - 1] : -1;
  const uint32_t bits = i0 < N ? static_cast<uint32_t>(cl[i0 >> 3]) >> (i0 & 7) : 0u;
  // the warp's K * 32 consecutive results are gathered here and stored 128 bits at a time
  __shared__ alignas(16) int32_t cbuf[kBlock / 32][32 * K];
  __shared__ int2 pend[kBlock / 32][32 * K];
  int32_t* const cw = cbuf[threadIdx.x >> 5];
  int2* const pq = pend[threadIdx.x >> 5];
  const unsigned below = (1u << lane) - 1u;
  int total = 0;
  bool bad = false;
  int32_t R[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const int64_t x = i0 + q;
    bool go = false;
    R[q] = 0;
    const int32_t ax = A[q];
    if (x < N) {
      if (ax < 0 || ax >= N) bad = true;
      else if ((bits >> q) & 1u) R[q] = static_cast<int32_t>(x);
      else if (prev == ax) R[q] = ax;  // not the first of its run
      else go = true;
      prev = ax;
    }
    const unsigned m = __ballot_sync(0xffffffffu, go);
    if (go) pq[total + __popc(m & below)] = make_int2(K * lane + q, ax);
    total += __popc(m);
  }
  if (K == 4) {
    reinterpret_cast<int4*>(cw)[lane] = make_int4(R[0], R[1], R[2], R[3]);
  } else {
    cw[lane] = R[0];
  }
  __syncwarp();
  const uint32_t un = static_cast<uint32_t>(N);
  for (int e = lane; e < total; e += 32) {
    const int2 w = pq[e];
    int32_t z = w.y;
    for (int64_t steps = 0;; ++steps) {
      const int32_t y = a[z];
      const bool zhead = z == 0 || a[z - 1] != y;
      if (static_cast<uint32_t>(y) >= un || steps > N) {  // only a corrupted a can get here
        bad = true;
        break;
      }
      if (!zhead) {
        cw[w.x] = y;
        break;
      }
      z = y;
    }
  }
  __syncwarp();
  if (K == 4 && full && (reinterpret_cast<uintptr_t>(c) & 15u) == 0) {
    *reinterpret_cast<int4*>(c + i0) = reinterpret_cast<const int4*>(cw)[lane];
  } else {
#pragma unroll
    for (int q = 0; q < K; ++q)
      if (i0 + q < N) c[i0 + q] = cw[K * lane + q];
  }
  if (bad) flag_error(err, RS_ERR_ARG);
}

// Permute of any ancestry (permute_one) with four consecutive slots per thread: 128-bit slot
// loads, the four claim checks d[a_i] issued together, and the walks of failed claims run
// together (walk_queue). Same reads and writes per slot as permute_one, so c is the same.
__global__ void __launch_bounds__(kBlock)
permute4_kernel(const int32_t* __restrict__ a, const int32_t* __restrict__ d, int64_t N,
                int32_t* __restrict__ c, int* err) {
  pdl_wait();
  const int64_t i0 = 4 * (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x);
  // (no early exit: the walks are finished warp-wide; threads past N have no slots)
  const int32_t sentinel = static_cast<int32_t>(N);
  int32_t A[4], D[4];
  const bool vec = i0 + 3 < N &&
                   ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(d)) & 15u) == 0;
  if (vec) {
    const int4 va = *reinterpret_cast<const int4*>(a + i0);
    const int4 vd = *reinterpret_cast<const int4*>(d + i0);
    A[0] = va.x; A[1] = va.y; A[2] = va.z; A[3] = va.w;
    D[0] = vd.x; D[1] = vd.y; D[2] = vd.z; D[3] = vd.w;
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      A[q] = i0 + q < N ? a[i0 + q] : 0;
      D[q] = i0 + q < N ? d[i0 + q] : sentinel;
    }
  }
  bool ok[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    ok[q] = i0 + q < N;
    if (ok[q] && (A[q] < 0 || A[q] >= N)) {
      flag_error(err, RS_ERR_ARG);
      ok[q] = false;
    }
  }
  int32_t claim[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) claim[q] = ok[q] ? d[A[q]] : static_cast<int32_t>(i0 + q);
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (ok[q] && D[q] != sentinel) c[i0 + q] = static_cast<int32_t>(i0 + q);
  bool fail[4];
  int32_t x[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    fail[q] = ok[q] && claim[q] != static_cast<int32_t>(i0 + q);
    x[q] = static_cast<int32_t>(i0 + q);
  }
  __shared__ int2 pend[kBlock / 32][128];
  walk_queue<4>(ClaimsOf{d}, sentinel, c, x, D, A, fail, N, pend[threadIdx.x >> 5], err);
}

// Ancestors-to-Offspring (Code 12).
__global__ void __launch_bounds__(kBlock)
offspring_kernel(const int32_t* __restrict__ a, int64_t N, int32_t* __restrict__ o, int* err) {
  pdl_wait();
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int32_t ai = a[i];
  if (ai < 0 || ai >= N) {
    flag_error(err, RS_ERR_ARG);
    return;
  }
  atomicAdd(o + ai, 1);
}

// Adjacent-Difference: o_i = O_i - O_{i-1} (o_0 = O_0), four consecutive positions per thread
// (128-bit loads and stores when inside and aligned; O_{i0-1} from the previous lane).
__global__ void __launch_bounds__(kBlock)
adjacent_difference_kernel(const int32_t* __restrict__ O, int64_t N, int32_t* __restrict__ o) {
  pdl_wait();
  const int64_t i0 = 4 * (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x);
  const bool vec = i0 + 4 <= N &&
                   ((reinterpret_cast<uintptr_t>(O) | reinterpret_cast<uintptr_t>(o)) & 15u) == 0;
  int32_t x[4];
  if (vec) {
    const int4 u = __ldg(reinterpret_cast<const int4*>(O + i0));
    x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w;
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) x[q] = i0 + q < N ? O[i0 + q] : 0;
  }
  int32_t prev = __shfl_up_sync(0xffffffffu, x[3], 1);
  if ((threadIdx.x & 31) == 0) prev = (i0 > 0 && i0 - 1 < N) ? O[i0 - 1] : 0;
  if (i0 >= N) return;  // (after the shuffle: the whole warp takes part in it)
  const int32_t y[4] = {x[0] - prev, x[1] - x[0], x[2] - x[1], x[3] - x[2]};
  if (vec) {
    *reinterpret_cast<int4*>(o + i0) = make_int4(y[0], y[1], y[2], y[3]);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (i0 + q < N) o[i0 + q] = y[q];
  }
}

// Cumulative-Offspring-to-Ancestors (Code 11): particle i fills a[O_{i-1} .. O_i - 1]. One
// warp per kSeg particles (kPer consecutive per lane): the counts are checked as Code 11
// needs them (RS_ERR_ARG for a count below the one before it or outside [0, n], or a last
// count other than n; such counts are clamped, so that every write stays inside a), then
// warp_runs writes the warp's positions [O_{j0-1}, O_{j0+kSeg-1}) through its shared window
// with coalesced stores. For valid counts the writes are exactly Code 11's.
__global__ void __launch_bounds__(kBlock)
cumoff_to_ancestors_kernel(const int32_t* __restrict__ O, int64_t N, int32_t* __restrict__ a,
                           int* err) {
  pdl_wait();
  __shared__ alignas(16) int32_t win[kWarps][kRunWin];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t j0l = (static_cast<int64_t>(blockIdx.x) * kWarps + warp) * kSeg;
  if (j0l >= N) return;  // (warp-uniform: only warp-level synchronisation below)
  const int32_t n = static_cast<int32_t>(N);
  const int32_t j0 = static_cast<int32_t>(j0l);
  const int32_t i0 = j0 + kPer * lane;
  int32_t Oe[kPer];
  if (i0 + kPer <= n && (reinterpret_cast<uintptr_t>(O) & 15u) == 0) {
    const int4 u0 = __ldg(reinterpret_cast<const int4*>(O + i0));
    const int4 u1 = __ldg(reinterpret_cast<const int4*>(O + i0 + 4));
    Oe[0] = u0.x; Oe[1] = u0.y; Oe[2] = u0.z; Oe[3] = u0.w;
    Oe[4] = u1.x; Oe[5] = u1.y; Oe[6] = u1.z; Oe[7] = u1.w;
  } else {
#pragma unroll
    for (int q = 0; q < kPer; ++q) Oe[q] = i0 + q < n ? __ldg(O + i0 + q) : n;
  }
  int32_t prev = __shfl_up_sync(0xffffffffu, Oe[kPer - 1], 1);
  if (lane == 0) prev = j0 > 0 ? __ldg(O + j0 - 1) : 0;
  bool bad = false;
  {
    int32_t p = prev;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      if (i0 + q < n)
        bad |= p < 0 || Oe[q] < p || Oe[q] > n || (i0 + q == n - 1 && Oe[q] != n);
      p = Oe[q];
    }
    // clamped into [0, n] and made non-decreasing within the lane, then across the warp
    prev = min(max(prev, 0), n);
    p = prev;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      Oe[q] = min(max(Oe[q], p), n);
      p = Oe[q];
    }
    int32_t m = Oe[kPer - 1];
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, m, dd);
      if (lane >= dd) m = max(m, y);
    }
    const int32_t before = __shfl_up_sync(0xffffffffu, m, 1);
    if (lane > 0 && before > prev) {
      prev = before;
#pragma unroll
      for (int q = 0; q < kPer; ++q) Oe[q] = max(Oe[q], before);
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) flag_error(err, RS_ERR_ARG);
  warp_runs(Oe, prev, i0, a, win[warp]);
}

// Integer inclusive prefix sum, reduce-then-scan over tiles of 4096 (exact in int64):
// pass 1 writes tile totals and the last CTA scans them; pass 2 scans each tile again and
// adds its prefix.
constexpr int kIscanTile = 16 * kBlock;  // elements per CTA of the integer scan

__device__ __forceinline__ long long block_tile_scan(const int32_t* __restrict__ in, int64_t N,
                                                     int64_t base, long long (&v)[16],
                                                     long long* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // thread t owns the 16 consecutive elements base + 16 t .. base + 16 t + 15
  long long run = 0;
  const int64_t idx = base + 16 * threadIdx.x;
  int32_t x[16];
  if (idx + 16 <= N && (reinterpret_cast<uintptr_t>(in) & 15u) == 0) {  // four 128-bit loads
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int4 u = __ldg(reinterpret_cast<const int4*>(in + idx) + h);
      x[4 * h] = u.x; x[4 * h + 1] = u.y; x[4 * h + 2] = u.z; x[4 * h + 3] = u.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q) x[q] = (idx + q < N) ? in[idx + q] : 0;
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    run += x[q];
    v[q] = run;
  }
  long long incl = run;
#pragma unroll
  for (int dd = 1; dd < 32; dd <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, incl, dd);
    if (lane >= dd) incl += y;
  }
  if (lane == 31) sh[warp] = incl;
  __syncthreads();
  long long pw = 0;
  for (int k = 0; k < warp; ++k) pw += sh[k];
  const long long excl = pw + incl - run;
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] += excl;
  long long total = 0;
  for (int k = 0; k < kWarps; ++k) total += sh[k];
  return total;
}

// out[idx + q] = v[q] + p for the 16 consecutive positions idx .. idx + 15 inside [0, N)
// (four 128-bit stores when all are inside and aligned).
__device__ __forceinline__ void store16(int32_t* __restrict__ out, int64_t idx, int64_t N,
                                        const long long (&v)[16], long long p) {
  if (idx + 16 <= N && (reinterpret_cast<uintptr_t>(out) & 15u) == 0) {
#pragma unroll
    for (int h = 0; h < 4; ++h)
      reinterpret_cast<int4*>(out + idx)[h] = make_int4(
          static_cast<int32_t>(v[4 * h] + p), static_cast<int32_t>(v[4 * h + 1] + p),
          static_cast<int32_t>(v[4 * h + 2] + p), static_cast<int32_t>(v[4 * h + 3] + p));
  } else {
#pragma unroll
    for (int q = 0; q < 16; ++q)
      if (idx + q < N) out[idx + q] = static_cast<int32_t>(v[q] + p);
  }
}

__global__ void __launch_bounds__(kBlock)
iscan_sum_kernel(const int32_t* __restrict__ in, int64_t N, long long* tot, long long* pre,
                 unsigned int* ticket) {
  pdl_wait();
  __shared__ long long sh[kWarps];
  __shared__ bool am_last;
  long long v[16];
  const long long total =
      block_tile_scan(in, N, static_cast<int64_t>(blockIdx.x) * kIscanTile, v, sh);
  if (threadIdx.x == 0) {
    tot[blockIdx.x] = total;
    __threadfence();
    am_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  // exclusive scan of the tile totals: a contiguous chunk per thread, then a block scan
  const int T = static_cast<int>(gridDim.x);
  const int chunk = (T + kBlock - 1) / kBlock;
  const int t0 = min(T, static_cast<int>(threadIdx.x) * chunk), t1 = min(T, t0 + chunk);
  long long local = 0;
  for (int t = t0; t < t1; ++t) local += __ldcg(tot + t);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long incl = local;
#pragma unroll
  for (int dd = 1; dd < 32; dd <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, incl, dd);
    if (lane >= dd) incl += y;
  }
  __syncthreads();
  if (lane == 31) sh[warp] = incl;
  __syncthreads();
  long long p = incl - local;
  for (int k = 0; k < warp; ++k) p += sh[k];
  for (int t = t0; t < t1; ++t) {
    pre[t] = p;
    p += __ldcg(tot + t);
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

__global__ void __launch_bounds__(kBlock)
iscan_emit_kernel(const int32_t* __restrict__ in, int64_t N, const long long* pre,
                  int32_t* __restrict__ out) {
  pdl_wait();
  __shared__ long long sh[kWarps];
  long long v[16];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kIscanTile;
  block_tile_scan(in, N, base, v, sh);
  const long long p = pre[blockIdx.x];
  store16(out, base + 16 * threadIdx.x, N, v, p);
}

// The same scan as one cooperative launch: CTA c owns the contiguous tiles
// [c T / G, (c+1) T / G); it scans them in order (keeping each tile's exclusive in-range
// prefix and its range total), meets the others at a grid barrier, adds the totals of the
// ranges before its own (exact integers: any order gives the same sums) and writes its tiles.
__device__ __forceinline__ long long block_sum_ll(long long v, long long* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  long long t = 0;
  for (int k = 0; k < kWarps; ++k) t += sh[k];
  return t;
}

__global__ void __launch_bounds__(kBlock)
iscan_coop_kernel(const int32_t* __restrict__ in, int64_t N, int T, long long* tot,
                  long long* pre, int32_t* __restrict__ out, GridBar* bar, int* err) {
  __shared__ long long sh[kWarps];
  unsigned int target = 0;
  const int G = static_cast<int>(gridDim.x), c = static_cast<int>(blockIdx.x);
  const int t0 = static_cast<int>(static_cast<int64_t>(c) * T / G);
  const int t1 = static_cast<int>(static_cast<int64_t>(c + 1) * T / G);
  long long v[16];
  long long run = 0;
  for (int t = t0; t < t1; ++t) {
    const long long total = block_tile_scan(in, N, static_cast<int64_t>(t) * kIscanTile, v, sh);
    if (threadIdx.x == 0) pre[t] = run;
    run += total;
    __syncthreads();  // sh is rewritten by the next tile
  }
  if (threadIdx.x == 0) tot[c] = run;
  grid_barrier(bar, target, err);
  long long part = 0;
  for (int k = threadIdx.x; k < c; k += kBlock) part += __ldcg(tot + k);
  const long long CP = block_sum_ll(part, sh);
  for (int t = t0; t < t1; ++t) {
    __syncthreads();
    const int64_t base = static_cast<int64_t>(t) * kIscanTile;
    block_tile_scan(in, N, base, v, sh);
    const long long p = CP + __ldcg(pre + t);
    store16(out, base + 16 * threadIdx.x, N, v, p);
  }
  grid_exit(bar, target);
}

// Self-check of the bounded grid barrier: the barrier's target is one arrival more than the
// grid makes, so every CTA waits until the handle's timeout, records RS_ERR_TIMEOUT and goes
// on; the exit arrivals then cannot return the counter to 0 (rs_last_error resets it).
__global__ void __launch_bounds__(kBlock) barrier_timeout_probe_kernel(GridBar* bar, int* err) {
  unsigned int target = 1;
  grid_barrier(bar, target, err);
  grid_exit(bar, target);
}

inline int grid_for(int64_t N) { return static_cast<int>((N + kBlock - 1) / kBlock); }

}  // namespace

cudaError_t launch_fill(int32_t* p, int64_t N, int32_t v, cudaStream_t st) {
  int64_t g = (N / 4 + kBlock - 1) / kBlock;
  if (g < 1) g = 1;
  const int64_t cap = static_cast<int64_t>(device_sm_count()) * 16;  // 16 CTAs per SM
  if (g > cap) g = cap;
  launch_pdl(fill_kernel, static_cast<int>(g), kBlock, st, p, N, v);
  return cudaGetLastError();
}

cudaError_t launch_prepermute(const Scratch& s, const int32_t* a, int64_t N, int32_t* d,
                              bool init, cudaStream_t st) {
  if (init) {
    trace_mark(s.trace, "fill", st);
    const cudaError_t e = launch_fill(d, N, static_cast<int32_t>(N), st);
    if (e != cudaSuccess) return e;
  }
  trace_mark(s.trace, "prepermute", st);
  launch_pdl(prepermute_kernel, grid_for(N), kBlock, st, a, N, d, s.err);
  return cudaGetLastError();
}

// Four slots per thread (permute4_kernel) from kPermute4MinN slots; below, one slot per
// thread keeps more threads in flight. (Handing the walks that outlast a few rounds to a tail
// kernel through a queue measured 3x slower at 2^24: every queued walk takes an atomic on one
// counter.)
constexpr int64_t kPermute4MinN = int64_t{1} << 18;

cudaError_t launch_permute(const Scratch& s, const int32_t* a, const int32_t* d, int64_t N,
                           int32_t* c, cudaStream_t st) {
  trace_mark(s.trace, "permute", st);
  if (N >= kPermute4MinN)
    launch_pdl(permute4_kernel, static_cast<int>((N + 4 * kBlock - 1) / (4 * kBlock)), kBlock,
               st, a, d, N, c, s.err);
  else
    launch_pdl(permute_kernel, grid_for(N), kBlock, st, a, d, N, c, s.err);
  return cudaGetLastError();
}

// Four slots per thread from 2^18 slots (measured 2 % faster at 2^20, 9 % at 2^22, 18 % at
// 2^24); below, one slot per thread keeps more threads in flight.
constexpr int64_t kSorted4MinN = int64_t{1} << 18;

cudaError_t launch_permute_sorted_bits(const Scratch& s, const int32_t* a, const uint8_t* cl,
                                       int64_t N, int32_t* c, cudaStream_t st) {
  trace_mark(s.trace, "permute_sorted", st);
  if (N >= kSorted4MinN)
    launch_pdl(permute_sorted_bits_kernel<4>, static_cast<int>((N + 4 * kBlock - 1) / (4 * kBlock)),
               kBlock, st, a, cl, N, c, s.err);
  else
    launch_pdl(permute_sorted_bits_kernel<1>, grid_for(N), kBlock, st, a, cl, N, c, s.err);
  return cudaGetLastError();
}

cudaError_t launch_offspring(const Scratch& s, const int32_t* a, int64_t N, int32_t* o,
                             cudaStream_t st) {
  trace_mark(s.trace, "fill", st);
  cudaError_t e = launch_fill(o, N, 0, st);
  if (e != cudaSuccess) return e;
  trace_mark(s.trace, "offspring", st);
  launch_pdl(offspring_kernel, grid_for(N), kBlock, st, a, N, o, s.err);
  return cudaGetLastError();
}

cudaError_t launch_inclusive_scan_i32(const Scratch& s, const int32_t* o, int64_t N,
                                      int32_t* O, cudaStream_t st) {
  const int tiles = static_cast<int>((N + kIscanTile - 1) / kIscanTile);
  long long* tot = s.irec;
  long long* pre = s.irec + (s.max_tiles + 2);
  if (s.coop && s.launch_mode != RS_LAUNCH_SEPARATE) {
    const int cap = coop_capacity(reinterpret_cast<const void*>(iscan_coop_kernel));
    if (cap > 0) {
      const int grid = tiles < cap ? tiles : cap;
      trace_mark(s.trace, "iscan", st);
      return coop_launch(iscan_coop_kernel, grid, st, o, N, tiles, tot, pre, O,
                         &s.glob->bar, s.err);
    }
  }
  trace_mark(s.trace, "iscan_sum", st);
  launch_pdl(iscan_sum_kernel, tiles, kBlock, st, o, N, tot, pre, &s.glob->ticket_iscan);
  trace_mark(s.trace, "iscan_emit", st);
  launch_pdl(iscan_emit_kernel, tiles, kBlock, st, o, N, pre, O);
  return cudaGetLastError();
}

cudaError_t launch_barrier_timeout_probe(const Scratch& s, cudaStream_t st) {
  const int cap = coop_capacity(reinterpret_cast<const void*>(barrier_timeout_probe_kernel));
  if (cap < 1) return cudaErrorCooperativeLaunchTooLarge;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = sms < cap ? sms : cap;
  trace_mark(s.trace, "barrier_timeout_probe", st);
  return coop_launch(barrier_timeout_probe_kernel, grid, st, &s.glob->bar, s.err);
}

cudaError_t launch_adjacent_difference(const int32_t* O, int64_t N, int32_t* o,
                                       cudaStream_t st) {
  launch_pdl(adjacent_difference_kernel, static_cast<int>((N + 4 * kBlock - 1) / (4 * kBlock)),
             kBlock, st, O, N, o);
  return cudaGetLastError();
}

cudaError_t launch_cumoff_to_ancestors(const Scratch& s, const int32_t* O, int64_t N,
                                       int32_t* a, cudaStream_t st) {
  trace_mark(s.trace, "cumoff_to_ancestors", st);
  launch_pdl(cumoff_to_ancestors_kernel, static_cast<int>((N + kTile - 1) / kTile), kBlock, st,
             O, N, a, s.err);
  return cudaGetLastError();
}

}  // namespace rsk
