// permute.cuh -- one slot of the parallel Permute of Code 10 (Appendix C), shared by the
// single-filter and batched kernels. The claims d (Prepermute: d[j] = lowest i with a[i] = j,
// or the sentinel n) must be complete before any thread runs this.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace rsk {
namespace {

// Second procedure of Code 10 fused with its gather c^i = a^{d^i}, for index i of a vector
// of n ancestors (local indices):
//  - a claimed slot i (d_i < n) keeps its own particle: c_i = a[d_i] = i;
//  - a particle whose claim failed (d[a_i] != i) walks x = i, d[x], d[d[x]], ... to the
//    first unclaimed slot x and writes c_x = a_i there.
// The walks start at indices absent from d and d is injective on claimed slots, so the
// walks are disjoint and end at distinct unclaimed slots (the termination argument of
// Appendix C): they only read d, and every slot of c is written exactly once, in any order.
// kCoherent: a and d were written earlier in the same kernel launch (by other CTAs), so they
// are read through L2 only.
template <bool kCoherent>
__device__ __forceinline__ int32_t ld_i32(const int32_t* p) {
  if constexpr (kCoherent) return __ldcg(p); else return *p;
}
template <bool kCoherent = false>
__device__ __forceinline__ void permute_one(const int32_t* __restrict__ a,
                                            const int32_t* __restrict__ d, int64_t n,
                                            int32_t* __restrict__ c, int64_t i, int* err) {
  const int32_t sentinel = static_cast<int32_t>(n);
  const int32_t ai = ld_i32<kCoherent>(a + i);
  if (ai < 0 || ai >= n) {
    flag_error(err, RS_ERR_ARG);
    return;
  }
  if (ld_i32<kCoherent>(d + i) != sentinel) c[i] = static_cast<int32_t>(i);
  if (ld_i32<kCoherent>(d + ai) != static_cast<int32_t>(i)) {
    int64_t x = i;
    int64_t steps = 0;
    for (;;) {
      const int32_t dx = ld_i32<kCoherent>(d + x);
      if (dx == sentinel) break;
      if (dx < 0 || dx > sentinel || ++steps > n) {  // only a corrupted d can get here
        flag_error(err, RS_ERR_ARG);
        return;
      }
      x = dx;
    }
    c[x] = ai;
  }
}

// Claims of Code 10 read from the Prepermute vector d (d[x] = the lowest position whose
// ancestor is x, or the sentinel n).
struct ClaimsOf {
  const int32_t* __restrict__ d;
  __device__ __forceinline__ int32_t operator()(int32_t x) const { return d[x]; }
};

// Walks of Code 10 for a whole warp, K walkers per lane, queued: walker q stands at slot
// x[q] with dx[q] = claim(x[q]) already loaded (claim: the Prepermute claim of a slot, the
// sentinel n for an unclaimed one) and ends at the first unclaimed slot, where c receives
// val[q]. A walker whose claim ends at its own slot (dx = the sentinel) is done at once; the
// others take their first step and are collected, by ballot, into the warp's shared list
// `pend` (32 K entries), which the lanes then work off one walk each to its end (lane l takes
// entries l, l + 32, ...), so every lane runs only walks that go on. The walks start at
// distinct failed claims and are disjoint (see permute_one): c is the same as walking each
// one alone. Called by all 32 lanes (lanes without walkers pass act = false).
template <int K, typename Claim>
__device__ __forceinline__ void walk_queue(const Claim& claim, int32_t sentinel,
                                           int32_t* __restrict__ c, const int32_t (&x)[K],
                                           const int32_t (&dx)[K], const int32_t (&val)[K],
                                           const bool (&act)[K], int64_t n, int2* pend,
                                           int* err) {
  const uint32_t us = static_cast<uint32_t>(sentinel);
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  bool bad = false;
  int total = 0;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    bool go = false;
    if (act[q]) {
      const uint32_t v = static_cast<uint32_t>(dx[q]);
      if (v == us) c[x[q]] = val[q];  // its own slot is unclaimed: the walk ends there
      else if (v > us) bad = true;    // (only a corrupted claim vector)
      else go = true;
    }
    const unsigned m = __ballot_sync(0xffffffffu, go);
    if (go) pend[total + __popc(m & below)] = make_int2(dx[q], val[q]);  // one step taken
    total += __popc(m);
  }
  __syncwarp();
  for (int e = lane; e < total; e += 32) {
    const int2 w = pend[e];
    int32_t xs = w.x;
    for (int64_t steps = 0;; ++steps) {
      const uint32_t v = static_cast<uint32_t>(claim(xs));
      if (v == us) {
        c[xs] = w.y;
        break;
      }
      if (v > us || steps > n) {  // only a corrupted claim vector can get here
        bad = true;
        break;
      }
      xs = static_cast<int32_t>(v);
    }
  }
  __syncwarp();
  if (bad) flag_error(err, RS_ERR_ARG);
}

}  // namespace
}  // namespace rsk
