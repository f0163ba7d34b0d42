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

// The same slot when a is non-decreasing and d holds its claims (the systematic and stratified
// ancestries of Code 11): the lowest claimant of particle a_i is the first position of its
// run, so the claim of position i failed exactly when i > 0 and a_{i-1} = a_i. That replaces
// the dependent load of d[a_i] by a load next to a_i; the writes are those of permute_one.
__device__ __forceinline__ void permute_sorted_one(const int32_t* __restrict__ a,
                                                   const int32_t* __restrict__ d, int64_t n,
                                                   int32_t* __restrict__ c, int64_t i, int* err) {
  const int32_t sentinel = static_cast<int32_t>(n);
  const int32_t ai = a[i];
  if (ai < 0 || ai >= n) {
    flag_error(err, RS_ERR_ARG);
    return;
  }
  const int32_t di = d[i];
  if (di != sentinel) c[i] = static_cast<int32_t>(i);
  if (i > 0 && a[i - 1] == ai) {
    int64_t x = i;
    int32_t dx = di;
    int64_t steps = 0;
    while (dx != sentinel) {
      if (dx < 0 || dx > sentinel || ++steps > n) {  // only a corrupted d can get here
        flag_error(err, RS_ERR_ARG);
        return;
      }
      x = dx;
      dx = d[x];
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

// Walks of Code 10 for a whole warp, K walkers per lane: walker q stands at slot x[q] with
// dx[q] = claim(x[q]) already loaded (claim: the Prepermute claim of a slot, the sentinel n
// for an unclaimed one) and ends at the first unclaimed slot, where c receives val[q]. First
// every lane moves its live walkers for at most kWalkRounds rounds, each round moving every
// live walker one step and then issuing the claim loads of all of them together (up to K
// dependent chains in flight per thread); then the walks still going are compacted into the
// warp's shared list `pend` (32 K entries: slot reached and value) and finished one walk per
// lane, 32 at a time. A warp otherwise runs as many rounds as its longest walk takes, with
// most lanes predicated off. The walks start at distinct failed claims and are disjoint (see
// permute_one), so every walk ends at its own unclaimed slot: c is the same as walking each
// one alone. Called by all 32 lanes (lanes without walkers pass act = false).
constexpr uint32_t kWalkRounds = 2;

template <int K, typename Claim>
__device__ __forceinline__ void walk_warp(const Claim& claim, int32_t sentinel,
                                          int32_t* __restrict__ c, int32_t (&x)[K],
                                          int32_t (&dx)[K], const int32_t (&val)[K],
                                          bool (&act)[K], int64_t n, int2* pend, int* err) {
  const uint32_t us = static_cast<uint32_t>(sentinel);
  const int lane = threadIdx.x & 31;
  bool bad = false;
  for (uint32_t r = 0; r < kWalkRounds; ++r) {
    bool any = false;
#pragma unroll
    for (int q = 0; q < K; ++q) {
      if (!act[q]) continue;
      const uint32_t v = static_cast<uint32_t>(dx[q]);
      if (v >= us) {  // the sentinel (the walk ends here), or a corrupted claim
        if (v == us) c[x[q]] = val[q]; else bad = true;
        act[q] = false;
      } else {
        x[q] = dx[q];
        any = true;
      }
    }
    if (!any) break;  // (per lane)
#pragma unroll
    for (int q = 0; q < K; ++q)
      if (act[q]) dx[q] = claim(x[q]);
  }
  // compaction of the walks still going (each at slot x with its claim loaded as dx)
  int mine = 0;
#pragma unroll
  for (int q = 0; q < K; ++q) mine += static_cast<int>(act[q]);
  int incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  if (total > 0) {
    int pos = incl - mine;
#pragma unroll
    for (int q = 0; q < K; ++q)
      if (act[q]) pend[pos++] = make_int2(x[q], val[q]);
    __syncwarp();
    for (int b = 0; b < total; b += 32) {
      if (b + lane < total) {
        const int2 e = pend[b + lane];
        int32_t xs = e.x;
        for (int64_t steps = 0;; ++steps) {
          const uint32_t v = static_cast<uint32_t>(claim(xs));
          if (v == us) {
            c[xs] = e.y;
            break;
          }
          if (v > us || steps > n) {  // only a corrupted claim vector can get here
            bad = true;
            break;
          }
          xs = static_cast<int32_t>(v);
        }
      }
    }
    __syncwarp();
  }
  if (bad) flag_error(err, RS_ERR_ARG);
}

// The same walks, queued: a walker whose claim ends at its own slot (dx = the sentinel) is
// done at once; the others take their first step and are collected, by ballot, into the warp's
// shared list `pend` (32 K entries), which the lanes then work off one walk each to its end
// (lane l takes entries l, l + 32, ...). Every lane runs only the walks that go on, instead of
// K predicated walkers per round. c is the same as walking each one alone. Called by all 32
// lanes.
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
