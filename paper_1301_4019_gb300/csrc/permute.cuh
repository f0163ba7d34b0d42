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

// Up to four walks of Code 10 at once: walker q stands at slot x[q] with dx[q] = d[x[q]]
// already loaded, and ends at the first unclaimed slot, where c receives val[q]. Each round
// moves every live walker one step and then issues the loads of all live walkers together,
// so up to four dependent chains are in flight per thread; the walks are disjoint (see
// permute_one), so the writes are those of four separate walks.
__device__ __forceinline__ void walk4(const int32_t* __restrict__ d, int32_t sentinel,
                                      int32_t* __restrict__ c, int32_t (&x)[4],
                                      int32_t (&dx)[4], const int32_t (&val)[4],
                                      bool (&act)[4], int64_t n, int* err) {
  const uint32_t us = static_cast<uint32_t>(sentinel);
  bool bad = false;
  for (uint32_t steps = 0; act[0] | act[1] | act[2] | act[3]; ++steps) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (!act[q]) continue;
      const uint32_t v = static_cast<uint32_t>(dx[q]);
      if (v >= us) {  // the sentinel (the walk ends here), or a corrupted d
        if (v == us) c[x[q]] = val[q]; else bad = true;
        act[q] = false;
      } else {
        x[q] = dx[q];
      }
    }
    if (steps >= static_cast<uint32_t>(n)) {  // only a corrupted d can get here
      bad = true;
      break;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (act[q]) dx[q] = d[x[q]];
  }
  if (bad) flag_error(err, RS_ERR_ARG);
}

// Walks of the four-slot kernels in two stages, for a whole warp: first every lane moves its
// (up to) four walkers for at most kWalkRounds rounds (walk4's loop), which ends most walks;
// then the walks still going are compacted into the warp's shared list `pend` (128 entries:
// slot reached and value) and finished one walk per lane, 32 at a time. A warp otherwise
// runs as many four-walker rounds as its longest walk takes, with most lanes predicated off.
// Every walk still moves through the same slots and ends at the same unclaimed slot, so c is
// the same as with walk4.
constexpr uint32_t kWalkRounds = 2;

__device__ __forceinline__ void walk4_warp(const int32_t* __restrict__ d, int32_t sentinel,
                                           int32_t* __restrict__ c, int32_t (&x)[4],
                                           int32_t (&dx)[4], const int32_t (&val)[4],
                                           bool (&act)[4], int64_t n, int2* pend, int* err) {
  const uint32_t us = static_cast<uint32_t>(sentinel);
  const int lane = threadIdx.x & 31;
  bool bad = false;
  for (uint32_t r = 0; r < kWalkRounds && (act[0] | act[1] | act[2] | act[3]); ++r) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (!act[q]) continue;
      const uint32_t v = static_cast<uint32_t>(dx[q]);
      if (v >= us) {  // the sentinel (the walk ends here), or a corrupted d
        if (v == us) c[x[q]] = val[q]; else bad = true;
        act[q] = false;
      } else {
        x[q] = dx[q];
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (act[q]) dx[q] = d[x[q]];
  }
  // compaction of the walks still going (each at slot x with d[x] loaded as dx)
  const int mine = static_cast<int>(act[0]) + act[1] + act[2] + act[3];
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
    for (int q = 0; q < 4; ++q)
      if (act[q]) pend[pos++] = make_int2(x[q], val[q]);
    __syncwarp();
    for (int b = 0; b < total; b += 32) {
      if (b + lane < total) {
        const int2 e = pend[b + lane];
        int32_t xs = e.x;
        for (int64_t steps = 0;; ++steps) {
          const uint32_t v = static_cast<uint32_t>(d[xs]);
          if (v == us) {
            c[xs] = e.y;
            break;
          }
          if (v > us || steps > n) {  // only a corrupted d can get here
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

}  // namespace
}  // namespace rsk
