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
__device__ __forceinline__ void permute_one(const int32_t* __restrict__ a,
                                            const int32_t* __restrict__ d, int64_t n,
                                            int32_t* __restrict__ c, int64_t i, int* err) {
  const int32_t sentinel = static_cast<int32_t>(n);
  const int32_t ai = a[i];
  if (ai < 0 || ai >= n) {
    flag_error(err, RS_ERR_ARG);
    return;
  }
  if (d[i] != sentinel) c[i] = static_cast<int32_t>(i);
  if (d[ai] != static_cast<int32_t>(i)) {
    int64_t x = i;
    int64_t steps = 0;
    for (;;) {
      const int32_t dx = d[x];
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

}  // namespace
}  // namespace rsk
