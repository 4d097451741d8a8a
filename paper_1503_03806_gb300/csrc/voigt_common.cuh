// voigt_common.cuh -- pieces shared by the Voigt kernel files and the tile
// map: the time limit of the bulk-copy barrier waits, the occupancy
// helpers of the persistent launches, and a warp-cooperative search of the
// lines' sorted reference indices.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "helk_internal.cuh"

namespace helk {

// Time limit of a bulk-copy barrier wait: a chunk's copy and the slowest
// warp's work on the chunks before it take microseconds, so 100 ms is only
// reached when something is wrong.
constexpr unsigned long long WAIT_LIMIT_NS = 100ull * 1000 * 1000;

template <typename K>
static int resident_ctas(helk_ctx *c, K kern, int block) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, 0) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  return occ * c->num_sms;
}

template <typename K>
static unsigned persistent_grid(helk_ctx *c, K kern, int block, int64_t nitems) {
  const int64_t slots = resident_ctas(c, kern, block);
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(slots, nitems));
}

// First index in [lo, hi) whose key is not below x (strict: key > x when
// `upper`), else hi.  All lanes take part and get the result.  K: the key
// type (double, or int32_t compared as integers against an int64_t x).
template <typename K, typename X>
__device__ __forceinline__ int64_t warp_search(const K *__restrict__ key, int64_t lo, int64_t hi, X x, bool upper) {
  const int lane = threadIdx.x & 31;
  // invariant: the answer lies in [lo, hi]
  while (hi - lo > 32) {
    const int64_t step = (hi - lo + 31) / 32;
    const int64_t p = lo + (int64_t)lane * step;
    const bool below = p < hi && (upper ? (X)key[p] <= x : (X)key[p] < x);
    const int c = __popc(__ballot_sync(0xffffffffu, below));
    const int64_t nlo = c > 0 ? lo + (int64_t)(c - 1) * step + 1 : lo;
    const int64_t nhi = c > 0 ? min(hi, lo + (int64_t)c * step) : lo;
    lo = nlo;
    hi = nhi;
  }
  const int64_t p = lo + lane;
  const bool below = p < hi && (upper ? (X)key[p] <= x : (X)key[p] < x);
  return lo + __popc(__ballot_sync(0xffffffffu, below));
}

}  // namespace helk
