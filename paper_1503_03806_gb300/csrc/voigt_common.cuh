// voigt_common.cuh -- pieces shared by the two Voigt kernel files: the
// bounded-wait limit of the bulk-copy barriers and the occupancy helpers of
// the persistent launches.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "helk_internal.cuh"

namespace helk {

constexpr long long WAIT_LIMIT = 1ll << 24;  // polls of a bulk-copy barrier

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

}  // namespace helk
