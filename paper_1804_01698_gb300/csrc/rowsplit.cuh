// Splitting one row's products over several blocks (heavy rows of skewed
// inputs): part `part` of `parts` takes a contiguous range of the row's
// stored a_ik holding an equal share of its flop.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace sg {

// Part `part` of `parts` of row i's stored a_ik: the contiguous range
// [*j_lo, *j_hi) of entries whose products start in the part's equal share
// of the row's flop (an entry belongs to the share holding its first
// product).  Whole block.
__device__ __forceinline__ void part_range(const Args &a, int32_t i, int part, int parts, int32_t *j_lo,
                                           int32_t *j_hi) {
  __shared__ long long s_ll[33];
  const int32_t j0 = a.arp[i], j1 = a.arp[i + 1];
  long long f = 0;
  for (int32_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    const int32_t c = a.aci[j];
    f += a.brp[c + 1] - a.brp[c];
  }
  const long long F = block_sum(f, s_ll);
  const long long lo_f = F / parts * part + F % parts * part / parts;
  const long long hi_f = F / parts * (part + 1) + F % parts * (part + 1) / parts;
  long long below_lo = 0, below_hi = 0, carry = 0;
  for (int32_t base = j0; base < j1; base += blockDim.x) {
    const int32_t j = base + threadIdx.x;
    long long len = 0;
    if (j < j1) {
      const int32_t c = a.aci[j];
      len = a.brp[c + 1] - a.brp[c];
    }
    long long tot;
    const long long excl = carry + block_excl_scan(len, s_ll, &tot);
    if (j < j1) {
      below_lo += excl < lo_f;
      below_hi += excl < hi_f;
    }
    carry += tot;
  }
  const long long n_lo = block_sum(below_lo, s_ll), n_hi = block_sum(below_hi, s_ll);
  *j_lo = part == 0 ? j0 : j0 + (int32_t)n_lo;
  *j_hi = part == parts - 1 ? j1 : j0 + (int32_t)n_hi;
}

}  // namespace sg
