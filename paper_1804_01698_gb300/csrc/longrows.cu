// Long rows of B for the symbolic phase of the bitmap rows of A.
//
// A heavy row of A (one that takes the column-bitmap path) meets the same
// few long rows of B again and again: in R-MAT A*A at scale 16, 119 rows of
// B with 1024 or more entries carry two thirds of all products.  For those
// rows the plan keeps the column bitmap of the row (words = ceil(k/32)
// words), and the symbolic phase ORs it word by word into the bitmap of C's
// row instead of setting one bit per product.  The count is the one the
// paper's symbolic phase defines (Fig. "Hash_SpGEMM"): the distinct columns
// of the row's products.
//
//   long_mark_row   per row of B (in the flop pass's k_merge_starts): long
//                   (entries >= long_min) or not; long rows get an index d
//   k_long_build    per long row: its column bitmap
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace sg {

// One block per long row d: its column bitmap.  Columns outside B raise
// kErrCsr and are left out.
__global__ void __launch_bounds__(256)
    k_long_build(const int32_t *__restrict__ brp, const int32_t *__restrict__ bci, int32_t ncols, int words,
                 const int32_t *__restrict__ lrow, uint32_t *__restrict__ bits, uint32_t *err) {
  extern __shared__ uint32_t sm_lbits[];
  const int d = blockIdx.x;
  const int32_t k = lrow[d];
  const int32_t b0 = brp[k], len = brp[k + 1] - b0;
  for (int w = threadIdx.x; w < words; w += blockDim.x) sm_lbits[w] = 0u;
  __syncthreads();
  for (int32_t q = threadIdx.x; q < len; q += blockDim.x) {
    const int32_t c = bci[b0 + q];
    if (!((uint32_t)c < (uint32_t)ncols)) {
      raise_err(err, kErrCsr);
      continue;
    }
    atomicOr(&sm_lbits[c >> 5], 1u << (c & 31));
  }
  __syncthreads();
  uint32_t *bw = bits + (size_t)d * words;
  for (int w = threadIdx.x; w < words; w += blockDim.x) bw[w] = sm_lbits[w];
}

cudaError_t long_rows_build(spgemm_plan_s *p) {
  p->long_ready = false;
  if (p->long_min <= 0 || p->n_long <= 0 || p->long_tot <= 0) return cudaSuccess;
  const size_t words = (size_t)p->bm_words;
  const size_t bytes = (size_t)p->n_long * words * 4;
  cudaError_t e = cudaMallocAsync(&p->long_ws, bytes, p->stream);
  if (e != cudaSuccess) {
    p->long_ws = nullptr;
    return e;
  }
  p->long_ws_bytes = bytes;
  p->lbits = static_cast<uint32_t *>(p->long_ws);
  const size_t smem = words * 4;
  e = set_dynamic_smem(reinterpret_cast<const void *>(k_long_build), smem);
  if (e != cudaSuccess) return e;
  {
    KernelScope ks(p, "long_build");
    k_long_build<<<(unsigned)p->n_long, 256, smem, p->stream>>>(p->brp, p->bci, (int32_t)p->k, (int)words, p->lrow,
                                                                p->lbits, &p->dc->err);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) p->long_ready = true;
  return e;
}

}  // namespace sg
