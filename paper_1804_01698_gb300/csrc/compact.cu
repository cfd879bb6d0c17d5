// Compacted copy of A for products where most stored a_ik select an empty
// row of B (the BFS-frontier product A * F of Sec. 5.5: F has a few entries
// per column, so almost every row of F is empty).  Such entries add nothing
// to C (Fig. "RowWise_SpGEMM" loops over the entries of the selected row of
// B), yet every hash-bin kernel would still stage them and read their row
// bounds.  The plan therefore hands the phases a copy of A holding only the
// entries whose row of B is not empty, row by row in stored order.
//
//   k_compact_keep  per entry: kept (its row of B is not empty), read from
//                   the flop pass's prefix of B-row lengths
//   k_compact_a     from the exclusive scan of the keep flags: the copy's
//                   row pointers, columns and the source entry of each
//   k_compact_vals  values of the copy, before every numeric phase
// Every kernel runs one thread per entry or per row, so a hub row of
// thousands of entries costs no more than as many short rows.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace sg {

// keep[j] = 1 when P[j + 1] > P[j] (P: exclusive prefix of the B-row lengths).
__global__ void __launch_bounds__(256)
    k_compact_keep(const long long *__restrict__ P, int64_t nnz_a, int32_t *__restrict__ keep) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz_a; j += (int64_t)gridDim.x * blockDim.x)
    keep[j] = P[j + 1] > P[j] ? 1 : 0;
}

// pos: exclusive scan of the keep flags (nnz_a + 1 entries).  Row i of the
// copy starts at pos[rp[i]]; a kept entry j goes to pos[j].
__global__ void __launch_bounds__(256)
    k_compact_a(const int32_t *__restrict__ arp, const int32_t *__restrict__ aci, int64_t m, int64_t nnz_a,
                const int32_t *__restrict__ pos, int32_t *__restrict__ karp, int32_t *__restrict__ kaci,
                int32_t *__restrict__ asrc) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz_a; j += stride) {
    const int32_t q = pos[j];
    if (pos[j + 1] > q) {
      kaci[q] = aci[j];
      asrc[q] = (int32_t)j;
    }
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= m; i += stride) karp[i] = pos[arp[i]];
}

template <typename T>
__global__ void __launch_bounds__(256)
    k_compact_vals(const int32_t *__restrict__ asrc, int64_t n, const T *__restrict__ av, T *__restrict__ kav) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    kav[e] = av[asrc[e]];
}

static unsigned grid_for(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (unsigned)(b < 1 ? 1 : b > 4096 ? 4096 : b);
}

cudaError_t compact_a_keep(spgemm_plan_s *p, int32_t *pos) {
  k_compact_keep<<<grid_for(p->nnz_a), 256, 0, p->stream>>>(p->eflop, p->nnz_a, pos);
  return cudaGetLastError();
}

cudaError_t compact_a_gather(spgemm_plan_s *p, const int32_t *pos) {
  k_compact_a<<<grid_for(std::max<int64_t>(p->nnz_a, p->m + 1)), 256, 0, p->stream>>>(
      p->arp, p->aci, p->m, p->nnz_a, pos, p->karp, p->kaci, p->asrc);
  return cudaGetLastError();
}

cudaError_t compact_a_values(spgemm_plan_s *p) {
  if (!p->a_compact || p->nnz_a_used == 0) return cudaSuccess;
  const int64_t n = p->nnz_a_used;
  const unsigned blocks = grid_for(n);
  KernelScope ks(p, "compact_vals");
  switch (p->dtype) {
    case SPGEMM_F64:
      k_compact_vals<double><<<blocks, 256, 0, p->stream>>>(p->asrc, n, (const double *)p->av, (double *)p->kav);
      break;
    case SPGEMM_F32:
      k_compact_vals<float><<<blocks, 256, 0, p->stream>>>(p->asrc, n, (const float *)p->av, (float *)p->kav);
      break;
    default:
      k_compact_vals<int64_t><<<blocks, 256, 0, p->stream>>>(p->asrc, n, (const int64_t *)p->av, (int64_t *)p->kav);
      break;
  }
  return cudaGetLastError();
}

}  // namespace sg
