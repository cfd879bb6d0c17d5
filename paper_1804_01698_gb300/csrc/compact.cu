// Compacted copy of A for products where most stored a_ik select an empty
// row of B (the BFS-frontier product A * F of Sec. 5.5: F has a few entries
// per column, so almost every row of F is empty).  Such entries add nothing
// to C (Fig. "RowWise_SpGEMM" loops over the entries of the selected row of
// B), yet every hash-bin kernel would still stage them and read their row
// bounds.  The plan therefore hands the phases a copy of A holding only the
// entries whose row of B is not empty, row by row (in stored order, but for
// the parts of a row that several threads share, which may change places).
//
//   (row pointers: the exclusive scan of the flop pass's per-row counts)
//   k_compact_a     the copy's columns and the source entry of each, from
//                   the flop pass's per-tile lists of kept entries (tiles
//                   with too many are walked again)
//   k_compact_vals  values of the copy, before every numeric phase
// Every kernel runs a fixed number of items per thread, so a hub row of
// thousands of entries costs no more than as many short rows.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace sg {

// The kept entries of every row (row of B not empty) go to the row's range
// [karp[i], karp[i + 1]) of the copy, with their source entries.  One block
// per merge-path tile.  A tile whose kept entries the flop pass listed
// (klist_n[t] >= 0) places them from that list, one reservation of the
// row's cursor each; a tile with more walks its items again, and there a row
// inside one thread's items keeps its stored order while the parts of a
// shared row reserve their places from the cursor (cursor[i], zeroed first).
// The products of a row do not depend on the order of its stored a_ik.
__global__ void __launch_bounds__(kMergeThreads)
    k_compact_a(Args a, int64_t nnz_a, int64_t nnz_b, const long long *__restrict__ starts,
                const int2 *__restrict__ klist, const int32_t *__restrict__ klist_n, const int32_t *__restrict__ karp,
                int32_t *__restrict__ cursor, int32_t *__restrict__ kaci, int32_t *__restrict__ asrc) {
  __shared__ int32_t lens[kMergeTile];
  __shared__ int32_t ends[kMergeTile];
  __shared__ long long coords[4];
  const int nl = klist_n[blockIdx.x];
  if (nl >= 0) {
    const int2 *list = klist + (size_t)blockIdx.x * kKeptListCap;
    for (int t = threadIdx.x; t < nl; t += blockDim.x) {
      const int2 e = list[t];
      const int32_t pos = karp[e.x] + atomicAdd(cursor + e.x, 1);
      kaci[pos] = __ldg(a.aci + e.y);
      asrc[pos] = e.y;
    }
    return;
  }
  merge_tile_walk(a.arp, a.aci, a.brp, a.m, nnz_a, a.n, nnz_b, a.err, starts, lens, ends, coords,
                  [&](int64_t i, long long, int kp, bool whole, int64_t j, const int32_t *len, int n) {
                    if (kp == 0) return;
                    int32_t pos = karp[i] + (whole ? 0 : atomicAdd(cursor + i, kp));
                    for (int q = 0; q < n; ++q) {
                      if (len[q] > 0) {
                        kaci[pos] = __ldg(a.aci + j + q);
                        asrc[pos] = (int32_t)(j + q);
                        ++pos;
                      }
                    }
                  });
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

cudaError_t compact_a_gather(spgemm_plan_s *p) {
  Args a{p->m, p->n, p->k, p->arp, p->aci, p->brp, p->bci, p->av, p->bv, p->G, &p->dc->err};
  const int64_t tiles = (p->m + p->nnz_a + kMergeTile - 1) / kMergeTile;
  k_compact_a<<<(unsigned)tiles, kMergeThreads, 0, p->stream>>>(a, p->nnz_a, p->nnz_b, p->mstarts, p->klist,
                                                                 p->klist_n, p->karp, p->kept, p->kaci, p->asrc);
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
