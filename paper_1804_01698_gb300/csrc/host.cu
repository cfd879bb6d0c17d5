// Products whose operands and result live in host memory (spgemm_host).
//
// One plan runs the flop pass and the symbolic phase of the whole product,
// which give C's row pointers and nnz(C), so C is allocated once.  The rows
// are then split into contiguous blocks by their share of C's entries (the
// partition of paper Sec. 4.1, Fig. "RowsToThreads", steps 1-2, applied to
// blocks instead of threads), and the numeric phase runs block after block
// (spgemm_numeric_rows) on the caller's stream while a copy stream moves
// each finished block's columns and values to the host.  Rows of C are
// independent (Fig. "RowWise_SpGEMM"), so the result does not depend on the
// blocking.
//
// On GB300 the host link, not the GPU, bounds this path: the copy of C runs
// at the link's rate whatever issues it, and the blocking hides the numeric
// phase (apart from the first block's) under that copy.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace sg {
namespace {

int cuda_fail(cudaError_t e, const char *where) {
  set_last_error(std::string("spgemm_host: ") + where + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? SPGEMM_ERR_OUT_OF_MEMORY : SPGEMM_ERR_DEVICE;
}

bool host_desc_ok(const spgemm_csr *c) {
  if (!c || c->nrows < 0 || c->ncols < 0 || c->nnz < 0) return false;
  if (c->nrows > INT32_MAX || c->ncols > INT32_MAX || c->nnz > INT32_MAX) return false;
  if (!c->row_ptr) return false;
  return c->nnz == 0 || (c->col_idx && c->vals);
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// The row blocks, in the order they run: `parts` contiguous ranges of
// rows, the r-th to run holding a share of C's entries proportional to
// 2^min(r, kShareCap).  The shares double, so the first block, whose numeric
// phase no copy hides, is small, and every later block's numeric phase (at
// most twice the entries of the block before it) still runs under the copy
// of the block before it, which moves C about 3 times slower than the
// numeric phase writes it on GB300.  The blocks are cut from the first row
// on or from the last row back, whichever gives the first block more rows:
// a first block of a few heavy rows keeps few SMs busy (in R-MAT the
// heaviest rows come first).  Each cut is a lower-bound search of its
// cumulative share over C's row pointers (as Fig. "RowsToThreads" searches
// the flop prefix for threads); empty blocks are possible and skipped by
// the caller.
constexpr int kShareCap = 6;

std::vector<std::pair<int64_t, int64_t>> nnz_blocks(const int32_t *c_rp, int64_t m, int parts) {
  const __int128 total = c_rp[m];
  std::vector<__int128> cum(parts + 1, 0);  // cumulative shares
  for (int r = 0; r < parts; ++r) cum[r + 1] = cum[r] + ((__int128)1 << std::min(r, kShareCap));
  std::vector<int64_t> fwd(parts + 1, 0), bwd(parts + 1, 0);  // boundaries in running order
  fwd[0] = 0;
  fwd[parts] = m;
  bwd[0] = m;
  bwd[parts] = 0;
  for (int r = 1; r < parts; ++r) {
    const int64_t head = (int64_t)(total * cum[r] / cum[parts]);
    fwd[r] = std::max<int64_t>(std::lower_bound(c_rp, c_rp + m, (int32_t)head) - c_rp, fwd[r - 1]);
    const int64_t tail = (int64_t)(total - total * cum[r] / cum[parts]);
    bwd[r] = std::min<int64_t>(std::lower_bound(c_rp, c_rp + m, (int32_t)tail) - c_rp, bwd[r - 1]);
  }
  std::vector<std::pair<int64_t, int64_t>> out;
  const bool from_end = parts > 1 && bwd[0] - bwd[1] > fwd[1] - fwd[0];
  for (int r = 0; r < parts; ++r)
    out.push_back(from_end ? std::make_pair(bwd[r + 1], bwd[r]) : std::make_pair(fwd[r], fwd[r + 1]));
  return out;
}

// Everything the call holds on the device, released in one place.
struct HostCall {
  cudaStream_t st = nullptr, cs = nullptr;
  spgemm_plan_t plan = nullptr;
  std::vector<cudaEvent_t> events;
  void *d_ops = nullptr;    // A (and B) on the device
  void *d_rp = nullptr;     // C's row pointers
  void *d_c = nullptr;      // C's columns and values
  ~HostCall() {
    if (cs) cudaStreamSynchronize(cs);
    if (plan) spgemm_plan_destroy(plan);
    for (cudaEvent_t e : events) cudaEventDestroy(e);
    if (d_c) cudaFreeAsync(d_c, st);
    if (d_rp) cudaFreeAsync(d_rp, st);
    if (d_ops) cudaFreeAsync(d_ops, st);
    if (cs) cudaStreamDestroy(cs);
  }
};

constexpr int kDefaultRowBlocks = 6;
constexpr int64_t kRowBlockMinFlop = int64_t(1) << 26;

}  // namespace
}  // namespace sg

using namespace sg;

// A's row pointers are read on the host: refuse device memory, which the
// host cannot dereference.  Without a usable driver the call cannot tell,
// and the pointer is taken for host memory.
static bool device_only(const void *ptr) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice;
}

static int spgemm_host_impl(const spgemm_csr *A, const spgemm_csr *B, int dtype, unsigned flags, void *stream,
                            int row_blocks, spgemm_alloc_fn host_alloc, void *alloc_ctx, int32_t **c_row_ptr,
                            int32_t **c_col_idx, void **c_vals, int64_t *nnz_c);

extern "C" int spgemm_host(const spgemm_csr *A, const spgemm_csr *B, int dtype, unsigned flags, void *stream,
                           int row_blocks, spgemm_alloc_fn host_alloc, void *alloc_ctx, int32_t **c_row_ptr,
                           int32_t **c_col_idx, void **c_vals, int64_t *nnz_c) {
  // nothing may throw across the C boundary: host-side vectors sized by m
  // can fail to allocate
  try {
    return spgemm_host_impl(A, B, dtype, flags, stream, row_blocks, host_alloc, alloc_ctx, c_row_ptr, c_col_idx,
                            c_vals, nnz_c);
  } catch (const std::bad_alloc &) {
    set_last_error("spgemm_host: host memory exhausted");
    return SPGEMM_ERR_OUT_OF_MEMORY;
  } catch (...) {
    set_last_error("spgemm_host: unexpected host-side failure");
    return SPGEMM_ERR_DEVICE;
  }
}

static int spgemm_host_impl(const spgemm_csr *A, const spgemm_csr *B, int dtype, unsigned flags, void *stream,
                            int row_blocks, spgemm_alloc_fn host_alloc, void *alloc_ctx, int32_t **c_row_ptr,
                            int32_t **c_col_idx, void **c_vals, int64_t *nnz_c) {
  NvtxRange nvtx("spgemm_host");
  if (!host_alloc || !c_row_ptr || !c_col_idx || !c_vals || !nnz_c) return SPGEMM_ERR_INVALID_ARGUMENT;
  *c_row_ptr = nullptr;
  *c_col_idx = nullptr;
  *c_vals = nullptr;
  *nnz_c = 0;
  set_last_error("");
  if (!host_desc_ok(A) || !host_desc_ok(B) || A->ncols != B->nrows) return SPGEMM_ERR_INVALID_ARGUMENT;
  if (dtype != SPGEMM_I64 && dtype != SPGEMM_F32 && dtype != SPGEMM_F64) return SPGEMM_ERR_INVALID_ARGUMENT;
  if (flags & SPGEMM_TIMING) {
    set_last_error("spgemm_host: SPGEMM_TIMING needs a plan the caller keeps; use spgemm_plan_create");
    return SPGEMM_ERR_INVALID_ARGUMENT;
  }
  if (device_only(A->row_ptr)) {
    set_last_error("spgemm_host: A's row_ptr is device memory; spgemm_host takes host arrays (see spgemm())");
    return SPGEMM_ERR_INVALID_ARGUMENT;
  }
  const int64_t m = A->nrows;
  // A's arrays are copied by its nnz, which its row pointers must agree with
  if (A->row_ptr[0] != 0 || A->row_ptr[m] != A->nnz) {
    set_last_error("spgemm_host: A's row_ptr must start at 0 and end at nnz");
    return SPGEMM_ERR_INVALID_CSR;
  }
  const size_t vs = dtype == SPGEMM_F32 ? 4 : 8;
  const bool same = A->row_ptr == B->row_ptr && A->col_idx == B->col_idx && A->vals == B->vals &&
                    A->nrows == B->nrows && A->ncols == B->ncols && A->nnz == B->nnz;

  HostCall h;
  h.st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;

  // 1. operands to the device
  const size_t a_rp = up256((size_t)(m + 1) * 4), a_ci = up256((size_t)A->nnz * 4), a_v = up256((size_t)A->nnz * vs);
  const size_t b_rp = same ? 0 : up256((size_t)(B->nrows + 1) * 4), b_ci = same ? 0 : up256((size_t)B->nnz * 4),
               b_v = same ? 0 : up256((size_t)B->nnz * vs);
  e = cudaMallocAsync(&h.d_ops, a_rp + a_ci + a_v + b_rp + b_ci + b_v, h.st);
  if (e != cudaSuccess) {
    h.d_ops = nullptr;
    return cuda_fail(e, "allocating operands");
  }
  char *ops = (char *)h.d_ops;
  spgemm_csr dA{m, A->ncols, A->nnz, (const int32_t *)ops, (const int32_t *)(ops + a_rp), ops + a_rp + a_ci};
  spgemm_csr dB = dA;
  if (!same) {
    char *ob = ops + a_rp + a_ci + a_v;
    dB = spgemm_csr{B->nrows, B->ncols, B->nnz, (const int32_t *)ob, (const int32_t *)(ob + b_rp), ob + b_rp + b_ci};
  }
  struct Copy {
    const void *dst;
    const void *src;
    size_t bytes;
  };
  std::vector<Copy> in = {{dA.row_ptr, A->row_ptr, (size_t)(m + 1) * 4},
                          {dA.col_idx, A->col_idx, (size_t)A->nnz * 4},
                          {dA.vals, A->vals, (size_t)A->nnz * vs}};
  if (!same) {
    in.push_back({dB.row_ptr, B->row_ptr, (size_t)(B->nrows + 1) * 4});
    in.push_back({dB.col_idx, B->col_idx, (size_t)B->nnz * 4});
    in.push_back({dB.vals, B->vals, (size_t)B->nnz * vs});
  }
  for (const Copy &c : in) {
    if (c.bytes == 0) continue;
    e = cudaMemcpyAsync(const_cast<void *>(c.dst), c.src, c.bytes, cudaMemcpyDefault, h.st);
    if (e != cudaSuccess) return cuda_fail(e, "copying operands to the device");
  }

  // 2. flop pass and symbolic phase of the whole product (the flop pass
  //    also checks both operands on the device): C's row pointers, nnz(C)
  int rc = spgemm_plan_create(&h.plan, &dA, &dB, dtype, flags, stream);
  if (rc != SPGEMM_OK) return rc;
  spgemm_stats ws;
  rc = spgemm_plan_stats(h.plan, &ws);
  if (rc != SPGEMM_OK) return rc;
  e = cudaMallocAsync(&h.d_rp, (size_t)(m + 1) * 4, h.st);
  if (e != cudaSuccess) {
    h.d_rp = nullptr;
    return cuda_fail(e, "allocating C's row pointers");
  }
  int32_t *d_rp = (int32_t *)h.d_rp;
  int64_t nnz = 0;
  rc = spgemm_symbolic(h.plan, d_rp, &nnz);
  if (rc != SPGEMM_OK) return rc;
  *nnz_c = nnz;

  // 3. C's row pointers on the host, and the row blocks from them
  int32_t *h_rp = (int32_t *)host_alloc((size_t)(m + 1) * 4, alloc_ctx);
  *c_row_ptr = h_rp;
  if (!h_rp) return SPGEMM_ERR_OUT_OF_MEMORY;
  e = cudaMemcpyAsync(h_rp, d_rp, (size_t)(m + 1) * 4, cudaMemcpyDefault, h.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h.st);
  if (e != cudaSuccess) return cuda_fail(e, "copying row pointers");
  int parts = row_blocks > 0 ? row_blocks : (ws.total_flop >= kRowBlockMinFlop ? kDefaultRowBlocks : 1);
  parts = (int)std::max<int64_t>(1, std::min<int64_t>(parts, m));
  std::vector<std::pair<int64_t, int64_t>> blocks;  // [r0, r1) of every non-empty block, in running order
  if (m > 0)
    for (const auto &bk : nnz_blocks(h_rp, m, parts))
      if (bk.second > bk.first) blocks.push_back(bk);
  const int nb = (int)blocks.size();

  // 4. C's columns and values: on the host through the callback, and on the device
  int32_t *h_ci = (int32_t *)host_alloc(nnz > 0 ? (size_t)nnz * 4 : 16, alloc_ctx);
  *c_col_idx = h_ci;
  void *h_cv = h_ci ? host_alloc(nnz > 0 ? (size_t)nnz * vs : 16, alloc_ctx) : nullptr;
  *c_vals = h_cv;
  if (!h_ci || !h_cv) return SPGEMM_ERR_OUT_OF_MEMORY;
  const size_t c_ci_b = up256((size_t)nnz * 4);
  e = cudaMallocAsync(&h.d_c, c_ci_b + up256((size_t)nnz * vs), h.st);
  if (e != cudaSuccess) {
    h.d_c = nullptr;
    return cuda_fail(e, "allocating C");
  }
  int32_t *d_ci = (int32_t *)h.d_c;
  char *d_cv = (char *)h.d_c + c_ci_b;

  // 5. numeric phases on the caller's stream, copies on the copy stream
  e = cudaStreamCreateWithFlags(&h.cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    h.cs = nullptr;
    return cuda_fail(e, "creating the copy stream");
  }
  h.events.assign(nb, nullptr);
  for (auto &ev : h.events) {
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      ev = nullptr;
      return cuda_fail(e, "creating events");
    }
  }
  for (int b = 0; b < nb; ++b) {
    const int64_t r0 = blocks[b].first, r1 = blocks[b].second;
    rc = spgemm_numeric_rows(h.plan, r0, r1, d_rp, d_ci, d_cv);
    if (rc != SPGEMM_OK) return rc;
    const int64_t e0 = h_rp[r0], n = (int64_t)h_rp[r1] - e0;
    if (n == 0) continue;
    e = cudaEventRecord(h.events[b], h.st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h.cs, h.events[b], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_ci + e0, d_ci + e0, (size_t)n * 4, cudaMemcpyDefault, h.cs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((char *)h_cv + e0 * vs, d_cv + e0 * vs, (size_t)n * vs, cudaMemcpyDefault, h.cs);
    if (e != cudaSuccess) return cuda_fail(e, "copying C to the host");
  }
  e = cudaStreamSynchronize(h.cs);
  if (e != cudaSuccess) return cuda_fail(e, "copy stream");
  // the numeric phase's device-side checks (reads the plan's counters)
  spgemm_stats s;
  return spgemm_plan_stats(h.plan, &s);
}
