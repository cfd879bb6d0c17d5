// Products whose operands and result live in host memory (spgemm_host).
//
// The rows of A are split into contiguous blocks by flop, the partition of
// paper Sec. 4.1 (Fig. "RowsToThreads", steps 1-2) applied to blocks
// instead of threads, and every block runs as a product of its own
// (one plan each).  The symbolic phases of all blocks give nnz(C), so C is
// allocated once; the numeric phases then run block after block on the
// caller's stream while a copy stream moves each finished block's columns
// and values to the host.  Rows of C are independent (Fig.
// "RowWise_SpGEMM"), so the result does not depend on the blocking.
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

// out[i] = rp[r0 + i] - rp[r0] for i = 0..n: the row pointers of rows
// r0 .. r0+n-1 of A, rebased to start at entry 0.
__global__ void k_rebase_rows(const int32_t *__restrict__ rp, int64_t r0, int64_t n, int32_t *__restrict__ out) {
  const int32_t base = rp[r0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = rp[r0 + i] - base;
}

// c_rp[r0 + i] = rp_b[i] + e0 for i = 0..n: a block's row pointers placed
// at its first row and first entry of C.
__global__ void k_place_rows(const int32_t *__restrict__ rp_b, int64_t n, int64_t r0, int32_t e0,
                             int32_t *__restrict__ c_rp) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
    c_rp[r0 + i] = rp_b[i] + e0;
}

unsigned grid_for(int64_t n) { return (unsigned)std::min<int64_t>((n + 256) / 256, 1024); }

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

// First row of each of `parts` row blocks; offs[parts] = m.  Block r gets
// a share of the flop proportional to 2^min(r, kShareCap): the shares
// double, so the first block, whose numeric phase no copy hides, is small,
// and every later block's numeric phase (at most twice the flop of the block
// before it) still runs under the copy of the block before it, which moves
// about 2.6 times as many bytes as the numeric phase writes per unit of time
// on GB300.  Block r starts at the first row whose exclusive flop prefix
// reaches its cumulative share (a lower-bound search over the prefix, as
// Fig. "RowsToThreads" does for threads); empty blocks are possible and
// skipped by the caller.
constexpr int kShareCap = 6;

std::vector<int64_t> flop_blocks(const std::vector<int64_t> &flop, int parts) {
  const int64_t m = (int64_t)flop.size();
  std::vector<int64_t> pre(m + 1, 0);
  for (int64_t i = 0; i < m; ++i) pre[i + 1] = pre[i] + flop[i];
  const __int128 total = pre[m];
  std::vector<__int128> cum(parts + 1, 0);  // cumulative shares
  for (int r = 0; r < parts; ++r) cum[r + 1] = cum[r] + ((__int128)1 << std::min(r, kShareCap));
  std::vector<int64_t> offs(parts + 1, 0);
  offs[parts] = m;
  for (int r = 1; r < parts; ++r) {
    const int64_t target = (int64_t)(total * cum[r] / cum[parts]);
    offs[r] = std::lower_bound(pre.begin(), pre.begin() + m, target) - pre.begin();
    offs[r] = std::max(offs[r], offs[r - 1]);
  }
  return offs;
}

// Everything the call holds on the device, released in one place.
struct HostCall {
  cudaStream_t st = nullptr, cs = nullptr;
  std::vector<spgemm_plan_t> plans;
  std::vector<cudaEvent_t> events;
  void *d_ops = nullptr;    // A (and B) on the device
  void *d_rows = nullptr;   // rebased A row pointers and per-block C row pointers
  void *d_c = nullptr;      // C: row pointers, columns, values
  ~HostCall() {
    if (cs) cudaStreamSynchronize(cs);
    for (spgemm_plan_t p : plans) spgemm_plan_destroy(p);
    for (cudaEvent_t e : events) cudaEventDestroy(e);
    if (d_c) cudaFreeAsync(d_c, st);
    if (d_rows) cudaFreeAsync(d_rows, st);
    if (d_ops) cudaFreeAsync(d_ops, st);
    if (cs) cudaStreamDestroy(cs);
  }
};

constexpr int kDefaultRowBlocks = 3;
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
  // the blocks index A's arrays from its host row pointers: check them first
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

  // 2. flop pass of the whole product (it also checks both operands on the
  //    device) and the row blocks
  spgemm_plan_t whole = nullptr;
  int rc = spgemm_plan_create(&whole, &dA, &dB, dtype, flags, stream);
  if (rc != SPGEMM_OK) return rc;
  h.plans.push_back(whole);
  spgemm_stats ws;
  rc = spgemm_plan_stats(whole, &ws);
  if (rc != SPGEMM_OK) return rc;
  int parts = row_blocks > 0 ? row_blocks : (ws.total_flop >= kRowBlockMinFlop ? kDefaultRowBlocks : 1);
  parts = (int)std::max<int64_t>(1, std::min<int64_t>(parts, m));
  std::vector<int64_t> offs = {0, m};
  if (parts > 1) {
    int64_t *d_flop = nullptr;
    e = cudaMallocAsync((void **)&d_flop, (size_t)m * 8, h.st);
    if (e != cudaSuccess) return cuda_fail(e, "allocating the flop array");
    std::vector<int64_t> flop(m);
    rc = spgemm_plan_row_flop(whole, d_flop);
    if (rc == SPGEMM_OK) {
      e = cudaMemcpyAsync(flop.data(), d_flop, (size_t)m * 8, cudaMemcpyDeviceToHost, h.st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h.st);
    }
    cudaFreeAsync(d_flop, h.st);
    if (rc != SPGEMM_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "reading the row flop");
    offs = flop_blocks(flop, parts);
    spgemm_plan_destroy(whole);
    h.plans.clear();
  }
  const bool keep_whole = parts == 1;  // the whole product is the only block
  std::vector<std::pair<int64_t, int64_t>> blocks;  // [r0, r1) of every non-empty block
  for (size_t r = 0; r + 1 < offs.size(); ++r)
    if (offs[r + 1] > offs[r]) blocks.push_back({offs[r], offs[r + 1]});
  const int nb = (int)blocks.size();

  // 3. symbolic phase of every block: per-block C row pointers, nnz(C)
  //    d_rows: rebased A row pointers of every block, then C's per block
  const size_t rows_total = (size_t)(m + nb);
  e = cudaMallocAsync(&h.d_rows, 2 * up256(rows_total * 4), h.st);
  if (e != cudaSuccess) {
    h.d_rows = nullptr;
    return cuda_fail(e, "allocating block row pointers");
  }
  int32_t *a_rows = (int32_t *)h.d_rows;
  int32_t *c_rows = (int32_t *)((char *)h.d_rows + up256(rows_total * 4));
  std::vector<int64_t> row_at(nb), nnz_b(nb), first(nb + 1, 0);
  int64_t at = 0;
  for (int b = 0; b < nb; ++b) {
    const int64_t r0 = blocks[b].first, rows = blocks[b].second - r0;
    row_at[b] = at;
    if (!keep_whole) {
      const int64_t e0 = A->row_ptr[r0], e1 = A->row_ptr[r0 + rows];
      if (e0 < 0 || e1 < e0 || e1 > A->nnz) {
        set_last_error("spgemm_host: A's row_ptr is not monotone");
        return SPGEMM_ERR_INVALID_CSR;
      }
      k_rebase_rows<<<grid_for(rows), 256, 0, h.st>>>(dA.row_ptr, r0, rows, a_rows + at);
      e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e, "rebasing row pointers");
      const spgemm_csr Ab{rows, A->ncols, e1 - e0, a_rows + at, dA.col_idx + e0, (const char *)dA.vals + e0 * vs};
      spgemm_plan_t p = nullptr;
      rc = spgemm_plan_create(&p, &Ab, &dB, dtype, flags, stream);
      if (rc != SPGEMM_OK) return rc;
      h.plans.push_back(p);
    }
    int64_t nz = 0;
    rc = spgemm_symbolic(h.plans[b], c_rows + at, &nz);
    if (rc != SPGEMM_OK) return rc;
    nnz_b[b] = nz;
    first[b + 1] = first[b] + nz;
    at += rows + 1;
  }
  const int64_t nnz = first[nb];
  if (nnz > INT32_MAX) {
    set_last_error("spgemm_host: nnz(C) exceeds int32 indexing");
    return SPGEMM_ERR_INDEX_OVERFLOW;
  }
  *nnz_c = nnz;

  // 4. C: on the host through the callback, and on the device
  int32_t *h_rp = (int32_t *)host_alloc((size_t)(m + 1) * 4, alloc_ctx);
  *c_row_ptr = h_rp;
  if (!h_rp) return SPGEMM_ERR_OUT_OF_MEMORY;
  int32_t *h_ci = (int32_t *)host_alloc(nnz > 0 ? (size_t)nnz * 4 : 16, alloc_ctx);
  *c_col_idx = h_ci;
  void *h_cv = h_ci ? host_alloc(nnz > 0 ? (size_t)nnz * vs : 16, alloc_ctx) : nullptr;
  *c_vals = h_cv;
  if (!h_ci || !h_cv) return SPGEMM_ERR_OUT_OF_MEMORY;
  const size_t c_rp_b = up256((size_t)(m + 1) * 4), c_ci_b = up256((size_t)nnz * 4);
  e = cudaMallocAsync(&h.d_c, c_rp_b + c_ci_b + up256((size_t)nnz * vs), h.st);
  if (e != cudaSuccess) {
    h.d_c = nullptr;
    return cuda_fail(e, "allocating C");
  }
  int32_t *d_rp = (int32_t *)h.d_c;
  int32_t *d_ci = (int32_t *)((char *)h.d_c + c_rp_b);
  char *d_cv = (char *)h.d_c + c_rp_b + c_ci_b;
  for (int b = 0; b < nb; ++b) {
    const int64_t rows = blocks[b].second - blocks[b].first;
    k_place_rows<<<grid_for(rows), 256, 0, h.st>>>(c_rows + row_at[b], rows, blocks[b].first, (int32_t)first[b],
                                                   d_rp);
  }
  if (nb == 0) {
    e = cudaMemsetAsync(d_rp, 0, (size_t)(m + 1) * 4, h.st);
    if (e != cudaSuccess) return cuda_fail(e, "clearing row pointers");
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "placing row pointers");

  // 5. numeric phases on the caller's stream, copies on the copy stream
  e = cudaStreamCreateWithFlags(&h.cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    h.cs = nullptr;
    return cuda_fail(e, "creating the copy stream");
  }
  h.events.assign(nb + 1, nullptr);
  for (auto &ev : h.events) {
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      ev = nullptr;
      return cuda_fail(e, "creating events");
    }
  }
  e = cudaEventRecord(h.events[nb], h.st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h.cs, h.events[nb], 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_rp, d_rp, (size_t)(m + 1) * 4, cudaMemcpyDefault, h.cs);
  if (e != cudaSuccess) return cuda_fail(e, "copying row pointers");
  for (int b = 0; b < nb; ++b) {
    rc = spgemm_numeric(h.plans[b], c_rows + row_at[b], d_ci + first[b], d_cv + first[b] * vs);
    if (rc != SPGEMM_OK) return rc;
    if (nnz_b[b] == 0) continue;
    e = cudaEventRecord(h.events[b], h.st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h.cs, h.events[b], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h_ci + first[b], d_ci + first[b], (size_t)nnz_b[b] * 4, cudaMemcpyDefault, h.cs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync((char *)h_cv + first[b] * vs, d_cv + first[b] * vs, (size_t)nnz_b[b] * vs,
                          cudaMemcpyDefault, h.cs);
    if (e != cudaSuccess) return cuda_fail(e, "copying C to the host");
  }
  e = cudaStreamSynchronize(h.cs);
  if (e != cudaSuccess) return cuda_fail(e, "copy stream");
  // device-side checks of every block (reads each plan's counters)
  for (spgemm_plan_t p : h.plans) {
    spgemm_stats s;
    rc = spgemm_plan_stats(p, &s);
    if (rc != SPGEMM_OK) return rc;
  }
  return SPGEMM_OK;
}
