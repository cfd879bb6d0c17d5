// Batched products: C_p = A_p * B_p for p = 0 .. P-1 in one plan.
//
// The P products are independent, so they form one product of block-
// diagonal operands: A = diag(A_0, ..., A_{P-1}) and B = diag(B_0, ...),
// whose result is diag(C_0, ...).  k_batch_pack builds the packed operands
// on the device (row pointers shifted by the entries of the products before,
// A's columns by the rows of B before, B's columns by the columns of B
// before, values copied), the regular plan runs the whole batch with the
// same number of kernel launches and host synchronisations as one product,
// and k_batch_unpack turns C's column indices back into each product's own
// columns.  Product p's rows of C are rows row_off[p] .. row_off[p+1]-1 of
// the packed C.
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace sg {

struct BatchDev {
  spgemm_csr a, b;
  long long a_row, a_nnz, b_row, b_nnz, b_col;  // offsets of this product in the packed operands
  long long chunk0;                              // first pack chunk of this product
};

// Elements of each operand array one block copies: a product of n elements
// in its largest array gets ceil(n / kPackChunk) blocks, so the copy of a
// large product spreads over the GPU instead of one SM.
constexpr int64_t kPackChunk = 8192;
constexpr int kPackUnroll = 8;

int64_t pack_chunks(const spgemm_csr &a, const spgemm_csr &b) {
  int64_t n = a.nrows + 1;
  if (a.nnz > n) n = a.nnz;
  if (b.nrows + 1 > n) n = b.nrows + 1;
  if (b.nnz > n) n = b.nnz;
  return (n + kPackChunk - 1) / kPackChunk;
}

// dst[i] = op(src[i], i) for i in [lo, hi): kPackUnroll loads in flight per
// thread before the stores.
template <typename W, typename Op>
__device__ __forceinline__ void pack_range(const W *__restrict__ src, W *__restrict__ dst, int64_t lo, int64_t hi,
                                           Op op) {
  for (int64_t base = lo + threadIdx.x; base < hi; base += (int64_t)blockDim.x * kPackUnroll) {
    W v[kPackUnroll];
#pragma unroll
    for (int u = 0; u < kPackUnroll; ++u) {
      const int64_t i = base + (int64_t)u * blockDim.x;
      if (i < hi) v[u] = src[i];
    }
#pragma unroll
    for (int u = 0; u < kPackUnroll; ++u) {
      const int64_t i = base + (int64_t)u * blockDim.x;
      if (i < hi) dst[i] = op(v[u], i);
    }
  }
}

// Copies one operand (row pointers shifted by `nnz_off`, column indices by
// `col_off`, values as words) of a product: chunk `c` of each array.
template <typename W>
__device__ __forceinline__ void pack_operand(const spgemm_csr &m, int64_t c, long long row_at, long long nnz_off,
                                             long long col_off, int32_t *rp, int32_t *ci, unsigned char *vals,
                                             uint32_t *err) {
  const int64_t lo = c * kPackChunk;
  const int32_t nnz = (int32_t)m.nnz;
  const int64_t ncols = m.ncols;
  // row pointers 0..nrows are checked; 0..nrows-1 are written (the packed
  // array's last entry is written by the host)
  {
    const int64_t hi = lo + kPackChunk < m.nrows + 1 ? lo + kPackChunk : m.nrows + 1;
    const int64_t nrows = m.nrows;
    pack_range<int32_t>(m.row_ptr, rp + row_at, lo, hi < nrows ? hi : nrows, [&](int32_t x, int64_t) {
      if (x < 0 || x > nnz) raise_err(err, kErrCsr);
      return (int32_t)(x + nnz_off);
    });
    if (threadIdx.x == 0 && lo == 0 && m.row_ptr[0] != 0) raise_err(err, kErrCsr);
    if (threadIdx.x == 0 && lo <= nrows && nrows < hi && m.row_ptr[nrows] != nnz) raise_err(err, kErrCsr);
  }
  const int64_t hi = lo + kPackChunk < m.nnz ? lo + kPackChunk : m.nnz;
  if (lo >= hi) return;
  pack_range<int32_t>(m.col_idx, ci + nnz_off, lo, hi, [&](int32_t c2, int64_t) {
    if ((uint64_t)(int64_t)c2 >= (uint64_t)ncols) raise_err(err, kErrCsr);
    return (int32_t)(c2 + col_off);
  });
  pack_range<W>(static_cast<const W *>(m.vals), reinterpret_cast<W *>(vals) + nnz_off, lo, hi,
                [](W v, int64_t) { return v; });
}

// Block b copies chunk (b - chunk0[p]) of product p, the product found by a
// binary search over the products' first chunks; indices are checked.
__global__ void __launch_bounds__(256)
    k_batch_pack(const BatchDev *__restrict__ d, int64_t nprod, int vsize, int32_t *__restrict__ arp,
                 int32_t *__restrict__ aci, unsigned char *__restrict__ av, int32_t *__restrict__ brp,
                 int32_t *__restrict__ bci, unsigned char *__restrict__ bv, uint32_t *err) {
  const int64_t blk = blockIdx.x;
  int64_t lo = 0, hi = nprod - 1;  // last product whose first chunk is <= blk
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (d[mid].chunk0 <= blk) lo = mid;
    else hi = mid - 1;
  }
  const BatchDev &p = d[lo];
  const int64_t c = blk - p.chunk0;
  if (vsize == 8) {
    pack_operand<unsigned long long>(p.a, c, p.a_row, p.a_nnz, p.b_row, arp, aci, av, err);
    pack_operand<unsigned long long>(p.b, c, p.b_row, p.b_nnz, p.b_col, brp, bci, bv, err);
  } else {
    pack_operand<uint32_t>(p.a, c, p.a_row, p.a_nnz, p.b_row, arp, aci, av, err);
    pack_operand<uint32_t>(p.b, c, p.b_row, p.b_nnz, p.b_col, brp, bci, bv, err);
  }
}

// One warp per row of C: subtract the column offset of the row's product.
__global__ void __launch_bounds__(256)
    k_batch_unpack(const int32_t *__restrict__ c_rp, int32_t *__restrict__ c_ci, int64_t m,
                   const long long *__restrict__ row_off, const long long *__restrict__ col_off, int64_t nprod) {
  const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= m) return;
  int64_t lo = 0, hi = nprod - 1;  // last product whose first row is <= row
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (row_off[mid] <= row) lo = mid;
    else hi = mid - 1;
  }
  const int32_t off = (int32_t)col_off[lo];
  for (int32_t j = c_rp[row] + lane; j < c_rp[row + 1]; j += 32) c_ci[j] -= off;
}

}  // namespace sg

using namespace sg;

struct spgemm_batch_s {
  int64_t nprod;
  int dtype;
  cudaStream_t stream;
  spgemm_plan_t plan;
  void *ws;                 // packed operands, offsets, error word
  int32_t *arp, *aci, *brp, *bci;
  void *av, *bv;
  long long *d_row_off, *d_col_off;
  uint32_t *d_err;
  std::vector<long long> row_off;  // host copy, nprod + 1
  int64_t m, k;
  int state;  // 0 planned, 1 symbolic done, 2 numeric done
};

namespace {

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

int bad(const spgemm_csr &c) {
  return c.nrows < 0 || c.ncols < 0 || c.nnz < 0 || !c.row_ptr || (c.nnz > 0 && (!c.col_idx || !c.vals));
}

}  // namespace

extern "C" {

int spgemm_batch_create(spgemm_batch_t *out, int64_t nprod, const spgemm_csr *A, const spgemm_csr *B, int dtype,
                        unsigned flags, void *stream) {
  return spgemm_batch_create_tuned(out, nprod, A, B, dtype, flags, stream, nullptr);
}

int spgemm_batch_create_tuned(spgemm_batch_t *out, int64_t nprod, const spgemm_csr *A, const spgemm_csr *B,
                              int dtype, unsigned flags, void *stream, const spgemm_tuning *tuning) {
  NvtxRange nvtx("spgemm_batch_create");
  if (!out) return SPGEMM_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  set_last_error("");
  if (nprod < 1 || !A || !B) return SPGEMM_ERR_INVALID_ARGUMENT;
  if (dtype != SPGEMM_I64 && dtype != SPGEMM_F32 && dtype != SPGEMM_F64) return SPGEMM_ERR_INVALID_ARGUMENT;
  const int vsize = dtype == SPGEMM_F32 ? 4 : 8;
  std::vector<BatchDev> h((size_t)nprod);
  long long am = 0, an = 0, bm = 0, bn = 0, bk = 0, chunks = 0;
  for (int64_t p = 0; p < nprod; ++p) {
    if (bad(A[p]) || bad(B[p]) || A[p].ncols != B[p].nrows) {
      set_last_error("product " + std::to_string(p) + ": bad descriptor or inner dimensions differ");
      return SPGEMM_ERR_INVALID_ARGUMENT;
    }
    h[p] = BatchDev{A[p], B[p], am, an, bm, bn, bk, chunks};
    chunks += pack_chunks(A[p], B[p]);
    am += A[p].nrows;
    an += A[p].nnz;
    bm += B[p].nrows;
    bn += B[p].nnz;
    bk += B[p].ncols;
  }
  if (am >= INT32_MAX || an > INT32_MAX || bm >= INT32_MAX || bn > INT32_MAX || bk > INT32_MAX ||
      chunks > INT32_MAX) {
    set_last_error("the packed batch exceeds int32 indexing");
    return SPGEMM_ERR_INDEX_OVERFLOW;
  }
  spgemm_batch_s *b = new (std::nothrow) spgemm_batch_s();
  if (!b) return SPGEMM_ERR_OUT_OF_MEMORY;
  b->nprod = nprod;
  b->dtype = dtype;
  b->stream = (cudaStream_t)stream;
  b->m = am;
  b->k = bk;
  b->row_off.resize((size_t)nprod + 1);
  std::vector<long long> col_off((size_t)nprod + 1);
  for (int64_t p = 0; p < nprod; ++p) {
    b->row_off[p] = h[p].a_row;
    col_off[p] = h[p].b_col;
  }
  b->row_off[nprod] = am;
  col_off[nprod] = bk;

  // workspace: descriptors, offsets, error word, packed A and B
  size_t off = 0;
  const size_t o_desc = off;
  off = up256(off + sizeof(BatchDev) * (size_t)nprod);
  const size_t o_roff = off;
  off = up256(off + 8 * ((size_t)nprod + 1));
  const size_t o_coff = off;
  off = up256(off + 8 * ((size_t)nprod + 1));
  const size_t o_err = off;
  off = up256(off + 4);
  const size_t o_arp = off;
  off = up256(off + 4 * ((size_t)am + 1));
  const size_t o_aci = off;
  off = up256(off + 4 * (size_t)an);
  const size_t o_av = off;
  off = up256(off + (size_t)vsize * an);
  const size_t o_brp = off;
  off = up256(off + 4 * ((size_t)bm + 1));
  const size_t o_bci = off;
  off = up256(off + 4 * (size_t)bn);
  const size_t o_bv = off;
  off = up256(off + (size_t)vsize * bn);
  cudaError_t e = cudaMallocAsync(&b->ws, off, b->stream);
  if (e != cudaSuccess) {
    delete b;
    set_last_error(std::string("batch workspace: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SPGEMM_ERR_OUT_OF_MEMORY : SPGEMM_ERR_DEVICE;
  }
  char *w = (char *)b->ws;
  BatchDev *d_desc = (BatchDev *)(w + o_desc);
  b->d_row_off = (long long *)(w + o_roff);
  b->d_col_off = (long long *)(w + o_coff);
  b->d_err = (uint32_t *)(w + o_err);
  b->arp = (int32_t *)(w + o_arp);
  b->aci = (int32_t *)(w + o_aci);
  b->av = w + o_av;
  b->brp = (int32_t *)(w + o_brp);
  b->bci = (int32_t *)(w + o_bci);
  b->bv = w + o_bv;
  const int32_t a_end = (int32_t)an, b_end = (int32_t)bn;
  e = cudaMemcpyAsync(d_desc, h.data(), sizeof(BatchDev) * (size_t)nprod, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_row_off, b->row_off.data(), 8 * ((size_t)nprod + 1), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_col_off, col_off.data(), 8 * ((size_t)nprod + 1), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, 4, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->arp + am, &a_end, 4, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->brp + bm, &b_end, 4, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) {
    k_batch_pack<<<(unsigned)chunks, 256, 0, b->stream>>>(d_desc, nprod, vsize, b->arp, b->aci,
                                                           (unsigned char *)b->av, b->brp, b->bci,
                                                           (unsigned char *)b->bv, b->d_err);
    e = cudaGetLastError();
  }
  uint32_t err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, b->d_err, 4, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess || err) {
    cudaFreeAsync(b->ws, b->stream);
    delete b;
    if (e != cudaSuccess) {
      set_last_error(std::string("batch packing: ") + cudaGetErrorString(e));
      return SPGEMM_ERR_DEVICE;
    }
    set_last_error("a product of the batch has an index out of range or a malformed row_ptr");
    return SPGEMM_ERR_INVALID_CSR;
  }
  spgemm_csr pa{am, bm, an, b->arp, b->aci, b->av};
  spgemm_csr pb{bm, bk, bn, b->brp, b->bci, b->bv};
  int rc = spgemm_plan_create_tuned(&b->plan, &pa, &pb, dtype, flags, stream, tuning);
  if (rc != SPGEMM_OK) {
    cudaFreeAsync(b->ws, b->stream);
    delete b;
    return rc;
  }
  // a row of the packed C spans at most its own product's columns: the block
  // bins' sort window is sized from the widest product, not the packed k
  int64_t widest = 0;
  for (int64_t q = 0; q < nprod; ++q) widest = B[q].ncols > widest ? B[q].ncols : widest;
  b->plan->span_cols = widest;
  b->state = 0;
  *out = b;
  return SPGEMM_OK;
}

int spgemm_batch_symbolic(spgemm_batch_t b, int32_t *c_row_ptr, int64_t *nnz_c, int64_t *row_off) {
  if (!b) return SPGEMM_ERR_INVALID_ARGUMENT;
  if (b->state != 0) return SPGEMM_ERR_BAD_STATE;
  int rc = spgemm_symbolic(b->plan, c_row_ptr, nnz_c);
  if (rc != SPGEMM_OK) return rc;
  if (row_off)
    for (int64_t p = 0; p <= b->nprod; ++p) row_off[p] = b->row_off[p];
  b->state = 1;
  return SPGEMM_OK;
}

int spgemm_batch_numeric(spgemm_batch_t b, const int32_t *c_row_ptr, int32_t *c_col_idx, void *c_vals) {
  if (!b) return SPGEMM_ERR_INVALID_ARGUMENT;
  if (b->state != 1) return SPGEMM_ERR_BAD_STATE;
  int rc = spgemm_numeric(b->plan, c_row_ptr, c_col_idx, c_vals);
  if (rc != SPGEMM_OK) return rc;
  if (b->m > 0 && c_col_idx) {
    KernelScope ks(b->plan, "batch_unpack");
    k_batch_unpack<<<(unsigned)((b->m + 7) / 8), 256, 0, b->stream>>>(c_row_ptr, c_col_idx, b->m, b->d_row_off,
                                                                      b->d_col_off, b->nprod);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_last_error(std::string("batch unpack: ") + cudaGetErrorString(e));
      return SPGEMM_ERR_DEVICE;
    }
  }
  b->state = 2;
  return SPGEMM_OK;
}

spgemm_plan_t spgemm_batch_plan(spgemm_batch_t b) { return b ? b->plan : nullptr; }

int spgemm_batch_destroy(spgemm_batch_t b) {
  if (!b) return SPGEMM_OK;
  spgemm_plan_destroy(b->plan);
  if (b->ws) cudaFreeAsync(b->ws, b->stream);
  delete b;
  return SPGEMM_OK;
}

}  // extern "C"
