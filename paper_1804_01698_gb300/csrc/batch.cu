// Batched products: C_p = A_p * B_p for p = 0 .. P-1 in one plan.
//
// The P products are independent, so they form one product of block-
// diagonal operands: A = diag(A_0, ..., A_{P-1}) and B = diag(B_0, ...),
// whose result is diag(C_0, ...).  k_batch_pack builds the packed operands
// on the device (row pointers shifted by the entries of the products before,
// A's columns by the rows of B before, B's columns by the columns of B
// before, values copied), the regular plan runs the whole batch with the
// same number of kernel launches and host synchronisations as one product,
// and the numeric kernels store each row's columns less its product's
// column offset (cbase, written by k_batch_pack), so C holds every
// product's own columns.  Product p's rows of C are rows row_off[p] ..
// row_off[p+1]-1 of the packed C.
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
                 int32_t *__restrict__ bci, unsigned char *__restrict__ bv, int32_t *__restrict__ cbase,
                 uint32_t *err) {
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
  // the rows of C this product's rows of A produce store its own columns
  const int64_t r0 = c * kPackChunk, r1 = r0 + kPackChunk < p.a.nrows ? r0 + kPackChunk : p.a.nrows;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) cbase[p.a_row + r] = (int32_t)p.b_col;
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
  int32_t *cbase;           // per packed row: the column offset of its product (Args::col_base)
  uint32_t *d_err;
  std::vector<long long> row_off;  // host copy, nprod + 1
  int64_t m, k;
  int state;  // 0 planned, 1 symbolic done, 2 numeric done
  // packing (batch graphs repack on every launch)
  sg::BatchDev *d_desc;
  int64_t chunks, an, bm, bn, widest;
  int vsize;
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

}  // extern "C"

namespace sg {

// Checks the products, allocates the packed operands and their offsets and
// packs them once (synchronising `stream` to read the packing's error word).
// The batch has no plan yet.
int batch_pack(spgemm_batch_s **out, int64_t nprod, const spgemm_csr *A, const spgemm_csr *B, int dtype,
               cudaStream_t stream) {
  *out = nullptr;
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
  const size_t o_cbase = off;
  off = up256(off + 4 * (size_t)am);
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
  b->cbase = (int32_t *)(w + o_cbase);
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
                                                           (unsigned char *)b->bv, b->cbase, b->d_err);
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
  b->chunks = chunks;
  b->d_desc = d_desc;
  b->vsize = vsize;
  b->an = an;
  b->bm = bm;
  b->bn = bn;
  int64_t widest = 0;
  for (int64_t q = 0; q < nprod; ++q) widest = B[q].ncols > widest ? B[q].ncols : widest;
  b->widest = widest;
  *out = b;
  return SPGEMM_OK;
}

// The packing kernel again (the operands' current contents), on `st`.
cudaError_t batch_repack(spgemm_batch_s *b, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(b->d_err, 0, 4, st);
  if (e != cudaSuccess) return e;
  k_batch_pack<<<(unsigned)b->chunks, 256, 0, st>>>(b->d_desc, b->nprod, b->vsize, b->arp, b->aci,
                                                      (unsigned char *)b->av, b->brp, b->bci, (unsigned char *)b->bv,
                                                      b->cbase, b->d_err);
  return cudaGetLastError();
}

void batch_free(spgemm_batch_s *b) {
  if (!b) return;
  if (b->plan) spgemm_plan_destroy(b->plan);
  if (b->ws) cudaFreeAsync(b->ws, b->stream);
  delete b;
}

}  // namespace sg

extern "C" {

int spgemm_batch_create_tuned(spgemm_batch_t *out, int64_t nprod, const spgemm_csr *A, const spgemm_csr *B,
                              int dtype, unsigned flags, void *stream, const spgemm_tuning *tuning) {
  NvtxRange nvtx("spgemm_batch_create");
  if (!out) return SPGEMM_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  set_last_error("");
  spgemm_batch_s *b = nullptr;
  int rc = batch_pack(&b, nprod, A, B, dtype, (cudaStream_t)stream);
  if (rc != SPGEMM_OK) return rc;
  spgemm_csr pa{b->m, b->bm, b->an, b->arp, b->aci, b->av};
  spgemm_csr pb{b->bm, b->k, b->bn, b->brp, b->bci, b->bv};
  rc = spgemm_plan_create_tuned(&b->plan, &pa, &pb, dtype, flags, stream, tuning);
  if (rc != SPGEMM_OK) {
    b->plan = nullptr;
    batch_free(b);
    return rc;
  }
  // a row of the packed C spans at most its own product's columns: the block
  // bins' sort window is sized from the widest product, not the packed k
  b->plan->span_cols = b->widest;
  b->plan->col_base = b->cbase;
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
  b->state = 2;
  return SPGEMM_OK;
}

spgemm_plan_t spgemm_batch_plan(spgemm_batch_t b) { return b ? b->plan : nullptr; }

int spgemm_batch_destroy(spgemm_batch_t b) {
  batch_free(b);
  return SPGEMM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batch graphs: every product of a batch in ONE CUDA graph launch.
//
// The products are split into waves (consecutive products whose C fits
// int32 indexing and a stated pool).  Each wave keeps its packed operands, a
// graph-mode plan (sized by a planning pass at creation: no host reads of
// counts while it runs) and its pool for C.  The graph holds, for every
// wave: the packing of its products, the flop pass, the symbolic bins, the
// row_ptr scan, the numeric bins (storing every product's own columns) and
// the copy of the per-product entry counts and error words to pinned host
// memory.  A launch
// is one cudaGraphLaunch on the caller's stream, with no host
// synchronisation until the caller waits for it; it recomputes every
// product from the current contents of the operands, so new values, or a
// new structure that fits the planned capacities, give new products.

namespace sg {

// out[p] = entries of C before product p's first row (c_rp[row_off[p]]),
// p = 0 .. nprod (so out[nprod] = nnz of the wave's C).
__global__ void k_wave_prod_nnz(const int32_t *__restrict__ c_rp, const long long *__restrict__ row_off, int64_t nprod,
                                const uint32_t *abort, long long *__restrict__ out) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p > nprod) return;
  const bool stop = *(volatile const uint32_t *)abort & (kErrOverflow | kErrCapacity);
  out[p] = stop ? 0 : c_rp[row_off[p]];
}

// Sum of v over the rows of each product (planning pass): block p, rows
// row_off[p] .. row_off[p+1]-1.
template <typename V>
__global__ void __launch_bounds__(256)
    k_prod_sum(const V *__restrict__ v, const long long *__restrict__ row_off, long long *__restrict__ out) {
  __shared__ long long red[33];
  const int64_t p = blockIdx.x;
  long long s = 0;
  for (int64_t r = row_off[p] + threadIdx.x; r < row_off[p + 1]; r += blockDim.x) s += v[r];
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[p] = s;
}

}  // namespace sg

struct GraphWave {
  int64_t p0 = 0, p1 = 0;          // products p0 .. p1-1
  spgemm_batch_s *b = nullptr;     // packed operands and offsets (its own plan freed)
  spgemm_plan_s *plan = nullptr;   // graph-mode plan on the packed operands
  void *cws = nullptr;             // C: row_ptr (m+1), col_idx and values (nnz_cap each)
  int32_t *c_rp = nullptr, *c_ci = nullptr;
  void *c_v = nullptr;
  int64_t nnz_cap = 0;
  long long *d_pnnz = nullptr;     // entries before each product (p1-p0+1)
};

struct spgemm_bgraph_s {
  int64_t nprod = 0;
  int dtype = 0;
  cudaStream_t stream = nullptr;
  std::vector<GraphWave> waves;
  std::vector<int64_t> wave_of;        // per product
  cudaGraphExec_t exec = nullptr;
  int64_t kernel_nodes = 0;
  long long *h_pnnz = nullptr;         // pinned: per wave, p1-p0+1 counts (written by the graph)
  uint32_t *h_err = nullptr;           // pinned: per wave, plan and packing error words
  std::vector<int64_t> h_off;          // per wave, offset into h_pnnz
  size_t bytes = 0;
  bool launched = false;
  cudaStream_t last_stream = nullptr;
};

namespace {

using sg::GraphCaps;

// Products [p0, p1) fit one packed batch (int32 indexing of its operands).
bool packable(const spgemm_csr *A, const spgemm_csr *B, int64_t p0, int64_t p1) {
  long long am = 0, an = 0, bm = 0, bn = 0, bk = 0, ch = 0;
  for (int64_t p = p0; p < p1; ++p) {
    am += A[p].nrows;
    an += A[p].nnz;
    bm += B[p].nrows;
    bn += B[p].nnz;
    bk += B[p].ncols;
    ch += sg::pack_chunks(A[p], B[p]);
  }
  return am < INT32_MAX && an <= INT32_MAX && bm < INT32_MAX && bn <= INT32_MAX && bk <= INT32_MAX && ch <= INT32_MAX;
}

// What the planning pass learns about the products of one packed group.
struct Planned {
  std::vector<long long> flop, nnz;  // per product
  int64_t max_flop = 0, max_bound = 0, max_nnz = 0;
};

// Planning pass of products [p0, p1): pack them, run the flop pass and the
// symbolic phase once (host-driven, no bitmap rows so that the heavy rows
// show their global-table sizes), and read per-product flop and nnz(C).
int plan_group(const spgemm_csr *A, const spgemm_csr *B, int64_t p0, int64_t p1, int dtype, unsigned flags,
               cudaStream_t st, const spgemm_tuning *tuning, Planned *out) {
  spgemm_tuning t{};
  if (tuning) t = *tuning;
  t.bitmap_min_bound = -1;
  t.long_row_min = -1;
  t.max_nnz_c = 0;
  spgemm_batch_s *b = nullptr;
  const int64_t np = p1 - p0;
  int rc = spgemm_batch_create_tuned(&b, np, A + p0, B + p0, dtype, flags & ~SPGEMM_TIMING, st, &t);
  if (rc != SPGEMM_OK) return rc;
  int32_t *rp = nullptr;
  long long *sums = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&rp, (size_t)(b->m + 1) * 4, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&sums, (size_t)np * 2 * 8, st);
  if (e != cudaSuccess) {
    if (rp) cudaFreeAsync(rp, st);
    sg::batch_free(b);
    sg::set_last_error(std::string("batch graph planning: ") + cudaGetErrorString(e));
    return SPGEMM_ERR_OUT_OF_MEMORY;
  }
  int64_t nnz = 0;
  rc = spgemm_batch_symbolic(b, rp, &nnz, nullptr);
  // a group whose C passes int32 indexing still has every row's count
  if (rc == SPGEMM_ERR_INDEX_OVERFLOW) rc = SPGEMM_OK;
  if (rc == SPGEMM_OK) {
    spgemm_plan_s *p = b->plan;
    sg::k_prod_sum<int32_t><<<(unsigned)np, 256, 0, st>>>(p->nnz_row, b->d_row_off, sums);
    sg::k_prod_sum<int64_t><<<(unsigned)np, 256, 0, st>>>(p->flop, b->d_row_off, sums + np);
    out->nnz.resize((size_t)np);
    out->flop.resize((size_t)np);
    e = cudaMemcpyAsync(out->nnz.data(), sums, (size_t)np * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out->flop.data(), sums + np, (size_t)np * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      sg::set_last_error(std::string("batch graph planning: ") + cudaGetErrorString(e));
      rc = SPGEMM_ERR_DEVICE;
    }
    out->max_flop = p->max_flop;
    out->max_bound = (int64_t)p->hc->max_bound_global;
    out->max_nnz = (int64_t)p->hc->max_nnz_global;
  }
  cudaFreeAsync(sums, st);
  cudaFreeAsync(rp, st);
  sg::batch_free(b);
  return rc;
}

// Planning pass of one wave on its packed operands (host-driven, no bitmap
// rows): the bins' row counts, the largest heavy row, the flop and nnz(C)
// the graph-mode plan is sized for.  The planning plan is freed.
int plan_wave(const spgemm_csr *pa, const spgemm_csr *pb, int dtype, unsigned flags, cudaStream_t st,
              const spgemm_tuning *tuning, GraphCaps *c) {
  spgemm_tuning t{};
  if (tuning) t = *tuning;
  t.bitmap_min_bound = -1;
  t.long_row_min = -1;
  t.max_nnz_c = 0;
  spgemm_plan_t hp = nullptr;
  int rc = spgemm_plan_create_tuned(&hp, pa, pb, dtype, flags & ~SPGEMM_TIMING, st, &t);
  if (rc != SPGEMM_OK) return rc;
  int32_t *rp = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&rp, (size_t)(pa->nrows + 1) * 4, st);
  int64_t nnz = 0;
  if (e != cudaSuccess) rc = SPGEMM_ERR_OUT_OF_MEMORY;
  if (rc == SPGEMM_OK) rc = spgemm_symbolic(hp, rp, &nnz);
  if (rc == SPGEMM_OK) {
    c->total_flop = hp->total_flop;
    c->max_flop = hp->max_flop;
    c->max_bound = (int64_t)hp->hc->max_bound_global;
    c->max_nnz = (int64_t)hp->hc->max_nnz_global;
    c->nnz_cap = nnz;
    for (int b = 0; b < sg::kNumSymBins; ++b) c->sym_rows[b] = hp->sym_count[b];
    for (int b = 0; b < sg::kNumNumBins; ++b) c->num_rows[b] = hp->num_count[b];
  }
  if (rp) cudaFreeAsync(rp, st);
  spgemm_plan_destroy(hp);
  return rc;
}

void free_graph(spgemm_bgraph_s *g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  for (auto &w : g->waves) {
    if (w.plan) sg::plan_free(w.plan);
    if (w.cws) cudaFreeAsync(w.cws, g->stream);
    if (w.d_pnnz) cudaFreeAsync(w.d_pnnz, g->stream);
    sg::batch_free(w.b);
  }
  if (g->h_pnnz) cudaFreeHost(g->h_pnnz);
  if (g->h_err) cudaFreeHost(g->h_err);
  delete g;
}

}  // namespace

namespace {

// out[i] = in[i] - sub, i < n (one product's row pointers, rebased to 0).
__global__ void k_rebase_rp(const int32_t *__restrict__ in, int64_t n, int32_t sub, int32_t *__restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i] - sub;
}

// Captures every wave, in order, into one graph on a private stream (the
// caller's stream may be a default stream, which cannot be captured), and
// instantiates it.
int bgraph_capture(spgemm_bgraph_s *g) {
  cudaError_t e = cudaStreamSynchronize(g->stream);  // planning passes and allocations done
  size_t tot = 0;
  for (auto &w : g->waves) {
    g->h_off.push_back((int64_t)tot);
    tot += (size_t)(w.p1 - w.p0 + 1);
  }
  if (e == cudaSuccess) e = cudaMallocHost((void **)&g->h_pnnz, tot * 8);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&g->h_err, 2 * g->waves.size() * 4 + 4);
  if (e != cudaSuccess) {
    set_last_error(std::string("batch graph: ") + cudaGetErrorString(e));
    return SPGEMM_ERR_OUT_OF_MEMORY;
  }
  std::memset(g->h_pnnz, 0, tot * 8);
  std::memset(g->h_err, 0, 2 * g->waves.size() * 4 + 4);
  cudaStream_t cap = nullptr;
  e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    set_last_error(std::string("batch graph capture stream: ") + cudaGetErrorString(e));
    return SPGEMM_ERR_DEVICE;
  }
  for (auto &w : g->waves) {
    w.plan->stream = cap;
    w.b->stream = cap;
  }
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  cudaError_t el = cudaSuccess;
  for (size_t i = 0; i < g->waves.size() && e == cudaSuccess && el == cudaSuccess; ++i) {
    GraphWave &w = g->waves[i];
    const int64_t np = w.p1 - w.p0;
    const uint32_t *abort = &w.plan->dc->err;
    el = sg::batch_repack(w.b, cap);
    if (el == cudaSuccess) el = sg::plan_enqueue_graph(w.plan, w.c_rp, w.c_ci, w.c_v);
    if (el == cudaSuccess) {
      sg::k_wave_prod_nnz<<<(unsigned)((np + 256) / 256), 256, 0, cap>>>(w.c_rp, w.b->d_row_off, np, abort,
                                                                          w.d_pnnz);
      el = cudaGetLastError();
    }
    if (el == cudaSuccess)
      el = cudaMemcpyAsync(g->h_pnnz + g->h_off[i], w.d_pnnz, (size_t)(np + 1) * 8, cudaMemcpyDeviceToHost, cap);
    if (el == cudaSuccess) el = cudaMemcpyAsync(g->h_err + 2 * i, abort, 4, cudaMemcpyDeviceToHost, cap);
    if (el == cudaSuccess) el = cudaMemcpyAsync(g->h_err + 2 * i + 1, w.b->d_err, 4, cudaMemcpyDeviceToHost, cap);
  }
  cudaGraph_t graph = nullptr;
  if (e == cudaSuccess) e = cudaStreamEndCapture(cap, &graph);
  for (auto &w : g->waves) {
    w.plan->stream = g->stream;
    w.b->stream = g->stream;
  }
  if (e == cudaSuccess && el == cudaSuccess) {
    size_t n = 0;
    e = cudaGraphGetNodes(graph, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    if (e == cudaSuccess && n > 0) e = cudaGraphGetNodes(graph, nodes.data(), &n);
    for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++g->kernel_nodes;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, graph, 0);
  }
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cap);
  if (el != cudaSuccess || e != cudaSuccess) {
    g->exec = nullptr;
    set_last_error(std::string("batch graph capture: ") + cudaGetErrorString(el != cudaSuccess ? el : e));
    return SPGEMM_ERR_DEVICE;
  }
  return SPGEMM_OK;
}

}  // namespace

extern "C" {

int spgemm_bgraph_create(spgemm_bgraph_t *out, int64_t nprod, const spgemm_csr *A, const spgemm_csr *B, int dtype,
                         unsigned flags, void *stream, const spgemm_tuning *tuning, int64_t wave_nnz,
                         double pool_slack) {
  NvtxRange nvtx("spgemm_bgraph_create");
  if (!out) return SPGEMM_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  set_last_error("");
  if (nprod < 1 || !A || !B || wave_nnz < 0 || wave_nnz > INT32_MAX || !(pool_slack >= 0.0 && pool_slack <= 16.0))
    return SPGEMM_ERR_INVALID_ARGUMENT;
  if (flags & (SPGEMM_TIMING | SPGEMM_COUNT_PROBES)) {
    set_last_error("a batch graph replays captured kernels: SPGEMM_TIMING and SPGEMM_COUNT_PROBES do not apply");
    return SPGEMM_ERR_INVALID_ARGUMENT;
  }
  for (int64_t p = 0; p < nprod; ++p)
    if (bad(A[p]) || bad(B[p]) || A[p].ncols != B[p].nrows) {
      set_last_error("product " + std::to_string(p) + ": bad descriptor or inner dimensions differ");
      return SPGEMM_ERR_INVALID_ARGUMENT;
    }
  const int64_t limit = wave_nnz > 0 ? wave_nnz : INT32_MAX;
  cudaStream_t st = (cudaStream_t)stream;
  spgemm_bgraph_s *g = new (std::nothrow) spgemm_bgraph_s();
  if (!g) return SPGEMM_ERR_OUT_OF_MEMORY;
  g->nprod = nprod;
  g->dtype = dtype;
  g->stream = st;
  g->wave_of.assign((size_t)nprod, 0);
  int rc = SPGEMM_OK;
  // 1. groups that pack (int32 operands), planned one after another; waves:
  //    consecutive products of a group whose nnz(C) stays within the limit
  std::vector<std::pair<int64_t, int64_t>> waves;
  std::vector<GraphCaps> caps;
  for (int64_t g0 = 0; g0 < nprod && rc == SPGEMM_OK;) {
    int64_t g1 = g0 + 1;
    while (g1 < nprod && packable(A, B, g0, g1 + 1)) ++g1;
    if (!packable(A, B, g0, g1)) {
      set_last_error("product " + std::to_string(g0) + " alone exceeds int32 indexing");
      rc = SPGEMM_ERR_INDEX_OVERFLOW;
      break;
    }
    Planned pl;
    rc = plan_group(A, B, g0, g1, dtype, flags, st, tuning, &pl);
    for (int64_t p = g0; p < g1 && rc == SPGEMM_OK;) {
      GraphCaps c{};
      int64_t q = p, nnz = 0;
      while (q < g1 && nnz + pl.nnz[(size_t)(q - g0)] <= limit) nnz += pl.nnz[(size_t)(q++ - g0)];
      if (q == p) {
        set_last_error("product " + std::to_string(p) + ": nnz(C) exceeds the wave limit");
        rc = SPGEMM_ERR_INDEX_OVERFLOW;
        break;
      }
      for (int64_t r = p; r < q; ++r) {
        c.total_flop += pl.flop[(size_t)(r - g0)];
        c.span_cols = std::max<int64_t>(c.span_cols, B[r].ncols);
      }

      waves.push_back({p, q});
      caps.push_back(c);
      p = q;
    }
    g0 = g1;
  }
  // 2. per wave: packed operands, graph-mode plan, pool for C
  const size_t vs = dtype == SPGEMM_F32 ? 4 : 8;
  for (size_t w = 0; w < waves.size() && rc == SPGEMM_OK; ++w) {
    GraphWave gw;
    gw.p0 = waves[w].first;
    gw.p1 = waves[w].second;
    const int64_t np = gw.p1 - gw.p0;
    rc = sg::batch_pack(&gw.b, np, A + gw.p0, B + gw.p0, dtype, st);
    if (rc != SPGEMM_OK) break;
    spgemm_csr pa{gw.b->m, gw.b->bm, gw.b->an, gw.b->arp, gw.b->aci, gw.b->av};
    spgemm_csr pb{gw.b->bm, gw.b->k, gw.b->bn, gw.b->brp, gw.b->bci, gw.b->bv};
    rc = plan_wave(&pa, &pb, dtype, flags, st, tuning, &caps[w]);
    if (rc != SPGEMM_OK) break;
    caps[w].nnz_cap = std::min<int64_t>(INT32_MAX, (int64_t)((double)caps[w].nnz_cap * (1.0 + pool_slack)) + 1);
    rc = sg::plan_create_graph(&gw.plan, &pa, &pb, dtype, flags, st, tuning, caps[w]);
    if (rc == SPGEMM_OK) gw.plan->col_base = gw.b->cbase;
    gw.nnz_cap = caps[w].nnz_cap;
    const size_t o_ci = up256((size_t)(gw.b->m + 1) * 4);
    const size_t o_v = o_ci + up256((size_t)gw.nnz_cap * 4);
    const size_t bytes = o_v + up256((size_t)gw.nnz_cap * vs);
    if (rc == SPGEMM_OK) {
      cudaError_t e = cudaMallocAsync(&gw.cws, bytes, st);
      if (e == cudaSuccess) e = cudaMallocAsync((void **)&gw.d_pnnz, (size_t)(np + 1) * 8, st);
      if (e != cudaSuccess) {
        set_last_error(std::string("batch graph pools: ") + cudaGetErrorString(e));
        rc = SPGEMM_ERR_OUT_OF_MEMORY;
      } else {
        gw.c_rp = static_cast<int32_t *>(gw.cws);
        gw.c_ci = reinterpret_cast<int32_t *>(static_cast<char *>(gw.cws) + o_ci);
        gw.c_v = static_cast<char *>(gw.cws) + o_v;
        g->bytes += bytes;
      }
    }
    for (int64_t p = gw.p0; p < gw.p1; ++p) g->wave_of[(size_t)p] = (int64_t)g->waves.size();
    g->waves.push_back(gw);
  }
  if (rc == SPGEMM_OK) rc = bgraph_capture(g);
  if (rc != SPGEMM_OK) {
    cudaStreamSynchronize(st);
    free_graph(g);
    return rc;
  }
  *out = g;
  return SPGEMM_OK;
}

}  // extern "C"

extern "C" {

int spgemm_bgraph_launch(spgemm_bgraph_t g, void *stream) {
  if (!g || !g->exec) return SPGEMM_ERR_INVALID_ARGUMENT;
  const cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_last_error(std::string("batch graph launch: ") + cudaGetErrorString(e));
    return SPGEMM_ERR_DEVICE;
  }
  g->launched = true;
  g->last_stream = (cudaStream_t)stream;
  return SPGEMM_OK;
}

int spgemm_bgraph_wait(spgemm_bgraph_t g) {
  if (!g) return SPGEMM_ERR_INVALID_ARGUMENT;
  if (!g->launched) return SPGEMM_ERR_BAD_STATE;
  const cudaError_t e = cudaStreamSynchronize(g->last_stream);
  if (e != cudaSuccess) {
    set_last_error(std::string("batch graph: ") + cudaGetErrorString(e));
    return SPGEMM_ERR_DEVICE;
  }
  for (size_t i = 0; i < g->waves.size(); ++i) {
    const uint32_t pe = g->h_err[2 * i], be = g->h_err[2 * i + 1];
    const std::string at = "batch graph wave " + std::to_string(i) + ": ";
    if (be || (pe & kErrCsr)) {
      set_last_error(at + "a product has an index out of range or a malformed row_ptr");
      return SPGEMM_ERR_INVALID_CSR;
    }
    if (pe & (kErrOverflow | kErrCapacity)) {
      set_last_error(at + "C or one of its rows exceeds the capacity the graph was planned with");
      return SPGEMM_ERR_OUT_OF_MEMORY;
    }
    if (pe) {
      set_last_error(at + "device-side check failed (hash probe or atomic retry bound)");
      return SPGEMM_ERR_DEVICE;
    }
  }
  return SPGEMM_OK;
}

int spgemm_bgraph_product_nnz(spgemm_bgraph_t g, int64_t p, int64_t *nnz) {
  if (!g || !nnz || p < 0 || p >= g->nprod) return SPGEMM_ERR_INVALID_ARGUMENT;
  if (!g->launched) return SPGEMM_ERR_BAD_STATE;
  const size_t w = (size_t)g->wave_of[(size_t)p];
  const int64_t i = p - g->waves[w].p0;
  const long long *c = g->h_pnnz + g->h_off[w];
  *nnz = c[i + 1] - c[i];
  return SPGEMM_OK;
}

int spgemm_bgraph_product_copy(spgemm_bgraph_t g, int64_t p, int32_t *c_row_ptr, int32_t *c_col_idx, void *c_vals,
                               void *stream) {
  if (!g || !c_row_ptr || p < 0 || p >= g->nprod) return SPGEMM_ERR_INVALID_ARGUMENT;
  if (!g->launched) return SPGEMM_ERR_BAD_STATE;
  const size_t w = (size_t)g->wave_of[(size_t)p];
  const GraphWave &gw = g->waves[w];
  const int64_t i = p - gw.p0;
  const long long first = g->h_pnnz[g->h_off[w] + i];
  const long long nnz = g->h_pnnz[g->h_off[w] + i + 1] - first;
  if (nnz > 0 && (!c_col_idx || !c_vals)) return SPGEMM_ERR_INVALID_ARGUMENT;
  const int64_t row0 = gw.b->row_off[(size_t)i], rows = gw.b->row_off[(size_t)i + 1] - row0;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t vs = g->dtype == SPGEMM_F32 ? 4 : 8;
  const int64_t nb = (rows + 1 + 255) / 256;
  k_rebase_rp<<<(unsigned)(nb < 4096 ? nb : 4096), 256, 0, st>>>(gw.c_rp + row0, rows + 1, (int32_t)first, c_row_ptr);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && nnz > 0)
    e = cudaMemcpyAsync(c_col_idx, gw.c_ci + first, (size_t)nnz * 4, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && nnz > 0)
    e = cudaMemcpyAsync(c_vals, static_cast<char *>(gw.c_v) + (size_t)first * vs, (size_t)nnz * vs,
                        cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) {
    set_last_error(std::string("batch graph product copy: ") + cudaGetErrorString(e));
    return SPGEMM_ERR_DEVICE;
  }
  return SPGEMM_OK;
}

int spgemm_bgraph_info(spgemm_bgraph_t g, int64_t *waves, int64_t *kernel_nodes, int64_t *bytes) {
  if (!g) return SPGEMM_ERR_INVALID_ARGUMENT;
  if (waves) *waves = (int64_t)g->waves.size();
  if (kernel_nodes) *kernel_nodes = g->kernel_nodes;
  if (bytes) *bytes = (int64_t)g->bytes;
  return SPGEMM_OK;
}

int spgemm_bgraph_destroy(spgemm_bgraph_t g) {
  if (!g) return SPGEMM_OK;
  if (g->launched) cudaStreamSynchronize(g->last_stream);
  free_graph(g);
  return SPGEMM_OK;
}

}  // extern "C"
