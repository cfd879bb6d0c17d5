// Long rows of B for the bitmap rows of A.
//
// A heavy row of A (one that takes the column-bitmap path) meets the same
// few long rows of B again and again: in R-MAT A*A at scale 16, 119 rows of
// B with 1024 or more entries carry two thirds of all products.  For those
// rows the plan keeps
//   * the column bitmap of the row (words = ceil(k/32) words), which the
//     symbolic phase ORs word by word into the bitmap of C's row, and
//   * a copy of the row's (column, value) entries sorted by column, with the
//     start of each of kLongRanges column ranges in it.  The ranges split
//     the columns into intervals of equal mass over all long rows (R-MAT
//     columns are skewed: the low ones are far denser), and warp w of a
//     numeric bitmap block owns its share of the ranges for every long row:
//     its lanes take consecutive entries of one long row's slice at a time
//     (distinct columns, so distinct output ranks), and add their products
//     with plain shared-memory loads and stores instead of atomics.
// A long row with a repeated column (a precondition violation that the
// method still sums) is left to the atomic path.  The result is the product
// the paper defines (Fig. "RowWise_SpGEMM"): only the order in which each
// row's products are visited changes.
//
//   k_long_mark     per row of B: long (entries >= long_min) or not; long
//                   rows get an index d and a range of the copy
//   k_long_build    per long row: bitmap, sorted copy and its sources,
//                   word histogram of its columns
//   k_long_ranges   the column ranges: quantiles of the word histogram
//   k_long_offsets  per long row: the start of every range in its copy
//   k_long_vals     before every numeric phase: the copies' values from B
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace sg {

__global__ void __launch_bounds__(256)
    k_long_mark(const int32_t *__restrict__ brp, int64_t n, int64_t nnz_b, int64_t long_min, int64_t cap,
                int32_t *__restrict__ lmap, int32_t *__restrict__ lrow, int32_t *__restrict__ lbase,
                DevCounters *dc) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int64_t b0 = brp[k], b1 = brp[k + 1];
  int32_t d = -1;
  // a malformed row is never long (the flop pass reports it when A selects it)
  if (0 <= b0 && b0 <= b1 && b1 <= nnz_b && b1 - b0 >= long_min) {
    const unsigned long long idx = atomicAdd(&dc->n_long, 1ull);
    if ((int64_t)idx < cap) {
      d = (int32_t)idx;
      lrow[d] = (int32_t)k;
      lbase[d] = (int32_t)atomicAdd(&dc->long_tot, (unsigned long long)(b1 - b0));
    }
  }
  lmap[k] = d;
}

// Exclusive prefix of popc over `words` bitmap words in shared memory, into
// pre[] (shared); each thread owns a contiguous run of words.  Whole block.
__device__ __forceinline__ void words_prefix(const uint32_t *bits, int *pre, int words, int *red) {
  const int per = (words + blockDim.x - 1) / blockDim.x;
  const int w0 = threadIdx.x * per, w1 = min(words, w0 + per);
  int local = 0;
  for (int w = w0; w < w1; ++w) local += __popc(bits[w]);
  int tot;
  int run = block_excl_scan(local, red, &tot);
  for (int w = w0; w < w1; ++w) {
    pre[w] = run;
    run += __popc(bits[w]);
  }
  __syncthreads();
}

// One block per long row d.  Columns outside B raise kErrCsr and are left
// out; a repeated column excludes the row (lmap[k] = -1).  The copy is
// written sorted by column: an entry's position is its column's rank in the
// row's bitmap.
__global__ void __launch_bounds__(256)
    k_long_build(const int32_t *__restrict__ brp, const int32_t *__restrict__ bci, int32_t ncols, int words,
                 const int32_t *__restrict__ lrow, const int32_t *__restrict__ lbase, int32_t *__restrict__ lmap,
                 uint32_t *__restrict__ bits, char *__restrict__ ent, int ent_bytes, int32_t *__restrict__ lsrc,
                 int32_t *__restrict__ whist, uint32_t *err) {
  extern __shared__ uint32_t sm_lbits[];  // words bitmap words, then words prefix counts
  int *pre = reinterpret_cast<int *>(sm_lbits + words);
  __shared__ int red[33];
  __shared__ int s_dup;
  const int d = blockIdx.x;
  const int32_t k = lrow[d];
  const int32_t base = lbase[d];
  const int32_t b0 = brp[k], len = brp[k + 1] - b0;
  for (int w = threadIdx.x; w < words; w += blockDim.x) sm_lbits[w] = 0u;
  if (threadIdx.x == 0) s_dup = 0;
  __syncthreads();
  for (int32_t q = threadIdx.x; q < len; q += blockDim.x) {
    const int32_t c = bci[b0 + q];
    if (!((uint32_t)c < (uint32_t)ncols)) {
      raise_err(err, kErrCsr);
      continue;
    }
    const uint32_t bit = 1u << (c & 31);
    if (atomicOr(&sm_lbits[c >> 5], bit) & bit) s_dup = 1;
  }
  __syncthreads();
  if (s_dup) {  // whole block: the row keeps the atomic path
    if (threadIdx.x == 0) lmap[k] = -1;
    return;
  }
  words_prefix(sm_lbits, pre, words, red);
  for (int32_t q = threadIdx.x; q < len; q += blockDim.x) {
    const int32_t c = bci[b0 + q];
    if (!((uint32_t)c < (uint32_t)ncols)) continue;
    const int pos = base + pre[c >> 5] + __popc(sm_lbits[c >> 5] & ((1u << (c & 31)) - 1u));
    *reinterpret_cast<int32_t *>(ent + (size_t)pos * ent_bytes) = c;
    lsrc[pos] = b0 + q;
  }
  uint32_t *bw = bits + (size_t)d * words;
  for (int w = threadIdx.x; w < words; w += blockDim.x) {
    const uint32_t x = sm_lbits[w];
    bw[w] = x;
    if (x) atomicAdd(&whist[w], __popc(x));
  }
}

// One block: word boundaries rw[0..kLongRanges] of the column ranges, range
// r holding words [rw[r], rw[r+1]) and about 1/kLongRanges of the long
// rows' entries (rw[0] = 0, rw[kLongRanges] = words).
__global__ void __launch_bounds__(1024)
    k_long_ranges(const int32_t *__restrict__ whist, int words, int32_t *__restrict__ rw) {
  __shared__ long long red[33];
  __shared__ long long s_tot;
  long long carry = 0;
  // pass 1: the total
  long long local = 0;
  for (int w = threadIdx.x; w < words; w += blockDim.x) local += whist[w];
  const long long tot = block_sum(local, red);
  if (threadIdx.x <= kLongRanges) rw[threadIdx.x] = threadIdx.x == kLongRanges ? words : 0;
  if (threadIdx.x == 0) s_tot = tot;
  __syncthreads();
  // pass 2: range r starts at the first word whose exclusive prefix reaches r * tot / R
  for (int c0 = 0; c0 < words; c0 += blockDim.x) {
    const int w = c0 + threadIdx.x;
    const long long v = w < words ? whist[w] : 0;
    long long t;
    const long long ex = carry + block_excl_scan(v, red, &t);
    if (w < words && v > 0) {
      // the threshold of range r lies in (ex, ex + v]: word w + 1 is the first
      // word whose exclusive prefix reaches it
      for (int r = 1; r < kLongRanges; ++r) {
        const long long thr = s_tot * r / kLongRanges;
        if (ex < thr && thr <= ex + v) rw[r] = w + 1;
      }
    }
    carry += t;
  }
  __syncthreads();
  // ranges never started (thresholds inside one heavy word, or no entries):
  // make the boundaries non-decreasing
  if (threadIdx.x == 0) {
    for (int r = 1; r < kLongRanges; ++r) {
      if (rw[r] < rw[r - 1]) rw[r] = rw[r - 1];
      if (rw[r] > words) rw[r] = words;
    }
  }
}

// One block per long row: off[d * (kLongRanges + 1) + r] = base + entries of
// the row in words below rw[r].
__global__ void __launch_bounds__(256)
    k_long_offsets(const int32_t *__restrict__ lrow, const int32_t *__restrict__ lbase,
                   const int32_t *__restrict__ lmap, const uint32_t *__restrict__ bits, int words,
                   const int32_t *__restrict__ rw, int32_t *__restrict__ off) {
  extern __shared__ uint32_t sm_lo[];
  int *pre = reinterpret_cast<int *>(sm_lo + words);
  __shared__ int red[33];
  const int d = blockIdx.x;
  if (lmap[lrow[d]] != d) return;  // excluded (repeated column): never read
  const uint32_t *bw = bits + (size_t)d * words;
  for (int w = threadIdx.x; w < words; w += blockDim.x) sm_lo[w] = bw[w];
  __syncthreads();
  words_prefix(sm_lo, pre, words, red);
  if (threadIdx.x <= kLongRanges) {
    const int w = rw[threadIdx.x];
    const int below = w >= words ? pre[words - 1] + __popc(sm_lo[words - 1]) : pre[w];
    off[(size_t)d * (kLongRanges + 1) + threadIdx.x] = lbase[d] + below;
  }
}

template <typename T>
__global__ void __launch_bounds__(256)
    k_long_vals(const int32_t *__restrict__ lsrc, int64_t n, const T *__restrict__ bv, LEnt<T> *__restrict__ ent) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    ent[e].v = bv[lsrc[e]];
}

size_t long_entry_bytes(int dtype) { return dtype == SPGEMM_F32 ? sizeof(LEnt<float>) : sizeof(LEnt<double>); }

cudaError_t long_rows_mark(spgemm_plan_s *p) {
  if (p->long_min <= 0 || p->n == 0) return cudaSuccess;
  KernelScope ks(p, "long_mark");
  k_long_mark<<<(unsigned)((p->n + 255) / 256), 256, 0, p->stream>>>(p->brp, p->n, p->nnz_b, p->long_min,
                                                                      p->long_cap, p->lmap, p->lrow, p->lbase, p->dc);
  return cudaGetLastError();
}

cudaError_t long_rows_build(spgemm_plan_s *p) {
  p->long_ready = false;
  if (p->long_min <= 0 || p->n_long <= 0 || p->long_tot <= 0) return cudaSuccess;
  const size_t words = (size_t)p->bm_words;
  const size_t eb = long_entry_bytes(p->dtype);
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t o_bits = 0;
  const size_t o_off = o_bits + up((size_t)p->n_long * words * 4);
  const size_t o_ent = o_off + up((size_t)p->n_long * (kLongRanges + 1) * 4);
  const size_t o_src = o_ent + up((size_t)p->long_tot * eb);
  const size_t o_hist = o_src + up((size_t)p->long_tot * 4);
  const size_t o_rw = o_hist + up(words * 4);
  const size_t bytes = o_rw + up((kLongRanges + 1) * 4);
  cudaError_t e = cudaMallocAsync(&p->long_ws, bytes, p->stream);
  if (e != cudaSuccess) {
    p->long_ws = nullptr;
    return e;
  }
  p->long_ws_bytes = bytes;
  char *b = static_cast<char *>(p->long_ws);
  p->lbits = reinterpret_cast<uint32_t *>(b + o_bits);
  p->loff = reinterpret_cast<int32_t *>(b + o_off);
  p->lent = b + o_ent;
  p->lsrc = reinterpret_cast<int32_t *>(b + o_src);
  int32_t *whist = reinterpret_cast<int32_t *>(b + o_hist);
  int32_t *rw = reinterpret_cast<int32_t *>(b + o_rw);
  // entries left out (columns outside B) keep source 0, a valid index of B
  e = cudaMemsetAsync(p->lsrc, 0, (size_t)p->long_tot * 4, p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(whist, 0, words * 4, p->stream);
  if (e != cudaSuccess) return e;
  const size_t smem = words * 8;
  e = set_dynamic_smem(reinterpret_cast<const void *>(k_long_build), smem);
  if (e == cudaSuccess) e = set_dynamic_smem(reinterpret_cast<const void *>(k_long_offsets), smem);
  if (e != cudaSuccess) return e;
  {
    KernelScope ks(p, "long_build");
    k_long_build<<<(unsigned)p->n_long, 256, smem, p->stream>>>(p->brp, p->bci, (int32_t)p->k, (int)words, p->lrow,
                                                                p->lbase, p->lmap, p->lbits, (char *)p->lent, (int)eb,
                                                                p->lsrc, whist, &p->dc->err);
    k_long_ranges<<<1, 1024, 0, p->stream>>>(whist, (int)words, rw);
    k_long_offsets<<<(unsigned)p->n_long, 256, smem, p->stream>>>(p->lrow, p->lbase, p->lmap, p->lbits, (int)words,
                                                                  rw, p->loff);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) p->long_ready = true;
  return e;
}

cudaError_t long_rows_values(spgemm_plan_s *p) {
  if (!p->long_ready) return cudaSuccess;
  const int64_t n = p->long_tot;
  const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
  KernelScope ks(p, "long_vals");
  switch (p->dtype) {
    case SPGEMM_F64:
      k_long_vals<double><<<blocks, 256, 0, p->stream>>>(p->lsrc, n, (const double *)p->bv, (LEnt<double> *)p->lent);
      break;
    case SPGEMM_F32:
      k_long_vals<float><<<blocks, 256, 0, p->stream>>>(p->lsrc, n, (const float *)p->bv, (LEnt<float> *)p->lent);
      break;
    default:
      k_long_vals<int64_t><<<blocks, 256, 0, p->stream>>>(p->lsrc, n, (const int64_t *)p->bv,
                                                          (LEnt<int64_t> *)p->lent);
      break;
  }
  return cudaGetLastError();
}

}  // namespace sg
