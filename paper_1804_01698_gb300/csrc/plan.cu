// Host side of the GB300 hash SpGEMM: the C ABI of include/spgemm.h, the
// plan object, and the small kernels around the two phases:
//
//   k_row_flop      flop[i] = sum over stored a_ik of nnz(b_k*)
//                   (paper Sec. 4.1, Fig. "RowsToThreads", step 1), plus
//                   the symbolic bin of every row and the input checks
//   k_bin_scatter   rows grouped by bin (the GPU form of step 2 of
//                   "RowsToThreads": instead of equal-flop row ranges per
//                   thread, rows of similar size share one kernel)
//   k_scan_*        exclusive scan of nnz(c_i*) into C's row_ptr
//                   (Fig. "Hash_SpGEMM": rpts_C is allocated and filled
//                   between the symbolic and the numeric phase)
//   k_num_classify  numeric bins from the exact row counts
//   k_bm_items_*    work items (row, rank window, part) of heavy bitmap rows
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace sg {

const BinCfg kSymBins[kNumSymBins] = {
    {kWarp, 64, kWarpsPerBlock * 32, 32},      {kWarp, 128, kWarpsPerBlock * 32, 64},
    {kWarp, 256, kWarpsPerBlock * 32, 128},    {kWarp, 512, kWarpsPerBlock * 32, 256},
    {kWarp, 1024, kWarpsPerBlock * 32, 512},   {kBlock, 2048, 256, 1536},
    {kBlock, 4096, 512, 3072},                 {kBlock, 8192, 1024, 6144},
    {kBlock, 16384, 1024, 12288},              {kBlock, 32768, 1024, 24576},
    {kBitmap, 0, 256, INT64_MAX},              {kBitmap, 0, 256, kBitmapMidMax},
    {kGlobal, 0, 1024, INT64_MAX}};

const BinCfg kNumBins[kNumNumBins] = {
    {kWarp, 64, kWarpsPerBlock * 32, 32},      {kWarp, 128, kWarpsPerBlock * 32, 64},
    {kWarp, 256, kWarpsPerBlock * 32, 128},    {kWarp, 512, kWarpsPerBlock * 32, 256},
    {kWarp, 1024, kWarpsPerBlock * 32, 512},   {kBlock, 2048, 256, 1536},
    {kBlock, 4096, 512, 3072},                 {kBlock, 8192, 1024, 6144},
    {kBlock, 16384, 1024, 12288},              {kBitmap, 0, kBmThreadsL, INT64_MAX},
    {kGlobal, 0, 1024, INT64_MAX},             {kBitmap, 0, kBmThreadsS, INT64_MAX},
    {kBitmap, 0, kBmThreadsM, INT64_MAX}};

cudaError_t launch_numeric_f64(spgemm_plan_s *p, const int32_t *c_rp, int32_t *c_ci, void *c_v);
cudaError_t launch_numeric_f32(spgemm_plan_s *p, const int32_t *c_rp, int32_t *c_ci, void *c_v);
cudaError_t launch_numeric_i64(spgemm_plan_s *p, const int32_t *c_rp, int32_t *c_ci, void *c_v);

HashCaps hash_caps(int warp_load_pct, int block_load_pct) {
  const int wp = warp_load_pct > 0 ? warp_load_pct : 50;
  const int bp = block_load_pct > 0 ? block_load_pct : 75;
  HashCaps c{};
  for (int t = 0; t < 9; ++t) {
    const long long slots = 64LL << t;
    c.cap[t] = slots * (t < 5 ? wp : bp) / 100;
  }
  return c;
}

__device__ __forceinline__ int hash_bin_of(int64_t b, const HashCaps &caps) {
#pragma unroll
  for (int t = 0; t < 9; ++t)
    if (b <= caps.cap[t]) return t;
  return 9;
}

__device__ __forceinline__ int sym_bin_of(int64_t b, int64_t bitmap_min, const HashCaps &caps) {
  if (b <= 0) return 255;
  if (bitmap_min > 0 && b > bitmap_min) return b > kBitmapMidMax ? kSymBitmapBin : kSymBitmapMidBin;
  const int t = hash_bin_of(b, caps);
  if (t < 9) return t;
  if (b <= kBlockSymMax) return 9;
  return kSymGlobalBin;
}

__device__ __forceinline__ bool is_bitmap_row(int sym_bin) {
  return sym_bin == kSymBitmapBin || sym_bin == kSymBitmapMidBin;
}

__device__ __forceinline__ int num_bin_of(int64_t nnz, const HashCaps &caps) {
  if (nnz <= 0) return 255;
  const int t = hash_bin_of(nnz, caps);
  return t < 9 ? t : kNumGlobalBin;
}

// The flop pass (Sec. 4.1, Fig. "RowsToThreads", step 1) in two sweeps, so
// that no thread walks a row: every stored a_ik first gets the length of the
// row of B it selects, an exclusive prefix sum P of those lengths follows,
// and row i's flop is then P[rp[i+1]] - P[rp[i]].  One thread per entry and
// per row keeps every SM busy whatever the row lengths (a warp per row would
// wait on its dependent loads row after row, and a hub row of thousands of
// entries would hold it for len/32 steps).

__global__ void __launch_bounds__(256)
    k_merge_starts(const int32_t *__restrict__ rp, int64_t m, int64_t nnz, int64_t tiles, long long *__restrict__ starts,
                   int64_t *__restrict__ flop, int32_t *__restrict__ kept, LongMark lm, DevCounters *dc) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // long rows of B (long_min 0: none), in the same launch
  if (lm.long_min > 0)
    for (int64_t k = t0; k < lm.n; k += stride) long_mark_row(lm, k, dc);
  for (int64_t i = t0; i < m; i += stride) {
    if (flop) {
      flop[i] = 0;
      kept[i] = 0;
    }
    const int64_t r0 = __ldg(rp + i), r1 = __ldg(rp + i + 1);
    if (r0 < 0 || r0 > r1 || r1 > nnz) continue;
    const int64_t hi = i + r1;
    for (int64_t D = (i + r0 + kMergeTile - 1) / kMergeTile * kMergeTile; D <= hi; D += kMergeTile) {
      const int64_t t = D / kMergeTile;
      if (t >= tiles) break;
      starts[2 * t] = i;
      starts[2 * t + 1] = D - i;
    }
  }
  if (t0 == 0) {
    starts[2 * tiles] = m;
    starts[2 * tiles + 1] = nnz;
  }
}

// flop[i] = sum over the stored a_ik of row i of nnz(b_k*), and kept[i], the
// number of those a_ik whose row of B is not empty, by a merge-path walk over
// A's row ends and entries: every thread takes kMergeIPT consecutive items,
// so a hub row of A is shared by as many threads as its length asks and no
// per-entry array is written.  A row that lies in one thread's items is
// stored; the parts of the others are added with atomics into flop and
// kept, which the caller zeroes first.  Columns outside B and malformed rows
// of B raise kErrCsr and count 0.  Counts the entries that select a
// non-empty row of B.
__global__ void __launch_bounds__(kMergeThreads)
    k_row_flop(Args a, int64_t nnz_a, int64_t nnz_b, const long long *__restrict__ starts, int64_t *__restrict__ flop,
               int32_t *__restrict__ kept, int2 *__restrict__ klist, int32_t *__restrict__ klist_n, DevCounters *dc) {
  __shared__ int32_t lens[kMergeTile];
  __shared__ int32_t ends[kMergeTile];
  __shared__ long long coords[4];
  __shared__ unsigned long long s_nz;
  __shared__ int s_nk;
  if (threadIdx.x == 0) {
    s_nz = 0;
    s_nk = 0;
  }
  unsigned long long nz = 0;
  int2 *list = klist + (size_t)blockIdx.x * kKeptListCap;
  merge_tile_walk(a.arp, a.aci, a.brp, a.m, nnz_a, a.n, nnz_b, a.err, starts, lens, ends, coords,
                  [&](int64_t i, long long sum, int kp, bool whole, int64_t j, const int32_t *len, int n) {
                    nz += (unsigned long long)kp;
                    if (whole) {
                      flop[i] = sum;
                      kept[i] = kp;
                    } else {
                      if (sum) atomicAdd(reinterpret_cast<unsigned long long *>(flop + i), (unsigned long long)sum);
                      if (kp) atomicAdd(kept + i, kp);
                    }
                    if (kp > 0) {
                      const int at = atomicAdd(&s_nk, kp);
                      for (int q = 0, w = at; q < n && w < kKeptListCap; ++q)
                        if (len[q] > 0) list[w++] = make_int2((int)i, (int)(j + q));
                    }
                  });
  nz = warp_sum(nz);
  if ((threadIdx.x & 31) == 0 && nz) atomicAdd(&s_nz, nz);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_nz) atomicAdd(&dc->nnz_a_used, s_nz);
    klist_n[blockIdx.x] = s_nk <= kKeptListCap ? s_nk : -1;
  }
}

// Row i (grid-stride): its symbolic bin from flop[i] (k_row_flop) and the
// plan's counters.  Row pointers must run from 0 to nnz(A) without
// decreasing; a row that breaks it raises kErrCsr and counts no flop.
__global__ void __launch_bounds__(256)
    k_row_bin(Args a, int64_t nnz_a, int64_t bitmap_min, HashCaps caps, int64_t gcap, int64_t *__restrict__ flop,
              uint8_t *__restrict__ rbin, int32_t *__restrict__ nnz_row, long long *__restrict__ sym_off,
              DevCounters *dc) {
  __shared__ unsigned int hist[kNumSymBins];
  __shared__ unsigned long long hflop[kNumSymBins];
  __shared__ unsigned long long s_tot, s_max, s_maxg, s_extra;
  if (threadIdx.x < kNumSymBins) {
    hist[threadIdx.x] = 0;
    hflop[threadIdx.x] = 0;
  }
  if (threadIdx.x == 0) s_tot = s_max = s_maxg = s_extra = 0;
  __syncthreads();
  unsigned long long tot = 0, mx = 0, mxg = 0, extra = 0;
  // every lane of a warp takes the same number of steps (warp_hist_add)
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < a.m; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = base + threadIdx.x;
    int64_t f = 0, bound = 0;
    int bin = 255;
    if (row < a.m) {
      const int64_t r0 = a.arp[row], r1 = a.arp[row + 1];
      if (0 <= r0 && r0 <= r1 && r1 <= nnz_a && (row > 0 || r0 == 0) && (row < a.m - 1 || r1 == nnz_a)) {
        f = flop[row];
      } else {
        raise_err(a.err, kErrCsr);
        flop[row] = 0;
      }
      bound = f < a.k ? f : a.k;
      bin = sym_bin_of(bound, bitmap_min, caps);
      if (bin == kSymGlobalBin && gcap >= 0 && bound >= gcap) {
        // graph mode: no table was planned for a row this large
        raise_err(a.err, kErrCapacity);
        bin = 255;
      }
      rbin[row] = (uint8_t)bin;
      if (bin == 255) nnz_row[row] = 0;
    }
    warp_hist_add(bin, (unsigned long long)f, kNumSymBins, hist, hflop);
    if (row >= a.m) continue;
    if (bin == kSymGlobalBin && (unsigned long long)bound > mxg) mxg = (unsigned long long)bound;
    if (bin == kSymBitmapBin && sym_split_parts(f) > 1) extra += (unsigned long long)(sym_split_parts(f) - 1);
    tot += (unsigned long long)f;
    if ((unsigned long long)f > mx) mx = (unsigned long long)f;
  }
  tot = warp_sum(tot);
  extra = warp_sum(extra);
  mx = warp_max(mx);
  mxg = warp_max(mxg);
  if ((threadIdx.x & 31) == 0) {
    if (tot) atomicAdd(&s_tot, tot);
    if (extra) atomicAdd(&s_extra, extra);
    if (mx) atomicMax(&s_max, mx);
    if (mxg) atomicMax(&s_maxg, mxg);
  }
  __syncthreads();
  if (threadIdx.x < kNumSymBins && hist[threadIdx.x]) {
    atomicAdd(&dc->sym_count[threadIdx.x], hist[threadIdx.x]);
    atomicAdd(&dc->sym_flop[threadIdx.x], hflop[threadIdx.x]);
  }
  if (threadIdx.x == 0) {
    if (s_tot) atomicAdd(&dc->total_flop, s_tot);
    if (s_extra) atomicAdd(&dc->sym_split_extra, s_extra);
    if (s_max) atomicMax(&dc->max_flop, s_max);
    if (s_maxg) atomicMax(&dc->max_bound_global, s_maxg);
  }
  // the symbolic bins' offsets on the device (bin kernels find their rows by them)
  last_block_offsets(dc->sym_count, kNumSymBins, sym_off, &dc->sym_ticket);
}


// Rows i with bin_of[i] != 255 go to perm[off[bin] + arbitrary rank].
__global__ void __launch_bounds__(256)
    k_bin_scatter(const uint8_t *__restrict__ bin_of, int64_t m, const long long *__restrict__ off,
                  unsigned long long *cursor, int32_t *__restrict__ perm, int nbins) {
  __shared__ unsigned int hist[16];
  __shared__ unsigned long long base[16];
  if (threadIdx.x < 16) hist[threadIdx.x] = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = i < m ? bin_of[i] : 255;
  unsigned int local = 0;
  if (b < nbins) local = atomicAdd(&hist[b], 1u);
  __syncthreads();
  if (threadIdx.x < nbins && hist[threadIdx.x]) base[threadIdx.x] = atomicAdd(&cursor[threadIdx.x], hist[threadIdx.x]);
  __syncthreads();
  if (b < nbins) perm[off[b] + (long long)base[b] + local] = (int32_t)i;
}

constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanThreads * kScanPer;

template <typename InT>
__global__ void __launch_bounds__(kScanThreads)
    k_scan_reduce(const InT *__restrict__ x, int64_t m, long long *__restrict__ partial) {
  __shared__ long long red[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  long long s = 0;
#pragma unroll
  for (int u = 0; u < kScanPer; ++u)
    if (base + u < m) s += x[base + u];
  s = block_sum(s, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kScanThreads)
    k_scan_spine(long long *partial, int64_t nblk, long long max_nnz, unsigned long long *total, uint32_t *err) {
  __shared__ long long red[33];
  long long carry = 0;
  for (int64_t c0 = 0; c0 < nblk; c0 += kScanThreads) {
    const int64_t t = c0 + threadIdx.x;
    const long long v = t < nblk ? partial[t] : 0;
    long long tot;
    const long long ex = block_excl_scan(v, red, &tot);
    if (t < nblk) partial[t] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    *total = (unsigned long long)carry;
    if (carry > max_nnz) raise_err(err, kErrOverflow);
  }
}

// out[i] = x[0] + ... + x[i-1] for i = 0..m; out may be x itself (each thread
// reads its elements before it writes them, and the reduce pass is done).
// With zero_in, x[] is zeroed once read (x not out).
template <typename InT, typename OutT>
__global__ void __launch_bounds__(kScanThreads)
    k_scan_apply(InT *x, int64_t m, const long long *__restrict__ partial, OutT *out, bool zero_in = false) {
  __shared__ long long red[33];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  InT v[kScanPer];
  long long s = 0;
#pragma unroll
  for (int u = 0; u < kScanPer; ++u) {
    v[u] = base + u < m ? x[base + u] : 0;
    s += v[u];
    if (zero_in && base + u < m) x[base + u] = 0;
  }
  long long tot;
  long long run = partial[blockIdx.x] + block_excl_scan(s, red, &tot);
#pragma unroll
  for (int u = 0; u < kScanPer; ++u) {
    if (base + u < m) out[base + u] = (OutT)run;
    run += v[u];
    if (base + u == m - 1) out[m] = (OutT)run;
  }
}

__global__ void __launch_bounds__(256)
    k_num_classify(const int32_t *__restrict__ nnz_row, const uint8_t *__restrict__ rbin,
                   const int64_t *__restrict__ flop, int64_t m, HashCaps caps, int64_t gcap,
                   uint8_t *__restrict__ rbin2, long long *__restrict__ num_off, DevCounters *dc) {
  __shared__ unsigned int hist[kNumNumBins];
  __shared__ unsigned long long hflop[kNumNumBins];
  __shared__ unsigned long long s_maxg;
  if (threadIdx.x < kNumNumBins) {
    hist[threadIdx.x] = 0;
    hflop[threadIdx.x] = 0;
  }
  if (threadIdx.x == 0) s_maxg = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int b = 255;
  unsigned long long f = 0;
  if (i < m) {
    if (!is_bitmap_row(rbin[i])) {
      const int32_t z = nnz_row[i];
      b = num_bin_of(z, caps);
      if (b == kNumGlobalBin && gcap >= 0 && (int64_t)z * 4 / 3 >= gcap) {
        raise_err(&dc->err, kErrCapacity);  // graph mode: the planned tables are too small
        b = 255;
      }
      if (b == kNumGlobalBin) atomicMax(&s_maxg, (unsigned long long)z);
    }
    rbin2[i] = (uint8_t)b;
    if (b != 255) f = (unsigned long long)flop[i];
  }
  warp_hist_add(b, f, kNumNumBins, hist, hflop);
  __syncthreads();
  if (threadIdx.x < kNumNumBins && hist[threadIdx.x]) atomicAdd(&dc->num_count[threadIdx.x], hist[threadIdx.x]);
  if (threadIdx.x < kNumNumBins && hflop[threadIdx.x]) atomicAdd(&dc->num_flop[threadIdx.x], hflop[threadIdx.x]);
  if (threadIdx.x == 0 && s_maxg) atomicMax(&dc->max_nnz_global, s_maxg);
  last_block_offsets(dc->num_count, kNumNumBins, num_off, &dc->num_ticket);
}

struct BmCaps {
  long long cap[3];              // small, medium, large (0 = class unused)
  long long off[3][kBmBuckets];  // item offsets of the classes' weight buckets (fill only)
};

// Class of a bitmap row with nnz entries and its number of rank windows
// (work items per part): one, or none for an empty row.  A large-class row
// with more entries than its shared array holds keeps the first cap[2]
// ranks there and adds the products of its other ranks straight into C
// (k_num_bitmap), so it needs no second window walking all its products
// again.
__device__ __forceinline__ int bm_class(long long nnz, const BmCaps &c, long long *windows) {
  *windows = nnz > 0 ? 1 : 0;
  if (nnz <= c.cap[0]) return 0;
  if (nnz <= c.cap[1]) return 1;
  return 2;
}

__global__ void __launch_bounds__(256)
    k_bm_items_count(const int32_t *__restrict__ rows, int64_t n, const int32_t *__restrict__ nnz_row,
                     const int64_t *__restrict__ flop, BmCaps caps, DevCounters *dc) {
  __shared__ unsigned long long s_items[3], s_flop[3], s_bucket[3 * kBmBuckets];
  if (threadIdx.x < 3) s_items[threadIdx.x] = s_flop[threadIdx.x] = 0;
  if (threadIdx.x < 3 * kBmBuckets) s_bucket[threadIdx.x] = 0;
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    const int32_t i = rows[t];
    long long w;
    const int c = bm_class(nnz_row[i], caps, &w);
    if (w > 0) {
      const int parts = bm_split_parts(flop[i], nnz_row[i]);
      w *= parts;
      atomicAdd(&s_items[c], (unsigned long long)w);
      atomicAdd(&s_bucket[c * kBmBuckets + bm_bucket_of(flop[i], parts)], (unsigned long long)w);
      atomicAdd(&s_flop[c], (unsigned long long)flop[i]);
    }
  }
  __syncthreads();
  if (threadIdx.x < 3 && s_items[threadIdx.x]) {
    atomicAdd(&dc->bm_items[threadIdx.x], s_items[threadIdx.x]);
    atomicAdd(&dc->bm_flop[threadIdx.x], s_flop[threadIdx.x]);
  }
  if (threadIdx.x < 3 * kBmBuckets && s_bucket[threadIdx.x])
    atomicAdd(&dc->bm_bucket[threadIdx.x / kBmBuckets][threadIdx.x % kBmBuckets], s_bucket[threadIdx.x]);
}

__global__ void __launch_bounds__(256)
    k_bm_items_fill(const int32_t *__restrict__ rows, int64_t n, const int32_t *__restrict__ nnz_row,
                    const int64_t *__restrict__ flop, BmCaps caps, DevCounters *dc, int4 *__restrict__ items) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int32_t i = rows[t];
  long long w;
  const int c = bm_class(nnz_row[i], caps, &w);
  if (w == 0) return;
  const int parts = bm_split_parts(flop[i], nnz_row[i]);
  const int bk = bm_bucket_of(flop[i], parts);
  const unsigned long long base = caps.off[c][bk] + atomicAdd(&dc->bm_cursor[c][bk], (unsigned long long)(w * parts));
  for (int q = 0; q < (int)w; ++q)
    for (int pt = 0; pt < parts; ++pt) items[base + (unsigned long long)q * parts + pt] = make_int4((int)t, q, pt, parts);
}

// ---------------------------------------------------------------------------
int max_smem_per_block() {
  static int cached[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 48 * 1024;
  if (cached[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0)
      v = 48 * 1024;
    cached[dev] = v;
  }
  return cached[dev];
}

cudaError_t set_dynamic_smem(const void *kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void *, int>, size_t> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(mu);
  size_t &have = done[{kernel, dev}];
  if (bytes <= have) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) have = bytes;
  return e;
}

static int sm_count() {
  static int cached[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 1;
  if (cached[dev] == 0) {
    int v = 1;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 1;
  }
  return cached[dev];
}

int64_t launch_blocks(const spgemm_plan_s *, const void *, int, size_t, int64_t exact) {
  return std::max<int64_t>(1, exact);
}

int64_t ddrive_bin_rows(const spgemm_plan_s *p, int b, bool symbolic) {
  // graph mode has no bitmap rows; the global bin runs only with its tables;
  // every other bin runs (one block at least) whatever the planned count
  if (symbolic) {
    if (b == kSymBitmapBin || b == kSymBitmapMidBin) return 0;
    if (b == kSymGlobalBin && !p->gtab) return 0;
    return std::max<int64_t>(1, p->sym_count[b]);
  }
  if (b == kNumBitmapBin || b == kNumBitmapSBin || b == kNumBitmapMBin) return 0;
  if (b == kNumGlobalBin && !p->gtab) return 0;
  return std::max<int64_t>(1, p->num_count[b]);
}

// Side streams and their fork/join events come from a per-device pool: a
// plan takes a set at its first fork and returns it when destroyed, so
// repeated plans do not pay for creating streams.  A returned set may still
// hold the old plan's work; the next plan's kernels queue behind it.
struct SideSet {
  cudaStream_t s[4];
  cudaEvent_t fork_ev, join_ev[4];
};
static std::mutex g_side_mu;
static std::vector<SideSet> g_side_free[64];

static cudaError_t acquire_side(spgemm_plan_s *p) {
  SideSet set{};
  bool have = false;
  if (p->device >= 0 && p->device < 64) {
    std::lock_guard<std::mutex> g(g_side_mu);
    if (!g_side_free[p->device].empty()) {
      set = g_side_free[p->device].back();
      g_side_free[p->device].pop_back();
      have = true;
    }
  }
  if (!have) {
    bool ok = true;
    for (int i = 0; i < 4 && ok; ++i) ok = cudaStreamCreateWithFlags(&set.s[i], cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&set.fork_ev, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < 4 && ok; ++i) ok = cudaEventCreateWithFlags(&set.join_ev[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) return cudaGetLastError() == cudaSuccess ? cudaErrorUnknown : cudaGetLastError();
  }
  for (int i = 0; i < 4; ++i) {
    p->side[i] = set.s[i];
    p->join_ev[i] = set.join_ev[i];
  }
  p->fork_ev = set.fork_ev;
  p->side_ready = true;
  return cudaSuccess;
}

static void release_side(spgemm_plan_s *p) {
  if (!p->side_ready) return;
  SideSet set{};
  for (int i = 0; i < 4; ++i) {
    set.s[i] = p->side[i];
    set.join_ev[i] = p->join_ev[i];
  }
  set.fork_ev = p->fork_ev;
  p->side_ready = false;
  if (p->device >= 0 && p->device < 64) {
    std::lock_guard<std::mutex> g(g_side_mu);
    g_side_free[p->device].push_back(set);
    return;
  }
  for (int i = 0; i < 4; ++i) {
    cudaStreamDestroy(set.s[i]);
    cudaEventDestroy(set.join_ev[i]);
  }
  cudaEventDestroy(set.fork_ev);
}

cudaError_t fork(spgemm_plan_s *p) {
  if (!p->side_ready) {
    const cudaError_t ea = acquire_side(p);
    if (ea != cudaSuccess) return ea;
  }
  cudaError_t e = cudaEventRecord(p->fork_ev, p->stream);
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(p->side[i], p->fork_ev, 0);
  return e;
}

cudaStream_t bin_stream(spgemm_plan_s *p, int i) { return p->side_ready ? p->side[i & 3] : p->stream; }

cudaError_t join(spgemm_plan_s *p) {
  if (!p->side_ready) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) {
    e = cudaEventRecord(p->join_ev[i], p->side[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->stream, p->join_ev[i], 0);
  }
  return e;
}

static size_t value_size(int dtype) { return dtype == SPGEMM_F32 ? 4 : 8; }

// Values per numeric bitmap window for a block of `budget` bytes of shared
// memory: what remains after the bitmap with its prefix counts and the
// block's static arrays.
int64_t bitmap_capacity(int dtype, int bm_words, int64_t budget) {
  const int64_t avail = budget - kStaticSmemReserve - (int64_t)bm_words * 8;
  int64_t cap = avail / (int64_t)value_size(dtype);
  cap = (cap / 256) * 256;
  return cap > 0 ? cap : 0;
}

}  // namespace sg

namespace {
thread_local std::string g_last_error;
}  // namespace

void sg::set_last_error(const std::string &text) { g_last_error = text; }

using namespace sg;

namespace {

int fail_cuda(cudaError_t e, const char *where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return SPGEMM_ERR_OUT_OF_MEMORY;
  return SPGEMM_ERR_DEVICE;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

std::mutex g_pool_mu;
bool g_pool_done[64];

// Keep freed workspace in the device's default memory pool instead of
// returning it to the driver, so repeated plans do not pay for allocation.
void keep_pool(int dev) {
  std::lock_guard<std::mutex> g(g_pool_mu);
  if (dev < 0 || dev >= 64 || g_pool_done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  g_pool_done[dev] = true;
}

int read_counters(spgemm_plan_s *p) {
  cudaError_t e = cudaMemcpyAsync(p->hc, p->dc, sizeof(DevCounters), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return fail_cuda(e, "reading plan counters");
  const unsigned err = p->hc->err;
  if (err & kErrCsr) {
    g_last_error = "input CSR has an index out of range or a malformed row_ptr";
    return SPGEMM_ERR_INVALID_CSR;
  }
  if (err & kErrCapacity) {
    g_last_error = "C or one of its rows exceeds the capacity the batch graph was planned with";
    return SPGEMM_ERR_OUT_OF_MEMORY;
  }
  if (err & kErrOverflow) {
    g_last_error = p->ddrive ? "nnz(C) exceeds the pool the batch graph was planned with"
                             : "nnz(C) exceeds int32 indexing";
    return p->ddrive ? SPGEMM_ERR_OUT_OF_MEMORY : SPGEMM_ERR_INDEX_OVERFLOW;
  }
  if (err) {
    g_last_error = "device-side check failed (hash probe or atomic retry bound)";
    return SPGEMM_ERR_DEVICE;
  }
  return SPGEMM_OK;
}

int64_t pow2_above(int64_t x) {  // smallest power of two strictly greater than x
  int64_t s = 1;
  while (s <= x) s <<= 1;
  return s;
}

int valid_csr_desc(const spgemm_csr *c) {
  if (!c) return 0;
  if (c->nrows < 0 || c->ncols < 0 || c->nnz < 0) return 0;
  if (c->nrows > INT32_MAX || c->ncols > INT32_MAX || c->nnz > INT32_MAX) return 0;
  if (!c->row_ptr) return 0;
  if (c->nnz > 0 && (!c->col_idx || !c->vals)) return 0;
  return 1;
}

void free_events(spgemm_plan_s *p) {
  for (auto &t : p->timed) {
    if (t.start) cudaEventDestroy(t.start);
    if (t.stop) cudaEventDestroy(t.stop);
  }
  p->timed.clear();
}

void free_ws(spgemm_plan_s *p) {
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  p->graph_exec = nullptr;
  free_events(p);
  release_side(p);
  if (p->ws_fixed) cudaFreeAsync(p->ws_fixed, p->stream);
  if (p->bitmaps) cudaFreeAsync(p->bitmaps, p->stream);
  if (p->bm_items) cudaFreeAsync(p->bm_items, p->stream);
  if (p->sym_items) cudaFreeAsync(p->sym_items, p->stream);
  if (p->gtab) cudaFreeAsync(p->gtab, p->stream);
  if (p->long_ws) cudaFreeAsync(p->long_ws, p->stream);
  if (p->acmp_ws) cudaFreeAsync(p->acmp_ws, p->stream);
  p->acmp_ws = nullptr;
  p->a_compact = false;
  p->long_ws = nullptr;
  p->long_ready = false;
  p->ws_fixed = nullptr;
  p->bitmaps = nullptr;
  p->bm_items = nullptr;
  p->sym_items = nullptr;
  p->sym_tickets = nullptr;
  p->gtab = nullptr;
}

int alloc_gtab(spgemm_plan_s *p, int64_t slots, size_t entry_bytes, int64_t rows) {
  // Blocks that work on heavy rows at once: two per SM, fewer when the
  // tables would pass 4 GiB.
  int64_t blocks = std::min<int64_t>(rows, 2 * (int64_t)sm_count());
  const size_t per = (size_t)slots * entry_bytes;
  const size_t budget = (size_t)4 << 30;
  while (blocks > 1 && per * (size_t)blocks > budget) blocks >>= 1;
  const size_t need = per * (size_t)blocks;
  if (p->gtab && p->gtab_bytes >= need) {
    p->gtab_slots = slots;
    p->gtab_blocks = blocks;
    return SPGEMM_OK;
  }
  if (p->gtab) cudaFreeAsync(p->gtab, p->stream);
  p->gtab = nullptr;
  cudaError_t e = cudaMallocAsync(&p->gtab, need, p->stream);
  if (e != cudaSuccess) {
    p->gtab = nullptr;
    return fail_cuda(e, "allocating heavy-row hash tables");
  }
  p->gtab_bytes = need;
  p->gtab_slots = slots;
  p->gtab_blocks = blocks;
  return SPGEMM_OK;
}

// Compacted A (Sec. 4.1's flop pass counts, per row, the stored a_ik whose
// row of B is not empty): when fewer than half of A's entries select a
// non-empty row of B, as in the BFS-frontier product A * F, the phases walk
// a copy of A without the others, which add nothing to C.  Row pointers are
// the scan of the counts; the copy's columns and sources are gathered once,
// its values before every numeric phase.
int compact_a(spgemm_plan_s *p) {
  const int64_t m = p->m, nz = p->nnz_a_used;
  const size_t vs = value_size(p->dtype);
  const size_t o_rp = 0;
  const size_t o_ci = align_up((size_t)(m + 1) * 4, 256);
  const size_t o_v = o_ci + align_up((size_t)nz * 4, 256);
  const size_t o_src = o_v + align_up((size_t)nz * vs, 256);
  const size_t bytes = o_src + align_up((size_t)nz * 4, 256);
  cudaError_t e = cudaMallocAsync(&p->acmp_ws, bytes, p->stream);
  if (e != cudaSuccess) {
    p->acmp_ws = nullptr;
    return fail_cuda(e, "allocating the compacted A");
  }
  p->acmp_bytes = bytes;
  char *b = static_cast<char *>(p->acmp_ws);
  p->karp = reinterpret_cast<int32_t *>(b + o_rp);
  p->kaci = reinterpret_cast<int32_t *>(b + o_ci);
  p->kav = b + o_v;
  p->asrc = reinterpret_cast<int32_t *>(b + o_src);
  // the copy's row pointers: the exclusive scan of the flop pass's per-row
  // counts; kept[] then serves as the per-row cursor of the gather
  const int64_t nblk = (m + kScanTile - 1) / kScanTile;
  long long *partial = (long long *)((char *)p->perm2 + align_up((size_t)m * 4, 256));
  {
    KernelScope ks(p, "compact_a");
    k_scan_reduce<<<(unsigned)nblk, kScanThreads, 0, p->stream>>>(p->kept, m, partial);
    k_scan_spine<<<1, kScanThreads, 0, p->stream>>>(partial, nblk, INT32_MAX, &p->dc->scan_total, &p->dc->err);
    k_scan_apply<<<(unsigned)nblk, kScanThreads, 0, p->stream>>>(p->kept, m, partial, p->karp, true);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = compact_a_gather(p);
  }
  if (e != cudaSuccess) return fail_cuda(e, "compacting A");
  p->a_compact = true;
  return SPGEMM_OK;
}

}  // namespace

extern "C" {

const char *spgemm_status_string(int status) {
  switch (status) {
    case SPGEMM_OK: return "ok";
    case SPGEMM_ERR_INVALID_ARGUMENT: return "invalid argument";
    case SPGEMM_ERR_INVALID_CSR: return "invalid CSR input";
    case SPGEMM_ERR_OUT_OF_MEMORY: return "out of device memory";
    case SPGEMM_ERR_INDEX_OVERFLOW: return "index overflow (nnz(C) > 2^31-1)";
    case SPGEMM_ERR_BAD_STATE: return "call out of order";
    case SPGEMM_ERR_DEVICE: return "device error";
    case SPGEMM_ERR_TIMEOUT: return "timeout";
    default: return "unknown status";
  }
}

const char *spgemm_last_error(void) { return g_last_error.c_str(); }

int spgemm_plan_create(spgemm_plan_t *out, const spgemm_csr *A, const spgemm_csr *B, int dtype, unsigned flags,
                       void *stream) {
  return spgemm_plan_create_tuned(out, A, B, dtype, flags, stream, nullptr);
}

}  // extern "C"

namespace sg {

// Validates the arguments, fills the plan and allocates its fixed
// workspace.  A graph-mode plan has no bitmap rows and no long rows.
int plan_init(spgemm_plan_s **out, const spgemm_csr *A, const spgemm_csr *B, int dtype, unsigned flags,
              cudaStream_t stream, const spgemm_tuning *tuning, bool graph) {
  if (!out) return SPGEMM_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  g_last_error.clear();
  if (tuning) {
    const int g = tuning->lanes_per_entry;
    auto pct_ok = [](int v) { return v == 0 || (v >= 5 && v <= 95); };
    if ((g != 0 && g != 4 && g != 8 && g != 16 && g != 32) || tuning->reserved != 0 ||
        tuning->bitmap_min_bound < -1 || tuning->max_nnz_c < 0 || tuning->max_nnz_c > INT32_MAX ||
        tuning->long_row_min < -1 || !pct_ok(tuning->warp_load_pct) || !pct_ok(tuning->block_load_pct)) {
      set_last_error("tuning: lanes_per_entry must be 0, 4, 8, 16 or 32, bitmap_min_bound >= -1, "
                     "0 <= max_nnz_c <= 2^31-1, long_row_min >= -1 and the load percentages 0 or 5..95");
      return SPGEMM_ERR_INVALID_ARGUMENT;
    }
  }
  if (!valid_csr_desc(A) || !valid_csr_desc(B) || A->ncols != B->nrows) return SPGEMM_ERR_INVALID_ARGUMENT;
  if (dtype != SPGEMM_I64 && dtype != SPGEMM_F32 && dtype != SPGEMM_F64) return SPGEMM_ERR_INVALID_ARGUMENT;
  if (flags & ~(SPGEMM_SORTED | SPGEMM_VALIDATE | SPGEMM_TIMING | SPGEMM_SERIAL | SPGEMM_PROBE_CHUNK4 |
                SPGEMM_COUNT_PROBES | SPGEMM_HASH_LOW_BITS))
    return SPGEMM_ERR_INVALID_ARGUMENT;

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_cuda(e, "cudaGetDevice");
  keep_pool(dev);

  spgemm_plan_s *p = new (std::nothrow) spgemm_plan_s();
  if (!p) return SPGEMM_ERR_OUT_OF_MEMORY;
  p->hc = new (std::nothrow) DevCounters();
  if (!p->hc) {
    delete p;
    return SPGEMM_ERR_OUT_OF_MEMORY;
  }
  p->m = A->nrows;
  p->n = A->ncols;
  p->k = B->ncols;
  p->nnz_a = A->nnz;
  p->nnz_b = B->nnz;
  p->arp = A->row_ptr;
  p->aci = A->col_idx;
  p->brp = B->row_ptr;
  p->bci = B->col_idx;
  p->av = A->vals;
  p->bv = B->vals;
  p->dtype = dtype;
  p->flags = flags;
  p->stream = stream;
  p->device = dev;
  p->G = 32;  // set from the flop pass below
  p->tune_G = tuning ? tuning->lanes_per_entry : 0;
  p->tune_bm_min = tuning ? tuning->bitmap_min_bound : 0;
  p->max_nnz_c = tuning && tuning->max_nnz_c > 0 ? tuning->max_nnz_c : INT32_MAX;
  p->span_cols = p->k;
  p->bitmap_ok = !graph && p->k <= kBitmapMaxCols;
  p->ddrive = graph;
  p->bm_words = (int)((p->k + 31) / 32);
  // bitmap classes: 3, 2 and 1 blocks per SM (228 KB per SM, 1 KB per block kept by the system)
  p->bm_cap[2] = bitmap_capacity(dtype, p->bm_words, max_smem_per_block());
  p->bm_cap[1] = bitmap_capacity(dtype, p->bm_words, 110 * 1024);
  p->bm_cap[0] = bitmap_capacity(dtype, p->bm_words, 72 * 1024);
  p->bm_threads[0] = kNumBins[kNumBitmapSBin].threads;
  p->bm_threads[1] = kNumBins[kNumBitmapMBin].threads;
  p->bm_threads[2] = kNumBins[kNumBitmapBin].threads;
  if (p->bitmap_ok && p->bm_cap[2] < 256) p->bitmap_ok = false;
  p->caps = hash_caps(tuning ? tuning->warp_load_pct : 0, tuning ? tuning->block_load_pct : 0);
  {
    const int64_t lt = tuning ? tuning->long_row_min : 0;
    p->long_min = !p->bitmap_ok || lt < 0 || p->nnz_b == 0 ? 0 : lt > 0 ? lt : long_row_min_default(p->k);
    p->long_cap = p->long_min > 0 ? p->nnz_b / p->long_min + 1 : 0;
  }

  // fixed workspace: counters, then per-row arrays
  const int64_t m = p->m;
  const int64_t nblk = (m + kScanTile - 1) / kScanTile + 1;
  size_t off = 0;
  const size_t o_dc = off;
  off = align_up(off + sizeof(DevCounters), 256);
  const size_t o_flop = off;
  off = align_up(off + (size_t)m * 8, 256);
  const size_t o_rbin = off;
  off = align_up(off + (size_t)m, 256);
  const size_t o_perm = off;
  off = align_up(off + (size_t)m * 4, 256);
  const size_t o_nnz = off;
  off = align_up(off + (size_t)m * 4, 256);
  const size_t o_rbin2 = off;
  off = align_up(off + (size_t)m, 256);
  const size_t o_perm2 = off;
  off = align_up(off + (size_t)m * 4, 256);
  const size_t o_part = off;
  off = align_up(off + (size_t)nblk * 8, 256);
  const size_t o_kept = off;
  off = align_up(off + (size_t)m * 4, 256);
  const int64_t mtiles = (m + p->nnz_a) / kMergeTile + 2;
  const size_t o_mstarts = off;
  off = align_up(off + (size_t)mtiles * 2 * sizeof(long long), 256);
  const size_t o_klist = off;
  off = align_up(off + (size_t)mtiles * kKeptListCap * sizeof(int2), 256);
  const size_t o_klist_n = off;
  off = align_up(off + (size_t)mtiles * sizeof(int32_t), 256);
  const size_t o_doff = off;
  off = align_up(off + 2 * 16 * sizeof(long long), 256);
  const size_t o_lmap = off;
  if (p->long_min > 0) off = align_up(off + (size_t)p->n * 4, 256);
  const size_t o_lrow = off;
  if (p->long_min > 0) off = align_up(off + (size_t)p->long_cap * 4, 256);
  e = cudaMallocAsync(&p->ws_fixed, off, p->stream);
  if (e != cudaSuccess) {
    p->ws_fixed = nullptr;
    int rc = fail_cuda(e, "allocating plan workspace");
    delete p->hc;
    delete p;
    return rc;
  }
  p->ws_fixed_bytes = off;
  char *base = (char *)p->ws_fixed;
  p->dc = (DevCounters *)(base + o_dc);
  p->flop = (int64_t *)(base + o_flop);
  p->rbin = (uint8_t *)(base + o_rbin);
  p->perm = (int32_t *)(base + o_perm);
  p->nnz_row = (int32_t *)(base + o_nnz);
  p->rbin2 = (uint8_t *)(base + o_rbin2);
  p->perm2 = (int32_t *)(base + o_perm2);
  (void)o_part;
  p->kept = (int32_t *)(base + o_kept);
  p->mstarts = (long long *)(base + o_mstarts);
  p->klist = (int2 *)(base + o_klist);
  p->klist_n = (int32_t *)(base + o_klist_n);
  p->d_sym_off = (long long *)(base + o_doff);
  p->d_num_off = p->d_sym_off + 16;
  if (p->long_min > 0) {
    p->lmap = (int32_t *)(base + o_lmap);
    p->lrow = (int32_t *)(base + o_lrow);
  }

  *out = p;
  return SPGEMM_OK;
}

// The flop pass, the symbolic bin offsets and the long rows' marks, on the
// plan's stream (Sec. 4.1, Fig. "RowsToThreads", step 1).
cudaError_t enqueue_flop(spgemm_plan_s *p) {
  const int64_t m = p->m;
  cudaError_t e = cudaMemsetAsync(p->dc, 0, sizeof(DevCounters), p->stream);
  if (e != cudaSuccess || m == 0) return e;
  Args a{p->m, p->n, p->k, p->arp, p->aci, p->brp, p->bci, p->av, p->bv, p->G, &p->dc->err};
  {
    KernelScope ks(p, "row_flop");
    const int64_t bm_min = !p->bitmap_ok || p->tune_bm_min < 0 ? 0
                           : p->tune_bm_min > 0                 ? p->tune_bm_min
                                                                : bitmap_min_bound(p->k);
    const int64_t tiles = (m + p->nnz_a + kMergeTile - 1) / kMergeTile;
    const LongMark lm{p->brp, p->n, p->nnz_b, p->long_min, p->long_cap, p->lmap, p->lrow};
    const int64_t items = std::max<int64_t>(m, p->long_min > 0 ? p->n : 0);
    k_merge_starts<<<(unsigned)std::min<int64_t>((items + 255) / 256, 8 * (int64_t)sm_count()), 256, 0, p->stream>>>(
        p->arp, m, p->nnz_a, tiles, p->mstarts, p->flop, p->kept, lm, p->dc);
    k_row_flop<<<(unsigned)tiles, kMergeThreads, 0, p->stream>>>(a, p->nnz_a, p->nnz_b, p->mstarts, p->flop, p->kept,
                                                                 p->klist, p->klist_n, p->dc);
    const int64_t rb = std::min<int64_t>((m + 255) / 256, 8 * (int64_t)sm_count());
    k_row_bin<<<(unsigned)rb, 256, 0, p->stream>>>(a, p->nnz_a, bm_min, p->caps, p->gcap_bound, p->flop, p->rbin,
                                                   p->nnz_row, p->d_sym_off, p->dc);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

// The symbolic kernels, the scan of the row counts into c_row_ptr (with the
// nnz(C) limit), the numeric bins and their device offsets.
cudaError_t enqueue_symbolic(spgemm_plan_s *p, int32_t *c_row_ptr) {
  cudaError_t e = launch_symbolic(p);
  if (e != cudaSuccess) return e;
  const int64_t m = p->m;
  if (m == 0) {
    e = cudaMemsetAsync(c_row_ptr, 0, sizeof(int32_t), p->stream);
  } else {
    const int64_t nblk = (m + kScanTile - 1) / kScanTile;
    // partial[] is the last segment of the fixed workspace, after perm2
    long long *partial = (long long *)((char *)p->perm2 + align_up((size_t)m * 4, 256));
    {
      KernelScope ks(p, "scan_reduce");
      k_scan_reduce<<<(unsigned)nblk, kScanThreads, 0, p->stream>>>(p->nnz_row, m, partial);
    }
    {
      KernelScope ks(p, "scan_spine");
      k_scan_spine<<<1, kScanThreads, 0, p->stream>>>(partial, nblk, p->max_nnz_c, &p->dc->nnz_c, &p->dc->err);
    }
    {
      KernelScope ks(p, "scan_apply");
      k_scan_apply<<<(unsigned)nblk, kScanThreads, 0, p->stream>>>(p->nnz_row, m, partial, c_row_ptr);
    }
    {
      KernelScope ks(p, "num_classify");
      k_num_classify<<<(unsigned)((m + 255) / 256), 256, 0, p->stream>>>(p->nnz_row, p->rbin, p->flop, m, p->caps,
                                                                         p->gcap_nnz, p->rbin2, p->d_num_off, p->dc);
    }
    const int64_t nbm = p->sym_count[kSymBitmapBin] + p->sym_count[kSymBitmapMidBin];
    if (nbm > 0) {
      KernelScope ks(p, "bm_items_count");
      BmCaps caps{{p->bm_cap[0], p->bm_cap[1], p->bm_cap[2]}, {}};
      k_bm_items_count<<<(unsigned)((nbm + 255) / 256), 256, 0, p->stream>>>(
          p->perm + p->sym_off[kSymBitmapBin], nbm, p->nnz_row, p->flop, caps, p->dc);
    }
    e = cudaGetLastError();
  }
  return e;
}

// Rows grouped by numeric bin (after enqueue_symbolic).
cudaError_t enqueue_num_scatter(spgemm_plan_s *p) {
  if (p->m == 0) return cudaSuccess;
  KernelScope ks(p, "bin_rows_num");
  k_bin_scatter<<<(unsigned)((p->m + 255) / 256), 256, 0, p->stream>>>(p->rbin2, p->m, p->d_num_off,
                                                                      p->dc->num_cursor, p->perm2, kNumNumBins);
  return cudaGetLastError();
}

// Rows grouped by symbolic bin (after enqueue_flop).
cudaError_t enqueue_sym_scatter(spgemm_plan_s *p) {
  if (p->m == 0) return cudaSuccess;
  KernelScope ks(p, "bin_rows_sym");
  k_bin_scatter<<<(unsigned)((p->m + 255) / 256), 256, 0, p->stream>>>(p->rbin, p->m, p->d_sym_off, p->dc->sym_cursor,
                                                                      p->perm, kNumSymBins);
  return cudaGetLastError();
}

}  // namespace sg

extern "C" {

int spgemm_plan_create_tuned(spgemm_plan_t *out, const spgemm_csr *A, const spgemm_csr *B, int dtype,
                             unsigned flags, void *stream, const spgemm_tuning *tuning) {
  NvtxRange nvtx("spgemm_plan_create");
  if (!out) return SPGEMM_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  spgemm_plan_s *p = nullptr;
  {
    const int rc0 = plan_init(&p, A, B, dtype, flags, (cudaStream_t)stream, tuning, false);
    if (rc0 != SPGEMM_OK) return rc0;
  }
  const int64_t m = p->m;
  int rc = SPGEMM_OK;
  cudaError_t e = enqueue_flop(p);
  if (e != cudaSuccess) rc = fail_cuda(e, "row flop pass");
  if (rc == SPGEMM_OK) rc = read_counters(p);
  if (rc == SPGEMM_OK) {
    p->total_flop = (int64_t)p->hc->total_flop;
    p->max_flop = (int64_t)p->hc->max_flop;
    // lanes per stored a_ik: the mean length of the B rows the products come
    // from (flop / nnz(A)), so that long rows get whole warps
    p->nnz_a_used = (int64_t)p->hc->nnz_a_used;
    const bool compact = m > 0 && p->total_flop > 0 && 2 * p->nnz_a_used < p->nnz_a;
    const int64_t walked = compact ? p->nnz_a_used : p->nnz_a;
    const double per_entry = walked > 0 ? (double)p->total_flop / (double)walked : 0.0;
    p->G = per_entry >= 24 ? 32 : per_entry >= 12 ? 16 : per_entry >= 6 ? 8 : 4;
    if (p->tune_G) p->G = p->tune_G;
    p->sym_off[0] = 0;
    for (int b = 0; b < kNumSymBins; ++b) {
      p->sym_flop[b] = (int64_t)p->hc->sym_flop[b];
      p->sym_count[b] = (int64_t)p->hc->sym_count[b];
      p->sym_off[b + 1] = p->sym_off[b] + p->sym_count[b];
    }
    if (compact) rc = compact_a(p);
    const int64_t nbm = p->sym_count[kSymBitmapBin] + p->sym_count[kSymBitmapMidBin];
    p->n_long = p->long_min > 0 ? std::min<int64_t>((int64_t)p->hc->n_long, p->long_cap) : 0;
    p->long_tot = p->long_min > 0 ? (int64_t)p->hc->long_tot : 0;
    if (rc == SPGEMM_OK && nbm > 0 && p->n_long > 0) {
      e = long_rows_build(p);
      if (e != cudaSuccess) rc = fail_cuda(e, "long rows of B");
    }
    if (rc == SPGEMM_OK && nbm > 0) {
      p->bitmaps_bytes = (size_t)nbm * p->bm_words * 4;
      e = cudaMallocAsync((void **)&p->bitmaps, p->bitmaps_bytes, p->stream);
      if (e != cudaSuccess) {
        p->bitmaps = nullptr;
        rc = fail_cuda(e, "allocating row bitmaps");
      }
    }
    if (rc == SPGEMM_OK && p->sym_count[kSymGlobalBin] > 0)
      // at least 64 slots: chunked probing reads 4 at a time
      rc = alloc_gtab(p, std::max<int64_t>(64, pow2_above((int64_t)p->hc->max_bound_global)), 4,
                      p->sym_count[kSymGlobalBin]);
    if (rc == SPGEMM_OK && m > 0) {
      e = enqueue_sym_scatter(p);
      if (e != cudaSuccess) rc = fail_cuda(e, "row binning");
    }
  }
  if (rc != SPGEMM_OK) {
    free_ws(p);
    delete p->hc;
    delete p;
    return rc;
  }
  p->state = 0;
  *out = p;
  return SPGEMM_OK;
}

int spgemm_symbolic(spgemm_plan_t p, int32_t *c_row_ptr, int64_t *nnz_c) {
  NvtxRange nvtx("spgemm_symbolic");
  if (!p || !c_row_ptr || !nnz_c) return SPGEMM_ERR_INVALID_ARGUMENT;
  if (p->state != 0) return SPGEMM_ERR_BAD_STATE;
  g_last_error.clear();
  cudaError_t e = enqueue_symbolic(p, c_row_ptr);
  if (e != cudaSuccess) return fail_cuda(e, "symbolic phase");
  const int64_t m = p->m;
  int rc = read_counters(p);
  if (rc != SPGEMM_OK) return rc;
  p->nnz_c = m > 0 ? (int64_t)p->hc->nnz_c : 0;
  p->num_off[0] = 0;
  for (int b = 0; b < kNumNumBins; ++b) {
    p->num_flop[b] = (int64_t)p->hc->num_flop[b];
    p->num_count[b] = (int64_t)p->hc->num_count[b];
    p->num_off[b + 1] = p->num_off[b] + p->num_count[b];
  }
  // the bitmap bins hold work items (row, rank window, part), not rows of perm2
  const int bm_bins[3] = {kNumBitmapSBin, kNumBitmapMBin, kNumBitmapBin};
  p->bm_item_off[0] = 0;
  for (int c = 0; c < 3; ++c) {
    p->num_count[bm_bins[c]] = (int64_t)p->hc->bm_items[c];
    p->num_flop[bm_bins[c]] = (int64_t)p->hc->bm_flop[c];
    p->bm_item_off[c + 1] = p->bm_item_off[c] + p->num_count[bm_bins[c]];
    int64_t at = p->bm_item_off[c];  // heaviest bucket first
    for (int q = 0; q < kBmBuckets; ++q) {
      p->bm_bucket_off[c][q] = at;
      at += (int64_t)p->hc->bm_bucket[c][q];
    }
  }
  *nnz_c = p->nnz_c;
  p->c_rp = c_row_ptr;
  p->state = 1;
  return SPGEMM_OK;
}

// Structure-only part of the numeric phase (bitmap work items, global
// tables, rows grouped by numeric bin): run by the first numeric call.
static int numeric_prepare(spgemm_plan_t p) {
  const int64_t m = p->m;
  cudaError_t e = cudaSuccess;
  const int64_t nitems = p->bm_item_off[3];
  if (nitems > 0) {
    p->bm_items_bytes = (size_t)nitems * sizeof(int4);
    e = cudaMallocAsync((void **)&p->bm_items, p->bm_items_bytes, p->stream);
    if (e != cudaSuccess) {
      p->bm_items = nullptr;
      return fail_cuda(e, "allocating bitmap work items");
    }
    const int64_t nbm = p->sym_count[kSymBitmapBin] + p->sym_count[kSymBitmapMidBin];
    KernelScope ks(p, "bm_items_fill");
    BmCaps caps{{p->bm_cap[0], p->bm_cap[1], p->bm_cap[2]}, {}};
    for (int c = 0; c < 3; ++c)
      for (int q = 0; q < kBmBuckets; ++q) caps.off[c][q] = p->bm_bucket_off[c][q];
    k_bm_items_fill<<<(unsigned)((nbm + 255) / 256), 256, 0, p->stream>>>(
        p->perm + p->sym_off[kSymBitmapBin], nbm, p->nnz_row, p->flop, caps, p->dc, p->bm_items);
  }
  if (p->num_count[kNumGlobalBin] > 0) {
    const int64_t slots = std::max<int64_t>(64, pow2_above((int64_t)p->hc->max_nnz_global * 4 / 3));
    const int rc = alloc_gtab(p, slots, 4 + value_size(p->dtype), p->num_count[kNumGlobalBin]);
    if (rc != SPGEMM_OK) return rc;
  }
  (void)m;
  e = enqueue_num_scatter(p);
  if (e != cudaSuccess) return fail_cuda(e, "numeric binning");
  return SPGEMM_OK;
}

// Value-dependent part: the numeric kernels of every bin.
static cudaError_t numeric_launch(spgemm_plan_t p, const int32_t *c_row_ptr, int32_t *c_col_idx, void *c_vals) {
  switch (p->dtype) {
    case SPGEMM_F64: return launch_numeric_f64(p, c_row_ptr, c_col_idx, c_vals);
    case SPGEMM_F32: return launch_numeric_f32(p, c_row_ptr, c_col_idx, c_vals);
    default: return launch_numeric_i64(p, c_row_ptr, c_col_idx, c_vals);
  }
}

// The numeric kernels of rows [lo, hi) (every row: 0, INT32_MAX).
static int numeric_run(spgemm_plan_t p, const int32_t *c_row_ptr, int32_t *c_col_idx, void *c_vals, int32_t lo,
                       int32_t hi) {
  if (p->state != 1 && p->state != 2) return SPGEMM_ERR_BAD_STATE;
  if (p->nnz_c > 0 && (!c_col_idx || !c_vals)) return SPGEMM_ERR_INVALID_ARGUMENT;
  g_last_error.clear();
  if (p->nnz_c > 0) {
    if (lo >= hi) return SPGEMM_OK;  // no rows: the plan's state is unchanged
    if (p->state == 1) {
      const int rc = numeric_prepare(p);
      if (rc != SPGEMM_OK) return rc;
      p->state = 2;
    }
    p->row_lo = lo;
    p->row_hi = hi;
    const cudaError_t e = numeric_launch(p, c_row_ptr, c_col_idx, c_vals);
    p->row_lo = 0;
    p->row_hi = INT32_MAX;
    if (e != cudaSuccess) return fail_cuda(e, "numeric kernels");
  }
  p->state = 2;
  return SPGEMM_OK;
}

int spgemm_numeric(spgemm_plan_t p, const int32_t *c_row_ptr, int32_t *c_col_idx, void *c_vals) {
  NvtxRange nvtx("spgemm_numeric");
  if (!p || !c_row_ptr) return SPGEMM_ERR_INVALID_ARGUMENT;
  return numeric_run(p, c_row_ptr, c_col_idx, c_vals, 0, INT32_MAX);
}

int spgemm_numeric_rows(spgemm_plan_t p, int64_t row_begin, int64_t row_end, const int32_t *c_row_ptr,
                        int32_t *c_col_idx, void *c_vals) {
  NvtxRange nvtx("spgemm_numeric_rows");
  if (!p || !c_row_ptr || row_begin < 0 || row_end < row_begin || row_end > p->m) return SPGEMM_ERR_INVALID_ARGUMENT;
  return numeric_run(p, c_row_ptr, c_col_idx, c_vals, (int32_t)row_begin, (int32_t)row_end);
}

int spgemm_numeric_graph(spgemm_plan_t p, const int32_t *c_row_ptr, int32_t *c_col_idx, void *c_vals) {
  NvtxRange nvtx("spgemm_numeric_graph");
  if (!p || !c_row_ptr) return SPGEMM_ERR_INVALID_ARGUMENT;
  if (p->state != 2) return SPGEMM_ERR_BAD_STATE;
  if (p->flags & SPGEMM_TIMING) {
    set_last_error("spgemm_numeric_graph: plans created with SPGEMM_TIMING time every kernel; use spgemm_numeric");
    return SPGEMM_ERR_INVALID_ARGUMENT;
  }
  if (p->nnz_c > 0 && (!c_col_idx || !c_vals)) return SPGEMM_ERR_INVALID_ARGUMENT;
  g_last_error.clear();
  if (p->nnz_c == 0) return SPGEMM_OK;
  cudaError_t e = cudaSuccess;
  const bool same = p->graph_exec && p->graph_rp == c_row_ptr && p->graph_ci == c_col_idx && p->graph_cv == c_vals;
  if (!same) {
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    p->graph_exec = nullptr;
    cudaGraph_t graph = nullptr;
    // the default streams cannot be captured: capture on a private stream
    // (the graph does not depend on the stream that recorded it) and launch
    // the graph into the plan's stream
    cudaStream_t cap = p->stream;
    const bool private_stream = p->stream == nullptr || p->stream == cudaStreamLegacy ||
                                p->stream == cudaStreamPerThread;
    if (private_stream) {
      e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
      if (e != cudaSuccess) return fail_cuda(e, "numeric graph capture stream");
    }
    const cudaStream_t saved = p->stream;
    p->stream = cap;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    cudaError_t el = cudaSuccess;
    if (e == cudaSuccess) {
      el = numeric_launch(p, c_row_ptr, c_col_idx, c_vals);
      e = cudaStreamEndCapture(cap, &graph);
    }
    p->stream = saved;
    if (private_stream) cudaStreamDestroy(cap);
    if (el != cudaSuccess || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return fail_cuda(el != cudaSuccess ? el : e, "numeric graph capture");
    }
    e = cudaGraphInstantiate(&p->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      p->graph_exec = nullptr;
      return fail_cuda(e, "numeric graph instantiation");
    }
    p->graph_rp = c_row_ptr;
    p->graph_ci = c_col_idx;
    p->graph_cv = c_vals;
  }
  e = cudaGraphLaunch(p->graph_exec, p->stream);
  if (e != cudaSuccess) return fail_cuda(e, "numeric graph launch");
  return SPGEMM_OK;
}

int spgemm_plan_destroy(spgemm_plan_t p) {
  if (!p) return SPGEMM_OK;
  free_ws(p);
  delete p->hc;
  delete p;
  return SPGEMM_OK;
}

int spgemm_plan_kernel_times(spgemm_plan_t p, spgemm_kernel_time *out, int max_entries, int *n_out) {
  if (!p || !n_out || (max_entries > 0 && !out)) return SPGEMM_ERR_INVALID_ARGUMENT;
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return fail_cuda(e, "timing sync");
  std::vector<std::string> names;
  std::vector<float> ms;
  std::vector<int> cnt;
  for (auto &t : p->timed) {
    float x = 0.f;
    if (cudaEventElapsedTime(&x, t.start, t.stop) != cudaSuccess) x = 0.f;
    size_t j = 0;
    while (j < names.size() && names[j] != t.name) ++j;
    if (j == names.size()) {
      names.push_back(t.name);
      ms.push_back(0.f);
      cnt.push_back(0);
    }
    ms[j] += x;
    cnt[j] += 1;
  }
  *n_out = (int)names.size();
  for (int j = 0; j < (int)names.size() && j < max_entries; ++j) {
    std::memset(out[j].name, 0, sizeof(out[j].name));
    std::strncpy(out[j].name, names[j].c_str(), sizeof(out[j].name) - 1);
    out[j].ms = ms[j];
    out[j].launches = cnt[j];
  }
  return SPGEMM_OK;
}

int spgemm_plan_workspace_bytes(spgemm_plan_t p, size_t *bytes) {
  if (!p || !bytes) return SPGEMM_ERR_INVALID_ARGUMENT;
  *bytes = p->ws_fixed_bytes + (p->bitmaps ? p->bitmaps_bytes : 0) + (p->bm_items ? p->bm_items_bytes : 0) +
           (p->gtab ? p->gtab_bytes : 0) + (p->long_ws ? p->long_ws_bytes : 0) + (p->acmp_ws ? p->acmp_bytes : 0);
  return SPGEMM_OK;
}

int spgemm_plan_stats(spgemm_plan_t p, spgemm_stats *s) {
  if (!p || !s) return SPGEMM_ERR_INVALID_ARGUMENT;
  int rc = read_counters(p);
  std::memset(s, 0, sizeof(*s));
  s->m = p->m;
  s->n = p->n;
  s->k = p->k;
  s->total_flop = p->total_flop;
  s->max_row_flop = p->max_flop;
  s->nnz_c = p->nnz_c;
  {
    long long acc[4] = {0, 0, 0, 0};
    for (int r = 0; r < 4; ++r)
      for (int j = 0; j < kProbeSlots; ++j) acc[r] += (long long)p->hc->probe_stats[r][j];
    s->sym_probes = acc[0];
    s->sym_inserts = acc[1];
    s->num_probes = acc[2];
    s->num_inserts = acc[3];
  }
  s->n_sym_bins = kNumSymBins;
  s->n_num_bins = kNumNumBins;
  for (int b = 0; b < kNumSymBins; ++b) {
    s->sym_bin_flop[b] = p->sym_flop[b];
    s->sym_bin_rows[b] = p->sym_count[b];
    s->sym_bin_table[b] = kSymBins[b].table;
  }
  for (int b = 0; b < kNumNumBins; ++b) {
    s->num_bin_flop[b] = p->num_flop[b];
    s->num_bin_rows[b] = p->num_count[b];
    s->num_bin_table[b] = kNumBins[b].table;
  }
  size_t ws = 0;
  spgemm_plan_workspace_bytes(p, &ws);
  s->workspace_bytes = (int64_t)ws;
  s->kernel_launches = p->launches;
  s->state = p->state;
  s->nnz_a_walked = p->a_compact ? p->nnz_a_used : p->nnz_a;
  s->long_rows = p->long_ready ? p->n_long : 0;
  s->long_entries = p->long_ready ? p->long_tot : 0;
  return rc;
}

int spgemm_plan_row_flop(spgemm_plan_t p, int64_t *flop_out) {
  if (!p || (!flop_out && p->m > 0)) return SPGEMM_ERR_INVALID_ARGUMENT;
  if (p->m == 0) return SPGEMM_OK;
  cudaError_t e = cudaMemcpyAsync(flop_out, p->flop, (size_t)p->m * 8, cudaMemcpyDeviceToDevice, p->stream);
  return e == cudaSuccess ? SPGEMM_OK : fail_cuda(e, "copy flop");
}

int spgemm_plan_sym_bins(spgemm_plan_t p, int32_t *perm_out, int64_t *offsets) {
  if (!p || !offsets || (!perm_out && p->m > 0)) return SPGEMM_ERR_INVALID_ARGUMENT;
  for (int b = 0; b <= kNumSymBins; ++b) offsets[b] = p->sym_off[b];
  const int64_t n = p->sym_off[kNumSymBins];
  if (n == 0) return SPGEMM_OK;
  cudaError_t e = cudaMemcpyAsync(perm_out, p->perm, (size_t)n * 4, cudaMemcpyDeviceToDevice, p->stream);
  return e == cudaSuccess ? SPGEMM_OK : fail_cuda(e, "copy perm");
}

int spgemm_plan_row_nnz(spgemm_plan_t p, int32_t *nnz_out) {
  if (!p || (!nnz_out && p->m > 0)) return SPGEMM_ERR_INVALID_ARGUMENT;
  if (p->state < 1) return SPGEMM_ERR_BAD_STATE;
  if (p->m == 0) return SPGEMM_OK;
  cudaError_t e = cudaMemcpyAsync(nnz_out, p->nnz_row, (size_t)p->m * 4, cudaMemcpyDeviceToDevice, p->stream);
  return e == cudaSuccess ? SPGEMM_OK : fail_cuda(e, "copy nnz_row");
}

int spgemm(const spgemm_csr *A, const spgemm_csr *B, int dtype, unsigned flags, void *stream, spgemm_alloc_fn alloc,
           void *alloc_ctx, int32_t **c_row_ptr, int32_t **c_col_idx, void **c_vals, int64_t *nnz_c) {
  if (!alloc || !c_row_ptr || !c_col_idx || !c_vals || !nnz_c || !A) return SPGEMM_ERR_INVALID_ARGUMENT;
  *c_row_ptr = nullptr;
  *c_col_idx = nullptr;
  *c_vals = nullptr;
  *nnz_c = 0;
  spgemm_plan_t p = nullptr;
  int rc = spgemm_plan_create(&p, A, B, dtype, flags, stream);
  if (rc != SPGEMM_OK) return rc;
  int32_t *rp = (int32_t *)alloc((size_t)(A->nrows + 1) * 4, alloc_ctx);
  if (!rp) {
    spgemm_plan_destroy(p);
    return SPGEMM_ERR_OUT_OF_MEMORY;
  }
  rc = spgemm_symbolic(p, rp, nnz_c);
  if (rc == SPGEMM_OK) {
    const size_t nz = (size_t)*nnz_c;
    const size_t vs = dtype == SPGEMM_F32 ? 4 : 8;
    int32_t *ci = (int32_t *)alloc(nz > 0 ? nz * 4 : 16, alloc_ctx);
    void *cv = alloc(nz > 0 ? nz * vs : 16, alloc_ctx);
    if (!ci || !cv) rc = SPGEMM_ERR_OUT_OF_MEMORY;
    if (rc == SPGEMM_OK) rc = spgemm_numeric(p, rp, ci, cv);
    *c_col_idx = ci;
    *c_vals = cv;
  }
  *c_row_ptr = rp;
  spgemm_plan_destroy(p);
  return rc;
}

}  // extern "C"

namespace sg {

int plan_create_graph(spgemm_plan_s **out, const spgemm_csr *A, const spgemm_csr *B, int dtype, unsigned flags,
                      cudaStream_t stream, const spgemm_tuning *tuning, const GraphCaps &gc) {
  if (!out) return SPGEMM_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  if (flags & (SPGEMM_TIMING | SPGEMM_COUNT_PROBES)) {
    set_last_error("a batch graph replays captured kernels: SPGEMM_TIMING and SPGEMM_COUNT_PROBES do not apply");
    return SPGEMM_ERR_INVALID_ARGUMENT;
  }
  if (gc.nnz_cap < 0 || gc.nnz_cap > INT32_MAX) return SPGEMM_ERR_INVALID_ARGUMENT;
  spgemm_plan_s *p = nullptr;
  int rc = plan_init(&p, A, B, dtype, flags, stream, tuning, true);
  if (rc != SPGEMM_OK) return rc;
  p->total_flop = gc.total_flop;
  p->max_flop = gc.max_flop;
  const double per_entry = p->nnz_a > 0 ? (double)gc.total_flop / (double)p->nnz_a : 0.0;
  p->G = per_entry >= 24 ? 32 : per_entry >= 12 ? 16 : per_entry >= 6 ? 8 : 4;
  if (p->tune_G) p->G = p->tune_G;
  p->max_nnz_c = gc.nnz_cap;
  if (gc.span_cols > 0) p->span_cols = gc.span_cols;
  for (int b = 0; b < kNumSymBins; ++b) p->sym_count[b] = gc.sym_rows[b];
  for (int b = 0; b < kNumNumBins; ++b) p->num_count[b] = gc.num_rows[b];
  // global tables, for the largest heavy row the planning pass saw
  const int64_t sym_slots = gc.max_bound > kBlockSymMax ? std::max<int64_t>(64, pow2_above(gc.max_bound)) : 0;
  const int64_t num_slots =
      gc.max_nnz > p->caps.cap[8] ? std::max<int64_t>(64, pow2_above(gc.max_nnz * 4 / 3)) : 0;
  const int64_t slots = std::max(sym_slots, num_slots);
  p->gcap_bound = p->gcap_nnz = slots;
  if (slots > 0) rc = alloc_gtab(p, slots, 4 + value_size(dtype), 2 * (int64_t)sm_count());
  if (rc == SPGEMM_OK && use_side_streams(p)) {
    const cudaError_t e = acquire_side(p);  // before any capture
    if (e != cudaSuccess) rc = fail_cuda(e, "side streams");
  }
  if (rc != SPGEMM_OK) {
    plan_free(p);
    return rc;
  }
  p->state = 1;
  *out = p;
  return SPGEMM_OK;
}

cudaError_t plan_enqueue_graph(spgemm_plan_s *p, int32_t *c_rp, int32_t *c_ci, void *c_v) {
  cudaError_t e = enqueue_flop(p);
  if (e == cudaSuccess) e = enqueue_sym_scatter(p);
  if (e == cudaSuccess) e = enqueue_symbolic(p, c_rp);
  if (e == cudaSuccess) e = enqueue_num_scatter(p);
  if (e == cudaSuccess && p->m > 0) e = numeric_launch(p, c_rp, c_ci, c_v);
  return e;
}

void plan_free(spgemm_plan_s *p) {
  if (!p) return;
  free_ws(p);
  delete p->hc;
  delete p;
}

}  // namespace sg
