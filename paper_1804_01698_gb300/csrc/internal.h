// Plan object and kernel launchers of the GB300 hash SpGEMM (host side).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/spgemm.h"
#include "common.cuh"

namespace sg {

// ---------------------------------------------------------------------------
// Row bins.  The paper balances rows over threads by flop (Sec. 4.1) and
// sizes each thread's hash table from the largest flop of its rows
// (Sec. 4.2.1); GPU hash SpGEMM instead bins rows by density and runs one
// kernel per bin (Sec. 2).  Here a row goes to the smallest bin whose table
// holds its key bound with the bin's load factor:
//   symbolic bound  = min(flop_i, ncols(B))      (Fig. "Hash_SpGEMM")
//   numeric  bound  = nnz(c_i*)                  (exact, from symbolic)
// Warp bins: one warp per row, table in shared memory.
// Block bins: one thread block per row, table in shared memory.
// Heavy rows: a column bitmap in shared memory when ncols(B) is small
// enough (BITMAP), otherwise a hash table in global memory (GLOBAL).
enum BinKind { kWarp = 0, kBlock = 1, kBitmap = 2, kGlobal = 3 };

struct BinCfg {
  int kind;
  int table;    // hash table slots (power of two), 0 for bitmap/global bins
  int threads;  // threads per block
  int64_t cap;  // largest bound this bin accepts
};

constexpr int kNumHashBins = 10;     // warp 64..1024, block 2048..32768
constexpr int kSymBitmapBin = 10;    // bitmap rows with bound > kBitmapMidMax (split into parts)
constexpr int kSymBitmapMidBin = 11; // bitmap rows with bound <= kBitmapMidMax (256 threads)
constexpr int kSymGlobalBin = 12;
constexpr int kNumSymBins = 13;
// numeric bins 0..8 are hash bins; bitmap rows become work items in three
// classes by row size: small (3 blocks per SM), medium (2), large (1; the
// ranks of a row beyond one block's shared array go straight into C)
constexpr int kNumBitmapBin = 9;     // large class
constexpr int kNumGlobalBin = 10;
constexpr int kNumBitmapSBin = 11;   // small class
constexpr int kNumBitmapMBin = 12;   // medium class
constexpr int kNumNumBins = 13;
constexpr int kWarpsPerBlock = 4;  // warp bins: rows per block
// shared memory kept free beside a bitmap kernel's dynamic allocation for
// its static arrays (staging of 256 entries and their long-row list,
// reductions)
constexpr int kStaticSmemReserve = 256 * 24 + 2048;

// Symbolic bins 0..9: tables 64 .. 32768 slots, load factor 1/2 for warp
// tables and 3/4 for block tables (the bound overestimates the key count
// by the compression ratio, so the true load is lower).
extern const BinCfg kSymBins[kNumSymBins];
// Numeric bins 0..8: tables 64 .. 16384 slots, same load factors.
extern const BinCfg kNumBins[kNumNumBins];

// Rows whose symbolic bound exceeds bitmap_min_bound(k) (at least
// kBitmapMinBound) use a column bitmap when B has at most kBitmapMaxCols
// columns: the symbolic phase builds and saves the bitmap, the numeric phase
// turns it into output positions.  Without bitmaps, rows above the largest
// shared-memory table (3/4 of 32768 keys) use global-memory hash tables.
constexpr int64_t kBitmapMinBound = 512;

// Launch shapes of the numeric bitmap classes (threads a block, blocks an
// SM): small, medium, large.  Shared memory per block is sized so that the
// blocks fit an SM; the registers a thread then gets follow from the shape
// (small 40, medium 64, large 64).  Measured on R-MAT A*A, scale 16: medium
// blocks of 512 threads ran 10% faster than 1024 (which spill at 32
// registers); small blocks of 256 threads 20% slower than 512.
constexpr int kBmThreadsS = 512, kBmBlocksS = 3;
constexpr int kBmThreadsM = 512, kBmBlocksM = 2;
constexpr int kBmThreadsL = 1024;

constexpr int64_t kBitmapMidMax = 24576;
constexpr int64_t kBlockSymMax = 24576;      // 3/4 of 32768 (global-table inputs)
constexpr int64_t kBitmapMaxCols = 1 << 18;  // bitmap + prefix <= 64 KB
// Bitmap threshold for B with k columns (0: no bitmaps): rows whose
// symbolic bound exceeds max(kBitmapMinBound, words / 2), words = k/32,
// take the bitmap path.  A bitmap row pays for its words (zeroing,
// counting, saving, prefix, output walk) whatever its size, so the
// threshold grows with the word count; measured on R-MAT16 (2048 words),
// moving it from 3072 to 1024 cut the product by 4%.
inline int64_t bitmap_min_bound(int64_t k) {
  if (k > kBitmapMaxCols) return 0;
  const int64_t half_words = (k + 31) / 32 / 2;
  return half_words > kBitmapMinBound ? half_words : kBitmapMinBound;
}

// A bitmap row whose flop is large next to its output is split over several
// blocks, each taking a contiguous range of the row's stored a_ik (equal
// flop) and adding its partial sums into C with global atomics.  Every part
// keeps at least max(kSplitMinFlop, kSplitFlopPerEntry * nnz) products, so
// the atomic adds stay a small fraction of its products.
constexpr long long kSplitMinFlop = 65536;
constexpr long long kSplitFlopPerEntry = 8;
constexpr long long kSplitMaxParts = 64;

// The symbolic phase of a heavy bitmap row (bin kSymBitmapBin) is split the
// same way when its flop reaches kSymSplitFlop: one part per kSymSplitFlop
// products, each ORing its partial bitmap into the row's saved bitmap; the
// last part to finish counts it.  With 256-thread blocks, parts of 32768
// products ran the heavy symbolic rows of R-MAT A*A (scale 16) 22% faster
// and those of the triangle product 37% faster than parts of 131072.
constexpr long long kSymSplitFlop = 32768;
__host__ __device__ inline int sym_split_parts(long long flop) {
  long long parts = flop / kSymSplitFlop;
  if (parts < 1) parts = 1;
  if (parts > kSplitMaxParts) parts = kSplitMaxParts;
  return (int)parts;
}

__host__ __device__ inline int bm_split_parts(long long flop, long long nnz) {
  const long long unit = kSplitMinFlop > kSplitFlopPerEntry * nnz ? kSplitMinFlop : kSplitFlopPerEntry * nnz;
  long long parts = flop / unit;
  if (parts < 1) parts = 1;
  if (parts > kSplitMaxParts) parts = kSplitMaxParts;
  return (int)parts;
}
// Numeric bitmap work items run heaviest first within each class: an item
// of a row with flop f in `parts` parts walks f / parts products, and the
// items go to kBmBuckets buckets by that weight (bucket 0: 2^20 products
// and more, each next bucket half the weight of the one before, the last
// every lighter item).  Blocks start roughly in index order, so a heavy
// item no longer starts near the end of the launch while the other SMs run
// dry (longest processing time first, bucketed).
constexpr int kBmBuckets = 8;
__host__ __device__ inline int bm_bucket_of(long long flop, int parts) {
  const long long w = flop / (parts > 0 ? parts : 1);
  int lg = 0;
  while (lg < 62 && (w >> (lg + 1)) > 0) ++lg;  // floor(log2(w)), 0 for w <= 1
  const int b = 20 - lg;
  return b < 0 ? 0 : b > kBmBuckets - 1 ? kBmBuckets - 1 : b;
}
// Long rows of B.  Inside bitmap rows of A, the symbolic phase does not take
// the products of a row k of B with at least long_row_min entries one by
// one: it ORs k's saved column bitmap into the row's bitmap.  The rule below
// is the default threshold (spgemm_tuning).
// Measured on R-MAT A*A, scale 16 (k = 2^16): thresholds 256, 512 and 1024
// gave 4.26, 4.23 and 4.25 ms per product; 64 and 128 were 10-30% slower.
inline int64_t long_row_min_default(int64_t k) {
  const int64_t q = k / 128;
  return q > 512 ? q : 512;
}

// Device view of a plan's long rows (map == nullptr: none).
struct LongRows {
  const int32_t *map;    // per row of B: its long-row index d, or -1
  const uint32_t *bits;  // column bitmap of long row d: bits[d * words + w]
};

// Rows of one bin: perm[off[bin]] .. perm[off[bin + 1] - 1].  The offsets
// live in device memory, written by a kernel from the bin counts, so that
// the bin kernels also find their rows when the host has not read the
// counts (a captured CUDA graph of whole products); the kernels walk their
// rows grid-stride, with exact grids when the host knows the counts and
// persistent grids otherwise.
struct BinRows {
  const int32_t *perm;
  const long long *off;
  int bin;
};

// Largest key bound of each hash bin (warp tables 64..1024 slots, block
// tables 2048..16384): a row goes to the first bin whose cap holds its
// bound.  Default loads: 1/2 of a warp table, 3/4 of a block table.
struct HashCaps {
  long long cap[9];
};
HashCaps hash_caps(int warp_load_pct, int block_load_pct);

// block-bin sort: a row whose columns span at most 4096 words (131072
// columns) is ranked through a bitmap of its window; measured on R-MAT
// scale 17 A*A (2^17 columns), 4096 words ran sorted output 17% faster than
// 2048 (whose wider rows fell back to bitonic sorting)
constexpr int64_t kSortWindowWords = 4096;

// Device counters of a plan (zeroed at creation).
struct DevCounters {
  unsigned long long sym_count[kNumSymBins];
  unsigned long long sym_cursor[kNumSymBins];
  unsigned long long num_count[kNumNumBins];
  unsigned long long num_cursor[kNumNumBins];
  unsigned long long sym_flop[kNumSymBins];
  unsigned long long num_flop[kNumNumBins];
  unsigned long long total_flop;
  unsigned long long max_flop;
  unsigned long long max_bound_global;  // largest symbolic bound in the global bin
  unsigned long long nnz_c;
  unsigned long long max_nnz_global;    // largest nnz in the numeric global bin
  unsigned long long bm_items[3];       // numeric bitmap work items per class (small, medium, large)
  unsigned long long bm_bucket[3][kBmBuckets];  // the same per weight bucket (bm_bucket_of)
  unsigned long long bm_cursor[3][kBmBuckets];
  unsigned long long bm_flop[3];        // flop of the rows of each class
  unsigned long long sym_split_extra;   // heavy symbolic bitmap rows: parts beyond one per row
  unsigned long long sym_item_cursor;
  unsigned long long n_long;            // long rows of B, and their entries
  unsigned long long long_tot;
  unsigned long long nnz_a_used;        // stored a_ik whose row of B is not empty
  unsigned long long scan_total;        // total of the compacted A's row scan
  // SPGEMM_COUNT_PROBES: rows 0/1 symbolic probes/inserts, 2/3 numeric,
  // each spread over kProbeSlots counters to limit atomic contention
  unsigned long long probe_stats[4][kProbeSlots];
  unsigned int err;
  unsigned int sym_ticket;  // blocks of k_row_bin done (the last one writes the symbolic bin offsets)
  unsigned int num_ticket;  // the same for k_num_classify and the numeric bin offsets
  unsigned int pad;
};

// Hash-table variants of a plan (Args::probe bits).
constexpr int kProbeChunk = 1;   // chunks of 4 slots per probe
constexpr int kProbeHashHi = 2;  // slot from the top bits of col * kHashScale (default)
inline int probe_mode(unsigned flags) {
  return ((flags & SPGEMM_PROBE_CHUNK4) ? kProbeChunk : 0) | ((flags & SPGEMM_HASH_LOW_BITS) ? 0 : kProbeHashHi);
}

// Kernel arguments common to all phases.
// Merge-path split of a CSR matrix's rows (Merrill and Garland's merge-based
// CSR traversal): the items are the m row ends and the nnz stored entries,
// in the order a row-by-row walk meets them (row i's entries, then its
// end).  Diagonal d (0 <= d <= m + nnz) of that walk is at row i, entry j
// with i + j = d: rows below i are finished and entries below j consumed.
// Threads and items (row ends + entries) per thread of the merge-path kernels.
constexpr int kMergeThreads = 256, kMergeIPT = 8, kMergeTile = kMergeThreads * kMergeIPT;
// Kept entries (row of B not empty) that the flop pass lists per tile for the
// compaction; a tile with more is walked again.
constexpr int kKeptListCap = 128;

// Start (row, entry) of every merge-path tile: row i's entries and end take
// diagonals [i + rp[i], i + rp[i + 1]], and tile t starts at diagonal
// t * kMergeTile.  One coalesced pass over the row pointers instead of a
// binary search per tile; starts[2 * tiles] = (m, nnz) ends the last tile.
// A malformed row (its range outside [0, m + nnz]) writes nothing, and the
// walk clamps what it reads.  Also zeroes flop[] and kept[] (null: not) for
// the atomics of the walk that follows.
// Long rows of B (see longrows.cu): row k of B is long when it has at least
// long_min entries; long rows get an index d (lmap[k] = d, lrow[d] = k).
struct LongMark {
  const int32_t *brp;
  int64_t n, nnz_b, long_min, cap;
  int32_t *lmap, *lrow;
};
__device__ __forceinline__ void long_mark_row(const LongMark &lm, int64_t k, DevCounters *dc) {
  const int64_t b0 = lm.brp[k], b1 = lm.brp[k + 1];
  int32_t d = -1;
  // a malformed row is never long (the flop pass reports it when A selects it)
  if (0 <= b0 && b0 <= b1 && b1 <= lm.nnz_b && b1 - b0 >= lm.long_min) {
    const unsigned long long idx = atomicAdd(&dc->n_long, 1ull);
    if ((int64_t)idx < lm.cap) {
      d = (int32_t)idx;
      lm.lrow[d] = (int32_t)k;
      atomicAdd(&dc->long_tot, (unsigned long long)(b1 - b0));
    }
  }
  lm.lmap[k] = d;
}

__global__ void __launch_bounds__(256)
    k_merge_starts(const int32_t *__restrict__ rp, int64_t m, int64_t nnz, int64_t tiles, long long *__restrict__ starts,
                   int64_t *__restrict__ flop, int32_t *__restrict__ kept, LongMark lm, DevCounters *dc);

// One tile of kMergeTile items of a merge-path walk over A, one block (tile
// blockIdx.x, its start and end read from starts[]): the
// B-row length of each of the tile's entries is gathered into shared memory
// (lens[j - j0]; entries whose column is outside B, or whose row of B is
// malformed, count 0 and raise kErrCsr), the row ends into ends[], and each
// thread walks kMergeIPT consecutive items.  For every row that ends in its
// items, the thread calls row(i, sum, kept, whole, j, len, n): the sum of
// the lengths of the row's entries among the thread's items, how many are
// non-zero, whether the row lies wholly in the thread's items, the first of
// those entries (j), their lengths (len[0..n)) and their number; for the row
// that continues past its items, it calls it with whole false if it met any
// of the row's entries.  rp must be monotone for the sums to be the rows'
// (the caller's row check reports it otherwise).  coords: 4 shared words.

template <typename F>
__device__ __forceinline__ void merge_tile_walk(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                                const int32_t *__restrict__ brp, int64_t m, int64_t nnz, int64_t nb,
                                                int64_t nnz_b, uint32_t *err, const long long *__restrict__ starts,
                                                int32_t *lens, int32_t *ends, long long *coords, F &&row) {
  const int64_t N = m + nnz;
  const int64_t D0 = (int64_t)blockIdx.x * kMergeTile;
  const int64_t D1 = D0 + kMergeTile < N ? D0 + kMergeTile : N;
  if (threadIdx.x < 4) coords[threadIdx.x] = starts[2 * (int64_t)blockIdx.x + threadIdx.x];
  __syncthreads();
  // for monotone row pointers both spans lie in A and within the tile;
  // clamped for any others
  auto clamp = [](int64_t v, int64_t lo, int64_t hi) { return v < lo ? lo : v > hi ? hi : v; };
  const int64_t ib0 = clamp(coords[0], 0, m), jb0 = clamp(coords[1], 0, nnz);
  const int64_t ni = clamp(coords[2] - ib0, 0, m - ib0 < kMergeTile ? m - ib0 : kMergeTile);
  const int64_t nj = clamp(coords[3] - jb0, 0, nnz - jb0 < kMergeTile ? nnz - jb0 : kMergeTile);
  for (int64_t t = threadIdx.x; t < nj; t += blockDim.x) {
    const int32_t kk = __ldg(ci + jb0 + t);
    int32_t len = 0;
    if ((uint64_t)(int64_t)kk < (uint64_t)nb) {
      const int32_t b0 = __ldg(brp + kk), b1 = __ldg(brp + kk + 1);
      if (0 <= b0 && b0 <= b1 && (int64_t)b1 <= nnz_b) len = b1 - b0;
      else raise_err(err, kErrCsr);
    } else {
      raise_err(err, kErrCsr);
    }
    lens[t] = len;
  }
  for (int64_t t = threadIdx.x; t < ni; t += blockDim.x) ends[t] = __ldg(rp + ib0 + t + 1);
  __syncthreads();
  // this thread's items: diagonals [d0, d1) of the tile, searched in the tile's lists
  auto local_search = [&](int64_t d, int64_t *i, int64_t *j) {
    int64_t lo = d - nj > 0 ? d - nj : 0, hi = d < ni ? d : ni;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if ((int64_t)ends[mid] - jb0 <= d - mid - 1) lo = mid + 1;
      else hi = mid;
    }
    *i = lo;
    *j = d - lo;
  };
  const int64_t span = D1 - D0;
  const int64_t d0 = (int64_t)threadIdx.x * kMergeIPT < span ? (int64_t)threadIdx.x * kMergeIPT : span;
  const int64_t d1 = d0 + kMergeIPT < span ? d0 + kMergeIPT : span;
  if (d0 >= d1) return;
  int64_t i, j, ie, je;
  local_search(d0, &i, &j);
  local_search(d1, &ie, &je);
  // the thread's first row lies wholly in its items when it starts at them
  bool whole = i < ni && (int64_t)__ldg(rp + ib0 + i) >= jb0 + j;
  for (; i < ie; ++i) {
    int64_t e = (int64_t)ends[i] - jb0;
    e = e < j ? j : e > je ? je : e;
    const int64_t first = j;
    long long sum = 0;
    int kept = 0;
    for (; j < e; ++j) {
      sum += lens[j];
      kept += lens[j] > 0;
    }
    row(ib0 + i, sum, kept, whole, jb0 + first, (const int32_t *)lens + first, (int)(e - first));
    whole = true;
  }
  if (j < je && ib0 + i < m) {
    const int64_t first = j;
    long long sum = 0;
    int kept = 0;
    for (; j < je; ++j) {
      sum += lens[j];
      kept += lens[j] > 0;
    }
    row(ib0 + i, sum, kept, false, jb0 + first, (const int32_t *)lens + first, (int)(je - first));
  }
}

struct Args {
  int64_t m, n, k;
  const int32_t *arp, *aci, *brp, *bci;
  const void *av, *bv;
  int G;  // lanes per stored a_ik
  uint32_t *err;
  int probe = 0;  // hash tables: kProbeChunk (SPGEMM_PROBE_CHUNK4) | kProbeHashHi (unless SPGEMM_HASH_LOW_BITS)
  // SPGEMM_COUNT_PROBES: this phase's probe counters (inserts at +kProbeSlots), else null
  unsigned long long *probe_ctr = nullptr;
  // graph mode: the plan's error word; a numeric kernel returns at once when
  // it holds kErrOverflow or kErrCapacity (C would not fit its buffers)
  const uint32_t *abort = nullptr;
  // per row of C, a column offset that the numeric kernels subtract from the
  // columns they store (a packed batch's rows store their product's own
  // columns); null: none
  const int32_t *col_base = nullptr;
  // numeric phase: only rows row_lo <= i < row_hi of C are computed and
  // written (spgemm_numeric_rows); the symbolic phase takes every row
  int32_t row_lo = 0, row_hi = INT32_MAX;
};

// Row i is inside the numeric phase's row range.
__device__ __forceinline__ bool in_rows(const Args &a, int32_t i) { return i >= a.row_lo && i < a.row_hi; }

// A numeric kernel of a graph-mode plan skips its work when the symbolic
// phase found that C does not fit the planned buffers.
__device__ __forceinline__ bool aborted(const Args &a) {
  return a.abort && (*(volatile const uint32_t *)a.abort & (kErrOverflow | kErrCapacity));
}

}  // namespace sg

namespace sg {
// An NVTX range for the lifetime of a scope (shown by profilers; no cost
// without one attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace sg

struct spgemm_plan_s {
  int64_t m, n, k, nnz_a, nnz_b;
  const int32_t *arp, *aci, *brp, *bci;
  const void *av, *bv;
  int dtype;
  unsigned flags;
  cudaStream_t stream;
  int device;
  int state;  // 0 planned, 1 symbolic done, 2 numeric done
  int G;
  int tune_G;            // spgemm_tuning::lanes_per_entry (0: chosen from the flop pass)
  int64_t tune_bm_min;   // spgemm_tuning::bitmap_min_bound (0: default rule, -1: no bitmaps)
  int64_t max_nnz_c;     // largest nnz(C) accepted (spgemm_tuning::max_nnz_c, default 2^31-1)
  int64_t span_cols;     // bound on the column span of any row of C: k, or a batch's widest product
  sg::HashCaps caps;     // hash-bin key caps (spgemm_tuning load factors)
  // long rows of B (spgemm_tuning::long_row_min; long_min 0: none)
  int64_t long_min;
  int64_t long_cap;      // room in lrow: nnz(B) / long_min + 1
  int64_t n_long, long_tot;
  int32_t *lmap;         // per row of B (fixed workspace)
  int32_t *lrow;         // per long row: its row of B (fixed workspace)
  void *long_ws;         // the long rows' bitmaps
  size_t long_ws_bytes;
  uint32_t *lbits;
  bool long_ready;       // built: the plan has bitmap rows and long rows
  const int32_t *col_base;  // Args::col_base of the numeric phase (a packed batch's), or null
  int32_t row_lo = 0, row_hi = INT32_MAX;  // Args::row_lo / row_hi of the numeric kernels (spgemm_numeric_rows)
  // compacted A (entries selecting a non-empty row of B), walked by the
  // phases instead of A when it holds fewer than half of A's entries
  int32_t *kept;         // flop pass: per row, its stored a_ik whose row of B is not empty (fixed
                         // workspace); the compaction's cursor afterwards
  long long *mstarts;    // merge-path tile starts (row, entry) over A (fixed workspace)
  int2 *klist;           // per merge-path tile: its kept entries (row, entry), kKeptListCap at most
  int32_t *klist_n;      // per tile: the number of them, or -1 when they did not fit
  int64_t nnz_a_used;
  bool a_compact;
  void *acmp_ws;
  size_t acmp_bytes;
  int32_t *karp, *kaci, *asrc;
  void *kav;
  // spgemm_numeric_graph: the captured numeric launches and the output buffers baked into them
  cudaGraphExec_t graph_exec;
  const void *graph_rp, *graph_ci, *graph_cv;
  bool bitmap_ok;
  int bm_words;

  // workspace (device)
  void *ws_fixed;  // counters + per-row arrays
  size_t ws_fixed_bytes;
  sg::DevCounters *dc;
  int64_t *flop;
  uint8_t *rbin;   // symbolic bin of each row (255 = none)
  int32_t *perm;   // rows grouped by symbolic bin
  int32_t *nnz_row;
  uint8_t *rbin2;  // numeric bin of each row
  int32_t *perm2;  // rows grouped by numeric bin
  long long *d_sym_off, *d_num_off;  // device bin offsets (16 each), as sym_off / num_off
  // graph mode (batched products replayed as one CUDA graph): no host read
  // of counts; bins are launched with persistent grids over device ranges,
  // and the workspace is sized from capacities instead of counts
  bool ddrive;
  // graph mode: the largest symbolic bound and row nnz the global tables
  // were planned for (-1: not graph mode, no check)
  int64_t gcap_bound = -1, gcap_nnz = -1;
  uint32_t *bitmaps;  // one bitmap per row of the symbolic bitmap bin
  size_t bitmaps_bytes;
  int4 *bm_items;     // numeric bitmap work items (bitmap index, window, part, parts)
  int4 *sym_items;    // split heavy symbolic rows: work items (index in the bin, part, parts)
  unsigned *sym_tickets;  // per heavy symbolic row: parts finished
  int64_t n_sym_items;
  size_t bm_items_bytes;
  void *gtab;         // global hash tables (heavy rows without bitmaps)
  size_t gtab_bytes;
  int64_t gtab_slots;  // table slots per block
  int64_t gtab_blocks;

  // host copies
  sg::DevCounters *hc;  // pinned
  int64_t sym_count[sg::kNumSymBins], sym_off[sg::kNumSymBins + 1];
  int64_t num_count[sg::kNumNumBins], num_off[sg::kNumNumBins + 1];
  int64_t sym_flop[sg::kNumSymBins], num_flop[sg::kNumNumBins];
  int64_t total_flop, max_flop, nnz_c;
  int64_t bm_cap[3];      // values per numeric bitmap window, per class
  int bm_threads[3];       // threads per block, per class
  int64_t bm_item_off[4];  // item offsets per class
  int64_t bm_bucket_off[3][sg::kBmBuckets];  // item offsets per class and weight bucket
  int32_t launches;
  const int32_t *c_rp;

  // side streams for bins that run concurrently (fork/join on `stream`)
  cudaStream_t side[4];
  cudaEvent_t fork_ev, join_ev[4];
  bool side_ready;

  // per-kernel CUDA events (SPGEMM_TIMING)
  struct Timed {
    std::string name;
    cudaEvent_t start, stop;
  };
  std::vector<Timed> timed;
};

namespace sg {
// Brackets one kernel launch with CUDA events when the plan records timings,
// and counts the launch.
struct KernelScope {
  spgemm_plan_s *p;
  cudaStream_t s;
  int idx = -1;
  KernelScope(spgemm_plan_s *plan, const std::string &name) : KernelScope(plan, name, plan->stream) {}
  KernelScope(spgemm_plan_s *plan, const std::string &name, cudaStream_t stream) : p(plan), s(stream) {
    p->launches++;
    if (!(p->flags & SPGEMM_TIMING)) return;
    spgemm_plan_s::Timed t{name, nullptr, nullptr};
    if (cudaEventCreate(&t.start) != cudaSuccess || cudaEventCreate(&t.stop) != cudaSuccess) return;
    cudaEventRecord(t.start, s);
    p->timed.push_back(t);
    idx = (int)p->timed.size() - 1;
  }
  ~KernelScope() {
    if (idx >= 0) cudaEventRecord(p->timed[idx].stop, s);
  }
};

// Concurrent bins: fork() makes the side streams wait for the plan's stream,
// bin_stream(i) picks the stream of the i-th launched bin, join() makes the
// plan's stream wait for every side stream.  Without side streams all bins
// run on the plan's stream.
cudaError_t fork(spgemm_plan_s *p);
// Bins run on side streams unless SPGEMM_SERIAL is set or the product is
// small (total flop below kSideStreamMinFlop), where the fork and join cost
// more than the overlap gains.
constexpr int64_t kSideStreamMinFlop = 1 << 20;
inline bool use_side_streams(const spgemm_plan_s *p) {
  return !(p->flags & SPGEMM_SERIAL) && p->total_flop >= kSideStreamMinFlop;
}
cudaStream_t bin_stream(spgemm_plan_s *p, int i);
cudaError_t join(spgemm_plan_s *p);

// Long rows: marked with the flop pass (k_merge_starts), then their bitmaps
// are built (when bitmap rows exist).
cudaError_t long_rows_build(spgemm_plan_s *p);
inline LongRows long_rows(const spgemm_plan_s *p) {
  if (!p->long_ready) return LongRows{nullptr, nullptr};
  return LongRows{p->lmap, p->lbits};
}
// Compacted A: keep flags of the entries (from the flop pass's prefix),
// then, from their exclusive scan pos, the copy's row pointers, columns and
// sources; its values before every numeric phase.
cudaError_t compact_a_gather(spgemm_plan_s *p);
cudaError_t compact_a_values(spgemm_plan_s *p);
// Arguments of the phase kernels: the compacted A when the plan has one.
inline Args phase_args(const spgemm_plan_s *p, uint32_t *err, int probe, unsigned long long *ctr) {
  const bool c = p->a_compact;
  Args a{p->m, p->n, p->k, c ? p->karp : p->arp, c ? p->kaci : p->aci, p->brp, p->bci,
         c ? (const void *)p->kav : p->av, p->bv, p->G, err, probe, ctr};
  a.col_base = p->col_base;
  a.row_lo = p->row_lo;
  a.row_hi = p->row_hi;
  return a;
}

// Blocks of a bin launch: one per row (or per 4 rows) of the count the host
// read, or, in graph mode, of the planning pass's count (at least one
// block: the kernels walk their actual rows grid-stride).
int64_t launch_blocks(const spgemm_plan_s *p, const void *kernel, int threads, size_t smem, int64_t exact);
// Graph mode: an upper bound on the rows of bin b (0: the bin never runs).
int64_t ddrive_bin_rows(const spgemm_plan_s *p, int b, bool symbolic);

// Graph mode (batched products replayed as one CUDA graph): what a plan is
// sized for, taken from a planning pass.  A replay whose product exceeds it
// reports SPGEMM_ERR_OUT_OF_MEMORY and writes nothing out of bounds.
struct GraphCaps {
  int64_t total_flop;  // sets the lanes per stored a_ik and the side streams
  int64_t max_flop;
  int64_t max_bound;   // largest symbolic bound of a row (global tables above 3/4 of 32768)
  int64_t max_nnz;     // largest nnz of a row (global tables above the largest shared table)
  int64_t nnz_cap;     // room for nnz(C)
  int64_t span_cols;   // bound on the column span of a row of C
  // rows per bin in the planning pass: the launch sizes of the bin kernels
  // (they walk their actual rows grid-stride, so any count stays correct)
  int64_t sym_rows[kNumSymBins];
  int64_t num_rows[kNumNumBins];
};
int plan_create_graph(spgemm_plan_s **out, const spgemm_csr *A, const spgemm_csr *B, int dtype, unsigned flags,
                      cudaStream_t stream, const spgemm_tuning *tuning, const GraphCaps &caps);
// Enqueues the whole product (flop pass, symbolic phase, row_ptr scan,
// numeric phase) on the plan's stream without any host synchronisation.
cudaError_t plan_enqueue_graph(spgemm_plan_s *p, int32_t *c_rp, int32_t *c_ci, void *c_v);
// Frees a plan (the public spgemm_plan_destroy).
void plan_free(spgemm_plan_s *p);

// Launchers (return a cudaError_t from the launch).
cudaError_t launch_symbolic(spgemm_plan_s *p);
cudaError_t launch_numeric(spgemm_plan_s *p, const int32_t *c_rp, int32_t *c_ci, void *c_v);
int64_t bitmap_capacity(int dtype, int bm_words, int64_t budget);
// Raises a kernel's dynamic shared memory limit to at least `bytes` (once per
// kernel, device and size; the static arrays count against the default 48 KB).
cudaError_t set_dynamic_smem(const void *kernel, size_t bytes);
// Text returned by spgemm_last_error() on this thread.
void set_last_error(const std::string &text);
int max_smem_per_block();
}  // namespace sg
