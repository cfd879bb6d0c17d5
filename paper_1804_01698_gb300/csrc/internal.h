// Plan object and kernel launchers of the GB300 hash SpGEMM (host side).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/spgemm.h"

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
constexpr int kSymBitmapBin = 10;    // bitmap rows with bound > kBitmapMidMax (1024 threads)
constexpr int kSymBitmapMidBin = 11; // bitmap rows with bound <= kBitmapMidMax (256 threads)
constexpr int kSymGlobalBin = 12;
constexpr int kNumSymBins = 13;
// numeric bins 0..8 are hash bins; bitmap rows become work items in three
// classes by row size: small (3 blocks per SM), medium (2), large (1, rank
// windows for rows longer than one block holds)
constexpr int kNumBitmapBin = 9;     // large class
constexpr int kNumGlobalBin = 10;
constexpr int kNumBitmapSBin = 11;   // small class
constexpr int kNumBitmapMBin = 12;   // medium class
constexpr int kNumNumBins = 13;
constexpr int kWarpsPerBlock = 4;  // warp bins: rows per block
// shared memory kept free beside a bitmap kernel's dynamic allocation for
// its static arrays (staging of 256 entries, reductions)
constexpr int kStaticSmemReserve = 256 * 20 + 2048;

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
// last part to finish counts it.
constexpr long long kSymSplitFlop = 131072;
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
  unsigned long long bm_cursor[3];
  unsigned long long bm_flop[3];        // flop of the rows of each class
  unsigned long long sym_split_extra;   // heavy symbolic bitmap rows: parts beyond one per row
  unsigned long long sym_item_cursor;
  // SPGEMM_COUNT_PROBES: rows 0/1 symbolic probes/inserts, 2/3 numeric,
  // each spread over kProbeSlots counters to limit atomic contention
  unsigned long long probe_stats[4][kProbeSlots];
  unsigned int err;
  unsigned int pad;
};

// Hash-table variants of a plan (Args::probe bits).
constexpr int kProbeChunk = 1;   // chunks of 4 slots per probe
constexpr int kProbeHashHi = 2;  // slot from the top bits of col * kHashScale (default)
inline int probe_mode(unsigned flags) {
  return ((flags & SPGEMM_PROBE_CHUNK4) ? kProbeChunk : 0) | ((flags & SPGEMM_HASH_LOW_BITS) ? 0 : kProbeHashHi);
}

// Kernel arguments common to all phases.
struct Args {
  int64_t m, n, k;
  const int32_t *arp, *aci, *brp, *bci;
  const void *av, *bv;
  int G;  // lanes per stored a_ik
  uint32_t *err;
  int probe = 0;  // hash tables: kProbeChunk (SPGEMM_PROBE_CHUNK4) | kProbeHashHi (unless SPGEMM_HASH_LOW_BITS)
  // SPGEMM_COUNT_PROBES: this phase's probe counters (inserts at +kProbeSlots), else null
  unsigned long long *probe_ctr = nullptr;
};

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
