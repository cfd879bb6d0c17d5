// Device helpers shared by the SpGEMM kernels: the hash function of the
// paper's Hash SpGEMM (Sec. 4.2.1), value-type accumulation, warp and block
// reductions and scans, and the device error word.
#pragma once

#include <climits>
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace sg {

// Sec. 4.2.1: the key (a column index) is multiplied by a constant and the
// remainder modulo the power-of-two table size picks the slot; collisions
// are resolved by linear probing.  The constant is Knuth's multiplicative
// hashing constant (TAOCP Vol. 3, Sec. 6.4), floor(2^32 / golden ratio).
constexpr uint32_t kHashScale = 2654435761u;
constexpr int32_t kEmpty = -1;  // Sec. 4.2.1: tables are initialised with -1

// The slot of a key in a table of mask+1 (a power of two) slots: with `hi`
// (the default) the top log2(size) bits of col * kHashScale (Fibonacci
// hashing), which depend on every bit of the column; otherwise its low bits,
// the remainder modulo the table size of Sec. 4.2.1 (SPGEMM_HASH_LOW_BITS).
__device__ __forceinline__ uint32_t hash_slot(int32_t col, uint32_t mask, int hi = 0) {
  const uint32_t x = (uint32_t)col * kHashScale;
  return hi ? x >> (32 - __popc(mask)) : x & mask;
}

// Bits of the device error word (DevCounters::err).
enum : uint32_t {
  kErrCsr = 1u,       // an index outside its matrix, or a malformed row_ptr
  kErrProbe = 2u,     // a probe sequence visited the whole table without a slot
  kErrOverflow = 4u,  // nnz(C) does not fit int32 indexing
  kErrRetry = 8u,     // an atomic update retried past its bound
  kErrCapacity = 16u, // graph mode: C or a heavy row exceeds what was planned
};

__device__ __forceinline__ void raise_err(uint32_t *err, uint32_t bit) { atomicOr(err, bit); }

// Bound on compare-and-swap retries of one accumulation; contention on a
// single slot is limited by the number of threads of a block, so this bound
// is never reached by a correct kernel.
constexpr int kMaxCasRetries = 1 << 20;

// ---------------------------------------------------------------------------
// Value types.  acc_shared/acc_global add a*b into *p with atomics; the f64
// form folds the multiply into the add with one fused multiply-add inside a
// compare-and-swap loop, because GB300's FP64 pipe is the scarce resource
// and a separate multiply plus the hardware's own CAS-loop add would cost
// two FP64 operations per product.
// Four consecutive keys of a table, slot h a multiple of 4 (16-byte
// aligned), read fresh: a volatile shared load, or an L2 load for tables in
// global memory (other lanes claim slots with atomics, which L1 does not see).
template <bool GLOBAL_MEM>
__device__ __forceinline__ int4 load_chunk(const int32_t *tab, uint32_t h) {
  if (GLOBAL_MEM) return __ldcg(reinterpret_cast<const int4 *>(tab + h));
  int4 k;
  const unsigned addr = (unsigned)__cvta_generic_to_shared(tab + h);
  asm volatile("ld.volatile.shared.v4.s32 {%0, %1, %2, %3}, [%4];"
               : "=r"(k.x), "=r"(k.y), "=r"(k.z), "=r"(k.w)
               : "r"(addr));
  return k;
}

// Chunked probing (the GPU form of HashVector, Sec. 4.2.2): the table is
// read 4 slots at a time from the chunk holding the key's hash slot, and a
// key is claimed in the first empty slot of its chunk, moving to the next
// chunk only when this one is full.  Slots are claimed in order within a
// chunk and never freed, so a key is absent from the table when its chunk
// has an empty slot and no match.  Returns the key's slot and sets *fresh
// when this call claimed it; -1 after a failed bound (err raised).
constexpr int kProbeSlots = 32;  // counters per phase for SPGEMM_COUNT_PROBES

// SPGEMM_COUNT_PROBES: adds one insertion of `probes` probes to the phase's
// counters (spread over kProbeSlots addresses).
__device__ __forceinline__ void count_probes(unsigned long long *ctr, unsigned probes) {
  if (!ctr) return;
  const unsigned slot = (blockIdx.x * 7u + threadIdx.x) % kProbeSlots;
  atomicAdd(ctr + slot, (unsigned long long)probes);
  atomicAdd(ctr + kProbeSlots + slot, 1ull);
}

template <bool GLOBAL_MEM>
__device__ __forceinline__ int chunk_find_or_claim(int32_t *tab, uint32_t mask, int32_t c, bool *fresh,
                                                   uint32_t *err, unsigned *probes, int hi) {
  uint32_t h = hash_slot(c, mask, hi) & ~3u;
  int retries = 0;
  for (uint32_t chunk = 0; chunk <= (mask >> 2);) {
    ++*probes;
    const int4 k4 = load_chunk<GLOBAL_MEM>(tab, h);
    const int32_t kk[4] = {k4.x, k4.y, k4.z, k4.w};
    int e = -1;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (e < 0 && kk[j] == c) {
        *fresh = false;
        return (int)(h + j);
      }
      if (e < 0 && kk[j] == kEmpty) e = j;
    }
    if (e < 0) {
      h = (h + 4) & mask;
      ++chunk;
      continue;
    }
    const int32_t old = atomicCAS(tab + h + e, kEmpty, c);
    if (old == kEmpty || old == c) {
      *fresh = old == kEmpty;
      return (int)(h + e);
    }
    if (++retries > kMaxCasRetries) {
      raise_err(err, kErrRetry);
      return -1;
    }
  }
  raise_err(err, kErrProbe);
  return -1;
}

template <typename T> struct Val;

template <> struct Val<double> {
  static __device__ __forceinline__ bool acc_shared(double *p, double a, double b) {
    unsigned long long *q = reinterpret_cast<unsigned long long *>(p);
    unsigned long long old = *reinterpret_cast<volatile unsigned long long *>(q);
    for (int it = 0; it < kMaxCasRetries; ++it) {
      unsigned long long assumed = old;
      double nv = fma(a, b, __longlong_as_double((long long)assumed));
      old = atomicCAS(q, assumed, (unsigned long long)__double_as_longlong(nv));
      if (old == assumed) return true;
    }
    return false;
  }
  static __device__ __forceinline__ void acc_global(double *p, double a, double b) { atomicAdd(p, a * b); }
  static __device__ __forceinline__ void add_global(double *p, double v) { atomicAdd(p, v); }
};

template <> struct Val<float> {
  static __device__ __forceinline__ bool acc_shared(float *p, float a, float b) {
    atomicAdd(p, a * b);
    return true;
  }
  static __device__ __forceinline__ void acc_global(float *p, float a, float b) { atomicAdd(p, a * b); }
  static __device__ __forceinline__ void add_global(float *p, float v) { atomicAdd(p, v); }
};

template <> struct Val<int64_t> {
  static __device__ __forceinline__ bool acc_shared(int64_t *p, int64_t a, int64_t b) {
    atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)a * (unsigned long long)b);
    return true;
  }
  static __device__ __forceinline__ void acc_global(int64_t *p, int64_t a, int64_t b) {
    atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)a * (unsigned long long)b);
  }
  static __device__ __forceinline__ void add_global(int64_t *p, int64_t v) {
    atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
  }
};

// After every block of a grid has added into count[0..nbins): the last block
// to finish writes off[b] = count[0] + ... + count[b-1] for b = 0..nbins
// (ticket: a counter zeroed before the launch).  Every thread of every block
// calls it, at the end of the kernel.
__device__ __forceinline__ void last_block_offsets(const unsigned long long *count, int nbins, long long *off,
                                                   unsigned int *ticket) {
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    long long run = 0;
    for (int b = 0; b < nbins; ++b) {
      off[b] = run;
      run += (long long)*reinterpret_cast<const volatile unsigned long long *>(count + b);
    }
    off[nbins] = run;
  }
}

// ---------------------------------------------------------------------------
// Reductions and scans.
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

template <typename T> __device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T w = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += w;
  }
  return v;
}

// Adds one row of flop v to bin b (b < nb; others add nothing) of a block's
// shared histogram: one shared atomic pair per distinct bin of the warp
// instead of one per lane, since most rows of a warp share a bin and
// atomics on one address serialise.  Every lane of the warp calls it.
__device__ __forceinline__ void warp_hist_add(int b, unsigned long long v, int nb, unsigned int *hist,
                                              unsigned long long *hflop) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  unsigned pending = __ballot_sync(full, b < nb);
  while (pending != 0u) {
    const int leader = __ffs(pending) - 1;
    const int lb = __shfl_sync(full, b, leader);
    const unsigned grp = __ballot_sync(full, b == lb);
    unsigned long long sum = b == lb ? v : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(full, sum, o);
    if (lane == leader) {
      atomicAdd(&hist[lb], (unsigned)__popc(grp));
      if (sum) atomicAdd(&hflop[lb], sum);
    }
    pending &= ~grp;
  }
}

// Block-wide sum; every thread of the block must call it.  `scratch` holds
// at least 32 elements and is reused, so callers separate two calls with a
// barrier (the function ends with one).
template <typename T> __device__ __forceinline__ T block_sum(T v, T *scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  T r = (threadIdx.x < nw) ? scratch[threadIdx.x] : T(0);
  if (wid == 0) r = warp_sum(r);
  if (threadIdx.x == 0) scratch[0] = r;
  __syncthreads();
  r = scratch[0];
  __syncthreads();
  return r;
}

// Block-wide minimum / maximum of an int; same calling rules as block_sum.
__device__ __forceinline__ int block_min(int v, int *scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  int r = threadIdx.x < nw ? scratch[threadIdx.x] : INT_MAX;
  if (wid == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = min(r, __shfl_xor_sync(0xffffffffu, r, o));
  }
  if (threadIdx.x == 0) scratch[0] = r;
  __syncthreads();
  r = scratch[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ int block_max(int v, int *scratch) { return -block_min(-v, scratch); }

// Block-wide exclusive scan; returns this thread's exclusive prefix and the
// block total through *total.  Same calling rules as block_sum.
template <typename T> __device__ __forceinline__ T block_excl_scan(T v, T *scratch, T *total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  T inc = warp_incl_scan(v);
  if (lane == 31) scratch[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T s = (lane < nw) ? scratch[lane] : T(0);
    T si = warp_incl_scan(s);
    if (lane < nw) scratch[lane] = si - s;
    if (lane == 31) scratch[32] = si;
  }
  __syncthreads();
  T r = scratch[wid] + inc - v;
  *total = scratch[32];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// The row loop shared by every phase (paper Fig. "RowWise_SpGEMM"): for
// each stored a_ik of row i and each stored b_kj, call f(j, a_ik, b_kj).
// A group of G lanes (a power of two dividing 32) takes one a_ik at a time
// and strides over row k of B, so consecutive lanes read consecutive
// entries of B (coalesced); groups take a_ik in turn.  U entries of B are
// loaded before any is processed, to keep several loads in flight.
// Columns of B outside [0, ncols) raise kErrCsr and are skipped.
template <int U, bool NEED_VAL, typename T, typename F>
__device__ __forceinline__ void for_row_products(int64_t a0, int64_t a1, int group, int ngroups, int lig, int G,
                                                 const int32_t *__restrict__ aci, const T *__restrict__ av,
                                                 const int32_t *__restrict__ brp, const int32_t *__restrict__ bci,
                                                 const T *__restrict__ bv, int32_t ncols, uint32_t *err, F &&f) {
  for (int64_t j = a0 + group; j < a1; j += ngroups) {
    const int32_t kk = __ldg(aci + j);
    T a = T(0);
    if (NEED_VAL) a = __ldg(av + j);
    const int32_t bs = __ldg(brp + kk), be = __ldg(brp + kk + 1);
    for (int32_t q = bs + lig; q < be; q += G * U) {
      int32_t c[U];
      T v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int32_t qq = q + u * G;
        c[u] = qq < be ? __ldg(bci + qq) : -1;
        if (NEED_VAL) v[u] = qq < be ? __ldg(bv + qq) : T(0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (q + u * G < be) {
          if ((uint32_t)c[u] < (uint32_t)ncols) f(c[u], a, NEED_VAL ? v[u] : T(0));
          else raise_err(err, kErrCsr);
        }
      }
    }
  }
}


// ---------------------------------------------------------------------------
// Staged, flattened row loop.  The stored a_ik of a row are processed in
// rounds of up to kStageN entries.  Per round, the start of row k of B and
// a_ik of each entry are staged in shared memory (the dependent loads
// col_idx(A) -> row_ptr(B) are issued in bulk), together with the exclusive
// prefix sum of the B row lengths.  The round's products then form one
// flat index range [0, total): product p belongs to the last entry e with
// pre[e] <= p and reads B entry bstart[e] + (p - pre[e]).  Groups of G lanes
// claim chunks of the range from a shared counter (dynamic balance); inside
// a chunk lane l takes products l, l+G, l+2G, ..., finds its first entry by
// binary search and then advances its entry cursor incrementally, so short
// rows of B keep every lane busy and consecutive lanes still read
// consecutive entries of B.  U products per lane are gathered before any is
// handed to f(col, a_ik, b_kj).
constexpr int kStageN = 256;  // entries staged per round (block form)

// One staged entry: products [start, end) of the round read B entries
// off + p, and carry a_ik.  16 bytes, read with one shared-memory load.
template <typename T> struct alignas(16) Entry {
  int end;
  int off;
  T a;
};

template <typename T> struct Stage {
  Entry<T> *ent;    // kStageN entries
  int *next;        // next unclaimed chunk
  long long *wsum;  // scratch for the scan (8 warp totals)
  int *lidx = nullptr;  // long-row loop: staged entries of long rows (kStageN)
  int *lcnt = nullptr;  // long-row loop: long entries per staging warp (8)
};

// Processes flat products [p0, p1) of a staged round of n entries, lane l
// of the group taking p0 + l, p0 + l + G, ...  All indices of a round fit in
// int32 (a round ends before its product count passes 2^31 - 1).
template <int U, bool NEED_VAL, typename T, typename F>
__device__ __forceinline__ void process_flat(const Entry<T> *ent, int n, int p0, int p1, int G, int lig,
                                             const int32_t *__restrict__ bci, const T *__restrict__ bv, int32_t ncols,
                                             uint32_t *err, F &&f) {
  int p = p0 + lig;
  if (p >= p1) return;
  int lo = 0, hi = n - 1;  // first entry e with end[e] > p
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (ent[mid].end > p) hi = mid;
    else lo = mid + 1;
  }
  int e = lo;
  Entry<T> cur = ent[e];
  while (p < p1) {
    int32_t q[U];
    T au[U];
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      ok[u] = p < p1;
      if (ok[u]) {
        while (p >= cur.end) cur = ent[++e];
        q[u] = cur.off + p;
        au[u] = cur.a;
      }
      p += G;
    }
    int32_t c[U];
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      c[u] = ok[u] ? __ldg(bci + q[u]) : -1;
      if (NEED_VAL) v[u] = ok[u] ? __ldg(bv + q[u]) : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (ok[u]) {
        if ((uint32_t)c[u] < (uint32_t)ncols) f(c[u], NEED_VAL ? au[u] : T(0), NEED_VAL ? v[u] : T(0));
        else raise_err(err, kErrCsr);
      }
    }
  }
}

// Block-wide form: every thread of the block calls it (blockDim.x >= kStageN).
template <int U, bool NEED_VAL, typename T, typename F>
__device__ __forceinline__ void block_row_products(int64_t a0, int64_t a1, int G, const int32_t *__restrict__ aci,
                                                   const T *__restrict__ av, const int32_t *__restrict__ brp,
                                                   const int32_t *__restrict__ bci, const T *__restrict__ bv,
                                                   int32_t ncols, uint32_t *err, Stage<T> st, F &&f) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, lig = tid & (G - 1);
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const int leader = lane & ~(G - 1);
  const int ngroups = blockDim.x / G;
  int64_t j0 = a0;
  while (j0 < a1) {
    const int n0 = (int)((a1 - j0) < kStageN ? (a1 - j0) : kStageN);
    long long len = 0;
    int32_t bs = 0;
    T av_t = T(0);
    if (tid < n0) {
      const int32_t kk = __ldg(aci + j0 + tid);
      bs = __ldg(brp + kk);
      len = __ldg(brp + kk + 1) - bs;
      if (NEED_VAL) av_t = __ldg(av + j0 + tid);
    }
    // inclusive scan of the lengths over the first kStageN threads (8 warps)
    long long inc = len;
    if (wid < kStageN / 32) {
      inc = warp_incl_scan(len);
      if (lane == 31) st.wsum[wid] = inc;
    }
    if (tid == 0) *st.next = 0;
    __syncthreads();
    if (wid < kStageN / 32) {
      long long base = 0;
      for (int w = 0; w < wid; ++w) base += st.wsum[w];
      inc += base;
    }
    // the round keeps the entries whose products end below 2^31 (at least one)
    const bool keep = tid < n0 && (tid == 0 || inc <= 2147483647LL);
    const int n = __syncthreads_count(keep);
    if (keep) st.ent[tid] = Entry<T>{(int)inc, (int)(bs - (inc - len)), av_t};
    __syncthreads();
    const int total = st.ent[n - 1].end;
    // chunk size: one chunk per group (every product costs about the same, so
    // equal shares balance; measured on R-MAT A*A, scale 16, four smaller
    // chunks per group ran the symbolic bitmap kernels 7-13% slower), at
    // least 4 products per lane
    long long chunk = ((long long)total + ngroups - 1) / ngroups;
    chunk = chunk < 4LL * G ? 4LL * G : chunk;
    chunk = (chunk + G - 1) / G * G;
    const int nchunks = (int)(((long long)total + chunk - 1) / chunk);
    for (;;) {
      int cidx = 0;
      if (lig == 0) cidx = atomicAdd(st.next, 1);
      cidx = __shfl_sync(gmask, cidx, leader);
      if (cidx >= nchunks) break;
      const long long p0 = (long long)cidx * chunk;
      const long long p1 = p0 + chunk < total ? p0 + chunk : total;
      process_flat<U, NEED_VAL>(st.ent, n, (int)p0, (int)p1, G, lig, bci, bv, ncols, err, f);
    }
    __syncthreads();
    j0 += n;
  }
}

// Processes flat products [p0, p1) like process_flat, but hands each lane's
// U gathered products to fb(c, a, b, ok) at once (ok[u]: product u exists
// and its column is inside B).  With PIPE, software-pipelined: the loads of
// the next U products are issued before fb works on the current ones, so
// their L2 latency overlaps fb's shared-memory updates (a second set of
// registers, which kernels at 32-40 registers a thread would spill).
template <int U, bool NEED_VAL, bool PIPE, typename T, typename FB>
__device__ __forceinline__ void process_flat_batch(const Entry<T> *ent, int n, int p0, int p1, int G, int lig,
                                                   const int32_t *__restrict__ bci, const T *__restrict__ bv,
                                                   int32_t ncols, uint32_t *err, FB &&fb) {
  if constexpr (!PIPE) {
    // the same without the second set of registers (kernels at 32-40
    // registers a thread would spill it): U products loaded, then handed over
    int p = p0 + lig;
    if (p >= p1) return;
    int lo = 0, hi = n - 1;  // first entry e with end[e] > p
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (ent[mid].end > p) hi = mid;
      else lo = mid + 1;
    }
    int e = lo;
    Entry<T> cur = ent[e];
    while (p < p1) {
      int32_t c[U];
      T au[U], v[U];
      bool ok[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        ok[u] = p < p1;
        c[u] = -1;
        au[u] = v[u] = T(0);
        if (ok[u]) {
          while (p >= cur.end) cur = ent[++e];
          const int32_t q = cur.off + p;
          c[u] = __ldg(bci + q);
          if (NEED_VAL) {
            au[u] = cur.a;
            v[u] = __ldg(bv + q);
          }
        }
        p += G;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (ok[u] && (uint32_t)c[u] >= (uint32_t)ncols) {
          raise_err(err, kErrCsr);
          ok[u] = false;
        }
      }
      fb(c, au, v, ok);
    }
    return;
  }
  int p = p0 + lig;
  if (p >= p1) return;
  int lo = 0, hi = n - 1;  // first entry e with end[e] > p
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (ent[mid].end > p) hi = mid;
    else lo = mid + 1;
  }
  int e = lo;
  Entry<T> cur = ent[e];
  // the next U products of this lane: columns, values, a_ik, presence
  auto gather = [&](int32_t(&c)[U], T(&v)[U], T(&au)[U], bool(&ok)[U]) {
    int32_t q[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      ok[u] = p < p1;
      q[u] = 0;
      au[u] = T(0);
      if (ok[u]) {
        while (p >= cur.end) cur = ent[++e];
        q[u] = cur.off + p;
        au[u] = cur.a;
      }
      p += G;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      c[u] = ok[u] ? __ldg(bci + q[u]) : -1;
      v[u] = (NEED_VAL && ok[u]) ? __ldg(bv + q[u]) : T(0);
    }
  };
  int32_t c0[U], c1[U];
  T v0[U], v1[U], a0[U], a1[U];
  bool k0[U], k1[U];
  gather(c0, v0, a0, k0);
  while (k0[0]) {
    gather(c1, v1, a1, k1);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k0[u] && !((uint32_t)c0[u] < (uint32_t)ncols)) {
        raise_err(err, kErrCsr);
        k0[u] = false;
      }
    }
    fb(c0, a0, v0, k0);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      c0[u] = c1[u];
      v0[u] = v1[u];
      a0[u] = a1[u];
      k0[u] = k1[u];
    }
  }
}

// Passed as `flong` below: the caller takes the long entries elsewhere and
// the loop only leaves them out.
struct SkipLong {
  __device__ void operator()(int, const int *) const {}
};

// Block-wide row loop of the bitmap rows, with long rows of B (lmap[k] >= 0,
// lmap null: none).  Like block_row_products, except that a staged entry
// whose row of B is long adds no flat products: its staged record keeps the
// long-row index in `off` (and a_ik), and after the round's flat products
// and a barrier every thread calls flong(nlong, lidx), lidx[0..nlong) being
// the round's long entries in stored order; a barrier follows (neither with
// flong = SkipLong).  Flat products go to fb (process_flat_batch).  Every
// thread of the block calls it (blockDim.x >= kStageN).
template <int U, bool NEED_VAL, bool PIPE, typename T, typename FB, typename FL>
__device__ __forceinline__ void block_row_products_long(int64_t a0, int64_t a1, int G,
                                                        const int32_t *__restrict__ aci, const T *__restrict__ av,
                                                        const int32_t *__restrict__ brp,
                                                        const int32_t *__restrict__ bci, const T *__restrict__ bv,
                                                        int32_t ncols, uint32_t *err, const int32_t *__restrict__ lmap,
                                                        Stage<T> st, FB &&fb, FL &&flong) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, lig = tid & (G - 1);
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const int leader = lane & ~(G - 1);
  const int ngroups = blockDim.x / G;
  int64_t j0 = a0;
  while (j0 < a1) {
    const int n0 = (int)((a1 - j0) < kStageN ? (a1 - j0) : kStageN);
    long long len = 0;
    int32_t bs = 0, d = -1;
    T av_t = T(0);
    if (tid < n0) {
      const int32_t kk = __ldg(aci + j0 + tid);
      if (lmap) d = __ldg(lmap + kk);
      if (d < 0) {
        bs = __ldg(brp + kk);
        len = __ldg(brp + kk + 1) - bs;
      }
      if (NEED_VAL) av_t = __ldg(av + j0 + tid);
    }
    long long inc = len;
    if (wid < kStageN / 32) {
      inc = warp_incl_scan(len);
      if (lane == 31) st.wsum[wid] = inc;
    }
    if (tid == 0) *st.next = 0;
    __syncthreads();
    if (wid < kStageN / 32) {
      long long base = 0;
      for (int w = 0; w < wid; ++w) base += st.wsum[w];
      inc += base;
    }
    const bool keep = tid < n0 && (tid == 0 || inc <= 2147483647LL);
    const int n = __syncthreads_count(keep);
    unsigned lm = 0;
    if (keep) st.ent[tid] = Entry<T>{(int)inc, d < 0 ? (int)(bs - (inc - len)) : d, av_t};
    if (!std::is_same<typename std::decay<FL>::type, SkipLong>::value && wid < kStageN / 32) {
      lm = __ballot_sync(0xffffffffu, keep && d >= 0);
      if (lane == 0) st.lcnt[wid] = __popc(lm);
    }
    __syncthreads();
    constexpr bool kList = !std::is_same<typename std::decay<FL>::type, SkipLong>::value;
    int nlong = 0;
    if (kList && lmap) {
#pragma unroll
      for (int w = 0; w < kStageN / 32; ++w) {
        if (w == wid && keep && d >= 0) st.lidx[nlong + __popc(lm & ((1u << lane) - 1u))] = tid;
        nlong += st.lcnt[w];
      }
    }
    const int total = st.ent[n - 1].end;
    if (total > 0) {
      long long chunk = ((long long)total + ngroups - 1) / ngroups;  // as in block_row_products
      chunk = chunk < 4LL * G ? 4LL * G : chunk;
      chunk = (chunk + G - 1) / G * G;
      const int nchunks = (int)(((long long)total + chunk - 1) / chunk);
      for (;;) {
        int cidx = 0;
        if (lig == 0) cidx = atomicAdd(st.next, 1);
        cidx = __shfl_sync(gmask, cidx, leader);
        if (cidx >= nchunks) break;
        const long long p0 = (long long)cidx * chunk;
        const long long p1 = p0 + chunk < total ? p0 + chunk : total;
        process_flat_batch<U, NEED_VAL, PIPE>(st.ent, n, (int)p0, (int)p1, G, lig, bci, bv, ncols, err, fb);
      }
    }
    __syncthreads();
    if (nlong > 0) {
      flong(nlong, (const int *)st.lidx);
      __syncthreads();
    }
    j0 += n;
  }
}

// Warp form: the 32 lanes of one warp work on one row as one group;
// `st` points to this warp's own staging area (32 entries).
template <int U, bool NEED_VAL, typename T, typename F>
__device__ __forceinline__ void warp_row_products(int64_t a0, int64_t a1, int /*G*/, const int32_t *__restrict__ aci,
                                                  const T *__restrict__ av, const int32_t *__restrict__ brp,
                                                  const int32_t *__restrict__ bci, const T *__restrict__ bv,
                                                  int32_t ncols, uint32_t *err, Stage<T> st, F &&f) {
  const int lane = threadIdx.x & 31;
  int64_t j0 = a0;
  while (j0 < a1) {
    const int n0 = (int)((a1 - j0) < 32 ? (a1 - j0) : 32);
    long long len = 0;
    int32_t bs = 0;
    T av_t = T(0);
    if (lane < n0) {
      const int32_t kk = __ldg(aci + j0 + lane);
      bs = __ldg(brp + kk);
      len = __ldg(brp + kk + 1) - bs;
      if (NEED_VAL) av_t = __ldg(av + j0 + lane);
    }
    const long long inc = warp_incl_scan(len);
    const bool keep = lane < n0 && (lane == 0 || inc <= 2147483647LL);
    const int n = __popc(__ballot_sync(0xffffffffu, keep));
    if (keep) st.ent[lane] = Entry<T>{(int)inc, (int)(bs - (inc - len)), av_t};
    __syncwarp();
    const int total = st.ent[n - 1].end;
    process_flat<U, NEED_VAL>(st.ent, n, 0, total, 32, lane, bci, bv, ncols, err, f);
    __syncwarp();
    j0 += n;
  }
}

}  // namespace sg
