// Numeric phase (paper Sec. 4.2.1; Fig. "Hash_SpGEMM", step Numeric): the
// keys are inserted again and a_ik*b_kj is added to the value of the key's
// slot; the finished row is then stored, sorted by column when requested.
//
//   k_num_warp<T,S>   one warp per row, S-slot table (keys + values) in smem
//   k_num_block<T,S>  one block per row, S-slot table in smem
//   k_num_bitmap<T,NT,MINB>  heavy rows with a column bitmap saved by the
//                     symbolic phase: the rank of column j among the row's
//                     columns is its output position, so values accumulate in
//                     a dense array indexed by rank and come out sorted.  A
//                     row with more entries than fit in shared memory keeps
//                     its first ranks there and adds the others straight into
//                     C, and a row with much more flop than output is split
//                     into parts of its stored a_ik (one block per part);
//                     three size classes, each with its own launch shape,
//                     their work items heaviest first.
//   k_num_global<T>   heavy rows without bitmaps: hash table in global memory.
//
// Tables are sized from the exact row count found by the symbolic phase,
// so they are smaller than the symbolic tables.
#pragma once

#include <algorithm>
#include <string>

#include "common.cuh"
#include "internal.h"
#include "rowsplit.cuh"

namespace sg {

constexpr int kUN = 4;  // B entries (column + value) loaded ahead per lane

// Every variant of the insert (see insert_key_any).
template <typename T, bool GLOBAL_MEM>
__device__ __forceinline__ void insert_acc_any(int32_t *keys, T *vals, uint32_t mask, int32_t c, T a, T b,
                                            uint32_t *err, int probe, unsigned long long *ctr) {
  if (probe & kProbeChunk) {
    bool fresh = false;
    unsigned probes = 0;
    const int h = chunk_find_or_claim<GLOBAL_MEM>(keys, mask, c, &fresh, err, &probes, probe & kProbeHashHi);
    count_probes(ctr, probes);
    if (h < 0) return;
    if (GLOBAL_MEM) {
      Val<T>::acc_global(vals + h, a, b);
    } else if (!Val<T>::acc_shared(vals + h, a, b)) {
      raise_err(err, kErrRetry);
    }
    return;
  }
  uint32_t h = hash_slot(c, mask, probe & kProbeHashHi);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const int32_t old = atomicCAS(keys + h, kEmpty, c);
    if (old == kEmpty || old == c) {
      count_probes(ctr, probe + 1);
      if (GLOBAL_MEM) {
        Val<T>::acc_global(vals + h, a, b);
      } else if (!Val<T>::acc_shared(vals + h, a, b)) {
        raise_err(err, kErrRetry);
      }
      return;
    }
    h = (h + 1) & mask;
  }
  raise_err(err, kErrProbe);
}

// Finds or claims the slot of key c and accumulates a*b there.  The default
// plan (linear probing, top-bits hash, no counting) runs the loop inline.
template <typename T, bool GLOBAL_MEM>
__device__ __forceinline__ void insert_acc(int32_t *keys, T *vals, uint32_t mask, int32_t c, T a, T b,
                                           uint32_t *err, int probe, unsigned long long *ctr) {
  if (probe != kProbeHashHi || ctr) {
    insert_acc_any<T, GLOBAL_MEM>(keys, vals, mask, c, a, b, err, probe, ctr);
    return;
  }
  uint32_t h = hash_slot(c, mask, 1);
  for (uint32_t q = 0; q <= mask; ++q) {
    const int32_t old = atomicCAS(keys + h, kEmpty, c);
    if (old == kEmpty || old == c) {
      if (GLOBAL_MEM) {
        Val<T>::acc_global(vals + h, a, b);
      } else if (!Val<T>::acc_shared(vals + h, a, b)) {
        raise_err(err, kErrRetry);
      }
      return;
    }
    h = (h + 1) & mask;
  }
  raise_err(err, kErrProbe);
}

template <typename T>
__device__ __forceinline__ void swap_entry(uint32_t *keys, T *vals, int i, int l) {
  const uint32_t ki = keys[i];
  keys[i] = keys[l];
  keys[l] = ki;
  const T vi = vals[i];
  vals[i] = vals[l];
  vals[l] = vi;
}

// Bitonic sort of n (power of two) entries by unsigned key; empty slots
// (-1 = 0xffffffff) sort last.  Threads t0, t0+tstride, ... take the n/2
// compare-exchange pairs of each stage; `sync` separates the stages.
template <typename T, typename Sync>
__device__ __forceinline__ void bitonic_sort(uint32_t *keys, T *vals, int n, int t0, int tstride, Sync &&sync) {
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = t0; t < (n >> 1); t += tstride) {
        const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
        const int l = i + j;
        const bool asc = (i & k) == 0;
        const uint32_t ki = keys[i], kl = keys[l];
        if ((ki > kl) == asc) swap_entry(keys, vals, i, l);
      }
      sync();
    }
  }
}

// Compare-exchange of registers r and r | JR of every lane (strides of 32 or
// more of the bitonic network below), ascending where bit kk of the element
// index is clear.
template <typename T, int R, int JR>
__device__ __forceinline__ void reg_stage(uint32_t (&k)[R], T (&v)[R], int kk) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if ((r & JR) == 0) {
      const bool asc = ((r * 32) & kk) == 0;
      const int q = r | JR;
      if ((k[r] > k[q]) == asc) {
        const uint32_t tk = k[r];
        k[r] = k[q];
        k[q] = tk;
        const T tv = v[r];
        v[r] = v[q];
        v[q] = tv;
      }
    }
  }
}

// Sorted store of a warp's row: the nnz compacted (key, value) pairs are
// sorted by a bitonic network held in registers, element e = r * 32 + lane
// in register r of lane `lane`; strides of 32 or more swap registers of one
// lane, shorter strides exchange with lane ^ stride by shuffles.  The stage
// loops stay loops (only the register index is unrolled) to keep the code
// small.  Padding keys (-1, the largest as unsigned) sort last and are not
// stored.
template <typename T, int R>
__device__ __forceinline__ void warp_sort_store(const int32_t *keys, const T *vals, int nnz, int lane,
                                                int32_t *__restrict__ out_ci, T *__restrict__ out_v, int32_t cb) {
  uint32_t k[R];
  T v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int e = r * 32 + lane;
    k[r] = e < nnz ? (uint32_t)keys[e] : 0xffffffffu;
    v[r] = e < nnz ? vals[e] : T(0);
  }
#pragma unroll 1
  for (int kk = 2; kk <= 32 * R; kk <<= 1) {
#pragma unroll 1
    for (int j = kk >> 1; j > 0; j >>= 1) {
      if (j >= 32) {
        switch (j >> 5) {
          case 1: reg_stage<T, R, 1>(k, v, kk); break;
          case 2: if (R > 2) reg_stage<T, R, (R > 2 ? 2 : 1)>(k, v, kk); break;
          case 4: if (R > 4) reg_stage<T, R, (R > 4 ? 4 : 1)>(k, v, kk); break;
          default: if (R > 8) reg_stage<T, R, (R > 8 ? 8 : 1)>(k, v, kk); break;
        }
      } else {
        const bool lower = (lane & j) == 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int e = r * 32 + lane;
          const uint32_t pk = __shfl_xor_sync(0xffffffffu, k[r], j);
          const T pv = __shfl_xor_sync(0xffffffffu, v[r], j);
          const bool asc = (e & kk) == 0;
          if ((lower == asc) ? (pk < k[r]) : (pk > k[r])) {
            k[r] = pk;
            v[r] = pv;
          }
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int e = r * 32 + lane;
    if (e < nnz) {
      out_ci[e] = (int32_t)k[r] - cb;
      out_v[e] = v[r];
    }
  }
}

// ---------------------------------------------------------------------------
// Sorted store of a warp's compacted row by bucket ranks: a counting sort on
// a monotone bucket of the column, (col - cmin) >> shift with at most nb
// buckets (nb = the power of two >= cnt), then each entry's rank inside its
// bucket by comparison with the bucket's other entries.  The rank is the
// entry's position in the sorted row, so it is stored there directly.
// Space: the warp tables hold cnt <= S/2 entries, so after compaction the
// upper halves of keys (bucket counters) and of vals (entry indices grouped
// by bucket) are free.  Returns false, having stored nothing and left the
// compacted entries in place, when a bucket holds more than kMaxBucket
// entries (columns clustered within the range): the caller then sorts by
// the bitonic network.
constexpr int kMaxBucket = 32;

template <typename T, int S>
__device__ __forceinline__ bool bucket_sort_store(int32_t *keys, T *vals, int cnt, int lane,
                                                  int32_t *__restrict__ out_ci, T *__restrict__ out_v, int32_t cb) {
  static_assert(S >= 64, "warp tables hold at least 64 slots");
  int32_t *bcnt = keys + S / 2;
  int32_t *grp = reinterpret_cast<int32_t *>(vals + S / 2);
  int32_t lo = 0x7fffffff, hi = 0;
  for (int e = lane; e < cnt; e += 32) {
    const int32_t c = keys[e];
    lo = min(lo, c);
    hi = max(hi, c);
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  int nb = 32;
  while (nb < cnt) nb <<= 1;  // nb <= S/2
  const uint32_t span = (uint32_t)(hi - lo);
  int shift = 0;
  while ((span >> shift) >= (uint32_t)nb) ++shift;  // buckets 0 .. nb-1
  for (int b = lane; b < nb; b += 32) bcnt[b] = 0;
  __syncwarp();
  for (int e = lane; e < cnt; e += 32) atomicAdd(&bcnt[(uint32_t)(keys[e] - lo) >> shift], 1);
  __syncwarp();
  // exclusive scan of the counters; lane l owns counters l*per .. l*per+per-1
  const int per = nb >> 5;
  int sum = 0, mx = 0;
  for (int j = 0; j < per; ++j) {
    const int v = bcnt[lane * per + j];
    sum += v;
    mx = max(mx, v);
  }
  if (__reduce_max_sync(0xffffffffu, mx) > kMaxBucket) return false;
  int incl = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += t;
  }
  int run = incl - sum;
  for (int j = 0; j < per; ++j) {
    const int v = bcnt[lane * per + j];
    bcnt[lane * per + j] = run;
    run += v;
  }
  __syncwarp();
  // group entry indices by bucket; afterwards bcnt[b] is the end of bucket b
  for (int e = lane; e < cnt; e += 32) grp[atomicAdd(&bcnt[(uint32_t)(keys[e] - lo) >> shift], 1)] = e;
  __syncwarp();
  for (int q = lane; q < cnt; q += 32) {
    const int e = grp[q];
    const int32_t c = keys[e];
    const int b = (int)((uint32_t)(c - lo) >> shift);
    const int b1 = bcnt[b];
    int r = b > 0 ? bcnt[b - 1] : 0;
    for (int t = r; t < b1; ++t) r += keys[grp[t]] < c;
    out_ci[r] = c - cb;
    out_v[r] = vals[e];
  }
  return true;
}

// One row of a warp bin: accumulate into the warp's table, then store the
// row (sorted when requested).
template <typename T, int S>
__device__ __forceinline__ void num_warp_row(const Args &a, int32_t i, int32_t *keys, T *vals, Entry<T> *ent,
                                             int *next, const int32_t *__restrict__ c_rp, int32_t *__restrict__ c_ci,
                                             T *__restrict__ c_v, int sorted, int lane) {
  for (int s = lane; s < S; s += 32) {
    keys[s] = kEmpty;
    vals[s] = T(0);
  }
  __syncwarp();
  const int G = a.G;
  warp_row_products<kUN, true, T>(a.arp[i], a.arp[i + 1], G, a.aci, (const T *)a.av, a.brp, a.bci, (const T *)a.bv,
                                  (int32_t)a.k, a.err, Stage<T>{ent, next, nullptr},
                                 [&](int32_t c, T av, T bv) { insert_acc<T, false>(keys, vals, S - 1, c, av, bv, a.err, a.probe, a.probe_ctr); });
  __syncwarp();
  const int32_t rp = c_rp[i];
  const int32_t nnz = c_rp[i + 1] - rp;
  const int32_t cb = a.col_base ? a.col_base[i] : 0;
  if (sorted) {
    // Compact the occupied slots to the front (in place: chunk by chunk, every
    // lane reads its slot before any lane writes, and a chunk only writes
    // positions at or below its own), pad to the next power of two with the
    // empty key (-1, largest as unsigned) and sort only that prefix.
    int base = 0;
    for (int s0 = 0; s0 < S; s0 += 32) {
      const int32_t kk = keys[s0 + lane];
      const T vv = vals[s0 + lane];
      const bool occ = kk != kEmpty;
      const unsigned m = __ballot_sync(0xffffffffu, occ);
      __syncwarp();
      if (occ) {
        const int pos = base + __popc(m & ((1u << lane) - 1u));
        keys[pos] = kk;
        vals[pos] = vv;
      }
      base += __popc(m);
      __syncwarp();
    }
    const int cnt = min(base, nnz);
    if (cnt <= 32) warp_sort_store<T, 1>(keys, vals, cnt, lane, c_ci + rp, c_v + rp, cb);
    else if (cnt <= S / 2 && bucket_sort_store<T, S>(keys, vals, cnt, lane, c_ci + rp, c_v + rp, cb)) {
    } else if (cnt <= 64) warp_sort_store<T, 2>(keys, vals, cnt, lane, c_ci + rp, c_v + rp, cb);
    else if (cnt <= 128) warp_sort_store<T, 4>(keys, vals, cnt, lane, c_ci + rp, c_v + rp, cb);
    else if (cnt <= 256) warp_sort_store<T, 8>(keys, vals, cnt, lane, c_ci + rp, c_v + rp, cb);
    else {
      // longer rows: the same network in shared memory (measured faster here)
      int P = 512;
      while (P < cnt) P <<= 1;
      for (int r = cnt + lane; r < P; r += 32) keys[r] = kEmpty;
      __syncwarp();
      bitonic_sort(reinterpret_cast<uint32_t *>(keys), vals, P, lane, 32, [] { __syncwarp(); });
      for (int r = lane; r < cnt; r += 32) {
        c_ci[rp + r] = keys[r] - cb;
        c_v[rp + r] = vals[r];
      }
    }
    if (lane == 0 && base != nnz) raise_err(a.err, kErrProbe);
  } else {
    int base = 0;
    for (int s0 = 0; s0 < S; s0 += 32) {
      const int s = s0 + lane;
      const int32_t kk = keys[s];
      const bool occ = kk != kEmpty;
      const unsigned m = __ballot_sync(0xffffffffu, occ);
      const int pos = base + __popc(m & ((1u << lane) - 1u));
      if (occ && pos < nnz) {
        c_ci[rp + pos] = kk - cb;
        c_v[rp + pos] = vals[s];
      }
      base += __popc(m);
    }
    if (lane == 0 && base != nnz) raise_err(a.err, kErrProbe);
  }
}

template <typename T, int S>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 8)
    k_num_warp(Args a, BinRows br, const int32_t *__restrict__ c_rp, int32_t *__restrict__ c_ci,
               T *__restrict__ c_v, int sorted) {
  extern __shared__ __align__(16) unsigned char sm_num_warp[];
  __shared__ Entry<T> s_ent[kWarpsPerBlock][32];
  __shared__ int s_next[kWarpsPerBlock];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (aborted(a)) return;
  const long long o0 = br.off[br.bin], nrows = br.off[br.bin + 1] - o0;
  int32_t *keys = reinterpret_cast<int32_t *>(sm_num_warp) + warp * S;
  T *vals = reinterpret_cast<T *>(sm_num_warp + (size_t)kWarpsPerBlock * S * sizeof(int32_t)) + warp * S;
  // one warp per row (no block barrier below)
  for (int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + warp; w < nrows; w += (int64_t)gridDim.x * kWarpsPerBlock) {
    const int32_t i = br.perm[o0 + w];
    if (!in_rows(a, i)) continue;
    num_warp_row<T, S>(a, i, keys, vals, s_ent[warp], &s_next[warp], c_rp, c_ci, c_v, sorted, lane);
    __syncwarp();
  }
}

// sort_mode: 0 unsorted, 1 bitonic sort of the table, 2 rank by column
// bitmap (needs 2 * words * 4 bytes more shared memory).
// Threads of the block bins (as kNumBins) and the blocks per SM their shared
// memory allows (table, sort window and staging): the register budget is
// set so that the registers do not cap the blocks per SM below that.
template <int S> constexpr int num_block_threads() { return S <= 2048 ? 256 : S <= 4096 ? 512 : 1024; }
template <int S> constexpr int num_block_min_blocks() { return S <= 2048 ? 5 : S <= 4096 ? 3 : 1; }

// One row of a block bin (whole block).
template <typename T, int S>
__device__ __forceinline__ void num_block_row(const Args &a, int32_t i, const int32_t *__restrict__ c_rp,
                                              int32_t *__restrict__ c_ci, T *__restrict__ c_v, int sort_mode,
                                              int words) {
  extern __shared__ __align__(16) unsigned char sm_num_block[];
  __shared__ int red[33];
  __shared__ Entry<T> s_ent[kStageN];
  __shared__ long long s_wsum[8];
  __shared__ int s_next;
  __shared__ int cursor;
  int32_t *keys = reinterpret_cast<int32_t *>(sm_num_block);
  T *vals = reinterpret_cast<T *>(sm_num_block + (size_t)S * sizeof(int32_t));
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    keys[s] = kEmpty;
    vals[s] = T(0);
  }
  if (threadIdx.x == 0) cursor = 0;
  __syncthreads();
  const int G = a.G;
  block_row_products<kUN, true, T>(a.arp[i], a.arp[i + 1], G, a.aci, (const T *)a.av, a.brp, a.bci,
                                   (const T *)a.bv, (int32_t)a.k, a.err, Stage<T>{s_ent, &s_next, s_wsum},
                                 [&](int32_t c, T av, T bv) { insert_acc<T, false>(keys, vals, S - 1, c, av, bv, a.err, a.probe, a.probe_ctr); });
  __syncthreads();
  const int32_t rp = c_rp[i];
  const int32_t nnz = c_rp[i + 1] - rp;
  const int32_t cb = a.col_base ? a.col_base[i] : 0;
  if (sort_mode == 1) {
    bitonic_sort(reinterpret_cast<uint32_t *>(keys), vals, S, (int)threadIdx.x, (int)blockDim.x, [] { __syncthreads(); });
    for (int r = threadIdx.x; r < nnz; r += blockDim.x) {
      c_ci[rp + r] = keys[r] - cb;
      c_v[rp + r] = vals[r];
    }
  } else if (sort_mode == 2) {
    // Rank by a bitmap over the row's own column window [cmin, cmax] (the
    // words of shared memory reserved for it hold `words` x 32 columns); a row
    // whose columns spread wider is sorted with the bitonic network instead.
    int cmin = INT_MAX, cmax = -1;
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
      const int32_t kk = keys[s];
      if (kk != kEmpty) {
        cmin = min(cmin, (int)kk);
        cmax = max(cmax, (int)kk);
      }
    }
    cmin = block_min(cmin, red);
    cmax = block_max(cmax, red);
    const int base = cmin & ~31;
    const int used = nnz > 0 ? ((cmax - base) >> 5) + 1 : 0;
    if (used <= words) {
      uint32_t *bm = reinterpret_cast<uint32_t *>(sm_num_block + (size_t)S * (sizeof(int32_t) + sizeof(T)));
      int32_t *pre = reinterpret_cast<int32_t *>(bm + words);
      for (int w = threadIdx.x; w < used; w += blockDim.x) bm[w] = 0u;
      __syncthreads();
      for (int s = threadIdx.x; s < S; s += blockDim.x) {
        const int32_t kk = keys[s];
        if (kk != kEmpty) atomicOr(bm + ((kk - base) >> 5), 1u << ((kk - base) & 31));
      }
      __syncthreads();
      // exclusive prefix of popcounts: each thread owns a contiguous run of words
      const int per = (used + blockDim.x - 1) / blockDim.x;
      const int w0 = threadIdx.x * per, w1 = min(used, w0 + per);
      int local = 0;
      for (int w = w0; w < w1; ++w) local += __popc(bm[w]);
      int tot;
      int run = block_excl_scan(local, red, &tot);
      for (int w = w0; w < w1; ++w) {
        pre[w] = run;
        run += __popc(bm[w]);
      }
      __syncthreads();
      for (int s = threadIdx.x; s < S; s += blockDim.x) {
        const int32_t kk = keys[s];
        if (kk != kEmpty) {
          const int o = kk - base;
          const int r = pre[o >> 5] + __popc(bm[o >> 5] & ((1u << (o & 31)) - 1u));
          if (r < nnz) {
            c_ci[rp + r] = kk - cb;
            c_v[rp + r] = vals[s];
          }
        }
      }
      if (threadIdx.x == 0 && tot != nnz) raise_err(a.err, kErrProbe);
    } else {
      bitonic_sort(reinterpret_cast<uint32_t *>(keys), vals, S, (int)threadIdx.x, (int)blockDim.x,
                   [] { __syncthreads(); });
      for (int r = threadIdx.x; r < nnz; r += blockDim.x) {
        c_ci[rp + r] = keys[r] - cb;
        c_v[rp + r] = vals[r];
      }
    }
  } else {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int s0 = warp * 32; s0 < S; s0 += nw * 32) {
      const int s = s0 + lane;
      const int32_t kk = keys[s];
      const bool occ = kk != kEmpty;
      const unsigned m = __ballot_sync(0xffffffffu, occ);
      int base = 0;
      if (lane == 0 && m) base = atomicAdd(&cursor, __popc(m));
      base = __shfl_sync(0xffffffffu, base, 0);
      const int pos = base + __popc(m & ((1u << lane) - 1u));
      if (occ && pos < nnz) {
        c_ci[rp + pos] = kk - cb;
        c_v[rp + pos] = vals[s];
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && cursor != nnz) raise_err(a.err, kErrProbe);
  }
}

template <typename T, int S>
__global__ void __launch_bounds__(num_block_threads<S>(), num_block_min_blocks<S>())
    k_num_block(Args a, BinRows br, const int32_t *__restrict__ c_rp, int32_t *__restrict__ c_ci,
                T *__restrict__ c_v, int sort_mode, int words) {
  if (aborted(a)) return;
  const long long o0 = br.off[br.bin], nrows = br.off[br.bin + 1] - o0;
  for (int64_t b = blockIdx.x; b < nrows; b += gridDim.x) {  // one block per row
    const int32_t i = br.perm[o0 + b];
    if (!in_rows(a, i)) continue;
    num_block_row<T, S>(a, i, c_rp, c_ci, c_v, sort_mode, words);
    __syncthreads();  // the shared table is cleared for the next row
  }
}

// Values that the bitmap kernels add into C start at zero: every value of a
// split row (its parts add theirs), and the ranks from cap_l on of a row
// with more entries than the large class's shared array holds (their
// products are added straight into C).  One warp per bitmap row.
template <typename T>
__global__ void __launch_bounds__(256)
    k_bm_zero_split(const int32_t *__restrict__ bm_rows, int64_t nbm, const int64_t *__restrict__ flop,
                    const int32_t *__restrict__ c_rp, T *__restrict__ c_v, int32_t row_lo, int32_t row_hi,
                    int64_t cap_l) {
  const int64_t t = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (t >= nbm) return;
  const int32_t i = bm_rows[t];
  if (i < row_lo || i >= row_hi) return;
  const int32_t rp = c_rp[i], nnz = c_rp[i + 1] - rp;
  const int32_t z0 = bm_split_parts(flop[i], nnz) >= 2 ? 0 : nnz > cap_l ? (int32_t)cap_l : nnz;
  for (int32_t r = z0 + (threadIdx.x & 31); r < nnz; r += 32) c_v[rp + r] = T(0);
}

// Rows whose flop is at least kAggregateMinRatio times their output size
// send many products to the same columns at once (hub columns of skewed
// graphs), and the compare-and-swap loops on those slots serialise.  In such
// rows the lanes that are converged at an accumulation and hold the same
// output rank first sum their products by shuffles (__match_any_sync), and
// one of them adds the sum.  Measured: worth it only for such rows; for rows
// of smaller ratio the match costs more than the contention it removes.
constexpr long long kAggregateMinRatio = 32;

// Heavy rows with a saved column bitmap.  Item (t, wdw, part, parts): bitmap
// t of the symbolic bitmap bin (row bm_rows[t]), output ranks
// [wdw*cap, (wdw+1)*cap) in shared memory, products of the part'th of
// `parts` ranges of the row's stored a_ik.  A row in one part stores its
// values; a split row's parts add theirs into C (zeroed by k_bm_zero_split)
// and part 0 stores the columns.  The items of a row with more than cap
// entries (window 0) add the products of ranks from cap on straight into C
// (zeroed there by k_bm_zero_split) with global atomics, and part 0 stores
// every column of the row.
// Every product goes through compare-and-swap accumulation (f64) or atomic
// adds into the rank-indexed values.
template <typename T, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_num_bitmap(Args a, const int32_t *__restrict__ bm_rows, const int4 *__restrict__ items,
                 const int64_t *__restrict__ flop, const uint32_t *__restrict__ bitmaps, int words, int cap,
                 const int32_t *__restrict__ c_rp,
                 int32_t *__restrict__ c_ci, T *__restrict__ c_v) {
  extern __shared__ __align__(16) unsigned char sm_num_bm[];
  __shared__ int red[33];
  __shared__ Entry<T> s_ent[kStageN];
  __shared__ long long s_wsum[8];
  __shared__ int s_next;
  T *vals = reinterpret_cast<T *>(sm_num_bm);
  // word w of the row's column bitmap and the number of set bits before it
  uint2 *rk = reinterpret_cast<uint2 *>(sm_num_bm + (size_t)cap * sizeof(T));
  const int4 item = items[blockIdx.x];
  const int32_t i = bm_rows[item.x];
  if (!in_rows(a, i)) return;
  const int part = item.z, parts = item.w;
  const bool agg = flop[i] >= kAggregateMinRatio * (c_rp[i + 1] - c_rp[i]);
  const int32_t rp = c_rp[i];
  const int32_t nnz = c_rp[i + 1] - rp;
  const int32_t cb = a.col_base ? a.col_base[i] : 0;
  const int32_t lo = item.y * cap;
  const int32_t hi = min(nnz, lo + cap);
  // ranks [hi, nnz) are added straight into C (rows with more than cap entries)
  const bool ovf = lo == 0 && hi < nnz;
  T *const c_row = c_v + rp;
  const uint32_t *src = bitmaps + (size_t)item.x * words;
  int32_t j_lo = a.arp[i], j_hi = a.arp[i + 1];
  if (parts > 1) part_range(a, i, part, parts, &j_lo, &j_hi);
  const int per = (words + blockDim.x - 1) / blockDim.x;
  const int w0 = threadIdx.x * per, w1 = min(words, w0 + per);
  int local = 0;
  for (int w = w0; w < w1; ++w) {
    const uint32_t b = src[w];
    rk[w].x = b;
    local += __popc(b);
  }
  int tot;
  int run = block_excl_scan(local, red, &tot);
  for (int w = w0; w < w1; ++w) {
    rk[w].y = (uint32_t)run;
    run += __popc(rk[w].x);
  }
  for (int r = threadIdx.x; r < hi - lo; r += blockDim.x) vals[r] = T(0);
  __syncthreads();
  const int span = hi - lo;
  // rank of column c among the row's columns, relative to the window
  auto rank_of = [&](int32_t c) {
    const uint2 word = rk[c >> 5];
    return (int)word.y + __popc(word.x & ((1u << (c & 31)) - 1u)) - lo;
  };
  block_row_products_long<kUN, true, false, T>(
      j_lo, j_hi, a.G, a.aci, (const T *)a.av, a.brp, a.bci, (const T *)a.bv, (int32_t)a.k, a.err, nullptr,
      Stage<T>{s_ent, &s_next, s_wsum},
      [&](const int32_t (&c)[kUN], const T (&av)[kUN], const T (&bv)[kUN], const bool (&ok)[kUN]) {
        int r[kUN];
        bool act[kUN];
#pragma unroll
        for (int u = 0; u < kUN; ++u) {
          r[u] = ok[u] ? rank_of(c[u]) : -1;
          act[u] = ok[u] && (unsigned)r[u] < (unsigned)span;
          if (ovf && ok[u] && r[u] >= span && r[u] < nnz) Val<T>::acc_global(c_row + r[u], av[u], bv[u]);
        }
        if (!agg) {
          // one product after another (measured: issuing the kUN swaps together
          // retried more and ran the large class 30% slower)
#pragma unroll
          for (int u = 0; u < kUN; ++u)
            if (act[u] && !Val<T>::acc_shared(vals + r[u], av[u], bv[u])) raise_err(a.err, kErrRetry);
          return;
        }
#pragma unroll
        for (int u = 0; u < kUN; ++u) {
          if (!act[u]) continue;
          const unsigned actm = __activemask();
          const unsigned grp = __match_any_sync(actm, r[u]);
          const int ln = threadIdx.x & 31;
          if (grp != (1u << ln)) {
            const T v = av[u] * bv[u];
            T sum = T(0);
            for (unsigned m = grp; m; m &= m - 1) sum += __shfl_sync(grp, v, __ffs(m) - 1);
            if (ln == __ffs(grp) - 1 && !Val<T>::acc_shared(vals + r[u], sum, T(1))) raise_err(a.err, kErrRetry);
            continue;
          }
          if (!Val<T>::acc_shared(vals + r[u], av[u], bv[u])) raise_err(a.err, kErrRetry);
        }
      },
      SkipLong{});
  __syncthreads();
  // Store ranks [lo, hi).  vals[] is already in rank order, so the block
  // copies it out with coalesced writes (a split row's parts add theirs).
  // Columns are then staged in the same shared array: thread t takes bitmap
  // words t, t + blockDim.x, ...; the set bits of word w, in order, are the
  // entries of ranks prefix[w], prefix[w] + 1, ..., so no entry needs a
  // search for its word; the staged columns go out with coalesced writes.
  if (parts == 1) {
    for (int r = threadIdx.x; r < hi - lo; r += blockDim.x) c_v[rp + lo + r] = vals[r];
  } else {
    for (int r = threadIdx.x; r < hi - lo; r += blockDim.x) {
      const T v = vals[r];
      if (v != T(0)) Val<T>::add_global(c_v + rp + lo + r, v);
    }
  }
  if (part == 0) {
    __syncthreads();
    int32_t *cols = reinterpret_cast<int32_t *>(vals);
    const int32_t top = ovf ? nnz : hi;  // ranks [hi, top) go straight to C
    for (int w = threadIdx.x; w < words; w += blockDim.x) {
      const uint2 wd = rk[w];
      int r = (int)wd.y;
      if (r >= top || r + __popc(wd.x) <= lo) continue;
      for (unsigned bits = wd.x; bits != 0u; bits &= bits - 1u, ++r) {
        const int32_t col = w * 32 + __ffs(bits) - 1;
        if (r >= lo && r < hi) cols[r - lo] = col;
        else if (r >= hi && r < top) c_ci[rp + r] = col - cb;
      }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < hi - lo; r += blockDim.x) c_ci[rp + lo + r] = cols[r] - cb;
  }
  if (threadIdx.x == 0 && tot != nnz) raise_err(a.err, kErrProbe);
}

// Heavy rows without bitmaps: block b owns table b (S slots of keys and
// values in global memory) and walks rows b, b+gridDim.x, ...  Sorted
// output ranks the row's columns window by window with a shared-memory
// bitmap of win_words words.
template <typename T>
__global__ void __launch_bounds__(1024, 1)
    k_num_global(Args a, BinRows br, int32_t *__restrict__ keys_all, T *__restrict__ vals_all, int64_t S,
                 const int32_t *__restrict__ c_rp, int32_t *__restrict__ c_ci, T *__restrict__ c_v, int sorted,
                 int win_words) {
  extern __shared__ __align__(16) unsigned char sm_num_gl[];
  __shared__ int red[33];
  __shared__ Entry<T> s_ent[kStageN];
  __shared__ long long s_wsum[8];
  __shared__ int s_next;
  __shared__ int cursor;
  if (aborted(a)) return;
  int32_t *keys = keys_all + (size_t)blockIdx.x * S;
  T *vals = vals_all + (size_t)blockIdx.x * S;
  const uint32_t mask = (uint32_t)(S - 1);
  const int G = a.G;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const long long o0 = br.off[br.bin], nrows = br.off[br.bin + 1] - o0;
  for (int64_t r = blockIdx.x; r < nrows; r += gridDim.x) {
    if (!in_rows(a, br.perm[o0 + r])) continue;
    for (int64_t s = threadIdx.x; s < S; s += blockDim.x) {
      keys[s] = kEmpty;
      vals[s] = T(0);
    }
    if (threadIdx.x == 0) cursor = 0;
    __syncthreads();
    const int32_t i = br.perm[o0 + r];
    block_row_products<kUN, true, T>(a.arp[i], a.arp[i + 1], G, a.aci, (const T *)a.av, a.brp, a.bci,
                                   (const T *)a.bv, (int32_t)a.k, a.err, Stage<T>{s_ent, &s_next, s_wsum},
                                   [&](int32_t c, T av, T bv) { insert_acc<T, true>(keys, vals, mask, c, av, bv, a.err, a.probe, a.probe_ctr); });
    __syncthreads();
    const int32_t rp = c_rp[i];
    const int32_t nnz = c_rp[i + 1] - rp;
    const int32_t cb = a.col_base ? a.col_base[i] : 0;
    if (!sorted) {
      for (int64_t s0 = (int64_t)warp * 32; s0 < S; s0 += (int64_t)nw * 32) {
        const int64_t s = s0 + lane;
        const int32_t kk = keys[s];
        const bool occ = kk != kEmpty;
        const unsigned m = __ballot_sync(0xffffffffu, occ);
        int base = 0;
        if (lane == 0 && m) base = atomicAdd(&cursor, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        const int pos = base + __popc(m & ((1u << lane) - 1u));
        if (occ && pos < nnz) {
          c_ci[rp + pos] = kk - cb;
          c_v[rp + pos] = vals[s];
        }
      }
      __syncthreads();
      if (threadIdx.x == 0 && cursor != nnz) raise_err(a.err, kErrProbe);
    } else {
      uint32_t *bm = reinterpret_cast<uint32_t *>(sm_num_gl);
      int32_t *pre = reinterpret_cast<int32_t *>(bm + win_words);
      const int64_t wcols = (int64_t)win_words * 32;
      int base = 0;
      for (int64_t c0 = 0; c0 < a.k; c0 += wcols) {
        for (int w = threadIdx.x; w < win_words; w += blockDim.x) bm[w] = 0u;
        __syncthreads();
        for (int64_t s = threadIdx.x; s < S; s += blockDim.x) {
          const int32_t kk = keys[s];
          if (kk != kEmpty && kk >= c0 && kk < c0 + wcols) {
            const int32_t o = (int32_t)(kk - c0);
            atomicOr(bm + (o >> 5), 1u << (o & 31));
          }
        }
        __syncthreads();
        const int per = (win_words + blockDim.x - 1) / blockDim.x;
        const int w0 = threadIdx.x * per, w1 = min(win_words, w0 + per);
        int local = 0;
        for (int w = w0; w < w1; ++w) local += __popc(bm[w]);
        int tot;
        int run = block_excl_scan(local, red, &tot);
        for (int w = w0; w < w1; ++w) {
          pre[w] = run;
          run += __popc(bm[w]);
        }
        __syncthreads();
        for (int64_t s = threadIdx.x; s < S; s += blockDim.x) {
          const int32_t kk = keys[s];
          if (kk != kEmpty && kk >= c0 && kk < c0 + wcols) {
            const int32_t o = (int32_t)(kk - c0);
            const int rr = base + pre[o >> 5] + __popc(bm[o >> 5] & ((1u << (o & 31)) - 1u));
            if (rr < nnz) {
              c_ci[rp + rr] = kk - cb;
              c_v[rp + rr] = vals[s];
            }
          }
        }
        base += tot;
        __syncthreads();
      }
      if (threadIdx.x == 0 && base != nnz) raise_err(a.err, kErrProbe);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Raises the kernel's dynamic shared memory limit once per size (the
// static arrays count against the default 48 KB as well).
template <typename K>
static cudaError_t prep_num(K kernel, size_t smem) {
  return set_dynamic_smem(reinterpret_cast<const void *>(kernel), smem);
}

template <typename T, int S>
static cudaError_t num_warp(spgemm_plan_s *p, cudaStream_t st, const Args &a, BinRows br, int64_t n,
                            const int32_t *c_rp, int32_t *c_ci, T *c_v) {
  const size_t smem = (size_t)kWarpsPerBlock * S * (sizeof(int32_t) + sizeof(T));
  cudaError_t e = prep_num(k_num_warp<T, S>, smem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = launch_blocks(p, reinterpret_cast<const void *>(k_num_warp<T, S>), kWarpsPerBlock * 32, smem,
                                       (n + kWarpsPerBlock - 1) / kWarpsPerBlock);
  {
    KernelScope ks(p, "num_warp_" + std::to_string(S), st);
    k_num_warp<T, S><<<(unsigned)blocks, kWarpsPerBlock * 32, smem, st>>>(a, br, c_rp, c_ci, c_v,
                                                                           (p->flags & SPGEMM_SORTED) ? 1 : 0);
  }
  return cudaGetLastError();
}

template <typename T, int S>
static cudaError_t num_block(spgemm_plan_s *p, cudaStream_t st, const Args &a, BinRows br, int64_t n,
                             int threads, const int32_t *c_rp, int32_t *c_ci, T *c_v) {
  size_t smem = (size_t)S * (sizeof(int32_t) + sizeof(T));
  int mode = 0;
  // sorted output: rank by a bitmap over each row's column window of up to
  // kSortWindowWords x 32 columns (the whole of B's columns when they fit)
  const int words = (int)std::min<int64_t>((p->span_cols + 31) / 32, kSortWindowWords);
  if (p->flags & SPGEMM_SORTED) {
    const size_t extra = (size_t)words * 8;
    if (smem + extra + kStaticSmemReserve <= (size_t)max_smem_per_block()) {
      mode = 2;
      smem += extra;
    } else {
      mode = 1;
    }
  }
  cudaError_t e = prep_num(k_num_block<T, S>, smem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = launch_blocks(p, reinterpret_cast<const void *>(k_num_block<T, S>), threads, smem, n);
  {
    KernelScope ks(p, "num_block_" + std::to_string(S), st);
    k_num_block<T, S><<<(unsigned)blocks, threads, smem, st>>>(a, br, c_rp, c_ci, c_v, mode, words);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_numeric_t(spgemm_plan_s *p, const int32_t *c_rp, int32_t *c_ci, T *c_v) {
  Args a = phase_args(p, &p->dc->err, probe_mode(p->flags),
                      (p->flags & SPGEMM_COUNT_PROBES) ? &p->dc->probe_stats[2][0] : nullptr);
  if (p->ddrive) a.abort = &p->dc->err;
  // bitmap classes first (small, medium, large), then the hash bins from the
  // heaviest, each bin on the next side stream.  Measured: the triangle
  // product (small and medium classes only) ran 1.26 -> 1.13 ms with the small
  // class launched before the medium one; R-MAT A*A (scale 16) was unchanged.
  static const int order[kNumNumBins] = {kNumBitmapSBin, kNumBitmapMBin, kNumBitmapBin, kNumGlobalBin, 8, 7, 6, 5,
                                         4, 3, 2, 1, 0};
  const bool concurrent = use_side_streams(p);
  cudaError_t e = cudaSuccess;
  const int64_t nbm = p->sym_count[kSymBitmapBin] + p->sym_count[kSymBitmapMidBin];
  if (p->a_compact) e = compact_a_values(p);
  if (e == cudaSuccess && nbm > 0 && p->bm_item_off[3] > 0) {
    // before the fork: every bitmap launch adds into the zeroed split rows
    KernelScope ks(p, "bm_zero_split");
    k_bm_zero_split<T><<<(unsigned)((nbm + 7) / 8), 256, 0, p->stream>>>(
        p->perm + p->sym_off[kSymBitmapBin], nbm, p->flop, c_rp, c_v, a.row_lo, a.row_hi, p->bm_cap[2]);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && concurrent) e = fork(p);
  int launched = 0;
  for (int o = 0; o < kNumNumBins && e == cudaSuccess; ++o) {
    const int b = order[o];
    // a graph-mode plan launches every bin it may need (counts unknown on the host)
    const int64_t n = p->ddrive ? ddrive_bin_rows(p, b, false) : p->num_count[b];
    if (n == 0) continue;
    const BinRows br{p->perm2, p->d_num_off, b};
    const BinCfg &c = kNumBins[b];
    cudaStream_t st = concurrent ? bin_stream(p, launched++) : p->stream;
    switch (b) {
      case 0: e = num_warp<T, 64>(p, st, a, br, n, c_rp, c_ci, c_v); break;
      case 1: e = num_warp<T, 128>(p, st, a, br, n, c_rp, c_ci, c_v); break;
      case 2: e = num_warp<T, 256>(p, st, a, br, n, c_rp, c_ci, c_v); break;
      case 3: e = num_warp<T, 512>(p, st, a, br, n, c_rp, c_ci, c_v); break;
      case 4: e = num_warp<T, 1024>(p, st, a, br, n, c_rp, c_ci, c_v); break;
      case 5: e = num_block<T, 2048>(p, st, a, br, n, c.threads, c_rp, c_ci, c_v); break;
      case 6: e = num_block<T, 4096>(p, st, a, br, n, c.threads, c_rp, c_ci, c_v); break;
      case 7: e = num_block<T, 8192>(p, st, a, br, n, c.threads, c_rp, c_ci, c_v); break;
      case 8: e = num_block<T, 16384>(p, st, a, br, n, c.threads, c_rp, c_ci, c_v); break;
      case kNumBitmapSBin:
      case kNumBitmapMBin:
      case kNumBitmapBin: {
        const int cls = b == kNumBitmapSBin ? 0 : b == kNumBitmapMBin ? 1 : 2;
        const size_t smem = (size_t)p->bm_cap[cls] * sizeof(T) + (size_t)p->bm_words * 8;
        // register budgets that let each class keep its shared-memory occupancy
        auto kern = cls == 0   ? k_num_bitmap<T, kBmThreadsS, kBmBlocksS>
                    : cls == 1 ? k_num_bitmap<T, kBmThreadsM, kBmBlocksM>
                               : k_num_bitmap<T, kBmThreadsL, 1>;
        e = prep_num(kern, smem);
        if (e != cudaSuccess) break;
        {
          KernelScope ks(p, cls == 0 ? "num_bitmap_s" : cls == 1 ? "num_bitmap_m" : "num_bitmap_l", st);
          kern<<<(unsigned)n, p->bm_threads[cls], smem, st>>>(
              a, p->perm + p->sym_off[kSymBitmapBin], p->bm_items + p->bm_item_off[cls], p->flop, p->bitmaps, p->bm_words,
              (int)p->bm_cap[cls], c_rp, c_ci, c_v);
        }
        e = cudaGetLastError();
        break;
      }
      case kNumGlobalBin: {
        const int win_words = 8192;  // 2^18 columns per window: 32 KB bitmap + 32 KB prefix
        const size_t smem = (p->flags & SPGEMM_SORTED) ? (size_t)win_words * 8 : 0;
        e = prep_num(k_num_global<T>, smem);
        if (e != cudaSuccess) break;
        int32_t *keys = (int32_t *)p->gtab;
        T *vals = reinterpret_cast<T *>((char *)p->gtab + (size_t)p->gtab_blocks * p->gtab_slots * sizeof(int32_t));
        {
          KernelScope ks(p, "num_global", st);
          k_num_global<T><<<(unsigned)p->gtab_blocks, c.threads, smem, st>>>(
              a, br, keys, vals, p->gtab_slots, c_rp, c_ci, c_v, (p->flags & SPGEMM_SORTED) ? 1 : 0, win_words);
        }
        e = cudaGetLastError();
        break;
      }
      default: break;
    }
  }
  if (concurrent && e == cudaSuccess) e = join(p);
  return e;
}

}  // namespace sg
