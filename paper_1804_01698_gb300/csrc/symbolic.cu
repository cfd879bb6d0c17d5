// Symbolic phase (paper Sec. 4.2.1: only keys, no values, go into the hash
// table): nnz(c_i*) = number of distinct keys inserted for row i.
//
//   k_sym_warp<S>    one warp per row, S-slot table in shared memory
//   k_sym_block<S>   one block per row, S-slot table in shared memory
//   k_sym_bitmap     heavy rows, one block per row, a bit per column of B in
//                    shared memory; the bitmap is saved for the numeric phase
//   k_sym_global     heavy rows when B has too many columns for a bitmap:
//                    the hash table lives in global memory (L2)
//
// Keys are inserted with atomicCAS on the int32 key (empty = -1) and
// linear probing (Sec. 4.2.1), or by chunks of 4 slots under
// SPGEMM_PROBE_CHUNK4 (Sec. 4.2.2); an insert that finds -1 claims the slot
// and counts one new column.
#include <algorithm>
#include <string>

#include "common.cuh"
#include "internal.h"
#include "rowsplit.cuh"

namespace sg {

constexpr int kU = 4;  // B entries loaded ahead per lane

// Inserts key c into an S-slot table; returns 1 when c was new.
// Every variant of the insert: chunked or linear probing, either hash,
// optional probe counting.  Only ablations and measurement runs take it.
// (Measured: an out-of-line call here, never taken, still slowed the default
// path of the warp bins by 5%, so it stays inline.)
template <bool GLOBAL_MEM>
__device__ __forceinline__ int insert_key_any(int32_t *tab, uint32_t mask, int32_t c, uint32_t *err, int probe,
                                           unsigned long long *ctr) {
  if (probe & kProbeChunk) {
    bool fresh = false;
    unsigned probes = 0;
    chunk_find_or_claim<GLOBAL_MEM>(tab, mask, c, &fresh, err, &probes, probe & kProbeHashHi);
    count_probes(ctr, probes);
    return fresh ? 1 : 0;
  }
  uint32_t h = hash_slot(c, mask, probe & kProbeHashHi);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const int32_t old = atomicCAS(tab + h, kEmpty, c);
    if (old == kEmpty || old == c) {
      count_probes(ctr, probe + 1);
      return old == kEmpty ? 1 : 0;
    }
    h = (h + 1) & mask;
  }
  raise_err(err, kErrProbe);
  return 0;
}

// Inserts key c; returns 1 when c was new.  The default plan (linear
// probing, top-bits hash, no counting) runs the loop inline.
template <bool GLOBAL_MEM>
__device__ __forceinline__ int insert_key(int32_t *tab, uint32_t mask, int32_t c, uint32_t *err, int probe,
                                          unsigned long long *ctr) {
  if (probe != kProbeHashHi || ctr) return insert_key_any<GLOBAL_MEM>(tab, mask, c, err, probe, ctr);
  uint32_t h = hash_slot(c, mask, 1);
  for (uint32_t q = 0; q <= mask; ++q) {
    const int32_t old = atomicCAS(tab + h, kEmpty, c);
    if (old == kEmpty) return 1;
    if (old == c) return 0;
    h = (h + 1) & mask;
  }
  raise_err(err, kErrProbe);
  return 0;
}

template <int S>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 8)
    k_sym_warp(Args a, BinRows br, int32_t *__restrict__ nnz_row) {
  extern __shared__ int32_t sm_sym_warp[];
  __shared__ Entry<int32_t> s_ent[kWarpsPerBlock][32];
  __shared__ int s_next[kWarpsPerBlock];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long o0 = br.off[br.bin], nrows = br.off[br.bin + 1] - o0;
  int32_t *tab = sm_sym_warp + warp * S;
  const int G = a.G;
  Stage<int32_t> st{s_ent[warp], &s_next[warp], nullptr};
  // one warp per row (no block barrier below)
  for (int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + warp; w < nrows; w += (int64_t)gridDim.x * kWarpsPerBlock) {
    for (int s = lane; s < S; s += 32) tab[s] = kEmpty;
    __syncwarp();
    const int32_t i = br.perm[o0 + w];
    int cnt = 0;
    warp_row_products<kU, false, int32_t>(a.arp[i], a.arp[i + 1], G, a.aci, (const int32_t *)nullptr, a.brp, a.bci,
                                          (const int32_t *)nullptr, (int32_t)a.k, a.err, st,
                                          [&](int32_t c, int32_t, int32_t) { cnt += insert_key<false>(tab, S - 1, c, a.err, a.probe, a.probe_ctr); });
    cnt = warp_sum(cnt);
    if (lane == 0) nnz_row[i] = cnt;
    __syncwarp();
  }
}

// Threads of the block bins (as kSymBins) and blocks per SM: a key table of
// S slots leaves room for these, so the register budget is set to match.
template <int S> constexpr int sym_block_threads() { return S <= 2048 ? 256 : S <= 4096 ? 512 : 1024; }
template <int S> constexpr int sym_block_min_blocks() { return S <= 2048 ? 8 : S <= 4096 ? 4 : S <= 16384 ? 2 : 1; }

template <int S>
__global__ void __launch_bounds__(sym_block_threads<S>(), sym_block_min_blocks<S>())
    k_sym_block(Args a, BinRows br, int32_t *__restrict__ nnz_row) {
  extern __shared__ int32_t sm_sym_block[];
  __shared__ int red[33];
  __shared__ Entry<int32_t> s_ent[kStageN];
  __shared__ long long s_wsum[8];
  __shared__ int s_next;
  int32_t *tab = sm_sym_block;
  const long long o0 = br.off[br.bin], nrows = br.off[br.bin + 1] - o0;
  const int G = a.G;
  for (int64_t b = blockIdx.x; b < nrows; b += gridDim.x) {  // one block per row
    for (int s = threadIdx.x; s < S; s += blockDim.x) tab[s] = kEmpty;
    __syncthreads();
    const int32_t i = br.perm[o0 + b];
    int cnt = 0;
    block_row_products<kU, false, int32_t>(a.arp[i], a.arp[i + 1], G, a.aci, (const int32_t *)nullptr,
                                           a.brp, a.bci, (const int32_t *)nullptr, (int32_t)a.k, a.err,
                                           Stage<int32_t>{s_ent, &s_next, s_wsum},
                                           [&](int32_t c, int32_t, int32_t) { cnt += insert_key<false>(tab, S - 1, c, a.err, a.probe, a.probe_ctr); });
    cnt = block_sum(cnt, red);  // ends with a barrier: the table may be cleared again
    if (threadIdx.x == 0) nnz_row[i] = cnt;
  }
}

// Heavy rows with a bitmap over the columns of B.  words = ceil(k / 32).
// A stored a_ik whose row of B is a long row (lr.map) sets that row's
// columns by ORing its saved bitmap, word by word, into the row's bitmap
// (thread t owns words t, t + NT, ...), instead of one atomic per entry.
template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_sym_bitmap(Args a, const int32_t *__restrict__ rows, const int4 *__restrict__ items,
                 int32_t *__restrict__ nnz_row, uint32_t *__restrict__ bitmaps, int words,
                 unsigned *__restrict__ tickets, LongRows lr) {
  extern __shared__ uint32_t sm_bm[];
  __shared__ int red[33];
  __shared__ Entry<int32_t> s_ent[kStageN];
  __shared__ long long s_wsum[8];
  __shared__ int s_next;
  __shared__ int s_last;
  __shared__ int s_lidx[kStageN];
  __shared__ int s_lcnt[kStageN / 32];
  // block b is row b of the bin, or, for split rows, work item b (row t of
  // the bin, part `part` of `parts`)
  int t = blockIdx.x, part = 0, parts = 1;
  if (items) {
    const int4 it = items[blockIdx.x];
    t = it.x;
    part = it.y;
    parts = it.z;
  }
  for (int w = threadIdx.x; w < words; w += blockDim.x) sm_bm[w] = 0u;
  const int32_t i = rows[t];
  int32_t j_lo = a.arp[i], j_hi = a.arp[i + 1];
  if (parts > 1) part_range(a, i, part, parts, &j_lo, &j_hi);
  __syncthreads();
  const int G = a.G;
  block_row_products_long<kU, false, true, int32_t>(
      j_lo, j_hi, G, a.aci, (const int32_t *)nullptr, a.brp, a.bci, (const int32_t *)nullptr, (int32_t)a.k, a.err,
      lr.map, Stage<int32_t>{s_ent, &s_next, s_wsum, s_lidx, s_lcnt},
      [&](const int32_t (&c)[kU], const int32_t (&)[kU], const int32_t (&)[kU], const bool (&ok)[kU]) {
#pragma unroll
        for (int u = 0; u < kU; ++u)
          if (ok[u]) atomicOr(sm_bm + (c[u] >> 5), 1u << (c[u] & 31));
      },
      [&](int nlong, const int *lidx) {
        // this thread's words, 4 at a time: OR of the round's long rows
        for (int w0 = threadIdx.x; w0 < words; w0 += 4 * NT) {
          uint32_t x[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) x[q] = 0u;
#pragma unroll 8
          for (int l = 0; l < nlong; ++l) {
            const uint32_t *bw = lr.bits + (size_t)s_ent[lidx[l]].off * words;
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (w0 + q * NT < words) x[q] |= __ldg(bw + w0 + q * NT);
          }
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (w0 + q * NT < words && x[q]) sm_bm[w0 + q * NT] |= x[q];
        }
      });
  uint32_t *out = bitmaps + (size_t)t * words;
  if (parts == 1) {
    int cnt = 0;
    for (int w = threadIdx.x; w < words; w += blockDim.x) {
      const uint32_t b = sm_bm[w];
      out[w] = b;
      cnt += __popc(b);
    }
    cnt = block_sum(cnt, red);
    if (threadIdx.x == 0) nnz_row[i] = cnt;
    return;
  }
  // a part ORs its bits into the row's bitmap (zeroed before the launch);
  // the last part to finish counts the union
  for (int w = threadIdx.x; w < words; w += blockDim.x) {
    const uint32_t b = sm_bm[w];
    if (b) atomicOr(out + w, b);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(tickets + t, 1u) == (unsigned)(parts - 1);
  __syncthreads();
  if (s_last) {
    __threadfence();
    int cnt = 0;
    for (int w = threadIdx.x; w < words; w += blockDim.x) cnt += __popc(__ldcg(out + w));
    cnt = block_sum(cnt, red);
    if (threadIdx.x == 0) nnz_row[i] = cnt;
  }
}

// Work items of the split heavy bitmap rows: row t of the bin (rows[t]) gets
// sym_split_parts(flop) items (t, part, parts).
__global__ void __launch_bounds__(256)
    k_sym_items_fill(const int32_t *__restrict__ rows, int64_t n, const int64_t *__restrict__ flop, DevCounters *dc,
                     int4 *__restrict__ items) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int parts = sym_split_parts(flop[rows[t]]);
  const unsigned long long base = atomicAdd(&dc->sym_item_cursor, (unsigned long long)parts);
  for (int q = 0; q < parts; ++q) items[base + q] = make_int4((int)t, q, parts, 0);
}

// Heavy rows, hash table in global memory: block b owns tables[b*S .. b*S+S)
// and walks rows b, b+gridDim.x, ...
__global__ void __launch_bounds__(1024, 1)
    k_sym_global(Args a, BinRows br, int32_t *__restrict__ nnz_row, int32_t *__restrict__ tables, int64_t S) {
  __shared__ int red[33];
  __shared__ Entry<int32_t> s_ent[kStageN];
  __shared__ long long s_wsum[8];
  __shared__ int s_next;
  int32_t *tab = tables + (size_t)blockIdx.x * S;
  const uint32_t mask = (uint32_t)(S - 1);
  const int G = a.G;
  const long long o0 = br.off[br.bin], nrows = br.off[br.bin + 1] - o0;
  for (int64_t r = blockIdx.x; r < nrows; r += gridDim.x) {
    for (int64_t s = threadIdx.x; s < S; s += blockDim.x) tab[s] = kEmpty;
    __syncthreads();
    const int32_t i = br.perm[o0 + r];
    int cnt = 0;
    block_row_products<kU, false, int32_t>(a.arp[i], a.arp[i + 1], G, a.aci, (const int32_t *)nullptr,
                                         a.brp, a.bci, (const int32_t *)nullptr, (int32_t)a.k, a.err,
                                         Stage<int32_t>{s_ent, &s_next, s_wsum},
                                         [&](int32_t c, int32_t, int32_t) { cnt += insert_key<true>(tab, mask, c, a.err, a.probe, a.probe_ctr); });
    cnt = block_sum(cnt, red);
    if (threadIdx.x == 0) nnz_row[i] = cnt;
  }
}

// ---------------------------------------------------------------------------
// Raises the kernel's dynamic shared memory limit once per size (the
// static arrays count against the default 48 KB as well).
template <typename K>
static cudaError_t prep(K kernel, size_t smem) {
  return set_dynamic_smem(reinterpret_cast<const void *>(kernel), smem);
}

template <int S>
static cudaError_t sym_warp(spgemm_plan_s *p, cudaStream_t st, const Args &a, BinRows br, int64_t n) {
  const size_t smem = (size_t)kWarpsPerBlock * S * sizeof(int32_t);
  cudaError_t e = prep(k_sym_warp<S>, smem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = launch_blocks(p, reinterpret_cast<const void *>(k_sym_warp<S>), kWarpsPerBlock * 32, smem,
                                       (n + kWarpsPerBlock - 1) / kWarpsPerBlock);
  {
    KernelScope ks(p, "sym_warp_" + std::to_string(S), st);
    k_sym_warp<S><<<(unsigned)blocks, kWarpsPerBlock * 32, smem, st>>>(a, br, p->nnz_row);
  }
  return cudaGetLastError();
}

template <int S>
static cudaError_t sym_block(spgemm_plan_s *p, cudaStream_t st, const Args &a, BinRows br, int64_t n, int threads) {
  const size_t smem = (size_t)S * sizeof(int32_t);
  cudaError_t e = prep(k_sym_block<S>, smem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = launch_blocks(p, reinterpret_cast<const void *>(k_sym_block<S>), threads, smem, n);
  {
    KernelScope ks(p, "sym_block_" + std::to_string(S), st);
    k_sym_block<S><<<(unsigned)blocks, threads, smem, st>>>(a, br, p->nnz_row);
  }
  return cudaGetLastError();
}

cudaError_t launch_symbolic(spgemm_plan_s *p) {
  const Args a = phase_args(p, &p->dc->err, probe_mode(p->flags),
                            (p->flags & SPGEMM_COUNT_PROBES) ? &p->dc->probe_stats[0][0] : nullptr);
  // heavy bins first.  The two bitmap bins take side streams 0 and 1, the
  // other bins streams 2 and 3 in turn, so that no hash bin waits behind a
  // bitmap launch on its stream.  Measured against one bin per next stream:
  // the triangle product ran 1.07 -> 1.02 ms, R-MAT A*A (scale 16) the same.
  static const int order[kNumSymBins] = {kSymBitmapBin, kSymBitmapMidBin, kSymGlobalBin, 9, 8, 7, 6, 5, 4, 3, 2, 1, 0};
  const bool concurrent = use_side_streams(p);
  cudaError_t e = cudaSuccess;
  // split heavy bitmap rows: work items, zeroed tickets and bitmaps (on the
  // plan's stream, before the side streams fork from it)
  const int64_t nheavy = p->sym_count[kSymBitmapBin];
  const int64_t extra = (int64_t)p->hc->sym_split_extra;
  p->n_sym_items = 0;
  if (nheavy > 0 && extra > 0) {
    const int64_t n_items = nheavy + extra;
    const size_t items_bytes = ((size_t)n_items * sizeof(int4) + 255) / 256 * 256;
    e = cudaMallocAsync((void **)&p->sym_items, items_bytes + (size_t)nheavy * sizeof(unsigned), p->stream);
    if (e != cudaSuccess) {
      p->sym_items = nullptr;
      return e;
    }
    p->sym_tickets = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(p->sym_items) + items_bytes);
    e = cudaMemsetAsync(p->sym_tickets, 0, (size_t)nheavy * sizeof(unsigned), p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->bitmaps, 0, (size_t)nheavy * p->bm_words * sizeof(uint32_t), p->stream);
    if (e == cudaSuccess) {
      KernelScope ks(p, "sym_items_fill");
      k_sym_items_fill<<<(unsigned)((nheavy + 255) / 256), 256, 0, p->stream>>>(p->perm + p->sym_off[kSymBitmapBin],
                                                                                nheavy, p->flop, p->dc, p->sym_items);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    p->n_sym_items = n_items;
  }
  if (concurrent) e = fork(p);
  int launched = 0;
  for (int o = 0; o < kNumSymBins && e == cudaSuccess; ++o) {
    const int b = order[o];
    // a graph-mode plan launches every bin it may need (counts unknown on the host)
    const int64_t n = p->ddrive ? ddrive_bin_rows(p, b, true) : p->sym_count[b];
    if (n == 0) continue;
    const int32_t *rows = p->perm + p->sym_off[b];
    const BinRows br{p->perm, p->d_sym_off, b};
    const BinCfg &c = kSymBins[b];
    const int si = b == kSymBitmapBin ? 0 : b == kSymBitmapMidBin ? 1 : 2 + (launched++ & 1);
    cudaStream_t st = concurrent ? bin_stream(p, si) : p->stream;
    switch (b) {
      case 0: e = sym_warp<64>(p, st, a, br, n); break;
      case 1: e = sym_warp<128>(p, st, a, br, n); break;
      case 2: e = sym_warp<256>(p, st, a, br, n); break;
      case 3: e = sym_warp<512>(p, st, a, br, n); break;
      case 4: e = sym_warp<1024>(p, st, a, br, n); break;
      case 5: e = sym_block<2048>(p, st, a, br, n, c.threads); break;
      case 6: e = sym_block<4096>(p, st, a, br, n, c.threads); break;
      case 7: e = sym_block<8192>(p, st, a, br, n, c.threads); break;
      case 8: e = sym_block<16384>(p, st, a, br, n, c.threads); break;
      case 9: e = sym_block<32768>(p, st, a, br, n, c.threads); break;
      case kSymBitmapBin:
      case kSymBitmapMidBin: {
        // bitmaps of both bins are stored in perm order from the first bitmap bin on
        const size_t smem = (size_t)p->bm_words * sizeof(uint32_t);
        // heavy and medium rows alike 8 x 256 threads per SM: the register
        // budget (32 per thread) that lets the bitmaps' shared memory set the
        // occupancy (measured 22% faster than 64 registers).  The two bins run
        // side by side on their own streams, and blocks of one shape interleave
        // on the SMs.  Measured on R-MAT A*A, scale 16: heavy rows at 2 x 1024
        // threads per SM ran the whole product 8% slower (4.02 against 3.70 ms),
        // at 4 x 512 1% slower.
        auto kern = k_sym_bitmap<256, 8>;
        e = prep(kern, smem);
        if (e != cudaSuccess) break;
        {
          KernelScope ks(p, b == kSymBitmapBin ? "sym_bitmap_heavy" : "sym_bitmap_mid", st);
          uint32_t *bm = p->bitmaps + (size_t)(p->sym_off[b] - p->sym_off[kSymBitmapBin]) * p->bm_words;
          const bool split = b == kSymBitmapBin && p->n_sym_items > 0;
          kern<<<(unsigned)(split ? p->n_sym_items : n), c.threads, smem, st>>>(
              a, rows, split ? p->sym_items : nullptr, p->nnz_row, bm, p->bm_words, split ? p->sym_tickets : nullptr,
              long_rows(p));
        }
        e = cudaGetLastError();
        break;
      }
      case kSymGlobalBin: {
        {
          KernelScope ks(p, "sym_global", st);
          k_sym_global<<<(unsigned)p->gtab_blocks, c.threads, 0, st>>>(a, br, p->nnz_row, (int32_t *)p->gtab,
                                                                      p->gtab_slots);
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
