// Symbolic phase without any device allocation.
//
// Some callers cannot allocate device memory while they run: code inside a
// custom allocator or a memory-pool callback, a real-time or latency-bound
// loop that must never reach the driver's allocator, or a host that has
// handed all device memory to another framework.  For them this file offers
// spgemm_symbolic_noalloc(): it counts the entries of every row of C = A*B
// and writes C's row_ptr and nnz(C), like spgemm_symbolic, but its scratch
// (the per-block hash tables and a few counters) is one file-scope device
// array, g_noalloc_scratch, that is placed on a device when the library's
// module is first used there (CUDA loads modules lazily: at the first kernel
// launch of this library or this entry point's first cudaGetSymbolAddress
// on that device) and stays until the process exits.  So the first call on
// each device, or any earlier call of this library on it, must come before
// the region in which the caller cannot allocate; later calls make no
// cudaMalloc or cudaFree call and call no library routine that allocates.
//
// The kernel is the global-table form of the symbolic phase: block b owns
// one hash table of kNoallocSlots keys inside the array and walks rows b,
// b + kNoallocBlocks, ...; each row is hashed into the first 2^s slots with
// 2^s > min(flop_i, k) (paper Sec. 4.2.1), so a row whose bound reaches
// kNoallocSlots is refused with SPGEMM_ERR_INVALID_ARGUMENT.
#include <cstring>
#include <mutex>
#include <string>

#include "common.cuh"
#include "internal.h"

namespace sg {

constexpr int kNoallocBlocks = 64;
constexpr int64_t kNoallocSlots = 1 << 17;  // keys per block table (512 KiB)
constexpr size_t kNoallocHeader = 256;      // counters at the start of the array
constexpr size_t kNoallocBytes = kNoallocHeader + (size_t)kNoallocBlocks * kNoallocSlots * sizeof(int32_t);

// Shared by every call on a device (32 MiB + 256 B, allocated when the
// library's module is loaded).  Only host code needs its device address,
// obtained once per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

struct NoallocHeader {
  unsigned long long total;      // nnz(C)
  unsigned long long max_bound;  // largest refused row bound
  unsigned int err;              // kErr* bits, plus kErrTooLarge
  unsigned int pad;
};
constexpr uint32_t kErrTooLarge = 16u;

__global__ void __launch_bounds__(1024, 1)
    k_noalloc_count(Args a, int64_t nnz_a, int64_t nnz_b, int32_t *__restrict__ c_row_ptr, unsigned char *scratch) {
  __shared__ long long red[33];
  __shared__ Entry<int32_t> s_ent[kStageN];
  __shared__ long long s_wsum[8];
  __shared__ int s_next;
  NoallocHeader *hdr = reinterpret_cast<NoallocHeader *>(scratch);
  int32_t *tab = reinterpret_cast<int32_t *>(scratch + kNoallocHeader) + (size_t)blockIdx.x * kNoallocSlots;
  const int G = a.G;
  for (int64_t i = blockIdx.x; i < a.m; i += gridDim.x) {
    // row flop and input checks (as in the flop pass)
    int64_t r0 = a.arp[i], r1 = a.arp[i + 1];
    const bool bad_rp = !(0 <= r0 && r0 <= r1 && r1 <= nnz_a);
    long long f = 0, nbad = 0;
    if (!bad_rp) {
      for (int64_t j = r0 + threadIdx.x; j < r1; j += blockDim.x) {
        const int32_t kk = a.aci[j];
        if ((uint64_t)(int64_t)kk >= (uint64_t)a.n) {
          ++nbad;
          continue;
        }
        const int64_t b0 = a.brp[kk], b1 = a.brp[kk + 1];
        if (!(0 <= b0 && b0 <= b1 && b1 <= nnz_b)) {
          ++nbad;
          continue;
        }
        f += b1 - b0;
      }
    }
    f = block_sum(f, red);
    // A row with a column outside A, or one that selects a malformed row of
    // B, is never hashed: the row loop below would read B's row_ptr and
    // col_idx at the unchecked addresses.
    nbad = block_sum(nbad, red);
    const bool bad = bad_rp || nbad > 0;
    if (bad && threadIdx.x == 0) raise_err(a.err, kErrCsr);
    const long long bound = f < a.k ? f : a.k;
    int cnt = 0;
    if (!bad && bound > 0) {
      if (bound >= kNoallocSlots) {
        if (threadIdx.x == 0) {
          raise_err(a.err, kErrTooLarge);
          atomicMax(&hdr->max_bound, (unsigned long long)bound);
        }
      } else {
        int64_t S = 32;
        while (S <= bound) S <<= 1;
        for (int64_t s = threadIdx.x; s < S; s += blockDim.x) tab[s] = kEmpty;
        __syncthreads();
        const uint32_t mask = (uint32_t)(S - 1);
        block_row_products<4, false, int32_t>(
            r0, r1, G, a.aci, (const int32_t *)nullptr, a.brp, a.bci, (const int32_t *)nullptr, (int32_t)a.k, a.err,
            Stage<int32_t>{s_ent, &s_next, s_wsum}, [&](int32_t c, int32_t, int32_t) {
              uint32_t h = hash_slot(c, mask);
              for (uint32_t probe = 0; probe <= mask; ++probe) {
                const int32_t old = atomicCAS(tab + h, kEmpty, c);
                if (old == kEmpty) {
                  ++cnt;
                  return;
                }
                if (old == c) return;
                h = (h + 1) & mask;
              }
              raise_err(a.err, kErrProbe);
            });
      }
    }
    long long total = block_sum((long long)cnt, red);
    if (threadIdx.x == 0) c_row_ptr[i + 1] = (int32_t)total;
    __syncthreads();
  }
}

// In-place scan: c_row_ptr[1..m] hold the row counts on entry and the
// inclusive prefix on exit; c_row_ptr[0] = 0.  One block.
__global__ void __launch_bounds__(1024) k_noalloc_scan(int32_t *c_row_ptr, int64_t m, unsigned char *scratch) {
  __shared__ long long red[33];
  NoallocHeader *hdr = reinterpret_cast<NoallocHeader *>(scratch);
  long long carry = 0;
  for (int64_t c0 = 0; c0 < m; c0 += blockDim.x) {
    const int64_t t = c0 + threadIdx.x;
    const long long v = t < m ? c_row_ptr[t + 1] : 0;
    long long tot;
    const long long ex = block_excl_scan(v, red, &tot);
    if (t < m) c_row_ptr[t + 1] = (int32_t)(carry + ex + v);
    carry += tot;
  }
  if (threadIdx.x == 0) {
    c_row_ptr[0] = 0;
    hdr->total = (unsigned long long)carry;
    if (carry > 2147483647LL) hdr->err |= kErrOverflow;
  }
}

}  // namespace sg

using namespace sg;

namespace {

std::mutex g_noalloc_mu;
unsigned char *g_noalloc_ptr[64];  // device address of the array, per device

// Once per device, with that device current: the device address of the
// scratch array.  In host code the symbol's name is only a host-side
// stand-in, so kernels are always given this address.
cudaError_t noalloc_setup(int dev, unsigned char **out) {
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

int bad_desc(const spgemm_csr *c) {
  if (!c || c->nrows < 0 || c->ncols < 0 || c->nnz < 0) return 1;
  if (c->nrows > INT32_MAX || c->ncols > INT32_MAX || c->nnz > INT32_MAX) return 1;
  if (!c->row_ptr || (c->nnz > 0 && !c->col_idx)) return 1;
  return 0;
}

}  // namespace

extern "C" {

int spgemm_symbolic_noalloc(const spgemm_csr *A, const spgemm_csr *B, int32_t *c_row_ptr, int64_t *nnz_c,
                            void *stream) {
  set_last_error("");
  if (bad_desc(A) || bad_desc(B) || A->ncols != B->nrows || !c_row_ptr || !nnz_c) return SPGEMM_ERR_INVALID_ARGUMENT;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  unsigned char *scratch = nullptr;
  if (e == cudaSuccess) e = noalloc_setup(dev, &scratch);
  if (e != cudaSuccess) {
    set_last_error(std::string("scratch setup: ") + cudaGetErrorString(e));
    return SPGEMM_ERR_DEVICE;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // the array keeps the previous call's contents: clear the counters
  e = cudaMemsetAsync(scratch, 0, kNoallocHeader, s);
  const int64_t m = A->nrows;
  const double avg_b = B->nrows > 0 ? (double)B->nnz / (double)B->nrows : 0.0;
  Args a{m, A->ncols, B->ncols, A->row_ptr, A->col_idx, B->row_ptr, B->col_idx, nullptr, nullptr,
         avg_b >= 24 ? 32 : avg_b >= 12 ? 16 : avg_b >= 6 ? 8 : 4,
         &reinterpret_cast<NoallocHeader *>(scratch)->err};
  if (e == cudaSuccess && m > 0) {
    k_noalloc_count<<<kNoallocBlocks, 1024, 0, s>>>(a, A->nnz, B->nnz, c_row_ptr, scratch);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_noalloc_scan<<<1, 1024, 0, s>>>(c_row_ptr, m, scratch);
    e = cudaGetLastError();
  }
  NoallocHeader h;
  std::memset(&h, 0, sizeof(h));
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, scratch, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return SPGEMM_ERR_DEVICE;
  }
  if (h.err & kErrTooLarge) {
    set_last_error("a row of C needs a hash table for " + std::to_string(h.max_bound) +
                      " keys; spgemm_symbolic_noalloc holds at most " + std::to_string(kNoallocSlots - 1) +
                      " keys per row");
    return SPGEMM_ERR_INVALID_ARGUMENT;
  }
  if (h.err & kErrCsr) {
    set_last_error("input CSR has an index out of range or a malformed row_ptr");
    return SPGEMM_ERR_INVALID_CSR;
  }
  if (h.err & kErrOverflow) {
    set_last_error("nnz(C) exceeds int32 indexing");
    return SPGEMM_ERR_INDEX_OVERFLOW;
  }
  if (h.err) {
    set_last_error("device-side check failed");
    return SPGEMM_ERR_DEVICE;
  }
  *nnz_c = (int64_t)h.total;
  return SPGEMM_OK;
}

}  // extern "C"
