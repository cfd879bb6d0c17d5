/*
 * spgemm.h - C ABI of the GB300 hash SpGEMM library (libspgemm_gb300.so).
 *
 * Computes C = A*B for sparse A (m x n) and B (n x k) in CSR form with
 * Gustavson's row-wise algorithm (paper Sec. 2, Fig. "RowWise_SpGEMM"):
 * row i of C accumulates a_ik * b_k* over the stored a_ik of row i of A,
 * in a hash table keyed by column index (Sec. 4.2.1).  The work runs in two
 * phases (the two-phase approach of Sec. 2; Sec. 4.2.1, Fig. "Hash_SpGEMM"):
 * a symbolic phase counts the entries of every output row so that C can be
 * allocated exactly, then a numeric phase computes the values.
 *
 * Call sequence:
 *     spgemm_plan_create   -> per-row flop count and row binning (Sec. 4.1)
 *     spgemm_symbolic      -> nnz per output row, C row_ptr, nnz(C) to host
 *     (caller allocates C col_idx and vals for nnz(C) entries)
 *     spgemm_numeric       -> C col_idx and vals, rows sorted if requested
 *     spgemm_plan_destroy
 * or the one-shot spgemm(), which takes a caller allocator, or spgemm_host()
 * for operands and result in host memory.
 *
 * Memory and ownership:
 *   - Every matrix pointer is a DEVICE pointer on the current CUDA device,
 *     except in spgemm_host(), whose operands and result are in host memory.
 *   - The caller owns A, B and all C buffers.  A plan borrows A and B: they
 *     must stay valid and unmodified until spgemm_numeric has completed on
 *     the plan's stream.
 *   - The plan owns its workspace (row flop, bins, row counts, heavy-row
 *     bitmaps and tables), allocated stream-ordered from the device's
 *     memory pool and released by spgemm_plan_destroy.
 *   - All device work is ordered on the stream given to spgemm_plan_create
 *     (a cudaStream_t passed as void*, NULL = legacy default stream).
 *   - spgemm_plan_create and spgemm_symbolic each synchronise that stream
 *     once, to read a few counters (bin sizes, nnz(C)) back to the host.
 *
 * Layout: CSR, 0-based, int32 row_ptr (nrows+1 entries) and col_idx.
 * Column indices inside an input row may be in any order (Table
 * "Summary of SpGEMM codes": Hash accepts any input order) and should be
 * distinct; a column repeated within a row is summed like separate entries.  Values are int64, float or double (spgemm_dtype); A, B and C
 * share one value type.  Output rows are column-sorted when flags has
 * SPGEMM_SORTED, otherwise their order is unspecified (Sec. 4.2.1 makes the
 * sort an optional last step of the numeric phase).
 *
 * Arithmetic: plus-times.  int64 wraps modulo 2^64.  Floating-point sums
 * are taken in an unspecified order (atomic accumulation), so results may
 * differ in the last bits between runs; every structural entry is stored,
 * including entries whose value sums to zero.
 *
 * Errors: every function returns an int status (spgemm_status); nothing
 * aborts or throws across this boundary.  The kernels check, as they read
 * them, that A's row_ptr is monotone within [0, nnz], that every column
 * index lies inside its matrix and that every touched row of B has a
 * monotone row_ptr; a violation skips the access and sets a device error
 * word.  That word (and any hash probe that ran past its table) is read
 * back at the plan's next host synchronisation: spgemm_plan_create,
 * spgemm_symbolic, or spgemm_plan_stats after spgemm_numeric.
 */
#ifndef SPGEMM_GB300_H
#define SPGEMM_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SPGEMM_API __attribute__((visibility("default")))
#else
#define SPGEMM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPGEMM_OK = 0,
    SPGEMM_ERR_INVALID_ARGUMENT = -1, /* null pointer, dims mismatch, bad dtype/flags, negative size */
    SPGEMM_ERR_INVALID_CSR = -2,      /* row_ptr not monotone or an index out of range (validated calls) */
    SPGEMM_ERR_OUT_OF_MEMORY = -3,    /* workspace allocation failed */
    SPGEMM_ERR_INDEX_OVERFLOW = -4,   /* nnz(C) does not fit int32 indexing */
    SPGEMM_ERR_BAD_STATE = -5,        /* calls out of order (numeric before symbolic, ...) */
    SPGEMM_ERR_DEVICE = -6,           /* CUDA error, or a device-side check failed */
    SPGEMM_ERR_TIMEOUT = -7           /* a bounded device-side wait gave up */
} spgemm_status;

typedef enum { SPGEMM_I64 = 0, SPGEMM_F32 = 1, SPGEMM_F64 = 2 } spgemm_dtype;

#define SPGEMM_UNSORTED 0u /* output columns in any order within a row */
#define SPGEMM_SORTED 1u   /* output columns ascending within each row */
#define SPGEMM_VALIDATE 2u /* accepted; the device checks listed under Errors always run */
#define SPGEMM_TIMING 4u   /* record CUDA events around every kernel (spgemm_plan_kernel_times) */
#define SPGEMM_SERIAL 8u   /* run the bins of a phase one after another on the plan's stream
                              (default: concurrently on side streams joined back to it) */
#define SPGEMM_HASH_LOW_BITS 64u /* hash slot = the low log2(size) bits of col * 2654435761, the remainder
                                    modulo the table size that Sec. 4.2.1 describes.  The default takes the
                                    top log2(size) bits instead (Fibonacci hashing): the low bits depend only
                                    on the column's low bits, which skewed (R-MAT) inputs share, and measured
                                    R-MAT A*A probes 2.75 slots per insert with them against 1.25.  The
                                    result is the same either way. */
#define SPGEMM_COUNT_PROBES 32u /* count hash-table probes and inserts (spgemm_stats::sym_probes etc.):
                                   the collision factor c of Eq. 2 is probes / inserts.  Adds global
                                   atomics to every hash insert: for measurement, not for timing. */
#define SPGEMM_PROBE_CHUNK4 16u /* hash tables probed 4 slots at a time: one 16-byte load reads the
                                   chunk holding the key's slot, a key is claimed in the chunk's first
                                   empty slot and the next chunk is tried only when this one is full
                                   (the GPU form of HashVector's chunked probing, Sec. 4.2.2); the
                                   default is one slot at a time (linear probing, Sec. 4.2.1).  The
                                   result is the same either way. */

/* A CSR operand (device pointers). */
typedef struct {
    int64_t nrows;
    int64_t ncols;
    int64_t nnz;
    const int32_t *row_ptr; /* nrows+1 entries, row_ptr[0] == 0, row_ptr[nrows] == nnz */
    const int32_t *col_idx; /* nnz entries in [0, ncols) */
    const void *vals;       /* nnz entries of the plan's value type */
} spgemm_csr;

/* Statistics of a plan (host struct, filled by spgemm_plan_stats). */
#define SPGEMM_MAX_BINS 24
typedef struct {
    int64_t m, n, k;           /* A is m x n, B is n x k */
    int64_t total_flop;        /* sum over rows of flop[i] (Sec. 4.1) */
    int64_t max_row_flop;      /* max over rows of flop[i] */
    int64_t nnz_c;             /* nnz(C), valid after spgemm_symbolic */
    int32_t n_sym_bins;        /* number of symbolic bins */
    int32_t n_num_bins;        /* number of numeric bins */
    int64_t sym_bin_rows[SPGEMM_MAX_BINS]; /* rows per symbolic bin */
    int64_t num_bin_rows[SPGEMM_MAX_BINS]; /* rows per numeric bin (bitmap bins: work items, a row per part) */
    int32_t sym_bin_table[SPGEMM_MAX_BINS]; /* table slots per bin (0 = bitmap or global table) */
    int32_t num_bin_table[SPGEMM_MAX_BINS];
    int64_t workspace_bytes;   /* device workspace currently held by the plan */
    int32_t kernel_launches;   /* kernels launched by this plan so far */
    int32_t state;             /* 0 planned, 1 symbolic done, 2 numeric done */
    int64_t sym_bin_flop[SPGEMM_MAX_BINS]; /* sum of flop[i] over the rows of each symbolic bin */
    int64_t num_bin_flop[SPGEMM_MAX_BINS]; /* same for numeric bins (bitmap bin: its rows, once) */
    int64_t sym_probes, sym_inserts;       /* hash-table slot reads (chunk reads under SPGEMM_PROBE_CHUNK4) and
                                              key insertions of the symbolic phase (SPGEMM_COUNT_PROBES only) */
    int64_t num_probes, num_inserts;       /* the same for the numeric phase */
    int64_t nnz_a_walked;      /* stored a_ik the phases walk: nnz(A), or fewer when the plan dropped the
                                  entries that select an empty row of B (fewer than half of A's were kept) */
    int64_t long_rows;         /* long rows of B whose bitmaps the symbolic bitmap rows OR in whole
                                  (spgemm_tuning::long_row_min) */
    int64_t long_entries;      /* their entries */
} spgemm_stats;

typedef struct spgemm_plan_s *spgemm_plan_t;

/*
 * Create a plan for C = A*B with value type `dtype` and `flags`
 * (SPGEMM_SORTED / SPGEMM_UNSORTED, optionally | SPGEMM_VALIDATE).
 * Runs the per-row flop pass, flop[i] = sum over stored a_ik of nnz(b_k*)
 * (Sec. 4.1, Fig. "RowsToThreads", step 1), and bins the rows by the hash
 * table size they need (GPU form of the load balancing of Sec. 4.1 and of
 * the density binning of GPU codes, Sec. 2).  Requires A->ncols ==
 * B->nrows.  Synchronises `stream` once.  On error *out is NULL.
 */
SPGEMM_API int spgemm_plan_create(spgemm_plan_t *out, const spgemm_csr *A, const spgemm_csr *B,
                       int dtype, unsigned flags, void *stream);

/*
 * Tuning of a plan's two main decisions (all zeros: the defaults).  The
 * result does not depend on them; only the time does.  The paper tunes its
 * recipe per input class (Sec. 4.2.4, Sec. 5.7); this is the GPU form.
 *   lanes_per_entry   G, the lanes that share one stored a_ik in the row
 *                     loop of the block kernels: 0 = chosen from the mean
 *                     B-row length flop/nnz(A) (>= 24: 32, >= 12: 16,
 *                     >= 6: 8, else 4); otherwise 4, 8, 16 or 32.
 *   bitmap_min_bound  rows whose symbolic bound min(flop_i, k) exceeds it
 *                     take the column-bitmap path (B with at most 2^18
 *                     columns): 0 = max(512, k/64); -1 = no bitmap rows;
 *                     otherwise a positive bound.
 *   max_nnz_c         the largest nnz(C) the plan accepts before
 *                     spgemm_symbolic returns SPGEMM_ERR_INDEX_OVERFLOW:
 *                     0 = 2^31-1 (int32 indexing); a smaller limit caps the
 *                     output memory of a product (and lets tests reach the
 *                     overflow path on small inputs).
 *   long_row_min      rows of B with at least this many entries are "long
 *                     rows": inside bitmap rows of A the symbolic phase ORs
 *                     their saved column bitmaps word by word instead of
 *                     setting one bit per product: 0 = max(512, k/128);
 *                     -1 = no long rows; otherwise a positive length.
 *   warp_load_pct     largest key bound of a warp hash table, in percent of
 *                     its slots (Sec. 4.2.1 sizes a table from the row's
 *                     bound; lower loads shorten probes): 0 = 50; else
 *                     5..95.
 *   block_load_pct    the same for block hash tables: 0 = 75; else 5..95.
 */
typedef struct {
    int32_t lanes_per_entry;
    int32_t reserved; /* must be 0 */
    int64_t bitmap_min_bound;
    int64_t max_nnz_c;
    int64_t long_row_min;
    int32_t warp_load_pct;
    int32_t block_load_pct;
} spgemm_tuning;

/* spgemm_plan_create with a tuning (NULL: the defaults).  Out-of-range
 * tuning values give SPGEMM_ERR_INVALID_ARGUMENT. */
SPGEMM_API int spgemm_plan_create_tuned(spgemm_plan_t *out, const spgemm_csr *A, const spgemm_csr *B, int dtype,
                                        unsigned flags, void *stream, const spgemm_tuning *tuning);

/*
 * Symbolic phase (Sec. 4.2.1: only keys, no values, go into the hash
 * table): counts the distinct columns of every output row, writes the
 * exclusive prefix sum to c_row_ptr (device, m+1 int32, caller-owned) and
 * returns nnz(C) in *nnz_c (host).  Synchronises the stream once.  Returns
 * SPGEMM_ERR_INDEX_OVERFLOW if nnz(C) > 2^31-1.
 */
SPGEMM_API int spgemm_symbolic(spgemm_plan_t plan, int32_t *c_row_ptr, int64_t *nnz_c);

/*
 * Numeric phase (Sec. 4.2.1; Fig. "Hash_SpGEMM", last step): accumulates
 * c_ij = sum_k a_ik*b_kj in per-row tables and stores every row at
 * c_row_ptr[i] .. c_row_ptr[i+1]-1 of c_col_idx (device, nnz(C) int32) and
 * c_vals (device, nnz(C) values), column-sorted when the plan has
 * SPGEMM_SORTED.  c_row_ptr must be the array filled by spgemm_symbolic.
 * Asynchronous: results are ready when the plan's stream reaches this point.
 * May be called again on the same plan, with the same or new output
 * buffers, after the VALUES of A and B changed: the row structure (row_ptr
 * and col_idx of A and B) must be unchanged, as in the repeated products of
 * multigrid setup.  The first call also prepares the structure-only work
 * (row grouping, heavy-row work items); later calls run only the kernels.
 */
SPGEMM_API int spgemm_numeric(spgemm_plan_t plan, const int32_t *c_row_ptr, int32_t *c_col_idx, void *c_vals);

/*
 * The numeric phase of rows row_begin .. row_end-1 of C only.  Rows of C
 * are independent (Fig. "RowWise_SpGEMM"), so calls over disjoint row
 * ranges that cover 0 .. m-1 give the result of one spgemm_numeric, and
 * each call writes nothing but its own rows' entries, c_row_ptr[row_begin]
 * .. c_row_ptr[row_end]-1 of c_col_idx and c_vals.  It lets a caller move
 * finished rows elsewhere (to the host, say) while later rows are computed.
 * Arguments, buffers, state and asynchrony as for spgemm_numeric; every
 * call launches the kernels of all bins, whose blocks skip the rows outside
 * the range.  SPGEMM_ERR_INVALID_ARGUMENT unless 0 <= row_begin <= row_end
 * <= m; an empty range does nothing.
 */
SPGEMM_API int spgemm_numeric_rows(spgemm_plan_t plan, int64_t row_begin, int64_t row_end, const int32_t *c_row_ptr,
                                   int32_t *c_col_idx, void *c_vals);

/*
 * The numeric phase as a CUDA graph.  The first call after a spgemm_numeric
 * on this plan captures the plan's numeric kernels (all bins, their side
 * streams and joins) for these output buffers and launches the graph; later
 * calls with the same buffers only launch it again, with one API call
 * instead of one per kernel.  New buffers capture a new graph.  Same rules
 * as a repeated spgemm_numeric: only the values of A and B may change.
 * Returns SPGEMM_ERR_BAD_STATE before the first spgemm_numeric, and
 * SPGEMM_ERR_INVALID_ARGUMENT for plans created with SPGEMM_TIMING (whose
 * per-kernel events cannot be timed inside a graph).
 */
SPGEMM_API int spgemm_numeric_graph(spgemm_plan_t plan, const int32_t *c_row_ptr, int32_t *c_col_idx, void *c_vals);

/* Release the plan and its workspace (stream-ordered).  NULL is accepted. */
SPGEMM_API int spgemm_plan_destroy(spgemm_plan_t plan);

/* Device workspace held by the plan, in bytes. */
SPGEMM_API int spgemm_plan_workspace_bytes(spgemm_plan_t plan, size_t *bytes);

/* Copy the plan's statistics into *out (host).  Synchronises the plan's
 * stream and returns the device error status of all work issued so far
 * (SPGEMM_OK, or the error the device checks recorded). */
SPGEMM_API int spgemm_plan_stats(spgemm_plan_t plan, spgemm_stats *out);

/* Time of every kernel the plan launched, summed by kernel name (plans
 * created with SPGEMM_TIMING only).  Synchronises the stream.  Writes at
 * most max_entries records and the number of distinct names to *n_out. */
typedef struct {
    char name[40];
    float ms;          /* summed CUDA-event time on the plan's stream */
    int32_t launches;  /* launches under this name */
} spgemm_kernel_time;
SPGEMM_API int spgemm_plan_kernel_times(spgemm_plan_t plan, spgemm_kernel_time *out, int max_entries, int *n_out);

/*
 * Inspection of the intermediate results, for tests: copy flop[m] (int64),
 * the symbolic row permutation perm[m] (int32; rows grouped by bin, bin b
 * occupying sym_bin_offsets[b]..sym_bin_offsets[b+1]-1) and nnz_row[m]
 * (int32, after spgemm_symbolic) into caller DEVICE buffers.
 * sym_bin_offsets is a HOST array of n_sym_bins+1 int64.
 */
SPGEMM_API int spgemm_plan_row_flop(spgemm_plan_t plan, int64_t *flop_out);
SPGEMM_API int spgemm_plan_sym_bins(spgemm_plan_t plan, int32_t *perm_out, int64_t *sym_bin_offsets);
SPGEMM_API int spgemm_plan_row_nnz(spgemm_plan_t plan, int32_t *nnz_out);

/* Allocator callback for spgemm(): returns a device pointer of `bytes`
 * bytes (16-byte aligned) or NULL.  The caller owns what it returns. */
typedef void *(*spgemm_alloc_fn)(size_t bytes, void *ctx);

/*
 * One-shot C = A*B: plan, symbolic, allocate C through `alloc`
 * (row_ptr: (m+1)*4 bytes, col_idx: nnz*4 bytes, vals: nnz*sizeof(value)),
 * numeric, destroy.  The three C pointers are returned through c_row_ptr,
 * c_col_idx and c_vals.  Results are ready when `stream` reaches the end
 * of the call's work.
 */
SPGEMM_API int spgemm(const spgemm_csr *A, const spgemm_csr *B, int dtype, unsigned flags, void *stream,
           spgemm_alloc_fn alloc, void *alloc_ctx,
           int32_t **c_row_ptr, int32_t **c_col_idx, void **c_vals, int64_t *nnz_c);

/*
 * Batched products C_p = A_p * B_p, p = 0 .. nprod-1, in one plan (batching
 * of independent products; the paper's products are single).  A and B are
 * HOST arrays of nprod device CSR descriptors.  The batch is packed on the
 * device into the block-diagonal product diag(A_p) * diag(B_p) (a copy of
 * the operands, owned by the batch) and runs with the launches and host
 * synchronisations of one product.
 *
 * spgemm_batch_create     packs, checks every product's indices
 *                         (SPGEMM_ERR_INVALID_CSR names none in particular),
 *                         runs the flop pass and binning; syncs `stream`.
 * spgemm_batch_symbolic   c_row_ptr (device, sum of nrows(A_p) + 1 int32)
 *                         receives the packed row pointers, *nnz_c the total,
 *                         row_off (host, nprod + 1, optional) the first row
 *                         of each product: product p owns rows
 *                         row_off[p] .. row_off[p+1]-1 and entries
 *                         c_row_ptr[row_off[p]] .. c_row_ptr[row_off[p+1]]-1.
 * spgemm_batch_numeric    columns (local to each product) and values.
 * spgemm_batch_plan       the underlying plan (statistics, timings).
 * Sizes of the packed batch must fit int32 indexing
 * (SPGEMM_ERR_INDEX_OVERFLOW otherwise).
 */
typedef struct spgemm_batch_s *spgemm_batch_t;
SPGEMM_API int spgemm_batch_create(spgemm_batch_t *out, int64_t nprod, const spgemm_csr *A, const spgemm_csr *B,
                                   int dtype, unsigned flags, void *stream);
/* spgemm_batch_create with a tuning for the batch's plan (NULL: defaults). */
SPGEMM_API int spgemm_batch_create_tuned(spgemm_batch_t *out, int64_t nprod, const spgemm_csr *A,
                                         const spgemm_csr *B, int dtype, unsigned flags, void *stream,
                                         const spgemm_tuning *tuning);
SPGEMM_API int spgemm_batch_symbolic(spgemm_batch_t batch, int32_t *c_row_ptr, int64_t *nnz_c, int64_t *row_off);
SPGEMM_API int spgemm_batch_numeric(spgemm_batch_t batch, const int32_t *c_row_ptr, int32_t *c_col_idx, void *c_vals);
SPGEMM_API spgemm_plan_t spgemm_batch_plan(spgemm_batch_t batch);
SPGEMM_API int spgemm_batch_destroy(spgemm_batch_t batch);

/*
 * Batched products in ONE CUDA graph launch.  The paper runs one product at
 * a time; balancing rows by flop over the workers (Sec. 4.1, Fig.
 * "RowsToThreads") is what this batched form applies across products: every
 * row of every product goes to the row bin its flop selects, and the bins
 * run over all products together.
 *
 * spgemm_bgraph_create plans the batch once: it splits the products into
 * waves of consecutive products whose C fits int32 indexing and `wave_nnz`
 * entries (0: 2^31-1), runs a planning pass (flop pass and symbolic phase,
 * host-synchronised) to size every workspace and a pool for each wave's C
 * (its nnz(C) times 1 + pool_slack), and captures, for every wave in order,
 * the packing of its operands, the flop pass, the symbolic kernels, the
 * row_ptr scan, the numeric kernels, the column unpacking and the copy of
 * the per-product counts to pinned host memory into one CUDA graph.  No
 * step of the graph reads a count on the host: the bin kernels find their
 * rows in device memory and walk them with grids sized to stay resident.
 * A and B are arrays of nprod device CSR descriptors, borrowed until
 * destroy; flags as for spgemm_plan_create without SPGEMM_TIMING and
 * SPGEMM_COUNT_PROBES; column bitmaps are not used (rows above the shared
 * tables use global-memory tables sized by the planning pass).
 *
 * spgemm_bgraph_launch enqueues the whole batch as one cudaGraphLaunch on
 * `stream`, recomputing every product from the operands' current contents.
 * spgemm_bgraph_wait synchronises that stream and returns the status:
 * SPGEMM_ERR_OUT_OF_MEMORY when a product no longer fits what was planned
 * (nothing is then written outside the pools), SPGEMM_ERR_INVALID_CSR for
 * malformed input.  spgemm_bgraph_product_nnz gives nnz(C_p) (host) and
 * spgemm_bgraph_product_copy copies C_p into caller buffers (device: m_p+1
 * row pointers from 0, nnz col_idx and values), stream-ordered on `stream`.
 * spgemm_bgraph_info reports the waves, the kernel nodes of the graph and
 * the device bytes held.  There are no waits on the device inside the
 * graph: its kernels follow each other in stream order.
 */
typedef struct spgemm_bgraph_s *spgemm_bgraph_t;
SPGEMM_API int spgemm_bgraph_create(spgemm_bgraph_t *out, int64_t nprod, const spgemm_csr *A, const spgemm_csr *B,
                                    int dtype, unsigned flags, void *stream, const spgemm_tuning *tuning,
                                    int64_t wave_nnz, double pool_slack);
SPGEMM_API int spgemm_bgraph_launch(spgemm_bgraph_t graph, void *stream);
SPGEMM_API int spgemm_bgraph_wait(spgemm_bgraph_t graph);
SPGEMM_API int spgemm_bgraph_product_nnz(spgemm_bgraph_t graph, int64_t p, int64_t *nnz);
SPGEMM_API int spgemm_bgraph_product_copy(spgemm_bgraph_t graph, int64_t p, int32_t *c_row_ptr, int32_t *c_col_idx,
                                          void *c_vals, void *stream);
SPGEMM_API int spgemm_bgraph_info(spgemm_bgraph_t graph, int64_t *waves, int64_t *kernel_nodes, int64_t *bytes);
SPGEMM_API int spgemm_bgraph_destroy(spgemm_bgraph_t graph);

/*
 * C = A*B with A, B and C in HOST memory, the copy of C to the host
 * overlapped with the computation.  The paper's products run on one
 * machine's memory and have no transfer step; this entry point serves
 * callers whose operands live in host memory.
 *
 * A and B describe host arrays (the same CSR layout as spgemm_csr; if the
 * descriptors point to the same arrays, B is copied once).  The memory
 * `host_alloc` returns for C must be host memory; page-locked memory
 * (cudaHostAlloc, cudaHostRegister) is needed for the copies to overlap,
 * and so it is for A and B.  `host_alloc` is called three times, after the
 * symbolic phase: row_ptr ((m+1)*4 bytes), col_idx (nnz*4) and vals
 * (nnz*sizeof(value)); the caller owns what it returns, also on error.
 *
 * The call copies A and B to the device and runs the flop pass and the
 * symbolic phase of the whole product (one plan), which give C's row
 * pointers and nnz(C); C is then allocated through `host_alloc`.  The rows
 * are split into `row_blocks` contiguous blocks by C's entries (the
 * partition of Sec. 4.1, Fig. "RowsToThreads", steps 1-2), the r-th block
 * to run taking a share proportional to 2^min(r, 6): the first block, whose
 * numeric phase no copy hides, is small, and each later block's numeric
 * phase fits under the copy of the block before it.  The blocks are cut
 * from the first row on or from the last row back, whichever gives the
 * first block more rows (more rows keep more of the GPU busy).  The
 * numeric phase runs block after block on `stream` (spgemm_numeric_rows)
 * while a second stream copies each finished block's columns and values to
 * the host, so the copy of block b overlaps the numeric phase of block b+1.  The result is the
 * same for every row_blocks.  row_blocks <= 0 picks a default (6 blocks
 * from 2^26 flop, else 1); it is capped at m.  flags as for
 * spgemm_plan_create, without SPGEMM_TIMING.
 *
 * Returns when C is complete in host memory.  The device memory it used is
 * released (stream-ordered on `stream`).  Errors as for spgemm(); on error
 * the pointers already allocated are returned and the rest are NULL.
 */
SPGEMM_API int spgemm_host(const spgemm_csr *A, const spgemm_csr *B, int dtype, unsigned flags, void *stream,
                           int row_blocks, spgemm_alloc_fn host_alloc, void *alloc_ctx, int32_t **c_row_ptr,
                           int32_t **c_col_idx, void **c_vals, int64_t *nnz_c);

/*
 * Symbolic phase for callers that cannot allocate device memory.  The paper
 * has no counterpart: this entry point exists for callers that must not
 * reach the CUDA allocator while they run (code inside an allocator or
 * memory-pool callback, a latency-bound loop that never calls into the
 * driver's allocator, a host whose device memory is owned by another
 * framework).
 *
 * Same result as spgemm_plan_create + spgemm_symbolic: c_row_ptr (device,
 * A->nrows+1 int32, caller-owned) receives the row pointers of C = A*B and
 * *nnz_c (host) receives nnz(C).  A and B are device CSR as for
 * spgemm_plan_create; their values are not read.  Work is ordered on
 * `stream`, which is synchronised once before the call returns.
 *
 * It allocates nothing: no cudaMalloc, no cudaFree, no allocating library
 * routine.  Its scratch is one static device array of 32 MiB + 256 bytes.
 * CUDA places it on a device when the library's module is first used there
 * (modules load lazily: at the first kernel launch of this library on that
 * device, or at this entry point's first call, which looks up the array's
 * device address), and it stays until the process exits.  So make the first
 * call on each device, or any other call of this library on it, before the
 * region in which the caller cannot allocate, and before any stream
 * capture.  The array holds 64 hash tables of 131072 keys; a row of C whose
 * key bound min(flop_i, ncols(B)) is 131072 or more is refused with
 * SPGEMM_ERR_INVALID_ARGUMENT and a message in spgemm_last_error().
 * Malformed CSR input (a column index outside its matrix, a bad row_ptr)
 * gives SPGEMM_ERR_INVALID_CSR; such rows are never hashed.
 *
 * Every call shares the array (the call clears the counters it needs):
 * calls that overlap on the GPU, from different streams or threads, race
 * and give wrong results.
 */
SPGEMM_API int spgemm_symbolic_noalloc(const spgemm_csr *A, const spgemm_csr *B, int32_t *c_row_ptr,
                                       int64_t *nnz_c, void *stream);

/* Human-readable name of a status code (static string). */
SPGEMM_API const char *spgemm_status_string(int status);

/* Last CUDA error text recorded by the library on this thread ("" if none). */
SPGEMM_API const char *spgemm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SPGEMM_GB300_H */
