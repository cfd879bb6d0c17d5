/*
 * CPU oracle for row-wise SpGEMM C = A*B on CSR inputs.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file's library.  The GPU
 * library shares no code with it.
 *
 * What it computes (paper Sec. 2, Fig. "RowWise_SpGEMM"): for every row i
 * of A and every stored a_ik, every stored b_kj contributes a_ik*b_kj to
 * c_ij; c_ij is created on the first contribution and summed afterwards.
 * Every structural entry is kept, even one whose sum is zero, because the
 * method inserts on presence and never tests values.
 *
 * Accumulator: Gustavson's dense sparse accumulator (SPA, paper Sec. 2):
 * a dense value array over the k columns of B, a marker array telling
 * whether column j was touched in the current row, and the list of touched
 * columns.  The list is sorted ascending before a row is emitted, so the
 * oracle's output is always column-sorted.
 *
 * Row flop (paper Sec. 4.1, Fig. "RowsToThreads", step 1):
 *     flop[i] = sum over stored a_ik of nnz(b_k*).
 *
 * Multi-threaded variant (for timing only; identical results): rows are
 * split among threads by Fig. "RowsToThreads", step 2: a prefix sum of the
 * flop vector, then thread t starts at the first row whose prefix reaches
 * t * (total / nthreads) (the paper's lowbnd).
 *
 * Arithmetic: floating point in double (inputs of narrower types are
 * widened exactly by the caller), summed in stored order of A then B,
 * compiled without FMA contraction.  int64 values are summed as uint64, so
 * overflow wraps modulo 2^64.
 *
 * All functions return 0 on success and a negative number when an index
 * is out of range.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define ORACLE_BAD_INDEX (-2)
#define ORACLE_NO_MEMORY (-3)

/* flop[i] = sum_{j in row i of A} nnz(B row cols_A[j])  (Sec. 4.1). */
int oracle_row_flop(int64_t m, const int32_t *a_rp, const int32_t *a_ci,
                    int64_t n, const int32_t *b_rp, int64_t *flop)
{
    for (int64_t i = 0; i < m; ++i) {
        int64_t f = 0;
        for (int64_t j = a_rp[i]; j < a_rp[i + 1]; ++j) {
            int64_t kk = a_ci[j];
            if (kk < 0 || kk >= n) return ORACLE_BAD_INDEX;
            f += (int64_t)b_rp[kk + 1] - (int64_t)b_rp[kk];
        }
        flop[i] = f;
    }
    return 0;
}

static int cmp_i32(const void *x, const void *y)
{
    int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

/* Per-thread SPA state. */
typedef struct {
    int64_t *mark;   /* mark[j] == row id when column j is in the current row */
    double *acc;     /* dense FP accumulator */
    uint64_t *acci;  /* dense integer accumulator */
    double *absacc;  /* dense accumulator of |a_ik|*|b_kj| */
    int32_t *list;   /* touched columns of the current row */
} spa_t;

static int spa_init(spa_t *s, int64_t k, int want_fp, int want_int)
{
    memset(s, 0, sizeof(*s));
    size_t kk = (size_t)(k > 0 ? k : 1);
    s->mark = (int64_t *)malloc(kk * sizeof(int64_t));
    s->list = (int32_t *)malloc(kk * sizeof(int32_t));
    if (want_fp) {
        s->acc = (double *)malloc(kk * sizeof(double));
        s->absacc = (double *)malloc(kk * sizeof(double));
    }
    if (want_int) s->acci = (uint64_t *)malloc(kk * sizeof(uint64_t));
    if (!s->mark || !s->list || (want_fp && (!s->acc || !s->absacc)) || (want_int && !s->acci))
        return ORACLE_NO_MEMORY;
    for (size_t j = 0; j < kk; ++j) s->mark[j] = -1;
    return 0;
}

static void spa_free(spa_t *s)
{
    free(s->mark); free(s->list); free(s->acc); free(s->absacc); free(s->acci);
}

/* Symbolic: nnz of row i = number of distinct columns touched. */
static int row_symbolic(spa_t *s, int64_t i, const int32_t *a_rp, const int32_t *a_ci,
                        int64_t n, const int32_t *b_rp, const int32_t *b_ci, int64_t k,
                        int32_t *nnz_row)
{
    int64_t cnt = 0;
    for (int64_t ja = a_rp[i]; ja < a_rp[i + 1]; ++ja) {
        int64_t kk = a_ci[ja];
        if (kk < 0 || kk >= n) return ORACLE_BAD_INDEX;
        for (int64_t jb = b_rp[kk]; jb < b_rp[kk + 1]; ++jb) {
            int64_t j = b_ci[jb];
            if (j < 0 || j >= k) return ORACLE_BAD_INDEX;
            if (s->mark[j] != i) { s->mark[j] = i; ++cnt; }
        }
    }
    nnz_row[i] = (int32_t)cnt;
    return 0;
}

/* Numeric for one row, FP (double) or integer (uint64) values. */
static int row_numeric(spa_t *s, int64_t i, const int32_t *a_rp, const int32_t *a_ci,
                       const double *a_vf, const int64_t *a_vi, int64_t n, int64_t k,
                       const int32_t *b_rp, const int32_t *b_ci,
                       const double *b_vf, const int64_t *b_vi,
                       const int32_t *c_rp, int32_t *c_ci, double *c_vf, int64_t *c_vi,
                       double *c_abs)
{
    int64_t len = 0;
    for (int64_t ja = a_rp[i]; ja < a_rp[i + 1]; ++ja) {
        int64_t kk = a_ci[ja];
        if (kk < 0 || kk >= n) return ORACLE_BAD_INDEX;
        for (int64_t jb = b_rp[kk]; jb < b_rp[kk + 1]; ++jb) {
            int32_t j = b_ci[jb];
            if (j < 0 || j >= k) return ORACLE_BAD_INDEX;
            if (s->mark[j] != i) {              /* c_ij not yet in row: insert */
                s->mark[j] = i;
                s->list[len++] = j;
                if (a_vf) { s->acc[j] = 0.0; s->absacc[j] = 0.0; }
                else s->acci[j] = 0;
            }
            if (a_vf) {                          /* c_ij <- c_ij + a_ik * b_kj */
                double p = a_vf[ja] * b_vf[jb];
                s->acc[j] = s->acc[j] + p;
                s->absacc[j] = s->absacc[j] + (p < 0 ? -p : p);
            } else {
                s->acci[j] = s->acci[j] + (uint64_t)a_vi[ja] * (uint64_t)b_vi[jb];
            }
        }
    }
    if (len != (int64_t)c_rp[i + 1] - (int64_t)c_rp[i]) return ORACLE_BAD_INDEX;
    qsort(s->list, (size_t)len, sizeof(int32_t), cmp_i32);
    int64_t base = c_rp[i];
    for (int64_t t = 0; t < len; ++t) {
        int32_t j = s->list[t];
        c_ci[base + t] = j;
        if (a_vf) {
            c_vf[base + t] = s->acc[j];
            if (c_abs) c_abs[base + t] = s->absacc[j];
        } else {
            c_vi[base + t] = (int64_t)s->acci[j];
        }
    }
    return 0;
}

/* nnz_row[i] for rows [r0, r1). */
int oracle_symbolic_rows(int64_t r0, int64_t r1, const int32_t *a_rp, const int32_t *a_ci,
                         int64_t n, const int32_t *b_rp, const int32_t *b_ci, int64_t k,
                         int32_t *nnz_row)
{
    spa_t s;
    int rc = spa_init(&s, k, 0, 0);
    for (int64_t i = r0; rc == 0 && i < r1; ++i)
        rc = row_symbolic(&s, i, a_rp, a_ci, n, b_rp, b_ci, k, nnz_row);
    spa_free(&s);
    return rc;
}

/* Numeric phase for rows [r0, r1) into caller buffers laid out by c_rp (FP). */
int oracle_numeric_rows_f64(int64_t r0, int64_t r1,
                            const int32_t *a_rp, const int32_t *a_ci, const double *a_v, int64_t n,
                            const int32_t *b_rp, const int32_t *b_ci, const double *b_v, int64_t k,
                            const int32_t *c_rp, int32_t *c_ci, double *c_v, double *c_abs)
{
    spa_t s;
    int rc = spa_init(&s, k, 1, 0);
    for (int64_t i = r0; rc == 0 && i < r1; ++i)
        rc = row_numeric(&s, i, a_rp, a_ci, a_v, NULL, n, k, b_rp, b_ci, b_v, NULL, c_rp, c_ci, c_v, NULL, c_abs);
    spa_free(&s);
    return rc;
}

/* Numeric phase for rows [r0, r1), int64 values (wrapping). */
int oracle_numeric_rows_i64(int64_t r0, int64_t r1,
                            const int32_t *a_rp, const int32_t *a_ci, const int64_t *a_v, int64_t n,
                            const int32_t *b_rp, const int32_t *b_ci, const int64_t *b_v, int64_t k,
                            const int32_t *c_rp, int32_t *c_ci, int64_t *c_v)
{
    spa_t s;
    int rc = spa_init(&s, k, 0, 1);
    for (int64_t i = r0; rc == 0 && i < r1; ++i)
        rc = row_numeric(&s, i, a_rp, a_ci, NULL, a_v, n, k, b_rp, b_ci, NULL, b_v, c_rp, c_ci, NULL, c_v, NULL);
    spa_free(&s);
    return rc;
}

/* ---------------- RowsToThreads partition (Sec. 4.1, step 2) ---------------- */

/* offset[0..t] from the flop vector: inclusive prefix sum, then thread tid
 * starts at the first row whose prefix is >= tid * average (lowbnd). */
int oracle_rows_to_threads(int64_t m, const int64_t *flop, int64_t t, int64_t *offset)
{
    int64_t *ps = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));
    if (!ps) return ORACLE_NO_MEMORY;
    ps[0] = 0;
    for (int64_t i = 0; i < m; ++i) ps[i + 1] = ps[i] + flop[i];
    double ave = (double)ps[m] / (double)t;
    offset[0] = 0;
    for (int64_t tid = 1; tid < t; ++tid) {
        double target = ave * (double)tid;
        /* lowbnd: smallest id with ps[id] >= target, searched over ps[0..m]. */
        int64_t lo = 0, hi = m;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if ((double)ps[mid] >= target) hi = mid; else lo = mid + 1;
        }
        offset[tid] = lo;
    }
    offset[t] = m;
    free(ps);
    return 0;
}

typedef struct {
    int64_t r0, r1;
    int phase; /* 0 symbolic, 1 numeric f64, 2 numeric i64 */
    const int32_t *a_rp, *a_ci, *b_rp, *b_ci, *c_rp;
    const void *a_v, *b_v;
    int64_t n, k;
    int32_t *nnz_row, *c_ci;
    void *c_v;
    double *c_abs;
    int rc;
} job_t;

static void *run_job(void *p)
{
    job_t *j = (job_t *)p;
    if (j->phase == 0)
        j->rc = oracle_symbolic_rows(j->r0, j->r1, j->a_rp, j->a_ci, j->n, j->b_rp, j->b_ci, j->k, j->nnz_row);
    else if (j->phase == 1)
        j->rc = oracle_numeric_rows_f64(j->r0, j->r1, j->a_rp, j->a_ci, (const double *)j->a_v, j->n, j->b_rp, j->b_ci,
                                        (const double *)j->b_v, j->k, j->c_rp, j->c_ci, (double *)j->c_v, j->c_abs);
    else
        j->rc = oracle_numeric_rows_i64(j->r0, j->r1, j->a_rp, j->a_ci, (const int64_t *)j->a_v, j->n, j->b_rp, j->b_ci,
                                        (const int64_t *)j->b_v, j->k, j->c_rp, j->c_ci, (int64_t *)j->c_v);
    return NULL;
}

/* Runs one phase over all rows with nthreads threads split by offset[]. */
int oracle_phase_mt(int phase, int64_t nthreads, const int64_t *offset,
                    const int32_t *a_rp, const int32_t *a_ci, const void *a_v,
                    int64_t n, const int32_t *b_rp, const int32_t *b_ci, const void *b_v, int64_t k,
                    int32_t *nnz_row, const int32_t *c_rp, int32_t *c_ci, void *c_v, double *c_abs)
{
    if (nthreads < 1) return ORACLE_BAD_INDEX;
    job_t *jobs = (job_t *)calloc((size_t)nthreads, sizeof(job_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return ORACLE_NO_MEMORY; }
    for (int64_t t = 0; t < nthreads; ++t) {
        job_t *j = &jobs[t];
        j->r0 = offset[t]; j->r1 = offset[t + 1]; j->phase = phase;
        j->a_rp = a_rp; j->a_ci = a_ci; j->a_v = a_v; j->n = n;
        j->b_rp = b_rp; j->b_ci = b_ci; j->b_v = b_v; j->k = k;
        j->nnz_row = nnz_row; j->c_rp = c_rp; j->c_ci = c_ci; j->c_v = c_v; j->c_abs = c_abs;
    }
    for (int64_t t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, run_job, &jobs[t]);
    run_job(&jobs[0]);
    int rc = jobs[0].rc;
    for (int64_t t = 1; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        if (jobs[t].rc != 0) rc = jobs[t].rc;
    }
    free(jobs); free(th);
    return rc;
}
