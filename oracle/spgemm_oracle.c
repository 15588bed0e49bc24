/*
 * CPU oracle for the sparsity-aware 1D SpGEMM C = A*B.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file; only the test-suite, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header or constant with the CUDA path.
 *
 * Everything here is the plain definition, written for a reader to check by eye:
 *
 *   - Product (Section 2, problem statement): C = A*B, A is m x k, B is k x n,
 *     all in compressed sparse column (CSC) form.  Column j of C is
 *     C(:,j) = sum over stored b_kj of A(:,k) * b_kj  (column-by-column,
 *     Gustavson form; the paper's local multiply runs column by column,
 *     Section 3.1 and Algorithm 1).  Computed with a dense sparse accumulator
 *     (SPA) of length m.  A position (r, j) of C is structurally present iff
 *     at least one product a_rk * b_kj exists, even when the sum cancels to 0.
 *     Rows within each output column ascend.
 *   - Values: double (sum in ascending k, then ascending r) or the integer
 *     (+, x) semiring on 64-bit two's-complement words (wrapping).
 *   - For every double output entry the oracle also returns
 *     S_rj = sum |a_rk * b_kj|, the scale of the accuracy bound
 *     |c - c_ref| <= 1e-12 * S_rj.
 *   - Planning quantities of Algorithm 1 for one column block B_i
 *     (columns [c0, c1)):  H_i, the dense boolean of the nonzero rows of B_i
 *     (Table 1, Algorithm 1 step "store non-zero rows");  D~_i = H_i AND D with
 *     D the nonempty columns of A (Algorithm 1, "required columns");  the
 *     fetch-block choice of Algorithm 2 (a block of b consecutive column ids is
 *     chosen iff it contains a required column);  the gathered matrix A~_i that
 *     holds exactly the required columns (Algorithm 1, "create a new sparse
 *     matrix");  per output column the sparse flop count
 *     flops_j = sum over k in B(:,j) of nnz(A(:,k)) (Section 3.2, the inner
 *     product of column counts of A with row counts of B).
 *   - The local product C_i = A~_i * B_i (Algorithm 1, last step), where row k
 *     of B_i addresses column map[k] of A~_i.
 *
 * Parallelism: an optional OpenMP loop over output columns, each thread with
 * its own SPA.  No blocking, fusion or reordering of the arithmetic.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t nrows, ncols;
    const int64_t *colptr;   /* ncols + 1 */
    const int64_t *rowidx;   /* colptr[ncols] */
    const void *vals;        /* double or int64 (see the calling function) */
} orc_csc;

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Symbolic count: for each selected column j = cols[s], nnz_out[s] = number of
 * distinct rows r with some product a_rk*b_kj, flops_out[s] = number of products.
 */
int orc_count(const orc_csc *A, const orc_csc *B, const int64_t *cols, int64_t nsel,
              int64_t *nnz_out, int64_t *flops_out, int nthreads)
{
    if (A->ncols != B->nrows) return -1;
    const int64_t m = A->nrows;
    set_threads(nthreads);
    int bad = 0;
#pragma omp parallel
    {
        int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
        if (!mark) {
#pragma omp atomic write
            bad = 1;
        } else {
            for (int64_t r = 0; r < m; r++) mark[r] = -1;
#pragma omp for schedule(dynamic, 16)
            for (int64_t s = 0; s < nsel; s++) {
                int64_t j = cols[s], cnt = 0, fl = 0;
                for (int64_t p = B->colptr[j]; p < B->colptr[j + 1]; p++) {
                    int64_t k = B->rowidx[p];
                    for (int64_t q = A->colptr[k]; q < A->colptr[k + 1]; q++) {
                        int64_t r = A->rowidx[q];
                        fl++;
                        if (mark[r] != s) { mark[r] = s; cnt++; }
                    }
                }
                nnz_out[s] = cnt;
                flops_out[s] = fl;
            }
            free(mark);
        }
    }
    return bad ? -2 : 0;
}

/*
 * Numeric fill for the selected columns.  out_colptr has nsel + 1 entries and
 * must hold the exclusive prefix sum of the counts from orc_count.  vals_mode:
 * 0 = double (A->vals, B->vals are double; absum receives S_rj), 1 = int64
 * wrapping semiring (A->vals, B->vals are int64; absum may be NULL).
 */
int orc_fill(const orc_csc *A, const orc_csc *B, const int64_t *cols, int64_t nsel,
             const int64_t *out_colptr, int64_t *out_rowidx, void *out_vals,
             double *out_absum, int vals_mode, int nthreads)
{
    if (A->ncols != B->nrows) return -1;
    const int64_t m = A->nrows;
    set_threads(nthreads);
    int bad = 0;
#pragma omp parallel
    {
        int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
        double *accd = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
        uint64_t *acci = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1));
        double *sabs = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
        int64_t *list = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
        if (!mark || !accd || !acci || !sabs || !list) {
#pragma omp atomic write
            bad = 1;
        } else {
            for (int64_t r = 0; r < m; r++) mark[r] = -1;
#pragma omp for schedule(dynamic, 16)
            for (int64_t s = 0; s < nsel; s++) {
                int64_t j = cols[s], len = 0;
                for (int64_t p = B->colptr[j]; p < B->colptr[j + 1]; p++) {
                    int64_t k = B->rowidx[p];
                    for (int64_t q = A->colptr[k]; q < A->colptr[k + 1]; q++) {
                        int64_t r = A->rowidx[q];
                        if (mark[r] != s) {
                            mark[r] = s;
                            list[len++] = r;
                            accd[r] = 0.0; acci[r] = 0; sabs[r] = 0.0;
                        }
                        if (vals_mode == 0) {
                            double prod = ((const double *)A->vals)[q] * ((const double *)B->vals)[p];
                            accd[r] += prod;
                            sabs[r] += fabs(prod);
                        } else {
                            uint64_t a = (uint64_t)((const int64_t *)A->vals)[q];
                            uint64_t b = (uint64_t)((const int64_t *)B->vals)[p];
                            acci[r] += a * b;   /* unsigned: wraps modulo 2^64 */
                        }
                    }
                }
                qsort(list, (size_t)len, sizeof(int64_t), cmp_i64);
                int64_t base = out_colptr[s];
                if (out_colptr[s + 1] - base != len) {
#pragma omp atomic write
                    bad = 1;
                    continue;
                }
                for (int64_t t = 0; t < len; t++) {
                    int64_t r = list[t];
                    out_rowidx[base + t] = r;
                    if (vals_mode == 0) {
                        ((double *)out_vals)[base + t] = accd[r];
                        if (out_absum) out_absum[base + t] = sabs[r];
                    } else {
                        ((int64_t *)out_vals)[base + t] = (int64_t)acci[r];
                    }
                }
            }
        }
        free(mark); free(accd); free(acci); free(sabs); free(list);
    }
    return bad ? -2 : 0;
}

/*
 * Planning quantities of Algorithm 1 for one block B_i = B(:, c0:c1).
 *   H (k bytes):        H[h] = 1 iff row h of B_i holds a nonzero.
 *   dtilde (k entries): the ascending required column ids h with H[h] = 1
 *                       and nnz(A(:,h)) > 0; *n_dtilde receives their count.
 *   fetch (ceil(k/b)):  fetch[t] = 1 iff block t = [t*b, min((t+1)*b, k))
 *                       contains a required column (Algorithm 2: a group is
 *                       chosen as soon as one of its columns is hit).
 *   vol_exact / vol_block: nonzeros of A inside the required columns / inside
 *                       the chosen fetch blocks.
 */
int orc_plan_block(const orc_csc *A, const orc_csc *B, int64_t c0, int64_t c1, int64_t b,
                   uint8_t *H, int64_t *dtilde, int64_t *n_dtilde, uint8_t *fetch,
                   int64_t *vol_exact, int64_t *vol_block)
{
    const int64_t k = B->nrows;
    if (A->ncols != k || b <= 0 || c0 < 0 || c1 > B->ncols || c0 > c1) return -1;
    memset(H, 0, (size_t)k);
    for (int64_t j = c0; j < c1; j++)
        for (int64_t p = B->colptr[j]; p < B->colptr[j + 1]; p++)
            H[B->rowidx[p]] = 1;
    int64_t nd = 0, ve = 0, vb = 0;
    for (int64_t h = 0; h < k; h++)
        if (H[h] && A->colptr[h + 1] > A->colptr[h]) {
            dtilde[nd++] = h;
            ve += A->colptr[h + 1] - A->colptr[h];
        }
    int64_t nblk = (k + b - 1) / b;
    memset(fetch, 0, (size_t)nblk);
    for (int64_t s = 0; s < nd; s++) fetch[dtilde[s] / b] = 1;
    for (int64_t t = 0; t < nblk; t++)
        if (fetch[t]) {
            int64_t lo = t * b, hi = (t + 1) * b < k ? (t + 1) * b : k;
            vb += A->colptr[hi] - A->colptr[lo];
        }
    *n_dtilde = nd;
    *vol_exact = ve;
    *vol_block = vb;
    return 0;
}

/*
 * A~ = A(:, dtilde): column s of A~ is column dtilde[s] of A, copied whole.
 * out_colptr must have nd + 1 entries; out arrays must hold the exact volume.
 * elem_bytes is the size of one value (8 for double / int64).
 */
int orc_gather(const orc_csc *A, const int64_t *dtilde, int64_t nd, int64_t *out_colptr,
               int64_t *out_rowidx, void *out_vals, int elem_bytes)
{
    out_colptr[0] = 0;
    for (int64_t s = 0; s < nd; s++) {
        int64_t h = dtilde[s];
        int64_t lo = A->colptr[h], len = A->colptr[h + 1] - lo;
        memcpy(out_rowidx + out_colptr[s], A->rowidx + lo, sizeof(int64_t) * (size_t)len);
        memcpy((char *)out_vals + (size_t)out_colptr[s] * elem_bytes,
               (const char *)A->vals + (size_t)lo * elem_bytes, (size_t)len * elem_bytes);
        out_colptr[s + 1] = out_colptr[s] + len;
    }
    return 0;
}

/*
 * Per-column features of the products feeding column j (j in [c0, c1)):
 *   flops_j  = sum over k in B(:,j) of nnz(A(:,k))
 *   nnzb_j   = nnz(B(:,j))
 *   maxa_j   = max over k in B(:,j) of nnz(A(:,k))   (0 for an empty column)
 */
int orc_column_features(const orc_csc *A, const orc_csc *B, int64_t c0, int64_t c1,
                        int64_t *flops, int64_t *nnzb, int64_t *maxa)
{
    for (int64_t j = c0; j < c1; j++) {
        int64_t f = 0, mx = 0;
        for (int64_t p = B->colptr[j]; p < B->colptr[j + 1]; p++) {
            int64_t k = B->rowidx[p];
            int64_t len = A->colptr[k + 1] - A->colptr[k];
            f += len;
            if (len > mx) mx = len;
        }
        flops[j - c0] = f;
        nnzb[j - c0] = B->colptr[j + 1] - B->colptr[j];
        maxa[j - c0] = mx;
    }
    return 0;
}
