/*
 * Oracle for the SpMV / CG hot path of "Morpheus unleashed: Fast cross-platform
 * SpMV on emerging architectures" (arXiv 2304.09511).
 *
 * TEST INFRASTRUCTURE ONLY. This file is a plain, slow, obviously correct CPU
 * statement of what the method computes, in FP64, written so that it can be
 * checked against the paper by eye. Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product path never does.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Build: plain C11, no intrinsics, -ffp-contract=off so that every a*b+c is a
 * rounded multiply followed by a rounded add, exactly as the algorithms print it.
 *
 * What each function follows:
 *   orc_coo_canonicalize  COO storage (Sec. II-B-1). The paper puts no order on
 *                         COO; the canonical form sorts by (row, col), stable,
 *                         and sums duplicates in input order (a reading: the
 *                         paper fixes neither).
 *   orc_coo_to_csr        CSR row pointers (Sec. II-B-2): irp(i) = first entry of
 *                         row i, irp(nrows) = NNZ.
 *   orc_dia_offsets,
 *   orc_coo_to_dia        DIA storage (Sec. II-B-3): one column of AV per
 *                         diagonal, DOFF holds each diagonal's offset col-row,
 *                         out-of-matrix slots zero. Layout here is diagonal-major
 *                         AV[j*npad + i], npad = n rounded up to 32 (a reading:
 *                         the paper's SVE code indexes AV row-major).
 *   orc_dia_to_coo,
 *   orc_csr_to_coo        inverse maps, used by the round-trip pins.
 *   orc_spmv_coo          Algorithm 1, with y cleared first (a reading: the
 *                         printed += is taken as an overwrite of y).
 *   orc_spmv_csr          Algorithm 2.
 *   orc_spmv_dia          Algorithm 3 (bounds check 0 <= k < N).
 *   orc_round_values      storage rounding of matrix values to FP32 / BF16
 *                         (round to nearest, ties to even, from FP64).
 *   orc_cg                unpreconditioned conjugate gradient, the loop the
 *                         paper's HPCG validation runs with the preconditioner
 *                         disabled (Sec. VI, HPCG experiments), textbook form.
 *   orc_cg_ir             FP64 iterative refinement around an inner CG on the
 *                         low-precision matrix. Not in the paper: pinned step by
 *                         step by the dense stationary recursion
 *                         x += Alo^-1 (b - A64 x) and by its final FP64 residual.
 *   orc_cg_ru             one CG on the low-precision matrix whose residual is
 *                         replaced by the true FP64 residual b - A64 x at
 *                         "reliable updates" (Sleijpen and van der Vorst). Not in
 *                         the paper: pinned by finite termination, by reducing
 *                         to orc_cg when both matrices are equal and by its
 *                         final FP64 residual.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/* The CPU-baseline timing copy of this file is compiled with OpenMP: the row loops of the
 * CSR and DIA SpMV and the vector loops of orc_cg then run on all host cores, and dot
 * products become reductions (so their rounding order changes there). The parity build
 * has no OpenMP and these markers expand to nothing. */
#ifdef _OPENMP
#include <omp.h>
#define ORC_ROWS_PARALLEL _Pragma("omp parallel for schedule(static)")
#define ORC_SUM_PARALLEL _Pragma("omp parallel for schedule(static) reduction(+:s)")   /* sums into s */
#else
#define ORC_ROWS_PARALLEL
#define ORC_SUM_PARALLEL
#endif

/* Threads the timing copy uses (1 in the parity build). */
int32_t orc_threads(void) {
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* COO canonicalisation: stable merge sort on (row, col), then coalesce.      */
/* ------------------------------------------------------------------------- */

static int key_less(const int32_t* rows, const int32_t* cols, int64_t a, int64_t b) {
    if (rows[a] != rows[b]) return rows[a] < rows[b];
    return cols[a] < cols[b];
}

/* Top-down merge sort of the permutation perm[lo, hi). Ties keep the left
 * run's element first, so the sort is stable. */
static void merge_sort(int64_t* perm, int64_t* tmp, int64_t lo, int64_t hi,
                       const int32_t* rows, const int32_t* cols) {
    if (hi - lo < 2) return;
    int64_t mid = lo + (hi - lo) / 2;
    merge_sort(perm, tmp, lo, mid, rows, cols);
    merge_sort(perm, tmp, mid, hi, rows, cols);
    int64_t i = lo, j = mid, k = lo;
    while (i < mid && j < hi) {
        if (key_less(rows, cols, perm[j], perm[i])) tmp[k++] = perm[j++];
        else tmp[k++] = perm[i++];
    }
    while (i < mid) tmp[k++] = perm[i++];
    while (j < hi) tmp[k++] = perm[j++];
    for (k = lo; k < hi; k++) perm[k] = tmp[k];
}

int64_t orc_coo_canonicalize(int32_t nrows, int32_t ncols, int64_t nnz,
                             const int32_t* rows, const int32_t* cols, const double* vals,
                             int32_t* out_rows, int32_t* out_cols, double* out_vals) {
    if (nrows < 0 || ncols < 0 || nnz < 0) return -1;
    for (int64_t e = 0; e < nnz; e++) {
        if (rows[e] < 0 || rows[e] >= nrows || cols[e] < 0 || cols[e] >= ncols) return -1;
    }
    if (nnz == 0) return 0;
    int64_t* perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)nnz);
    int64_t* tmp = (int64_t*)malloc(sizeof(int64_t) * (size_t)nnz);
    if (!perm || !tmp) { free(perm); free(tmp); return -2; }
    for (int64_t e = 0; e < nnz; e++) perm[e] = e;
    merge_sort(perm, tmp, 0, nnz, rows, cols);

    int64_t out = 0;
    int64_t e = 0;
    while (e < nnz) {
        int64_t p = perm[e];
        double sum = vals[p];
        int64_t f = e + 1;
        /* equal keys are adjacent after sorting; they appear in input order */
        while (f < nnz && rows[perm[f]] == rows[p] && cols[perm[f]] == cols[p]) {
            sum = sum + vals[perm[f]];
            f++;
        }
        out_rows[out] = rows[p];
        out_cols[out] = cols[p];
        out_vals[out] = sum;
        out++;
        e = f;
    }
    free(perm);
    free(tmp);
    return out;
}

/* ------------------------------------------------------------------------- */
/* CSR (Sec. II-B-2)                                                          */
/* ------------------------------------------------------------------------- */

void orc_coo_to_csr(int32_t nrows, int64_t nnz, const int32_t* rows, int32_t* irp) {
    for (int32_t i = 0; i <= nrows; i++) irp[i] = 0;
    for (int64_t e = 0; e < nnz; e++) irp[rows[e] + 1] += 1;     /* row lengths */
    for (int32_t i = 0; i < nrows; i++) irp[i + 1] += irp[i];    /* running sum */
}

void orc_csr_to_coo(int32_t nrows, const int32_t* irp, int32_t* rows) {
    for (int32_t i = 0; i < nrows; i++)
        for (int32_t j = irp[i]; j < irp[i + 1]; j++) rows[j] = i;
}

/* ------------------------------------------------------------------------- */
/* DIA (Sec. II-B-3)                                                          */
/* ------------------------------------------------------------------------- */

int32_t orc_dia_offsets(int32_t n, int64_t nnz, const int32_t* rows, const int32_t* cols,
                        int32_t* doff) {
    if (n <= 0) return 0;
    /* offsets col-row range over -(n-1) .. n-1 */
    int64_t span = 2 * (int64_t)n - 1;
    unsigned char* seen = (unsigned char*)calloc((size_t)span, 1);
    if (!seen) return -2;
    for (int64_t e = 0; e < nnz; e++) seen[(int64_t)cols[e] - rows[e] + (n - 1)] = 1;
    int32_t nd = 0;
    for (int64_t k = 0; k < span; k++)
        if (seen[k]) doff[nd++] = (int32_t)(k - (n - 1));
    free(seen);
    return nd;
}

void orc_coo_to_dia(int32_t n, int64_t nnz, const int32_t* rows, const int32_t* cols,
                    const double* vals, int32_t ndiags, const int32_t* doff, int32_t npad,
                    double* av) {
    for (int64_t s = 0; s < (int64_t)ndiags * npad; s++) av[s] = 0.0;
    for (int64_t e = 0; e < nnz; e++) {
        int32_t off = cols[e] - rows[e];
        /* locate the diagonal by binary search in the ascending offset list */
        int32_t lo = 0, hi = ndiags - 1, j = -1;
        while (lo <= hi) {
            int32_t mid = lo + (hi - lo) / 2;
            if (doff[mid] == off) { j = mid; break; }
            if (doff[mid] < off) lo = mid + 1; else hi = mid - 1;
        }
        av[(int64_t)j * npad + rows[e]] = vals[e];
    }
    (void)n;
}

int64_t orc_dia_to_coo(int32_t n, int32_t ndiags, const int32_t* doff, int32_t npad,
                       const double* av, int32_t* rows, int32_t* cols, double* vals) {
    /* emit nonzero slots in (row, col) order; zero slots are padding */
    int64_t out = 0;
    for (int32_t i = 0; i < n; i++) {
        for (int32_t j = 0; j < ndiags; j++) {
            int64_t k = (int64_t)i + doff[j];
            if (k < 0 || k >= n) continue;
            double v = av[(int64_t)j * npad + i];
            if (v != 0.0) {
                rows[out] = i;
                cols[out] = (int32_t)k;
                vals[out] = v;
                out++;
            }
        }
    }
    return out;
}

/* ------------------------------------------------------------------------- */
/* SpMV: Algorithms 1-3                                                       */
/* ------------------------------------------------------------------------- */

void orc_spmv_coo(int32_t nrows, int64_t nnz, const int32_t* ai, const int32_t* aj,
                  const double* av, const double* x, double* y) {
    for (int32_t i = 0; i < nrows; i++) y[i] = 0.0;
    for (int64_t e = 0; e < nnz; e++) y[ai[e]] += av[e] * x[aj[e]];
}

void orc_spmv_csr(int32_t nrows, const int32_t* irp, const int32_t* aj, const double* av,
                  const double* x, double* y) {
    ORC_ROWS_PARALLEL
    for (int32_t i = 0; i < nrows; i++) {
        double sum = 0.0;
        for (int32_t j = irp[i]; j < irp[i + 1]; j++) sum += av[j] * x[aj[j]];
        y[i] = sum;
    }
}

void orc_spmv_dia(int32_t n, int32_t ndiags, const int32_t* doff, int32_t npad,
                  const double* av, const double* x, double* y) {
    ORC_ROWS_PARALLEL
    for (int32_t i = 0; i < n; i++) {
        double sum = 0.0;
        for (int32_t j = 0; j < ndiags; j++) {
            int64_t k = (int64_t)i + doff[j];
            if (k >= 0 && k < n) sum += av[(int64_t)j * npad + i] * x[k];
        }
        y[i] = sum;
    }
}

/* ------------------------------------------------------------------------- */
/* Storage rounding of matrix values (low-precision values, FP64 arithmetic)  */
/* ------------------------------------------------------------------------- */

/* FP64 -> BF16 value, round to nearest, ties to even, directly from FP64.
 * BF16 carries 8 significant bits and the FP32 exponent range, so a normal
 * value v = m * 2^e (0.5 <= |m| < 1) rounds to nearbyint(m * 2^8) * 2^(e-8);
 * below the smallest normal (2^-126) the quantum is fixed at 2^-133. */
static double round_bf16(double v) {
    if (v == 0.0 || isnan(v) || isinf(v)) return v;
    int e;
    double m = frexp(v, &e);
    double q;
    if (e - 1 >= -126) q = ldexp(nearbyint(ldexp(m, 8)), e - 8);
    else q = ldexp(nearbyint(ldexp(v, 133)), -133);
    if (fabs(q) >= ldexp(1.0, 128)) q = copysign(INFINITY, v);
    return q;
}

void orc_round_values(int64_t count, const double* in, int32_t value_type, double* out) {
    for (int64_t e = 0; e < count; e++) {
        if (value_type == ORC_F32) out[e] = (double)(float)in[e];
        else if (value_type == ORC_BF16) out[e] = round_bf16(in[e]);
        else out[e] = in[e];
    }
}

/* ------------------------------------------------------------------------- */
/* Conjugate gradient                                                         */
/* ------------------------------------------------------------------------- */

static void matvec(const orc_matrix* A, const double* x, double* y) {
    if (A->fmt == ORC_COO) orc_spmv_coo(A->nrows, A->nnz, A->ai, A->aj, A->av, x, y);
    else if (A->fmt == ORC_CSR) orc_spmv_csr(A->nrows, A->irp, A->aj, A->av, x, y);
    else orc_spmv_dia(A->nrows, A->ndiags, A->doff, A->npad, A->av, x, y);
}

static double dot(int32_t n, const double* u, const double* v) {
    double s = 0.0;
    ORC_SUM_PARALLEL
    for (int32_t i = 0; i < n; i++) s += u[i] * v[i];
    return s;
}

/* sqrt((u - w)^T A (u - w)), the A-norm of an error vector */
static double anorm_err(const orc_matrix* A, const double* u, const double* w, double* e, double* Ae) {
    int32_t n = A->nrows;
    for (int32_t i = 0; i < n; i++) e[i] = u[i] - w[i];
    matvec(A, e, Ae);
    double s = dot(n, e, Ae);
    return sqrt(s > 0.0 ? s : 0.0);
}

/* Textbook (Hestenes-Stiefel) CG on A x = b from the given x0:
 *   r0 = b - A x0, p0 = r0, rho0 = r0.r0
 *   per iteration: q = A p; alpha = rho / (p.q); x += alpha p; r -= alpha q;
 *                  rho' = r.r; stop when sqrt(rho') <= tol * ||b||;
 *                  beta = rho' / rho; p = r + beta p.
 * tol <= 0 runs exactly maxit iterations (stopping early only on rho' == 0).
 * ||b|| == 0 returns x = 0 after zero iterations. p.q <= 0 or a non-finite
 * alpha is a breakdown; x then holds the last completed iterate. */
int32_t orc_cg(const orc_matrix* A, const double* b, double* x, double tol, int32_t maxit,
               int32_t* iters, double* relres, double* res_hist,
               const double* xstar, double* aerr_hist) {
    int32_t n = A->nrows;
    double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* p = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* q = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* e = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int32_t status = ORC_OK;
    *iters = 0;
    *relres = 0.0;

    double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) {
        for (int32_t i = 0; i < n; i++) x[i] = 0.0;
        if (res_hist) res_hist[0] = 0.0;
        goto done;
    }
    matvec(A, x, q);
    ORC_ROWS_PARALLEL
    for (int32_t i = 0; i < n; i++) { r[i] = b[i] - q[i]; p[i] = r[i]; }
    double rho = dot(n, r, r);
    if (res_hist) res_hist[0] = sqrt(rho) / bnorm;
    if (xstar && aerr_hist) aerr_hist[0] = anorm_err(A, x, xstar, e, q);
    int converged = (sqrt(rho) <= tol * bnorm);
    int32_t k = 0;
    while (!converged && k < maxit) {
        matvec(A, p, q);
        double pq = dot(n, p, q);
        double alpha = rho / pq;
        if (!(pq > 0.0) || !isfinite(alpha)) { status = ORC_BREAKDOWN; break; }
        ORC_ROWS_PARALLEL
        for (int32_t i = 0; i < n; i++) x[i] = x[i] + alpha * p[i];
        ORC_ROWS_PARALLEL
        for (int32_t i = 0; i < n; i++) r[i] = r[i] - alpha * q[i];
        double rho_new = dot(n, r, r);
        k++;
        if (res_hist) res_hist[k] = sqrt(rho_new) / bnorm;
        if (xstar && aerr_hist) aerr_hist[k] = anorm_err(A, x, xstar, e, q);
        if (sqrt(rho_new) <= tol * bnorm) { rho = rho_new; converged = 1; break; }
        double beta = rho_new / rho;
        rho = rho_new;
        ORC_ROWS_PARALLEL
        for (int32_t i = 0; i < n; i++) p[i] = r[i] + beta * p[i];
    }
    *iters = k;
    *relres = sqrt(rho) / bnorm;
    if (status == ORC_OK && !converged && tol > 0.0) status = ORC_NOTCONV;
done:
    free(r); free(p); free(q); free(e);
    return status;
}

/* Iterative refinement (not in the paper): outer loop in FP64 on A64,
 *   r = b - A64 x; stop when ||r|| / ||b|| <= tol;
 *   inner CG on Alo d = r from d = 0 to relative tolerance inner_tol
 *   (at most maxit_inner iterations); x += d. */
int32_t orc_cg_ir(const orc_matrix* A64, const orc_matrix* Alo, const double* b, double* x,
                  double tol, double inner_tol, int32_t max_outer, int32_t maxit_inner,
                  int32_t* outer_iters, int32_t* inner_iters_total, double* relres) {
    int32_t n = A64->nrows;
    double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* d = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int32_t status = ORC_NOTCONV;
    *outer_iters = 0;
    *inner_iters_total = 0;
    *relres = 0.0;
    double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) {
        for (int32_t i = 0; i < n; i++) x[i] = 0.0;
        status = ORC_OK;
        goto done;
    }
    for (int32_t k = 0;; k++) {
        matvec(A64, x, r);
        for (int32_t i = 0; i < n; i++) r[i] = b[i] - r[i];
        double rel = sqrt(dot(n, r, r)) / bnorm;
        *relres = rel;
        *outer_iters = k;
        if (rel <= tol) { status = ORC_OK; break; }
        if (k == max_outer) { status = ORC_NOTCONV; break; }
        for (int32_t i = 0; i < n; i++) d[i] = 0.0;
        int32_t it = 0;
        double inner_rel = 0.0;
        int32_t st = orc_cg(Alo, r, d, inner_tol, maxit_inner, &it, &inner_rel, NULL, NULL, NULL);
        *inner_iters_total += it;
        if (st == ORC_BREAKDOWN) { status = ORC_BREAKDOWN; break; }
        for (int32_t i = 0; i < n; i++) x[i] = x[i] + d[i];
    }
done:
    free(r); free(d);
    return status;
}

/* Reliable updates (not in the paper). One CG runs on Alo throughout; x stays in
 * FP64 and the low-precision iteration accumulates its correction y:
 *   x from x0; r = b - A64 x; stop at once when ||r|| <= tol ||b||;
 *   y = 0; p = r; rho = r.r; rlast = ||r||
 *   per iteration: q = Alo p; alpha = rho / (p.q); y += alpha p; r -= alpha q;
 *     an update is due when ||r|| <= delta * rlast, ||r|| <= tol ||b|| or the
 *     iteration count reaches maxit; it does x += y; y = 0; r = b - A64 x;
 *     rlast = ||r||, and stops when ||r|| <= tol ||b|| (OK) or after max_updates
 *     updates or maxit iterations (NOTCONV);
 *     then (r being the recursive or the replaced residual)
 *     beta = r.r / rho; rho = r.r; p = r + beta p.
 * p.q <= 0 or a non-finite alpha is a breakdown (x then holds the last update).
 * updates counts the updates done; iters the iterations on Alo. */
int32_t orc_cg_ru(const orc_matrix* A64, const orc_matrix* Alo, const double* b, double* x,
                  double tol, double delta, int32_t max_updates, int32_t maxit,
                  int32_t* updates, int32_t* iters, double* relres) {
    int32_t n = A64->nrows;
    size_t sz = sizeof(double) * (size_t)(n > 0 ? n : 1);
    double* r = (double*)malloc(sz);
    double* p = (double*)malloc(sz);
    double* q = (double*)malloc(sz);
    double* y = (double*)malloc(sz);
    int32_t status = ORC_NOTCONV;
    int32_t k = 0;
    *updates = 0;
    *iters = 0;
    *relres = 0.0;
    double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) {
        for (int32_t i = 0; i < n; i++) x[i] = 0.0;
        status = ORC_OK;
        goto done;
    }
    matvec(A64, x, q);
    for (int32_t i = 0; i < n; i++) r[i] = b[i] - q[i];
    double rho = dot(n, r, r);
    double rlast = sqrt(rho);
    *relres = rlast / bnorm;
    if (rlast <= tol * bnorm) { status = ORC_OK; goto done; }
    for (int32_t i = 0; i < n; i++) { p[i] = r[i]; y[i] = 0.0; }
    for (;;) {
        if (k < maxit) {
            matvec(Alo, p, q);
            double pq = dot(n, p, q);
            double alpha = rho / pq;
            if (!(pq > 0.0) || !isfinite(alpha)) { status = ORC_BREAKDOWN; break; }
            for (int32_t i = 0; i < n; i++) y[i] = y[i] + alpha * p[i];
            for (int32_t i = 0; i < n; i++) r[i] = r[i] - alpha * q[i];
            k++;
        }
        double rr = dot(n, r, r);
        double rn = sqrt(rr);
        if (rn <= delta * rlast || rn <= tol * bnorm || k >= maxit) {
            for (int32_t i = 0; i < n; i++) { x[i] = x[i] + y[i]; y[i] = 0.0; }
            matvec(A64, x, q);
            for (int32_t i = 0; i < n; i++) r[i] = b[i] - q[i];
            rr = dot(n, r, r);
            rlast = sqrt(rr);
            *updates += 1;
            *relres = rlast / bnorm;
            if (rlast <= tol * bnorm) { status = ORC_OK; break; }
            if (*updates >= max_updates || k >= maxit) { status = ORC_NOTCONV; break; }
        }
        double beta = rr / rho;
        rho = rr;
        for (int32_t i = 0; i < n; i++) p[i] = r[i] + beta * p[i];
    }
    *iters = k;
done:
    free(r); free(p); free(q); free(y);
    return status;
}
