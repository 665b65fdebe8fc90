/*
 * Oracle for the SpMV / CG hot path of arXiv 2304.09511. TEST INFRASTRUCTURE
 * ONLY: loaded by the test suite, the smoke check and the benchmark's CPU
 * baseline, never by the product path. Shares nothing with the CUDA library.
 * Each function's paper passage is named beside its definition in oracle.c.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

enum { ORC_COO = 0, ORC_CSR = 1, ORC_DIA = 2 };
enum { ORC_F64 = 0, ORC_F32 = 1, ORC_BF16 = 2 };
enum { ORC_OK = 0, ORC_NOTCONV = 1, ORC_BREAKDOWN = 2 };

/* A matrix in one of the three formats; only the arrays of `fmt` are read. */
typedef struct {
    int32_t fmt;
    int32_t nrows, ncols;
    int64_t nnz;
    const int32_t* ai;    /* COO rows */
    const int32_t* aj;    /* COO / CSR columns */
    const int32_t* irp;   /* CSR row pointers, nrows + 1 */
    const double* av;     /* values: nnz (COO/CSR) or ndiags * npad (DIA) */
    int32_t ndiags;
    const int32_t* doff;  /* DIA offsets, ascending */
    int32_t npad;
} orc_matrix;

int64_t orc_coo_canonicalize(int32_t nrows, int32_t ncols, int64_t nnz,
                             const int32_t* rows, const int32_t* cols, const double* vals,
                             int32_t* out_rows, int32_t* out_cols, double* out_vals);
void orc_coo_to_csr(int32_t nrows, int64_t nnz, const int32_t* rows, int32_t* irp);
void orc_csr_to_coo(int32_t nrows, const int32_t* irp, int32_t* rows);
int32_t orc_dia_offsets(int32_t n, int64_t nnz, const int32_t* rows, const int32_t* cols,
                        int32_t* doff);
void orc_coo_to_dia(int32_t n, int64_t nnz, const int32_t* rows, const int32_t* cols,
                    const double* vals, int32_t ndiags, const int32_t* doff, int32_t npad,
                    double* av);
int64_t orc_dia_to_coo(int32_t n, int32_t ndiags, const int32_t* doff, int32_t npad,
                       const double* av, int32_t* rows, int32_t* cols, double* vals);
void orc_spmv_coo(int32_t nrows, int64_t nnz, const int32_t* ai, const int32_t* aj,
                  const double* av, const double* x, double* y);
void orc_spmv_csr(int32_t nrows, const int32_t* irp, const int32_t* aj, const double* av,
                  const double* x, double* y);
void orc_spmv_dia(int32_t n, int32_t ndiags, const int32_t* doff, int32_t npad,
                  const double* av, const double* x, double* y);
void orc_round_values(int64_t count, const double* in, int32_t value_type, double* out);
int32_t orc_cg(const orc_matrix* A, const double* b, double* x, double tol, int32_t maxit,
               int32_t* iters, double* relres, double* res_hist,
               const double* xstar, double* aerr_hist);
int32_t orc_cg_ir(const orc_matrix* A64, const orc_matrix* Alo, const double* b, double* x,
                  double tol, double inner_tol, int32_t max_outer, int32_t maxit_inner,
                  int32_t* outer_iters, int32_t* inner_iters_total, double* relres);
int32_t orc_threads(void);
int32_t orc_cg_ru(const orc_matrix* A64, const orc_matrix* Alo, const double* b, double* x,
                  double tol, double delta, int32_t max_updates, int32_t maxit,
                  int32_t* updates, int32_t* iters, double* relres);

#endif
