/*
 * mspv — sparse matrix-vector multiply and conjugate gradient on GB300 (sm_103a).
 *
 * C ABI of libmspv.so. The operations follow the problem statement of
 * "Morpheus unleashed: Fast cross-platform SpMV on emerging architectures"
 * (arXiv 2304.09511): a sparse matrix held in one of the three storage formats of
 * Sec. II-B (COO, CSR, DIA), the SpMV of Algorithms 1-3, and the unpreconditioned
 * conjugate-gradient loop the paper runs in its HPCG experiments (Sec. VI, with the
 * preconditioner disabled). The handle lifecycle mirrors the create -> optimise ->
 * execute -> destroy sequence the paper describes for vendor sparse handles
 * (Sec. III): mspv_create_coo / mspv_convert / mspv_spmv / mspv_destroy.
 *
 * Conventions (every entry point):
 *  - Indices are 0-based int32. nnz is int64 but must stay below 2^31.
 *  - Matrix values are given in FP64. A handle may store them as FP64, FP32 or
 *    BF16 (mspv_value_type); arithmetic inside SpMV is always FP64 (values are
 *    widened exactly before each multiply-add).
 *  - Vectors passed to mspv_spmv / mspv_cg_* are DEVICE pointers to FP64 arrays,
 *    owned by the caller, which must stay valid until the stream work completes.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream. mspv_spmv is asynchronous on that stream. mspv_create_coo,
 *    mspv_convert, mspv_export and the CG solvers synchronise the stream before
 *    they return.
 *  - Handles own device copies of everything they hold (inputs are copied in,
 *    never aliased). A handle must not be used by two calls that overlap in time.
 *  - No C++ exception crosses this boundary. Every call returns a status; the
 *    calling thread's last error message is kept for mspv_last_error().
 *  - Device faults are never used to signal errors: bounds, sizes and numerical
 *    breakdown are detected and returned as statuses.
 */
#ifndef MSPV_H
#define MSPV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define MSPV_API __attribute__((visibility("default")))
#else
#define MSPV_API
#endif

typedef struct mspv_matrix* mspv_matrix_t;

/* Storage formats of Sec. II-B. */
typedef enum { MSPV_COO = 0, MSPV_CSR = 1, MSPV_DIA = 2 } mspv_format;

/* Storage type of matrix values; accumulation is always FP64. */
typedef enum { MSPV_F64 = 0, MSPV_F32 = 1, MSPV_BF16 = 2 } mspv_value_type;

typedef enum {
    MSPV_OK = 0,
    MSPV_EINVAL = 1,      /* bad argument: null pointer, negative size, index out of range */
    MSPV_ENOMEM = 2,      /* device allocation failed or exceeded MSPV_MAX_BYTES */
    MSPV_ETOOBIG = 3,     /* DIA storage would exceed its fill cap or 2^31 - 1 padded rows, or nnz >= 2^31 */
    MSPV_EFORMAT = 4,     /* operation not defined for this format (e.g. DIA of a non-square matrix) */
    MSPV_ECUDA = 5,       /* a CUDA runtime call failed; see mspv_last_error() */
    MSPV_ENOTCONV = 6,    /* CG reached its iteration limit above the tolerance */
    MSPV_EBREAKDOWN = 7   /* CG found p.Ap <= 0 or a non-finite step (matrix not SPD) */
} mspv_status;

/* Description of a handle, filled by mspv_info. */
typedef struct {
    int32_t format;          /* mspv_format */
    int32_t value_type;      /* mspv_value_type */
    int32_t nrows, ncols;
    int64_t nnz;             /* stored entries (COO/CSR); for DIA the entries it was built from */
    int32_t ndiags;          /* DIA: number of stored diagonals, else 0 */
    int32_t npad;            /* DIA: padded row count of each diagonal (multiple of 32), else 0 */
    int32_t csr_vector;      /* CSR: lanes per row (1..32), or 0 for the staged kernels */
    int32_t row_max;         /* longest row */
    double row_mean;         /* mean row length */
    double row_std;          /* standard deviation of row lengths */
    int64_t empty_rows;      /* rows with no stored entry */
    int64_t device_bytes;    /* device memory the handle holds */
} mspv_matrix_info;

/*
 * Create a COO handle from triplets (Sec. II-B-1: arrays AI, AJ, AV of length NNZ,
 * in no particular order). rows/cols/vals are host pointers when on_device == 0,
 * device pointers otherwise; they are read, never kept. The handle stores the
 * canonical form: entries sorted by (row, col), stable, with duplicate (row, col)
 * pairs summed in input order; explicit zeros are kept.
 * Errors: EINVAL for nrows/ncols/nnz < 0, null arrays with nnz > 0, or any index
 * outside [0, nrows) x [0, ncols); ETOOBIG for nnz >= 2^31; ENOMEM; ECUDA.
 * On error *out is set to NULL.
 */
MSPV_API mspv_status mspv_create_coo(int32_t nrows, int32_t ncols, int64_t nnz,
                                     const int32_t* rows, const int32_t* cols,
                                     const double* vals, int on_device, void* stream,
                                     mspv_matrix_t* out);

/*
 * Build a new handle holding A in format `format` with values stored as
 * `value_type` (rounded to nearest even from FP64). A is not modified.
 *  - CSR (Sec. II-B-2): IRP[nrows + 1] = exclusive scan of the row lengths, AJ and
 *    AV in canonical order.
 *  - DIA (Sec. II-B-3): DOFF = ascending distinct offsets col - row; AV is stored
 *    diagonal-major, AV[j * npad + i] multiplying x[i + DOFF[j]], with
 *    npad = ceil(nrows / 32) * 32 and zeros in every slot outside the matrix or
 *    without an entry. Square matrices only (EFORMAT otherwise). ETOOBIG when
 *    ndiags * npad exceeds max(32 * nnz, 2^20) slots (DIA's storage blow-up on
 *    scattered patterns), or the MSPV_DIA_MAX_FILL override of the factor 32, and when npad
 *    would exceed 2^31 - 1 (nrows > 2^31 - 32).
 *  - COO: a copy, possibly with another value type.
 * A may be COO or CSR; converting from DIA returns EFORMAT.
 */
MSPV_API mspv_status mspv_convert(mspv_matrix_t A, mspv_format format,
                                  mspv_value_type value_type, void* stream,
                                  mspv_matrix_t* out);

/*
 * y = A x (overwrite), by Algorithm 1 (COO), 2 (CSR) or 3 (DIA) for A's format.
 * x has ncols entries, y has nrows entries; both are device FP64 arrays and must
 * not overlap. Rows without entries get y = 0. Asynchronous on `stream`.
 * Summation order inside a row differs from the sequential order of the
 * algorithms (FP64 fused multiply-adds and tree reductions); results agree with
 * the sequential sum within 2 (k + 2) u sum_j |a_ij x_j| for a row of k entries.
 * Repeated calls on the same inputs give bit-identical y.
 */
MSPV_API mspv_status mspv_spmv(mspv_matrix_t A, const double* x, double* y, void* stream);

/*
 * Unpreconditioned conjugate gradient on A x = b (A square, assumed SPD), started
 * from the x passed in and overwritten with the result:
 *   r = b - A x, p = r, rho = r.r; per iteration q = A p, alpha = rho / p.q,
 *   x += alpha p, r -= alpha q, rho' = r.r; stop when sqrt(rho') <= tol ||b||_2;
 *   beta = rho' / rho, p = r + beta p.
 * tol <= 0 runs exactly maxit iterations (earlier only if r becomes exactly 0)
 * and returns OK. ||b|| = 0 sets x = 0 with zero iterations.
 * Outputs (host pointers, may be NULL): *iters = iterations done, *relres =
 * sqrt(rho) / ||b|| (the recursively updated residual).
 * Returns OK, ENOTCONV (maxit reached with tol > 0; x holds the last iterate) or
 * EBREAKDOWN (p.q <= 0 or non-finite alpha; x holds the last completed iterate).
 * Vector work runs on the device with device-resident scalars (||b|| = 0 included); the
 * host launches batches of MSPV_CG_CHECK_EVERY iterations (default 10; with tol <= 0, a
 * fixed count, up to 256 unless that variable is set) and reads the convergence flag after
 * each batch; launches past convergence are no-ops, so results do not depend on that
 * interval. The call returns once the solve has ended (it synchronises the stream).
 * Workspace (3 vectors + reduction partials) is allocated once per handle.
 */
MSPV_API mspv_status mspv_cg_solve(mspv_matrix_t A, const double* b, double* x, double tol,
                                   int32_t maxit, void* stream, int32_t* iters,
                                   double* relres);

/*
 * Mixed-precision CG with iterative refinement (not in the paper). A64 and Alo hold
 * the same matrix; Alo typically stores FP32 or BF16 values (any format). Outer loop
 * in FP64 on A64: r = b - A64 x; stop when ||r|| / ||b|| <= tol; otherwise solve
 * Alo d = r approximately from d = 0 to relative tolerance inner_tol (at most
 * maxit_inner iterations), then x += d. At most max_outer corrections.
 * inner_fp32 = 0: the inner CG is mspv_cg_solve's FP64 iteration on Alo (values widened
 *   exactly, FP64 FMAs and vectors).
 * inner_fp32 = 1: the inner CG runs in FP32 arithmetic (FP32 vectors and FMAs) on the
 *   unit-norm right-hand side r / ||r||, with alpha, beta, rho and the cross-CTA sums of
 *   every dot product kept in FP64; x += ||r|| d in FP64. Alo must store FP32 or BF16
 *   values (EFORMAT otherwise). On GB300, whose FP64 pipe is ~1/64 of its FP32 pipe,
 *   this is the mode that makes refinement faster than plain FP64 CG.
 * inner_fp32 = 2: reliable updates instead of restarts. One FP32-arithmetic CG on Alo
 *   (scalars in FP64, as for 1) runs throughout and accumulates a correction y; x and
 *   the residual stay in FP64. When its recursive residual has fallen by the factor
 *   inner_tol since the last update, or to tol ||b||, the update does x += y, r = b -
 *   A64 x in FP64, stops when ||r|| / ||b|| <= tol, and otherwise continues the same CG
 *   from the replaced residual with p = r + beta p, beta = ||r||^2 / (r.r before the
 *   last iteration), so the search direction is kept (Sleijpen and van der Vorst's
 *   reliable updated residuals). inner_tol <= 0 selects 1e-2 for FP32 values and 1e-1
 *   for BF16 values. max_outer bounds the updates and maxit_inner the total FP32
 *   iterations; *outer_iters returns the updates and *inner_iters the FP32 iterations.
 *   With FP32 values this needs about as many iterations as FP64 CG.
 * inner_fp32 outside 0..2 is EINVAL.
 * Outputs (host, may be NULL): *outer_iters, *inner_iters (sum over corrections),
 * *relres = final ||b - A64 x|| / ||b||. Returns OK, ENOTCONV or EBREAKDOWN.
 */
MSPV_API mspv_status mspv_cg_solve_ir(mspv_matrix_t A64, mspv_matrix_t Alo, const double* b,
                                      double* x, double tol, double inner_tol,
                                      int32_t max_outer, int32_t maxit_inner, int32_t inner_fp32,
                                      void* stream, int32_t* outer_iters, int32_t* inner_iters,
                                      double* relres);

/*
 * COO SpMV y = A x that allocates no device memory (the paper has no counterpart; this
 * is a library convenience). For callers that cannot call cudaMalloc: applications
 * whose device memory is reserved up front or strictly budgeted by their own
 * allocator (for example a framework's caching allocator holding the free memory),
 * where one more allocation would fail or break the budget.
 * rows/cols/vals are DEVICE arrays of nnz triplets with row indices non-decreasing
 * (any column order, duplicates allowed: they are summed); x has ncols and y nrows
 * device FP64 entries. The per-window scratch of the COO kernel lives in a fixed
 * 1.5 MiB device array compiled into the library, present on every GPU that loads it
 * until the process exits; nnz above 201,326,592 (65,536 windows of 3,072 entries)
 * returns ETOOBIG. EINVAL for an index outside the shape or decreasing rows (checked on
 * the device; the call synchronises `stream` once to read the check). The first call on
 * a device looks up the array's device address (call it once before any stream
 * capture) and keeps it for the life of the process: after cudaDeviceReset, which unloads
 * the library's device code, this entry point must not be called again in that process.
 * All calls share the array: calls that overlap on the GPU race on it.
 */
MSPV_API mspv_status mspv_spmv_coo_noalloc(int32_t nrows, int32_t ncols, int64_t nnz,
                                           const int32_t* rows, const int32_t* cols,
                                           const double* vals, const double* x, double* y,
                                           void* stream);

/*
 * y = A x in FP32 arithmetic (the inner SpMV of mspv_cg_solve_ir with inner_fp32 = 1): A stores
 * FP32 or BF16 values (EFORMAT for FP64 values), x (ncols) and y (nrows) are DEVICE FP32 arrays,
 * both 16-byte aligned (EINVAL otherwise), x and y must not overlap. Products and sums in FP32
 * (BF16 values widened exactly). Asynchronous on `stream`.
 */
MSPV_API mspv_status mspv_spmv_f32(mspv_matrix_t A, const float* x, float* y, void* stream);

/*
 * y += A x: the accumulating form of mspv_spmv (same arguments, layouts and errors). Rows of A
 * without entries leave y unchanged. With mspv_split_columns it forms y = A_local x_local +
 * A_remote x_remote, one call per part.
 */
MSPV_API mspv_status mspv_spmv_add(mspv_matrix_t A, const double* x, double* y, void* stream);

/*
 * Local/remote split (the paper's distributed HPCG, Sec. VI: each process's matrix is split
 * into a structured local part and an unstructured remote part so that each can take its own
 * format). For a COO or CSR handle A (nrows x ncols) and 0 <= ncols_local <= ncols, *local
 * receives the entries with column < ncols_local (nrows x ncols_local) and *remote those with
 * column >= ncols_local, renumbered from 0 (nrows x (ncols - ncols_local)); both are new
 * canonical COO handles with A's value type, to be converted and destroyed independently.
 * A x = local x[0:ncols_local] + remote x[ncols_local:]. EFORMAT for a DIA handle, EINVAL for
 * ncols_local outside [0, ncols]. Synchronous.
 */
MSPV_API mspv_status mspv_split_columns(mspv_matrix_t A, int32_t ncols_local, void* stream,
                                        mspv_matrix_t* local, mspv_matrix_t* remote);

/*
 * ---- Format selection ----
 * The paper's distributed HPCG chooses each process's format with a run-first auto-tuner
 * (Sec. VI: time every format, keep the fastest), and its related work cites learned
 * selectors (Sec. VII). mspv_tune_format is the run-first tuner; the features and the
 * small FP32 MLP below are a learned selector trained on its labels, so that a format
 * can be chosen without building and timing all three.
 */
#define MSPV_NUM_FEATURES 10
#define MSPV_SELECTOR_PARAMS 5099

/*
 * The sparsity features of A's stored structure, rounded to FP32, into HOST out[10]:
 *   0 log2 max(nrows, 1)            5 shortest row (entries)
 *   1 log2 max(nnz, 1)              6 log2 max(ndiags, 1), ndiags = distinct col - row
 *   2 mean row length nnz / nrows   7 DIA fill nnz / (ndiags * nrows) (0 if ndiags = 0)
 *   3 population std of row length  8 empty rows / nrows
 *   4 longest row (entries)         9 max |col - row| / nrows
 * Row-based entries are 0 for nrows = 0. Counts are taken on the device (integers); the
 * ratios are formed in FP64 on the host. Any format. Synchronous.
 */
MSPV_API mspv_status mspv_features(mspv_matrix_t A, float* out, void* stream);

/*
 * Run-first tuner: builds A in each other format (FP64 values), times `reps` SpMV launches
 * of each (x = 1, after two warm-up launches) with CUDA events on `stream`, frees the copies,
 * and writes the mean milliseconds per SpMV to HOST ms[3] (indexed by mspv_format; +inf for
 * DIA when A is not square or DIA storage would exceed its fill cap) and the fastest format
 * to *best. Ties: starting from CSR, then DIA, then COO, a format replaces the current
 * choice only when it is more than 1% faster. A must be a COO or CSR handle (EFORMAT for
 * DIA); reps >= 1. Synchronous; the temporary handles are allocated and freed inside.
 */
MSPV_API mspv_status mspv_tune_format(mspv_matrix_t A, int32_t reps, void* stream, double* ms,
                                      mspv_format* best);

/*
 * Trains the selector MLP (10 -> 64 -> 64 -> 3, ReLU, softmax cross-entropy; class k is
 * mspv_format k) in one CTA on HOST features X[N * 10] (row-major, as mspv_features writes
 * them) and HOST labels y[N] in {0, 1, 2}. Features are standardised by the training set's
 * mean and population standard deviation (1 where that is below 1e-6), and their minimum and
 * maximum are kept: at prediction every feature is first clamped to that training range, so a
 * matrix beyond the training set (e.g. larger) is judged like the most extreme ones seen. Weights start as
 * uniform Glorot values drawn from SplitMix64 output k (seed `seed`) for trained parameter k
 * in layout order, biases at 0. Each epoch runs Adam (Kingma & Ba 2015: beta1 0.9, beta2
 * 0.999, eps 1e-8, step size lr) over minibatches of 64 consecutive samples in index order
 * (the last one may be shorter), each gradient the mean over its minibatch. Writes
 * MSPV_SELECTOR_PARAMS floats to HOST params in the layout
 *   mu[10] sd[10] lo[10] hi[10] W1[64][10] b1[64] W2[64][64] b2[64] W3[3][64] b3[3]   (W[out][in]).
 * Deterministic (fixed summation order). EINVAL for N < 1, epochs < 0, lr <= 0 or a label
 * outside {0, 1, 2}. Synchronous.
 */
MSPV_API mspv_status mspv_selector_train(const float* X, const int32_t* y, int32_t N,
                                         int32_t epochs, float lr, uint64_t seed, float* params,
                                         void* stream);

/*
 * Predicted class for each row of HOST features X[N * 10] under HOST params (the layout
 * above): features clamped to [lo, hi], standardised, arg max of the logits (the lowest class
 * on ties); into HOST out[N]. N >= 0.
 * Synchronous.
 */
MSPV_API mspv_status mspv_selector_predict(const float* params, const float* X, int32_t N,
                                           int32_t* out, void* stream);

/*
 * The format to use for A. params == NULL: the run-first tuner (mspv_tune_format, 10
 * reps; A must be COO or CSR). Otherwise the MLP on mspv_features(A); a DIA prediction for
 * a matrix that is not square or whose DIA storage would exceed the fill cap becomes CSR.
 * Synchronous.
 */
MSPV_API mspv_status mspv_select_format(mspv_matrix_t A, const float* params, void* stream,
                                        mspv_format* best);

/* Fill *info with the handle's shape, format and row statistics. */
MSPV_API mspv_status mspv_info(mspv_matrix_t A, mspv_matrix_info* info);

/*
 * Copy the handle's stored structure to HOST arrays (values widened exactly to FP64):
 *   COO: idx0 = rows[nnz], idx1 = cols[nnz], vals[nnz]
 *   CSR: idx0 = irp[nrows + 1], idx1 = cols[nnz], vals[nnz]
 *   DIA: idx0 = doff[ndiags], idx1 unused (may be NULL), vals[ndiags * npad]
 * Sizes come from mspv_info. Synchronous.
 */
MSPV_API mspv_status mspv_export(mspv_matrix_t A, int32_t* idx0, int32_t* idx1, double* vals,
                                 void* stream);

/* Free the handle and its device memory (after synchronising its device). NULL is a no-op. */
MSPV_API void mspv_destroy(mspv_matrix_t A);

/* The calling thread's last error message ("" if none). Valid until the next call. */
MSPV_API const char* mspv_last_error(void);

/* Name of a status code. */
MSPV_API const char* mspv_status_string(mspv_status s);

/*
 * CSR SpMV kernel choice for the given row-length statistics (host only, no device
 * access): V lanes per row, 4 while the mean row length is at most 48, then 8 (<= 96),
 * 16 (<= 192), 32 (warp per row). Rows longer than 32 V entries are listed when the CSR
 * handle is built and reduced by one CTA each. MSPV_CSR_VEC (1, 2, 4, 8, 16, 32) overrides
 * V; MSPV_CSR_VEC=0 selects the staged kernels (values and gathered x staged in shared
 * memory, one row per thread; MSPV_CSR_KERNEL=block for CTA row blocks instead of warp
 * slices). Exposed for tests and tuning.
 */
MSPV_API int32_t mspv_csr_vector_width(double row_mean, double row_std, int32_t row_max);

/*
 * FP64 fused multiply-add rate of the current device, in TFLOP/s (2 flops per FMA); device
 * characterisation, not part of the paper's method. On GB300 the FP64 pipe bounds the FP64
 * DIA SpMV, whose roofline takes this rate as its peak. One full wave of CTAs (as many as the
 * device holds at once) runs 4, 8 or 16 independent FMA chains per thread, each a running
 * sum acc = m * y + acc like an SpMV row (8 chains for `iters`
 * steps, the same FMA count for the others); for each, one warm-up launch, then the fastest of
 * `repeats` launches timed with CUDA events on `stream`; the fastest configuration is the rate.
 * Synchronous; allocates and frees a small device buffer. EINVAL for iters outside
 * [1, 2^30], repeats < 1 or tflops NULL.
 */
MSPV_API mspv_status mspv_fp64_fma_rate(int64_t iters, int32_t repeats, void* stream, double* tflops);

/* Library version, as MAJOR * 10000 + MINOR * 100 + PATCH. */
MSPV_API int32_t mspv_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MSPV_H */
