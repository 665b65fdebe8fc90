// C-ABI entry points of libmspv.so (declared in include/mspv.h): argument checks,
// device-memory accounting, error strings, and dispatch into the converters, the
// SpMV kernels and the CG solvers. No exception leaves this file.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

namespace mspv {

// ---------------------------------------------------------------------------
// errors (thread-local message)
// ---------------------------------------------------------------------------
static thread_local char g_err[1024] = "";

mspv_status set_error(mspv_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

void clear_error() { g_err[0] = '\0'; }

// ---------------------------------------------------------------------------
// device memory accounting; MSPV_MAX_BYTES caps the bytes held by the library
// ---------------------------------------------------------------------------
static std::mutex g_mem_mu;
static std::unordered_map<void*, size_t> g_sizes;
static int64_t g_live = 0;

static int64_t byte_cap() {
    const char* s = std::getenv("MSPV_MAX_BYTES");
    if (!s || !*s) return 0;
    const long long v = std::atoll(s);
    return v > 0 ? (int64_t)v : 0;
}

mspv_status dev_alloc(void** p, size_t bytes) {
    *p = nullptr;
    const int64_t cap = byte_cap();
    {
        std::lock_guard<std::mutex> lk(g_mem_mu);
        if (cap > 0 && g_live + (int64_t)bytes > cap)
            return set_error(MSPV_ENOMEM, "allocation of %zu bytes would exceed MSPV_MAX_BYTES=%lld (held %lld)",
                             bytes, (long long)cap, (long long)g_live);
    }
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();   // allocation failures are not sticky; clear it
        *p = nullptr;
        if (e == cudaErrorMemoryAllocation)
            return set_error(MSPV_ENOMEM, "cudaMalloc of %zu bytes failed", bytes);
        return set_error(MSPV_ECUDA, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    std::lock_guard<std::mutex> lk(g_mem_mu);
    g_sizes[*p] = bytes;
    g_live += (int64_t)bytes;
    return MSPV_OK;
}

void dev_free(void* p, size_t) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(g_mem_mu);
        auto it = g_sizes.find(p);
        if (it != g_sizes.end()) {
            g_live -= (int64_t)it->second;
            g_sizes.erase(it);
        }
    }
    cudaFree(p);
}

// ---------------------------------------------------------------------------
// SM count of the current device, cached per device ordinal
// ---------------------------------------------------------------------------
constexpr int kMaxDevices = 64;
static std::atomic<int> g_sms[kMaxDevices];

int num_sms() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return 152;   // GB300's count; only reached without a usable device
    }
    int v = g_sms[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
        cudaGetLastError();
        v = 152;
    }
    g_sms[dev].store(v, std::memory_order_relaxed);
    return v;
}

}  // namespace mspv

using namespace mspv;

#define MSPV_GUARD_BEGIN try {
#define MSPV_GUARD_END                                                                   \
    }                                                                                    \
    catch (const std::bad_alloc&) {                                                      \
        return set_error(MSPV_ENOMEM, "host allocation failed");                         \
    }                                                                                    \
    catch (...) {                                                                        \
        return set_error(MSPV_ECUDA, "internal error");                                  \
    }

static inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

extern "C" {

MSPV_API const char* mspv_last_error(void) { return g_err; }

MSPV_API const char* mspv_status_string(mspv_status s) {
    switch (s) {
        case MSPV_OK: return "MSPV_OK";
        case MSPV_EINVAL: return "MSPV_EINVAL";
        case MSPV_ENOMEM: return "MSPV_ENOMEM";
        case MSPV_ETOOBIG: return "MSPV_ETOOBIG";
        case MSPV_EFORMAT: return "MSPV_EFORMAT";
        case MSPV_ECUDA: return "MSPV_ECUDA";
        case MSPV_ENOTCONV: return "MSPV_ENOTCONV";
        case MSPV_EBREAKDOWN: return "MSPV_EBREAKDOWN";
    }
    return "MSPV_UNKNOWN";
}

MSPV_API int32_t mspv_version(void) { return 100; }

MSPV_API int32_t mspv_csr_vector_width(double row_mean, double row_std, int32_t row_max) {
    return choose_csr_vector(row_mean, row_std, row_max);
}

MSPV_API void mspv_destroy(mspv_matrix_t A) {
    if (!A) return;
    free_matrix(A);
    delete A;
}

MSPV_API mspv_status mspv_create_coo(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t* rows,
                                     const int32_t* cols, const double* vals, int on_device,
                                     void* stream, mspv_matrix_t* out) {
    MSPV_GUARD_BEGIN
    if (!out) return set_error(MSPV_EINVAL, "create_coo: out is NULL");
    *out = nullptr;
    if (nrows < 0 || ncols < 0 || nnz < 0)
        return set_error(MSPV_EINVAL, "create_coo: negative size (nrows=%d ncols=%d nnz=%lld)", nrows, ncols,
                         (long long)nnz);
    if (nnz >= (int64_t)1 << 31) return set_error(MSPV_ETOOBIG, "create_coo: nnz=%lld >= 2^31", (long long)nnz);
    if (nnz > 0 && (!rows || !cols || !vals)) return set_error(MSPV_EINVAL, "create_coo: NULL triplet array");
    if (nnz > 0 && (nrows == 0 || ncols == 0))
        return set_error(MSPV_EINVAL, "create_coo: entries given for an empty shape");
    if (!on_device) {   // host triplets are checked before any device work
        for (int64_t e = 0; e < nnz; ++e)
            if (rows[e] < 0 || rows[e] >= nrows || cols[e] < 0 || cols[e] >= ncols)
                return set_error(MSPV_EINVAL, "create_coo: entry %lld at (%d, %d) outside [0,%d) x [0,%d)",
                                 (long long)e, rows[e], cols[e], nrows, ncols);
    }
    cudaStream_t s = as_stream(stream);
    mspv_matrix* M = new mspv_matrix();
    cudaGetDevice(&M->device);
    DevBuf dr, dc, dv;
    const int32_t* r = rows;
    const int32_t* c = cols;
    const double* v = vals;
    mspv_status st = MSPV_OK;
    if (!on_device && nnz > 0) {
        if ((st = dr.alloc(4 * (size_t)nnz)) == MSPV_OK && (st = dc.alloc(4 * (size_t)nnz)) == MSPV_OK &&
            (st = dv.alloc(8 * (size_t)nnz)) == MSPV_OK) {
            cudaError_t e1 = cudaMemcpyAsync(dr.ptr, rows, 4 * nnz, cudaMemcpyHostToDevice, s);
            cudaError_t e2 = cudaMemcpyAsync(dc.ptr, cols, 4 * nnz, cudaMemcpyHostToDevice, s);
            cudaError_t e3 = cudaMemcpyAsync(dv.ptr, vals, 8 * nnz, cudaMemcpyHostToDevice, s);
            if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)
                st = set_error(MSPV_ECUDA, "create_coo: host-to-device copy failed: %s",
                               cudaGetErrorString(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3)));
        }
        r = dr.as<int32_t>();
        c = dc.as<int32_t>();
        v = dv.as<double>();
    }
    if (st == MSPV_OK) st = build_coo(nrows, ncols, nnz, r, c, v, s, M);
    if (st == MSPV_OK) st = finish_coo_stats(M, s);
    if (st == MSPV_OK) st = ensure_coo_carry(M, s);
    if (st != MSPV_OK) {
        cudaStreamSynchronize(s);
        mspv_destroy(M);
        return st;
    }
    *out = M;
    clear_error();
    return MSPV_OK;
    MSPV_GUARD_END
}

MSPV_API mspv_status mspv_convert(mspv_matrix_t A, mspv_format format, mspv_value_type value_type,
                                  void* stream, mspv_matrix_t* out) {
    MSPV_GUARD_BEGIN
    if (!out) return set_error(MSPV_EINVAL, "convert: out is NULL");
    *out = nullptr;
    if (!A) return set_error(MSPV_EINVAL, "convert: A is NULL");
    if (format < MSPV_COO || format > MSPV_DIA) return set_error(MSPV_EINVAL, "convert: unknown format %d", (int)format);
    if (value_type < MSPV_F64 || value_type > MSPV_BF16)
        return set_error(MSPV_EINVAL, "convert: unknown value type %d", (int)value_type);
    cudaStream_t s = as_stream(stream);
    mspv_matrix* M = new mspv_matrix();
    M->device = A->device;
    mspv_status st = build_from(A, format, value_type, s, M);
    if (st != MSPV_OK) {
        cudaStreamSynchronize(s);
        mspv_destroy(M);
        return st;
    }
    *out = M;
    clear_error();
    return MSPV_OK;
    MSPV_GUARD_END
}

MSPV_API mspv_status mspv_spmv(mspv_matrix_t A, const double* x, double* y, void* stream) {
    MSPV_GUARD_BEGIN
    if (!A) return set_error(MSPV_EINVAL, "spmv: A is NULL");
    if ((!x && A->ncols > 0) || (!y && A->nrows > 0)) return set_error(MSPV_EINVAL, "spmv: NULL vector");
    if (x == y && A->nrows > 0) return set_error(MSPV_EINVAL, "spmv: x and y must not overlap");
    return launch_spmv(A, x, y, as_stream(stream), DotEpilogue{nullptr, nullptr});
    MSPV_GUARD_END
}

MSPV_API mspv_status mspv_cg_solve(mspv_matrix_t A, const double* b, double* x, double tol, int32_t maxit,
                                   void* stream, int32_t* iters, double* relres) {
    MSPV_GUARD_BEGIN
    if (!A) return set_error(MSPV_EINVAL, "cg: A is NULL");
    if ((!b || !x) && A->nrows > 0) return set_error(MSPV_EINVAL, "cg: NULL vector");
    mspv_status st = cg_solve(A, b, x, tol, maxit, as_stream(stream), iters, relres);
    if (st == MSPV_OK) clear_error();
    return st;
    MSPV_GUARD_END
}

MSPV_API mspv_status mspv_cg_solve_ir(mspv_matrix_t A64, mspv_matrix_t Alo, const double* b, double* x,
                                      double tol, double inner_tol, int32_t max_outer, int32_t maxit_inner,
                                      int32_t inner_fp32, void* stream, int32_t* outer_iters,
                                      int32_t* inner_iters, double* relres) {
    MSPV_GUARD_BEGIN
    if (!A64 || !Alo) return set_error(MSPV_EINVAL, "cg_ir: NULL matrix");
    if ((!b || !x) && A64->nrows > 0) return set_error(MSPV_EINVAL, "cg_ir: NULL vector");
    return cg_solve_ir(A64, Alo, b, x, tol, inner_tol, max_outer, maxit_inner, inner_fp32,
                       as_stream(stream), outer_iters, inner_iters, relres);
    MSPV_GUARD_END
}

MSPV_API mspv_status mspv_info(mspv_matrix_t A, mspv_matrix_info* info) {
    if (!A || !info) return set_error(MSPV_EINVAL, "info: NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->format = A->format;
    info->value_type = A->value_type;
    info->nrows = A->nrows;
    info->ncols = A->ncols;
    info->nnz = A->nnz;
    info->ndiags = A->ndiags;
    info->npad = A->npad;
    info->csr_vector = A->format == MSPV_CSR ? A->csr_vector : 0;
    info->row_max = A->row_max;
    info->row_mean = A->row_mean;
    info->row_std = A->row_std;
    info->empty_rows = A->empty_rows;
    info->device_bytes = A->bytes;
    return MSPV_OK;
}

MSPV_API mspv_status mspv_export(mspv_matrix_t A, int32_t* idx0, int32_t* idx1, double* vals, void* stream) {
    MSPV_GUARD_BEGIN
    if (!A) return set_error(MSPV_EINVAL, "export: A is NULL");
    return export_matrix(A, idx0, idx1, vals, as_stream(stream));
    MSPV_GUARD_END
}

MSPV_API mspv_status mspv_spmv_f32(mspv_matrix_t A, const float* x, float* y, void* stream) {
    MSPV_GUARD_BEGIN
    if (!A) return set_error(MSPV_EINVAL, "spmv_f32: A is NULL");
    if ((!x && A->ncols > 0) || (!y && A->nrows > 0)) return set_error(MSPV_EINVAL, "spmv_f32: NULL vector");
    if (x == y && A->nrows > 0) return set_error(MSPV_EINVAL, "spmv_f32: x and y must not overlap");
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15)
        return set_error(MSPV_EINVAL, "spmv_f32: x and y must be 16-byte aligned");
    return launch_spmv_f32(A, x, y, as_stream(stream), DotEpilogue{nullptr, nullptr});
    MSPV_GUARD_END
}

MSPV_API mspv_status mspv_spmv_add(mspv_matrix_t A, const double* x, double* y, void* stream) {
    MSPV_GUARD_BEGIN
    if (!A) return set_error(MSPV_EINVAL, "spmv_add: A is NULL");
    if ((!x && A->ncols > 0) || (!y && A->nrows > 0)) return set_error(MSPV_EINVAL, "spmv_add: NULL vector");
    if (x == y && A->nrows > 0) return set_error(MSPV_EINVAL, "spmv_add: x and y must not overlap");
    DotEpilogue ep{nullptr, nullptr};
    ep.acc = true;
    return launch_spmv(A, x, y, as_stream(stream), ep);
    MSPV_GUARD_END
}

MSPV_API mspv_status mspv_split_columns(mspv_matrix_t A, int32_t ncols_local, void* stream, mspv_matrix_t* local,
                                        mspv_matrix_t* remote) {
    MSPV_GUARD_BEGIN
    if (!local || !remote) return set_error(MSPV_EINVAL, "split_columns: NULL output");
    *local = nullptr;
    *remote = nullptr;
    if (!A) return set_error(MSPV_EINVAL, "split_columns: A is NULL");
    if (ncols_local < 0 || ncols_local > A->ncols)
        return set_error(MSPV_EINVAL, "split_columns: ncols_local = %d outside [0, %d]", ncols_local, A->ncols);
    cudaStream_t s = as_stream(stream);
    mspv_matrix* L = new mspv_matrix();
    mspv_matrix* R = new mspv_matrix();
    L->device = R->device = A->device;
    const mspv_status st = split_columns(A, ncols_local, s, L, R);
    if (st != MSPV_OK) {
        cudaStreamSynchronize(s);
        mspv_destroy(L);
        mspv_destroy(R);
        return st;
    }
    *local = L;
    *remote = R;
    clear_error();
    return MSPV_OK;
    MSPV_GUARD_END
}

MSPV_API mspv_status mspv_features(mspv_matrix_t A, float* out, void* stream) {
    MSPV_GUARD_BEGIN
    if (!A || !out) return set_error(MSPV_EINVAL, "features: NULL argument");
    MSPV_TRY(compute_features(A, out, as_stream(stream)));
    clear_error();
    return MSPV_OK;
    MSPV_GUARD_END
}

MSPV_API mspv_status mspv_tune_format(mspv_matrix_t A, int32_t reps, void* stream, double* ms,
                                      mspv_format* best) {
    MSPV_GUARD_BEGIN
    if (!A || !ms || !best) return set_error(MSPV_EINVAL, "tune_format: NULL argument");
    if (reps < 1) return set_error(MSPV_EINVAL, "tune_format: reps = %d < 1", reps);
    int32_t b = MSPV_CSR;
    MSPV_TRY(tune_formats(A, reps, as_stream(stream), ms, &b));
    *best = (mspv_format)b;
    return MSPV_OK;
    MSPV_GUARD_END
}

MSPV_API mspv_status mspv_selector_train(const float* X, const int32_t* y, int32_t N, int32_t epochs, float lr,
                                         uint64_t seed, float* params, void* stream) {
    MSPV_GUARD_BEGIN
    if (!X || !y || !params) return set_error(MSPV_EINVAL, "selector_train: NULL argument");
    if (N < 1 || epochs < 0 || !(lr > 0.0f))
        return set_error(MSPV_EINVAL, "selector_train: N = %d, epochs = %d, lr = %g", N, epochs, (double)lr);
    for (int32_t i = 0; i < N; ++i)
        if (y[i] < 0 || y[i] > 2) return set_error(MSPV_EINVAL, "selector_train: label %d of sample %d", y[i], i);
    MSPV_TRY(selector_train(X, y, N, epochs, lr, seed, params, as_stream(stream)));
    clear_error();
    return MSPV_OK;
    MSPV_GUARD_END
}

MSPV_API mspv_status mspv_selector_predict(const float* params, const float* X, int32_t N, int32_t* out,
                                           void* stream) {
    MSPV_GUARD_BEGIN
    if (N < 0) return set_error(MSPV_EINVAL, "selector_predict: N = %d", N);
    if (!params || (N > 0 && (!X || !out))) return set_error(MSPV_EINVAL, "selector_predict: NULL argument");
    MSPV_TRY(selector_predict(params, X, N, out, as_stream(stream)));
    clear_error();
    return MSPV_OK;
    MSPV_GUARD_END
}

MSPV_API mspv_status mspv_select_format(mspv_matrix_t A, const float* params, void* stream, mspv_format* best) {
    MSPV_GUARD_BEGIN
    if (!A || !best) return set_error(MSPV_EINVAL, "select_format: NULL argument");
    int32_t b = MSPV_CSR;
    MSPV_TRY(select_format(A, params, as_stream(stream), &b));
    *best = (mspv_format)b;
    clear_error();
    return MSPV_OK;
    MSPV_GUARD_END
}

}  // extern "C"
