// Internal declarations shared by the translation units of libmspv.so.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>

#include "mspv.h"

namespace mspv {

constexpr int kThreads = 256;       // threads per CTA for every kernel here
// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount; 152 on
// GB300), read once per device and cached. Grid caps are multiples of it.
int num_sms();

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
mspv_status set_error(mspv_status s, const char* fmt, ...);
void clear_error();

#define MSPV_CUDA_TRY(expr)                                                              \
    do {                                                                                 \
        cudaError_t _e = (expr);                                                         \
        if (_e != cudaSuccess)                                                           \
            return ::mspv::set_error(MSPV_ECUDA, "%s failed: %s (%s:%d)", #expr,         \
                                     cudaGetErrorString(_e), __FILE__, __LINE__);        \
    } while (0)

#define MSPV_TRY(expr)                              \
    do {                                            \
        mspv_status _s = (expr);                    \
        if (_s != MSPV_OK) return _s;               \
    } while (0)

// ---------------------------------------------------------------------------
// device memory: every allocation goes through here so that MSPV_MAX_BYTES can cap
// the total the library holds (ENOMEM is then returned without exhausting the GPU).
// ---------------------------------------------------------------------------
mspv_status dev_alloc(void** p, size_t bytes);
void dev_free(void* p, size_t bytes);

template <typename T>
mspv_status dev_alloc_n(T** p, int64_t count) {
    return dev_alloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)(count > 0 ? count : 1));
}

// A device buffer freed on scope exit (synchronous free; used by converters).
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { reset(); }
    void reset() {
        if (ptr) dev_free(ptr, bytes);
        ptr = nullptr;
        bytes = 0;
    }
    mspv_status alloc(size_t b) {
        reset();
        bytes = b > 0 ? b : 1;
        mspv_status s = dev_alloc(&ptr, bytes);
        if (s != MSPV_OK) bytes = 0;
        return s;
    }
    template <typename T>
    T* as() const { return static_cast<T*>(ptr); }
};

// ---------------------------------------------------------------------------
// value storage types
// ---------------------------------------------------------------------------
inline size_t value_size(int vt) { return vt == MSPV_F64 ? 8 : (vt == MSPV_F32 ? 4 : 2); }

// Exact FP32 -> FP64 widening with integer operations only. On GB300 the hardware
// conversion issues on the (narrow) FP64 pipe at the rate of an FP64 FMA; this costs a
// handful of integer instructions instead. IEEE binary32 -> binary64 is exact:
// sign kept, exponent rebiased by 1023 - 127 = 896, mantissa shifted left by 29;
// subnormals are normalised, infinities and NaNs keep their payload.
__device__ __forceinline__ double widen_f32_bits(uint32_t u) {
    const uint32_t sign = u & 0x80000000u;
    const uint32_t e = (u >> 23) & 0xffu;
    uint32_t m = u & 0x7fffffu;
    uint32_t e64;
    if (e == 0xffu) {
        e64 = 0x7ffu;
    } else if (e != 0u) {
        e64 = e + 896u;
    } else if (m == 0u) {
        e64 = 0u;
    } else {                                   // subnormal: m * 2^-149
        const int lz = __clz(m) - 8;           // shift that brings the leading 1 to bit 23
        m = (m << lz) & 0x7fffffu;
        e64 = 1023u - 126u - (uint32_t)lz;
    }
    const uint32_t hi = sign | (e64 << 20) | (m >> 3);
    return __hiloint2double((int)hi, (int)(m << 29));
}
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ double widen(float v) { return widen_f32_bits(__float_as_uint(v)); }
__device__ __forceinline__ double widen(__nv_bfloat16 v) {
    return widen_f32_bits((uint32_t)__bfloat16_as_ushort(v) << 16);
}

// ---------------------------------------------------------------------------
// CG device state: scalars live on the device so the loop needs no host sync.
// ---------------------------------------------------------------------------
enum CgPhase : int { CG_RUNNING = 0, CG_CONVERGED = 1, CG_MAXIT = 2, CG_BREAKDOWN = 3 };

struct CgState {
    double rho;      // r.r of the current residual
    double pq;       // p.q of the current step
    double alpha;
    double beta;
    double bnorm;    // ||b||_2
    double tol;
    int32_t iters;
    int32_t maxit;
    int32_t done;    // nonzero once converged, at maxit, or broken down
    int32_t phase;   // CgPhase
    double rho_prev; // r.r before the iteration that converged (reliable updates form the
                     // next direction from it)
};

// An SpMV kernel's optional epilogue for CG: each CTA writes its partial of the dot x.y
// of its input and output (p.q) to partials[blockIdx.x]; kernels return at entry once
// st->done is set. st == nullptr disables both.
struct DotEpilogue {
    CgState* st;
    double* partials;   // one per CTA of the launch
    bool pdl = false;   // launch as a programmatic dependent launch (inside the CG loop)
    bool acc = false;   // y += A x instead of y = A x (never together with a dot product)
};

// The one place each SpMV kernel writes a row of y: overwrite, or add (accumulating SpMV).
template <typename T>
__device__ __forceinline__ void store_y(T* y, int64_t i, T v, bool acc) {
    y[i] = acc ? y[i] + v : v;
}
// A row without entries: 0 when overwriting, untouched when accumulating.
template <typename T>
__device__ __forceinline__ void zero_y(T* y, int64_t i, bool acc) {
    if (!acc) y[i] = T(0);
}

// Programmatic dependent launch. A kernel launched with the programmatic-serialisation
// attribute may be scheduled while the previous kernel of its stream is still running; it
// waits for that kernel's completion and memory (griddepcontrol.wait) before reading
// anything. pdl_trigger lets the next such kernel be scheduled early. Both are no-ops in a
// kernel launched without the attribute. The wait ends when the previous grid completes.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void launch_kernel(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                          cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);   // errors surface via cudaGetLastError
}

// COO per-window carry record: rows that cross a window boundary leave partial sums.
struct CooCarry {
    int32_t row_first;
    int32_t row_last;
    double head;   // partial sum of row_first over the window
    double tail;   // partial sum of row_last over the window
};

// Entries per CTA window of the staged COO and CSR kernels: values and gathered x are
// staged in shared memory (16 B per entry, plus 4 B of row index for COO).
constexpr int kCooWindow = 3072;    // staged COO kernel (allocation-free entry point)
constexpr int kCooVecChunk = 256;   // run-vector COO kernel: entries per warp
constexpr int kCooRbRows = 32;      // row-block COO kernel: rows per warp (4 lanes each)
constexpr int kCsrWindow = 2560;     // a CTA takes the rows that start in its window

// CG workspace, owned by a handle and grown on demand.
struct CgWork {
    int64_t n = 0;
    double* r = nullptr;
    double* p = nullptr;
    double* q = nullptr;
    double* partials = nullptr;
    int64_t npartials = 0;
    CgState* st = nullptr;
    CgState* host_st = nullptr;   // pinned mirror
    // FP32 vectors of the FP32-arithmetic inner solver
    int64_t nf = 0;
    float* rf = nullptr;
    float* pf = nullptr;
    float* qf = nullptr;
};

// Last CTA of a fused p.q reduction: alpha = rho / p.q, or a breakdown when p.q <= 0
// or alpha is not finite (the matrix is not SPD, or the iteration has degenerated).
__device__ __forceinline__ void finish_alpha(CgState* st, double pq) {
    st->pq = pq;
    const double alpha = st->rho / pq;
    if (!(pq > 0.0) || !isfinite(alpha)) {
        st->phase = CG_BREAKDOWN;
        st->done = 1;
    } else {
        st->alpha = alpha;
    }
}

}  // namespace mspv

// The handle. Device arrays are owned; sizes in elements.
struct mspv_matrix {
    int32_t format = MSPV_COO;
    int32_t value_type = MSPV_F64;
    int32_t nrows = 0, ncols = 0;
    int64_t nnz = 0;
    int32_t ndiags = 0, npad = 0;
    int32_t csr_vector = 0;   // 0: staged kernel; 1..32: lanes per row
    int32_t csr_block = 0;    // staged kernel: 0 = warp-private staging, 1 = CTA row blocks
    int32_t row_max = 0;
    int32_t row_min = 0;
    double row_mean = 0.0, row_std = 0.0;
    int64_t empty_rows = 0;
    int device = 0;

    int32_t* ai = nullptr;    // COO rows
    int32_t* aj = nullptr;    // COO / CSR columns
    int32_t* irp = nullptr;   // CSR row pointers
    int32_t* doff = nullptr;  // DIA offsets
    int2* druns = nullptr;    // DIA: runs of consecutive offsets (first diagonal, length <= 3)
    int32_t ndruns = 0;
    void* av = nullptr;       // values (value_type)
    int64_t av_count = 0;

    mspv::CooCarry* carry = nullptr;   // COO: per-window carries
    int64_t nchunks = 0;               // COO chunks of kCooVecChunk entries
    int32_t coo_kernel = 0;            // COO: 0 lane-sequential segments, 1 run-vector, 2 row blocks (choose_coo_kernel)
    int32_t* coo_rb = nullptr;         // COO row-block kernel: first entry of every 32-row block, nrb + 1 entries
    int64_t coo_nrb = 0;
    int32_t coo_chunk = 256;           // run-vector kernel: entries per warp (256; MSPV_COO_CHUNK=512)
    int32_t* row_block = nullptr;      // CSR: first row of each window, nblocks + 1 entries
    int32_t* long_rows = nullptr;      // CSR vector kernel: rows longer than 32 * csr_vector
    int64_t nlong = 0;
    int64_t nblocks = 0;               // CSR windows

    mspv::CgWork cg;
    int64_t bytes = 0;        // device bytes held
};

namespace mspv {

// scan.cu / convert.cu
mspv_status exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t m, int32_t* d_total,
                               cudaStream_t s);
mspv_status build_coo(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t* rows,
                      const int32_t* cols, const double* vals, cudaStream_t s,
                      mspv_matrix* M);
mspv_status build_from(const mspv_matrix* A, int32_t format, int32_t vt, cudaStream_t s,
                       mspv_matrix* M);
mspv_status export_matrix(const mspv_matrix* A, int32_t* idx0, int32_t* idx1, double* vals,
                          cudaStream_t s);
void free_matrix(mspv_matrix* M);
// DIA slots (ndiags * npad) allowed for nnz entries: max(MSPV_DIA_MAX_FILL (32) * nnz, 2^20)
double dia_slot_cap(int64_t nnz);
mspv_status ensure_coo_carry(mspv_matrix* M, cudaStream_t s);   // stream-ordered after M->ai
mspv_status finish_coo_stats(mspv_matrix* M, cudaStream_t s);
// Local part (columns < c) and remote part (columns >= c, renumbered from 0) of a COO/CSR
// handle, both canonical COO handles with A's value type.
mspv_status split_columns(const mspv_matrix* A, int32_t c, cudaStream_t s, mspv_matrix* L, mspv_matrix* R);

// spmv.cu
mspv_status launch_spmv(const mspv_matrix* A, const double* x, double* y, cudaStream_t s,
                        DotEpilogue ep);
// FP32 arithmetic (FP32/BF16 stored values, FP32 vectors, 16-byte aligned): the inner solver of
// mixed-precision refinement. EFORMAT for FP64 stored values.
mspv_status launch_spmv_f32(const mspv_matrix* A, const float* x, float* y, cudaStream_t s,
                            DotEpilogue ep);
int64_t spmv_partials_count(const mspv_matrix* A, bool f32);   // CTAs of the fused-dot launch
int64_t spmv_partials_needed(const mspv_matrix* A);   // the larger of the FP64 and FP32 counts
mspv_status launch_coo_raw(int32_t nrows, int64_t nnz, const int32_t* ai, const int32_t* aj,
                           const double* av, const double* x, double* y, CooCarry* carry,
                           cudaStream_t s);
int32_t choose_csr_vector(double mean, double stdev, int32_t maxlen);
mspv_status build_csr_row_blocks(mspv_matrix* M, cudaStream_t s);
mspv_status build_csr_long_rows(mspv_matrix* M, cudaStream_t s);
int32_t choose_csr_block_kernel();   // MSPV_CSR_KERNEL=block selects CTA row blocks
int32_t choose_coo_kernel(int32_t row_max, int64_t nnz, int32_t nrows);   // 2 row blocks, 1 run-vector, 0 segments

// cg.cu
mspv_status cg_solve(mspv_matrix* A, const double* b, double* x, double tol, int32_t maxit,
                     cudaStream_t s, int32_t* iters, double* relres);
mspv_status cg_solve_ir(mspv_matrix* A64, mspv_matrix* Alo, const double* b, double* x,
                        double tol, double inner_tol, int32_t max_outer, int32_t maxit_inner,
                        int32_t inner_fp32, cudaStream_t s, int32_t* outer_iters,
                        int32_t* inner_iters, double* relres);

// select.cu: format selection features, run-first tuner, MLP selector
constexpr int kSelectorFeatures = 10;
constexpr int kSelectorParams = 5099;   // mu, sd, lo, hi, W1, b1, W2, b2, W3, b3
mspv_status compute_features(const mspv_matrix* A, float* out, cudaStream_t s, int64_t* ndiags = nullptr);
mspv_status select_format(const mspv_matrix* A, const float* params, cudaStream_t s, int32_t* best);
mspv_status tune_formats(const mspv_matrix* A, int32_t reps, cudaStream_t s, double* ms, int32_t* best);
mspv_status selector_train(const float* X, const int32_t* y, int32_t N, int32_t epochs, float lr,
                           uint64_t seed, float* params, cudaStream_t s);
mspv_status selector_predict(const float* params, const float* X, int32_t N, int32_t* out,
                             cudaStream_t s);

// block-wide reductions shared by the kernels (defined inline below)
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the CTA (kThreads threads); the result is valid in thread 0. Every value goes
// through shared memory and warp 0 adds 8 of them per lane before a 5-step shuffle
// reduction: 13 FP64 warp instructions per CTA instead of 45 for a shuffle reduction in
// every warp (FP64 issue slots are the scarce resource on GB300). smem holds kThreads
// doubles. The order is fixed, so the result is deterministic.
__device__ __forceinline__ double block_sum(double v, double* smem) {
    smem[threadIdx.x] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = smem[threadIdx.x];
#pragma unroll
        for (int k = 1; k < kThreads / 32; ++k) t += smem[threadIdx.x + 32 * k];
        t = warp_sum(t);
    }
    __syncthreads();
    return t;
}


}  // namespace mspv
