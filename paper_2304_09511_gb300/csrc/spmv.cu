// SpMV kernels for the three storage formats of Sec. II-B, y = A x in FP64.
//
//  DIA (Algorithm 3): diagonal-major values, each thread owns RPT consecutive rows
//      and walks the diagonals in order; value loads are 128-bit (FP64: 2 rows,
//      FP32: 4 rows, BF16: 8 rows), coalesced and streamed past L1. This is the
//      row-parallel, diagonal-sequential structure of the paper's outer-loop
//      vectorisation (Sec. III), with a warp's 32 lanes in place of SVE lanes and the
//      predicate 0 <= k < N kept per element.
//  CSR (Algorithm 2): V lanes per row (V in 1..32 from the row-length statistics),
//      strided accumulation then a butterfly reduction inside the V-lane group.
//  COO (Algorithm 1): each warp owns a contiguous chunk of 256 sorted entries and
//      does a segmented shuffle-scan keyed by row -- the GPU counterpart of the
//      paper's SVE COO kernel, which masks runs of equal row index and reduces them
//      horizontally. Rows that cross a chunk boundary leave partial sums in a carry
//      record; a fix-up pass adds them in chunk order. No floating-point atomics,
//      so y is bit-identical run to run.
//
// All three can fuse CG's p.q into the epilogue (DotEpilogue): the last CTA to
// finish reduces the per-CTA partials in index order and forms alpha.
#include <climits>
#include <cstdlib>

#include "internal.cuh"

namespace mspv {

// ---------------------------------------------------------------------------
// value loads: one scalar, or RPT consecutive values as one 128-bit load
// ---------------------------------------------------------------------------
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) { return (double)v; }
__device__ __forceinline__ double to_f64(__nv_bfloat16 v) {
    return (double)__uint_as_float((uint32_t)__bfloat16_as_ushort(v) << 16);
}

template <typename VT> struct DiaVec;
template <> struct DiaVec<double> {
    static constexpr int RPT = 2;
    __device__ __forceinline__ static void load(const double* p, double (&v)[RPT]) {
        const double2 t = __ldcs(reinterpret_cast<const double2*>(p));
        v[0] = t.x; v[1] = t.y;
    }
};
template <> struct DiaVec<float> {
    static constexpr int RPT = 4;
    __device__ __forceinline__ static void load(const float* p, double (&v)[RPT]) {
        const float4 t = __ldcs(reinterpret_cast<const float4*>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
};
template <> struct DiaVec<__nv_bfloat16> {
    static constexpr int RPT = 8;
    __device__ __forceinline__ static void load(const __nv_bfloat16* p, double (&v)[RPT]) {
        const uint4 t = __ldcs(reinterpret_cast<const uint4*>(p));
        const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[2 * k] = (double)__uint_as_float(w[k] << 16);
            v[2 * k + 1] = (double)__uint_as_float(w[k] & 0xffff0000u);
        }
    }
};

// ---------------------------------------------------------------------------
// DIA
// ---------------------------------------------------------------------------
constexpr int kDiaSmemDiags = 256;   // offsets cached in shared memory; more are read from global

template <typename VT>
__global__ void __launch_bounds__(kThreads) spmv_dia_kernel(
    int32_t n, int32_t ndiags, int32_t npad, const int32_t* __restrict__ doff,
    const VT* __restrict__ av, const double* __restrict__ x, double* __restrict__ y,
    DotEpilogue ep) {
    constexpr int RPT = DiaVec<VT>::RPT;
    if (ep.st && ep.st->done) return;   // uniform: CG already finished
    __shared__ int32_t s_off[kDiaSmemDiags];
    for (int k = threadIdx.x; k < ndiags && k < kDiaSmemDiags; k += kThreads) s_off[k] = doff[k];
    __syncthreads();

    const int64_t i0 = ((int64_t)blockIdx.x * kThreads + threadIdx.x) * RPT;
    double acc[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) acc[r] = 0.0;
    if (i0 < n) {
        const VT* col = av + i0;
#pragma unroll 3
        for (int j = 0; j < ndiags; ++j) {
            const int32_t off = (j < kDiaSmemDiags) ? s_off[j] : __ldg(doff + j);
            double a[RPT];
            DiaVec<VT>::load(col + (int64_t)j * npad, a);
            const int64_t k0 = i0 + off;
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                const int64_t k = k0 + r;
                const double xv = (k >= 0 && k < n) ? __ldg(x + k) : 0.0;
                acc[r] = fma(a[r], xv, acc[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < RPT; ++r)
            if (i0 + r < n) y[i0 + r] = acc[r];
    }
    if (ep.st) {
        double d = 0.0;
        if (i0 < n) {
#pragma unroll
            for (int r = 0; r < RPT; ++r)
                if (i0 + r < n) d = fma(__ldg(x + i0 + r), acc[r], d);
        }
        double tot;
        if (last_block_total(d, ep.partials, &ep.st->ticket, &tot) && threadIdx.x == 0)
            finish_alpha(ep.st, tot);
    }
}

// ---------------------------------------------------------------------------
// CSR, V lanes per row
// ---------------------------------------------------------------------------
template <typename VT, int V>
__global__ void __launch_bounds__(kThreads) spmv_csr_vector_kernel(
    int32_t nrows, const int32_t* __restrict__ irp, const int32_t* __restrict__ aj,
    const VT* __restrict__ av, const double* __restrict__ x, double* __restrict__ y,
    DotEpilogue ep) {
    if (ep.st && ep.st->done) return;
    const int64_t gt = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const int64_t row = gt / V;
    const int lane = threadIdx.x & (V - 1);
    double sum = 0.0;
    if (row < nrows) {
        const int32_t s = __ldg(irp + row), e = __ldg(irp + row + 1);
        int32_t j = s + lane;
        // two independent accumulators for memory-level parallelism
        double sum2 = 0.0;
        for (; j + V < e; j += 2 * V) {
            const int32_t c0 = __ldcs(aj + j), c1 = __ldcs(aj + j + V);
            const double a0 = to_f64(__ldcs(av + j)), a1 = to_f64(__ldcs(av + j + V));
            sum = fma(a0, __ldg(x + c0), sum);
            sum2 = fma(a1, __ldg(x + c1), sum2);
        }
        if (j < e) sum = fma(to_f64(__ldcs(av + j)), __ldg(x + __ldcs(aj + j)), sum);
        sum += sum2;
    }
#pragma unroll
    for (int o = V / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0 && row < nrows) y[row] = sum;
    if (ep.st) {
        const double d = (lane == 0 && row < nrows) ? __ldg(x + row) * sum : 0.0;
        double tot;
        if (last_block_total(d, ep.partials, &ep.st->ticket, &tot) && threadIdx.x == 0)
            finish_alpha(ep.st, tot);
    }
}

// ---------------------------------------------------------------------------
// COO, warp-segmented
// ---------------------------------------------------------------------------
template <typename VT>
__global__ void __launch_bounds__(kThreads) spmv_coo_kernel(
    int32_t nrows, int64_t nnz, const int32_t* __restrict__ ai, const int32_t* __restrict__ aj,
    const VT* __restrict__ av, const double* __restrict__ x, double* __restrict__ y,
    CooCarry* __restrict__ carry, int64_t nchunks, const CgState* st) {
    if (st && st->done) return;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    if (w >= nchunks) return;   // whole warp
    const int64_t c0 = w * kCooChunk;
    const int64_t c1 = (c0 + kCooChunk < nnz) ? c0 + kCooChunk : nnz;

    // all loads first, for memory-level parallelism
    int32_t rr[kCooWarpIters];
    double pp[kCooWarpIters];
    {
        int32_t cc[kCooWarpIters];
        double aa[kCooWarpIters];
#pragma unroll
        for (int it = 0; it < kCooWarpIters; ++it) {
            const int64_t e = c0 + it * 32 + lane;
            const bool valid = e < c1;
            rr[it] = valid ? __ldcs(ai + e) : INT_MAX;
            cc[it] = valid ? __ldcs(aj + e) : 0;
            aa[it] = valid ? to_f64(__ldcs(av + e)) : 0.0;
        }
#pragma unroll
        for (int it = 0; it < kCooWarpIters; ++it)
            pp[it] = (rr[it] != INT_MAX) ? aa[it] * __ldg(x + cc[it]) : 0.0;
    }
    const int32_t row_first = __shfl_sync(FULL, rr[0], 0);
    const int32_t row_before = (c0 > 0) ? __ldg(ai + c0 - 1) : -1;
    const int32_t row_after = (c1 < nnz) ? __ldg(ai + c1) : INT_MAX;
    const bool cont_prev = (row_before == row_first);

    int32_t carry_row = row_before;
    double carry_val = 0.0;
#pragma unroll
    for (int it = 0; it < kCooWarpIters; ++it) {
        const int32_t row = rr[it];
        double v = pp[it];
        // segmented inclusive scan over equal rows (rows are sorted, so runs are contiguous)
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double pv = __shfl_up_sync(FULL, v, o);
            const int32_t rv = __shfl_up_sync(FULL, row, o);
            if (lane >= o && rv == row) v += pv;
        }
        if (row == carry_row) v += carry_val;
        int32_t prev_row = __shfl_up_sync(FULL, row, 1);
        if (lane == 0) prev_row = carry_row;
        int32_t next_row = __shfl_down_sync(FULL, row, 1);
        // lane 31 looks at the first entry of the next step; after the last step the
        // run may continue into the next chunk, which the code after the loop decides
        const int32_t next_step_row =
            __shfl_sync(FULL, rr[(it + 1 < kCooWarpIters) ? it + 1 : it], 0);
        if (lane == 31) next_row = next_step_row;
        const bool may_end = (lane < 31) || (it + 1 < kCooWarpIters);
        if (row != INT_MAX) {
            // rows skipped between the previous entry and this one are empty
            if (row != prev_row)
                for (int32_t r = prev_row + 1; r < row; ++r) y[r] = 0.0;
            if (may_end && next_row != row) {   // the run of `row` ends inside the chunk
                if (row == row_first && cont_prev) carry[w].head = v;
                else y[row] = v;                // (such a run never continues past the chunk)
            }
        }
        carry_row = __shfl_sync(FULL, row, 31);
        carry_val = __shfl_sync(FULL, v, 31);
    }
    if (lane == 0) {
        int32_t row_last = carry_row;
        if (carry_row != INT_MAX) {   // the chunk's last entry sits in lane 31 of the last step
            const bool cont_next = (row_after == carry_row);
            const bool single = (carry_row == row_first);
            if (single && cont_prev) carry[w].head = carry_val;
            if (cont_next) carry[w].tail = carry_val;
            if (!cont_next && !(single && cont_prev)) y[carry_row] = carry_val;
        } else {
            row_last = __ldg(ai + c1 - 1);
        }
        carry[w].row_first = row_first;
        carry[w].row_last = row_last;
    }
    if (c1 == nnz) {   // trailing empty rows
        const int32_t last = __ldg(ai + nnz - 1);
        for (int32_t r = last + 1 + lane; r < nrows; r += 32) y[r] = 0.0;
    }
}

// Rows spanning chunks: the chunk where such a row starts adds its tail, the heads of
// the chunks it covers entirely, and the head of the chunk where it ends, in order.
__global__ void spmv_coo_fixup_kernel(const CooCarry* __restrict__ carry, int64_t nchunks,
                                      double* __restrict__ y, const CgState* st) {
    if (st && st->done) return;
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nchunks - 1) return;   // the last chunk cannot continue into another
    const CooCarry c = carry[w];
    const bool cont_next = carry[w + 1].row_first == c.row_last;
    const bool single = c.row_first == c.row_last;
    const bool cont_prev = (w > 0) && carry[w - 1].row_last == c.row_first;
    if (!cont_next || (single && cont_prev)) return;
    double sum = c.tail;
    int64_t v = w + 1;
    for (;;) {
        const CooCarry d = carry[v];
        sum += d.head;
        const bool d_single = d.row_first == d.row_last;
        const bool d_next = (v + 1 < nchunks) && carry[v + 1].row_first == d.row_last;
        if (d_single && d_next) ++v;
        else break;
    }
    y[c.row_last] = sum;
}

__global__ void fill_zero_kernel(double* __restrict__ y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = 0.0;
}

// p.q for the COO path (its SpMV has no single pass to fuse into); last CTA forms alpha.
__global__ void __launch_bounds__(kThreads) dot_alpha_kernel(int64_t n, const double* __restrict__ p,
                                                             const double* __restrict__ q,
                                                             DotEpilogue ep) {
    if (ep.st->done) return;
    double d = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kThreads)
        d = fma(p[i], q[i], d);
    double tot;
    if (last_block_total(d, ep.partials, &ep.st->ticket, &tot) && threadIdx.x == 0)
        finish_alpha(ep.st, tot);
}

// ---------------------------------------------------------------------------
// host dispatch
// ---------------------------------------------------------------------------
int32_t choose_csr_vector(double mean, double stdev, int32_t maxlen) {
    (void)stdev;
    (void)maxlen;
    if (const char* s = std::getenv("MSPV_CSR_VEC")) {
        int v = std::atoi(s);
        if (v == 1 || v == 2 || v == 4 || v == 8 || v == 16 || v == 32) return v;
    }
    int v = 2;
    while (v < 32 && (double)v < mean) v <<= 1;
    return v;
}

static inline unsigned blocks_for(int64_t threads) {
    return (unsigned)((threads + kThreads - 1) / kThreads);
}

static int64_t vector_grid(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)kNumSMs * 8;
    if (b > cap) b = cap;
    return b < 1 ? 1 : b;
}

int64_t spmv_partials_needed(const mspv_matrix* A) {
    switch (A->format) {
        case MSPV_DIA: {
            const int rpt = A->value_type == MSPV_F64 ? 2 : (A->value_type == MSPV_F32 ? 4 : 8);
            return blocks_for((A->nrows + rpt - 1) / rpt);
        }
        case MSPV_CSR:
            return blocks_for((int64_t)A->nrows * A->csr_vector);
        default:
            return vector_grid(A->nrows);
    }
}

template <typename VT>
static void launch_dia(const mspv_matrix* A, const double* x, double* y, cudaStream_t s,
                       DotEpilogue ep) {
    constexpr int RPT = DiaVec<VT>::RPT;
    const unsigned grid = blocks_for((A->nrows + RPT - 1) / RPT);
    spmv_dia_kernel<VT><<<grid, kThreads, 0, s>>>(A->nrows, A->ndiags, A->npad, A->doff,
                                                  static_cast<const VT*>(A->av), x, y, ep);
}

template <typename VT>
static void launch_csr(const mspv_matrix* A, const double* x, double* y, cudaStream_t s,
                       DotEpilogue ep) {
    const int V = A->csr_vector;
    const unsigned grid = blocks_for((int64_t)A->nrows * V);
    const VT* av = static_cast<const VT*>(A->av);
#define MSPV_CSR_CASE(VV)                                                                 \
    case VV:                                                                              \
        spmv_csr_vector_kernel<VT, VV><<<grid, kThreads, 0, s>>>(A->nrows, A->irp, A->aj, \
                                                                 av, x, y, ep);           \
        break;
    switch (V) {
        MSPV_CSR_CASE(1)
        MSPV_CSR_CASE(2)
        MSPV_CSR_CASE(4)
        MSPV_CSR_CASE(8)
        MSPV_CSR_CASE(16)
        default:
        MSPV_CSR_CASE(32)
    }
#undef MSPV_CSR_CASE
}

template <typename VT>
static void launch_coo(const mspv_matrix* A, const double* x, double* y, cudaStream_t s,
                       DotEpilogue ep) {
    const VT* av = static_cast<const VT*>(A->av);
    spmv_coo_kernel<VT><<<blocks_for(A->nchunks * 32), kThreads, 0, s>>>(
        A->nrows, A->nnz, A->ai, A->aj, av, x, y, A->carry, A->nchunks, ep.st);
    if (A->nchunks > 1)
        spmv_coo_fixup_kernel<<<blocks_for(A->nchunks), kThreads, 0, s>>>(A->carry, A->nchunks, y, ep.st);
    if (ep.st)
        dot_alpha_kernel<<<(unsigned)vector_grid(A->nrows), kThreads, 0, s>>>(A->nrows, x, y, ep);
}

mspv_status launch_spmv(const mspv_matrix* A, const double* x, double* y, cudaStream_t s,
                        DotEpilogue ep) {
    if (A->nrows == 0) return MSPV_OK;
    if (A->format == MSPV_COO && A->nnz == 0) {
        if (ep.st) return set_error(MSPV_EINVAL, "cg: matrix has no entries");
        fill_zero_kernel<<<(unsigned)vector_grid(A->nrows), kThreads, 0, s>>>(y, A->nrows);
        MSPV_CUDA_TRY(cudaGetLastError());
        return MSPV_OK;
    }
    const int vt = A->value_type;
    switch (A->format) {
        case MSPV_DIA:
            if (vt == MSPV_F64) launch_dia<double>(A, x, y, s, ep);
            else if (vt == MSPV_F32) launch_dia<float>(A, x, y, s, ep);
            else launch_dia<__nv_bfloat16>(A, x, y, s, ep);
            break;
        case MSPV_CSR:
            if (vt == MSPV_F64) launch_csr<double>(A, x, y, s, ep);
            else if (vt == MSPV_F32) launch_csr<float>(A, x, y, s, ep);
            else launch_csr<__nv_bfloat16>(A, x, y, s, ep);
            break;
        default:
            if (vt == MSPV_F64) launch_coo<double>(A, x, y, s, ep);
            else if (vt == MSPV_F32) launch_coo<float>(A, x, y, s, ep);
            else launch_coo<__nv_bfloat16>(A, x, y, s, ep);
            break;
    }
    MSPV_CUDA_TRY(cudaGetLastError());
    return MSPV_OK;
}

}  // namespace mspv
