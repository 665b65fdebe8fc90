// SpMV kernels for the three storage formats of Sec. II-B, y = A x (or y += A x), FP64
// arithmetic, plus the FP32-arithmetic kernels of the refinement's inner solver.
//
// On GB300 the FP64 pipe, not HBM, is the tighter limit for FP64 SpMV: one FP64 FMA
// per stored value is about as fast as HBM delivers that value, a warp instruction
// costs the same however many of its lanes are active, and the FP32 -> FP64
// conversion instruction issues on the same narrow pipe. Every kernel here therefore
// spends one FMA per value it must multiply with as many lanes busy as it can, widens
// FP32/BF16 values with integer instructions, and keeps FP64 shuffle reductions short.
//
//  DIA (Algorithm 3): diagonal-major values; each thread owns RPT consecutive rows
//      (FP64 arithmetic: 2 rows for FP64 values, 4 for FP32, 8 for BF16, one 128-bit
//      value load per diagonal) and walks the diagonals in order with the predicate
//      0 <= k < N -- the row-parallel, diagonal-sequential structure of the paper's
//      outer-loop SVE vectorisation (Sec. III), with warp lanes in place of SVE lanes.
//      The FP32-arithmetic kernel reads one x window per run of consecutive offsets, at
//      4 rows per thread for FP32 values and 8 (one 16-byte value load per diagonal,
//      kept packed until its FMAs) for BF16 values.
//  CSR (Algorithm 2): V lanes per row (V = 4 for short rows, chosen from the row-length
//      statistics). Up to V = 8 a warp owns 32 rows, runs V passes of 32 / V rows with
//      lane-strided FMAs and joins the passes' partial sums with one reduce-scatter
//      (V - 1 FP64 adds per lane); wider rows take a log2(V)-step shuffle reduction per
//      pass. Rows longer than 32 V entries are listed at conversion and reduced by one CTA
//      each. Inside CG the grid is capped and the warps stride. Kernels that stage values
//      and gathered x through shared memory (warp slices, CTA row blocks) are selectable.
//  COO (Algorithm 1): rows of at most 128 entries, at least 4 per row on average, take the
//      row-block kernel (a warp per 32 rows, whose entries a table of block starts gives;
//      row starts marked from the row indices, then the CSR kernel's FMA phase); sparser
//      short rows the run-vector kernel (a warp per 256 sorted entries: ballot-compacted run
//      starts, then 4 lanes per run); longer rows the lane-sequential segment kernel (16
//      entries per lane summed in order, a segmented scan joins rows across lanes) -- forms
//      of the paper's SVE COO idea of reducing runs of equal row index. Runs cut by a chunk
//      edge leave partial sums in a carry record that a fix-up pass adds in chunk order. A
//      staged window kernel serves the allocation-free entry point.
// No floating-point atomics anywhere: y is bit-identical run to run. Inside CG each
// SpMV kernel writes its CTA's partial of p.q (DotEpilogue); the partials are summed in
// index order by a one-CTA kernel. store_y is the single place a row of y is written
// (overwrite, or add for the accumulating SpMV).
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <string>

#include "internal.cuh"

namespace mspv {

constexpr int kStageCap = 3072;   // entries staged per CTA (values + gathered x)
constexpr int kLongRun = 128;     // runs longer than this are reduced by the whole CTA
constexpr int kMaxLongRuns = kStageCap / (kLongRun + 1) + 1;
constexpr int kRsCap = kStageCap + 4;   // run starts (+1 sentinel), padded so srow stays 16-byte aligned
static_assert(kCooWindow <= kStageCap, "COO window must fit the staging buffers");

// ---------------------------------------------------------------------------
// DIA
// ---------------------------------------------------------------------------
template <typename VT, typename T> struct DiaVec;
template <> struct DiaVec<double, double> {
    static constexpr int RPT = 2;
    __device__ __forceinline__ static void load(const double* p, double (&v)[RPT]) {
        const double2 t = __ldcs(reinterpret_cast<const double2*>(p));
        v[0] = t.x; v[1] = t.y;
    }
};
template <> struct DiaVec<float, double> {
    static constexpr int RPT = 4;
    __device__ __forceinline__ static void load(const float* p, double (&v)[RPT]) {
        const uint4 t = __ldcs(reinterpret_cast<const uint4*>(p));
        v[0] = widen_f32_bits(t.x); v[1] = widen_f32_bits(t.y);
        v[2] = widen_f32_bits(t.z); v[3] = widen_f32_bits(t.w);
    }
};
template <> struct DiaVec<__nv_bfloat16, double> {
    static constexpr int RPT = 8;
    __device__ __forceinline__ static void load(const __nv_bfloat16* p, double (&v)[RPT]) {
        const uint4 t = __ldcs(reinterpret_cast<const uint4*>(p));
        const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[2 * k] = widen_f32_bits(w[k] << 16);
            v[2 * k + 1] = widen_f32_bits(w[k] & 0xffff0000u);
        }
    }
};
// FP32 arithmetic: one 16-byte load per diagonal, kept packed (`raw`) until `unpack` turns it
// into RPT floats next to the FMAs that use them.
template <> struct DiaVec<float, float> {
    static constexpr int RPT = 4;
    __device__ __forceinline__ static uint4 raw(const float* p) { return __ldcs(reinterpret_cast<const uint4*>(p)); }
    __device__ __forceinline__ static void unpack(uint4 t, float (&v)[RPT]) {
        v[0] = __uint_as_float(t.x); v[1] = __uint_as_float(t.y);
        v[2] = __uint_as_float(t.z); v[3] = __uint_as_float(t.w);
    }
    __device__ __forceinline__ static void load(const float* p, float (&v)[RPT]) { unpack(raw(p), v); }
};
template <> struct DiaVec<__nv_bfloat16, float> {
    static constexpr int RPT = 8;   // a 16-byte value load per diagonal (half the requests of 4 rows)
    __device__ __forceinline__ static uint4 raw(const __nv_bfloat16* p) {
        return __ldcs(reinterpret_cast<const uint4*>(p));
    }
    __device__ __forceinline__ static void unpack(uint4 t, float (&v)[RPT]) {
        const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[2 * k] = __uint_as_float(w[k] << 16);
            v[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
        }
    }
    __device__ __forceinline__ static void load(const __nv_bfloat16* p, float (&v)[RPT]) { unpack(raw(p), v); }
};

constexpr int kDiaSmemDiags = 256;   // offsets cached in shared memory; more are read from global

// FMA in the arithmetic type (T = double: the FP64 path; T = float: the FP32-arithmetic
// path of the inner solver of mixed-precision refinement).
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
// Exact FP32 -> FP64 of a per-thread FP32 partial, with integer operations.
__device__ __forceinline__ double to_f64_exact(double v) { return v; }
__device__ __forceinline__ double to_f64_exact(float v) { return widen_f32_bits(__float_as_uint(v)); }

// Sum over the CTA in T (thread 0 holds the result); smem holds kThreads values.
template <typename T>
__device__ __forceinline__ T block_sum_t(T v, T* smem) {
    smem[threadIdx.x] = v;
    __syncthreads();
    T t = T(0);
    if (threadIdx.x < 32) {
        t = smem[threadIdx.x];
#pragma unroll
        for (int k = 1; k < kThreads / 32; ++k) t += smem[threadIdx.x + 32 * k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;
}

// Sum over a CTA of NT threads in T (thread 0 holds the result); smem holds NT values.
template <typename T, int NT>
__device__ __forceinline__ T block_sum_nt(T v, T* smem) {
    smem[threadIdx.x] = v;
    __syncthreads();
    T t = T(0);
    if (threadIdx.x < 32) {
        t = smem[threadIdx.x];
#pragma unroll
        for (int k = 1; k < NT / 32; ++k) t += smem[threadIdx.x + 32 * k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;
}

template <typename T, int NT>
__device__ __forceinline__ void finish_dot_nt(T dot, DotEpilogue ep) {
    __shared__ T s_dot[NT];
    const T cta = block_sum_nt<T, NT>(dot, s_dot);
    if (threadIdx.x == 0) ep.partials[blockIdx.x] = to_f64_exact(cta);
}

// Dot epilogue (CG's p.q): the CTA sums its threads' partials (in T) and thread 0 writes
// the CTA total, in FP64, to ep.partials[blockIdx.x]. The cross-CTA sum is a separate
// one-CTA kernel: no fence or atomic holds the CTA here.
template <typename T>
__device__ __forceinline__ void finish_dot(T dot, DotEpilogue ep) {
    __shared__ T s_dot[kThreads];
    const T cta = block_sum_t(dot, s_dot);
    if (threadIdx.x == 0) ep.partials[blockIdx.x] = to_f64_exact(cta);
}

// One thread per RPT consecutive rows, one CTA per strip of kThreads * RPT rows.
// ACC: y += A x (accumulating SpMV), a template argument so the y = A x path has no test
// in its store.
template <typename VT, typename T, bool ACC>
__global__ void __launch_bounds__(kThreads) spmv_dia_kernel(
    int32_t n, int32_t ndiags, int32_t npad, const int32_t* __restrict__ doff,
    const VT* __restrict__ av, const T* __restrict__ x, T* __restrict__ y, DotEpilogue ep) {
    constexpr int RPT = DiaVec<VT, T>::RPT;
    pdl_wait();
    pdl_trigger();
    if (ep.st && ep.st->done) return;   // uniform: CG already finished
    __shared__ int32_t s_off[kDiaSmemDiags];
    for (int k = threadIdx.x; k < ndiags && k < kDiaSmemDiags; k += kThreads) s_off[k] = doff[k];
    __syncthreads();

    const int64_t i0 = ((int64_t)blockIdx.x * kThreads + threadIdx.x) * RPT;
    T acc[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) acc[r] = T(0);
    T d = T(0);
    if (i0 < n) {
        const VT* col = av + i0;
#pragma unroll 3
        for (int j = 0; j < ndiags; ++j) {
            const int32_t off = (j < kDiaSmemDiags) ? s_off[j] : __ldg(doff + j);
            T a[RPT];
            DiaVec<VT, T>::load(col + (int64_t)j * npad, a);
            const int64_t k0 = i0 + off;
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                const int64_t k = k0 + r;
                if (k >= 0 && k < n) acc[r] = fma_t(a[r], __ldg(x + k), acc[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            if (i0 + r < n) {
                store_y(y, i0 + r, acc[r], ACC);
                if (ep.st) d = fma_t(__ldg(x + i0 + r), acc[r], d);
            }
        }
    }
    if (ep.st) finish_dot(d, ep);
}

// FP32-arithmetic DIA (inner solver of mixed-precision refinement; x and y are the
// library's own 16-byte-aligned FP32 vectors). Bound by loads, not arithmetic: the diagonals
// go in runs of consecutive offsets (at most 3, found at conversion; the 27-point stencil has
// 9 runs of 3), and one 12-float x window serves a whole run: the window starts at the first
// offset's index rounded down to a multiple of 4 and each diagonal t of the run picks its
// values at the shift m + t (m = that offset's index & 3, the same for the whole warp).
template <int M, int RPT, int W>
__device__ __forceinline__ void dia_f32_fma(const float (&a)[RPT], const float (&w)[W], float (&acc)[RPT]) {
    static_assert(M + RPT <= W, "window too short for the shift");
#pragma unroll
    for (int r = 0; r < RPT; ++r) acc[r] = fmaf(a[r], w[M + r], acc[r]);
}

// CTA size of the FP32-arithmetic DIA kernel: 256 threads, 8 rows per thread with BF16 values
// (48 registers, 2,048 rows per CTA) and 4 with FP32 values (1,024 rows). Inside CG the BF16
// strips of 2,048 rows halve the partials the alpha kernel sums against 128-thread CTAs of
// 1,024 rows (same SpMV time; reliable updates at 192^3 48.5 vs 49.1 ms).
template <typename VT> struct DiaF32Shape { static constexpr int NT = kThreads; };

template <typename VT>
__global__ void __launch_bounds__(DiaF32Shape<VT>::NT) spmv_dia_f32_kernel(
    int32_t n, int32_t ndiags, int32_t npad, const int32_t* __restrict__ doff, const int2* __restrict__ runs,
    int32_t nruns, const VT* __restrict__ av, const float* __restrict__ x, float* __restrict__ y, DotEpilogue ep) {
    constexpr int RPT = DiaVec<VT, float>::RPT;   // 4 (FP32 values) or 8 (BF16 values)
    constexpr int NT = DiaF32Shape<VT>::NT;
    static_assert(RPT == 4 || RPT == 8, "x windows come in whole float4s");
    constexpr int W = RPT + 8;                     // shift m + t <= 5 plus RPT rows, in float4s
    pdl_wait();
    pdl_trigger();
    if (ep.st && ep.st->done) return;
    // At 8 rows per thread the run table sits in shared memory, so that no global load heads
    // each run (192^3 BF16: 75.7 vs 86.3 us); at 4 rows the global read measured faster.
    constexpr bool kRunsInSmem = RPT == 8;
    __shared__ int32_t s_off[kDiaSmemDiags];
    __shared__ int2 s_runs[kRunsInSmem ? kDiaSmemDiags : 1];
    for (int k = threadIdx.x; k < ndiags && k < kDiaSmemDiags; k += NT) s_off[k] = doff[k];
    if constexpr (kRunsInSmem)
        for (int k = threadIdx.x; k < nruns && k < kDiaSmemDiags; k += NT) s_runs[k] = runs[k];
    __syncthreads();
    const int64_t i0 = ((int64_t)blockIdx.x * NT + threadIdx.x) * RPT;
    float acc[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) acc[r] = 0.0f;
    if (i0 < n) {
        const VT* col = av + i0;
        for (int q = 0; q < nruns; ++q) {
            const int2 run = (kRunsInSmem && q < kDiaSmemDiags) ? s_runs[q] : __ldg(runs + q);
            const int j0 = run.x, len = run.y;
            // The run's value loads are issued together and stay packed until their diagonal's
            // FMAs: unpacked all at once, the BF16 kernel held 56 registers (9 CTAs per SM);
            // packed it holds 48 (10 CTAs) and the 192^3 SpMV takes 67.6 instead of 77.9 us.
            uint4 araw[3];
#pragma unroll
            for (int t = 0; t < 3; ++t)
                araw[t] = t < len ? DiaVec<VT, float>::raw(col + (int64_t)(j0 + t) * npad) : make_uint4(0u, 0u, 0u, 0u);
            float a[RPT];
            const int32_t off = (j0 < kDiaSmemDiags) ? s_off[j0] : __ldg(doff + j0);
            const int64_t k0 = i0 + off;
            const int m = (int)(k0 & 3);
            const int64_t base = k0 - m;
            if (base >= 0 && base + W <= n) {
                float w[W];
#pragma unroll
                for (int u = 0; u < W / 4; ++u) {
                    const float4 t4 = __ldg(reinterpret_cast<const float4*>(x + base) + u);
                    w[4 * u] = t4.x; w[4 * u + 1] = t4.y; w[4 * u + 2] = t4.z; w[4 * u + 3] = t4.w;
                }
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    if (t < len) {
                        DiaVec<VT, float>::unpack(araw[t], a);
                        switch (m + t) {   // uniform across the warp
                            case 0: dia_f32_fma<0>(a, w, acc); break;
                            case 1: dia_f32_fma<1>(a, w, acc); break;
                            case 2: dia_f32_fma<2>(a, w, acc); break;
                            case 3: dia_f32_fma<3>(a, w, acc); break;
                            case 4: dia_f32_fma<4>(a, w, acc); break;
                            default: dia_f32_fma<5>(a, w, acc); break;
                        }
                    }
                }
            } else {   // a strip touching either end of x
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    if (t < len) {
                        DiaVec<VT, float>::unpack(araw[t], a);
#pragma unroll
                        for (int r = 0; r < RPT; ++r) {
                            const int64_t k = k0 + t + r;
                            if (k >= 0 && k < n) acc[r] = fmaf(a[r], __ldg(x + k), acc[r]);
                        }
                    }
                }
            }
        }
    }
    float d = 0.0f;
    if (!ep.acc && i0 + RPT <= n) {   // the vector store overwrites; accumulation goes below
#pragma unroll
        for (int u = 0; u < RPT / 4; ++u) {
            reinterpret_cast<float4*>(y + i0)[u] =
                make_float4(acc[4 * u], acc[4 * u + 1], acc[4 * u + 2], acc[4 * u + 3]);
            if (ep.st) {
                const float4 xv = __ldg(reinterpret_cast<const float4*>(x + i0) + u);
                d = fmaf(xv.x, acc[4 * u], d);
                d = fmaf(xv.y, acc[4 * u + 1], d);
                d = fmaf(xv.z, acc[4 * u + 2], d);
                d = fmaf(xv.w, acc[4 * u + 3], d);
            }
        }
    } else if (i0 < n) {
#pragma unroll
        for (int r = 0; r < RPT; ++r)
            if (i0 + r < n) {
                store_y(y, i0 + r, acc[r], ep.acc);
                if (ep.st) d = fmaf(__ldg(x + i0 + r), acc[r], d);
            }
    }
    if (ep.st) finish_dot_nt<float, NT>(d, ep);
}

// ---------------------------------------------------------------------------
// CSR, V lanes per row (long rows)
// ---------------------------------------------------------------------------
template <typename T, typename VT>
__device__ __forceinline__ T convert_value(VT v) {
    if constexpr (sizeof(T) == 8) return widen(v);
    else if constexpr (sizeof(VT) == 4) return v;
    else return __uint_as_float((uint32_t)__bfloat16_as_ushort(v) << 16);
}

// The FMA phase of the 32-row CSR and COO kernels. A warp owns 32 consecutive rows; lane
// (grp, sub) = (lane / V, lane % V) keeps V partial sums, one for each of the rows R t + grp
// (t < V, R = 32 / V rows per pass of the warp). The passes run one after another, each like a
// V-lanes-per-row pass over R consecutive rows (lane-strided FMAs, R segments of V consecutive
// values per load instruction), but the partial sums are not reduced per pass: a reduce-scatter
// at the end joins the V lanes of every row. At each of its log2(V) steps a lane keeps half of
// its partials, receives its partner's copy of that half and adds it, so lane (grp, sub) ends
// with the whole sum of row R sub + grp after V - 1 FP64 adds. A shuffle-add reduction after every pass costs log2(V)
// adds per pass, V log2(V) per 32 rows (8 against 3 for V = 4): on GB300's narrow FP64 pipe
// those adds are a fifth of a 27-entry row's FMA instructions.
// The matrix is read through the read-only path with normal cache priority: a row may start at
// any entry, so a lane group's V values often straddle two 32-byte sectors and the same warp's
// next load uses the rest. With streaming (evict-first) loads that remainder was often gone
// from L1 and the kernels ran 1.2-1.3x slower (192^3 stencil); an evict-first hint for L2
// alone was slower still inside the benchmark step.
// bounds(t, s, len) gives the first entry and the length of row R t + grp (len 0: a row written
// elsewhere); every lane calls it for every t outside divergent code, so it may shuffle.
template <typename VT, typename T, int V, typename Bounds>
__device__ __forceinline__ T rows32_sum(int sub, const int32_t* __restrict__ aj, const VT* __restrict__ av,
                                        const T* __restrict__ x, Bounds bounds) {
    const unsigned FULL = 0xffffffffu;
    T part[V];
#pragma unroll
    for (int t = 0; t < V; ++t) {
        int32_t s0, len;
        bounds(t, s0, len);
        T acc = T(0);
        for (int32_t off = sub; off < len; off += V) {
            const int64_t j = (int64_t)s0 + off;
            acc = fma_t(convert_value<T>(__ldg(av + j)), __ldg(x + __ldg(aj + j)), acc);
        }
        part[t] = acc;
    }
#pragma unroll
    for (int h = V / 2; h >= 1; h >>= 1) {
        const bool upper = (sub & h) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const T give = upper ? part[i] : part[i + h];
            const T keep = upper ? part[i + h] : part[i];
            part[i] = keep + __shfl_xor_sync(FULL, give, h);
        }
    }
    return part[0];
}

// CSR with V lanes per row (V = 1, 2, 4, 8), a warp per 32 consecutive rows (rows32_sum).
// The warp's 33 row pointers come from one coalesced load spread by shuffles. Rows longer
// than long_len are skipped here and reduced by spmv_csr_long_kernel. Lane (grp, sub) writes
// row R sub + grp of the warp: the 32 stores of a warp land in one 256-byte span.
template <typename VT, typename T, int V, bool STRIDE>
__global__ void __launch_bounds__(kThreads) spmv_csr_rows32_kernel(
    int32_t nrows, const int32_t* __restrict__ irp, const int32_t* __restrict__ aj,
    const VT* __restrict__ av, const T* __restrict__ x, T* __restrict__ y, int32_t long_len,
    DotEpilogue ep) {
    static_assert(V == 1 || V == 2 || V == 4 || V == 8, "lanes per row");
    constexpr int R = 32 / V;
    pdl_wait();
    pdl_trigger();
    if (ep.st && ep.st->done) return;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, sub = lane & (V - 1), grp = lane / V;
    const int64_t warp = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    // Inside CG (STRIDE) the grid is capped so the scalar kernels have fewer partials to sum,
    // and the warps stride over the rows, 32 rows per warp and pass.
    const int64_t step = STRIDE ? (int64_t)gridDim.x * kThreads : 0;
    T dot = T(0);
    for (int64_t base = warp * 32; base < nrows; base += step) {
        const int32_t p = __ldg(irp + min(base + lane, (int64_t)nrows));
        const int32_t pend = __ldg(irp + min(base + 32, (int64_t)nrows));
        const T sum = rows32_sum<VT, T, V>(sub, aj, av, x, [=](int t, int32_t& s0, int32_t& len) {
            const int r = R * t + grp;
            const int32_t a = __shfl_sync(FULL, p, r);
            const int32_t b1 = __shfl_sync(FULL, p, (r + 1) & 31);
            const int32_t l = (r == 31 ? pend : b1) - a;
            s0 = a;
            len = l > long_len ? 0 : l;
        });
        const int rr = R * sub + grp;
        const int32_t a = __shfl_sync(FULL, p, rr);
        const int32_t b1 = __shfl_sync(FULL, p, (rr + 1) & 31);
        const int64_t row = base + rr;
        if (row < nrows && (rr == 31 ? pend : b1) - a <= long_len) {
            store_y(y, row, sum, ep.acc);
            if (ep.st) dot = fma_t(__ldg(x + row), sum, dot);
        }
        if (!STRIDE) break;
    }
    if (ep.st) finish_dot(dot, ep);
}

// V lanes per row for wide rows (V = 16, 32), lane-strided FMAs and a log2(V)-step shuffle
// reduction per pass of 32 / V rows. Rows longer than long_len are skipped here and reduced by
// spmv_csr_long_kernel.
template <typename VT, typename T, int V, bool STRIDE>
__global__ void __launch_bounds__(kThreads) spmv_csr_vector_kernel(
    int32_t nrows, const int32_t* __restrict__ irp, const int32_t* __restrict__ aj,
    const VT* __restrict__ av, const T* __restrict__ x, T* __restrict__ y, int32_t long_len,
    DotEpilogue ep) {
    pdl_wait();
    pdl_trigger();
    if (ep.st && ep.st->done) return;
    // One V-lane group per row. Inside CG (STRIDE) the grid is capped, so the scalar kernels
    // have fewer partials to sum, and the groups stride over the rows; the loop bound is the
    // warp's first row, so all 32 lanes run every shuffle together.
    const int lane = threadIdx.x & (V - 1);
    const int grp = (threadIdx.x & 31) / V;
    const int64_t warp_row0 = ((int64_t)blockIdx.x * kThreads + (threadIdx.x & ~31)) / V;
    const int64_t stride = STRIDE ? (int64_t)gridDim.x * (kThreads / V) : 0;
    T dot = T(0);
    for (int64_t base = warp_row0; base < nrows; base += stride) {
        const int64_t row = base + grp;
        T sum = T(0);
        bool mine = row < nrows;
        if (mine) {
            const int32_t s = __ldg(irp + row), e = __ldg(irp + row + 1);
            if (e - s > long_len) {
                mine = false;   // written by the long-row kernel
            } else {
                for (int64_t j = s + lane; j < e; j += V)
                    sum = fma_t(convert_value<T>(__ldcs(av + j)), __ldg(x + __ldcs(aj + j)), sum);
            }
        }
#pragma unroll
        for (int o = V / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0 && mine) {
            store_y(y, row, sum, ep.acc);
            if (ep.st) dot = fma_t(x[row], sum, dot);
        }
        if (!STRIDE) break;
    }
    if (ep.st) finish_dot(dot, ep);
}

// One CTA per long row (listed at conversion): strided FMAs, then a CTA reduction.
template <typename VT, typename T>
__global__ void __launch_bounds__(kThreads) spmv_csr_long_kernel(
    const int32_t* __restrict__ long_rows, const int32_t* __restrict__ irp, const int32_t* __restrict__ aj,
    const VT* __restrict__ av, const T* __restrict__ x, T* __restrict__ y, DotEpilogue ep) {
    pdl_wait();
    pdl_trigger();
    if (ep.st && ep.st->done) return;
    __shared__ T s_red[kThreads];
    const int32_t row = long_rows[blockIdx.x];
    const int32_t s = __ldg(irp + row), e = __ldg(irp + row + 1);
    T part = T(0);
    for (int64_t j = s + threadIdx.x; j < e; j += kThreads)
        part = fma_t(convert_value<T>(__ldcs(av + j)), __ldg(x + __ldcs(aj + j)), part);
    const T sum = block_sum_t(part, s_red);
    if (threadIdx.x == 0) {
        store_y(y, row, sum, ep.acc);
        if (ep.st) ep.partials[blockIdx.x] = to_f64_exact(x[row] * sum);
    }
}

// Rows longer than long_len, listed in order: flag, scan, compact.
__global__ void csr_long_flag_kernel(const int32_t* __restrict__ irp, int32_t n, int32_t long_len,
                                     int32_t* __restrict__ flags) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        flags[r] = (irp[r + 1] - irp[r] > long_len) ? 1 : 0;
}
__global__ void csr_long_compact_kernel(const int32_t* __restrict__ flags, const int32_t* __restrict__ pos,
                                        int32_t n, int32_t* __restrict__ out) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        if (flags[r]) out[pos[r]] = (int32_t)r;
}

// ---------------------------------------------------------------------------
// Staged run-per-thread reduction (CSR and COO), generic in the arithmetic type T:
// T = double is the FP64 path; T = float is the FP32-arithmetic path used by the inner
// solver of mixed-precision refinement (FP32/BF16 values, FP32 vectors).
// ---------------------------------------------------------------------------
// Asynchronous global -> shared copies (LDGSTS). Completion is awaited with
// cp.async.wait_group, a hardware wait on the issuing thread's own copies.
template <int N>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
    static_assert(N == 4 || N == 8, "copy size");
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (N == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) { cp_async<4>(smem, gmem); }
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}


// Value slot k of the staging buffer as T. Values of the arithmetic type's size are
// staged as is; FP32 values on the FP64 path are staged as their 4 raw bytes and widened
// here; BF16 values are converted while staging.
template <typename VT, typename T>
__device__ __forceinline__ T staged_value(const T* a_s, int k) {
    if constexpr (sizeof(VT) == 4 && sizeof(T) == 8)
        return widen_f32_bits(reinterpret_cast<const uint32_t*>(a_s + k)[0]);
    else
        return a_s[k];
}

// Stage a window: a_s[k] = av[s+k], x_s[k] = x[aj[s+k]]. Every copy of a phase is in
// flight at once: first the values and column indices (the index lands in x_s[k]'s
// slot), then, per thread and for its own slots only, the gathers of x.
template <typename VT, typename T>
__device__ __forceinline__ void stage_window(const int32_t* __restrict__ aj,
                                             const VT* __restrict__ av,
                                             const T* __restrict__ x, int64_t s, int len,
                                             T* __restrict__ a_s, T* __restrict__ x_s) {
    constexpr int STRIDE = sizeof(T) / 4;   // int32 slots per staged entry
    int32_t* slot_idx = reinterpret_cast<int32_t*>(x_s);
    for (int k = threadIdx.x; k < len; k += kThreads) {
        if constexpr (sizeof(VT) == sizeof(T)) cp_async<sizeof(T)>(a_s + k, av + s + k);
        else if constexpr (sizeof(VT) == 4) cp_async4(a_s + k, av + s + k);
        else a_s[k] = convert_value<T>(__ldcs(av + s + k));
        cp_async4(slot_idx + STRIDE * k, aj + s + k);
    }
    cp_async_wait_all();
    for (int k = threadIdx.x; k < len; k += kThreads) cp_async<sizeof(T)>(x_s + k, x + slot_idx[STRIDE * k]);
    cp_async_wait_all();
}

// Left-to-right FMA chain over staged entries [b, e).
template <typename VT, typename T>
__device__ __forceinline__ T run_fma(const T* __restrict__ a_s, const T* __restrict__ x_s, int b, int e) {
    T sum = T(0);
    int j = b;
    for (; j + 4 <= e; j += 4) {
        sum = fma_t(staged_value<VT>(a_s, j), x_s[j], sum);
        sum = fma_t(staged_value<VT>(a_s, j + 1), x_s[j + 1], sum);
        sum = fma_t(staged_value<VT>(a_s, j + 2), x_s[j + 2], sum);
        sum = fma_t(staged_value<VT>(a_s, j + 3), x_s[j + 3], sum);
    }
    for (; j < e; ++j) sum = fma_t(staged_value<VT>(a_s, j), x_s[j], sum);
    return sum;
}


// Exclusive scan of one int per thread over the CTA; *total gets the sum.
__device__ __forceinline__ int block_excl_scan(int v, int* s_warp, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int w = (lane < kThreads / 32) ? s_warp[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < kThreads / 32) s_warp[lane] = wi - w;
        if (lane == kThreads / 32 - 1) s_warp[kThreads / 32] = wi;
    }
    __syncthreads();
    const int r = incl - v + s_warp[warp];
    *total = s_warp[kThreads / 32];
    __syncthreads();
    return r;
}

// Sum every run [rs[i], rs[i+1]) of the staged window, calling emit(i, sum) once per
// run: runs up to kLongRun entries in one thread each, longer runs by the whole CTA.
template <typename VT, typename T, typename Emit>
__device__ __forceinline__ void reduce_runs(const T* __restrict__ a_s, const T* __restrict__ x_s,
                                            const int32_t* __restrict__ rs, int nruns, Emit emit) {
    __shared__ int s_long[kMaxLongRuns];
    __shared__ int s_nlong;
    __shared__ T s_red_t[kThreads];
    if (threadIdx.x == 0) s_nlong = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < nruns; i += kThreads) {
        const int b = rs[i], e = rs[i + 1];
        if (e - b > kLongRun) {
            s_long[atomicAdd(&s_nlong, 1)] = i;   // processing order only; results unaffected
            continue;
        }
        emit(i, run_fma<VT>(a_s, x_s, b, e));
    }
    __syncthreads();
    const int nlong = s_nlong;
    for (int l = 0; l < nlong; ++l) {
        const int i = s_long[l];
        const int b = rs[i], e = rs[i + 1];
        T part = T(0);
        for (int j = b + threadIdx.x; j < e; j += kThreads) part = fma_t(staged_value<VT>(a_s, j), x_s[j], part);
        const T sum = block_sum_t(part, s_red_t);
        if (threadIdx.x == 0) emit(i, sum);
    }
}

template <typename T>
constexpr size_t csr_smem() { return 2 * kStageCap * sizeof(T) + kRsCap * sizeof(int32_t); }
template <typename T>
constexpr size_t coo_smem() { return csr_smem<T>() + kStageCap * sizeof(int32_t); }
static_assert(csr_smem<double>() % 16 == 0 && csr_smem<float>() % 16 == 0, "srow alignment");

// CSR: CTA b takes rows [row_block[b], row_block[b+1]), the rows whose first entry lies
// in entry window b. Blocks too large to stage are reduced row by row by the whole CTA.
template <typename VT, typename T>
__global__ void __launch_bounds__(kThreads) spmv_csr_stage_kernel(
    const int32_t* __restrict__ irp, const int32_t* __restrict__ aj, const VT* __restrict__ av,
    const int32_t* __restrict__ row_block, const T* __restrict__ x, T* __restrict__ y,
    DotEpilogue ep) {
    pdl_wait();
    pdl_trigger();
    if (ep.st && ep.st->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* a_s = reinterpret_cast<T*>(smem_raw);
    T* x_s = a_s + kStageCap;
    int32_t* rs = reinterpret_cast<int32_t*>(x_s + kStageCap);
    __shared__ T s_red_t[kThreads];
    const int32_t rb = row_block[blockIdx.x], re = row_block[blockIdx.x + 1];
    const int nr = re - rb;
    T dot = T(0);
    if (nr > 0) {
        const int32_t s = __ldg(irp + rb), e = __ldg(irp + re);
        const int len = e - s;
        if (len <= kStageCap && nr <= kStageCap) {
            for (int i = threadIdx.x; i <= nr; i += kThreads) rs[i] = __ldg(irp + rb + i) - s;
            stage_window(aj, av, x, s, len, a_s, x_s);
            __syncthreads();
            reduce_runs<VT>(a_s, x_s, rs, nr, [&](int i, T sum) {
                store_y(y, rb + i, sum, ep.acc);
                if (ep.st) dot = fma_t(x[rb + i], sum, dot);
            });
        } else {
            for (int32_t r = rb; r < re; ++r) {   // uniform over the CTA
                const int32_t a = __ldg(irp + r), b = __ldg(irp + r + 1);
                if (a == b) {
                    if (threadIdx.x == 0) zero_y(y, r, ep.acc);
                    continue;
                }
                T part = T(0);
                for (int64_t j = a + threadIdx.x; j < b; j += kThreads)
                    part = fma_t(convert_value<T>(__ldcs(av + j)), __ldg(x + __ldcs(aj + j)), part);
                const T sum = block_sum_t(part, s_red_t);
                if (threadIdx.x == 0) {
                    store_y(y, r, sum, ep.acc);
                    if (ep.st) dot = fma_t(x[r], sum, dot);
                }
            }
        }
    }
    if (ep.st) finish_dot(dot, ep);
}

// CSR, warp-private staging. Warp w of the grid takes row groups of 32 consecutive rows
// (grid-stride); lane l owns row 32g + l. The group's entries [irp[32g], irp[32g+32))
// are staged through the warp's own slice of shared memory in chunks of WCAP entries
// (values with cp.async, column indices into the x slots, then the x gathers), and each
// lane adds the FMAs of its row's part of the chunk, left to right. Warps synchronise
// only with __syncwarp, so one warp's loads overlap another's FMAs, and all 32 lanes
// work on rows of similar length (FP64 issue slots are spent on full warps). A group
// holding a row longer than kWarpLongRow is reduced row by row by the whole warp.
constexpr int kWarpLongRow = 256;
template <typename T, int WCAP, int NT>
constexpr size_t csr_warp_smem() { return (size_t)(NT / 32) * 2 * WCAP * sizeof(T); }

template <typename VT, typename T, int WCAP, int NT>
__global__ void __launch_bounds__(NT) spmv_csr_warp_kernel(
    int32_t nrows, const int32_t* __restrict__ irp, const int32_t* __restrict__ aj, const VT* __restrict__ av,
    const T* __restrict__ x, T* __restrict__ y, DotEpilogue ep) {
    pdl_wait();
    pdl_trigger();
    if (ep.st && ep.st->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T* a_s = reinterpret_cast<T*>(smem_raw) + (size_t)warp * 2 * WCAP;
    T* x_s = a_s + WCAP;
    constexpr int STRIDE = sizeof(T) / 4;
    int32_t* slot_idx = reinterpret_cast<int32_t*>(x_s);
    const int64_t ngroups = ((int64_t)nrows + 31) / 32;
    const int64_t wstride = (int64_t)gridDim.x * (NT / 32);
    T dot = T(0);
    for (int64_t g = (int64_t)blockIdx.x * (NT / 32) + warp; g < ngroups; g += wstride) {
        const int64_t r0 = g * 32;
        const int64_t row = r0 + lane;
        const bool has_row = row < nrows;
        const int32_t myb = has_row ? __ldg(irp + row) : 0;
        const int32_t mye = has_row ? __ldg(irp + row + 1) : 0;
        const int nr = (int)((nrows - r0 < 32) ? nrows - r0 : 32);
        const int32_t s = __shfl_sync(0xffffffffu, myb, 0);
        const int32_t e = __shfl_sync(0xffffffffu, mye, nr - 1);
        const bool long_row = has_row && (mye - myb > kWarpLongRow);
        if (__any_sync(0xffffffffu, long_row)) {
            // whole warp per row: lane-strided FMAs, then a shuffle reduction
            for (int q = 0; q < nr; ++q) {
                const int32_t a = __shfl_sync(0xffffffffu, myb, q), b = __shfl_sync(0xffffffffu, mye, q);
                T part = T(0);
                for (int64_t j = a + lane; j < b; j += 32)
                    part = fma_t(convert_value<T>(__ldcs(av + j)), __ldg(x + __ldcs(aj + j)), part);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                if (lane == q) {
                    store_y(y, row, part, ep.acc);
                    if (ep.st) dot = fma_t(x[row], part, dot);
                }
            }
            continue;
        }
        T sum = T(0);
        for (int64_t c0 = s; c0 < e; c0 += WCAP) {
            const int len = (int)((e - c0 < WCAP) ? e - c0 : WCAP);
            for (int k = lane; k < len; k += 32) {
                if constexpr (sizeof(VT) == sizeof(T)) cp_async<sizeof(T)>(a_s + k, av + c0 + k);
                else if constexpr (sizeof(VT) == 4) cp_async4(a_s + k, av + c0 + k);
                else a_s[k] = convert_value<T>(__ldcs(av + c0 + k));
                cp_async4(slot_idx + STRIDE * k, aj + c0 + k);
            }
            cp_async_wait_all();
            for (int k = lane; k < len; k += 32) cp_async<sizeof(T)>(x_s + k, x + slot_idx[STRIDE * k]);
            cp_async_wait_all();
            __syncwarp();
            const int b = (int)((myb - c0 > 0) ? myb - c0 : 0);
            const int en = (int)((mye - c0 < len) ? mye - c0 : len);
            if (has_row && b < en) {
                int j = b;
                for (; j + 4 <= en; j += 4) {
                    sum = fma_t(staged_value<VT>(a_s, j), x_s[j], sum);
                    sum = fma_t(staged_value<VT>(a_s, j + 1), x_s[j + 1], sum);
                    sum = fma_t(staged_value<VT>(a_s, j + 2), x_s[j + 2], sum);
                    sum = fma_t(staged_value<VT>(a_s, j + 3), x_s[j + 3], sum);
                }
                for (; j < en; ++j) sum = fma_t(staged_value<VT>(a_s, j), x_s[j], sum);
            }
            __syncwarp();   // the next chunk overwrites the slice
        }
        if (has_row) {
            store_y(y, row, sum, ep.acc);
            if (ep.st) dot = fma_t(x[row], sum, dot);
        }
    }
    if (ep.st) finish_dot_nt<T, NT>(dot, ep);
}

// First row of each entry window: row_block[w] = first r in [0, n] with irp[r] >= w*W,
// for w < nblocks; row_block[nblocks] = n.
__global__ void csr_row_block_kernel(const int32_t* __restrict__ irp, int32_t n, int64_t nblocks,
                                     int32_t* __restrict__ row_block) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lo = (r == 0) ? 0 : (int64_t)irp[r - 1] / kCsrWindow + 1;
        int64_t hi = (int64_t)irp[r] / kCsrWindow;
        if (hi > nblocks - 1) hi = nblocks - 1;
        for (int64_t w = lo; w <= hi; ++w) row_block[w] = (int32_t)r;
        if (r == n) row_block[nblocks] = n;
    }
}

// COO: CTA w takes entries [w*W, (w+1)*W) of the sorted arrays.
template <typename VT, typename T>
__global__ void __launch_bounds__(kThreads) spmv_coo_stage_kernel(
    int32_t nrows, int64_t nnz, const int32_t* __restrict__ ai, const int32_t* __restrict__ aj,
    const VT* __restrict__ av, const T* __restrict__ x, T* __restrict__ y,
    CooCarry* __restrict__ carry, const CgState* st, bool acc) {
    pdl_wait();
    pdl_trigger();
    if (st && st->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* a_s = reinterpret_cast<T*>(smem_raw);
    T* x_s = a_s + kStageCap;
    int32_t* rs = reinterpret_cast<int32_t*>(x_s + kStageCap);
    int32_t* srow = rs + kRsCap;
    __shared__ int s_warp[kThreads / 32 + 1];
    const int64_t w = blockIdx.x;
    const int64_t s = w * kCooWindow;
    const int len = (int)((nnz - s < kCooWindow) ? nnz - s : kCooWindow);
    for (int k = threadIdx.x; k < len; k += kThreads) cp_async4(srow + k, ai + s + k);
    stage_window(aj, av, x, s, len, a_s, x_s);
    const int32_t row_before = (s > 0) ? __ldg(ai + s - 1) : -1;
    const int32_t row_after = (s + len < nnz) ? __ldg(ai + s + len) : INT_MAX;
    __syncthreads();

    // run starts: positions whose row differs from the previous entry's. Thread t scans
    // the PER entries [t*PER, t*PER + PER) with 128-bit shared loads (48-byte stride:
    // conflict-free per quarter warp).
    constexpr int PER = kCooWindow / kThreads;
    static_assert(PER % 4 == 0, "compaction reads four rows at a time");
    const int kb = threadIdx.x * PER;
    int32_t rv[PER];
#pragma unroll
    for (int q = 0; q < PER / 4; ++q) {
        const int4 t4 = reinterpret_cast<const int4*>(srow + kb)[q];
        rv[4 * q] = t4.x; rv[4 * q + 1] = t4.y; rv[4 * q + 2] = t4.z; rv[4 * q + 3] = t4.w;
    }
    const int32_t before = (kb > 0 && kb <= len) ? srow[kb - 1] : INT_MIN;
    unsigned flags = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int k = kb + q;
        const int32_t prv = (q == 0) ? before : rv[q - 1];
        if (k < len && (k == 0 || rv[q] != prv)) flags |= 1u << q;
    }
    int nruns;
    int pos = block_excl_scan(__popc(flags), s_warp, &nruns);
    while (flags) {
        const int q = __ffs(flags) - 1;
        flags &= flags - 1;
        rs[pos++] = kb + q;
    }
    if (threadIdx.x == 0) rs[nruns] = len;
    __syncthreads();

    const int32_t row_first = srow[0], row_last = srow[len - 1];
    const bool cont_prev = (row_before == row_first);
    const bool cont_next = (row_after == row_last);
    reduce_runs<VT>(a_s, x_s, rs, nruns, [&](int i, T sum) {
        const int32_t r = srow[rs[i]];
        const bool to_head = (i == 0) && cont_prev;
        const bool to_tail = (i == nruns - 1) && cont_next;
        if (to_head) carry[w].head = to_f64_exact(sum);
        if (to_tail) carry[w].tail = to_f64_exact(sum);
        if (!to_head && !to_tail) store_y(y, r, sum, acc);
    });
    if (threadIdx.x == 0) {
        carry[w].row_first = row_first;
        carry[w].row_last = row_last;
    }
}

// COO, run-vector kernel. Warp c takes the chunk of CHUNK (256 or 512) sorted entries
// [c*C, (c+1)*C). Pass 1 (integer only): lanes read the row indices (coalesced), mark
// where the row changes, and compact the run starts with ballots into the warp's slice
// of shared memory, zeroing the rows skipped between runs. Pass 2: groups of 4 lanes
// take one run each, lane-strided FMAs over its entries, then 2 shuffle-adds -- the CSR
// V = 4 pattern, which on GB300 balances coalescing against FP64 issue slots. Runs cut
// by a chunk edge leave partial sums in the carry record, added by the fix-up pass.
template <typename VT, typename T, int CHUNK>
__global__ void __launch_bounds__(kThreads) spmv_coo_vec_kernel(
    int32_t nrows, int64_t nnz, const int32_t* __restrict__ ai, const int32_t* __restrict__ aj,
    const VT* __restrict__ av, const T* __restrict__ x, T* __restrict__ y, CooCarry* __restrict__ carry,
    int64_t nchunks, const CgState* st, bool acc) {
    pdl_wait();
    pdl_trigger();
    if (st && st->done) return;
    __shared__ int32_t s_rs[kThreads / 32][CHUNK + 1];
    __shared__ int32_t s_row[kThreads / 32][CHUNK];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * (kThreads / 32) + w;
    if (c >= nchunks) return;   // whole warp
    const int64_t c0 = c * CHUNK;
    const int len = (int)((nnz - c0 < CHUNK) ? nnz - c0 : CHUNK);
    const int32_t row_before = (c0 > 0) ? __ldg(ai + c0 - 1) : -1;
    const int32_t row_after = (c0 + len < nnz) ? __ldg(ai + c0 + len) : INT_MAX;
    int32_t* rs = s_rs[w];
    int32_t* rrow = s_row[w];

    int32_t rv[(CHUNK / 32)];
#pragma unroll
    for (int q = 0; q < (CHUNK / 32); ++q) {
        const int k = q * 32 + lane;
        rv[q] = (k < len) ? __ldcs(ai + c0 + k) : INT_MAX;
    }
    int nr = 0;
    int32_t carry_row = row_before;
#pragma unroll
    for (int q = 0; q < (CHUNK / 32); ++q) {
        const int k = q * 32 + lane;
        const int32_t r = rv[q];
        int32_t prev = __shfl_up_sync(FULL, r, 1);
        if (lane == 0) prev = carry_row;
        const bool start = (k < len) && (k == 0 || r != prev);
        const unsigned ballot = __ballot_sync(FULL, start);
        if (start) {
            const int pos = nr + __popc(ballot & ((1u << lane) - 1u));
            rs[pos] = k;
            rrow[pos] = r;
        }
        nr += __popc(ballot);
        carry_row = __shfl_sync(FULL, r, 31);
    }
    if (lane == 0) rs[nr] = len;
    __syncwarp();

    const bool cont_prev = (row_before == rrow[0]);
    const bool cont_next = (row_after == rrow[nr - 1]);
    const int grp = lane >> 2, sub = lane & 3;
    for (int i0 = 0; i0 < nr; i0 += 8) {
        const int i = i0 + grp;
        T sum = T(0);
        if (i < nr) {
            const int b = rs[i], e = rs[i + 1];
            for (int j = b + sub; j < e; j += 4)
                sum = fma_t(convert_value<T>(__ldcs(av + c0 + j)), __ldg(x + __ldcs(aj + c0 + j)), sum);
        }
        sum += __shfl_xor_sync(FULL, sum, 1);
        sum += __shfl_xor_sync(FULL, sum, 2);
        if (sub == 0 && i < nr) {
            const bool to_head = (i == 0) && cont_prev;
            const bool to_tail = (i == nr - 1) && cont_next;
            if (to_head) carry[c].head = to_f64_exact(sum);
            if (to_tail) carry[c].tail = to_f64_exact(sum);
            if (!to_head && !to_tail) store_y(y, rrow[i], sum, acc);
        }
    }
    if (lane == 0) {
        carry[c].row_first = rrow[0];
        carry[c].row_last = rrow[nr - 1];
    }
}

// COO, a warp per block of kCooRbRows = 32 consecutive rows. The block's entries
// [rb[b], rb[b+1]) come from a table built with the handle (one int per 32 rows); a row never
// crosses a block, so there are no carries and no fix-up pass. The warp reads the block's row
// indices in 16-byte groups (lane l the l-th group of each 128-entry stretch, every group of
// the block in flight at once for rows of stencil length), marks where each row starts (a row
// change against the previous entry) in shared memory, finds where each row ends by a suffix
// minimum over the next rows' starts, and then runs the FMA phase of the 32-row CSR kernel
// (rows32_sum, 4 lanes per row, reduce-scatter). Rows of the block without entries are
// written as 0 (left as they are for y += A x). For rows of at most 128 entries (longer ones
// take the segment kernel).
// The kernel waits on memory latency, so it is held to 32 registers for 8 CTAs per SM (block
// positions in 32 bits; a few bytes spill): 157.7-158.6 vs 161.7-162.7 us at 128^3 and 494-495
// vs 512 us at 192^3 against 40 registers and 6 CTAs.
template <typename VT, typename T>
__global__ void __launch_bounds__(kThreads, 8) spmv_coo_rb_kernel(
    int32_t nrows, int64_t nnz, const int32_t* __restrict__ ai, const int32_t* __restrict__ aj,
    const VT* __restrict__ av, const int32_t* __restrict__ rb, int64_t nrb, const T* __restrict__ x,
    T* __restrict__ y, const CgState* st, bool acc) {
    static_assert(kCooRbRows == 32, "a warp per block of 32 rows");
    constexpr int V = 4, R = 32 / V;
    pdl_wait();
    pdl_trigger();
    if (st && st->done) return;
    __shared__ int32_t s_start[kThreads / 32][kCooRbRows];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // 32-bit positions: entries lie below 2^31, so an entry index plus the 2,048 entries one
    // round reads past it, and a block's first row, fit in 32 unsigned bits.
    const uint32_t b = blockIdx.x * (kThreads / 32) + w;
    if ((int64_t)b >= nrb) return;   // whole warp
    const uint32_t row0 = b * kCooRbRows;
    const uint32_t e0 = (uint32_t)__ldg(rb + b);
    const uint32_t e1 = (uint32_t)__ldg(rb + b + 1);
    const uint32_t unnz = (uint32_t)nnz;
    const int cnt = (int)(e1 - e0);
    int32_t* start = s_start[w];
    start[lane] = -1;
    __syncwarp();
    // 16-byte groups from the multiple of 4 at or below e0; entries outside [e0, e1) are read
    // (when below nnz) but not marked. ai's allocation starts 256-byte aligned.
    const uint32_t a0 = e0 & ~3u;
    constexpr int kHeld = 4;   // groups loaded together: 512 entries (two rounds for 32 stencil rows)
    int32_t last = (int32_t)row0 - 1;   // the row before the first group (a row below the block)
    for (uint32_t g0 = a0; g0 < e1; g0 += 128 * kHeld) {
        int4 v[kHeld];
#pragma unroll
        for (int q = 0; q < kHeld; ++q) {
            const uint32_t g = g0 + 128 * q + 4 * lane;
            if (g + 3 < unnz) {
                v[q] = __ldg(reinterpret_cast<const int4*>(ai + g));
            } else {
                v[q].x = g < unnz ? __ldg(ai + g) : INT_MAX;
                v[q].y = g + 1 < unnz ? __ldg(ai + g + 1) : INT_MAX;
                v[q].z = g + 2 < unnz ? __ldg(ai + g + 2) : INT_MAX;
                v[q].w = INT_MAX;
            }
        }
#pragma unroll
        for (int q = 0; q < kHeld; ++q) {
            const uint32_t g = g0 + 128 * q + 4 * lane;
            int32_t prev = __shfl_up_sync(FULL, v[q].w, 1);
            if (lane == 0) prev = last;
            last = __shfl_sync(FULL, v[q].w, 31);
            const int32_t r[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int32_t pr = c == 0 ? prev : r[c - 1];
                if (g + c >= e0 && g + c < e1 && r[c] != pr) start[(int)((uint32_t)r[c] - row0)] = (int)(g + c - e0);
            }
        }
    }
    __syncwarp();
    // row (row0 + lane): its first entry (block-relative) and length; an empty row's end is the
    // next nonempty row's start, the minimum of the starts of the rows after it (or cnt)
    const int my = start[lane];
    int nxt = __shfl_down_sync(FULL, my >= 0 ? my : cnt, 1);
    if (lane == 31) nxt = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_down_sync(FULL, nxt, o);
        if (lane + o < 32) nxt = min(nxt, t);
    }
    const int32_t mylen = my >= 0 ? nxt - my : 0;
    const int sub = lane & (V - 1);
    const T sum = rows32_sum<VT, T, V>(sub, aj, av, x, [=](int t, int32_t& s0, int32_t& len) {
        const int r = R * t + lane / V;
        s0 = (int32_t)e0 + __shfl_sync(FULL, my, r);
        len = __shfl_sync(FULL, mylen, r);
    });
    const int rr = R * sub + lane / V;
    const bool has = __shfl_sync(FULL, mylen, rr) > 0;
    const int64_t row = (int64_t)row0 + rr;
    if (row < nrows) {
        if (has) store_y(y, row, sum, acc);
        else zero_y(y, row, acc);
    }
}

// Rows spanning windows: the window where such a row starts adds its tail, the heads of
// the windows it covers entirely, and the head of the window where it ends, in order.
template <typename T>
__global__ void spmv_coo_fixup_kernel(const CooCarry* __restrict__ carry, int64_t nwin,
                                      T* __restrict__ y, const CgState* st, bool acc) {
    pdl_wait();
    pdl_trigger();
    if (st && st->done) return;
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwin - 1) return;   // the last window cannot continue into another
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
        const bool d_next = (v + 1 < nwin) && carry[v + 1].row_first == d.row_last;
        if (d_single && d_next) ++v;
        else break;
    }
    store_y(y, c.row_last, (T)sum, acc);
}

// ---------------------------------------------------------------------------
// COO, lane-sequential segments
// ---------------------------------------------------------------------------
// A warp takes 512 consecutive (row-sorted) entries, each lane 16 of them in order: the
// lane multiplies and accumulates sequentially (every FP64 FMA issued by all 32 lanes),
// writes the rows that start and end inside its 16 entries, and keeps the partial sums of
// its first run (head) and last run (tail). A head-flag segmented scan over the lanes' tail
// sums (5 FP64 adds per warp) joins rows that span lanes; rows that span chunks leave the
// same carry records as the other COO kernels for spmv_coo_fixup_kernel.
constexpr int kCooSegPer = 16;
constexpr int kCooSegChunk = 32 * kCooSegPer;
static_assert(kCooSegChunk >= kCooVecChunk, "carry records are allocated for the smaller chunk");

template <typename VT, typename T>
__device__ __forceinline__ void load8_values(const VT* p, T (&v)[8]) {
    using L = DiaVec<VT, T>;
#pragma unroll
    for (int q = 0; q < 8 / L::RPT; ++q) {
        T t[L::RPT];
        L::load(p + q * L::RPT, t);
#pragma unroll
        for (int k = 0; k < L::RPT; ++k) v[q * L::RPT + k] = t[k];
    }
}

template <typename VT, typename T>
__global__ void __launch_bounds__(kThreads, 3) spmv_coo_seg_kernel(
    int32_t nrows, int64_t nnz, const int32_t* __restrict__ ai, const int32_t* __restrict__ aj,
    const VT* __restrict__ av, const T* __restrict__ x, T* __restrict__ y, CooCarry* __restrict__ carry,
    int64_t nchunks, const CgState* st, bool acc) {
    pdl_wait();
    pdl_trigger();
    if (st && st->done) return;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t c = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    if (c >= nchunks) return;   // whole warp
    const int64_t c0 = c * kCooSegChunk;
    const int len = (int)((nnz - c0 < kCooSegChunk) ? nnz - c0 : kCooSegChunk);
    const int32_t row_before = (c0 > 0) ? __ldg(ai + c0 - 1) : -1;
    const int32_t row_after = (c0 + len < nnz) ? __ldg(ai + c0 + len) : INT_MAX;
    const int32_t chunk_first = __ldg(ai + c0);
    const int32_t chunk_last = __ldg(ai + c0 + len - 1);
    const int b = lane * kCooSegPer;
    const int cnt = (len - b >= kCooSegPer) ? kCooSegPer : (len - b > 0 ? len - b : 0);
    const int64_t e0 = c0 + b;

    // Sequential pass over the lane's entries: each row change closes the run before it (the
    // lane's first run is kept as `head` for the joins below, later runs are written at once).
    // Rows without entries are not written here (the launcher zero-fills y first when the
    // matrix has any). A lane without entries acts as a single run of the chunk's last row
    // with sum 0 (transparent below).
    int32_t cur = chunk_last, first = chunk_last;
    T head = T(0), sum = T(0);
    bool closed = false;   // the lane's first run has ended inside the lane
    if (cnt > 0) {
        cur = (e0 > 0) ? __ldg(ai + e0 - 1) : -1;
        first = __ldg(ai + e0);
#pragma unroll
        for (int h = 0; h < kCooSegPer; h += 8) {
            int32_t rr[8], jj[8];
            T aa[8], xx[8];
            if (cnt == kCooSegPer) {
                const int4 r0 = __ldcs(reinterpret_cast<const int4*>(ai + e0 + h));
                const int4 r1 = __ldcs(reinterpret_cast<const int4*>(ai + e0 + h + 4));
                const int4 j0 = __ldcs(reinterpret_cast<const int4*>(aj + e0 + h));
                const int4 j1 = __ldcs(reinterpret_cast<const int4*>(aj + e0 + h + 4));
                rr[0] = r0.x; rr[1] = r0.y; rr[2] = r0.z; rr[3] = r0.w;
                rr[4] = r1.x; rr[5] = r1.y; rr[6] = r1.z; rr[7] = r1.w;
                jj[0] = j0.x; jj[1] = j0.y; jj[2] = j0.z; jj[3] = j0.w;
                jj[4] = j1.x; jj[5] = j1.y; jj[6] = j1.z; jj[7] = j1.w;
                load8_values<VT, T>(av + e0 + h, aa);
            } else {
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const bool ok = h + k < cnt;
                    rr[k] = ok ? __ldcs(ai + e0 + h + k) : 0;
                    jj[k] = ok ? __ldcs(aj + e0 + h + k) : 0;
                    aa[k] = ok ? convert_value<T>(__ldcs(av + e0 + h + k)) : T(0);
                }
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) xx[k] = (h + k < cnt) ? __ldg(x + jj[k]) : T(0);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (h + k < cnt) {
                    const int32_t r = rr[k];
                    if (r != cur) {
                        if (h + k > 0) {   // close run `cur`
                            if (!closed) { head = sum; closed = true; }
                            else store_y(y, cur, sum, acc);
                        }
                        cur = r;
                        sum = T(0);
                    }
                    sum = fma_t(aa[k], xx[k], sum);
                }
            }
        }
    }

    // Segmented inclusive scan of the tail sums: a lane without an internal row change whose
    // row equals the previous lane's last row continues that lane's last run.
    const int32_t prev_last = __shfl_up_sync(FULL, cur, 1);
    const bool cont = !closed && lane > 0 && first == prev_last;
    T S = sum;
    bool F = !cont;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T Su = __shfl_up_sync(FULL, S, d);
        const bool Fu = __shfl_up_sync(FULL, F, d);
        if (lane >= d) {
            if (!F) S += Su;
            F = F || Fu;
        }
    }
    const T prevS = __shfl_up_sync(FULL, S, 1);
    const int32_t next_first = __shfl_down_sync(FULL, first, 1);
    const bool cp = (row_before == chunk_first);   // the chunk's first run started before it
    const bool cn = (row_after == chunk_last);     // the chunk's last run continues after it

    if (cnt > 0 && closed) {   // the lane's first run ends inside the lane
        T tot = head;
        if (lane > 0 && first == prev_last) tot += prevS;
        if (first == chunk_first && cp) carry[c].head = to_f64_exact(tot);
        else store_y(y, first, tot, acc);
    }
    if (lane < 31 && cnt > 0 && next_first != cur) {   // the last run ends at the lane's end
        if (cur == chunk_first && cp) carry[c].head = to_f64_exact(S);
        else store_y(y, cur, S, acc);
    }
    if (lane == 31) {   // S is the chunk's last run
        const bool one_run = (chunk_first == chunk_last);
        if (cn) carry[c].tail = to_f64_exact(S);
        if (one_run && cp) carry[c].head = to_f64_exact(S);
        if (!cn && !(one_run && cp)) store_y(y, chunk_last, S, acc);
        carry[c].row_first = chunk_first;
        carry[c].row_last = chunk_last;
    }
}

// y = 0. Inside CG (st set) a launch after the iteration has stopped does nothing, like the
// other kernels of the iteration.
template <typename T>
__global__ void fill_zero_kernel(T* __restrict__ y, int64_t n, const CgState* st) {
    if (st && st->done) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = T(0);
}

// p.q for the COO path (its SpMV has no single pass to fuse into); last CTA forms alpha.
template <typename T>
__global__ void __launch_bounds__(kThreads) dot_alpha_kernel(int64_t n, const T* __restrict__ p,
                                                             const T* __restrict__ q, DotEpilogue ep) {
    pdl_wait();
    pdl_trigger();
    if (ep.st->done) return;
    T d = T(0);
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kThreads)
        d = fma_t(p[i], q[i], d);
    finish_dot(d, ep);
}

// ---------------------------------------------------------------------------
// host dispatch
// ---------------------------------------------------------------------------
int32_t choose_csr_vector(double mean, double stdev, int32_t maxlen) {
    (void)stdev;
    (void)maxlen;
    if (const char* s = std::getenv("MSPV_CSR_VEC")) {
        int v = std::atoi(s);
        if (v == 0 || v == 1 || v == 2 || v == 4 || v == 8 || v == 16 || v == 32) return v;
    }
    // V lanes per row: 4 for short rows (coalesced 32-byte segments; a warp's 32 rows joined
    // by a reduce-scatter of 3 FP64 adds per lane), wider as rows grow; rows longer than
    // 32 V entries are reduced by a CTA each. The staged kernels (0) are selected only
    // explicitly.
    if (mean <= 48.0) return 4;
    if (mean <= 96.0) return 8;
    if (mean <= 192.0) return 16;
    return 32;
}

mspv_status build_csr_long_rows(mspv_matrix* M, cudaStream_t s) {
    M->nlong = 0;
    if (M->nrows == 0) return MSPV_OK;
    const int32_t long_len = 32 * M->csr_vector;
    if (M->row_max <= long_len) return MSPV_OK;
    DevBuf flags, pos, total;
    MSPV_TRY(flags.alloc(sizeof(int32_t) * (size_t)M->nrows));
    MSPV_TRY(pos.alloc(sizeof(int32_t) * (size_t)M->nrows));
    MSPV_TRY(total.alloc(sizeof(int32_t)));
    unsigned grid = (unsigned)(((int64_t)M->nrows + kThreads - 1) / kThreads);
    if (grid > (unsigned)num_sms() * 64) grid = num_sms() * 64;
    csr_long_flag_kernel<<<grid, kThreads, 0, s>>>(M->irp, M->nrows, long_len, flags.as<int32_t>());
    MSPV_CUDA_TRY(cudaGetLastError());
    MSPV_TRY(exclusive_scan_i32(flags.as<int32_t>(), pos.as<int32_t>(), M->nrows, total.as<int32_t>(), s));
    int32_t nl = 0;
    MSPV_CUDA_TRY(cudaMemcpyAsync(&nl, total.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    MSPV_CUDA_TRY(cudaStreamSynchronize(s));
    if (nl == 0) return MSPV_OK;
    MSPV_TRY(dev_alloc_n(&M->long_rows, nl));
    M->bytes += (int64_t)nl * 4;
    csr_long_compact_kernel<<<grid, kThreads, 0, s>>>(flags.as<int32_t>(), pos.as<int32_t>(), M->nrows,
                                                      M->long_rows);
    MSPV_CUDA_TRY(cudaGetLastError());
    MSPV_CUDA_TRY(cudaStreamSynchronize(s));
    M->nlong = nl;
    return MSPV_OK;
}

mspv_status build_csr_row_blocks(mspv_matrix* M, cudaStream_t s) {
    M->nblocks = (M->nnz + kCsrWindow - 1) / kCsrWindow;
    if (M->nblocks < 1) M->nblocks = 1;
    MSPV_TRY(dev_alloc_n(&M->row_block, M->nblocks + 1));
    M->bytes += (M->nblocks + 1) * 4;
    const int64_t threads = (int64_t)M->nrows + 1;
    unsigned grid = (unsigned)((threads + kThreads - 1) / kThreads);
    if (grid > (unsigned)num_sms() * 64) grid = num_sms() * 64;
    csr_row_block_kernel<<<grid, kThreads, 0, s>>>(M->irp, M->nrows, M->nblocks, M->row_block);
    MSPV_CUDA_TRY(cudaGetLastError());
    return MSPV_OK;
}

static inline unsigned blocks_for(int64_t threads) {
    return (unsigned)((threads + kThreads - 1) / kThreads);
}

static int64_t vector_grid(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)num_sms() * 8;
    if (b > cap) b = cap;
    return b < 1 ? 1 : b;
}

// Raise a kernel's dynamic shared-memory limit once (per kernel instantiation).
template <auto Kernel>
static void allow_smem(size_t bytes) {
    static const bool ok = [bytes] {
        return cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
    }();
    (void)ok;
}

// DIA launch shape: one CTA per strip of kThreads * RPT consecutive rows. Consecutive
// CTAs run on consecutive strips, so the CTAs in flight read one contiguous stretch of
// each diagonal and of x (DRAM and L2 friendly). Spreading one wave of CTAs over distant
// equal row ranges instead balances the tail but measured ~10% slower on GB300.
// Rows per CTA of the DIA kernel that a value type and arithmetic launch (threads x rows per
// thread).
static int64_t dia_strip_rows(int vt, bool f32) {
    switch (vt) {
        case MSPV_F64: return (int64_t)kThreads * DiaVec<double, double>::RPT;
        case MSPV_F32:
            return f32 ? (int64_t)DiaF32Shape<float>::NT * DiaVec<float, float>::RPT
                       : (int64_t)kThreads * DiaVec<float, double>::RPT;
        default:
            return f32 ? (int64_t)DiaF32Shape<__nv_bfloat16>::NT * DiaVec<__nv_bfloat16, float>::RPT
                       : (int64_t)kThreads * DiaVec<__nv_bfloat16, double>::RPT;
    }
}

static int64_t csr_grid_for(const mspv_matrix* A, bool f32);

// CTAs of the fused-dot SpMV launch in FP64 or FP32 arithmetic: the number of p.q partials
// it writes, which the CG's alpha kernel sums. Only DIA launches differ between the two
// (BF16 values: 8 rows per thread in FP64, 4 in FP32).
int64_t spmv_partials_count(const mspv_matrix* A, bool f32) {
    switch (A->format) {
        case MSPV_DIA: {
            const int64_t strip = dia_strip_rows(A->value_type, f32);
            const int64_t g = ((int64_t)A->nrows + strip - 1) / strip;
            return g < 1 ? 1 : g;
        }
        case MSPV_CSR:
            return csr_grid_for(A, f32);
        default:
            return vector_grid(A->nrows);
    }
}

int64_t spmv_partials_needed(const mspv_matrix* A) {
    return std::max(spmv_partials_count(A, false), spmv_partials_count(A, true));
}

template <typename VT, typename T>
static void launch_dia(const mspv_matrix* A, const T* x, T* y, cudaStream_t s, DotEpilogue ep) {
    constexpr int RPT = DiaVec<VT, T>::RPT;
    constexpr int NT = sizeof(T) == 4 ? DiaF32Shape<VT>::NT : kThreads;
    const int64_t strip = (int64_t)NT * RPT;
    int64_t grid = ((int64_t)A->nrows + strip - 1) / strip;
    if (grid < 1) grid = 1;
    if constexpr (sizeof(T) == 4) {
        launch_kernel(ep.pdl, spmv_dia_f32_kernel<VT>, (unsigned)grid, NT, 0, s, A->nrows, A->ndiags,
                      A->npad, A->doff, (const int2*)A->druns, A->ndruns, static_cast<const VT*>(A->av), x, y, ep);
    } else {
        if (ep.acc)
            launch_kernel(ep.pdl, spmv_dia_kernel<VT, T, true>, (unsigned)grid, kThreads, 0, s, A->nrows,
                          A->ndiags, A->npad, A->doff, static_cast<const VT*>(A->av), x, y, ep);
        else
            launch_kernel(ep.pdl, spmv_dia_kernel<VT, T, false>, (unsigned)grid, kThreads, 0, s, A->nrows,
                          A->ndiags, A->npad, A->doff, static_cast<const VT*>(A->av), x, y, ep);
    }
}

// Warp slice: 1024 entries, so a 32-row group of rows up to 32 entries long is staged
// in one chunk and every lane's row is summed in the same pass (a group split over
// chunks leaves lanes idle while the warp still issues the longest lane's FMAs).
// 128-thread CTAs keep three CTAs (12 warps) per SM within shared memory at FP64.
constexpr int kCsrWarpCap = 1024;
constexpr int kCsrWarpThreads = 128;

// Which staged CSR kernel a new CSR handle uses: warp-private staging (default) or CTA
// row blocks (MSPV_CSR_KERNEL=block, read when the handle is built).
int32_t choose_csr_block_kernel() {
    const char* v = std::getenv("MSPV_CSR_KERNEL");
    return (v && std::string(v) == "block") ? 1 : 0;
}

template <typename VT, typename T>
static int64_t csr_warp_grid(int32_t nrows) {
    static const int per_sm = [] {
        int b = 0;
        constexpr auto K = spmv_csr_warp_kernel<VT, T, kCsrWarpCap, kCsrWarpThreads>;
        constexpr size_t smem = csr_warp_smem<T, kCsrWarpCap, kCsrWarpThreads>();
        allow_smem<K>(smem);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, K, kCsrWarpThreads, smem) != cudaSuccess || b < 1)
            b = 2;
        return b;
    }();
    const int64_t groups = ((int64_t)nrows + 31) / 32;
    int64_t g = (groups + kCsrWarpThreads / 32 - 1) / (kCsrWarpThreads / 32);
    const int64_t wave = (int64_t)num_sms() * per_sm;
    if (g > wave) g = wave;
    return g < 1 ? 1 : g;
}

// Resident CTAs per SM of the striding 32-row CSR kernel (the grid inside CG) for a value type
// and arithmetic, from the occupancy calculator; the V = 4 instantiation stands for every lane
// width.
template <typename VT, typename T>
static int csr_stride_ctas_per_sm() {
    static const int k = [] {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, spmv_csr_rows32_kernel<VT, T, 4, true>, kThreads, 0) !=
                cudaSuccess ||
            b < 1)
            b = 6;
        return b;
    }();
    return k;
}

static int csr_stride_ctas_per_sm(int vt, bool f32) {
    switch (vt) {
        case MSPV_F64: return csr_stride_ctas_per_sm<double, double>();   // FP32 arithmetic needs FP32/BF16 values
        case MSPV_F32: return f32 ? csr_stride_ctas_per_sm<float, float>() : csr_stride_ctas_per_sm<float, double>();
        default:
            return f32 ? csr_stride_ctas_per_sm<__nv_bfloat16, float>()
                       : csr_stride_ctas_per_sm<__nv_bfloat16, double>();
    }
}

// CTAs of the V-lane kernels (a CTA covers kThreads rows for V <= 8, kThreads / V rows for
// wider rows). With a dot-product epilogue (inside CG) the grid is capped, so the scalar kernels
// sum few partials, and the warps stride over the rows: two whole waves of the striding kernel in
// FP64 arithmetic, three in FP32 arithmetic. A fixed 16 CTAs per SM made a ragged third wave of
// the 40-register FP64 kernel, which holds 6 CTAs per SM (0.58 vs 0.54 ms per FP64 CG iteration
// at 192^3); the FP32-arithmetic kernels of the inner solver measured fastest at three waves.
static int64_t csr_vector_grid(const mspv_matrix* A, bool capped, bool f32) {
    const int64_t lanes_per_row = A->csr_vector <= 8 ? 1 : A->csr_vector;
    int64_t g = ((int64_t)A->nrows * lanes_per_row + kThreads - 1) / kThreads;
    if (capped) {
        const int64_t cap = (int64_t)num_sms() * csr_stride_ctas_per_sm(A->value_type, f32) * (f32 ? 3 : 2);
        if (g > cap) g = cap;
    }
    return g < 1 ? 1 : g;
}

static int64_t csr_grid_for(const mspv_matrix* A, bool f32) {
    if (A->csr_vector != 0) return csr_vector_grid(A, true, f32) + A->nlong;
    if (A->csr_block) return A->nblocks;
    if (A->value_type == MSPV_F64) return csr_warp_grid<double, double>(A->nrows);
    // FP32/BF16 values run the FP64-arithmetic or FP32-arithmetic instantiation; both
    // have one grid size per value type, the larger of the two bounds the partials
    const int64_t a = (A->value_type == MSPV_F32) ? csr_warp_grid<float, double>(A->nrows)
                                                  : csr_warp_grid<__nv_bfloat16, double>(A->nrows);
    const int64_t b = (A->value_type == MSPV_F32) ? csr_warp_grid<float, float>(A->nrows)
                                                  : csr_warp_grid<__nv_bfloat16, float>(A->nrows);
    return a > b ? a : b;
}

template <typename VT, typename T>
static void launch_csr(const mspv_matrix* A, const T* x, T* y, cudaStream_t s, DotEpilogue ep) {
    const VT* av = static_cast<const VT*>(A->av);
    const int V = A->csr_vector;
    if (V == 0 && !A->csr_block) {
        constexpr auto K = spmv_csr_warp_kernel<VT, T, kCsrWarpCap, kCsrWarpThreads>;
        constexpr size_t smem = csr_warp_smem<T, kCsrWarpCap, kCsrWarpThreads>();
        allow_smem<K>(smem);
        const int64_t grid = csr_warp_grid<VT, T>(A->nrows);
        launch_kernel(ep.pdl, K, (unsigned)grid, kCsrWarpThreads, smem, s, A->nrows, A->irp, A->aj, av, x, y, ep);
        return;
    }
    if (V == 0) {
        allow_smem<spmv_csr_stage_kernel<VT, T>>(csr_smem<T>());
        launch_kernel(ep.pdl, spmv_csr_stage_kernel<VT, T>, (unsigned)A->nblocks, kThreads, csr_smem<T>(), s,
                      A->irp, A->aj, av, A->row_block, x, y, ep);
        return;
    }
    const bool capped = ep.partials != nullptr;
    const unsigned grid = (unsigned)csr_vector_grid(A, capped, sizeof(T) == 4);
    const int32_t long_len = A->nlong > 0 ? 32 * V : INT_MAX;
#define MSPV_CSR_CASE(VV, KERNEL)                                                              \
    case VV:                                                                                   \
        if (capped)                                                                            \
            launch_kernel(ep.pdl, KERNEL<VT, T, VV, true>, grid, kThreads, 0, s,               \
                          A->nrows, A->irp, A->aj, av, x, y, long_len, ep);                    \
        else                                                                                   \
            launch_kernel(ep.pdl, KERNEL<VT, T, VV, false>, grid, kThreads, 0, s,              \
                          A->nrows, A->irp, A->aj, av, x, y, long_len, ep);                    \
        break;
    switch (V) {
        MSPV_CSR_CASE(1, spmv_csr_rows32_kernel)
        MSPV_CSR_CASE(2, spmv_csr_rows32_kernel)
        MSPV_CSR_CASE(4, spmv_csr_rows32_kernel)
        MSPV_CSR_CASE(8, spmv_csr_rows32_kernel)
        MSPV_CSR_CASE(16, spmv_csr_vector_kernel)
        default:
        MSPV_CSR_CASE(32, spmv_csr_vector_kernel)
    }
#undef MSPV_CSR_CASE
    if (A->nlong > 0) {
        DotEpilogue lep = ep;   // same flags; its partials follow the V-lane kernel's
        lep.partials = ep.partials ? ep.partials + grid : nullptr;
        launch_kernel(ep.pdl, spmv_csr_long_kernel<VT, T>, (unsigned)A->nlong, kThreads, 0, s, A->long_rows,
                      A->irp, A->aj, av, x, y, lep);
    }
}

template <typename VT, typename T>
static void launch_coo_windows(int32_t nrows, int64_t nnz, const int32_t* ai, const int32_t* aj, const VT* av,
                               const T* x, T* y, CooCarry* carry, int64_t nwin, cudaStream_t s, const CgState* st) {
    allow_smem<spmv_coo_stage_kernel<VT, T>>(coo_smem<T>());
    spmv_coo_stage_kernel<VT, T><<<(unsigned)nwin, kThreads, coo_smem<T>(), s>>>(nrows, nnz, ai, aj, av, x, y,
                                                                                 carry, st, false);
    if (nwin > 1) spmv_coo_fixup_kernel<T><<<blocks_for(nwin), kThreads, 0, s>>>(carry, nwin, y, st, false);
}

template <typename VT, typename T>
static void launch_coo(const mspv_matrix* A, const T* x, T* y, cudaStream_t s, DotEpilogue ep) {
    int64_t nch;
    // The chunked kernels write only rows that have entries: rows without any are zeroed here,
    // in parallel, before them (y = A x; for y += A x they stay as they are). The row-block
    // kernel writes every row of its blocks itself. A plain launch: it waits for its
    // predecessor.
    if (!(A->coo_kernel == 2 && A->coo_rb) && !ep.acc && A->empty_rows > 0)
        fill_zero_kernel<T><<<(unsigned)vector_grid(A->nrows), kThreads, 0, s>>>(y, (int64_t)A->nrows,
                                                                                   (const CgState*)ep.st);
    if (A->coo_kernel == 2 && A->coo_rb) {
        const unsigned g = (unsigned)((A->coo_nrb + kThreads / 32 - 1) / (kThreads / 32));
        launch_kernel(ep.pdl, spmv_coo_rb_kernel<VT, T>, g, kThreads, 0, s, A->nrows, A->nnz, A->ai, A->aj,
                      static_cast<const VT*>(A->av), (const int32_t*)A->coo_rb, A->coo_nrb, x, y,
                      (const CgState*)ep.st, ep.acc);
        nch = 0;   // no carries
    } else if (A->coo_kernel == 1) {
        const int chunk = A->coo_chunk == 512 ? 512 : kCooVecChunk;
        nch = (A->nnz + chunk - 1) / chunk;   // <= A->nchunks, the carry records allocated
        const unsigned g = (unsigned)((nch + kThreads / 32 - 1) / (kThreads / 32));
        if (chunk == 512)
            launch_kernel(ep.pdl, spmv_coo_vec_kernel<VT, T, 512>, g, kThreads, 0, s, A->nrows, A->nnz, A->ai,
                          A->aj, static_cast<const VT*>(A->av), x, y, A->carry, nch, (const CgState*)ep.st, ep.acc);
        else
            launch_kernel(ep.pdl, spmv_coo_vec_kernel<VT, T, kCooVecChunk>, g, kThreads, 0, s, A->nrows, A->nnz,
                          A->ai, A->aj, static_cast<const VT*>(A->av), x, y, A->carry, nch,
                          (const CgState*)ep.st, ep.acc);
    } else {
        nch = (A->nnz + kCooSegChunk - 1) / kCooSegChunk;
        launch_kernel(ep.pdl, spmv_coo_seg_kernel<VT, T>, (unsigned)((nch + kThreads / 32 - 1) / (kThreads / 32)),
                      kThreads, 0, s, A->nrows, A->nnz, A->ai, A->aj, static_cast<const VT*>(A->av), x, y,
                      A->carry, nch, (const CgState*)ep.st, ep.acc);
    }
    if (nch > 1)
        launch_kernel(ep.pdl, spmv_coo_fixup_kernel<T>, blocks_for(nch), kThreads, 0, s, (const CooCarry*)A->carry,
                      nch, y, (const CgState*)ep.st, ep.acc);
    if (ep.st)
        launch_kernel(ep.pdl, dot_alpha_kernel<T>, (unsigned)vector_grid(A->nrows), kThreads, 0, s,
                      (int64_t)A->nrows, x, (const T*)y, ep);
}

// COO SpMV on raw, row-sorted FP64 device triplets with caller-provided carry records
// (one per 3072-entry window); used by the allocation-free entry point.
mspv_status launch_coo_raw(int32_t nrows, int64_t nnz, const int32_t* ai, const int32_t* aj,
                           const double* av, const double* x, double* y, CooCarry* carry,
                           cudaStream_t s) {
    if (nrows == 0) return MSPV_OK;
    if (nnz == 0) {
        fill_zero_kernel<double><<<(unsigned)vector_grid(nrows), kThreads, 0, s>>>(y, nrows, nullptr);
        MSPV_CUDA_TRY(cudaGetLastError());
        return MSPV_OK;
    }
    const int64_t nwin = (nnz + kCooWindow - 1) / kCooWindow;
    // rows without entries (unknown for raw triplets) are zeroed first; the kernel writes the others
    fill_zero_kernel<double><<<(unsigned)vector_grid(nrows), kThreads, 0, s>>>(y, nrows, nullptr);
    launch_coo_windows<double, double>(nrows, nnz, ai, aj, av, x, y, carry, nwin, s, nullptr);
    MSPV_CUDA_TRY(cudaGetLastError());
    return MSPV_OK;
}

template <typename T>
static mspv_status launch_spmv_t(const mspv_matrix* A, const T* x, T* y, cudaStream_t s, DotEpilogue ep) {
    if (A->nrows == 0) return MSPV_OK;
    if (A->format == MSPV_COO && A->nnz == 0) {
        if (ep.st) return set_error(MSPV_EINVAL, "cg: matrix has no entries");
        fill_zero_kernel<T><<<(unsigned)vector_grid(A->nrows), kThreads, 0, s>>>(y, A->nrows, nullptr);
        MSPV_CUDA_TRY(cudaGetLastError());
        return MSPV_OK;
    }
    const int vt = A->value_type;
    if constexpr (sizeof(T) == 4) {
        if (vt == MSPV_F64)
            return set_error(MSPV_EFORMAT, "FP32 arithmetic needs FP32 or BF16 stored values");
    }
    switch (A->format) {
        case MSPV_DIA:
            if constexpr (sizeof(T) == 8) {
                if (vt == MSPV_F64) { launch_dia<double, T>(A, x, y, s, ep); break; }
            }
            if (vt == MSPV_F32) launch_dia<float, T>(A, x, y, s, ep);
            else launch_dia<__nv_bfloat16, T>(A, x, y, s, ep);
            break;
        case MSPV_CSR:
            if constexpr (sizeof(T) == 8) {
                if (vt == MSPV_F64) { launch_csr<double, T>(A, x, y, s, ep); break; }
            }
            if (vt == MSPV_F32) launch_csr<float, T>(A, x, y, s, ep);
            else launch_csr<__nv_bfloat16, T>(A, x, y, s, ep);
            break;
        default:
            if constexpr (sizeof(T) == 8) {
                if (vt == MSPV_F64) { launch_coo<double, T>(A, x, y, s, ep); break; }
            }
            if (vt == MSPV_F32) launch_coo<float, T>(A, x, y, s, ep);
            else launch_coo<__nv_bfloat16, T>(A, x, y, s, ep);
            break;
    }
    MSPV_CUDA_TRY(cudaGetLastError());
    return MSPV_OK;
}

mspv_status launch_spmv(const mspv_matrix* A, const double* x, double* y, cudaStream_t s, DotEpilogue ep) {
    return launch_spmv_t<double>(A, x, y, s, ep);
}

mspv_status launch_spmv_f32(const mspv_matrix* A, const float* x, float* y, cudaStream_t s, DotEpilogue ep) {
    return launch_spmv_t<float>(A, x, y, s, ep);
}

}  // namespace mspv
