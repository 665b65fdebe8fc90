// Unpreconditioned conjugate gradient, the solver the paper's HPCG experiments run
// with the preconditioner disabled (Sec. VI), and two mixed-precision solvers for
// low-precision matrix values (not in the paper): FP64 iterative refinement around a
// restarted inner CG, and one FP32 CG whose residual is replaced by the FP64 one at
// reliable updates.
//
// One iteration is five kernels on the caller's stream, chained by programmatic dependent
// launches; none of them waits on the host or on another CTA:
//   1. q = A p; each CTA also writes its partial sum of p.q;
//   2. (one CTA) p.q = sum of the partials in a fixed order; alpha = rho / p.q, or a
//      breakdown;
//   3. r -= alpha q; each CTA writes its partial of r.r;
//   4. (one CTA) rho' = r.r; convergence test, iteration count, beta = rho' / rho;
//   5. x += alpha p, then p = r + beta p (one pass over p).
// Every scalar lives in a device CgState. Once `done` is set all kernels return at
// entry, so the host may launch past convergence and polls the state only after every
// MSPV_CG_CHECK_EVERY iterations. Reductions are deterministic (fixed order) and use
// no fence or atomic: on GB300 a fused last-CTA reduction (fence + atomic ticket in
// every CTA) measured +16 us on a 60 us SpMV, more than two extra tiny launches.
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "internal.cuh"

namespace mspv {

static int64_t vec_grid(int64_t n) {   // upper bound of every wave_grid() (partials sizing)
    int64_t b = (n + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)num_sms() * 8;
    if (b > cap) b = cap;
    return b < 1 ? 1 : b;
}

// Grid of a grid-stride vector kernel: one full wave of resident CTAs (SM count x
// CTAs per SM at this kernel's register use), fewer when n is small.
template <auto Kernel>
static int64_t wave_grid(int64_t n) {
    static const int per_sm = [] {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, Kernel, kThreads, 0) != cudaSuccess || b < 1) b = 4;
        return b;
    }();
    int64_t g = (n + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)num_sms() * per_sm;
    if (g > cap) g = cap;
    return g < 1 ? 1 : g;
}

// FP64 value of an FP32 number, exactly, with integer operations only.
__device__ __forceinline__ double f32_to_f64(float v) { return widen_f32_bits(__float_as_uint(v)); }

__device__ __forceinline__ float block_sum_f32(float v, float* smem) {
    smem[threadIdx.x] = v;
    __syncthreads();
    float t = 0.0f;
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

// CTA partial of a per-thread value: written by thread 0 to partials[blockIdx.x].
__device__ __forceinline__ void write_partial(double v, double* partials) {
    __shared__ double s_red[kThreads];
    const double t = block_sum(v, s_red);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}
__device__ __forceinline__ void write_partial_f32(float v, double* partials) {
    __shared__ float s_red[kThreads];
    const float t = block_sum_f32(v, s_red);
    if (threadIdx.x == 0) partials[blockIdx.x] = f32_to_f64(t);
}

// Sum of count partials in index order (one CTA; valid in thread 0).
#define MSPV_SCALAR_LAUNCH(pdl, K, count, s, ...)                                              \
    ((count) > kScalarWideFrom ? launch_kernel(pdl, K<kScalarWide>, 1, kScalarWide, 0, s, __VA_ARGS__) \
                               : launch_kernel(pdl, K<kThreads>, 1, kThreads, 0, s, __VA_ARGS__))

// One-CTA scalar kernels run 256 threads, or 1024 when there are more than 16,384 partials
// to sum (large CSR/DIA grids); the partial count decides, so results stay deterministic.
constexpr int kScalarWide = 1024;
constexpr int64_t kScalarWideFrom = 16384;

// Sum of `count` per-CTA partials by one CTA of NT threads: thread t adds partials t, t + NT,
// t + 2 NT, ... into four accumulators (four loads in flight), then the warps and the CTA
// reduce in a fixed order, so a given count always gives the same result. The total is
// returned in thread 0.
template <int NT>
__device__ __forceinline__ double sum_partials(const double* partials, int64_t count) {
    __shared__ double s_warp[NT / 32];
    constexpr int64_t T = NT;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int64_t b = threadIdx.x;
    for (; b + 3 * T < count; b += 4 * T) {
        a0 += partials[b];
        a1 += partials[b + T];
        a2 += partials[b + 2 * T];
        a3 += partials[b + 3 * T];
    }
    for (; b < count; b += T) a0 += partials[b];
    const double v = warp_sum((a0 + a1) + (a2 + a3));
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) t = warp_sum(threadIdx.x < NT / 32 ? s_warp[threadIdx.x] : 0.0);
    __syncthreads();
    return t;
}

// ---------------------------------------------------------------------------
// scalar kernels (one CTA)
// ---------------------------------------------------------------------------
// rho = r.r, ||b||; converged at the start when r is already small enough (or b = 0).
template <int NT>
__global__ void __launch_bounds__(NT) cg_start_kernel(const double* __restrict__ prr,
                                                            const double* __restrict__ pbb, int64_t count,
                                                            CgState* st) {
    const double rr = sum_partials<NT>(prr, count);
    const double bb = sum_partials<NT>(pbb, count);
    if (threadIdx.x == 0) {
        st->rho = rr;
        st->bnorm = sqrt(bb);
        st->iters = 0;
        if (bb == 0.0 || sqrt(rr) <= st->tol * st->bnorm) {
            st->done = 1;
            st->phase = CG_CONVERGED;
        }
    }
}

// alpha = rho / p.q, or a breakdown when p.q <= 0 or alpha is not finite.
template <int NT>
__global__ void __launch_bounds__(NT) cg_alpha_kernel(const double* __restrict__ partials, int64_t count,
                                                            CgState* st) {
    pdl_wait();
    pdl_trigger();
    if (st->done) return;
    const double pq = sum_partials<NT>(partials, count);
    if (threadIdx.x == 0) finish_alpha(st, pq);
}

// rho' = r.r; stop when sqrt(rho') <= tol ||b||; beta = rho' / rho; iteration count.
template <int NT>
__global__ void __launch_bounds__(NT) cg_beta_kernel(const double* __restrict__ partials, int64_t count,
                                                           CgState* st) {
    pdl_wait();
    pdl_trigger();
    if (st->done) return;
    const double rr = sum_partials<NT>(partials, count);
    if (threadIdx.x == 0) {
        st->iters += 1;
        if (sqrt(rr) <= st->tol * st->bnorm) {
            st->rho_prev = st->rho;
            st->rho = rr;
            st->done = 1;
            st->phase = CG_CONVERGED;
        } else {
            st->beta = rr / st->rho;
            st->rho = rr;
            if (st->iters >= st->maxit) {
                st->done = 1;
                st->phase = CG_MAXIT;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// FP64 vector kernels
// ---------------------------------------------------------------------------
// r = b - q (q = A x0), p = r; partials of r.r and b.b.
__global__ void __launch_bounds__(kThreads) cg_init_kernel(int64_t n, const double* __restrict__ b,
                                                           const double* __restrict__ q, double* __restrict__ r,
                                                           double* __restrict__ p, double* __restrict__ prr,
                                                           double* __restrict__ pbb) {
    double rr = 0.0, bb = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        const double bi = b[i];
        const double ri = bi - q[i];
        r[i] = ri;
        p[i] = ri;
        rr = fma(ri, ri, rr);
        bb = fma(bi, bi, bb);
    }
    write_partial(rr, prr);
    write_partial(bb, pbb);
}

// r -= alpha q with the CTA partial of r.r. x is advanced by the p-update kernel, which reads
// p anyway (x += alpha p there saves one pass over p per iteration).
__global__ void __launch_bounds__(kThreads) cg_update_kernel(int64_t n, double* __restrict__ r,
                                                             const double* __restrict__ q,
                                                             double* __restrict__ partials, const CgState* st) {
    pdl_wait();
    pdl_trigger();
    if (st->done) return;
    const double alpha = st->alpha;
    double rr = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        rr = fma(ri, ri, rr);
    }
    write_partial(rr, partials);
}

// p = r + beta p
// Iteration `it`: x += alpha p, then p = r + beta p. Runs only when the iteration updated r
// (its beta kernel counted it: st->iters == it); on the iteration that converged or reached
// maxit only x is advanced.
__global__ void __launch_bounds__(kThreads) cg_pupdate_kernel(int64_t n, double* __restrict__ x,
                                                              const double* __restrict__ r,
                                                              double* __restrict__ p, const CgState* st,
                                                              int32_t it) {
    pdl_wait();
    pdl_trigger();
    if (st->iters != it) return;
    const double alpha = st->alpha, beta = st->beta;
    const bool more = !st->done;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        const double pi = p[i];
        x[i] = fma(alpha, pi, x[i]);
        if (more) p[i] = fma(beta, pi, r[i]);
    }
}

// Iterative refinement: r = b - q; partials of r.r and b.b.
__global__ void __launch_bounds__(kThreads) ir_residual_kernel(int64_t n, const double* __restrict__ b,
                                                               const double* __restrict__ q, double* __restrict__ r,
                                                               double* __restrict__ prr, double* __restrict__ pbb) {
    double rr = 0.0, bb = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        const double bi = b[i];
        const double ri = bi - q[i];
        r[i] = ri;
        rr = fma(ri, ri, rr);
        bb = fma(bi, bi, bb);
    }
    write_partial(rr, prr);
    write_partial(bb, pbb);
}

// rho = r.r and ||b|| of the refinement's outer residual.
template <int NT>
__global__ void __launch_bounds__(NT) ir_norms_kernel(const double* __restrict__ prr,
                                                            const double* __restrict__ pbb, int64_t count,
                                                            CgState* st) {
    const double rr = sum_partials<NT>(prr, count);
    const double bb = sum_partials<NT>(pbb, count);
    if (threadIdx.x == 0) {
        st->rho = rr;
        st->bnorm = sqrt(bb);
    }
}

__global__ void axpy1_kernel(int64_t n, double* __restrict__ x, const double* __restrict__ d) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += d[i];
}

// x = 0 when the start kernel found b = 0 (it then also marked the solve done).
__global__ void zero_if_b_zero_kernel(double* __restrict__ x, int64_t n, const CgState* st) {
    if (st->bnorm != 0.0) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = 0.0;
}

__global__ void zero_kernel(double* __restrict__ v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = 0.0;
}

// ---------------------------------------------------------------------------
// FP32-arithmetic inner solver of mixed-precision refinement: FP32 vectors and FMAs;
// alpha, beta, rho and the cross-CTA sums of every dot product in FP64. The FP32
// vectors are the library's own (16-byte aligned): the bulk is processed with 128-bit
// accesses, the n % 4 tail element by element.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) cgf_init_kernel(int64_t n, const float* __restrict__ b,
                                                            const float* __restrict__ q, float* __restrict__ r,
                                                            float* __restrict__ p, double* __restrict__ prr,
                                                            double* __restrict__ pbb) {
    float rr = 0.0f, bb = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        const float bi = b[i];
        const float ri = bi - q[i];
        r[i] = ri;
        p[i] = ri;
        rr = fmaf(ri, ri, rr);
        bb = fmaf(bi, bi, bb);
    }
    write_partial_f32(rr, prr);
    write_partial_f32(bb, pbb);
}

__global__ void __launch_bounds__(kThreads) cgf_update_kernel(int64_t n, float* __restrict__ r,
                                                              const float* __restrict__ q,
                                                              double* __restrict__ partials, const CgState* st) {
    pdl_wait();
    pdl_trigger();
    if (st->done) return;
    __shared__ float s_alpha;
    if (threadIdx.x == 0) s_alpha = (float)st->alpha;
    __syncthreads();
    const float alpha = s_alpha;
    float rr = 0.0f;
    const int64_t n4 = n / 4;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    const int64_t t0 = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    for (int64_t i = t0; i < n4; i += stride) {
        float4 rv = reinterpret_cast<float4*>(r)[i];
        const float4 qv = reinterpret_cast<const float4*>(q)[i];
        rv.x = fmaf(-alpha, qv.x, rv.x); rv.y = fmaf(-alpha, qv.y, rv.y);
        rv.z = fmaf(-alpha, qv.z, rv.z); rv.w = fmaf(-alpha, qv.w, rv.w);
        reinterpret_cast<float4*>(r)[i] = rv;
        rr = fmaf(rv.x, rv.x, rr); rr = fmaf(rv.y, rv.y, rr);
        rr = fmaf(rv.z, rv.z, rr); rr = fmaf(rv.w, rv.w, rr);
    }
    for (int64_t i = 4 * n4 + t0; i < n; i += stride) {
        const float ri = fmaf(-alpha, q[i], r[i]);
        r[i] = ri;
        rr = fmaf(ri, ri, rr);
    }
    write_partial_f32(rr, partials);
}

__global__ void __launch_bounds__(kThreads) cgf_pupdate_kernel(int64_t n, float* __restrict__ x,
                                                               const float* __restrict__ r,
                                                               float* __restrict__ p, const CgState* st,
                                                               int32_t it) {
    pdl_wait();
    pdl_trigger();
    if (st->iters != it) return;
    __shared__ float s_ab[2];
    if (threadIdx.x == 0) {
        s_ab[0] = (float)st->alpha;
        s_ab[1] = (float)st->beta;
    }
    __syncthreads();
    const float alpha = s_ab[0], beta = s_ab[1];
    const bool more = !st->done;
    const int64_t n4 = n / 4;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    const int64_t t0 = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    for (int64_t i = t0; i < n4; i += stride) {
        const float4 pv = reinterpret_cast<const float4*>(p)[i];
        float4 xv = reinterpret_cast<float4*>(x)[i];
        xv.x = fmaf(alpha, pv.x, xv.x); xv.y = fmaf(alpha, pv.y, xv.y);
        xv.z = fmaf(alpha, pv.z, xv.z); xv.w = fmaf(alpha, pv.w, xv.w);
        reinterpret_cast<float4*>(x)[i] = xv;
        if (more) {
            const float4 rv = reinterpret_cast<const float4*>(r)[i];
            float4 np;
            np.x = fmaf(beta, pv.x, rv.x); np.y = fmaf(beta, pv.y, rv.y);
            np.z = fmaf(beta, pv.z, rv.z); np.w = fmaf(beta, pv.w, rv.w);
            reinterpret_cast<float4*>(p)[i] = np;
        }
    }
    for (int64_t i = 4 * n4 + t0; i < n; i += stride) {
        const float pi = p[i];
        x[i] = fmaf(alpha, pi, x[i]);
        if (more) p[i] = fmaf(beta, pi, r[i]);
    }
}

// Refinement glue: r32 = (float)(r * scale); x += scale * (double)d32.
__global__ void ir_scale_down_kernel(int64_t n, const double* __restrict__ r, double scale,
                                     float* __restrict__ r32) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r32[i] = __double2float_rn(r[i] * scale);
}

__global__ void ir_correct_kernel(int64_t n, double* __restrict__ x, double scale, const float* __restrict__ d32) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = fma(scale, f32_to_f64(d32[i]), x[i]);
}

// Reliable-update glue: x += sigma * (double)y32 and y32 = 0 (the FP32 correction folded
// into the FP64 solution); r32 = (float)(r / sigma') with p32 = r32 + c p32 (c = 0: p32 = r32),
// the replaced residual in its new unit and the direction formed from it.
__global__ void ru_fold_kernel(int64_t n, double* __restrict__ x, double sigma, float* __restrict__ y32) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = fma(sigma, f32_to_f64(y32[i]), x[i]);
        y32[i] = 0.0f;
    }
}

__global__ void ru_restart_kernel(int64_t n, const double* __restrict__ r, double inv_sigma,
                                  float* __restrict__ r32, float* __restrict__ p32, float c) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float ri = __double2float_rn(r[i] * inv_sigma);
        r32[i] = ri;
        p32[i] = c == 0.0f ? ri : fmaf(c, p32[i], ri);
    }
}

__global__ void zero_f32_kernel(float* __restrict__ v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = 0.0f;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// Partials needed: one per CTA of the fused-dot SpMV or of a vector kernel, twice over
// (two dot products share the buffer in the init and residual kernels).
static int64_t partials_needed(const mspv_matrix* A) {
    return 2 * std::max<int64_t>(spmv_partials_needed(A), vec_grid(A->nrows));
}

static mspv_status ensure_cg_work(mspv_matrix* A) {
    CgWork& w = A->cg;
    const int64_t n = A->nrows;
    const int64_t need_partials = partials_needed(A);
    if (w.r && w.n == n && w.npartials >= need_partials) return MSPV_OK;
    auto f = [](void* p) { if (p) dev_free(p, 0); };
    f(w.r); f(w.p); f(w.q); f(w.partials); f(w.st);
    w.r = w.p = w.q = w.partials = nullptr;
    w.st = nullptr;
    MSPV_TRY(dev_alloc_n(&w.r, n));
    MSPV_TRY(dev_alloc_n(&w.p, n));
    MSPV_TRY(dev_alloc_n(&w.q, n));
    MSPV_TRY(dev_alloc_n(&w.partials, need_partials));
    MSPV_TRY(dev_alloc_n(&w.st, 2));   // [0] CG, [1] iterative-refinement outer loop
    if (!w.host_st) MSPV_CUDA_TRY(cudaMallocHost((void**)&w.host_st, 2 * sizeof(CgState)));
    w.n = n;
    w.npartials = need_partials;
    return MSPV_OK;
}

static mspv_status ensure_cg_work_f32(mspv_matrix* A) {
    MSPV_TRY(ensure_cg_work(A));
    CgWork& w = A->cg;
    const int64_t n = A->nrows;
    if (w.rf && w.nf == n) return MSPV_OK;
    auto f = [](void* p) { if (p) dev_free(p, 0); };
    f(w.rf); f(w.pf); f(w.qf);
    w.rf = w.pf = w.qf = nullptr;
    MSPV_TRY(dev_alloc_n(&w.rf, n));
    MSPV_TRY(dev_alloc_n(&w.pf, n));
    MSPV_TRY(dev_alloc_n(&w.qf, n));
    w.nf = n;
    return MSPV_OK;
}

// Programmatic dependent launches between the kernels of a CG iteration (MSPV_PDL=0 turns
// them off): each kernel's launch overlaps the end of the previous one.
static bool use_pdl() {
    const char* s = std::getenv("MSPV_PDL");
    return !(s && s[0] == '0');
}

static int check_every() {
    const char* s = std::getenv("MSPV_CG_CHECK_EVERY");
    const int v = s ? std::atoi(s) : 10;
    return v > 0 ? v : 10;
}

// Iterations launched between two polls of the stop flag: MSPV_CG_CHECK_EVERY when set, else
// 10; a run with tol <= 0 has a fixed count (only a breakdown or an exactly zero residual stops
// it early, and launches past that are no-ops), so it goes in batches of up to 256 and the GPU
// is rarely drained to poll.
static int32_t poll_batch(double tol, int32_t remaining) {
    if (tol <= 0.0 && !std::getenv("MSPV_CG_CHECK_EVERY")) return std::min<int32_t>(256, remaining);
    return std::min<int32_t>(check_every(), remaining);
}

// The CG iteration loop shared by the FP64 and the FP32-arithmetic solver: V is the
// vector type, Spmv(x, y, ep) launches the SpMV with its p.q partials.
template <typename V, typename SpmvFn, typename UpdateK, typename PupdateK>
static mspv_status cg_iterate(mspv_matrix* A, V* x, V* r, V* p, V* q, int32_t maxit, cudaStream_t s,
                              SpmvFn spmv, UpdateK update, PupdateK pupdate, unsigned Gu, unsigned Gp,
                              int32_t it0 = 0) {
    CgWork& w = A->cg;
    CgState* hst = w.host_st;
    const int64_t n = A->nrows;
    const int64_t P = spmv_partials_count(A, sizeof(V) == sizeof(float));   // exactly the partials the SpMV writes
    const bool pdl = use_pdl();
    const DotEpilogue ep{w.st, w.partials, pdl};
    const double tol = hst->tol;
    // Launch first and poll after each batch: the first batch follows the set-up kernels on the
    // stream without a host round trip (launches past a stop return at entry).
    int32_t launched = 0;
    for (;;) {
        const int32_t batch = poll_batch(tol, maxit - launched);
        for (int32_t k = 0; k < batch; ++k) {
            MSPV_TRY(spmv(p, q, ep));
            MSPV_SCALAR_LAUNCH(pdl, cg_alpha_kernel, P, s, (const double*)w.partials, P, w.st);
            launch_kernel(pdl, update, Gu, kThreads, 0, s, n, r, (const V*)q, w.partials, (const CgState*)w.st);
            MSPV_SCALAR_LAUNCH(pdl, cg_beta_kernel, (int64_t)Gu, s, (const double*)w.partials, (int64_t)Gu, w.st);
            launch_kernel(pdl, pupdate, Gp, kThreads, 0, s, n, x, (const V*)r, p, (const CgState*)w.st,
                          (int32_t)(it0 + launched + k + 1));
        }
        MSPV_CUDA_TRY(cudaGetLastError());
        launched += batch;
        MSPV_CUDA_TRY(cudaMemcpyAsync(hst, w.st, sizeof(CgState), cudaMemcpyDeviceToHost, s));
        MSPV_CUDA_TRY(cudaStreamSynchronize(s));
        if (hst->done || launched >= maxit) break;
    }
    return MSPV_OK;
}

mspv_status cg_solve(mspv_matrix* A, const double* b, double* x, double tol, int32_t maxit,
                     cudaStream_t s, int32_t* iters, double* relres) {
    if (A->nrows != A->ncols)
        return set_error(MSPV_EFORMAT, "cg: matrix is %d x %d, not square", A->nrows, A->ncols);
    if (maxit < 0) return set_error(MSPV_EINVAL, "cg: maxit < 0");
    const int64_t n = A->nrows;
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    if (n == 0) return MSPV_OK;
    if (A->format == MSPV_COO && A->nnz == 0) return set_error(MSPV_EINVAL, "cg: matrix has no entries");
    MSPV_TRY(ensure_cg_work(A));
    CgWork& w = A->cg;
    CgState* hst = w.host_st;
    *hst = CgState{};
    hst->tol = tol;
    hst->maxit = maxit;
    MSPV_CUDA_TRY(cudaMemcpyAsync(w.st, hst, sizeof(CgState), cudaMemcpyHostToDevice, s));
    const unsigned Gi = (unsigned)wave_grid<cg_init_kernel>(n);
    const unsigned Gu = (unsigned)wave_grid<cg_update_kernel>(n);
    const unsigned Gp = (unsigned)wave_grid<cg_pupdate_kernel>(n);
    const int64_t half = w.npartials / 2;

    MSPV_TRY(launch_spmv(A, x, w.q, s, DotEpilogue{nullptr, nullptr}));
    cg_init_kernel<<<Gi, kThreads, 0, s>>>(n, b, w.q, w.r, w.p, w.partials, w.partials + half);
    MSPV_SCALAR_LAUNCH(false, cg_start_kernel, (int64_t)Gi, s, (const double*)w.partials,
                       (const double*)(w.partials + half), (int64_t)Gi, w.st);
    // b = 0: the start kernel marks the solve done and the solution is 0 (decided on the device,
    // so the iterations follow without a host round trip)
    zero_if_b_zero_kernel<<<(unsigned)vec_grid(n), kThreads, 0, s>>>(x, n, w.st);
    MSPV_CUDA_TRY(cudaGetLastError());
    MSPV_TRY(cg_iterate(
        A, x, w.r, w.p, w.q, maxit, s,
        [&](const double* pp, double* qq, DotEpilogue ep) { return launch_spmv(A, pp, qq, s, ep); },
        cg_update_kernel, cg_pupdate_kernel, Gu, Gp));
    if (hst->bnorm == 0.0) return MSPV_OK;   // x = 0, no iterations, relres 0
    if (iters) *iters = hst->iters;
    if (relres) *relres = std::sqrt(hst->rho) / hst->bnorm;
    switch (hst->phase) {
        case CG_CONVERGED:
            return MSPV_OK;
        case CG_BREAKDOWN:
            return set_error(MSPV_EBREAKDOWN, "cg: breakdown at iteration %d (p.Ap = %g)", hst->iters, hst->pq);
        default:   // reached maxit (or maxit == 0)
            if (tol <= 0.0) return MSPV_OK;
            return set_error(MSPV_ENOTCONV, "cg: %d iterations, relative residual %g above %g", hst->iters,
                             std::sqrt(hst->rho) / hst->bnorm, tol);
    }
}

// CG in FP32 arithmetic on A (FP32 or BF16 stored values) for A x32 = b32, x32 from 0.
// Same iteration and stopping rule as cg_solve; the scalars live in FP64.
static mspv_status cg_solve_f32(mspv_matrix* A, const float* b32, float* x32, double tol, int32_t maxit,
                                cudaStream_t s, int32_t* iters) {
    const int64_t n = A->nrows;
    *iters = 0;
    MSPV_TRY(ensure_cg_work_f32(A));
    CgWork& w = A->cg;
    CgState* hst = w.host_st;
    *hst = CgState{};
    hst->tol = tol;
    hst->maxit = maxit;
    MSPV_CUDA_TRY(cudaMemcpyAsync(w.st, hst, sizeof(CgState), cudaMemcpyHostToDevice, s));
    const unsigned Gi = (unsigned)wave_grid<cgf_init_kernel>(n);
    const unsigned Gu = (unsigned)wave_grid<cgf_update_kernel>(n);
    const unsigned Gp = (unsigned)wave_grid<cgf_pupdate_kernel>(n);
    const int64_t half = w.npartials / 2;
    MSPV_TRY(launch_spmv_f32(A, x32, w.qf, s, DotEpilogue{nullptr, nullptr}));
    cgf_init_kernel<<<Gi, kThreads, 0, s>>>(n, b32, w.qf, w.rf, w.pf, w.partials, w.partials + half);
    MSPV_SCALAR_LAUNCH(false, cg_start_kernel, (int64_t)Gi, s, (const double*)w.partials,
                       (const double*)(w.partials + half), (int64_t)Gi, w.st);
    MSPV_CUDA_TRY(cudaGetLastError());
    MSPV_TRY(cg_iterate(
        A, x32, w.rf, w.pf, w.qf, maxit, s,
        [&](const float* pp, float* qq, DotEpilogue ep) { return launch_spmv_f32(A, pp, qq, s, ep); },
        cgf_update_kernel, cgf_pupdate_kernel, Gu, Gp));
    *iters = hst->iters;
    if (hst->phase == CG_BREAKDOWN)
        return set_error(MSPV_EBREAKDOWN, "cg (fp32 inner): breakdown at iteration %d", hst->iters);
    return MSPV_OK;
}

// Mixed precision with reliable updates (inner_fp32 = 2). One FP32-arithmetic CG on Alo runs
// throughout, on the residual in units of sigma (its FP64 norm at the last update), and
// accumulates its correction y32. The FP32 iteration stops itself, on the device, in the
// iteration where its recursive residual falls below delta (relative to the last update) or to
// the FP64 target; the update then folds sigma y32 into the FP64 x, recomputes the true
// residual b - A64 x in FP64, stops once it meets tol, and otherwise restarts the FP32
// iteration on the replaced residual in its new unit sigma' with the direction
//     p = r' + beta p,   beta = ||r'||^2 / rho_prev   (in the new unit: sigma' / (sigma rho_prev)),
// so the search direction, and with it the Krylov space, survives the update (reliable
// updated residuals, Sleijpen and van der Vorst). inner_tol <= 0 takes delta = 1e-2 for FP32
// values and 1e-1 for BF16 values, whose larger rounding of A needs more frequent updates.
static mspv_status cg_solve_ru(mspv_matrix* A64, mspv_matrix* Alo, const double* b, double* x, double tol,
                               double delta, int32_t max_updates, int32_t maxit, cudaStream_t s,
                               int32_t* updates, int32_t* iters, double* relres) {
    const int64_t n = A64->nrows;
    if (!(delta > 0.0)) delta = Alo->value_type == MSPV_BF16 ? 1e-1 : 1e-2;
    MSPV_TRY(ensure_cg_work(A64));
    MSPV_TRY(ensure_cg_work_f32(Alo));
    DevBuf rbuf, qbuf, ybuf;
    MSPV_TRY(rbuf.alloc(sizeof(double) * n));
    MSPV_TRY(qbuf.alloc(sizeof(double) * n));
    MSPV_TRY(ybuf.alloc(sizeof(float) * n));
    double* r = rbuf.as<double>();
    double* q = qbuf.as<double>();
    float* y32 = ybuf.as<float>();
    CgState* ost = A64->cg.st + 1;
    CgState* host = A64->cg.host_st + 1;
    *host = CgState{};
    MSPV_CUDA_TRY(cudaMemcpyAsync(ost, host, sizeof(CgState), cudaMemcpyHostToDevice, s));
    const unsigned G = (unsigned)vec_grid(n);
    const int64_t half = A64->cg.npartials / 2;
    auto true_residual = [&]() -> mspv_status {   // r = b - A64 x with ||r||, ||b|| in FP64
        MSPV_TRY(launch_spmv(A64, x, q, s, DotEpilogue{nullptr, nullptr}));
        ir_residual_kernel<<<G, kThreads, 0, s>>>(n, b, q, r, A64->cg.partials, A64->cg.partials + half);
        MSPV_SCALAR_LAUNCH(false, ir_norms_kernel, (int64_t)G, s, (const double*)A64->cg.partials,
                           (const double*)(A64->cg.partials + half), (int64_t)G, ost);
        MSPV_CUDA_TRY(cudaGetLastError());
        MSPV_CUDA_TRY(cudaMemcpyAsync(host, ost, sizeof(CgState), cudaMemcpyDeviceToHost, s));
        MSPV_CUDA_TRY(cudaStreamSynchronize(s));
        return MSPV_OK;
    };
    MSPV_TRY(true_residual());
    if (host->bnorm == 0.0) {
        zero_kernel<<<G, kThreads, 0, s>>>(x, n);
        MSPV_CUDA_TRY(cudaGetLastError());
        MSPV_CUDA_TRY(cudaStreamSynchronize(s));
        return MSPV_OK;
    }
    const double bnorm = host->bnorm;
    double sigma = std::sqrt(host->rho);
    if (relres) *relres = sigma / bnorm;
    if (sigma <= tol * bnorm) return MSPV_OK;

    CgWork& w = Alo->cg;
    CgState* hst = w.host_st;
    const unsigned Gu = (unsigned)wave_grid<cgf_update_kernel>(n);
    const unsigned Gp = (unsigned)wave_grid<cgf_pupdate_kernel>(n);
    ru_restart_kernel<<<G, kThreads, 0, s>>>(n, r, 1.0 / sigma, w.rf, w.pf, 0.0f);
    zero_f32_kernel<<<G, kThreads, 0, s>>>(y32, n);
    *hst = CgState{};
    hst->maxit = maxit;
    hst->bnorm = 1.0;   // the FP32 residual is measured in units of sigma
    int32_t done = 0, nupd = 0;
    mspv_status result = MSPV_ENOTCONV;
    for (;;) {
        // restart the FP32 iteration on r / sigma (unit norm); it stops below its threshold
        hst->rho = 1.0;
        hst->tol = std::max(delta, tol * bnorm / sigma);
        hst->done = 0;
        hst->phase = CG_RUNNING;
        MSPV_CUDA_TRY(cudaMemcpyAsync(w.st, hst, sizeof(CgState), cudaMemcpyHostToDevice, s));
        if (done < maxit)
            MSPV_TRY(cg_iterate(
                Alo, y32, w.rf, w.pf, w.qf, maxit - done, s,
                [&](const float* pp, float* qq, DotEpilogue ep) { return launch_spmv_f32(Alo, pp, qq, s, ep); },
                cgf_update_kernel, cgf_pupdate_kernel, Gu, Gp, done));
        if (hst->phase == CG_BREAKDOWN) {
            result = set_error(MSPV_EBREAKDOWN, "cg (reliable updates): breakdown at FP32 iteration %d", hst->iters);
            break;
        }
        done = hst->iters;
        // reliable update: fold the correction into x and replace the residual by the true one
        ru_fold_kernel<<<G, kThreads, 0, s>>>(n, x, sigma, y32);
        MSPV_TRY(true_residual());
        ++nupd;
        const double sigma_new = std::sqrt(host->rho);
        if (relres) *relres = sigma_new / bnorm;
        if (sigma_new <= tol * bnorm) { result = MSPV_OK; break; }
        if (nupd >= max_updates || done >= maxit) break;
        const double c = sigma_new / (sigma * hst->rho_prev);
        ru_restart_kernel<<<G, kThreads, 0, s>>>(n, r, 1.0 / sigma_new, w.rf, w.pf, (float)c);
        sigma = sigma_new;
    }
    if (updates) *updates = nupd;
    if (iters) *iters = done;
    MSPV_CUDA_TRY(cudaGetLastError());
    MSPV_CUDA_TRY(cudaStreamSynchronize(s));
    if (result == MSPV_ENOTCONV)
        return set_error(MSPV_ENOTCONV, "cg (reliable updates): %d FP32 iterations, %d updates, residual %g above %g",
                         done, nupd, relres ? *relres : 0.0, tol);
    if (result != MSPV_OK) return result;
    clear_error();
    return MSPV_OK;
}

mspv_status cg_solve_ir(mspv_matrix* A64, mspv_matrix* Alo, const double* b, double* x,
                        double tol, double inner_tol, int32_t max_outer, int32_t maxit_inner,
                        int32_t inner_fp32, cudaStream_t s, int32_t* outer_iters,
                        int32_t* inner_iters, double* relres) {
    if (A64->nrows != A64->ncols || Alo->nrows != A64->nrows || Alo->ncols != A64->ncols)
        return set_error(MSPV_EFORMAT, "cg_ir: matrices must be square and of equal size");
    if (max_outer < 0 || maxit_inner < 0) return set_error(MSPV_EINVAL, "cg_ir: negative iteration limit");
    if (inner_fp32 < 0 || inner_fp32 > 2) return set_error(MSPV_EINVAL, "cg_ir: inner_fp32 = %d", inner_fp32);
    if (inner_fp32 && Alo->value_type == MSPV_F64)
        return set_error(MSPV_EFORMAT, "cg_ir: FP32 inner arithmetic needs FP32 or BF16 values in Alo");
    const int64_t n = A64->nrows;
    if (outer_iters) *outer_iters = 0;
    if (inner_iters) *inner_iters = 0;
    if (relres) *relres = 0.0;
    if (n == 0) return MSPV_OK;
    if (inner_fp32 == 2)
        return cg_solve_ru(A64, Alo, b, x, tol, inner_tol, max_outer, maxit_inner, s, outer_iters, inner_iters,
                           relres);
    MSPV_TRY(ensure_cg_work(A64));
    // outer vectors are separate buffers so that Alo may be the same handle as A64
    DevBuf rbuf, dbuf, qbuf, r32buf, d32buf;
    MSPV_TRY(rbuf.alloc(sizeof(double) * n));
    MSPV_TRY(qbuf.alloc(sizeof(double) * n));
    if (inner_fp32) {
        MSPV_TRY(r32buf.alloc(sizeof(float) * n));
        MSPV_TRY(d32buf.alloc(sizeof(float) * n));
    } else {
        MSPV_TRY(dbuf.alloc(sizeof(double) * n));
    }
    double* r = rbuf.as<double>();
    double* d = dbuf.as<double>();
    double* q = qbuf.as<double>();
    float* r32 = r32buf.as<float>();
    float* d32 = d32buf.as<float>();
    CgState* ost = A64->cg.st + 1;
    CgState* host = A64->cg.host_st + 1;
    *host = CgState{};
    MSPV_CUDA_TRY(cudaMemcpyAsync(ost, host, sizeof(CgState), cudaMemcpyHostToDevice, s));
    const unsigned G = (unsigned)vec_grid(n);
    const int64_t half = A64->cg.npartials / 2;
    int32_t total_inner = 0;
    mspv_status result = MSPV_ENOTCONV;
    for (int32_t k = 0;; ++k) {
        MSPV_TRY(launch_spmv(A64, x, q, s, DotEpilogue{nullptr, nullptr}));
        ir_residual_kernel<<<G, kThreads, 0, s>>>(n, b, q, r, A64->cg.partials, A64->cg.partials + half);
        MSPV_SCALAR_LAUNCH(false, ir_norms_kernel, (int64_t)G, s, (const double*)A64->cg.partials,
                           (const double*)(A64->cg.partials + half), (int64_t)G, ost);
        MSPV_CUDA_TRY(cudaGetLastError());
        MSPV_CUDA_TRY(cudaMemcpyAsync(host, ost, sizeof(CgState), cudaMemcpyDeviceToHost, s));
        MSPV_CUDA_TRY(cudaStreamSynchronize(s));
        if (host->bnorm == 0.0) {
            zero_kernel<<<G, kThreads, 0, s>>>(x, n);
            MSPV_CUDA_TRY(cudaStreamSynchronize(s));
            result = MSPV_OK;
            break;
        }
        const double rnorm = std::sqrt(host->rho);
        const double rel = rnorm / host->bnorm;
        if (relres) *relres = rel;
        if (outer_iters) *outer_iters = k;
        if (rel <= tol) { result = MSPV_OK; break; }
        if (k == max_outer) { result = MSPV_ENOTCONV; break; }
        int32_t it = 0;
        mspv_status st;
        if (inner_fp32) {
            // solve A d = r / ||r|| in FP32 (a unit right-hand side keeps FP32 in range as
            // the outer residual shrinks), then x += ||r|| d in FP64
            ir_scale_down_kernel<<<G, kThreads, 0, s>>>(n, r, 1.0 / rnorm, r32);
            zero_f32_kernel<<<G, kThreads, 0, s>>>(d32, n);
            st = cg_solve_f32(Alo, r32, d32, inner_tol, maxit_inner, s, &it);
            if (st == MSPV_OK) ir_correct_kernel<<<G, kThreads, 0, s>>>(n, x, rnorm, d32);
        } else {
            zero_kernel<<<G, kThreads, 0, s>>>(d, n);
            double inner_rel = 0.0;
            st = cg_solve(Alo, r, d, inner_tol, maxit_inner, s, &it, &inner_rel);
            if (st == MSPV_OK || st == MSPV_ENOTCONV) {
                axpy1_kernel<<<G, kThreads, 0, s>>>(n, x, d);
                st = MSPV_OK;
            }
        }
        total_inner += it;
        if (st != MSPV_OK) {
            result = st;
            break;
        }
        MSPV_CUDA_TRY(cudaGetLastError());
    }
    if (inner_iters) *inner_iters = total_inner;
    MSPV_CUDA_TRY(cudaStreamSynchronize(s));
    if (result == MSPV_ENOTCONV)
        return set_error(MSPV_ENOTCONV, "cg_ir: %d corrections, residual above %g", max_outer, tol);
    if (result != MSPV_OK) return result;
    clear_error();
    return MSPV_OK;
}

}  // namespace mspv
