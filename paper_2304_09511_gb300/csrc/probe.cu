// Device characterisation for the roofline of the FP64 kernels: the FP64 fused multiply-add
// issue rate of the current device (not part of the paper's method). On GB300 the FP64 pipe,
// not HBM, bounds the FP64 DIA SpMV, so its roofline needs this rate as its peak; measuring it
// on the device that runs the benchmark replaces a rate derived from the SM count and clock.
#include <algorithm>
#include <climits>

#include "internal.cuh"

namespace mspv {

// Every thread runs C independent chains acc = m * y + acc for `iters` steps, the dependence
// running through the addend as in an SpMV row sum (the values stay near 1: no overflow, no
// subnormals), then stores their sum, so nothing is dead code. y comes in as an argument
// (a register, not a constant-bank operand); each chain has its own multiplicand.
template <int C>
__global__ void __launch_bounds__(kThreads) fp64_fma_probe_kernel(int32_t iters, double y,
                                                                  double* __restrict__ out) {
    const int64_t tid = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    double acc[C], m[C];
#pragma unroll
    for (int k = 0; k < C; ++k) {
        acc[k] = 1.0 + 1e-3 * k + 1e-9 * (double)threadIdx.x;
        m[k] = 1e-8 * (k + 1);
    }
    for (int32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < C; ++k) acc[k] = fma(m[k], y, acc[k]);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < C; ++k) s += acc[k];
    out[tid] = s;
}

// One full wave (the most CTAs of this kernel the device holds at once) launched `repeats` + 1
// times; the fastest of the timed launches, in FMA per second.
template <int C>
static mspv_status probe_rate(int32_t iters, int32_t repeats, cudaStream_t s, double* out_buf,
                              int64_t max_threads, cudaEvent_t e0, cudaEvent_t e1, double* fma_per_s) {
    int per_sm = 0;
    MSPV_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp64_fma_probe_kernel<C>, kThreads, 0));
    int64_t ctas = (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
    if (ctas * kThreads > max_threads) ctas = max_threads / kThreads;
    float best = 0.0f;
    for (int r = 0; r <= repeats; ++r) {   // the first launch warms up
        MSPV_CUDA_TRY(cudaEventRecord(e0, s));
        fp64_fma_probe_kernel<C><<<(unsigned)ctas, kThreads, 0, s>>>(iters, 0.999, out_buf);
        MSPV_CUDA_TRY(cudaGetLastError());
        MSPV_CUDA_TRY(cudaEventRecord(e1, s));
        MSPV_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.0f;
        MSPV_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (r > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    *fma_per_s = (double)ctas * kThreads * (double)iters * C / (best * 1e-3);
    return MSPV_OK;
}

}  // namespace mspv

using namespace mspv;

extern "C" MSPV_API mspv_status mspv_fp64_fma_rate(int64_t iters, int32_t repeats, void* stream,
                                                   double* tflops) {
    try {
        if (iters < 1 || iters > (1 << 30) || repeats < 1 || !tflops)
            return set_error(MSPV_EINVAL, "fp64_fma_rate: bad argument");
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        const int64_t max_threads = (int64_t)num_sms() * 2048;
        DevBuf out;
        MSPV_TRY(out.alloc(sizeof(double) * (size_t)max_threads));
        cudaEvent_t e0, e1;
        MSPV_CUDA_TRY(cudaEventCreate(&e0));
        if (cudaEventCreate(&e1) != cudaSuccess) {
            cudaEventDestroy(e0);
            return set_error(MSPV_ECUDA, "fp64_fma_rate: cudaEventCreate failed");
        }
        // 4, 8 and 16 independent chains per thread (the chain count changes how much FMA
        // latency the warps must hide); the fastest is the rate. Work per launch is kept
        // equal: iters scaled by 8 / C.
        double r4 = 0.0, r8 = 0.0, r16 = 0.0;
        const int32_t it = (int32_t)iters;
        mspv_status st = probe_rate<4>(2 * it, repeats, s, out.as<double>(), max_threads, e0, e1, &r4);
        if (st == MSPV_OK) st = probe_rate<8>(it, repeats, s, out.as<double>(), max_threads, e0, e1, &r8);
        if (st == MSPV_OK) st = probe_rate<16>(std::max<int32_t>(1, it / 2), repeats, s, out.as<double>(),
                                               max_threads, e0, e1, &r16);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (st != MSPV_OK) return st;
        *tflops = 2.0 * std::max(r4, std::max(r8, r16)) / 1e12;
        clear_error();
        return MSPV_OK;
    } catch (...) {
        return set_error(MSPV_ECUDA, "fp64_fma_rate: internal error");
    }
}
