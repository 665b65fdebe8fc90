// Format selection (not in the paper beyond its run-first auto-tuner, Sec. VI): the ten
// sparsity features of a matrix, the exhaustive "time every format" tuner, and a small
// FP32 MLP (10 -> 64 -> 64 -> 3, ReLU) that predicts the fastest of COO / CSR / DIA,
// trained and evaluated by hand-written kernels.
//
// Training is one CTA: Adam over minibatches of 64 samples taken in index order every
// epoch; every gradient entry is a sum over the minibatch in sample order, computed by
// one thread, so training is deterministic. Weights start from a SplitMix64 counter
// stream (uniform Glorot), identical to the host reference.
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdint>
#include <vector>

#include "internal.cuh"

namespace mspv {

// ---------------------------------------------------------------------------
// features
// ---------------------------------------------------------------------------
// Marks each diagonal offset present (flag index col - row + nrows - 1) and finds the largest
// |col - row|.
__global__ void diag_flags_coo_kernel(const int32_t* __restrict__ ai, const int32_t* __restrict__ aj, int64_t nnz,
                                      int32_t n, uint8_t* __restrict__ flags, int32_t* __restrict__ band) {
    int32_t b = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = aj[e] - ai[e];
        flags[(int64_t)d + n - 1] = 1;
        b = max(b, abs(d));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
    if ((threadIdx.x & 31) == 0) atomicMax(band, b);
}

__global__ void diag_flags_csr_kernel(const int32_t* __restrict__ irp, const int32_t* __restrict__ aj, int32_t n,
                                      uint8_t* __restrict__ flags, int32_t* __restrict__ band) {
    int32_t b = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        for (int32_t j = irp[r]; j < irp[r + 1]; ++j) {
            const int32_t d = aj[j] - (int32_t)r;
            flags[(int64_t)d + n - 1] = 1;
            b = max(b, abs(d));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
    if ((threadIdx.x & 31) == 0) atomicMax(band, b);
}

__global__ void count_flags_kernel(const uint8_t* __restrict__ flags, int64_t m, unsigned long long* count) {
    unsigned long long c = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        c += flags[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(count, c);
}

static unsigned grid_cap(int64_t m) {
    int64_t g = (m + kThreads - 1) / kThreads;
    if (g > (int64_t)num_sms() * 16) g = (int64_t)num_sms() * 16;
    return (unsigned)(g < 1 ? 1 : g);
}

// Distinct diagonals and bandwidth (integer counts on the device).
static mspv_status diag_stats(const mspv_matrix* A, cudaStream_t s, int64_t* ndiags, int64_t* band) {
    const int32_t n = A->nrows;
    *ndiags = 0;
    *band = 0;
    if (A->format == MSPV_DIA) {
        *ndiags = A->ndiags;
        if (A->ndiags > 0) {
            std::vector<int32_t> off(A->ndiags);
            MSPV_CUDA_TRY(cudaMemcpyAsync(off.data(), A->doff, 4 * A->ndiags, cudaMemcpyDeviceToHost, s));
            MSPV_CUDA_TRY(cudaStreamSynchronize(s));
            for (int32_t d : off) *band = std::max<int64_t>(*band, d < 0 ? -(int64_t)d : d);
        }
        return MSPV_OK;
    }
    if (n == 0 || A->ncols == 0 || A->nnz == 0) return MSPV_OK;
    const int64_t span = (int64_t)n + A->ncols - 1;   // offsets -(nrows - 1) .. ncols - 1
    DevBuf flags, cnt;
    MSPV_TRY(flags.alloc((size_t)span));
    MSPV_TRY(cnt.alloc(sizeof(unsigned long long) + sizeof(int32_t)));
    MSPV_CUDA_TRY(cudaMemsetAsync(flags.ptr, 0, (size_t)span, s));
    MSPV_CUDA_TRY(cudaMemsetAsync(cnt.ptr, 0, sizeof(unsigned long long) + sizeof(int32_t), s));
    unsigned long long* d_count = cnt.as<unsigned long long>();
    int32_t* d_band = reinterpret_cast<int32_t*>(d_count + 1);
    if (A->format == MSPV_COO)
        diag_flags_coo_kernel<<<grid_cap(A->nnz), kThreads, 0, s>>>(A->ai, A->aj, A->nnz, n, flags.as<uint8_t>(), d_band);
    else
        diag_flags_csr_kernel<<<grid_cap(n), kThreads, 0, s>>>(A->irp, A->aj, n, flags.as<uint8_t>(), d_band);
    count_flags_kernel<<<grid_cap(span), kThreads, 0, s>>>(flags.as<uint8_t>(), span, d_count);
    MSPV_CUDA_TRY(cudaGetLastError());
    unsigned long long h[2] = {0, 0};
    MSPV_CUDA_TRY(cudaMemcpyAsync(h, cnt.ptr, sizeof(unsigned long long) + sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    MSPV_CUDA_TRY(cudaStreamSynchronize(s));
    *ndiags = (int64_t)h[0];
    *band = (int64_t)(int32_t)(h[1] & 0xffffffffull);
    return MSPV_OK;
}

mspv_status compute_features(const mspv_matrix* A, float* out, cudaStream_t s, int64_t* ndiags) {
    int64_t nd = 0, band = 0;
    MSPV_TRY(diag_stats(A, s, &nd, &band));
    if (ndiags) *ndiags = nd;
    const double n = (double)A->nrows;
    const double nnz = (double)A->nnz;
    const double nn = n > 0 ? n : 1.0;
    double f[kSelectorFeatures];
    f[0] = std::log2(n > 1 ? n : 1.0);
    f[1] = std::log2(nnz > 1 ? nnz : 1.0);
    f[2] = A->row_mean;
    f[3] = A->row_std;
    f[4] = (double)A->row_max;
    f[5] = (double)A->row_min;
    f[6] = std::log2(nd > 1 ? (double)nd : 1.0);
    f[7] = nd > 0 ? nnz / ((double)nd * nn) : 0.0;
    f[8] = (double)A->empty_rows / nn;
    f[9] = (double)band / nn;
    for (int k = 0; k < kSelectorFeatures; ++k) out[k] = (float)f[k];
    return MSPV_OK;
}

// ---------------------------------------------------------------------------
// MLP 10 -> 64 -> 64 -> 3
// ---------------------------------------------------------------------------
constexpr int NF = kSelectorFeatures, NH = 64, NC = 3, NB = 64;
constexpr int OFF_MU = 0, OFF_SD = NF, OFF_LO = 2 * NF, OFF_HI = 3 * NF, OFF_W1 = 4 * NF,
              OFF_B1 = OFF_W1 + NH * NF, OFF_W2 = OFF_B1 + NH,
              OFF_B2 = OFF_W2 + NH * NH, OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NC * NH,
              NPARAM = OFF_B3 + NC;
static_assert(NPARAM == kSelectorParams, "parameter layout");

// Output k (0-based) of SplitMix64 seeded with `seed` (Steele, Lea, Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014): the state advances by the golden gamma
// before each output, so output k mixes seed + (k + 1) * gamma.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Initial value of parameter `a` (absolute index in the layout, a >= OFF_W1): a weight is
// (2u - 1) sqrt(6 / (fan_in + fan_out)) with u = (top 24 bits of SplitMix64 output
// a - OFF_W1) / 2^24 (uniform Glorot); biases start at zero.
__device__ __forceinline__ float init_param(uint64_t seed, int a) {
    int fan_in, fan_out;
    if (a < OFF_B1) { fan_in = NF; fan_out = NH; }
    else if (a < OFF_W2) return 0.0f;
    else if (a < OFF_B2) { fan_in = NH; fan_out = NH; }
    else if (a < OFF_W3) return 0.0f;
    else if (a < OFF_B3) { fan_in = NH; fan_out = NC; }
    else return 0.0f;
    const float u = (float)(splitmix64_at(seed, (uint64_t)(a - OFF_W1)) >> 40) * (1.0f / 16777216.0f);
    return (2.0f * u - 1.0f) * sqrtf(6.0f / (float)(fan_in + fan_out));
}

struct TrainSmem {
    float p[NPARAM];
    float m[NPARAM];
    float v[NPARAM];
    float g[NPARAM];
    float xb[NB][NF];
    float h1[NB][NH];
    float h2[NB][NH];   // reused for dH1
    float dh[NB][NH];   // dH2
    float lg[NB][NC];   // logits, then dL
};

__global__ void __launch_bounds__(kThreads) selector_train_kernel(const float* __restrict__ X,
                                                                  const int32_t* __restrict__ y, int32_t N,
                                                                  int32_t epochs, float lr, uint64_t seed,
                                                                  float* __restrict__ params) {
    extern __shared__ __align__(16) unsigned char raw[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(raw);
    const int t = threadIdx.x;
    // standardisation: per-feature mean and standard deviation (sequential, in order)
    if (t < NF) {
        double sm = 0.0, sq = 0.0;
        for (int i = 0; i < N; ++i) sm += X[(int64_t)i * NF + t];
        const double mu = sm / (N > 0 ? N : 1);
        for (int i = 0; i < N; ++i) {
            const double d = X[(int64_t)i * NF + t] - mu;
            sq += d * d;
        }
        const double sd = sqrt(sq / (N > 0 ? N : 1));
        float lo = X[t], hi = X[t];
        for (int i = 1; i < N; ++i) {
            lo = fminf(lo, X[(int64_t)i * NF + t]);
            hi = fmaxf(hi, X[(int64_t)i * NF + t]);
        }
        S.p[OFF_MU + t] = (float)mu;
        S.p[OFF_SD + t] = sd > 1e-6 ? (float)sd : 1.0f;
        S.p[OFF_LO + t] = lo;
        S.p[OFF_HI + t] = hi;
    }
    for (int k = OFF_W1 + t; k < NPARAM; k += kThreads) {
        S.p[k] = init_param(seed, k);
        S.m[k] = 0.0f;
        S.v[k] = 0.0f;
    }
    __syncthreads();
    const float b1c = 0.9f, b2c = 0.999f, eps = 1e-8f;
    float b1t = 1.0f, b2t = 1.0f;
    const int nchunks = (N + NB - 1) / NB;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int c = 0; c < nchunks; ++c) {
            const int i0 = c * NB;
            const int nb = (N - i0 < NB) ? N - i0 : NB;
            // forward
            for (int q = t; q < nb * NF; q += kThreads) {
                const int sidx = q / NF, f = q % NF;
                S.xb[sidx][f] = (X[(int64_t)(i0 + sidx) * NF + f] - S.p[OFF_MU + f]) / S.p[OFF_SD + f];
            }
            __syncthreads();
            for (int q = t; q < nb * NH; q += kThreads) {
                const int sidx = q / NH, j = q % NH;
                float a = S.p[OFF_B1 + j];
                for (int f = 0; f < NF; ++f) a = fmaf(S.p[OFF_W1 + j * NF + f], S.xb[sidx][f], a);
                S.h1[sidx][j] = a > 0.0f ? a : 0.0f;
            }
            __syncthreads();
            for (int q = t; q < nb * NH; q += kThreads) {
                const int sidx = q / NH, k = q % NH;
                float a = S.p[OFF_B2 + k];
                for (int j = 0; j < NH; ++j) a = fmaf(S.p[OFF_W2 + k * NH + j], S.h1[sidx][j], a);
                S.h2[sidx][k] = a > 0.0f ? a : 0.0f;
            }
            __syncthreads();
            for (int q = t; q < nb * NC; q += kThreads) {
                const int sidx = q / NC, cl = q % NC;
                float a = S.p[OFF_B3 + cl];
                for (int k = 0; k < NH; ++k) a = fmaf(S.p[OFF_W3 + cl * NH + k], S.h2[sidx][k], a);
                S.lg[sidx][cl] = a;
            }
            __syncthreads();
            // softmax cross-entropy gradient, mean over the minibatch
            if (t < nb) {
                const float l0 = S.lg[t][0], l1 = S.lg[t][1], l2 = S.lg[t][2];
                const float mx = fmaxf(l0, fmaxf(l1, l2));
                const float e0 = expf(l0 - mx), e1 = expf(l1 - mx), e2 = expf(l2 - mx);
                const float inv = 1.0f / (e0 + e1 + e2);
                const int lab = y[i0 + t];
                S.lg[t][0] = (e0 * inv - (lab == 0 ? 1.0f : 0.0f)) / (float)nb;
                S.lg[t][1] = (e1 * inv - (lab == 1 ? 1.0f : 0.0f)) / (float)nb;
                S.lg[t][2] = (e2 * inv - (lab == 2 ? 1.0f : 0.0f)) / (float)nb;
            }
            __syncthreads();
            // layer 3 gradients and dH2
            for (int q = t; q < NC * NH; q += kThreads) {
                const int cl = q / NH, k = q % NH;
                float a = 0.0f;
                for (int sidx = 0; sidx < nb; ++sidx) a = fmaf(S.lg[sidx][cl], S.h2[sidx][k], a);
                S.g[OFF_W3 + q] = a;
            }
            if (t < NC) {
                float a = 0.0f;
                for (int sidx = 0; sidx < nb; ++sidx) a += S.lg[sidx][t];
                S.g[OFF_B3 + t] = a;
            }
            for (int q = t; q < nb * NH; q += kThreads) {
                const int sidx = q / NH, k = q % NH;
                float a = 0.0f;
                for (int cl = 0; cl < NC; ++cl) a = fmaf(S.lg[sidx][cl], S.p[OFF_W3 + cl * NH + k], a);
                S.dh[sidx][k] = S.h2[sidx][k] > 0.0f ? a : 0.0f;
            }
            __syncthreads();
            // layer 2 gradients and dH1 (into h2)
            for (int q = t; q < NH * NH; q += kThreads) {
                const int k = q / NH, j = q % NH;
                float a = 0.0f;
                for (int sidx = 0; sidx < nb; ++sidx) a = fmaf(S.dh[sidx][k], S.h1[sidx][j], a);
                S.g[OFF_W2 + q] = a;
            }
            if (t < NH) {
                float a = 0.0f;
                for (int sidx = 0; sidx < nb; ++sidx) a += S.dh[sidx][t];
                S.g[OFF_B2 + t] = a;
            }
            for (int q = t; q < nb * NH; q += kThreads) {
                const int sidx = q / NH, j = q % NH;
                float a = 0.0f;
                for (int k = 0; k < NH; ++k) a = fmaf(S.dh[sidx][k], S.p[OFF_W2 + k * NH + j], a);
                S.h2[sidx][j] = S.h1[sidx][j] > 0.0f ? a : 0.0f;
            }
            __syncthreads();
            // layer 1 gradients
            for (int q = t; q < NH * NF; q += kThreads) {
                const int j = q / NF, f = q % NF;
                float a = 0.0f;
                for (int sidx = 0; sidx < nb; ++sidx) a = fmaf(S.h2[sidx][j], S.xb[sidx][f], a);
                S.g[OFF_W1 + q] = a;
            }
            if (t < NH) {
                float a = 0.0f;
                for (int sidx = 0; sidx < nb; ++sidx) a += S.h2[sidx][t];
                S.g[OFF_B1 + t] = a;
            }
            __syncthreads();
            // Adam
            b1t *= b1c;
            b2t *= b2c;
            for (int k = OFF_W1 + t; k < NPARAM; k += kThreads) {
                const float gk = S.g[k];
                const float mk = b1c * S.m[k] + (1.0f - b1c) * gk;
                const float vk = b2c * S.v[k] + (1.0f - b2c) * gk * gk;
                S.m[k] = mk;
                S.v[k] = vk;
                const float mh = mk / (1.0f - b1t), vh = vk / (1.0f - b2t);
                S.p[k] -= lr * mh / (sqrtf(vh) + eps);
            }
            __syncthreads();
        }
    }
    for (int k = t; k < NPARAM; k += kThreads) params[k] = S.p[k];
}

// One thread per sample: standardise, forward, arg max (lowest class on ties).
__global__ void selector_predict_kernel(const float* __restrict__ params, const float* __restrict__ X, int32_t N,
                                        int32_t* __restrict__ out) {
    __shared__ float p[NPARAM];
    for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) p[k] = params[k];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float xb[NF], h1[NH];
    // features outside the training range are clamped to it: a matrix larger (or more
    // skewed) than any training matrix is judged like the most extreme ones seen
    for (int f = 0; f < NF; ++f)
        xb[f] = (fminf(fmaxf(X[i * NF + f], p[OFF_LO + f]), p[OFF_HI + f]) - p[OFF_MU + f]) / p[OFF_SD + f];
    for (int j = 0; j < NH; ++j) {
        float a = p[OFF_B1 + j];
        for (int f = 0; f < NF; ++f) a = fmaf(p[OFF_W1 + j * NF + f], xb[f], a);
        h1[j] = a > 0.0f ? a : 0.0f;
    }
    float lg[NC];
    for (int cl = 0; cl < NC; ++cl) lg[cl] = p[OFF_B3 + cl];
    for (int k = 0; k < NH; ++k) {
        float a = p[OFF_B2 + k];
        for (int j = 0; j < NH; ++j) a = fmaf(p[OFF_W2 + k * NH + j], h1[j], a);
        const float h2 = a > 0.0f ? a : 0.0f;
        for (int cl = 0; cl < NC; ++cl) lg[cl] = fmaf(p[OFF_W3 + cl * NH + k], h2, lg[cl]);
    }
    int best = 0;
    for (int cl = 1; cl < NC; ++cl)
        if (lg[cl] > lg[best]) best = cl;
    out[i] = best;
}

mspv_status selector_train(const float* X, const int32_t* y, int32_t N, int32_t epochs, float lr, uint64_t seed,
                           float* params, cudaStream_t s) {
    DevBuf dX, dy, dp;
    MSPV_TRY(dX.alloc(sizeof(float) * (size_t)N * NF));
    MSPV_TRY(dy.alloc(sizeof(int32_t) * (size_t)N));
    MSPV_TRY(dp.alloc(sizeof(float) * NPARAM));
    MSPV_CUDA_TRY(cudaMemcpyAsync(dX.ptr, X, sizeof(float) * (size_t)N * NF, cudaMemcpyHostToDevice, s));
    MSPV_CUDA_TRY(cudaMemcpyAsync(dy.ptr, y, sizeof(int32_t) * (size_t)N, cudaMemcpyHostToDevice, s));
    const size_t smem = sizeof(TrainSmem);
    MSPV_CUDA_TRY(cudaFuncSetAttribute(selector_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    selector_train_kernel<<<1, kThreads, smem, s>>>(dX.as<float>(), dy.as<int32_t>(), N, epochs, lr, seed,
                                                    dp.as<float>());
    MSPV_CUDA_TRY(cudaGetLastError());
    MSPV_CUDA_TRY(cudaMemcpyAsync(params, dp.ptr, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, s));
    MSPV_CUDA_TRY(cudaStreamSynchronize(s));
    return MSPV_OK;
}

mspv_status selector_predict(const float* params, const float* X, int32_t N, int32_t* out, cudaStream_t s) {
    if (N == 0) return MSPV_OK;
    DevBuf dX, dp, dout;
    MSPV_TRY(dX.alloc(sizeof(float) * (size_t)N * NF));
    MSPV_TRY(dp.alloc(sizeof(float) * NPARAM));
    MSPV_TRY(dout.alloc(sizeof(int32_t) * (size_t)N));
    MSPV_CUDA_TRY(cudaMemcpyAsync(dX.ptr, X, sizeof(float) * (size_t)N * NF, cudaMemcpyHostToDevice, s));
    MSPV_CUDA_TRY(cudaMemcpyAsync(dp.ptr, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, s));
    selector_predict_kernel<<<(unsigned)((N + 127) / 128), 128, 0, s>>>(dp.as<float>(), dX.as<float>(), N,
                                                                        dout.as<int32_t>());
    MSPV_CUDA_TRY(cudaGetLastError());
    MSPV_CUDA_TRY(cudaMemcpyAsync(out, dout.ptr, sizeof(int32_t) * (size_t)N, cudaMemcpyDeviceToHost, s));
    MSPV_CUDA_TRY(cudaStreamSynchronize(s));
    return MSPV_OK;
}

// ---------------------------------------------------------------------------
// run-first tuning: time y = A x in every format that can be built
// ---------------------------------------------------------------------------
__global__ void fill_ones_kernel(double* __restrict__ v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = 1.0;
}

static mspv_status time_spmv(const mspv_matrix* M, const double* x, double* y, int32_t reps, cudaStream_t s,
                             double* ms) {
    cudaEvent_t e0, e1;
    MSPV_CUDA_TRY(cudaEventCreate(&e0));
    MSPV_CUDA_TRY(cudaEventCreate(&e1));
    mspv_status st = MSPV_OK;
    for (int w = 0; w < 2 && st == MSPV_OK; ++w) st = launch_spmv(M, x, y, s, DotEpilogue{nullptr, nullptr});
    if (st == MSPV_OK) {
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st == MSPV_OK; ++r) st = launch_spmv(M, x, y, s, DotEpilogue{nullptr, nullptr});
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        *ms = (double)t / (reps > 0 ? reps : 1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

mspv_status tune_formats(const mspv_matrix* A, int32_t reps, cudaStream_t s, double* ms, int32_t* best) {
    if (A->format == MSPV_DIA) return set_error(MSPV_EFORMAT, "tune: pass a COO or CSR handle");
    for (int k = 0; k < 3; ++k) ms[k] = INFINITY;
    DevBuf xb, yb;
    MSPV_TRY(xb.alloc(sizeof(double) * (size_t)(A->ncols > 0 ? A->ncols : 1)));
    MSPV_TRY(yb.alloc(sizeof(double) * (size_t)(A->nrows > 0 ? A->nrows : 1)));
    if (A->ncols > 0) fill_ones_kernel<<<grid_cap(A->ncols), kThreads, 0, s>>>(xb.as<double>(), A->ncols);
    for (int f = 0; f < 3; ++f) {
        if (f == A->format) {
            MSPV_TRY(time_spmv(A, xb.as<double>(), yb.as<double>(), reps, s, &ms[f]));
            continue;
        }
        mspv_matrix M;
        M.device = A->device;
        const mspv_status st = build_from(A, f, MSPV_F64, s, &M);
        if (st == MSPV_OK) {
            const mspv_status t = time_spmv(&M, xb.as<double>(), yb.as<double>(), reps, s, &ms[f]);
            cudaStreamSynchronize(s);
            free_matrix(&M);
            if (t != MSPV_OK) return t;
        } else {
            cudaStreamSynchronize(s);
            free_matrix(&M);
            if (st != MSPV_ETOOBIG && st != MSPV_EFORMAT) return st;   // DIA infeasible: stays +inf
        }
    }
    // fastest; ties within 1% prefer CSR, then DIA, then COO
    const int order[3] = {MSPV_CSR, MSPV_DIA, MSPV_COO};
    int b = order[0];
    for (int k = 1; k < 3; ++k)
        if (ms[order[k]] < ms[b] * 0.99) b = order[k];
    *best = b;
    clear_error();
    return MSPV_OK;
}

mspv_status select_format(const mspv_matrix* A, const float* params, cudaStream_t s, int32_t* best) {
    if (!params) {
        double ms[3];
        return tune_formats(A, 10, s, ms, best);
    }
    float f[kSelectorFeatures];
    int64_t nd = 0;
    MSPV_TRY(compute_features(A, f, s, &nd));
    int32_t pick = MSPV_CSR;
    MSPV_TRY(selector_predict(params, f, 1, &pick, s));
    if (pick == MSPV_DIA) {
        const double npad = (double)(((int64_t)A->nrows + 31) / 32 * 32);
        if (A->nrows != A->ncols || (double)nd * npad > dia_slot_cap(A->nnz)) pick = MSPV_CSR;
    }
    *best = pick;
    return MSPV_OK;
}

}  // namespace mspv
