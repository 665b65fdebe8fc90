// Allocation-free COO SpMV: mspv_spmv_coo_noalloc.
//
// Some callers cannot call cudaMalloc: applications whose device memory is reserved up
// front or strictly budgeted by their own allocator -- a framework's caching allocator
// that has already taken the free memory, or a service that accounts for every byte --
// where one more cudaMalloc would fail or break the budget. This entry point runs the COO SpMV on
// triplets the caller already holds on the device and keeps the kernel's only scratch
// -- one carry record per window of 3072 entries -- in a fixed-size array compiled
// into the library. The array lives in device memory on every GPU that loads the
// library, for as long as the process runs; it is shared by all calls, so calls that
// overlap on the GPU race on it.
#include <mutex>

#include "internal.cuh"

namespace mspv {

constexpr int64_t kNoAllocMaxWindows = 65536;                       // 1.5 MiB of carry records
constexpr int64_t kNoAllocMaxEntries = kNoAllocMaxWindows * kCooWindow;   // 201,326,592 entries
constexpr int kNoAllocMaxDevices = 64;

struct NoAllocScratch {
    CooCarry carry[kNoAllocMaxWindows];
    int32_t flags[4];   // [0]: index outside the shape, [1]: rows not non-decreasing
};

// The scratch array. Host code must not use this name as a device address: it is a
// host-side stand-in; the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

static std::mutex g_noalloc_mu;
static NoAllocScratch* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device
// (with that device current) and cached for the life of the process. cudaDeviceReset unloads
// the module and would leave the cached address stale: the entry point is documented as not
// callable after a device reset.
static mspv_status noalloc_scratch(NoAllocScratch** out) {
    int dev = 0;
    MSPV_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return set_error(MSPV_EINVAL, "spmv_coo_noalloc: device ordinal %d beyond %d", dev, kNoAllocMaxDevices);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        MSPV_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_addr[dev] = static_cast<NoAllocScratch*>(p);
    }
    *out = g_noalloc_addr[dev];
    return MSPV_OK;
}

// Flags entries outside [0, nrows) x [0, ncols) and rows that decrease.
__global__ void noalloc_check_kernel(const int32_t* __restrict__ ai, const int32_t* __restrict__ aj,
                                     int64_t nnz, int32_t nrows, int32_t ncols, int32_t* flags) {
    int bad = 0, unsorted = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = ai[e], c = aj[e];
        bad |= (r < 0) | (r >= nrows) | (c < 0) | (c >= ncols);
        if (e > 0) unsorted |= (ai[e - 1] > r);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&flags[0], 1);
    if (__any_sync(0xffffffffu, unsorted) && (threadIdx.x & 31) == 0) atomicOr(&flags[1], 1);
}

}  // namespace mspv

using namespace mspv;

extern "C" MSPV_API mspv_status mspv_spmv_coo_noalloc(int32_t nrows, int32_t ncols, int64_t nnz,
                                                      const int32_t* rows, const int32_t* cols,
                                                      const double* vals, const double* x, double* y,
                                                      void* stream) {
    try {
        if (nrows < 0 || ncols < 0 || nnz < 0)
            return set_error(MSPV_EINVAL, "spmv_coo_noalloc: negative size");
        if (nnz > kNoAllocMaxEntries)
            return set_error(MSPV_ETOOBIG, "spmv_coo_noalloc: %lld entries exceed the fixed scratch limit of %lld",
                             (long long)nnz, (long long)kNoAllocMaxEntries);
        if (nnz > 0 && (!rows || !cols || !vals || nrows == 0 || ncols == 0))
            return set_error(MSPV_EINVAL, "spmv_coo_noalloc: NULL triplet array or entries in an empty shape");
        if ((!x && ncols > 0) || (!y && nrows > 0)) return set_error(MSPV_EINVAL, "spmv_coo_noalloc: NULL vector");
        if (nrows == 0) return MSPV_OK;
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        NoAllocScratch* S = nullptr;
        MSPV_TRY(noalloc_scratch(&S));
        if (nnz > 0) {
            // the flags keep the previous call's contents: clear them first
            MSPV_CUDA_TRY(cudaMemsetAsync(S->flags, 0, sizeof(S->flags), s));
            int64_t grid = (nnz + kThreads - 1) / kThreads;
            if (grid > (int64_t)num_sms() * 8) grid = (int64_t)num_sms() * 8;
            noalloc_check_kernel<<<(unsigned)grid, kThreads, 0, s>>>(rows, cols, nnz, nrows, ncols, S->flags);
            MSPV_CUDA_TRY(cudaGetLastError());
            int32_t hflags[4] = {0, 0, 0, 0};
            MSPV_CUDA_TRY(cudaMemcpyAsync(hflags, S->flags, sizeof(hflags), cudaMemcpyDeviceToHost, s));
            MSPV_CUDA_TRY(cudaStreamSynchronize(s));
            if (hflags[0])
                return set_error(MSPV_EINVAL, "spmv_coo_noalloc: an entry lies outside [0,%d) x [0,%d)", nrows, ncols);
            if (hflags[1]) return set_error(MSPV_EINVAL, "spmv_coo_noalloc: row indices must be non-decreasing");
        }
        MSPV_TRY(launch_coo_raw(nrows, nnz, rows, cols, vals, x, y, S->carry, s));
        clear_error();
        return MSPV_OK;
    } catch (...) {
        return set_error(MSPV_ECUDA, "spmv_coo_noalloc: internal error");
    }
}
