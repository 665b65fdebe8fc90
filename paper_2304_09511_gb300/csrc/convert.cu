// Format converters (Sec. II-B): canonical COO (stable LSD radix sort on (row, col)
// + in-order coalescing of duplicates), CSR row pointers by exclusive scan of the
// row histogram, DIA offset discovery, padding and scatter. Integer work only, so
// every structure is bit-identical run to run. No kernel here waits on another CTA.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace mspv {

// ---------------------------------------------------------------------------
// exclusive scan of int32 (tile of 2048 = 256 threads x 8, then a scan of the
// tile totals, then an add; recursive on the number of tiles)
// ---------------------------------------------------------------------------
constexpr int kScanItems = 8;
constexpr int kScanTile = kThreads * kScanItems;

__device__ __forceinline__ int32_t warp_incl_scan_i32(int32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan of one tile per CTA; tile_sums[blockIdx.x] = tile total.
__global__ void __launch_bounds__(kThreads) scan_tiles_kernel(const int32_t* __restrict__ in,
                                                              int32_t* __restrict__ out, int64_t m,
                                                              int32_t* __restrict__ tile_sums) {
    __shared__ int32_t s[kScanTile + kScanTile / 32];   // padded against bank conflicts
    __shared__ int32_t s_warp[kThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    const int tid = threadIdx.x;
    auto pad = [](int i) { return i + (i >> 5); };
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int i = k * kThreads + tid;
        int64_t e = base + i;
        s[pad(i)] = (e < m) ? in[e] : 0;
    }
    __syncthreads();
    int32_t v[kScanItems];
    int32_t run = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = s[pad(tid * kScanItems + k)];
        run += v[k];
    }
    int32_t incl = warp_incl_scan_i32(run);
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int32_t w = (lane < kThreads / 32) ? s_warp[lane] : 0;
        int32_t wi = warp_incl_scan_i32(w);
        if (lane < kThreads / 32) s_warp[lane] = wi - w;   // exclusive warp offsets
    }
    __syncthreads();
    int32_t excl = incl - run + s_warp[warp];
    if (tid == kThreads - 1) tile_sums[blockIdx.x] = excl + run;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        s[pad(tid * kScanItems + k)] = excl;
        excl += v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int i = k * kThreads + tid;
        int64_t e = base + i;
        if (e < m) out[e] = s[pad(i)];
    }
}

__global__ void scan_add_kernel(int32_t* __restrict__ out, int64_t m,
                                const int32_t* __restrict__ tile_offsets) {
    const int64_t e = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
    const int32_t add = tile_offsets[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = e + (int64_t)k * kThreads;
        if (i < m) out[i] += add;
    }
}

mspv_status exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t m, int32_t* d_total,
                               cudaStream_t s) {
    if (m <= 0) {
        if (d_total) MSPV_CUDA_TRY(cudaMemsetAsync(d_total, 0, sizeof(int32_t), s));
        return MSPV_OK;
    }
    const int64_t ntiles = (m + kScanTile - 1) / kScanTile;
    if (ntiles == 1) {
        DevBuf tmp;
        int32_t* tot = d_total;
        if (!tot) {
            MSPV_TRY(tmp.alloc(sizeof(int32_t)));
            tot = tmp.as<int32_t>();
        }
        scan_tiles_kernel<<<1, kThreads, 0, s>>>(in, out, m, tot);
        MSPV_CUDA_TRY(cudaGetLastError());
        if (tmp.ptr) MSPV_CUDA_TRY(cudaStreamSynchronize(s));
        return MSPV_OK;
    }
    DevBuf sums, offs;
    MSPV_TRY(sums.alloc(sizeof(int32_t) * ntiles));
    MSPV_TRY(offs.alloc(sizeof(int32_t) * ntiles));
    scan_tiles_kernel<<<(unsigned)ntiles, kThreads, 0, s>>>(in, out, m, sums.as<int32_t>());
    MSPV_CUDA_TRY(cudaGetLastError());
    MSPV_TRY(exclusive_scan_i32(sums.as<int32_t>(), offs.as<int32_t>(), ntiles, d_total, s));
    scan_add_kernel<<<(unsigned)ntiles, kThreads, 0, s>>>(out, m, offs.as<int32_t>());
    MSPV_CUDA_TRY(cudaGetLastError());
    MSPV_CUDA_TRY(cudaStreamSynchronize(s));   // temporaries are freed on return
    return MSPV_OK;
}

// ---------------------------------------------------------------------------
// keys, validation, sortedness
// ---------------------------------------------------------------------------
static int bits_for(int64_t v) {   // bits needed to hold 0..v (v >= 0), at least 1
    int b = 1;
    while ((v >> b) != 0) ++b;
    return b;
}

// key = row << colbits | col; flags[0] |= index out of range, flags[1] |= keys not
// non-decreasing in input order.
__global__ void make_keys_kernel(const int32_t* __restrict__ rows, const int32_t* __restrict__ cols,
                                 int64_t m, int32_t nrows, int32_t ncols, int colbits,
                                 uint64_t* __restrict__ keys, int32_t* __restrict__ idx,
                                 int32_t* __restrict__ flags) {
    int bad = 0, unsorted = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        int32_t r = rows[e], c = cols[e];
        bool ok = (r >= 0) & (r < nrows) & (c >= 0) & (c < ncols);
        bad |= !ok;
        uint64_t k = ok ? (((uint64_t)(uint32_t)r << colbits) | (uint32_t)c) : 0ull;
        keys[e] = k;
        idx[e] = (int32_t)e;
        if (e > 0) {
            int32_t rp = rows[e - 1], cp = cols[e - 1];
            unsorted |= (rp > r) | ((rp == r) & (cp > c));
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&flags[0], 1);
    if (__any_sync(0xffffffffu, unsorted) && (threadIdx.x & 31) == 0) atomicOr(&flags[1], 1);
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (key, idx), 8-bit digits
// ---------------------------------------------------------------------------
constexpr int kRadixChunks = 16;                          // 256-element chunks per tile
constexpr int kRadixTile = kThreads * kRadixChunks;       // 4096 elements per CTA

__global__ void __launch_bounds__(kThreads) radix_hist_kernel(const uint64_t* __restrict__ keys,
                                                              int64_t m, int shift,
                                                              int32_t* __restrict__ counts,
                                                              int nblocks) {
    __shared__ int32_t h[256];
    const int tid = threadIdx.x, lane = tid & 31;
    h[tid] = 0;
    __syncthreads();
    const int64_t tile0 = (int64_t)blockIdx.x * kRadixTile;
    for (int c = 0; c < kRadixChunks; ++c) {
        int64_t e = tile0 + (int64_t)c * kThreads + tid;
        int d = (e < m) ? (int)((keys[e] >> shift) & 255u) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        if (d < 256 && lane == __ffs(peers) - 1) atomicAdd(&h[d], __popc(peers));
    }
    __syncthreads();
    counts[(int64_t)tid * nblocks + blockIdx.x] = h[tid];
}

// offsets = exclusive scan of counts laid out digit-major: the first output slot of
// digit d for this CTA. Elements of one digit keep their input order (stable).
__global__ void __launch_bounds__(kThreads) radix_scatter_kernel(
    const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin, uint64_t* __restrict__ kout,
    int32_t* __restrict__ vout, int64_t m, int shift, const int32_t* __restrict__ offsets,
    int nblocks) {
    __shared__ int32_t s_base[256];
    __shared__ int32_t s_wc[kThreads / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    s_base[tid] = offsets[(int64_t)tid * nblocks + blockIdx.x];
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) s_wc[w][tid] = 0;
    __syncthreads();
    const int64_t tile0 = (int64_t)blockIdx.x * kRadixTile;
    for (int c = 0; c < kRadixChunks; ++c) {
        const int64_t cbase = tile0 + (int64_t)c * kThreads;
        if (cbase >= m) break;   // uniform across the CTA
        int64_t e = cbase + tid;
        bool valid = e < m;
        uint64_t k = valid ? kin[e] : 0ull;
        int32_t v = valid ? vin[e] : 0;
        int d = valid ? (int)((k >> shift) & 255u) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && lane == __ffs(peers) - 1) s_wc[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int32_t pos = s_base[d] + rank;
            for (int w = 0; w < warp; ++w) pos += s_wc[w][d];
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        int32_t tot = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) {
            tot += s_wc[w][tid];
            s_wc[w][tid] = 0;
        }
        s_base[tid] += tot;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// coalescing: heads[e] = 1 where key[e] differs from key[e-1]; after an exclusive
// scan pos[e] is the output slot of the run starting at e. Each run is summed left to
// right in input order (the sort was stable), matching sequential accumulation.
// ---------------------------------------------------------------------------
__global__ void heads_kernel(const uint64_t* __restrict__ keys, int64_t m, int32_t* __restrict__ heads) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        heads[e] = (e == 0 || keys[e] != keys[e - 1]) ? 1 : 0;
}

__global__ void coalesce_kernel(const uint64_t* __restrict__ keys, const int32_t* __restrict__ idx,
                                const int32_t* __restrict__ pos, int64_t m,
                                const double* __restrict__ vals, int colbits,
                                int32_t* __restrict__ ai, int32_t* __restrict__ aj,
                                double* __restrict__ av) {
    const uint64_t cmask = (colbits >= 64) ? ~0ull : ((1ull << colbits) - 1ull);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[e];
        if (e > 0 && keys[e - 1] == k) continue;   // not a run head
        double sum = vals[idx[e]];
        for (int64_t f = e + 1; f < m && keys[f] == k; ++f) sum = sum + vals[idx[f]];
        const int32_t p = pos[e];
        ai[p] = (int32_t)(k >> colbits);
        aj[p] = (int32_t)(k & cmask);
        av[p] = sum;
    }
}

static unsigned grid_for(int64_t m, int per_thread = 1) {
    int64_t b = (m + (int64_t)kThreads * per_thread - 1) / ((int64_t)kThreads * per_thread);
    if (b < 1) b = 1;
    if (b > (int64_t)num_sms() * 64) b = (int64_t)num_sms() * 64;   // grid-stride beyond this
    return (unsigned)b;
}

mspv_status build_coo(int32_t nrows, int32_t ncols, int64_t nnz, const int32_t* rows,
                      const int32_t* cols, const double* vals, cudaStream_t s,
                      mspv_matrix* M) {
    M->format = MSPV_COO;
    M->value_type = MSPV_F64;
    M->nrows = nrows;
    M->ncols = ncols;
    if (nnz == 0) {
        M->nnz = 0;
        MSPV_TRY(dev_alloc_n(&M->ai, 1));
        MSPV_TRY(dev_alloc_n(&M->aj, 1));
        MSPV_TRY(dev_alloc(&M->av, 8));
        M->bytes += 16;
        return MSPV_OK;
    }
    const int colbits = bits_for(ncols > 0 ? ncols - 1 : 0);
    const int rowbits = bits_for(nrows > 0 ? nrows - 1 : 0);
    const int totbits = colbits + rowbits;

    DevBuf keys, idx, flags;
    MSPV_TRY(keys.alloc(sizeof(uint64_t) * nnz));
    MSPV_TRY(idx.alloc(sizeof(int32_t) * nnz));
    MSPV_TRY(flags.alloc(sizeof(int32_t) * 2));
    MSPV_CUDA_TRY(cudaMemsetAsync(flags.ptr, 0, sizeof(int32_t) * 2, s));
    make_keys_kernel<<<grid_for(nnz), kThreads, 0, s>>>(rows, cols, nnz, nrows, ncols, colbits,
                                                        keys.as<uint64_t>(), idx.as<int32_t>(),
                                                        flags.as<int32_t>());
    MSPV_CUDA_TRY(cudaGetLastError());
    int32_t hflags[2] = {0, 0};
    MSPV_CUDA_TRY(cudaMemcpyAsync(hflags, flags.ptr, sizeof(hflags), cudaMemcpyDeviceToHost, s));
    MSPV_CUDA_TRY(cudaStreamSynchronize(s));
    if (hflags[0]) return set_error(MSPV_EINVAL, "create_coo: an index lies outside [0,%d) x [0,%d)", nrows, ncols);

    uint64_t* kcur = keys.as<uint64_t>();
    int32_t* vcur = idx.as<int32_t>();
    DevBuf keys2, idx2, counts;
    if (hflags[1]) {   // not already in (row, col) order: sort
        MSPV_TRY(keys2.alloc(sizeof(uint64_t) * nnz));
        MSPV_TRY(idx2.alloc(sizeof(int32_t) * nnz));
        const int64_t nblocks = (nnz + kRadixTile - 1) / kRadixTile;
        MSPV_TRY(counts.alloc(sizeof(int32_t) * 256 * nblocks));
        uint64_t* kalt = keys2.as<uint64_t>();
        int32_t* valt = idx2.as<int32_t>();
        for (int shift = 0; shift < totbits; shift += 8) {
            radix_hist_kernel<<<(unsigned)nblocks, kThreads, 0, s>>>(kcur, nnz, shift,
                                                                     counts.as<int32_t>(), (int)nblocks);
            MSPV_CUDA_TRY(cudaGetLastError());
            MSPV_TRY(exclusive_scan_i32(counts.as<int32_t>(), counts.as<int32_t>(), 256 * nblocks,
                                        nullptr, s));
            radix_scatter_kernel<<<(unsigned)nblocks, kThreads, 0, s>>>(
                kcur, vcur, kalt, valt, nnz, shift, counts.as<int32_t>(), (int)nblocks);
            MSPV_CUDA_TRY(cudaGetLastError());
            uint64_t* tk = kcur; kcur = kalt; kalt = tk;
            int32_t* tv = vcur; vcur = valt; valt = tv;
        }
    }
    // coalesce duplicates
    DevBuf heads, total;
    MSPV_TRY(heads.alloc(sizeof(int32_t) * nnz));
    MSPV_TRY(total.alloc(sizeof(int32_t)));
    heads_kernel<<<grid_for(nnz), kThreads, 0, s>>>(kcur, nnz, heads.as<int32_t>());
    MSPV_CUDA_TRY(cudaGetLastError());
    MSPV_TRY(exclusive_scan_i32(heads.as<int32_t>(), heads.as<int32_t>(), nnz, total.as<int32_t>(), s));
    int32_t nout = 0;
    MSPV_CUDA_TRY(cudaMemcpyAsync(&nout, total.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    MSPV_CUDA_TRY(cudaStreamSynchronize(s));
    M->nnz = nout;
    MSPV_TRY(dev_alloc_n(&M->ai, nout));
    MSPV_TRY(dev_alloc_n(&M->aj, nout));
    MSPV_TRY(dev_alloc(&M->av, sizeof(double) * (size_t)nout));
    M->av_count = nout;
    M->bytes += (int64_t)nout * 16;
    coalesce_kernel<<<grid_for(nnz), kThreads, 0, s>>>(kcur, vcur, heads.as<int32_t>(), nnz, vals,
                                                       colbits, M->ai, M->aj, (double*)M->av);
    MSPV_CUDA_TRY(cudaGetLastError());
    MSPV_CUDA_TRY(cudaStreamSynchronize(s));
    return MSPV_OK;
}

// ---------------------------------------------------------------------------
// value storage: round FP64 to the stored type (to nearest, ties to even)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double load_value(const void* av, int vt, int64_t e) {
    if (vt == MSPV_F64) return static_cast<const double*>(av)[e];
    if (vt == MSPV_F32) return (double)static_cast<const float*>(av)[e];
    const uint16_t b = static_cast<const uint16_t*>(av)[e];
    return (double)__uint_as_float((uint32_t)b << 16);
}

__device__ __forceinline__ void store_value(void* av, int vt, int64_t e, double v) {
    if (vt == MSPV_F64) {
        static_cast<double*>(av)[e] = v;
    } else if (vt == MSPV_F32) {
        static_cast<float*>(av)[e] = __double2float_rn(v);
    } else {
        uint16_t b;
        asm("cvt.rn.bf16.f64 %0, %1;" : "=h"(b) : "d"(v));
        static_cast<uint16_t*>(av)[e] = b;
    }
}

__global__ void convert_values_kernel(const void* __restrict__ src, int svt, int64_t m,
                                      void* __restrict__ dst, int dvt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        store_value(dst, dvt, e, load_value(src, svt, e));
}

// ---------------------------------------------------------------------------
// row histogram and statistics
// ---------------------------------------------------------------------------
__global__ void row_count_kernel(const int32_t* __restrict__ ai, int64_t nnz, int32_t* __restrict__ counts) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // the loop trip count is uniform per warp so that __match_any_sync sees all lanes
    const int64_t trips = (nnz + stride - 1) / stride;
    for (int64_t t = 0; t < trips; ++t) {
        int64_t e = first + t * stride;
        int r = (e < nnz) ? ai[e] : -1;
        unsigned peers = __match_any_sync(0xffffffffu, r);
        if (r >= 0 && lane == __ffs(peers) - 1) atomicAdd(&counts[r], __popc(peers));
    }
}

struct RowStats {
    unsigned long long sum_sq;
    unsigned long long empty;
    int32_t max;
    int32_t min;
};

__global__ void row_stats_kernel(const int32_t* __restrict__ counts, int32_t n, RowStats* st) {
    unsigned long long sq = 0, empty = 0;
    int32_t mx = 0, mn = INT32_MAX;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = counts[i];
        sq += (unsigned long long)c * (unsigned long long)c;
        empty += (c == 0);
        mx = max(mx, c);
        mn = min(mn, c);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sq += __shfl_xor_sync(0xffffffffu, sq, o);
        empty += __shfl_xor_sync(0xffffffffu, empty, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&st->sum_sq, sq);
        atomicAdd(&st->empty, empty);
        atomicMax(&st->max, mx);
        atomicMin(&st->min, mn);
    }
}

static mspv_status compute_row_stats(const int32_t* ai, int64_t nnz, int32_t nrows, cudaStream_t s,
                                     mspv_matrix* M, DevBuf* counts_out) {
    DevBuf counts_local, stats;
    DevBuf& counts = counts_out ? *counts_out : counts_local;
    MSPV_TRY(counts.alloc(sizeof(int32_t) * ((size_t)nrows + 1)));
    MSPV_TRY(stats.alloc(sizeof(RowStats)));
    MSPV_CUDA_TRY(cudaMemsetAsync(counts.ptr, 0, sizeof(int32_t) * ((size_t)nrows + 1), s));
    MSPV_CUDA_TRY(cudaMemsetAsync(stats.ptr, 0, sizeof(RowStats), s));
    const int32_t big = INT32_MAX;
    MSPV_CUDA_TRY(cudaMemcpyAsync(&stats.as<RowStats>()->min, &big, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    if (nnz > 0) {
        row_count_kernel<<<grid_for(nnz), kThreads, 0, s>>>(ai, nnz, counts.as<int32_t>());
        MSPV_CUDA_TRY(cudaGetLastError());
    }
    if (nrows > 0) {
        row_stats_kernel<<<grid_for(nrows), kThreads, 0, s>>>(counts.as<int32_t>(), nrows,
                                                              stats.as<RowStats>());
        MSPV_CUDA_TRY(cudaGetLastError());
    }
    RowStats h{};
    MSPV_CUDA_TRY(cudaMemcpyAsync(&h, stats.ptr, sizeof(h), cudaMemcpyDeviceToHost, s));
    MSPV_CUDA_TRY(cudaStreamSynchronize(s));
    const double n = nrows > 0 ? (double)nrows : 1.0;
    M->row_mean = (double)nnz / n;
    double var = (double)h.sum_sq / n - M->row_mean * M->row_mean;
    M->row_std = std::sqrt(var > 0.0 ? var : 0.0);
    M->row_max = h.max;
    M->row_min = nrows > 0 ? h.min : 0;
    M->empty_rows = (int64_t)h.empty;
    return MSPV_OK;
}

mspv_status finish_coo_stats(mspv_matrix* M, cudaStream_t s) {
    return compute_row_stats(M->ai, M->nnz, M->nrows, s, M, nullptr);
}

// CSR rows -> COO rows: ai[j] = i for j in [irp[i], irp[i+1])
__global__ void expand_rows_kernel(const int32_t* __restrict__ irp, int32_t n, int32_t* __restrict__ ai) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        for (int32_t j = irp[i]; j < irp[i + 1]; ++j) ai[j] = (int32_t)i;
}

// ---------------------------------------------------------------------------
// DIA: offset flags over the 2n-1 possible diagonals, their scan gives the column
// of each diagonal in AV; then the scatter into the zeroed, padded array.
// ---------------------------------------------------------------------------
__global__ void dia_flag_kernel(const int32_t* __restrict__ ai, const int32_t* __restrict__ aj,
                                int64_t nnz, int32_t n, int32_t* __restrict__ flags) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x)
        flags[(int64_t)aj[e] - ai[e] + (n - 1)] = 1;
}

__global__ void dia_offsets_kernel(const int32_t* __restrict__ flags, const int32_t* __restrict__ map,
                                   int64_t span, int32_t n, int32_t* __restrict__ doff) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < span;
         k += (int64_t)gridDim.x * blockDim.x)
        if (flags[k]) doff[map[k]] = (int32_t)(k - (n - 1));
}

__global__ void zero_bytes_kernel(uint4* __restrict__ p, int64_t n16) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n16;
         e += (int64_t)gridDim.x * blockDim.x)
        p[e] = make_uint4(0, 0, 0, 0);
}

__global__ void dia_scatter_kernel(const int32_t* __restrict__ ai, const int32_t* __restrict__ aj,
                                   const void* __restrict__ av, int svt, int64_t nnz, int32_t n,
                                   int32_t npad, const int32_t* __restrict__ map,
                                   void* __restrict__ dav, int dvt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = ai[e];
        const int64_t j = map[(int64_t)aj[e] - i + (n - 1)];
        store_value(dav, dvt, j * npad + i, load_value(av, svt, e));
    }
}

static double dia_fill_cap() {
    const char* s = std::getenv("MSPV_DIA_MAX_FILL");
    double f = s ? std::atof(s) : 32.0;
    return f > 0.0 ? f : 32.0;
}

double dia_slot_cap(int64_t nnz) { return std::fmax(dia_fill_cap() * (double)nnz, (double)(1 << 20)); }

mspv_status build_from(const mspv_matrix* A, int32_t format, int32_t vt, cudaStream_t s,
                       mspv_matrix* M) {
    if (A->format == MSPV_DIA)
        return set_error(MSPV_EFORMAT, "convert: a DIA handle cannot be converted (build from COO or CSR)");
    M->format = format;
    M->value_type = vt;
    M->nrows = A->nrows;
    M->ncols = A->ncols;
    M->nnz = A->nnz;
    M->row_mean = A->row_mean;
    M->row_std = A->row_std;
    M->row_max = A->row_max;
    M->row_min = A->row_min;
    M->empty_rows = A->empty_rows;
    const int64_t nnz = A->nnz;
    const size_t vs = value_size(vt);

    // a COO view of the source
    DevBuf rows_tmp;
    const int32_t* src_ai = A->ai;
    if (A->format == MSPV_CSR) {
        MSPV_TRY(rows_tmp.alloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1)));
        if (A->nrows > 0) {
            expand_rows_kernel<<<grid_for(A->nrows), kThreads, 0, s>>>(A->irp, A->nrows, rows_tmp.as<int32_t>());
            MSPV_CUDA_TRY(cudaGetLastError());
        }
        src_ai = rows_tmp.as<int32_t>();
    }

    if (format == MSPV_COO || format == MSPV_CSR) {
        MSPV_TRY(dev_alloc_n(&M->aj, nnz));
        MSPV_TRY(dev_alloc(&M->av, vs * (size_t)(nnz > 0 ? nnz : 1)));
        M->av_count = nnz;
        M->bytes += nnz * (4 + (int64_t)vs);
        if (nnz > 0) {
            MSPV_CUDA_TRY(cudaMemcpyAsync(M->aj, A->aj, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, s));
            convert_values_kernel<<<grid_for(nnz), kThreads, 0, s>>>(A->av, A->value_type, nnz, M->av, vt);
            MSPV_CUDA_TRY(cudaGetLastError());
        }
        if (format == MSPV_COO) {
            MSPV_TRY(dev_alloc_n(&M->ai, nnz));
            M->bytes += nnz * 4;
            if (nnz > 0)
                MSPV_CUDA_TRY(cudaMemcpyAsync(M->ai, src_ai, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, s));
            MSPV_TRY(ensure_coo_carry(M, s));
        } else {
            // irp = exclusive scan of the row histogram; irp[nrows] = nnz
            MSPV_TRY(dev_alloc_n(&M->irp, (int64_t)M->nrows + 1));
            M->bytes += ((int64_t)M->nrows + 1) * 4;
            MSPV_CUDA_TRY(cudaMemsetAsync(M->irp, 0, sizeof(int32_t) * ((size_t)M->nrows + 1), s));
            if (nnz > 0) {
                row_count_kernel<<<grid_for(nnz), kThreads, 0, s>>>(src_ai, nnz, M->irp);
                MSPV_CUDA_TRY(cudaGetLastError());
            }
            MSPV_TRY(exclusive_scan_i32(M->irp, M->irp, M->nrows, M->irp + M->nrows, s));
            M->csr_vector = choose_csr_vector(M->row_mean, M->row_std, M->row_max);
            M->csr_block = choose_csr_block_kernel();
            if (M->csr_vector > 0) MSPV_TRY(build_csr_long_rows(M, s));
            MSPV_TRY(build_csr_row_blocks(M, s));
        }
        MSPV_CUDA_TRY(cudaStreamSynchronize(s));
        return MSPV_OK;
    }

    // DIA
    if (A->nrows != A->ncols)
        return set_error(MSPV_EFORMAT, "convert: DIA needs a square matrix (got %d x %d)", A->nrows, A->ncols);
    const int32_t n = A->nrows;
    const int64_t npad64 = ((int64_t)n + 31) / 32 * 32;   // checked before any workspace is allocated
    if (npad64 > INT32_MAX)
        return set_error(MSPV_ETOOBIG, "convert: %d rows padded to a multiple of 32 exceed 2^31 - 1", n);
    const int32_t npad = (int32_t)npad64;
    const int64_t span = n > 0 ? 2 * (int64_t)n - 1 : 0;
    DevBuf flags, map, total;
    MSPV_TRY(flags.alloc(sizeof(int32_t) * (size_t)(span > 0 ? span : 1)));
    MSPV_TRY(map.alloc(sizeof(int32_t) * (size_t)(span > 0 ? span : 1)));
    MSPV_TRY(total.alloc(sizeof(int32_t)));
    if (span > 0) MSPV_CUDA_TRY(cudaMemsetAsync(flags.ptr, 0, sizeof(int32_t) * span, s));
    if (nnz > 0) {
        dia_flag_kernel<<<grid_for(nnz), kThreads, 0, s>>>(src_ai, A->aj, nnz, n, flags.as<int32_t>());
        MSPV_CUDA_TRY(cudaGetLastError());
    }
    MSPV_TRY(exclusive_scan_i32(flags.as<int32_t>(), map.as<int32_t>(), span, total.as<int32_t>(), s));
    int32_t nd = 0;
    MSPV_CUDA_TRY(cudaMemcpyAsync(&nd, total.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    MSPV_CUDA_TRY(cudaStreamSynchronize(s));
    const double slots = (double)nd * (double)npad;
    const double cap = dia_slot_cap(nnz);
    if (slots > cap)
        return set_error(MSPV_ETOOBIG, "convert: DIA would store %d diagonals x %d rows = %.0f slots for %lld entries (cap %.0f)",
                         nd, npad, slots, (long long)nnz, cap);
    M->ndiags = nd;
    M->npad = npad;
    const int64_t nslots = (int64_t)nd * npad;
    MSPV_TRY(dev_alloc_n(&M->doff, nd));
    const size_t avbytes = ((vs * (size_t)(nslots > 0 ? nslots : 1)) + 15) & ~(size_t)15;
    MSPV_TRY(dev_alloc(&M->av, avbytes));
    M->av_count = nslots;
    M->bytes += (int64_t)nd * 4 + (int64_t)avbytes;
    if (span > 0) {
        dia_offsets_kernel<<<grid_for(span), kThreads, 0, s>>>(flags.as<int32_t>(), map.as<int32_t>(), span, n, M->doff);
        MSPV_CUDA_TRY(cudaGetLastError());
    }
    // runs of consecutive offsets (at most 3 long): the FP32-arithmetic kernel reads one x
    // window per run instead of one per diagonal
    if (nd > 0) {
        std::vector<int32_t> off(nd);
        MSPV_CUDA_TRY(cudaMemcpyAsync(off.data(), M->doff, sizeof(int32_t) * nd, cudaMemcpyDeviceToHost, s));
        MSPV_CUDA_TRY(cudaStreamSynchronize(s));
        std::vector<int2> runs;
        for (int32_t j = 0; j < nd;) {
            int32_t len = 1;
            while (j + len < nd && len < 3 && off[j + len] == off[j] + len) ++len;
            runs.push_back(make_int2(j, len));
            j += len;
        }
        M->ndruns = (int32_t)runs.size();
        MSPV_TRY(dev_alloc(reinterpret_cast<void**>(&M->druns), sizeof(int2) * runs.size()));
        M->bytes += (int64_t)(sizeof(int2) * runs.size());
        MSPV_CUDA_TRY(cudaMemcpyAsync(M->druns, runs.data(), sizeof(int2) * runs.size(), cudaMemcpyHostToDevice, s));
    }
    zero_bytes_kernel<<<grid_for((int64_t)(avbytes / 16)), kThreads, 0, s>>>((uint4*)M->av, (int64_t)(avbytes / 16));
    MSPV_CUDA_TRY(cudaGetLastError());
    if (nnz > 0) {
        dia_scatter_kernel<<<grid_for(nnz), kThreads, 0, s>>>(src_ai, A->aj, A->av, A->value_type, nnz, n,
                                                              npad, map.as<int32_t>(), M->av, vt);
        MSPV_CUDA_TRY(cudaGetLastError());
    }
    MSPV_CUDA_TRY(cudaStreamSynchronize(s));
    return MSPV_OK;
}

// ---------------------------------------------------------------------------
// column split: local part (columns < c) and remote part (columns >= c, shifted by -c)
// ---------------------------------------------------------------------------
__global__ void split_flag_kernel(const int32_t* __restrict__ aj, int64_t nnz, int32_t c, int32_t* __restrict__ flag) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        flag[e] = aj[e] < c ? 1 : 0;
}

template <typename W>
__global__ void split_scatter_kernel(const int32_t* __restrict__ ai, const int32_t* __restrict__ aj,
                                     const W* __restrict__ av, const int32_t* __restrict__ pos, int64_t nnz,
                                     int32_t c, int32_t* __restrict__ li, int32_t* __restrict__ lj,
                                     W* __restrict__ lv, int32_t* __restrict__ ri, int32_t* __restrict__ rj,
                                     W* __restrict__ rv) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = aj[e];
        const int64_t p = pos[e];   // local entries before e
        if (j < c) {
            li[p] = ai[e];
            lj[p] = j;
            lv[p] = av[e];
        } else {
            const int64_t q = e - p;
            ri[q] = ai[e];
            rj[q] = j - c;
            rv[q] = av[e];
        }
    }
}

static mspv_status alloc_coo_part(mspv_matrix* M, int32_t nrows, int32_t ncols, int64_t nnz, int32_t vt) {
    M->format = MSPV_COO;
    M->value_type = vt;
    M->nrows = nrows;
    M->ncols = ncols;
    M->nnz = nnz;
    const size_t vs = value_size(vt);
    MSPV_TRY(dev_alloc_n(&M->ai, nnz > 0 ? nnz : 1));
    MSPV_TRY(dev_alloc_n(&M->aj, nnz > 0 ? nnz : 1));
    MSPV_TRY(dev_alloc(&M->av, vs * (size_t)(nnz > 0 ? nnz : 1)));
    M->av_count = nnz;
    M->bytes += nnz * (8 + (int64_t)vs);
    return MSPV_OK;
}

mspv_status split_columns(const mspv_matrix* A, int32_t c, cudaStream_t s, mspv_matrix* L, mspv_matrix* R) {
    if (A->format == MSPV_DIA)
        return set_error(MSPV_EFORMAT, "split: pass a COO or CSR handle");
    const int64_t nnz = A->nnz;
    DevBuf rows_tmp, flag, pos, total;
    const int32_t* src_ai = A->ai;
    if (A->format == MSPV_CSR) {
        MSPV_TRY(rows_tmp.alloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1)));
        if (A->nrows > 0)
            expand_rows_kernel<<<grid_for(A->nrows), kThreads, 0, s>>>(A->irp, A->nrows, rows_tmp.as<int32_t>());
        src_ai = rows_tmp.as<int32_t>();
    }
    MSPV_TRY(flag.alloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1)));
    MSPV_TRY(pos.alloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1)));
    MSPV_TRY(total.alloc(sizeof(int32_t)));
    MSPV_CUDA_TRY(cudaMemsetAsync(total.ptr, 0, sizeof(int32_t), s));
    if (nnz > 0) {
        split_flag_kernel<<<grid_for(nnz), kThreads, 0, s>>>(A->aj, nnz, c, flag.as<int32_t>());
        MSPV_CUDA_TRY(cudaGetLastError());
        MSPV_TRY(exclusive_scan_i32(flag.as<int32_t>(), pos.as<int32_t>(), nnz, total.as<int32_t>(), s));
    }
    int32_t nloc = 0;
    MSPV_CUDA_TRY(cudaMemcpyAsync(&nloc, total.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    MSPV_CUDA_TRY(cudaStreamSynchronize(s));
    MSPV_TRY(alloc_coo_part(L, A->nrows, c, nloc, A->value_type));
    MSPV_TRY(alloc_coo_part(R, A->nrows, A->ncols - c, nnz - nloc, A->value_type));
    if (nnz > 0) {
        const unsigned g = grid_for(nnz);
        const int32_t* pp = pos.as<int32_t>();
        switch (value_size(A->value_type)) {
            case 8:
                split_scatter_kernel<uint64_t><<<g, kThreads, 0, s>>>(
                    src_ai, A->aj, static_cast<const uint64_t*>(A->av), pp, nnz, c, L->ai, L->aj,
                    static_cast<uint64_t*>(L->av), R->ai, R->aj, static_cast<uint64_t*>(R->av));
                break;
            case 4:
                split_scatter_kernel<uint32_t><<<g, kThreads, 0, s>>>(
                    src_ai, A->aj, static_cast<const uint32_t*>(A->av), pp, nnz, c, L->ai, L->aj,
                    static_cast<uint32_t*>(L->av), R->ai, R->aj, static_cast<uint32_t*>(R->av));
                break;
            default:
                split_scatter_kernel<uint16_t><<<g, kThreads, 0, s>>>(
                    src_ai, A->aj, static_cast<const uint16_t*>(A->av), pp, nnz, c, L->ai, L->aj,
                    static_cast<uint16_t*>(L->av), R->ai, R->aj, static_cast<uint16_t*>(R->av));
        }
        MSPV_CUDA_TRY(cudaGetLastError());
    }
    MSPV_TRY(finish_coo_stats(L, s));
    MSPV_TRY(ensure_coo_carry(L, s));
    MSPV_TRY(finish_coo_stats(R, s));
    MSPV_TRY(ensure_coo_carry(R, s));
    MSPV_CUDA_TRY(cudaStreamSynchronize(s));
    return MSPV_OK;
}

// COO kernel for the row lengths: short rows (at most 128 entries) take the row-block kernel
// (a warp per 32 consecutive rows, 4 lanes per row, chunks that never cut a row) when rows
// average at least 4 entries, and the run-vector kernel (fixed 256-entry chunks) when they are
// sparser: the row-block kernel spends a warp on every 32 rows, empty or not (the remote part of
// a process's matrix, ~95 % empty rows, took 3x longer). Longer rows take the lane-sequential
// segment kernel, which keeps every lane busy however the rows are cut. MSPV_COO_KERNEL=
// rb|vec|seg overrides.
int32_t choose_coo_kernel(int32_t row_max, int64_t nnz, int32_t nrows) {
    const char* k = std::getenv("MSPV_COO_KERNEL");
    if (k && std::strcmp(k, "rb") == 0) return 2;
    if (k && std::strcmp(k, "vec") == 0) return 1;
    if (k && std::strcmp(k, "seg") == 0) return 0;
    if (row_max > 128) return 0;
    return nnz >= 4 * (int64_t)nrows ? 2 : 1;
}

// First entry of every block of kCooRbRows rows in row-sorted COO (blocks past the last
// entry start at nnz): the entry where the row index first reaches or passes a block's first
// row records it, so every block boundary is written once.
__global__ void coo_row_blocks_kernel(const int32_t* __restrict__ ai, int64_t nnz, int32_t* __restrict__ rb) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = ai[e];
        const int32_t rp = e > 0 ? ai[e - 1] : -1;
        if (r == rp) continue;
        for (int64_t k = ((int64_t)rp + kCooRbRows) / kCooRbRows; k <= r / kCooRbRows; ++k) rb[k] = (int32_t)e;
    }
}

__global__ void fill_i32_kernel(int32_t* __restrict__ v, int64_t n, int32_t value) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = value;
}

mspv_status ensure_coo_carry(mspv_matrix* M, cudaStream_t s) {
    if (M->format != MSPV_COO || M->carry) return MSPV_OK;
    M->coo_kernel = choose_coo_kernel(M->row_max, M->nnz, M->nrows);
    const char* ch = std::getenv("MSPV_COO_CHUNK");
    M->coo_chunk = (ch && std::atoi(ch) == 512) ? 512 : kCooVecChunk;
    M->nchunks = (M->nnz + kCooVecChunk - 1) / kCooVecChunk;
    MSPV_TRY(dev_alloc_n(&M->carry, M->nchunks > 0 ? M->nchunks : 1));
    M->bytes += (M->nchunks > 0 ? M->nchunks : 1) * (int64_t)sizeof(CooCarry);
    if (M->coo_kernel == 2 && M->nrows > 0) {
        M->coo_nrb = ((int64_t)M->nrows + kCooRbRows - 1) / kCooRbRows;
        MSPV_TRY(dev_alloc_n(&M->coo_rb, M->coo_nrb + 1));
        M->bytes += (M->coo_nrb + 1) * (int64_t)sizeof(int32_t);
        fill_i32_kernel<<<grid_for(M->coo_nrb + 1), kThreads, 0, s>>>(M->coo_rb, M->coo_nrb + 1, (int32_t)M->nnz);
        if (M->nnz > 0) coo_row_blocks_kernel<<<grid_for(M->nnz), kThreads, 0, s>>>(M->ai, M->nnz, M->coo_rb);
        MSPV_CUDA_TRY(cudaGetLastError());
    }
    return MSPV_OK;
}

mspv_status export_matrix(const mspv_matrix* A, int32_t* idx0, int32_t* idx1, double* vals,
                          cudaStream_t s) {
    const int64_t nnz = A->nnz;
    if (A->format == MSPV_COO) {
        if (idx0 && nnz) MSPV_CUDA_TRY(cudaMemcpyAsync(idx0, A->ai, 4 * nnz, cudaMemcpyDeviceToHost, s));
        if (idx1 && nnz) MSPV_CUDA_TRY(cudaMemcpyAsync(idx1, A->aj, 4 * nnz, cudaMemcpyDeviceToHost, s));
    } else if (A->format == MSPV_CSR) {
        if (idx0) MSPV_CUDA_TRY(cudaMemcpyAsync(idx0, A->irp, 4 * ((int64_t)A->nrows + 1), cudaMemcpyDeviceToHost, s));
        if (idx1 && nnz) MSPV_CUDA_TRY(cudaMemcpyAsync(idx1, A->aj, 4 * nnz, cudaMemcpyDeviceToHost, s));
    } else {
        if (idx0 && A->ndiags) MSPV_CUDA_TRY(cudaMemcpyAsync(idx0, A->doff, 4 * (int64_t)A->ndiags, cudaMemcpyDeviceToHost, s));
    }
    const int64_t nv = A->av_count;
    if (vals && nv > 0) {
        if (A->value_type == MSPV_F64) {
            MSPV_CUDA_TRY(cudaMemcpyAsync(vals, A->av, 8 * nv, cudaMemcpyDeviceToHost, s));
        } else {
            DevBuf wide;
            MSPV_TRY(wide.alloc(8 * (size_t)nv));
            convert_values_kernel<<<grid_for(nv), kThreads, 0, s>>>(A->av, A->value_type, nv, wide.ptr, MSPV_F64);
            MSPV_CUDA_TRY(cudaGetLastError());
            MSPV_CUDA_TRY(cudaMemcpyAsync(vals, wide.ptr, 8 * nv, cudaMemcpyDeviceToHost, s));
            MSPV_CUDA_TRY(cudaStreamSynchronize(s));
        }
    }
    MSPV_CUDA_TRY(cudaStreamSynchronize(s));
    return MSPV_OK;
}

void free_matrix(mspv_matrix* M) {
    auto f = [](void* p) { if (p) dev_free(p, 0); };
    f(M->ai); f(M->aj); f(M->irp); f(M->doff); f(M->druns); f(M->av); f(M->carry); f(M->row_block); f(M->long_rows);
    f(M->coo_rb);
    M->coo_rb = nullptr;
    M->coo_nrb = 0;
    f(M->cg.r); f(M->cg.p); f(M->cg.q); f(M->cg.partials); f(M->cg.st);
    f(M->cg.rf); f(M->cg.pf); f(M->cg.qf);
    if (M->cg.host_st) cudaFreeHost(M->cg.host_st);
    M->ai = M->aj = M->irp = M->doff = nullptr;
    M->druns = nullptr;
    M->ndruns = 0;
    M->av = nullptr;
    M->carry = nullptr;
    M->row_block = nullptr;
    M->long_rows = nullptr;
    M->cg = CgWork{};
}

}  // namespace mspv
