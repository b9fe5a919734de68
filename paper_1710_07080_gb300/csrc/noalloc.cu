// noalloc.cu -- isira_apply_operator_noalloc: the trimmed, shifted, deflated operator without
// any device allocation.
//
// Who needs it: callers that must not allocate device memory themselves or let a library do
// it -- a host program whose device memory is entirely pre-reserved by its own pool allocator
// with a fixed budget, a latency-critical loop in which cudaMalloc/cudaFree (which may
// synchronise the device) are not acceptable, or a plug-in whose host application forbids
// allocations behind its back.  isira_create allocates its workspace, so those callers get this
// one handle-free entry point instead.  They still pass every input and output buffer.
//
// Scratch: the cross-CTA partial sums of 1^T x and Vh^T x live in the file-scope array
// g_isira_noalloc_scratch below (about 72 KB).  Every GPU that loads this library holds that
// array until the process exits.  Every call shares it, and it keeps the previous call's
// contents: the arrival counter is cleared at the start of each call (an in-stream memset,
// which allocates nothing) and every partial is written before it is read.  Calls whose work
// overlaps on the GPU (two streams, two host threads) race on the array and give wrong
// results; serialise them.
//
// Device address: in host code the name g_isira_noalloc_scratch is only a host-side stand-in,
// not a device address.  The first call on each device (with that device current) looks the
// address up with cudaGetSymbolAddress and caches it; make that first call before any stream
// capture begins on that device.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/isira.h"
#include "common.cuh"

namespace {

constexpr int kNaBlocks = 1024;                 // maximum CTAs of the reduction launch
constexpr int kNaCMax = 8;                      // maximum deflation rank c
constexpr int kNaSlots = 1 + kNaCMax;           // 1^T x and Vh^T x
constexpr int kNaPartial = kNaSlots * kNaBlocks;
constexpr int kNaCoef = kNaPartial;             // kNaSlots final sums
constexpr int kNaCounter = kNaPartial + 16;     // one double slot reused as the arrival counter
constexpr int kNaDoubles = kNaPartial + 32;
constexpr int kNaMaxDevices = 64;

}  // namespace

static __device__ __align__(256) double g_isira_noalloc_scratch[kNaDoubles];

namespace {

using namespace isira;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_na_reduce(const T* __restrict__ x, const double* __restrict__ V,
                                                        int64_t n, int64_t trim, int c, double* scratch) {
    T* partial = reinterpret_cast<T*>(scratch);
    T* coef = reinterpret_cast<T*>(scratch + kNaCoef);
    unsigned* counter = reinterpret_cast<unsigned*>(scratch + kNaCounter);
    __shared__ T red[kNaSlots];
    T acc[kNaSlots];
#pragma unroll
    for (int t = 0; t < kNaSlots; ++t) acc[t] = T(0);
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        if (r == trim) continue;
        const T xr = x[r];
        acc[0] += xr;
#pragma unroll
        for (int t = 0; t < kNaCMax; ++t)
            if (t < c) acc[1 + t] += (T)V[(int64_t)t * n + r] * xr;
    }
    if (block_partials_arrive<T, kNaSlots>(acc, 1 + c, partial, kNaBlocks, counter)) {
        last_block_sum(partial, kNaBlocks, gridDim.x, 1 + c, red, counter);
        for (int t = threadIdx.x; t < 1 + c; t += blockDim.x) coef[t] = red[t];
    }
}

// y_r = (deg_r - sigma) x_r - sum_{c in N(r), c != trim} x_c + sig_n 1^T x + delta sum_t V_rt (V^T x)_t,
// y_trim = 0.  Four lanes per row.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_na_apply(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                       int64_t n, int64_t trim, T sigma, T sig_n, T delta,
                                                       const T* __restrict__ x, const double* __restrict__ V, int c,
                                                       const double* scratch, T* __restrict__ y) {
    constexpr int G = 4;
    const T* coef = reinterpret_cast<const T*>(scratch + kNaCoef);
    const int lane = threadIdx.x & 31;
    const int64_t group = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / G;
    const int64_t iters = (n + ngroups - 1) / ngroups;   // uniform trip count keeps the warp converged
    for (int64_t it = 0; it < iters; ++it) {
        const int64_t r = group + it * ngroups;
        T s = 0;
        int64_t beg = 0, end = 0;
        if (r < n) {
            beg = rp[r];
            end = rp[r + 1];
            for (int64_t e = beg + (lane % G); e < end; e += G) {
                const int32_t col = ci[e];
                if (col != trim) s += x[col];
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
        if (r < n && (lane % G) == 0) {
            if (r == trim) {
                y[r] = T(0);
            } else {
                const T degT = (T)(end - beg);
                T v = (degT - sigma) * x[r] - s + sig_n * coef[0];
                for (int t = 0; t < c; ++t) v += delta * (T)V[(int64_t)t * n + r] * coef[1 + t];
                y[r] = v;
            }
        }
    }
}

std::mutex g_na_mutex;
double* g_na_addr[kNaMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t na_scratch(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_isira_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_na_addr[dev] = static_cast<double*>(p);
    }
    *out = g_na_addr[dev];
    return cudaSuccess;
}

template <typename T>
isira_status na_run(int64_t n, const int64_t* rp, const int32_t* ci, int64_t trim, double sigma, double delta,
                    int drop_rank1, int c, const double* V, const void* xv, void* yv, cudaStream_t s) {
    double* scratch = nullptr;
    if (na_scratch(&scratch) != cudaSuccess) return ISIRA_ERR_CUDA;
    const T* x = static_cast<const T*>(xv);
    T* y = static_cast<T*>(yv);
    if (cudaMemsetAsync(scratch + kNaCounter, 0, sizeof(double), s) != cudaSuccess) return ISIRA_ERR_CUDA;
    const int64_t want = (n + kThreads - 1) / kThreads;
    const int grid = (int)(want < kNaBlocks ? (want > 0 ? want : 1) : kNaBlocks);
    k_na_reduce<T><<<grid, kThreads, 0, s>>>(x, V, n, trim, c, scratch);
    const T sig_n = drop_rank1 ? T(0) : (T)(sigma / (double)n);
    const int64_t want2 = (n * 4 + kThreads - 1) / kThreads;
    const int grid2 = (int)(want2 < 4096 ? (want2 > 0 ? want2 : 1) : 4096);
    k_na_apply<T><<<grid2, kThreads, 0, s>>>(rp, ci, n, trim, (T)sigma, sig_n, (T)delta, x, V, c, scratch, y);
    if (cudaGetLastError() != cudaSuccess) return ISIRA_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return ISIRA_ERR_CUDA;
    return ISIRA_OK;
}

}  // namespace

extern "C" isira_status isira_apply_operator_noalloc(int64_t n, int64_t nnz, const int64_t* d_row_ptr,
                                                     const int32_t* d_col_idx, int64_t trim, int precision,
                                                     double sigma, double delta, int drop_rank1, int c,
                                                     const double* d_V, const void* d_x, void* d_y, void* stream) {
    if (n < 3 || nnz < 0 || !d_row_ptr || !d_col_idx || !d_x || !d_y || trim < 0 || trim >= n || c < 0 ||
        (c > 0 && !d_V) || (precision != ISIRA_FP64 && precision != ISIRA_MIXED) || !(delta >= 0.0))
        return ISIRA_ERR_INVALID_ARG;
    if (c > kNaCMax) return ISIRA_ERR_LIMIT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == ISIRA_FP64)
        return na_run<double>(n, d_row_ptr, d_col_idx, trim, sigma, delta, drop_rank1, c, d_V, d_x, d_y, s);
    return na_run<float>(n, d_row_ptr, d_col_idx, trim, sigma, delta, drop_rank1, c, d_V, d_x, d_y, s);
}
