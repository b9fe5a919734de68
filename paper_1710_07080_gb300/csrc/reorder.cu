// reorder.cu -- optional relabelling of the vertices by descending degree (stable: equal degrees
// keep their original order).  On power-law graphs most stored entries point at the few
// high-degree vertices; numbering them first packs their vector entries into a small block that
// stays in L1/L2, so the gathers of the SpMV mostly hit cache.  The relabelled CSR is owned by
// the solver; vectors cross the API in the caller's numbering.
#include <cub/cub.cuh>

#include "internal.h"

namespace isira {

__global__ void k_reorder_keys(const int64_t* rp, int64_t n, int64_t maxdeg, uint32_t* keys, int32_t* vals) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        keys[v] = (uint32_t)(maxdeg - (rp[v + 1] - rp[v]));
        vals[v] = (int32_t)v;
    }
}

__global__ void k_new_degrees(const int64_t* rp, const int32_t* perm, int64_t n, int64_t* deg_new, int32_t* inv) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
        if (i == n) {
            deg_new[n] = 0;
        } else {
            const int64_t o = perm[i];
            deg_new[i] = rp[o + 1] - rp[o];
            inv[o] = (int32_t)i;
        }
    }
}

// one warp per new row: copy the old row's neighbours, renamed (and their weights, if any)
__global__ void __launch_bounds__(kThreads) k_permute_cols(const int64_t* rp, const int32_t* ci, const double* w,
                                                           const int32_t* perm, const int32_t* inv, const int64_t* rp2,
                                                           int64_t n, int32_t* ci2, double* w2) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < n; i += nw) {
        const int64_t o = perm[i];
        const int64_t b = rp[o], d = rp[o + 1] - b, b2 = rp2[i];
        for (int64_t j = lane; j < d; j += 32) {
            ci2[b2 + j] = inv[ci[b + j]];
            if (w) w2[b2 + j] = w[b + j];
        }
    }
}

template <typename T>
__global__ void k_gather_perm(const T* src, const int32_t* perm, int64_t n, T* dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[perm[i]];
}

template <typename T>
__global__ void k_scatter_perm(const T* src, const int32_t* perm, int64_t n, T* dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[perm[i]] = src[i];
}

cudaError_t build_reordered_graph(const int64_t* rp, const int32_t* ci, const double* w, int64_t n, int64_t nnz,
                                  int64_t maxdeg, int64_t* rp2, int32_t* ci2, double* w2, int32_t* perm, int32_t* inv,
                                  cudaStream_t s) {
    uint32_t *k0 = nullptr, *k1 = nullptr;
    int32_t* v0 = nullptr;
    int64_t* deg = nullptr;
    void* tmp = nullptr;
    size_t tmp_bytes = 0, scan_bytes = 0;
    cudaError_t e = cudaSuccess;
    const int grid = 1024;
#define CK(x) do { e = (x); if (e != cudaSuccess) goto done; } while (0)
    CK(cudaMalloc(&k0, sizeof(uint32_t) * n));
    CK(cudaMalloc(&k1, sizeof(uint32_t) * n));
    CK(cudaMalloc(&v0, sizeof(int32_t) * n));
    CK(cudaMalloc(&deg, sizeof(int64_t) * (n + 1)));
    k_reorder_keys<<<grid, kThreads, 0, s>>>(rp, n, maxdeg, k0, v0);
    CK(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, k0, k1, v0, perm, (int)n, 0, 32, s));
    CK(cub::DeviceScan::ExclusiveSum(nullptr, scan_bytes, deg, rp2, (int)(n + 1), s));
    if (scan_bytes > tmp_bytes) tmp_bytes = scan_bytes;
    CK(cudaMalloc(&tmp, tmp_bytes));
    CK(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, k0, k1, v0, perm, (int)n, 0, 32, s));
    k_new_degrees<<<grid, kThreads, 0, s>>>(rp, perm, n, deg, inv);
    CK(cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, deg, rp2, (int)(n + 1), s));
    k_permute_cols<<<grid, kThreads, 0, s>>>(rp, ci, w, perm, inv, rp2, n, ci2, w2);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
#undef CK
done:
    if (k0) cudaFree(k0);
    if (k1) cudaFree(k1);
    if (v0) cudaFree(v0);
    if (deg) cudaFree(deg);
    if (tmp) cudaFree(tmp);
    (void)nnz;
    return e;
}

// ------------------------------------------------------------------ sliced ELL copy of the light rows
// Rows [light0, n) in slices of 32 consecutive rows.  Slice s has width w_s = the largest degree
// among its rows; entry q of its lane l (row light0 + 32 s + l) sits at off[s] + 32 q + l, so a
// warp reads one 128-byte line per q.  Rows shorter than w_s are padded with -1.  With the
// degree-descending numbering the rows of a slice have nearly equal degrees (little padding).

__global__ void __launch_bounds__(kThreads) k_sell_widths(const int64_t* rp, int64_t n, int64_t light0,
                                                          int64_t n_slices, int64_t* w32) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s <= n_slices;
         s += (int64_t)gridDim.x * blockDim.x) {
        int64_t w = 0;
        if (s < n_slices)
            for (int64_t r = light0 + 32 * s; r < light0 + 32 * s + 32 && r < n; ++r) {
                const int64_t d = rp[r + 1] - rp[r];
                w = d > w ? d : w;
            }
        w32[s] = 32 * w;
    }
}

__global__ void __launch_bounds__(kThreads) k_sell_fill(const int64_t* rp, const int32_t* ci, const double* w,
                                                        int64_t n, int64_t light0, int64_t n_slices, const int64_t* off,
                                                        int32_t* sci, double* sw) {
    const int64_t total = n_slices * 32;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = t >> 5, lane = t & 31;
        const int64_t row = light0 + t;
        const int64_t wid = (off[s + 1] - off[s]) >> 5;
        const int64_t b = row < n ? rp[row] : 0;
        const int64_t d = row < n ? rp[row + 1] - b : 0;
        for (int64_t q = 0; q < wid; ++q) {
            sci[off[s] + 32 * q + lane] = q < d ? ci[b + q] : -1;
            if (w) sw[off[s] + 32 * q + lane] = q < d ? w[b + q] : 0.0;
        }
    }
}

cudaError_t build_sell(const int64_t* rp, const int32_t* ci, const double* w, int64_t n, int64_t light0,
                       int64_t n_slices, int64_t* off, int32_t** sci, double** sw, int64_t* total, cudaStream_t s) {
    *sci = nullptr;
    if (sw) *sw = nullptr;
    *total = 0;
    int64_t* w32 = nullptr;
    void* tmp = nullptr;
    size_t tmp_bytes = 0;
    cudaError_t e = cudaSuccess;
#define CK(x) do { e = (x); if (e != cudaSuccess) goto done; } while (0)
    CK(cudaMalloc(&w32, sizeof(int64_t) * (size_t)(n_slices + 1)));
    k_sell_widths<<<1024, kThreads, 0, s>>>(rp, n, light0, n_slices, w32);
    CK(cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, w32, off, (int)(n_slices + 1), s));
    CK(cudaMalloc(&tmp, tmp_bytes));
    CK(cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, w32, off, (int)(n_slices + 1), s));
    CK(cudaMemcpyAsync(total, off + n_slices, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaMalloc(sci, sizeof(int32_t) * (size_t)(*total > 0 ? *total : 1)));
    if (w) CK(cudaMalloc(sw, sizeof(double) * (size_t)(*total > 0 ? *total : 1)));
    if (*total > 0) k_sell_fill<<<2048, kThreads, 0, s>>>(rp, ci, w, n, light0, n_slices, off, *sci, w ? *sw : nullptr);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
#undef CK
done:
    if (w32) cudaFree(w32);
    if (tmp) cudaFree(tmp);
    return e;
}

template <typename T>
void to_internal(const T* src, const int32_t* perm, int64_t n, T* dst, cudaStream_t s) {
    k_gather_perm<T><<<608, kThreads, 0, s>>>(src, perm, n, dst);
}

template <typename T>
void to_external(const T* src, const int32_t* perm, int64_t n, T* dst, cudaStream_t s) {
    k_scatter_perm<T><<<608, kThreads, 0, s>>>(src, perm, n, dst);
}

template void to_internal<float>(const float*, const int32_t*, int64_t, float*, cudaStream_t);
template void to_internal<double>(const double*, const int32_t*, int64_t, double*, cudaStream_t);
template void to_external<float>(const float*, const int32_t*, int64_t, float*, cudaStream_t);
template void to_external<double>(const double*, const int32_t*, int64_t, double*, cudaStream_t);

}  // namespace isira
