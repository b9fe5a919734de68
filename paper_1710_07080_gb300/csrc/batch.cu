// batch.cu -- many independent graphs solved concurrently (one solver and one CUDA stream per
// graph, driven by a pool of host threads that take graphs largest first).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <numeric>
#include <thread>
#include <vector>

#include "../../include/isira.h"

// default pool size: the threads mostly sleep on blocking-sync events, so the pool can be much
// larger than the host's core count; it bounds how many graphs are in flight on the GPU at once
constexpr int kBatchThreads = 64;

struct isira_batch_s {
    int G = 0;
    int device = 0;
    std::vector<isira_handle> h;
    std::vector<cudaStream_t> streams;
    std::vector<int64_t> n, nnz;
    std::vector<isira_status> status;
};

extern "C" {

isira_status isira_batch_create(isira_batch* out, int G, const int64_t* h_n, const int64_t* h_nnz,
                                const int64_t* const* d_row_ptr, const int32_t* const* d_col_idx,
                                const isira_opts* opts) {
    if (!out) return ISIRA_ERR_INVALID_ARG;
    *out = nullptr;
    if (G < 1 || !h_n || !h_nnz || !d_row_ptr || !d_col_idx) return ISIRA_ERR_INVALID_ARG;
    isira_batch b = new isira_batch_s();
    b->G = G;
    cudaGetDevice(&b->device);
    b->h.assign(G, nullptr);
    b->streams.assign(G, nullptr);
    b->n.assign(h_n, h_n + G);
    b->nnz.assign(h_nnz, h_nnz + G);
    b->status.assign(G, ISIRA_ERR_NOT_SOLVED);
    isira_opts o;
    if (opts) o = *opts;
    else isira_default_opts(&o);
    o.blocking_sync = 1;
    isira_status st = ISIRA_OK;
    for (int g = 0; g < G && st == ISIRA_OK; ++g) {
        if (cudaStreamCreateWithFlags(&b->streams[g], cudaStreamNonBlocking) != cudaSuccess) {
            st = ISIRA_ERR_CUDA;
            break;
        }
        st = isira_create(&b->h[g], h_n[g], h_nnz[g], d_row_ptr[g], d_col_idx[g], &o, b->streams[g]);
    }
    if (st != ISIRA_OK) {
        isira_batch_destroy(b);
        return st;
    }
    *out = b;
    return ISIRA_OK;
}

isira_status isira_batch_solve(isira_batch b, int k, double sigma, double tol_rel, int n_threads) {
    if (!b || !(tol_rel >= 0.0)) return ISIRA_ERR_INVALID_ARG;
    const int G = b->G;
    std::vector<int> order(G);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->nnz[a] + b->n[a] > b->nnz[c] + b->n[c]; });
    const int T = std::max(1, std::min(G, n_threads > 0 ? n_threads : kBatchThreads));
    std::atomic<int> next(0);
    auto worker = [&]() {
        cudaSetDevice(b->device);
        while (true) {
            const int i = next.fetch_add(1);
            if (i >= G) break;
            const int g = order[i];
            isira_stats st{};
            isira_get_stats(b->h[g], &st);
            b->status[g] = isira_solve(b->h[g], k, sigma, tol_rel * st.norm_L, nullptr);
        }
    };
    std::vector<std::thread> pool;
    for (int t = 0; t < T; ++t) pool.emplace_back(worker);
    for (auto& th : pool) th.join();
    for (int g = 0; g < G; ++g)
        if (b->status[g] != ISIRA_OK) return b->status[g];
    return ISIRA_OK;
}

isira_status isira_batch_status(isira_batch b, int g) {
    if (!b || g < 0 || g >= b->G) return ISIRA_ERR_INVALID_ARG;
    return b->status[g];
}

isira_status isira_batch_eigpairs(isira_batch b, int g, double* h_eigvals, double* d_eigvecs, double* h_true_resid,
                                  int* n_out) {
    if (!b || g < 0 || g >= b->G) return ISIRA_ERR_INVALID_ARG;
    return isira_eigpairs(b->h[g], h_eigvals, d_eigvecs, h_true_resid, n_out);
}

isira_status isira_batch_get_stats(isira_batch b, int g, isira_stats* out) {
    if (!b || g < 0 || g >= b->G) return ISIRA_ERR_INVALID_ARG;
    return isira_get_stats(b->h[g], out);
}

void isira_batch_destroy(isira_batch b) {
    if (!b) return;
    for (auto h : b->h)
        if (h) isira_destroy(h);
    for (auto s : b->streams)
        if (s) cudaStreamDestroy(s);
    delete b;
}

}  // extern "C"
