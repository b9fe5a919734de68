// multilevel.cu -- an aggregation multilevel preconditioner for the inner solve.
//
// The paper preconditions the trimmed systems with combinatorial multigrid (Sec. 3.2; Remark 3.2,
// with the deflated form of Eq. 3.6).  This file builds a multilevel preconditioner of the same
// kind for M ~ Lh, the trimmed Laplacian (Theorem 2.3: an SPD M-matrix):
//  * level 0 is the graph without the trimmed vertex, with the full degrees on the diagonal (the
//    trimmed vertex acts as a Dirichlet node for its neighbours);
//  * the vertices of a level are grouped into small connected clusters by greedy aggregation
//    (a vertex whose neighbours are all free starts a cluster with them; leftover vertices join
//    the neighbouring cluster they are most strongly tied to);
//  * each cluster becomes one vertex of the next level, whose matrix is the Galerkin product
//    P^T A P with the piecewise-constant P: again a weighted Laplacian, with edge weights summed
//    between clusters and the clusters' Dirichlet mass kept on the diagonal;
//  * levels stop at <= kMlCoarse vertices, whose matrix is inverted densely on the host.
// M^{-1} b is one V-cycle: on each level x0 = w D^{-1} b, the residual restricted to the next level,
// x1 = x0 + a P x_c, and one more damped Jacobi step x1 + w D^{-1} (b - A x1).  With the same
// smoother before and after the coarse correction the cycle is a symmetric operator, positive
// definite for w < 1 (the levels are diagonally dominant, so rho(D^{-1} A) <= 2) and any a > 0.
//
// Storage per level l >= 1: CSR (int32 row pointers) of the off-diagonal weights W (positive; the
// matrix is diag(d) - W), 1/d, the cluster map of level l-1 (fine vertex -> cluster) and the member
// lists of the clusters (CSR over the clusters).  Level 0 uses the solver's own gather for W x.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "internal.h"

namespace isira {

constexpr int kMlCoarse = 512;       // the coarsest level is solved with a dense inverse
constexpr int kMlMaxLevels = 12;

struct HostLevel {
    int64_t n = 0;
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    std::vector<double> w;       // off-diagonal weights (positive)
    std::vector<double> d;       // diagonal
};

// Greedy aggregation.  skip: a vertex excluded from every cluster (-1: none).  Returns the
// cluster id of every vertex (-1 for skip) and the cluster count.
static std::vector<int32_t> aggregate(const HostLevel& A, int64_t skip, int64_t* n_agg) {
    const int64_t n = A.n;
    std::vector<int32_t> agg(n, -1);
    std::vector<char> p1(n, 0);
    int32_t next = 0;
    // phase 1: a vertex whose neighbours are all free starts a cluster with all of them
    for (int64_t i = 0; i < n; ++i) {
        if (i == skip || agg[i] >= 0) continue;
        bool free_nb = true;
        for (int64_t e = A.rp[i]; e < A.rp[i + 1] && free_nb; ++e) {
            const int64_t j = A.ci[e];
            if (j != skip && agg[j] >= 0) free_nb = false;
        }
        if (!free_nb) continue;
        agg[i] = next;
        p1[i] = 1;
        for (int64_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
            const int64_t j = A.ci[e];
            if (j != skip) {
                agg[j] = next;
                p1[j] = 1;
            }
        }
        ++next;
    }
    // phase 2: every free vertex joins the phase-1 cluster it is most strongly tied to
    std::vector<int32_t> join(n, -1);
    for (int64_t i = 0; i < n; ++i) {
        if (i == skip || agg[i] >= 0) continue;
        double best = 0.0;
        int32_t bid = -1;
        for (int64_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
            const int64_t j = A.ci[e];
            if (j == skip || !p1[j]) continue;
            if (A.w[e] > best || (A.w[e] == best && agg[j] < bid)) {
                best = A.w[e];
                bid = agg[j];
            }
        }
        join[i] = bid;
    }
    for (int64_t i = 0; i < n; ++i)
        if (join[i] >= 0) agg[i] = join[i];
    // phase 3: what is still free forms clusters with its free neighbours
    for (int64_t i = 0; i < n; ++i) {
        if (i == skip || agg[i] >= 0) continue;
        agg[i] = next;
        for (int64_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
            const int64_t j = A.ci[e];
            if (j != skip && agg[j] < 0) agg[j] = next;
        }
        ++next;
    }
    *n_agg = next;
    return agg;
}

// Galerkin coarse matrix P^T A P for the piecewise-constant P of `agg`.
static HostLevel coarsen(const HostLevel& A, const std::vector<int32_t>& agg, int64_t nc) {
    HostLevel C;
    C.n = nc;
    C.d.assign(nc, 0.0);
    // members of each cluster, in fine order
    std::vector<int64_t> mrp(nc + 1, 0);
    for (int64_t i = 0; i < A.n; ++i)
        if (agg[i] >= 0) mrp[agg[i] + 1]++;
    for (int64_t I = 0; I < nc; ++I) mrp[I + 1] += mrp[I];
    std::vector<int64_t> mem(mrp[nc]);
    {
        std::vector<int64_t> pos(mrp.begin(), mrp.end() - 1);
        for (int64_t i = 0; i < A.n; ++i)
            if (agg[i] >= 0) mem[pos[agg[i]]++] = i;
    }
    std::vector<double> acc(nc, 0.0);
    std::vector<int32_t> mark(nc, -1);
    std::vector<int32_t> cols;
    C.rp.assign(nc + 1, 0);
    for (int64_t I = 0; I < nc; ++I) {
        cols.clear();
        double dI = 0.0;
        for (int64_t q = mrp[I]; q < mrp[I + 1]; ++q) {
            const int64_t i = mem[q];
            dI += A.d[i];
            for (int64_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
                const int32_t J = agg[A.ci[e]];
                if (J < 0) continue;                         // an edge to the excluded vertex
                if (J == I) {
                    dI -= A.w[e];                            // internal edge: P^T A P adds -w twice
                    continue;
                }
                if (mark[J] != I) {
                    mark[J] = (int32_t)I;
                    acc[J] = 0.0;
                    cols.push_back(J);
                }
                acc[J] += A.w[e];
            }
        }
        std::sort(cols.begin(), cols.end());
        for (int32_t J : cols) {
            C.ci.push_back(J);
            C.w.push_back(acc[J]);
        }
        C.d[I] = dI;
        C.rp[I + 1] = (int64_t)C.ci.size();
    }
    return C;
}

// Dense inverse of the SPD matrix of a (small) level by Cholesky; column-major n x n.  The row
// and column of `skip` (the trimmed vertex, when level 0 itself is the coarsest) become identity.
static bool dense_inverse(const HostLevel& A, int64_t skip, std::vector<double>& inv) {
    const int64_t n = A.n;
    std::vector<double> M(n * n, 0.0);
    for (int64_t i = 0; i < n; ++i) {
        M[i + i * n] = A.d[i];
        for (int64_t e = A.rp[i]; e < A.rp[i + 1]; ++e) M[i + (int64_t)A.ci[e] * n] -= A.w[e];
    }
    if (skip >= 0 && skip < n) {
        for (int64_t i = 0; i < n; ++i) {
            M[i + skip * n] = 0.0;
            M[skip + i * n] = 0.0;
        }
        M[skip + skip * n] = 1.0;
    }
    // Cholesky M = L L^T in place (lower triangle)
    for (int64_t j = 0; j < n; ++j) {
        double s = M[j + j * n];
        for (int64_t k = 0; k < j; ++k) s -= M[j + k * n] * M[j + k * n];
        if (!(s > 0.0)) return false;
        const double ljj = std::sqrt(s);
        M[j + j * n] = ljj;
        for (int64_t i = j + 1; i < n; ++i) {
            double t = M[i + j * n];
            for (int64_t k = 0; k < j; ++k) t -= M[i + k * n] * M[j + k * n];
            M[i + j * n] = t / ljj;
        }
    }
    inv.assign(n * n, 0.0);
    std::vector<double> y(n);
    for (int64_t c = 0; c < n; ++c) {
        for (int64_t i = 0; i < n; ++i) {
            double t = (i == c) ? 1.0 : 0.0;
            for (int64_t k = 0; k < i; ++k) t -= M[i + k * n] * y[k];
            y[i] = t / M[i + i * n];
        }
        for (int64_t i = n - 1; i >= 0; --i) {
            double t = y[i];
            for (int64_t k = i + 1; k < n; ++k) t -= M[k + i * n] * y[k];
            y[i] = t / M[i + i * n];
        }
        for (int64_t i = 0; i < n; ++i) inv[i + c * n] = y[i];
    }
    return true;
}

// ------------------------------------------------------------------ device kernels of the V-cycle

template <typename T>
__global__ void __launch_bounds__(kThreads) k_ml_scale(const T* __restrict__ b, const T* __restrict__ dinv, T om,
                                                       int64_t n, int64_t skip, T* __restrict__ x,
                                                       const int* __restrict__ done) {
    if (done && *done) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = i == skip ? T(0) : om * b[i] * dinv[i];
}

// (W x)_r for the rows of a coarse level, G lanes per row (strided over the row's entries, then a
// shuffle reduction); every warp runs the same number of passes so the shuffles stay converged
template <typename T, int G>
__device__ __forceinline__ T csr_row_sum(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                         const T* __restrict__ w, const T* __restrict__ x, int64_t row, bool valid) {
    T s = T(0);
    if (valid) {
        const int j = threadIdx.x & (G - 1);
        for (int32_t e = rp[row] + j; e < rp[row + 1]; e += G) s += w[e] * x[ci[e]];
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    return s;
}

// coarse level: r = b - A x0 at x0 = w D^{-1} b, i.e. (1 - w) b + W x0
template <typename T, int G>
__global__ void __launch_bounds__(kThreads) k_ml_resid(const T* __restrict__ b, const T* __restrict__ x0,
                                                       const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                       const T* __restrict__ w, T om, int64_t n, T* __restrict__ r,
                                                       const int* __restrict__ done) {
    if (done && *done) return;
    const int64_t groups = ((int64_t)gridDim.x * blockDim.x) / G;
    const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int64_t passes = (n + groups - 1) / groups;
    for (int64_t p = 0; p < passes; ++p) {
        const int64_t row = g0 + p * groups;
        const T s = csr_row_sum<T, G>(rp, ci, w, x0, row, row < n);
        if (row < n && (threadIdx.x & (G - 1)) == 0) r[row] = (T(1) - om) * b[row] + s;
    }
}

// bc[I] = sum over the members i of cluster I of (ob * b_i + add_i): level 0 passes ob = 1 - w and
// add = W x0 (the gather), so the summand is the residual (1 - w) b + W x0; coarser levels pass ob = 0
// and add = their residual.  One thread per cluster.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_ml_restrict(const T* __restrict__ b, const T* __restrict__ add, T ob,
                                                          const int64_t* __restrict__ mrp,
                                                          const int32_t* __restrict__ mem, int64_t nc,
                                                          T* __restrict__ bc, const int* __restrict__ done) {
    if (done && *done) return;
    for (int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += (int64_t)gridDim.x * blockDim.x) {
        T s = T(0);
        for (int64_t q = mrp[I]; q < mrp[I + 1]; ++q) {
            const int32_t i = mem[q];
            s += ob * b[i] + add[i];
        }
        bc[I] = s;
    }
}

// x1 = x0 + a xc[agg(i)] (x0 = w D^{-1} b recomputed); the excluded vertex stays 0
template <typename T>
__global__ void __launch_bounds__(kThreads) k_ml_prolong(const T* __restrict__ b, const T* __restrict__ dinv,
                                                         const int32_t* __restrict__ agg, const T* __restrict__ xc,
                                                         T om, T alpha, int64_t n, T* __restrict__ x1,
                                                         const int* __restrict__ done) {
    if (done && *done) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t I = agg[i];
        x1[i] = I < 0 ? T(0) : om * b[i] * dinv[i] + alpha * xc[I];
    }
}

// post-smoothing: out = x1 + w D^{-1} (b - d x1 + W x1); level 0 takes (W x1) from the gather
template <typename T>
__global__ void __launch_bounds__(kThreads) k_ml_post(const T* __restrict__ b, const T* __restrict__ dinv,
                                                      const T* __restrict__ x1, const T* __restrict__ wx1, T om,
                                                      int64_t n, int64_t skip, T* __restrict__ out,
                                                      const int* __restrict__ done) {
    if (done && *done) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (i == skip) {
            out[i] = T(0);
            continue;
        }
        const T xi = x1[i], di = dinv[i];
        out[i] = xi + om * (b[i] * di - xi + wx1[i] * di);
    }
}

// the same on a coarse level, (W x1) from its CSR with G lanes per row
template <typename T, int G>
__global__ void __launch_bounds__(kThreads) k_ml_post_csr(const T* __restrict__ b, const T* __restrict__ dinv,
                                                          const T* __restrict__ x1, const int32_t* __restrict__ rp,
                                                          const int32_t* __restrict__ ci, const T* __restrict__ w, T om,
                                                          int64_t n, T* __restrict__ out, const int* __restrict__ done) {
    if (done && *done) return;
    const int64_t groups = ((int64_t)gridDim.x * blockDim.x) / G;
    const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int64_t passes = (n + groups - 1) / groups;
    for (int64_t p = 0; p < passes; ++p) {
        const int64_t row = g0 + p * groups;
        const T s = csr_row_sum<T, G>(rp, ci, w, x1, row, row < n);
        if (row < n && (threadIdx.x & (G - 1)) == 0) {
            const T xi = x1[row], di = dinv[row];
            out[row] = xi + om * (b[row] * di - xi + s * di);
        }
    }
}

// coarsest level: x = A^{-1} b with the dense inverse, one warp per row (the inverse is symmetric,
// so row i is column i: coalesced)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_ml_dense(const T* __restrict__ inv, const T* __restrict__ b, int64_t n,
                                                       T* __restrict__ x, const int* __restrict__ done) {
    if (done && *done) return;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < n; i += nw) {
        T s = T(0);
        for (int64_t j = lane; j < n; j += 32) s += inv[j + i * n] * b[j];
        s = warp_sum(s);
        if (lane == 0) x[i] = s;
    }
}

// ------------------------------------------------------------------ hierarchy

template <typename T>
static void upload(T** dst, const std::vector<double>& src) {
    std::vector<T> tmp(src.begin(), src.end());
    CUDA_OK(cudaMalloc(dst, sizeof(T) * std::max<size_t>(1, tmp.size())));
    if (!tmp.empty()) CUDA_OK(cudaMemcpy(*dst, tmp.data(), sizeof(T) * tmp.size(), cudaMemcpyHostToDevice));
}

template <typename I>
static void upload_i(I** dst, const std::vector<I>& src) {
    CUDA_OK(cudaMalloc(dst, sizeof(I) * std::max<size_t>(1, src.size())));
    if (!src.empty()) CUDA_OK(cudaMemcpy(*dst, src.data(), sizeof(I) * src.size(), cudaMemcpyHostToDevice));
}

template <typename T>
cudaError_t ml_build(MlHierarchy<T>& H, const int64_t* d_rp, const int32_t* d_ci, const double* d_w, int64_t n,
                     int64_t ld, int64_t skip, cudaStream_t s) {
    try {
        HostLevel A0;
        A0.n = n;
        A0.rp.resize(n + 1);
        CUDA_OK(cudaMemcpyAsync(A0.rp.data(), d_rp, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s));
        CUDA_OK(cudaStreamSynchronize(s));
        A0.ci.resize(A0.rp[n]);
        CUDA_OK(cudaMemcpyAsync(A0.ci.data(), d_ci, sizeof(int32_t) * A0.rp[n], cudaMemcpyDeviceToHost, s));
        CUDA_OK(cudaStreamSynchronize(s));
        A0.w.assign(A0.rp[n], 1.0);
        if (d_w) {
            CUDA_OK(cudaMemcpyAsync(A0.w.data(), d_w, sizeof(double) * A0.rp[n], cudaMemcpyDeviceToHost, s));
            CUDA_OK(cudaStreamSynchronize(s));
        }
        A0.d.assign(n, 0.0);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t e = A0.rp[i]; e < A0.rp[i + 1]; ++e) A0.d[i] += A0.w[e];
        H.n0 = n;
        H.skip = skip;
        std::vector<HostLevel> levels;
        levels.push_back(std::move(A0));
        std::vector<std::vector<int32_t>> aggs;
        while ((int)levels.size() < kMlMaxLevels && levels.back().n > kMlCoarse) {
            int64_t nc = 0;
            const int64_t sk = levels.size() == 1 ? skip : -1;
            std::vector<int32_t> agg = aggregate(levels.back(), sk, &nc);
            if (nc >= levels.back().n * 9 / 10 || nc < 1) break;    // no useful coarsening left
            HostLevel C = coarsen(levels.back(), agg, nc);
            aggs.push_back(std::move(agg));
            levels.push_back(std::move(C));
        }
        const int L = (int)levels.size();
        H.nlev = L;
        H.lev.assign(L, MlLevel<T>{});
        for (int l = 0; l < L; ++l) {
            MlLevel<T>& D = H.lev[l];
            const HostLevel& A = levels[l];
            D.n = A.n;
            std::vector<double> dinv(l == 0 ? ld : A.n, 0.0);
            for (int64_t i = 0; i < A.n; ++i) dinv[i] = (l == 0 && i == skip) ? 0.0 : 1.0 / A.d[i];
            upload<T>(&D.dinv, dinv);
            if (l > 0) {
                std::vector<int32_t> rp32(A.n + 1);
                for (int64_t i = 0; i <= A.n; ++i) rp32[i] = (int32_t)A.rp[i];
                upload_i<int32_t>(&D.rp, rp32);
                upload_i<int32_t>(&D.ci, A.ci);
                upload<T>(&D.w, A.w);
            }
            const size_t nv = (size_t)(l == 0 ? ld : A.n);
            CUDA_OK(cudaMalloc(&D.b, sizeof(T) * nv));
            CUDA_OK(cudaMalloc(&D.x0, sizeof(T) * nv));
            CUDA_OK(cudaMalloc(&D.x1, sizeof(T) * nv));
            CUDA_OK(cudaMalloc(&D.x, sizeof(T) * nv));
            CUDA_OK(cudaMemsetAsync(D.x0, 0, sizeof(T) * nv, s));
            CUDA_OK(cudaMemsetAsync(D.x1, 0, sizeof(T) * nv, s));
            if (l + 1 < L) {
                const std::vector<int32_t>& agg = aggs[l];
                std::vector<int32_t> agg_pad(nv, -1);
                std::copy(agg.begin(), agg.end(), agg_pad.begin());
                upload_i<int32_t>(&D.agg, agg_pad);
                const int64_t nc = levels[l + 1].n;
                std::vector<int64_t> mrp(nc + 1, 0);
                for (int32_t I : agg)
                    if (I >= 0) mrp[I + 1]++;
                for (int64_t I = 0; I < nc; ++I) mrp[I + 1] += mrp[I];
                std::vector<int32_t> mem(mrp[nc]);
                std::vector<int64_t> pos(mrp.begin(), mrp.end() - 1);
                for (int64_t i = 0; i < (int64_t)agg.size(); ++i)
                    if (agg[i] >= 0) mem[pos[agg[i]]++] = (int32_t)i;
                upload_i<int64_t>(&D.mrp, mrp);
                upload_i<int32_t>(&D.mem, mem);
            }
        }
        std::vector<double> inv;
        if (!dense_inverse(levels[L - 1], L == 1 ? skip : -1, inv)) return cudaErrorInvalidValue;
        upload<T>(&H.inv, inv);
        H.n_coarse = levels[L - 1].n;
        CUDA_OK(cudaStreamSynchronize(s));
    } catch (CudaFailure& f) {
        return f.e;
    } catch (std::bad_alloc&) {
        return cudaErrorMemoryAllocation;
    }
    return cudaSuccess;
}

template <typename T>
void ml_free(MlHierarchy<T>& H) {
    for (MlLevel<T>& D : H.lev) {
        void* ptrs[] = {D.dinv, D.rp, D.ci, D.w, D.agg, D.mrp, D.mem, D.b, D.x0, D.x1, D.x};
        for (void* p : ptrs)
            if (p) cudaFree(p);
    }
    if (H.inv) cudaFree(H.inv);
    H.lev.clear();
    H.inv = nullptr;
    H.nlev = 0;
}

static int ml_grid(int64_t n) {
    const int64_t g = (n + kThreads - 1) / kThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 1216));
}

static int ml_warp_grid(int64_t n) {
    const int64_t g = (n * 32 + kThreads - 1) / kThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 2432));
}

static int ml_group_grid(int64_t n, int G) {
    const int64_t g = (n * G + kThreads - 1) / kThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 2432));
}

constexpr int kMlLanes = 4;          // lanes per coarse CSR row

// out = M^{-1} b (b on level 0, n-space, the trimmed entry ignored; out may alias nothing else).
// gather(x, g) must compute g = sum over neighbours of x for level 0 (the solver's gather).
template <typename T>
void ml_vcycle(MlHierarchy<T>& H, const T* b, T* out, const GatherFn<T>& gather, T omega, T alpha, const int* done,
               cudaStream_t s) {
    const int L = H.nlev;
    const T* bl = b;
    // downward: x0 = w D^{-1} b, restrict the residual
    for (int l = 0; l < L - 1; ++l) {
        MlLevel<T>& D = H.lev[l];
        MlLevel<T>& C = H.lev[l + 1];
        k_ml_scale<T><<<ml_grid(D.n), kThreads, 0, s>>>(bl, D.dinv, omega, D.n, l == 0 ? H.skip : -1, D.x0, done);
        if (l == 0) {
            gather(D.x0, D.x, s);                                    // D.x <- W x0
            k_ml_restrict<T><<<ml_grid(C.n), kThreads, 0, s>>>(bl, D.x, T(1) - omega, D.mrp, D.mem, C.n, C.b, done);
        } else {
            k_ml_resid<T, kMlLanes><<<ml_group_grid(D.n, kMlLanes), kThreads, 0, s>>>(bl, D.x0, D.rp, D.ci, D.w,
                                                                                        omega, D.n, D.x, done);
            k_ml_restrict<T><<<ml_grid(C.n), kThreads, 0, s>>>(bl, D.x, T(0), D.mrp, D.mem, C.n, C.b, done);
        }
        bl = C.b;
    }
    // coarsest
    MlLevel<T>& Lc = H.lev[L - 1];
    T* xc = L == 1 ? out : Lc.x;
    k_ml_dense<T><<<ml_warp_grid(Lc.n), kThreads, 0, s>>>(H.inv, L == 1 ? b : Lc.b, Lc.n, xc, done);
    // upward: prolong, post-smooth
    for (int l = L - 2; l >= 0; --l) {
        MlLevel<T>& D = H.lev[l];
        const T* bd = l == 0 ? b : D.b;
        k_ml_prolong<T><<<ml_grid(D.n), kThreads, 0, s>>>(bd, D.dinv, D.agg, xc, omega, alpha, D.n, D.x1, done);
        T* dst = l == 0 ? out : D.x;
        if (l == 0) {
            gather(D.x1, D.x0, s);                                   // D.x0 <- W x1 (x0 is free now)
            k_ml_post<T><<<ml_grid(D.n), kThreads, 0, s>>>(bd, D.dinv, D.x1, D.x0, omega, D.n, H.skip, dst, done);
        } else {
            k_ml_post_csr<T, kMlLanes><<<ml_group_grid(D.n, kMlLanes), kThreads, 0, s>>>(bd, D.dinv, D.x1, D.rp, D.ci,
                                                                                          D.w, omega, D.n, dst, done);
        }
        xc = dst;
    }
}

template <typename T>
int ml_launches(const MlHierarchy<T>& H) {
    return H.nlev <= 1 ? 1 : 6 + 5 * (H.nlev - 2) + 1;
}

#define ISIRA_INSTANTIATE_ML(T)                                                                              \
    template cudaError_t ml_build<T>(MlHierarchy<T>&, const int64_t*, const int32_t*, const double*, int64_t,  \
                                     int64_t, int64_t, cudaStream_t);                                        \
    template void ml_free<T>(MlHierarchy<T>&);                                                               \
    template void ml_vcycle<T>(MlHierarchy<T>&, const T*, T*, const GatherFn<T>&, T, T, const int*, cudaStream_t); \
    template int ml_launches<T>(const MlHierarchy<T>&);
ISIRA_INSTANTIATE_ML(float)
ISIRA_INSTANTIATE_ML(double)

}  // namespace isira
