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
//
// Launches of one V-cycle: level 0 takes the gather twice (W x0 and W x1) with a restriction and a
// prolongation / post-smoothing kernel around them (x0 itself usually comes from the caller's
// projection kernel); each level l >= 1 takes one fused kernel down and one up, forming x0 and x1 of
// the neighbours on the fly instead of storing them; the two coarsest levels, when small, run as
// one CTA (k_ml_tail).  Five levels (the 128^3 grid: 2.1M, 264K, 15K, 690, 38 vertices) take 9
// launches when the caller forms x0 and does level 0's post-smoothing in its own kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
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

// Fused kernels of the levels l >= 1 (no excluded vertex there).  With x0 = w D^{-1} b formed on the
// fly for every neighbour, the down sweep of a level is one kernel and so is the up sweep:
//   down  bc[I] = sum_{i in I} ((1 - w) b_i + w sum_{c in N(i)} w_ic b_c / d_c)      (restricted residual)
//   up    x1_i = w b_i / d_i + a xc[agg_i],  out_i = x1_i + w (b_i - d_i x1_i + sum_c w_ic x1_c) / d_i
// On levels l >= 1 the rows are ordered by cluster (ml_build), so the members of cluster I are the
// rows mrp[I] .. mrp[I+1]-1 and their entries one contiguous CSR range: one warp per cluster, lanes
// striding over the rows and over the entries (coalesced), G lanes per row in the up sweep.
// x0 / x1 (FP64 only, else null): the level's x0 = w D^{-1} b / x1 stored by a separate kernel, read
// instead of formed per entry: on this part an FP64 multiply costs as much as a load, so the FP64
// path stores the vectors and the FP32 path forms them on the fly.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_ml_down(const T* __restrict__ b, const T* __restrict__ dinv,
                                                      const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                      const T* __restrict__ w, const int64_t* __restrict__ mrp,
                                                      T om, int64_t nc, T* __restrict__ bc,
                                                      const T* __restrict__ x0, const int* __restrict__ done) {
    if (done && *done) return;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t I = w0; I < nc; I += nw) {
        const int64_t r_beg = mrp[I], r_end = mrp[I + 1];
        T own = T(0), s = T(0);
        for (int64_t i = r_beg + lane; i < r_end; i += 32) own += b[i];
        if (x0) {
            for (int32_t e = rp[r_beg] + lane; e < rp[r_end]; e += 32) s += w[e] * x0[ci[e]];
        } else {
            for (int32_t e = rp[r_beg] + lane; e < rp[r_end]; e += 32) {
                const int32_t c = ci[e];
                s += w[e] * (b[c] * dinv[c]);
            }
            s *= om;
        }
        const T acc = warp_sum((T(1) - om) * own + s);
        if (lane == 0) bc[I] = acc;
    }
}

template <typename T, int G>
__global__ void __launch_bounds__(kThreads) k_ml_up(const T* __restrict__ b, const T* __restrict__ dinv,
                                                    const int32_t* __restrict__ agg, const T* __restrict__ xc,
                                                    const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                    const T* __restrict__ w, T om, T alpha, int64_t n,
                                                    T* __restrict__ out, const T* __restrict__ x1v,
                                                    const int* __restrict__ done) {
    if (done && *done) return;
    const int64_t groups = ((int64_t)gridDim.x * blockDim.x) / G;
    const int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int64_t passes = (n + groups - 1) / groups;
    const int j = threadIdx.x & (G - 1);
    for (int64_t p = 0; p < passes; ++p) {
        const int64_t row = g0 + p * groups;
        const bool valid = row < n;
        T s = T(0);
        if (valid) {
            if (x1v) {
                for (int32_t e = rp[row] + j; e < rp[row + 1]; e += G) s += w[e] * x1v[ci[e]];
            } else {
                for (int32_t e = rp[row] + j; e < rp[row + 1]; e += G) {
                    const int32_t c = ci[e];
                    s += w[e] * (om * b[c] * dinv[c] + alpha * xc[agg[c]]);
                }
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
        if (valid && j == 0) {
            const T bi = b[row], di = dinv[row];
            const T x1 = x1v ? x1v[row] : om * bi * di + alpha * xc[agg[row]];
            out[row] = x1 + om * (bi * di - x1 + s * di);
        }
    }
}

// The two coarsest levels in one CTA: level t (n_t <= kMlTailMax rows, its CSR) and the dense
// coarsest level t + 1.  Restricted residual of t, dense solve, prolongation and post-smoothing of t,
// with the level-t vectors in shared memory; writes level t's output.
constexpr int kMlTailMax = 4096;
constexpr int kMlTailThreads = 1024;

template <typename T>
__global__ void __launch_bounds__(kMlTailThreads) k_ml_tail(const T* __restrict__ b, const T* __restrict__ dinv,
                                                            const int32_t* __restrict__ rp,
                                                            const int32_t* __restrict__ ci, const T* __restrict__ w,
                                                            const int32_t* __restrict__ agg,
                                                            const int64_t* __restrict__ mrp,
                                                            const int32_t* __restrict__ mem,
                                                            const T* __restrict__ inv, T om, T alpha, int nt, int nc,
                                                            T* __restrict__ out, const int* __restrict__ done) {
    if (done && *done) return;
    extern __shared__ __align__(16) unsigned char tail_sm[];
    T* r = reinterpret_cast<T*>(tail_sm);        // nt: residual, then x1
    T* bc = r + nt;                              // nc
    T* xc = bc + nc;                             // nc
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    for (int i = tid; i < nt; i += blockDim.x) {
        T s = T(0);
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
            const int32_t c = ci[e];
            s += w[e] * (b[c] * dinv[c]);
        }
        r[i] = (T(1) - om) * b[i] + om * s;
    }
    __syncthreads();
    for (int I = wp; I < nc; I += blockDim.x / 32) {
        T acc = T(0);
        for (int64_t q = mrp[I] + lane; q < mrp[I + 1]; q += 32) acc += r[mem[q]];
        acc = warp_sum(acc);
        if (lane == 0) bc[I] = acc;
    }
    __syncthreads();
    for (int I = wp; I < nc; I += blockDim.x / 32) {
        T acc = T(0);
        for (int J = lane; J < nc; J += 32) acc += inv[J + (int64_t)I * nc] * bc[J];
        acc = warp_sum(acc);
        if (lane == 0) xc[I] = acc;
    }
    __syncthreads();
    for (int i = tid; i < nt; i += blockDim.x) r[i] = om * b[i] * dinv[i] + alpha * xc[agg[i]];
    __syncthreads();
    for (int i = tid; i < nt; i += blockDim.x) {
        T s = T(0);
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) s += w[e] * r[ci[e]];
        const T x1 = r[i], di = dinv[i];
        out[i] = x1 + om * (b[i] * di - x1 + s * di);
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
        // Order the rows of every level l >= 1 that has a next level by cluster (stable), from the
        // coarse end down, so that cluster ids are final when their members are sorted: the members
        // of a cluster become consecutive rows in increasing cluster order, and the down sweep reads
        // one contiguous range per cluster.
        for (int l = (int)levels.size() - 2; l >= 1; --l) {
            const HostLevel& A = levels[l];
            std::vector<int32_t>& ag = aggs[l];
            std::vector<int64_t> order(A.n), pos(A.n);
            std::iota(order.begin(), order.end(), (int64_t)0);
            std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return ag[x] < ag[y]; });
            for (int64_t p = 0; p < A.n; ++p) pos[order[p]] = p;
            HostLevel B;
            B.n = A.n;
            B.rp.assign(A.n + 1, 0);
            B.d.resize(A.n);
            B.ci.reserve(A.ci.size());
            B.w.reserve(A.w.size());
            std::vector<int32_t> ag2(A.n);
            for (int64_t p = 0; p < A.n; ++p) {
                const int64_t i = order[p];
                B.d[p] = A.d[i];
                for (int64_t e = A.rp[i]; e < A.rp[i + 1]; ++e) {
                    B.ci.push_back((int32_t)pos[A.ci[e]]);
                    B.w.push_back(A.w[e]);
                }
                B.rp[p + 1] = (int64_t)B.ci.size();
                ag2[p] = ag[i];
            }
            levels[l] = std::move(B);
            ag = std::move(ag2);
            for (int32_t& x : aggs[l - 1])
                if (x >= 0) x = (int32_t)pos[x];
        }
        const int L = (int)levels.size();
        H.nlev = L;
        H.lev.assign(L, MlLevel<T>{});
        for (int l = 0; l < L; ++l) {
            MlLevel<T>& D = H.lev[l];
            const HostLevel& A = levels[l];
            D.n = A.n;
            D.nnz = (int64_t)A.ci.size();
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

// Whether the two coarsest levels run as one k_ml_tail CTA.
template <typename T>
static bool ml_use_tail(const MlHierarchy<T>& H) {
    return H.nlev >= 3 && H.lev[H.nlev - 2].n <= kMlTailMax && H.n_coarse <= kMlTailMax;
}

// out = M^{-1} b (b on level 0, n-space, the trimmed entry ignored; out may alias nothing else).
// gather(x, g) must compute g = sum over neighbours of x for level 0 (the solver's gather).
// x0_ready: level 0's x0 = w D^{-1} b is already in H.lev[0].x0 (written by the caller's kernel).
// skip_post0 (nlev >= 2): stop after the gather of x1 (W x1 in H.lev[0].x0); the caller's next kernel
// does level 0's post-smoothing (out is then not written).
template <typename T>
void ml_vcycle(MlHierarchy<T>& H, const T* b, T* out, const GatherFn<T>& gather, T omega, T alpha, const int* done,
               bool x0_ready, bool skip_post0, cudaStream_t s) {
    const int L = H.nlev;
    if (L == 1) {
        k_ml_dense<T><<<ml_warp_grid(H.lev[0].n), kThreads, 0, s>>>(H.inv, b, H.lev[0].n, out, done);
        return;
    }
    const bool tail = ml_use_tail(H);
    const int nmid = tail ? L - 3 : L - 2;        // levels 1..nmid take the fused down / up kernels
    MlLevel<T>& F = H.lev[0];
    // level 0 down: x0 = w D^{-1} b, its neighbour sums by the solver's gather, restricted residual
    if (!x0_ready)
        k_ml_scale<T><<<ml_grid(F.n), kThreads, 0, s>>>(b, F.dinv, omega, F.n, H.skip, F.x0, done);
    gather(F.x0, F.x, s);                                            // F.x <- W x0
    k_ml_restrict<T><<<ml_grid(H.lev[1].n), kThreads, 0, s>>>(b, F.x, T(1) - omega, F.mrp, F.mem, H.lev[1].n,
                                                              H.lev[1].b, done);
    constexpr bool store = sizeof(T) == 8;          // FP64: x0 and x1 stored, not formed per entry
    for (int l = 1; l <= nmid; ++l) {
        MlLevel<T>& D = H.lev[l];
        MlLevel<T>& C = H.lev[l + 1];
        if (store) k_ml_scale<T><<<ml_grid(D.n), kThreads, 0, s>>>(D.b, D.dinv, omega, D.n, -1, D.x0, done);
        k_ml_down<T><<<ml_warp_grid(C.n), kThreads, 0, s>>>(D.b, D.dinv, D.rp, D.ci, D.w, D.mrp, omega, C.n, C.b,
                                                            store ? D.x0 : nullptr, done);
    }
    if (tail) {
        static std::once_flag once;
        std::call_once(once, [] {
            cudaFuncSetAttribute(k_ml_tail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(T) * 3 * kMlTailMax));
        });
        MlLevel<T>& D = H.lev[L - 2];
        const int nt = (int)D.n, nc = (int)H.n_coarse;
        const int bytes = (int)(sizeof(T) * (nt + 2 * nc));
        k_ml_tail<T><<<1, kMlTailThreads, bytes, s>>>(D.b, D.dinv, D.rp, D.ci, D.w, D.agg, D.mrp, D.mem, H.inv, omega,
                                                      alpha, nt, nc, D.x, done);
    } else {
        MlLevel<T>& C = H.lev[L - 1];
        k_ml_dense<T><<<ml_warp_grid(C.n), kThreads, 0, s>>>(H.inv, C.b, C.n, C.x, done);
    }
    for (int l = nmid; l >= 1; --l) {
        MlLevel<T>& D = H.lev[l];
        if (store)
            k_ml_prolong<T><<<ml_grid(D.n), kThreads, 0, s>>>(D.b, D.dinv, D.agg, H.lev[l + 1].x, omega, alpha, D.n,
                                                              D.x1, done);
        k_ml_up<T, kMlLanes><<<ml_group_grid(D.n, kMlLanes), kThreads, 0, s>>>(D.b, D.dinv, D.agg, H.lev[l + 1].x, D.rp,
                                                                                D.ci, D.w, omega, alpha, D.n, D.x,
                                                                                store ? D.x1 : nullptr, done);
    }
    // level 0 up: prolong, neighbour sums of x1, post-smooth
    k_ml_prolong<T><<<ml_grid(F.n), kThreads, 0, s>>>(b, F.dinv, F.agg, H.lev[1].x, omega, alpha, F.n, F.x1, done);
    gather(F.x1, F.x0, s);                                           // F.x0 <- W x1 (x0 is free now)
    if (!skip_post0)
        k_ml_post<T><<<ml_grid(F.n), kThreads, 0, s>>>(b, F.dinv, F.x1, F.x0, omega, F.n, H.skip, out, done);
}

template <typename T>
int ml_launches(const MlHierarchy<T>& H, bool x0_ready, bool skip_post0) {
    if (H.nlev <= 1) return 1;
    const int nmid = ml_use_tail(H) ? H.nlev - 3 : H.nlev - 2;
    return (x0_ready ? 0 : 1) + 2 + (sizeof(T) == 8 ? 4 : 2) * nmid + 1 + (skip_post0 ? 2 : 3);
}

#define ISIRA_INSTANTIATE_ML(T)                                                                              \
    template cudaError_t ml_build<T>(MlHierarchy<T>&, const int64_t*, const int32_t*, const double*, int64_t,  \
                                     int64_t, int64_t, cudaStream_t);                                        \
    template void ml_free<T>(MlHierarchy<T>&);                                                               \
    template void ml_vcycle<T>(MlHierarchy<T>&, const T*, T*, const GatherFn<T>&, T, T, const int*, bool,     \
                               bool, cudaStream_t);                                                          \
    template int ml_launches<T>(const MlHierarchy<T>&, bool, bool);
ISIRA_INSTANTIATE_ML(float)
ISIRA_INSTANTIATE_ML(double)

}  // namespace isira
