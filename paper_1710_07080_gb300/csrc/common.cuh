// common.cuh -- device building blocks shared by the iSIRA kernels (sm_103a).
//
//  * deterministic block reductions with a "last block finishes" step: every block
//    writes its partial sums, the block that arrives last adds them in a fixed
//    order, so a reduction needs no second launch and gives the same bits on
//    every run;
//  * a three-tier CSR row scheduler for skewed (power-law) degrees: rows of
//    degree > kHeavyDeg get a whole CTA, rows above the light threshold get one
//    warp, and all other rows are processed in tiles of 32 consecutive rows by
//    G lanes per row, so that the per-row epilogue runs with one lane per row and
//    coalesced vector accesses;
//  * SplitMix64 (Vigna), the counter-based generator of replacement vectors.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace isira {

constexpr int kThreads = 256;         // threads per CTA for every kernel here
constexpr int kWarps = kThreads / 32;
constexpr int kCMax = 32;             // max locked vectors (deflation rank) supported
constexpr int kMMax = 64;             // max search-space dimension
constexpr int kHeavyDeg = 4096;       // rows above this degree get a whole CTA
constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------ host-visible status
// Written by the device (last blocks) into mapped pinned memory, read by the host
// after a stream synchronisation.
struct HostStatus {
    double rnorm;          // ||r||_2 of the current Ritz pair
    double theta[2];       // two smallest Ritz values
    double cgs_in;         // ||z|| entering orthogonalisation
    double cgs_out;        // ||z|| after two Gram-Schmidt passes
    double inner_relres;   // MINRES relative residual estimate
    double gram_dot;       // spare scalar channel
    int inner_done;
    int inner_iters;
    int eig_sweeps;        // Jacobi sweeps used (-1: not converged)
    int pad;
};

// ------------------------------------------------------------------ reductions
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Reduces NV per-thread values over the block; the block's sums go to
// partial[i * pstride + blockIdx.x] (i < nv).  Returns true in the last block to
// arrive, after which all partials of all blocks are visible to it.
template <typename T, int NV>
__device__ __forceinline__ bool block_partials_arrive(T (&v)[NV], int nv, T* partial, int pstride,
                                                      unsigned* counter) {
    __shared__ T red[kWarps][NV];
    __shared__ int last;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        if (i < nv) {
            T s = warp_sum(v[i]);
            if (lane == 0) red[w][i] = s;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
        T s = 0;
#pragma unroll
        for (int q = 0; q < kWarps; ++q) s += red[q][i];
        partial[(size_t)i * pstride + blockIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    return last != 0;
}

// In the last block: out[i] = sum over blocks of partial[i * pstride + b], in a fixed
// order (lane-strided, then a fixed shuffle tree).  out is shared memory.  Resets the
// arrival counter for the next launch.
template <typename T>
__device__ __forceinline__ void last_block_sum(const T* partial, int pstride, int nb, int nv, T* out,
                                               unsigned* counter) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = w; i < nv; i += kWarps) {
        T s = 0;
        for (int b = lane; b < nb; b += 32) s += __ldcg(partial + (size_t)i * pstride + b);
        s = warp_sum(s);
        if (lane == 0) out[i] = s;
    }
    if (threadIdx.x == 0) *counter = 0u;
    __syncthreads();
}

// Sum over the block, result valid in thread 0.
template <typename T>
__device__ __forceinline__ T block_sum0(T v) {
    __shared__ T s[kWarps];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    T r = 0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < kWarps; ++q) r += s[q];
    }
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------ row scheduler
// Grid layout of an SpMV-style launch: [heavy CTAs][medium CTAs][light CTAs].
struct RowSched {
    const int64_t* __restrict__ rp;
    const int32_t* __restrict__ ci;
    int64_t n;
    const int32_t* __restrict__ heavy;   // rows of degree > kHeavyDeg, ascending
    const int32_t* __restrict__ medium;  // rows of degree in (light_deg, kHeavyDeg], ascending
    int n_heavy, n_medium;
    int medium_blocks, light_blocks;
    int light_deg;
    __host__ __device__ int grid() const { return n_heavy + medium_blocks + light_blocks; }
};

// Calls epi(row, degree, sum_{c in N(row)} x[c]) exactly once for every row 0..n-1.
// G = lanes per light row (1, 2, 4, 8, 16 or 32).
template <typename T, int G, class Epi>
__device__ __forceinline__ void for_each_row_gather(const RowSched& S, const T* __restrict__ x, Epi& epi) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int b = blockIdx.x;
    if (b < S.n_heavy) {                                   // one CTA per heavy row
        const int64_t r = S.heavy[b];
        const int64_t beg = S.rp[r], end = S.rp[r + 1];
        T s0 = 0, s1 = 0;
        int64_t e = beg + threadIdx.x;
        for (; e + blockDim.x < end; e += 2 * blockDim.x) {
            s0 += __ldg(x + __ldg(S.ci + e));
            s1 += __ldg(x + __ldg(S.ci + e + blockDim.x));
        }
        if (e < end) s0 += __ldg(x + __ldg(S.ci + e));
        T s = block_sum0(s0 + s1);
        if (threadIdx.x == 0) epi(r, end - beg, s);
        return;
    }
    b -= S.n_heavy;
    if (b < S.medium_blocks) {                             // one warp per medium row
        for (int64_t i = (int64_t)b * kWarps + warp; i < S.n_medium; i += (int64_t)S.medium_blocks * kWarps) {
            const int64_t r = S.medium[i];
            const int64_t beg = S.rp[r], end = S.rp[r + 1];
            T s0 = 0, s1 = 0;
            int64_t e = beg + lane;
            for (; e + 32 < end; e += 64) {
                s0 += __ldg(x + __ldg(S.ci + e));
                s1 += __ldg(x + __ldg(S.ci + e + 32));
            }
            if (e < end) s0 += __ldg(x + __ldg(S.ci + e));
            T s = warp_sum(s0 + s1);
            if (lane == 0) epi(r, end - beg, s);
        }
        return;
    }
    b -= S.medium_blocks;
    constexpr int RPS = 32 / G;                            // rows per sub-pass
    const int64_t ntiles = (S.n + 31) >> 5;
    for (int64_t tile = (int64_t)b * kWarps + warp; tile < ntiles; tile += (int64_t)S.light_blocks * kWarps) {
        const int64_t row = tile * 32 + lane;
        const bool valid = row < S.n;
        const int64_t beg = valid ? S.rp[row] : 0;
        const int64_t end = valid ? S.rp[row + 1] : 0;
        const int light = valid && (end - beg) <= S.light_deg;
        T mine = 0;
#pragma unroll
        for (int sub = 0; sub < G; ++sub) {
            const int src = sub * RPS + lane / G;
            const int64_t sb = __shfl_sync(kFull, beg, src);
            const int64_t se = __shfl_sync(kFull, end, src);
            const int sl = __shfl_sync(kFull, light, src);
            T s = 0;
            if (sl) {
                int64_t e = sb + (lane % G);
                for (; e + G < se; e += 2 * G) s += __ldg(x + __ldg(S.ci + e)) + __ldg(x + __ldg(S.ci + e + G));
                if (e < se) s += __ldg(x + __ldg(S.ci + e));
            }
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
            const T t = __shfl_sync(kFull, s, (lane % RPS) * G);
            if (lane / RPS == sub) mine = t;
        }
        if (light) epi(row, end - beg, mine);
    }
}

// ------------------------------------------------------------------ SplitMix64
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t counter) {
    uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform_at(uint64_t seed, uint64_t counter) {
    return (double)(splitmix64_at(seed, counter) >> 11) * (1.0 / 9007199254740992.0);
}

}  // namespace isira
