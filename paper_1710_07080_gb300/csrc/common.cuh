// common.cuh -- device building blocks shared by the iSIRA kernels (sm_103a).
//
//  * deterministic block reductions with a "last block finishes" step: every block
//    writes its partial sums, the block that arrives last adds them in a fixed
//    order, so a reduction needs no second launch and gives the same bits on
//    every run;
//  * a CSR row scheduler for skewed (power-law) degrees (see "row scheduler" below):
//    light rows in tiles of 32 consecutive rows with G lanes per row, longer rows cut
//    into equal-size warp work items;
//  * SplitMix64 (Vigna), the counter-based generator of replacement vectors.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace isira {

constexpr int kThreads = 256;         // threads per CTA for every kernel here
constexpr int kWarps = kThreads / 32;
constexpr int kCMax = 32;             // max locked vectors (deflation rank) supported
constexpr int kMMax = 64;             // max search-space dimension
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
// Grid layout of an SpMV-style launch: [long-row CTAs][light-row CTAs].
//  * light rows (degree <= light_deg) are processed in tiles of 32 consecutive rows by one
//    warp, G lanes per row, so the per-row epilogue runs with one lane per row and coalesced
//    vector accesses;
//  * every longer row is cut into work items of at most kItemNnz stored entries, one warp per
//    item; a row with several items gets its sum from the warp that finishes its last item,
//    which adds the items' partial sums in item order (deterministic) and runs the epilogue.
// The row `skip` (the trimmed vertex, or -1) is never gathered: its epilogue runs from the
// light tiles with a zero sum.
constexpr int kItemNnz = 1024;

// Work units are the items (0 .. n_items-1) followed by the light tiles; setup cuts the unit
// list into n_warps ranges of equal estimated cost (one launch wave), warp w walking units
// [warp_start[w], warp_start[w+1]).  The static partition keeps every reduction deterministic.
constexpr int kTileRowCost = 12;   // estimated cost of one row epilogue, in gathered entries
constexpr int kItemCost = 32;      // fixed cost of one work item

struct RowSched {
    const int64_t* __restrict__ rp;
    const int32_t* __restrict__ ci;
    int64_t n;
    const int32_t* __restrict__ item_row;   // row of each work item (rows ascending)
    const int32_t* __restrict__ item_k;     // position of the item within its row
    void* item_partial;                     // one partial sum per item (type of the launch)
    unsigned* item_count;                   // arrival counters, used at each row's first item
    const int32_t* __restrict__ warp_start; // n_warps + 1 unit boundaries
    int n_items;
    int n_warps;
    int light_deg;
    int hub;                                // x[0:hub] is staged in shared memory (0: none)
    __host__ __device__ int grid() const { return n_warps / kWarps; }
};

// Calls epi(row, degree, sum_{c in N(row)} x[c]) exactly once for every row 0..n-1 (with a
// zero sum for row `skip`).  G = lanes per light row (1, 2, 4, 8, 16 or 32).
// Shared-memory capacity for the hub block of x: 16 KB per CTA.
template <typename T>
struct HubCap { static constexpr int value = 16384 / sizeof(T); };

template <typename T>
__device__ __forceinline__ T gather_x(const T* __restrict__ x, const T* sx, int hub, int32_t c) {
    return c < hub ? sx[c] : __ldg(x + c);
}

template <typename T, int G, class Epi>
__device__ __forceinline__ void for_each_row_gather(const RowSched& S, const T* __restrict__ x, Epi& epi,
                                                    int64_t skip) {
    // With the solver's degree-descending numbering the first `hub` vertices are the hubs most
    // entries point at; their x values are staged once per CTA and read from shared memory.
    __shared__ T sx[HubCap<T>::value];
    const int hub = S.hub < HubCap<T>::value ? S.hub : HubCap<T>::value;
    for (int i = threadIdx.x; i < hub; i += blockDim.x) sx[i] = x[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int u_beg = S.warp_start[gw], u_end = S.warp_start[gw + 1];
    // long rows: finished rows are collected one per lane and their epilogues run 32 at a time,
    // so the epilogue arithmetic uses every lane of the warp
    T* part = static_cast<T*>(S.item_partial);
    int64_t my_row = -1, my_deg = 0;
    T my_sum = 0;
    int nb = 0;                                            // rows collected (warp-uniform)
    const int it_end = u_end < S.n_items ? u_end : S.n_items;
    for (int it = u_beg; it < it_end; ++it) {
        const int64_t r = S.item_row[it];
        if (r == skip) continue;
        const int kpos = S.item_k[it];
        const int64_t rb = S.rp[r], re = S.rp[r + 1];
        const int64_t beg = rb + (int64_t)kpos * kItemNnz;
        const int64_t end = beg + kItemNnz < re ? beg + kItemNnz : re;
        T s0 = 0, s1 = 0;
        for (int64_t e = beg + lane; e < end; e += 256) {
            // a predicated batch of 8 independent index loads, then 8 independent gathers
            int32_t c[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) c[q] = (e + 32 * q < end) ? __ldcs(S.ci + e + 32 * q) : -1;
            T v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = c[q] >= 0 ? gather_x(x, sx, hub, c[q]) : T(0);
            s0 += (v[0] + v[1]) + (v[2] + v[3]);
            s1 += (v[4] + v[5]) + (v[6] + v[7]);
        }
        T s = warp_sum(s0 + s1);
        const int nit = (int)((re - rb + kItemNnz - 1) / kItemNnz);
        int done = 1;
        if (nit > 1) {
            // several items: the warp that finishes the row's last item adds all partials in order
            int last = 0;
            if (lane == 0) {
                const int64_t first = it - kpos;
                part[it] = s;
                __threadfence();
                const unsigned prev = atomicAdd(S.item_count + first, 1u);
                if (prev == (unsigned)(nit - 1)) {
                    __threadfence();
                    T tot = 0;
                    for (int q = 0; q < nit; ++q) tot += __ldcg(part + first + q);
                    S.item_count[first] = 0u;
                    s = tot;
                    last = 1;
                }
            }
            done = __shfl_sync(kFull, last, 0);
            s = __shfl_sync(kFull, s, 0);
        }
        if (done) {
            if (lane == nb) { my_row = r; my_deg = re - rb; my_sum = s; }
            if (++nb == 32) {
                epi(my_row, my_deg, my_sum);
                my_row = -1;
                nb = 0;
            }
        }
    }
    if (my_row >= 0) epi(my_row, my_deg, my_sum);
    // light tiles: 32 consecutive rows, G lanes per row, one lane per row for the epilogue
    constexpr int RPS = 32 / G;                            // rows per sub-pass
    const int t_beg = (u_beg > S.n_items ? u_beg : S.n_items) - S.n_items;
    const int t_end = u_end - S.n_items;
    for (int tile = t_beg; tile < t_end; ++tile) {
        const int64_t row = (int64_t)tile * 32 + lane;
        const bool valid = row < S.n;
        int64_t beg = valid ? S.rp[row] : 0;
        int64_t end = valid ? S.rp[row + 1] : 0;
        const int64_t deg = end - beg;
        const int light = valid && (deg <= S.light_deg || row == skip);
        if (row == skip) end = beg;                        // the skipped row gathers nothing
        T mine = 0;
#pragma unroll
        for (int sub = 0; sub < G; ++sub) {
            const int src = sub * RPS + lane / G;
            const int64_t sb = __shfl_sync(kFull, beg, src);
            const int64_t se = __shfl_sync(kFull, end, src);
            const int sl = __shfl_sync(kFull, light, src);
            T s = 0;
            if (sl) {
                for (int64_t e = sb + (lane % G); e < se; e += 8 * G) {
                    int32_t c[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) c[q] = (e + q * G < se) ? __ldcs(S.ci + e + q * G) : -1;
                    T v[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) v[q] = c[q] >= 0 ? gather_x(x, sx, hub, c[q]) : T(0);
                    s += ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
                }
            }
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
            const T t = __shfl_sync(kFull, s, (lane % RPS) * G);
            if (lane / RPS == sub) mine = t;
        }
        if (light) epi(row, deg, mine);
    }
}

// Epilogue of the plain gather: g[row] = sum over the row (0 for the skipped row).
template <typename T>
struct GatherStore {
    T* g;
    __device__ __forceinline__ void operator()(int64_t r, int64_t, T s) { g[r] = s; }
};

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
