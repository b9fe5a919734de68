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

#include <initializer_list>

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
    int eig_path;          // Rayleigh-Ritz: 0 Jacobi, 1 arrowhead, -1 arrowhead refused (run Jacobi)
    int dev_error;         // bit 0: a gather CTA's staging copy missed its wait limit (set by the
                           // device, cleared by the host at the start of each entry point)
};

// ------------------------------------------------------------------ reductions
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Warp sums of NV per-lane values by recursive halving: at each butterfly level a lane keeps
// half of its values and adds the partner's copy of that half, so a lane spends about 2P adds
// (P = NV rounded up to a power of two) instead of 5 NV.  Afterwards value i's total is in
// slot i % S of lane i / S when P >= 32 (S = P / 32 slots per lane), and in slot 0 of lanes
// i * (32 / P) ... i * (32 / P) + 32 / P - 1 when P < 32.  The summation order is fixed.
template <int NV>
struct MultiShape {
    static constexpr int P = NV <= 1 ? 1 : NV <= 2 ? 2 : NV <= 4 ? 4 : NV <= 8 ? 8 : NV <= 16 ? 16 : NV <= 32 ? 32 : 64;
    static constexpr int S = P >= 32 ? P / 32 : 1;
};

template <typename T, int O, int M, int P>
__device__ __forceinline__ void multi_level(T (&a)[P], int lane) {
    if constexpr (M > 1) {
        const bool up = (lane & O) != 0;
#pragma unroll
        for (int j = 0; j < M / 2; ++j) {
            const T send = up ? a[j] : a[j + M / 2];
            const T keep = up ? a[j + M / 2] : a[j];
            a[j] = keep + __shfl_xor_sync(kFull, send, O);
        }
    } else {
        a[0] += __shfl_xor_sync(kFull, a[0], O);
    }
    if constexpr (O > 1) multi_level<T, O / 2, (M > 1 ? M / 2 : 1), P>(a, lane);
}

template <typename T, int NV>
__device__ __forceinline__ void warp_reduce_multi(const T (&v)[NV], T (&out)[MultiShape<NV>::S]) {
    constexpr int P = MultiShape<NV>::P;
    T a[P];
#pragma unroll
    for (int i = 0; i < P; ++i) a[i] = i < NV ? v[i] : T(0);
    multi_level<T, 16, P, P>(a, threadIdx.x & 31);
#pragma unroll
    for (int q = 0; q < MultiShape<NV>::S; ++q) out[q] = a[q];
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
    constexpr int P = MultiShape<NV>::P, S = MultiShape<NV>::S;
    T out[S];
    warp_reduce_multi<T, NV>(v, out);
    if constexpr (P >= 32) {
#pragma unroll
        for (int q = 0; q < S; ++q) {
            const int i = lane * S + q;
            if (i < nv && i < NV) red[w][i] = out[q];
        }
    } else {
        const int i = lane / (32 / P);
        if (lane % (32 / P) == 0 && i < nv && i < NV) red[w][i] = out[0];
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
// Work of an SpMV-style gather launch, in units:
//  * every row longer than light_deg is cut into work items of at most kItemNnz stored
//    entries, summed by one warp; a row with several items gets its sum from the warp that
//    finishes its last item, which adds the items' partial sums in item order (deterministic);
//  * light rows (degree <= light_deg) are processed in tiles of 32 consecutive rows by one
//    warp, G lanes per row, so the per-row epilogue runs with one lane per row.
// The row `skip` (the trimmed vertex, or -1) is never gathered: its epilogue runs from the
// light tiles with a zero sum.
constexpr int kItemNnz = 1024;

// Work units are the items (0 .. n_items-1) followed by the light tiles.  By default warps take
// units from a device counter (dynamic distribution); alternatively setup cuts the unit list
// into n_warps ranges of equal estimated cost, warp w walking [warp_start[w], warp_start[w+1]).
// Either way every row's sum is computed in the same order.
constexpr int kUnitChunk = 2;      // default units a warp takes at a time (dynamic distribution)
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
    int hub;                                // x[0:hub] may be staged in shared memory (0: none)
    int hub_bytes;                          // dynamic shared memory of a gather CTA for that block
    int tpb;                                // threads per gather CTA (kThreads or kBigBlock)
    int ci_vec;                             // ci is 16-byte aligned and padded to a multiple of 4
                                            // entries: 128-bit index loads
    int dyn;                                // 1: dynamic unit distribution through sched
    unsigned* sched;                        // [next unit, warps finished], zero between launches
    int chunk;                              // units per take (1..32)
    unsigned* hub_timeouts;                 // CTAs whose staging copy missed the wait limit
    int* err;                               // device alias of HostStatus::dev_error (may be null)
    // sliced ELL copy of the light rows (see build_sell): with sell = 1 the rows [light0, n) are
    // gathered from sell_ci in slices of 32 rows instead of CSR tiles, and rows below light0 are
    // exactly the long rows (the degree-descending numbering puts them first)
    const int32_t* __restrict__ sell_ci;
    const int64_t* __restrict__ sell_off;   // n_slices + 1 offsets (multiples of 32)
    int64_t light0;
    int n_slices;
    int sell;
    // weighted Laplacian (all null: unit weights): edge weights aligned with ci and with sell_ci
    // (0 in the padding), in FP32 and FP64, and the weighted degrees (ld entries)
    const float* __restrict__ wf;
    const double* __restrict__ wd;
    const float* __restrict__ swf;
    const double* __restrict__ swd;
    const float* __restrict__ degwf;
    const double* __restrict__ degwd;
    template <typename T> __host__ __device__ const T* wts() const;
    template <typename T> __host__ __device__ const T* swts() const;
    template <typename T> __host__ __device__ const T* degw() const;
    __host__ __device__ int grid() const { return n_warps / (tpb / 32); }
    __host__ __device__ int n_units() const {
        return n_items + (sell ? n_slices : (int)((n + 31) / 32));
    }
};

template <> __host__ __device__ inline const float* RowSched::wts<float>() const { return wf; }
template <> __host__ __device__ inline const double* RowSched::wts<double>() const { return wd; }
template <> __host__ __device__ inline const float* RowSched::swts<float>() const { return swf; }
template <> __host__ __device__ inline const double* RowSched::swts<double>() const { return swd; }
template <> __host__ __device__ inline const float* RowSched::degw<float>() const { return degwf; }
template <> __host__ __device__ inline const double* RowSched::degw<double>() const { return degwd; }

// degree of row r in precision T: the weighted degree when the graph has weights
template <typename T>
__device__ __forceinline__ T row_degree(const RowSched& S, int64_t r) {
    const T* dw = S.degw<T>();
    return dw ? dw[r] : (T)(S.rp[r + 1] - S.rp[r]);
}

constexpr int kBigBlock = 1024;             // one gather CTA per SM holding a large hub block
constexpr int kDefaultHubBytes = 192 * 1024;  // hub block of a 1024-thread gather CTA

// Calls F(G, TPB) with compile-time lanes per light row and threads per gather CTA.
#define ISIRA_GATHER_DISPATCH(lanes, tpb, F) \
    do {                                     \
        if ((tpb) == kBigBlock) {            \
            switch (lanes) {                 \
                case 1: F(1, kBigBlock); break; \
                case 2: F(2, kBigBlock); break; \
                case 4: F(4, kBigBlock); break; \
                case 8: F(8, kBigBlock); break; \
                case 16: F(16, kBigBlock); break; \
                default: F(32, kBigBlock); break; \
            }                                \
        } else {                             \
            switch (lanes) {                 \
                case 1: F(1, kThreads); break; \
                case 2: F(2, kThreads); break; \
                case 4: F(4, kThreads); break; \
                case 8: F(8, kThreads); break; \
                case 16: F(16, kThreads); break; \
                default: F(32, kThreads); break; \
            }                                \
        }                                    \
    } while (0)

__device__ __forceinline__ unsigned atomic_add_acq_rel(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

template <typename T>
__device__ __forceinline__ T gather_x(const T* __restrict__ x, const T* sx, int hub, int32_t c) {
    return c < hub ? sx[c] : __ldg(x + c);
}

// ------------------------------------------------------------------ hub staging (TMA bulk copy)
// The dynamic shared memory of a gather launch holds the hub block x[0:hub).
extern __shared__ __align__(128) unsigned char g_dyn_smem[];

constexpr int kHubWaitPolls = 1 << 20;      // x ~64 ns: a bound far above the copy's microseconds
constexpr int kHubDrainPolls = 1 << 24;     // second bound, for a copy still in flight after a timeout

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity, int polls) {
    for (int i = 0; i < polls; ++i) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
        if (i >= 8) __nanosleep(64);
    }
    return false;
}

// Copies x[0:hub) into shared memory with one bulk asynchronous copy (the tensor memory
// accelerator) that an mbarrier tracks; returns the number of staged entries (a multiple of
// 16 bytes).  Should the copy not land within the wait limit, the CTA counts the event, sets
// bit 0 of the host-visible error word (the solve then fails with a device-timeout status),
// waits once more, with a longer but still finite limit, for the copy in flight, so that it
// does not leave while the copy can still write its shared memory, and returns -1: the CTA then
// gathers nothing.
template <typename T>
__device__ __forceinline__ int stage_hub(const RowSched& S, const T* __restrict__ x, T* sx) {
    constexpr int kUnit = 16 / (int)sizeof(T);
    int hub = S.hub < S.hub_bytes / (int)sizeof(T) ? S.hub : S.hub_bytes / (int)sizeof(T);
    hub = hub / kUnit * kUnit;
    if (hub <= 0) return 0;
    if ((reinterpret_cast<uintptr_t>(x) & 15u) != 0) {
        for (int i = threadIdx.x; i < hub; i += blockDim.x) sx[i] = x[i];
        __syncthreads();
        return hub;
    }
    __shared__ __align__(8) unsigned long long bar;
    const unsigned bar_a = smem_u32(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned bytes = (unsigned)hub * (unsigned)sizeof(T);
        asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}"
                     :: "r"(bar_a), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     :: "r"(smem_u32(sx)), "l"(x), "r"(bytes), "r"(bar_a) : "memory");
    }
    if (__syncthreads_and(mbar_wait_bounded(bar_a, 0, kHubWaitPolls))) return hub;
    if (threadIdx.x == 0) {
        atomicAdd(S.hub_timeouts, 1u);
        if (S.err) atomicOr_system(S.err, 1);
    }
    (void)__syncthreads_and(mbar_wait_bounded(bar_a, 0, kHubDrainPolls));
    return -1;
}

// Partial sum over the stored entries [beg, end) of ci taken by sub-lane j of a group of W lanes.
// Each pass loads a batch of independent indices first and then issues all their gathers, so a
// lane keeps a whole batch of loads in flight.  The summation order depends only on (beg, end,
// W), never on the launch shape.
//  * vector form (ci 16-byte aligned and padded): sub-lane j reads the 128-bit chunks starting at
//    (beg rounded down to 4) + 4j + 4W*u, u < NB, and masks the entries outside [beg, end);
//  * scalar form: sub-lane j reads entries beg + j + W*u, u < 8 (u < 4 in a short last pass).
template <typename T, int W, int NB>
__device__ __forceinline__ T seg_sum_vec(const int32_t* __restrict__ ci, const T* __restrict__ x, const T* sx,
                                         int hub, int64_t beg, int64_t end, int j) {
    T s0 = 0, s1 = 0;
    for (int64_t base = (beg & ~(int64_t)3) + 4 * j; base < end; base += 4 * W * NB) {
        int4 q[NB];
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int64_t p = base + 4 * W * u;
            q[u] = p < end ? __ldcs(reinterpret_cast<const int4*>(ci + p)) : make_int4(0, 0, 0, 0);
        }
        T v[4 * NB];
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int64_t p = base + 4 * W * u;
            const int32_t cc[4] = {q[u].x, q[u].y, q[u].z, q[u].w};
#pragma unroll
            for (int w = 0; w < 4; ++w)
                v[4 * u + w] = (p + w >= beg && p + w < end) ? gather_x(x, sx, hub, cc[w]) : T(0);
        }
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const T t = (v[4 * u] + v[4 * u + 1]) + (v[4 * u + 2] + v[4 * u + 3]);
            if (u & 1) s1 += t; else s0 += t;
        }
    }
    return s0 + s1;
}

// One pass of the scalar form: sub-lane j takes entries e + W*q, q < Q (e = pass base + j); with
// weights (wt not null) every gathered value is scaled by its edge's weight.
template <typename T, int W, int Q>
__device__ __forceinline__ void scalar_pass(const int32_t* __restrict__ ci, const T* __restrict__ wt,
                                            const T* __restrict__ x, const T* sx, int hub, int64_t e, int64_t end,
                                            T& s0, T& s1) {
    int32_t c[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) c[q] = (e + W * q < end) ? __ldcs(ci + e + W * q) : -1;
    T v[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) v[q] = c[q] >= 0 ? gather_x(x, sx, hub, c[q]) : T(0);
    if (wt) {
#pragma unroll
        for (int q = 0; q < Q; ++q) v[q] *= c[q] >= 0 ? __ldcs(wt + e + W * q) : T(0);
    }
    if constexpr (Q == 8) {
        s0 += (v[0] + v[1]) + (v[2] + v[3]);
        s1 += (v[4] + v[5]) + (v[6] + v[7]);
    } else {
        s0 += v[0] + v[1];
        s1 += v[2] + v[3];
    }
}

// Whole-warp segments (W = 32) end with a half-width pass when at most 4W entries remain, so
// the tail adds fewer padding zeros.
template <typename T, int W>
__device__ __forceinline__ T seg_sum_scalar(const int32_t* __restrict__ ci, const T* __restrict__ wt,
                                            const T* __restrict__ x, const T* sx, int hub, int64_t beg, int64_t end,
                                            int j) {
    T s0 = 0, s1 = 0;
    for (int64_t base = beg; base < end;) {
        if (W == 32 && end - base <= 4 * W) {
            scalar_pass<T, W, 4>(ci, wt, x, sx, hub, base + j, end, s0, s1);
            base += 4 * W;
        } else {
            scalar_pass<T, W, 8>(ci, wt, x, sx, hub, base + j, end, s0, s1);
            base += 8 * W;
        }
    }
    return s0 + s1;
}

// 128-bit index chunks per lane and pass: 16 indices in flight per lane for FP32, 8 for FP64
template <typename T>
struct VecChunks { static constexpr int value = sizeof(T) == 4 ? 4 : 2; };

template <typename T, int W>
__device__ __forceinline__ T seg_sum(const RowSched& S, const T* __restrict__ x, const T* sx, int hub, int64_t beg,
                                     int64_t end, int j) {
    // the 128-bit index path is for unweighted graphs (the solver turns it off with weights)
    return S.ci_vec ? seg_sum_vec<T, W, VecChunks<T>::value>(S.ci, x, sx, hub, beg, end, j)
                    : seg_sum_scalar<T, W>(S.ci, S.wts<T>(), x, sx, hub, beg, end, j);
}

// Calls epi(row, degree, sum_{c in N(row)} x[c]) exactly once for every row 0..n-1 (with a
// zero sum for row `skip`).  G = lanes per light row (1, 2, 4, 8, 16 or 32).
// Launched with S.grid() CTAs of S.tpb threads and S.hub_bytes of dynamic shared memory.
template <typename T, int G, class Epi>
__device__ __forceinline__ void for_each_row_gather(const RowSched& S, const T* __restrict__ x, Epi& epi,
                                                    int64_t skip) {
    // With the solver's degree-descending numbering the first `hub` vertices are the hubs most
    // entries point at; their x values are staged once per CTA and read from shared memory.
    T* sx = reinterpret_cast<T*>(g_dyn_smem);
    const int hub = stage_hub<T>(S, x, sx);
    const int lane = threadIdx.x & 31;
    // dynamic distribution: every warp reports once that it has finished taking units; the last
    // one resets the counters for the next launch
    auto finish_dyn = [&]() {
        if (lane == 0) {
            const unsigned n_warps = gridDim.x * (blockDim.x >> 5);
            __threadfence();
            if (atomicAdd(S.sched + 1, 1u) == n_warps - 1) {
                S.sched[0] = 0u;
                S.sched[1] = 0u;
            }
        }
    };
    if (hub < 0) {                      // staging timed out (reported): this CTA takes no units
        if (S.dyn) finish_dyn();
        return;
    }
    // long rows: finished rows are collected one per lane and their epilogues run 32 at a time,
    // so the epilogue arithmetic uses every lane of the warp
    T* part = static_cast<T*>(S.item_partial);
    int64_t my_row = -1, my_deg = 0;
    T my_sum = 0;
    int nb = 0;                                            // rows collected (warp-uniform)
    // item u's header (row, position in the row, row extent); loaded lane-parallel for a chunk
    int h_row = -1, h_k = 0;
    int64_t h_rb = 0, h_re = 0;
    auto load_headers = [&](int u0, int u1) {
        const int u = u0 + lane;
        h_row = -1;
        if (u < u1 && u < S.n_items) {
            h_row = S.item_row[u];
            h_k = S.item_k[u];
            h_rb = S.rp[h_row];
            h_re = S.rp[h_row + 1];
        }
    };
    // per-lane partial sum of the item whose header sits in lane j (zero for the skipped row)
    auto item_partial = [&](int j) -> T {
        const int64_t r = __shfl_sync(kFull, h_row, j);
        const int kpos = __shfl_sync(kFull, h_k, j);
        const int64_t rb = __shfl_sync(kFull, h_rb, j), re = __shfl_sync(kFull, h_re, j);
        if (r == skip) return T(0);
        const int64_t beg = rb + (int64_t)kpos * kItemNnz;
        const int64_t end = beg + kItemNnz < re ? beg + kItemNnz : re;
        return seg_sum<T, 32>(S, x, sx, hub, beg, end, lane);
    };
    // item it (header in lane j) with its warp total s: combine a split row, collect the row
    auto item_finish = [&](int it, int j, T s) {
        const int64_t r = __shfl_sync(kFull, h_row, j);
        if (r == skip) return;
        const int kpos = __shfl_sync(kFull, h_k, j);
        const int64_t rb = __shfl_sync(kFull, h_rb, j), re = __shfl_sync(kFull, h_re, j);
        const int nit = (int)((re - rb + kItemNnz - 1) / kItemNnz);
        int done = 1;
        if (nit > 1) {
            // several items: the warp that finishes the row's last item adds all partials in order
            int last = 0;
            if (lane == 0) {
                const int64_t first = it - kpos;
                part[it] = s;
                // one acquire-release add: publishes this partial and, in the last arriver,
                // makes every other item's partial visible (no full fences)
                const unsigned prev = atomic_add_acq_rel(S.item_count + first, 1u);
                if (prev == (unsigned)(nit - 1)) {
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
    };
    auto do_item = [&](int it, int j) { item_finish(it, j, warp_sum(item_partial(j))); };
    // two items share one butterfly reduction; it applies the same lane pairs in the same order
    // as two warp_sum calls, so the totals are bit-identical to reducing them one by one
    auto do_item_pair = [&](int it, int j) {
        const T v[2] = {item_partial(j), item_partial(j + 1)};
        T out[1];
        warp_reduce_multi<T, 2>(v, out);
        const T s0 = __shfl_sync(kFull, out[0], 0), s1 = __shfl_sync(kFull, out[0], 16);
        item_finish(it, j, s0);
        item_finish(it + 1, j + 1, s1);
    };
    // light tiles: 32 consecutive rows, G lanes per row, one lane per row for the epilogue
    constexpr int RPS = 32 / G;                            // rows per sub-pass
    auto do_tile = [&](int tile) {
        const int64_t row = (int64_t)tile * 32 + lane;
        const bool valid = row < S.n;
        int64_t beg = valid ? S.rp[row] : 0;
        int64_t end = valid ? S.rp[row + 1] : 0;
        const int64_t deg = end - beg;
        const int light = valid && (deg <= S.light_deg || row == skip);
        if (row == skip) end = beg;                        // the skipped row gathers nothing
        if (!__any_sync(kFull, light)) return;
        T mine = 0;
#pragma unroll
        for (int sub = 0; sub < G; ++sub) {
            const int src = sub * RPS + lane / G;
            const int64_t sb = __shfl_sync(kFull, beg, src);
            const int64_t se = __shfl_sync(kFull, end, src);
            const int sl = __shfl_sync(kFull, light, src);
            T s = sl ? seg_sum<T, G>(S, x, sx, hub, sb, se, lane % G) : T(0);
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
            const T t = __shfl_sync(kFull, s, (lane % RPS) * G);
            if (lane / RPS == sub) mine = t;
        }
        if (light) epi(row, deg, mine);
    };
    // sliced light rows: one lane per row, two slices at a time so that each lane keeps eight index
    // loads (four per row) in flight; a lane adds its row's entries in slice order
    const T* __restrict__ sw = S.swts<T>();
    auto do_slices = [&](int s0, int s1) {
        for (int sa = s0; sa < s1; sa += 2) {
            const bool two = sa + 1 < s1;
            const int64_t ra = S.light0 + (int64_t)sa * 32 + lane;
            const int64_t rb = ra + 32;
            const int64_t oa = S.sell_off[sa], ea = S.sell_off[sa + 1];
            const int64_t ob = two ? ea : 0, eb = two ? S.sell_off[sa + 2] : 0;
            const int wa = (int)((ea - oa) >> 5), wb = (int)((eb - ob) >> 5);
            const int w = wa > wb ? wa : wb;
            T s_a = 0, s_b = 0;
            for (int q = 0; q < w; q += 4) {
                int32_t ia[4], ib[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    ia[u] = q + u < wa ? __ldcs(S.sell_ci + oa + (int64_t)(q + u) * 32 + lane) : -1;
                    ib[u] = q + u < wb ? __ldcs(S.sell_ci + ob + (int64_t)(q + u) * 32 + lane) : -1;
                }
                T va[4], vb[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    va[u] = ia[u] >= 0 ? gather_x(x, sx, hub, ia[u]) : T(0);
                    vb[u] = ib[u] >= 0 ? gather_x(x, sx, hub, ib[u]) : T(0);
                }
                if (sw) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        va[u] *= ia[u] >= 0 ? __ldcs(sw + oa + (int64_t)(q + u) * 32 + lane) : T(0);
                        vb[u] *= ib[u] >= 0 ? __ldcs(sw + ob + (int64_t)(q + u) * 32 + lane) : T(0);
                    }
                }
                s_a += (va[0] + va[1]) + (va[2] + va[3]);
                s_b += (vb[0] + vb[1]) + (vb[2] + vb[3]);
            }
            if (ra < S.n) epi(ra, 0, ra == skip ? T(0) : s_a);
            if (two && rb < S.n) epi(rb, 0, rb == skip ? T(0) : s_b);
        }
    };
    auto do_range = [&](int u0, int u1) {             // u1 - u0 <= 32
        if (u0 < S.n_items) load_headers(u0, u1);
        for (int u = u0; u < u1;) {
            if (u + 1 < u1 && u + 1 < S.n_items) {
                do_item_pair(u, u - u0);
                u += 2;
            } else if (u >= S.n_items && S.sell) {
                do_slices(u - S.n_items, u1 - S.n_items);
                break;
            } else {
                if (u < S.n_items) do_item(u, u - u0); else do_tile(u - S.n_items);
                u += 1;
            }
        }
    };
    // a trimmed long row is skipped by its items; with slices no tile writes its zero sum
    if (S.sell && skip >= 0 && skip < S.light0 && blockIdx.x == 0 && threadIdx.x == 0) epi(skip, 0, T(0));
    const int n_units = S.n_units();
    if (S.dyn) {
        // dynamic: warps take chunks of S.chunk units from a counter; the last warp to finish
        // resets it for the next launch.  Which warp takes a unit never changes its sum.  With
        // sliced light rows only the long-row items are taken this way: the slices are many and
        // of nearly equal cost, so the warps walk them in a fixed grid-strided order instead of
        // contending for one counter.
        const int n_dyn = S.sell ? S.n_items : n_units;
        for (;;) {
            int u0 = 0;
            if (lane == 0) u0 = (int)atomicAdd(S.sched, (unsigned)S.chunk);
            u0 = __shfl_sync(kFull, u0, 0);
            if (u0 >= n_dyn) break;               // the failing take precedes the fence below
            do_range(u0, u0 + S.chunk < n_dyn ? u0 + S.chunk : n_dyn);
        }
        if (S.sell) {
            const int gw = blockIdx.x * (int)(blockDim.x >> 5) + (threadIdx.x >> 5);
            const int nw = gridDim.x * (int)(blockDim.x >> 5);
            for (int s0 = 2 * gw; s0 < S.n_slices; s0 += 2 * nw) do_slices(s0, s0 + 2 < S.n_slices ? s0 + 2 : S.n_slices);
        }
        finish_dyn();
    } else {
        const int gw = blockIdx.x * (int)(blockDim.x >> 5) + (threadIdx.x >> 5);
        const int u_beg = S.warp_start[gw], u_end = S.warp_start[gw + 1];
        for (int u = u_beg; u < u_end; u += 32) do_range(u, u + 32 < u_end ? u + 32 : u_end);
    }
    if (my_row >= 0) epi(my_row, my_deg, my_sum);
}

// Gather for graphs without long rows (every row in the sliced copy, no work items): warp w walks
// the slices w, w + W, ... (W warps in the grid), one lane per row, with the next slice's offsets
// loaded ahead and eight independent index loads per pass.  Few registers, so a full SM of warps
// keeps loads in flight.  A row's entries are added in slice order in two interleaved partial
// sums, whatever the launch shape (the result does not depend on the grid).
template <typename T, class Epi>
__device__ __forceinline__ void slices_only_gather(const RowSched& S, const T* __restrict__ x, Epi& epi, int64_t skip) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (int)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nw = gridDim.x * (int)(blockDim.x >> 5);
    const T* __restrict__ sw = S.swts<T>();
    int64_t o0 = 0, o1 = 0;
    if (gw < S.n_slices) { o0 = S.sell_off[gw]; o1 = S.sell_off[gw + 1]; }
    for (int s = gw; s < S.n_slices; s += nw) {
        const int64_t oa = o0;
        const int wa = (int)((o1 - o0) >> 5);
        if (s + nw < S.n_slices) { o0 = S.sell_off[s + nw]; o1 = S.sell_off[s + nw + 1]; }   // next slice
        T s0 = 0, s1 = 0;
        for (int q = 0; q < wa; q += 8) {
            int32_t ia[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) ia[u] = q + u < wa ? __ldcs(S.sell_ci + oa + (int64_t)(q + u) * 32 + lane) : -1;
            T va[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) va[u] = ia[u] >= 0 ? __ldg(x + ia[u]) : T(0);
            if (sw) {
#pragma unroll
                for (int u = 0; u < 8; ++u) va[u] *= ia[u] >= 0 ? __ldcs(sw + oa + (int64_t)(q + u) * 32 + lane) : T(0);
            }
            s0 += (va[0] + va[1]) + (va[2] + va[3]);
            s1 += (va[4] + va[5]) + (va[6] + va[7]);
        }
        const int64_t row = S.light0 + (int64_t)s * 32 + lane;
        if (row < S.n) epi(row, 0, row == skip ? T(0) : s0 + s1);
    }
    if (skip >= 0 && skip < S.light0 && blockIdx.x == 0 && threadIdx.x == 0) epi(skip, 0, T(0));
}

// The slices-only kernels are used when every row is sliced: relabelling on, sliced copy on, no
// work items.
__host__ __device__ inline bool slices_only(const RowSched& S) { return S.sell && S.n_items == 0; }
constexpr int kSliceBlocksPerSM = 8;

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
