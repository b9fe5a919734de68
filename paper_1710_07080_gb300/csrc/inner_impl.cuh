// inner_impl.cuh -- the inexact inner solve of Algorithm 2 on the GPU.
//
// Operator (Theorem 2.6, Eq. 2.14), applied in n-space with the trimmed entry i
// pinned to zero (x_i = 0 in every Krylov vector, y_i = 0):
//   (Mh x)_r = (deg_r - sigma) x_r - sum_{c in N(r)} x_c + (sigma/n) 1^T x + delta (Vh (Vh^T x))_r.
// Preconditioner (Remark 3.2 with a diagonal Mh_sigma, Eq. 3.6 for the deflation):
//   P = D + delta Vh Vh^T,  D = diag(max(deg_r - sigma, deg_r / 2)),
//   P^{-1} y = D^{-1} (y - Vh t),  t = C^{-1} Vh^T D^{-1} y,  C = delta^{-1} I + Vh^T D^{-1} Vh.
// Solver: preconditioned MINRES (Paige & Saunders 1975).  One iteration k is two
// launches:
//   phase 1: the SpMV with the whole row epilogue fused in: y1 = Mh v_k - (beta_k /
//            beta_{k-1}) r_{k-1}, with r_{k-1} = P z_{k-1} rebuilt from z_{k-1} (so the
//            Lanczos residual vectors are never stored), the deferred solution update
//            of iteration k-1 (w, x), and the reductions alpha_k = v_k^T y1 and
//            Vh^T D^{-1} y1;
//   phase 2: y = y1 - (alpha_k / beta_k) r_k, z_{k+1} = P^{-1} y (SMW), and the
//            reductions y^T z (beta_{k+1}^2), 1^T z, Vh^T z; its last block runs the
//            Givens recurrence and the stopping test.
// Vectors per row and iteration: z_k (gathered), z_{k-1}, Y, three rotating w
// buffers, x, and c columns of Vh.
#pragma once
#include <mutex>
#include <unordered_map>

#include "internal.h"

namespace isira {

template <typename T>
__device__ __forceinline__ T precond_diag(T deg, T sigma) {
    T m = deg - sigma;
    T h = deg * T(0.5);
    return m < h ? h : m;
}

// 1/D_r: from the FP64 array the prep kernel filled, or computed (FP32 mode)
template <typename T>
__device__ __forceinline__ T inv_diag(const T* dinv, int64_t r, T D) {
    return dinv ? dinv[r] : T(1) / D;
}

template <typename T>
__device__ __forceinline__ T* wbuf(const InnerArgs<T>& a, int j) {
    int r = j % 3;
    return r == 0 ? a.wb0 : (r == 1 ? a.wb1 : a.wb2);
}

// ------------------------------------------------------------------ vector access
// The row kernels move VN = 16 / sizeof(T) consecutive rows per thread with 16-byte loads and
// stores.  Every n-vector has ld >= n rows (ld a multiple of 32), so a vector access never leaves
// its buffer; rows >= n and the trimmed row are masked with selects (padding may hold anything).
template <typename T> struct Vec;
template <> struct Vec<float> { static constexpr int N = 4; using V = float4; using I = int4; };
template <> struct Vec<double> { static constexpr int N = 2; using V = double2; using I = int2; };

template <typename T>
__device__ __forceinline__ void vld(const T* __restrict__ p, T (&v)[Vec<T>::N]) {
    const typename Vec<T>::V q = __ldg(reinterpret_cast<const typename Vec<T>::V*>(p));
    if constexpr (Vec<T>::N == 4) { v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w; }
    else { v[0] = q.x; v[1] = q.y; }
}

// plain (coherent) load for buffers the kernel also writes
template <typename T>
__device__ __forceinline__ void vld_rw(const T* p, T (&v)[Vec<T>::N]) {
    const typename Vec<T>::V q = *reinterpret_cast<const typename Vec<T>::V*>(p);
    if constexpr (Vec<T>::N == 4) { v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w; }
    else { v[0] = q.x; v[1] = q.y; }
}

template <typename T>
__device__ __forceinline__ void vst(T* p, const T (&v)[Vec<T>::N]) {
    typename Vec<T>::V q;
    if constexpr (Vec<T>::N == 4) { q.x = v[0]; q.y = v[1]; q.z = v[2]; q.w = v[3]; }
    else { q.x = v[0]; q.y = v[1]; }
    *reinterpret_cast<typename Vec<T>::V*>(p) = q;
}

template <typename T>
__device__ __forceinline__ void vld_deg(const int32_t* __restrict__ p, int (&v)[Vec<T>::N]) {
    const typename Vec<T>::I q = __ldg(reinterpret_cast<const typename Vec<T>::I*>(p));
    if constexpr (Vec<T>::N == 4) { v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w; }
    else { v[0] = q.x; v[1] = q.y; }
}

// degrees of VN consecutive rows in precision T: the weighted degrees when the graph has weights,
// else the int32 degree array
template <typename T>
__device__ __forceinline__ void vld_degree(const InnerArgs<T>& a, int64_t r0, T (&d)[Vec<T>::N]) {
    const T* dw = a.rs.template degw<T>();
    if (dw) {
        vld(dw + r0, d);
    } else {
        int dg[Vec<T>::N];
        vld_deg<T>(a.deg + r0, dg);
#pragma unroll
        for (int e = 0; e < Vec<T>::N; ++e) d[e] = (T)dg[e];
    }
}

// deflation columns the per-thread accumulators of a bucket hold: c <= kCMax - 1 in every solve
template <int NC>
struct Ncols { static constexpr int value = NC < kCMax ? NC : kCMax - 1; };

// ------------------------------------------------------------------ MINRES scalar step
// Last CTA of phase 2 (one thread): beta_{k+1} = sqrt(bb) with bb = r_{k+1}^T P^{-1} r_{k+1}, then the
// Givens rotation of column k of the Lanczos tridiagonal matrix (Paige & Saunders 1975), the
// coefficients of the deferred w/x update, the stopping test phibar <= tau beta_1, and the host
// status.  init: the first preconditioned vector (k = 0).  ssum = 1^T z_{k+1}.
template <typename T>
__device__ __forceinline__ void minres_step(const InnerArgs<T>& a, InnerState<T>* st, T bb, T ssum, int init, int k,
                                            cudaGraphConditionalHandle cond, int has_cond) {
    const T bnew = bb > T(0) ? sqrt(bb) : T(0);
    int done;
    if (init) {
        st->beta1 = bnew;
        st->beta = bnew;
        st->oldb = T(0);
        st->phibar = bnew;
        st->cs = T(-1);
        st->sn = T(0);
        st->dbar = T(0);
        st->epsln = T(0);
        st->itn = 0;
        st->pending = 0;
        done = !(bnew > T(0));
    } else {
        const T alpha = st->alpha;
        const T cs = st->cs, sn = st->sn, dbar = st->dbar;
        const T oldeps = st->epsln;
        const T dlt = cs * dbar + sn * alpha;
        const T gbar = sn * dbar - cs * alpha;
        const T epsln = sn * bnew;
        const T dbar2 = -cs * bnew;
        T gamma = sqrt(gbar * gbar + bnew * bnew);
        if (!(gamma > T(0))) gamma = T(1e-30);
        const T cs2 = gbar / gamma, sn2 = bnew / gamma;
        const T phi = cs2 * st->phibar;
        const T phibar = sn2 * st->phibar;
        st->w_oldeps = oldeps;
        st->w_dlt = dlt;
        st->w_inv_gamma = T(1) / gamma;
        st->w_phi = phi;
        st->cs = cs2;
        st->sn = sn2;
        st->dbar = dbar2;
        st->epsln = epsln;
        st->phibar = phibar;
        st->oldb = st->beta;
        st->beta = bnew;
        st->itn = k;
        st->pending = 1;
        done = (phibar <= a.tau * st->beta1) || (k >= a.max_it) || !(bnew > T(0));
    }
    st->s_cur = ssum;
    st->done = done;
    if (has_cond) cudaGraphSetConditional(cond, done ? 0u : 1u);
    a.hs->inner_done = done;
    a.hs->inner_iters = st->itn;
    a.hs->inner_relres = st->beta1 > T(0) ? (double)(st->phibar / st->beta1) : 0.0;
}

// ------------------------------------------------------------------ phase 1
// Row epilogue of the operator from the gathered neighbour sums, one pass over the rows:
//   y'_r = ((deg_r - sigma) z_r - g_r + (sigma/n) s) / beta_k - (beta_k / beta_{k-1}) D_r zp_r   (r != trim)
// i.e. Mh v_k - (beta_k/beta_{k-1}) P z_{k-1} without their deflation parts, which phase 2 adds
// as Vh u1 (so phase 1 reads each Vh entry once and uses it at once).  Also the deferred w/x
// update of iteration k-1, and the reductions
//   alpha' = v_k^T y',   a_t = (Vh^T D^{-1} y')_t,   g_t = (Vh^T z_k)_t.
// The last CTA turns them into u1 = delta (g / beta_k - (beta_k / beta_{k-1}) g_prev),
// alpha_k = alpha' + (g / beta_k)^T u1, and phase 2's SMW coefficient
//   tv = C^{-1} Vh^T D^{-1} y,  Vh^T D^{-1} y = a + G u1 - (alpha_k / beta_k)(g + delta G g),
// with G = Vh^T D^{-1} Vh (so Vh^T D^{-1} (Vh u1) needs no pass over Vh).

// Gather of phase 1: g_r = sum_{c in N(r)} z_k[c] (the trimmed row gathers nothing).  Only this
// kernel walks the CSR; it keeps few registers so many warps keep loads in flight.
template <typename T, int G, int TPB>
__global__ void __launch_bounds__(TPB, TPB == kThreads ? 4 : 1) k_phase1_gather(InnerArgs<T> a) {
    const InnerState<T>* st = a.st;
    if (st->done) return;
    const int itn = st->itn;                 // iteration k = itn + 1 gathers z_k = z[itn & 1]
    const T* zc = (itn & 1) ? a.z1 : a.z0;
    GatherStore<T> epi{a.gsum};
    for_each_row_gather<T, G>(a.rs, zc, epi, a.trim);
}

// Partial sums of one CTA, already reduced over the CTA, to the per-block slots; returns true in
// the CTA that arrives last (all partials of all blocks are visible to it then).
template <typename T>
__device__ __forceinline__ bool block_values_arrive(const T* bv, int nv, T* partial, int pstride,
                                                    unsigned* counter) {
    __shared__ int last;
    for (int i = threadIdx.x; i < nv; i += blockDim.x) partial[(size_t)i * pstride + blockIdx.x] = bv[i];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    return last != 0;
}

// Rows are taken in tiles of kThreads * VN; after a tile's row arithmetic, z_k and D^{-1} y' of the
// tile sit in shared memory and every warp reads whole columns of Vh for the tile (coalesced
// 16-byte loads), so the deflation reductions need a few registers per warp, whatever c is.
template <typename T, int NC>
__global__ void __launch_bounds__(kThreads) k_phase1(InnerArgs<T> a) {
    constexpr int VN = Vec<T>::N;
    constexpr int NE = Ncols<NC>::value;
    constexpr int NA = 1 + 2 * NE;
    constexpr int TILE = kThreads * VN;
    constexpr int QW = (NE + kWarps - 1) / kWarps;          // columns per warp
    InnerState<T>* st = a.st;
    if (st->done) return;
    const int k = st->itn + 1;
    const int c = st->p_c;
    const T sigma = st->p_sigma;
    const T* __restrict__ zc = ((k - 1) & 1) ? a.z1 : a.z0;
    const T* __restrict__ zp = (k & 1) ? a.z1 : a.z0;
    const T beta = st->beta, oldb = st->oldb;
    const T inv_beta = T(1) / beta;
    const bool has_prev = k >= 2;
    const T cprev = has_prev ? beta / oldb : T(0);
    const T inv_oldb = has_prev ? T(1) / oldb : T(0);
    const T s_term = st->p_sig_n * st->s_cur;
    const int j = k - 1;                    // iteration whose w/x update is deferred to here
    const T* __restrict__ wo2 = wbuf(a, j + 1);   // w_{j-2}
    const T* __restrict__ wo1 = wbuf(a, j + 2);   // w_{j-1}
    T* __restrict__ wn = wbuf(a, j);              // w_j
    const T oldeps = st->w_oldeps, dlt = st->w_dlt, inv_gamma = st->w_inv_gamma, phi = st->w_phi;
    __shared__ __align__(16) T sz[NE > 0 ? TILE : 1];
    __shared__ __align__(16) T syd[NE > 0 ? TILE : 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T acc0 = T(0);
    T ca[QW > 0 ? QW : 1], cg[QW > 0 ? QW : 1];
#pragma unroll
    for (int q = 0; q < (QW > 0 ? QW : 1); ++q) { ca[q] = T(0); cg[q] = T(0); }
    const int64_t n = a.rs.n, trim = a.trim;
    const T* __restrict__ Vt = a.Vt;
    for (int64_t t0 = (int64_t)blockIdx.x * TILE; t0 < n; t0 += (int64_t)gridDim.x * TILE) {
        const int64_t r0 = t0 + (int64_t)threadIdx.x * VN;
        T z[VN], yd[VN];
#pragma unroll
        for (int e = 0; e < VN; ++e) { z[e] = T(0); yd[e] = T(0); }
        if (r0 < n) {
            T g[VN], y[VN];
            T dgv[VN];
            vld(a.gsum + r0, g);
            vld(zc + r0, z);
            vld_degree<T>(a, r0, dgv);
            T dinv[VN];
            if (a.dinv) vld(a.dinv + r0, dinv);
            T zpv[VN], w2[VN], w1[VN], xv[VN], wv[VN];
            if (has_prev) {
                vld(zp + r0, zpv);
                vld(wo2 + r0, w2);
                vld(wo1 + r0, w1);
                vld_rw(a.x + r0, xv);
            }
#pragma unroll
            for (int e = 0; e < VN; ++e) {
                const int64_t r = r0 + e;
                const bool ok = r < n && r != trim;
                const T degT = dgv[e];
                const T D = precond_diag(degT, sigma);
                const T di = a.dinv ? dinv[e] : T(1) / D;
                T base = ((degT - sigma) * z[e] - g[e] + s_term) * inv_beta;
                if (has_prev) {
                    base -= cprev * D * zpv[e];
                    const T w = (zpv[e] * inv_oldb - oldeps * w2[e] - dlt * w1[e]) * inv_gamma;
                    wv[e] = ok ? w : T(0);
                    xv[e] += ok ? phi * w : T(0);
                }
                y[e] = ok ? base : T(0);
                yd[e] = ok ? base * di : T(0);           // padding rows may have D = 0
                z[e] = ok ? z[e] : T(0);
                acc0 += z[e] * inv_beta * y[e];
            }
            vst(a.Y + r0, y);
            if (has_prev) {
                vst(wn + r0, wv);
                vst(a.x + r0, xv);
            }
        }
        if (NE > 0 && c > 0) {
#pragma unroll
            for (int e = 0; e < VN; ++e) {
                sz[threadIdx.x * VN + e] = z[e];
                syd[threadIdx.x * VN + e] = yd[e];
            }
            __syncthreads();
            // warp w owns columns w, w + kWarps, ...; a lane reads VN consecutive rows per step
#pragma unroll
            for (int q = 0; q < QW; ++q) {
                const int t = warp + q * kWarps;
                if (t < c) {
                    const T* col = Vt + (int64_t)t * a.ldv + t0;
#pragma unroll
                    for (int u = 0; u < TILE / (32 * VN); ++u) {
                        const int rr = (u * 32 + lane) * VN;
                        if (t0 + rr < n) {
                            T v[VN];
                            vld(col + rr, v);
#pragma unroll
                            for (int e = 0; e < VN; ++e) {
                                const T vm = t0 + rr + e < n ? v[e] : T(0);
                                ca[q] += vm * syd[rr + e];
                                cg[q] += vm * sz[rr + e];
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
    // CTA sums: alpha' by a block reduction, the column sums by warp reductions (one warp per column)
    __shared__ T bv[NA];
    const T a0 = block_sum0(acc0);
    if (threadIdx.x == 0) bv[0] = a0;
#pragma unroll
    for (int q = 0; q < QW; ++q) {
        const int t = warp + q * kWarps;
        const T sa = warp_sum(ca[q]), sg = warp_sum(cg[q]);
        if (lane == 0 && t < NE) {
            bv[1 + t] = t < c ? sa : T(0);
            bv[1 + NE + t] = t < c ? sg : T(0);
        }
    }
    __syncthreads();
    __shared__ T red[NA];
    if (block_values_arrive<T>(bv, NE > 0 ? NA : 1, a.partial, a.pstride, a.counter)) {
        last_block_sum(a.partial, a.pstride, gridDim.x, NE > 0 ? NA : 1, red, a.counter);
        __shared__ double u1d[kCMax], gcd[kCMax], rhs[kCMax];
        __shared__ double alpha_s;
        const double delta = (double)a.delta;
        const double cp = (double)cprev, bt = (double)beta;
        for (int t = threadIdx.x; t < c; t += blockDim.x) {
            const double gp = has_prev ? (double)st->g_cur[t] : 0.0;
            const double gn = (double)red[1 + NE + t];
            gcd[t] = gn;
            u1d[t] = delta * (gn / bt - cp * gp);
            st->g_prev[t] = (T)gp;
            st->g_cur[t] = (T)gn;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double al = (double)red[0];
            for (int t = 0; t < c; ++t) al += gcd[t] / bt * u1d[t];
            alpha_s = al;
            st->alpha = (T)al;
        }
        __syncthreads();
        const double coef = alpha_s / bt;
        for (int t = threadIdx.x; t < c; t += blockDim.x) {
            double gu = 0.0, gg = 0.0;
            for (int q = 0; q < c; ++q) {
                gu += a.Gm[t + q * c] * u1d[q];
                gg += a.Gm[t + q * c] * gcd[q];
            }
            rhs[t] = (double)red[1 + t] + gu - coef * (gcd[t] + delta * gg);
        }
        __syncthreads();
        for (int t = threadIdx.x; t < c; t += blockDim.x) {
            double tv = 0.0;
            for (int q = 0; q < c; ++q) tv += a.Cinv[t + q * c] * rhs[q];
            st->tv[t] = (T)tv;
            st->qv[t] = (T)(coef * delta * gcd[t]);
            st->u1[t] = (T)u1d[t];
        }
    }
}

// ------------------------------------------------------------------ phase 2
// y = y' - (alpha_k / beta_k) D z_k + Vh (u1 - qv)        (the Lanczos vector, qv = coef delta g)
// z_{k+1} = D^{-1} (y - Vh tv)                           (the SMW preconditioner, Eq. 3.6)
// and the reductions y^T z_{k+1} (= beta_{k+1}^2) and 1^T z_{k+1}.  Each Vh entry is read once and
// feeds both combinations.  The last CTA runs the Givens step and the stopping test.
template <typename T, int NC>
__global__ void __launch_bounds__(kThreads) k_phase2(InnerArgs<T> a, int init, cudaGraphConditionalHandle cond,
                                                     int has_cond) {
    constexpr int VN = Vec<T>::N;
    constexpr int NE = Ncols<NC>::value;
    InnerState<T>* st = a.st;
    if (!init && st->done) {
        // nothing left to do: make sure a surrounding WHILE node stops
        if (has_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
        return;
    }
    const int k = init ? 0 : st->itn + 1;
    const int c = st->p_c;
    const T sigma = st->p_sigma;
    const T* __restrict__ zc = ((k - 1) & 1) ? a.z1 : a.z0;
    T* __restrict__ zn = (k & 1) ? a.z1 : a.z0;
    const T coef = init ? T(0) : st->alpha / st->beta;
    __shared__ T as_[NE > 0 ? NE : 1], ts_[NE > 0 ? NE : 1];
    __shared__ T red[2];
    for (int t = threadIdx.x; t < c; t += blockDim.x) {
        ts_[t] = st->tv[t];
        as_[t] = init ? T(0) : st->u1[t] - st->qv[t];
    }
    __syncthreads();
    T acc[2] = {T(0), T(0)};
    const int64_t n = a.rs.n, trim = a.trim;
    const T* __restrict__ Vt = a.Vt;
    const int64_t step = (int64_t)gridDim.x * blockDim.x * VN;
    for (int64_t r0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * VN; r0 < n; r0 += step) {
        T yv[VN], zcv[VN], ya[VN], zt[VN], dinv[VN];
        T dgv[VN];
        vld(a.Y + r0, yv);
        if (!init) vld(zc + r0, zcv);
        vld_degree<T>(a, r0, dgv);
        if (a.dinv) vld(a.dinv + r0, dinv);
#pragma unroll
        for (int e = 0; e < VN; ++e) { ya[e] = T(0); zt[e] = T(0); }
#pragma unroll
        for (int t = 0; t < NE; ++t) {
            if (t < c) {
                T v[VN];
                vld(Vt + (int64_t)t * a.ldv + r0, v);
                const T ca = as_[t], ct = ts_[t];
#pragma unroll
                for (int e = 0; e < VN; ++e) {
                    ya[e] += v[e] * ca;
                    zt[e] += v[e] * ct;
                }
            }
        }
        T zo[VN];
#pragma unroll
        for (int e = 0; e < VN; ++e) {
            const int64_t r = r0 + e;
            const bool ok = r < n && r != trim;
            const T degT = dgv[e];
            const T D = precond_diag(degT, sigma);
            const T di = a.dinv ? dinv[e] : T(1) / D;
            T y = yv[e] + ya[e];
            if (!init) y -= coef * D * zcv[e];
            const T z = (y - zt[e]) * di;
            zo[e] = ok ? z : T(0);
            acc[0] += ok ? y * z : T(0);
            acc[1] += zo[e];
        }
        vst(zn + r0, zo);
    }
    if (block_partials_arrive<T, 2>(acc, 2, a.partial, a.pstride, a.counter)) {
        last_block_sum(a.partial, a.pstride, gridDim.x, 2, red, a.counter);
        if (threadIdx.x == 0) minres_step(a, st, red[0], red[1], init, k, cond, has_cond);
    }
}

// ------------------------------------------------------------------ stand-alone operator apply
// y_r = (deg_r - sigma) x_r - g_r + (sigma/n) 1^T x + delta (Vh (Vh^T x))_r for r != trim, y_trim = 0, with
// x in z0, its gathered sums in gsum and 1^T x, delta Vh^T x left in s_cur, u1 by k_opstats.
template <typename T, int NC>
__global__ void __launch_bounds__(kThreads) k_apply_rows(InnerArgs<T> a) {
    constexpr int VN = Vec<T>::N;
    constexpr int NE = Ncols<NC>::value;
    const InnerState<T>* st = a.st;
    const int c = st->p_c;
    const T sigma = st->p_sigma;
    const T s_term = st->p_sig_n * st->s_cur;
    __shared__ T u1s[NE > 0 ? NE : 1];
    for (int t = threadIdx.x; t < c; t += blockDim.x) u1s[t] = st->u1[t];
    __syncthreads();
    const int64_t n = a.rs.n, trim = a.trim;
    const int64_t step = (int64_t)gridDim.x * blockDim.x * VN;
    for (int64_t r0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * VN; r0 < n; r0 += step) {
        T g[VN], z[VN], y[VN], vd[VN];
        T dgv[VN];
        vld(a.gsum + r0, g);
        vld(a.z0 + r0, z);
        vld_degree<T>(a, r0, dgv);
#pragma unroll
        for (int e = 0; e < VN; ++e) vd[e] = T(0);
#pragma unroll
        for (int t = 0; t < NE; ++t) {
            if (t < c) {
                T v[VN];
                vld(a.Vt + (int64_t)t * a.ldv + r0, v);
#pragma unroll
                for (int e = 0; e < VN; ++e) vd[e] += v[e] * u1s[t];
            }
        }
#pragma unroll
        for (int e = 0; e < VN; ++e) {
            const int64_t r = r0 + e;
            const T degT = dgv[e];
            const T v = ((degT - sigma) * z[e] - g[e] + s_term) + vd[e];
            y[e] = (r < n && r != trim) ? v : T(0);
        }
        vst(a.Y + r0, y);
    }
}

// ------------------------------------------------------------------ prep: b = rh / ||r||, h1 = Vh^T D^{-1} b

template <typename T, int NC>
__global__ void __launch_bounds__(kThreads) k_prep(InnerArgs<T> a, const double* R, const double* rnorm_dev) {
    __shared__ T red[NC > 0 ? NC : 1];
    const double rn = *rnorm_dev;
    const double inv = rn > 0.0 ? 1.0 / rn : 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.st->p_sigma = a.sigma;
        a.st->p_sig_n = a.sig_n;
        a.st->p_c = a.c;
    }
    T acc[NC > 0 ? NC : 1];
#pragma unroll
    for (int t = 0; t < (NC > 0 ? NC : 1); ++t) acc[t] = T(0);
    const int64_t n = a.rs.n;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const T b = (r == a.trim) ? T(0) : (T)(R[r] * inv);
        a.Y[r] = b;
        a.x[r] = T(0);
        a.wb0[r] = T(0);
        a.wb1[r] = T(0);
        a.wb2[r] = T(0);
        if (a.dinv || NC > 0) {
            const T degT = row_degree<T>(a.rs, r);
            const T di = T(1) / precond_diag(degT, a.sigma);
            if (a.dinv) a.dinv[r] = di;
            if (NC > 0 && r != a.trim) {
                const T bd = b * di;
#pragma unroll
                for (int t = 0; t < NC; ++t)
                    if (t < a.c) acc[t] += a.Vt[(int64_t)t * a.ldv + r] * bd;
            }
        }
    }
    const int nv = NC > 0 ? a.c : 0;
    if (block_partials_arrive<T, (NC > 0 ? NC : 1)>(acc, nv, a.partial, a.pstride, a.counter)) {
        last_block_sum(a.partial, a.pstride, gridDim.x, nv, red, a.counter);
        InnerState<T>* st = a.st;
        for (int t = threadIdx.x; t < nv; t += blockDim.x) {
            double tv = 0.0;
            for (int s = 0; s < nv; ++s) tv += a.Cinv[t + s * nv] * (double)red[s];
            st->tv[t] = (T)tv;
            st->qv[t] = T(0);
        }
        if (threadIdx.x == 0) {
            st->done = 0;
            st->itn = 0;
            st->pending = 0;
            st->alpha = T(0);
            st->beta = T(1);
        }
    }
}

// ------------------------------------------------------------------ finalize: last deferred update, cast to FP64

template <typename T>
__global__ void __launch_bounds__(kThreads) k_finalize(InnerArgs<T> a, double* Z) {
    const InnerState<T>* st = a.st;
    const int j = st->itn;
    const int pend = st->pending;
    const T* zj = ((j - 1) & 1) ? a.z1 : a.z0;
    const T* wo2 = wbuf(a, j + 1);
    const T* wo1 = wbuf(a, j + 2);
    const T inv_oldb = pend ? T(1) / st->oldb : T(0);
    const T oldeps = st->w_oldeps, dlt = st->w_dlt, inv_gamma = st->w_inv_gamma, phi = st->w_phi;
    const int64_t n = a.rs.n;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        T xv = a.x[r];
        if (pend && r != a.trim) {
            const T w = (zj[r] * inv_oldb - oldeps * wo2[r] - dlt * wo1[r]) * inv_gamma;
            xv += phi * w;
        }
        Z[r] = (r == a.trim) ? 0.0 : (double)xv;
    }
}

// ------------------------------------------------------------------ operator statistics for a stand-alone apply

template <typename T, int NC>
__global__ void __launch_bounds__(kThreads) k_opstats(InnerArgs<T> a, const T* x) {
    __shared__ T red[1 + NC];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.st->p_sigma = a.sigma;
        a.st->p_sig_n = a.sig_n;
        a.st->p_c = a.c;
    }
    T acc[1 + NC];
#pragma unroll
    for (int t = 0; t < 1 + NC; ++t) acc[t] = T(0);
    const int64_t n = a.rs.n;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        if (r == a.trim) continue;
        const T xr = x[r];
        acc[0] += xr;
#pragma unroll
        for (int t = 0; t < NC; ++t)
            if (t < a.c) acc[1 + t] += a.Vt[(int64_t)t * a.ldv + r] * xr;
    }
    if (block_partials_arrive<T, 1 + NC>(acc, 1 + a.c, a.partial, a.pstride, a.counter)) {
        last_block_sum(a.partial, a.pstride, gridDim.x, 1 + a.c, red, a.counter);
        InnerState<T>* st = a.st;
        for (int t = threadIdx.x; t < a.c; t += blockDim.x) {
            st->g_cur[t] = red[1 + t];
            st->u1[t] = a.delta * red[1 + t];
        }
        if (threadIdx.x == 0) {
            st->s_cur = red[0];
            st->beta = T(1);
            st->oldb = T(0);
            st->itn = 0;
            st->done = 0;
            st->pending = 0;
        }
    }
}

// ------------------------------------------------------------------ Gram matrix Vh^T D^{-1} Vh and C^{-1}

constexpr int kGramTile = 128;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_gram(InnerArgs<T> a, double* G, double* Cinv, double* partial,
                                                   int pstride) {
    extern __shared__ double gsm[];     // [c][kGramTile + 1]
    const int c = a.c;
    const int ne = c * (c + 1) / 2;
    const int64_t n = a.rs.n;
    constexpr int kPer = 2;             // entries per thread (c <= 31 -> ne <= 496 <= 2 * 256)
    int ea[kPer], eb[kPer];
    double acc[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        int e = threadIdx.x + q * blockDim.x;
        acc[q] = 0.0;
        ea[q] = -1;
        eb[q] = -1;
        if (e < ne) {  // unrank e -> (p, s), p <= s, row-major over the upper triangle
            int p = 0, rem = e;
            while (rem >= c - p) { rem -= c - p; ++p; }
            ea[q] = p;
            eb[q] = p + rem;
        }
    }
    const int ldt = kGramTile + 1;
    for (int64_t r0 = (int64_t)blockIdx.x * kGramTile; r0 < n; r0 += (int64_t)gridDim.x * kGramTile) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < c * kGramTile; idx += blockDim.x) {
            const int col = idx / kGramTile, rr = idx % kGramTile;
            const int64_t r = r0 + rr;
            double v = 0.0;
            if (r < n && r != a.trim) {
                const T degT = row_degree<T>(a.rs, r);
                v = (double)a.Vt[(int64_t)col * a.ldv + r] * rsqrt((double)precond_diag(degT, a.sigma));
            }
            gsm[col * ldt + rr] = v;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            if (ea[q] >= 0) {
                const double* pa = gsm + ea[q] * ldt;
                const double* pb = gsm + eb[q] * ldt;
                double s = 0.0;
                for (int rr = 0; rr < kGramTile; ++rr) s += pa[rr] * pb[rr];
                acc[q] += s;
            }
        }
    }
    // per-block partials (one slot per entry), then the last block sums and factors
    for (int q = 0; q < kPer; ++q) {
        int e = threadIdx.x + q * blockDim.x;
        if (e < ne) partial[(size_t)e * pstride + blockIdx.x] = acc[q];
    }
    __threadfence();
    __syncthreads();
    __shared__ int last;
    if (threadIdx.x == 0) last = (atomicAdd(a.counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    __shared__ double Gs[kCMax * kCMax];
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(partial + (size_t)e * pstride + b);
        int p = 0, rem = e;
        while (rem >= c - p) { rem -= c - p; ++p; }
        Gs[p + (p + rem) * c] = s;
        Gs[(p + rem) + p * c] = s;
    }
    if (threadIdx.x == 0) *a.counter = 0u;
    __syncthreads();
    if (threadIdx.x == 0) {
        // C = delta^{-1} I + G (SPD), Cholesky C = L L^T, then C^{-1} column by column
        double Lc[kCMax * kCMax];
        const double dinv = 1.0 / (double)a.delta;
        for (int p = 0; p < c; ++p)
            for (int s = 0; s < c; ++s) {
                G[p + s * c] = Gs[p + s * c];
                Lc[p + s * c] = 0.0;
            }
        for (int s = 0; s < c; ++s) {
            double d = Gs[s + s * c] + dinv;
            for (int t = 0; t < s; ++t) d -= Lc[s + t * c] * Lc[s + t * c];
            d = sqrt(d > 0.0 ? d : 1e-300);
            Lc[s + s * c] = d;
            for (int p = s + 1; p < c; ++p) {
                double v = Gs[p + s * c];
                for (int t = 0; t < s; ++t) v -= Lc[p + t * c] * Lc[s + t * c];
                Lc[p + s * c] = v / d;
            }
        }
        for (int col = 0; col < c; ++col) {
            double y[kCMax];
            for (int p = 0; p < c; ++p) {
                double v = (p == col) ? 1.0 : 0.0;
                for (int t = 0; t < p; ++t) v -= Lc[p + t * c] * y[t];
                y[p] = v / Lc[p + p * c];
            }
            for (int p = c - 1; p >= 0; --p) {
                double v = y[p];
                for (int t = p + 1; t < c; ++t) v -= Lc[t + p * c] * y[t];
                y[p] = v / Lc[p + p * c];
            }
            for (int p = 0; p < c; ++p) Cinv[p + col * c] = y[p];
        }
    }
}

template <typename T>
__global__ void k_copy_vcol(const double* src, T* dst, int64_t n) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        dst[r] = (T)src[r];
}

// ------------------------------------------------------------------ multilevel-preconditioned MINRES
// Preconditioner (Remark 3.2; here with the multilevel M instead of a diagonal):
//   P^{-1} r = Pi M^{-1} Pi r + Vh D Vh^T r,   Pi = I - Vh Vh^T,   D = diag(1 / (lambda_t - sigma + delta)),
// with M^{-1} one V-cycle of the aggregation hierarchy (multilevel.cu) and lambda_t the locked
// eigenvalues.  It is symmetric positive definite and, for Vh made of eigenvectors, it inverts
// Lh + delta Vh Vh^T - sigma I on span Vh and approximates it on the complement.  It replaces the
// Sherman-Morrison-Woodbury form of Eq. 3.6 (exact for M + delta Vh Vh^T) because M^{-1} is ~1/lambda_1
// on the deflated directions: SMW subtracts two terms of that size to get one of size 1/delta,
// which in FP32 loses more than the inner tolerance; the projections never form those terms.
// P is not diagonal, so the unpreconditioned Lanczos vectors r_{k-1}, r_k are kept (buffers rprev,
// rcur, shifted in place).  One iteration k:
//   gather(z_k); ml_phase1: y' = ((deg - sigma) z_k - g + (sigma/n) s) / beta_k - (beta_k/beta_{k-1}) r_{k-1},
//       the deferred w/x update, alpha' = v_k^T y'; last CTA: u1 = delta g_k / beta_k,
//       alpha_k = alpha' + (g_k / beta_k)^T u1 with g_k = Vh^T z_k from the phase-2c launch before;
//   ml_phase2a: r_{k+1} = y' + Vh u1 - (alpha_k / beta_k) r_k and h = Vh^T r_{k+1};
//   ml_project: rin = r_{k+1} - Vh h (= Pi r);   V-cycle: w = M^{-1} rin;
//   ml_phase2b: the V-cycle's last level-0 step (w), Vh^T w, r^T w; last CTA: tv = D h - Vh^T w,
//       beta_{k+1}^2 = r^T w + h^T tv, Givens step;
//   ml_phase2c: z_{k+1} = w + Vh tv (= Pi w + Vh D h), 1^T z_{k+1} and g_{k+1} = Vh^T z_{k+1}.

template <typename T, int NC>
__global__ void __launch_bounds__(kThreads) k_ml_phase1(InnerArgs<T> a) {
    constexpr int VN = Vec<T>::N;
    InnerState<T>* st = a.st;
    if (st->done) return;
    const int k = st->itn + 1;
    const int c = st->p_c;
    const T sigma = st->p_sigma;
    const T* __restrict__ zc = ((k - 1) & 1) ? a.z1 : a.z0;
    const T* __restrict__ zp = (k & 1) ? a.z1 : a.z0;
    const T beta = st->beta, oldb = st->oldb;
    const T inv_beta = T(1) / beta;
    const bool has_prev = k >= 2;
    const T cprev = has_prev ? beta / oldb : T(0);
    const T inv_oldb = has_prev ? T(1) / oldb : T(0);
    const T s_term = st->p_sig_n * st->s_cur;
    const int j = k - 1;
    const T* __restrict__ wo2 = wbuf(a, j + 1);
    const T* __restrict__ wo1 = wbuf(a, j + 2);
    T* __restrict__ wn = wbuf(a, j);
    const T oldeps = st->w_oldeps, dlt = st->w_dlt, inv_gamma = st->w_inv_gamma, phi = st->w_phi;
    T acc0 = T(0);
    const int64_t n = a.rs.n, trim = a.trim;
    const int64_t step = (int64_t)gridDim.x * blockDim.x * VN;
    for (int64_t r0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * VN; r0 < n; r0 += step) {
        T z[VN];
#pragma unroll
        for (int e = 0; e < VN; ++e) z[e] = T(0);
        {
            T g[VN], y[VN], rpv[VN], dgv[VN];
            vld(a.gsum + r0, g);
            vld(zc + r0, z);
            vld_degree<T>(a, r0, dgv);
            T zpv[VN], w2[VN], w1[VN], xv[VN], wv[VN];
            if (has_prev) {
                vld(a.rprev + r0, rpv);
                vld(zp + r0, zpv);
                vld(wo2 + r0, w2);
                vld(wo1 + r0, w1);
                vld_rw(a.x + r0, xv);
            }
#pragma unroll
            for (int e = 0; e < VN; ++e) {
                const int64_t r = r0 + e;
                const bool ok = r < n && r != trim;
                T base = ((dgv[e] - sigma) * z[e] - g[e] + s_term) * inv_beta;
                if (has_prev) {
                    base -= cprev * rpv[e];
                    const T w = (zpv[e] * inv_oldb - oldeps * w2[e] - dlt * w1[e]) * inv_gamma;
                    wv[e] = ok ? w : T(0);
                    xv[e] += ok ? phi * w : T(0);
                }
                y[e] = ok ? base : T(0);
                z[e] = ok ? z[e] : T(0);
                acc0 += z[e] * inv_beta * y[e];
            }
            vst(a.Y + r0, y);
            if (has_prev) {
                vst(wn + r0, wv);
                vst(a.x + r0, xv);
            }
        }
    }
    __shared__ T red[1];
    T accv[1] = {acc0};
    if (block_partials_arrive<T, 1>(accv, 1, a.partial, a.pstride, a.counter)) {
        last_block_sum(a.partial, a.pstride, gridDim.x, 1, red, a.counter);
        if (threadIdx.x == 0) {
            // g_k = Vh^T z_k was reduced by the phase-2c launch that wrote z_k
            const double bt = (double)beta, delta = (double)a.delta;
            double al = (double)red[0];
            for (int t = 0; t < c; ++t) {
                const double gn = (double)st->g_cur[t];
                const double u = delta * gn / bt;
                st->u1[t] = (T)u;
                al += gn / bt * u;
            }
            st->alpha = (T)al;
        }
    }
}

// r_{k+1} = y' + Vh u1 - (alpha_k / beta_k) r_k (rprev <- r_k, rcur <- r_{k+1}) and h = Vh^T r_{k+1};
// init: h = Vh^T r_1 only (r_1 = rcur from the prep kernel)
template <typename T, int NC>
__global__ void __launch_bounds__(kThreads) k_ml_phase2a(InnerArgs<T> a, int init) {
    constexpr int VN = Vec<T>::N;
    constexpr int NE = Ncols<NC>::value;
    constexpr int TILE = kThreads * VN;
    constexpr int QW = (NE + kWarps - 1) / kWarps;
    InnerState<T>* st = a.st;
    if (!init && st->done) return;
    const int c = st->p_c;
    const T coef = init ? T(0) : st->alpha / st->beta;
    __shared__ T us[NE > 0 ? NE : 1];
    __shared__ __align__(16) T sr[NE > 0 ? TILE : 1];
    for (int t = threadIdx.x; t < c; t += blockDim.x) us[t] = init ? T(0) : st->u1[t];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T ch[QW > 0 ? QW : 1];
#pragma unroll
    for (int q = 0; q < (QW > 0 ? QW : 1); ++q) ch[q] = T(0);
    const int64_t n = a.rs.n, trim = a.trim;
    for (int64_t t0 = (int64_t)blockIdx.x * TILE; t0 < n; t0 += (int64_t)gridDim.x * TILE) {
        const int64_t r0 = t0 + (int64_t)threadIdx.x * VN;
        T rn[VN];
#pragma unroll
        for (int e = 0; e < VN; ++e) rn[e] = T(0);
        if (r0 < n) {
            T rc[VN];
            vld_rw(a.rcur + r0, rc);
            if (init) {
#pragma unroll
                for (int e = 0; e < VN; ++e) rn[e] = (r0 + e < n && r0 + e != trim) ? rc[e] : T(0);
            } else {
                T y[VN], vu[VN];
                vld(a.Y + r0, y);
#pragma unroll
                for (int e = 0; e < VN; ++e) vu[e] = T(0);
#pragma unroll
                for (int t = 0; t < NE; ++t) {
                    if (t < c) {
                        T v[VN];
                        vld(a.Vt + (int64_t)t * a.ldv + r0, v);
#pragma unroll
                        for (int e = 0; e < VN; ++e) vu[e] += v[e] * us[t];
                    }
                }
#pragma unroll
                for (int e = 0; e < VN; ++e) {
                    const int64_t r = r0 + e;
                    rn[e] = (r < n && r != trim) ? y[e] + vu[e] - coef * rc[e] : T(0);
                }
                vst(a.rprev + r0, rc);
                vst(a.rcur + r0, rn);
            }
        }
        if (NE > 0 && c > 0) {
#pragma unroll
            for (int e = 0; e < VN; ++e) sr[threadIdx.x * VN + e] = rn[e];
            __syncthreads();
#pragma unroll
            for (int q = 0; q < QW; ++q) {
                const int t = warp + q * kWarps;
                if (t < c) {
                    const T* col = a.Vt + (int64_t)t * a.ldv + t0;
#pragma unroll
                    for (int u = 0; u < TILE / (32 * VN); ++u) {
                        const int rr = (u * 32 + lane) * VN;
                        if (t0 + rr < n) {
                            T v[VN];
                            vld(col + rr, v);
#pragma unroll
                            for (int e = 0; e < VN; ++e) ch[q] += (t0 + rr + e < n ? v[e] : T(0)) * sr[rr + e];
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
    if (NE == 0) return;
    __shared__ T bv[NE > 0 ? NE : 1];
#pragma unroll
    for (int q = 0; q < QW; ++q) {
        const int t = warp + q * kWarps;
        const T sh = warp_sum(ch[q]);
        if (lane == 0 && t < NE) bv[t] = t < c ? sh : T(0);
    }
    __syncthreads();
    __shared__ T red[NE > 0 ? NE : 1];
    if (block_values_arrive<T>(bv, NE, a.partial, a.pstride, a.counter)) {
        last_block_sum(a.partial, a.pstride, gridDim.x, NE, red, a.counter);
        for (int t = threadIdx.x; t < c; t += blockDim.x) st->hv[t] = red[t];
    }
}

// rin = r_{k+1} - Vh h (Pi r); only for c > 0
template <typename T, int NC>
__global__ void __launch_bounds__(kThreads) k_ml_project(InnerArgs<T> a, int init) {
    constexpr int VN = Vec<T>::N;
    constexpr int NE = Ncols<NC>::value;
    InnerState<T>* st = a.st;
    if (!init && st->done) return;
    const int c = st->p_c;
    __shared__ T hs[NE > 0 ? NE : 1];
    for (int t = threadIdx.x; t < c; t += blockDim.x) hs[t] = st->hv[t];
    __syncthreads();
    const int64_t n = a.rs.n, trim = a.trim;
    const int64_t step = (int64_t)gridDim.x * blockDim.x * VN;
    for (int64_t r0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * VN; r0 < n; r0 += step) {
        T r[VN];
        vld(a.rcur + r0, r);
#pragma unroll
        for (int t = 0; t < NE; ++t) {
            if (t < c) {
                T v[VN];
                vld(a.Vt + (int64_t)t * a.ldv + r0, v);
#pragma unroll
                for (int e = 0; e < VN; ++e) r[e] -= v[e] * hs[t];
            }
        }
#pragma unroll
        for (int e = 0; e < VN; ++e) r[e] = (r0 + e < n && r0 + e != trim) ? r[e] : T(0);
        vst(a.rin + r0, r);
        if (a.ml_x0) {                        // the V-cycle's first smoothing step, x0 = w D^{-1} rin
            T di[VN];
            vld(a.ml_dinv0 + r0, di);
#pragma unroll
            for (int e = 0; e < VN; ++e) r[e] = a.ml_omega * r[e] * di[e];
            vst(a.ml_x0 + r0, r);
        }
    }
}

template <typename T, int NC>
__global__ void __launch_bounds__(kThreads) k_ml_phase2b(InnerArgs<T> a, int init, cudaGraphConditionalHandle cond,
                                                        int has_cond) {
    constexpr int VN = Vec<T>::N;
    constexpr int NE = Ncols<NC>::value;
    constexpr int NA = 1 + NE;               // r^T w, Vh^T w
    InnerState<T>* st = a.st;
    if (!init && st->done) {
        if (has_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
        return;
    }
    const int k = init ? 0 : st->itn + 1;
    const int c = st->p_c;
    T acc[NA];
#pragma unroll
    for (int t = 0; t < NA; ++t) acc[t] = T(0);
    const int64_t n = a.rs.n, trim = a.trim;
    const int64_t step = (int64_t)gridDim.x * blockDim.x * VN;
    for (int64_t r0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * VN; r0 < n; r0 += step) {
        T w[VN], r[VN];
        if (a.ml_fuse_post) {
            // the V-cycle's last step on level 0: w = x1 + w D^{-1} (b - D x1 + W x1), stored for phase 2c
            T bb[VN], di[VN], x1[VN], wx[VN];
            vld(a.ml_b0 + r0, bb);
            vld(a.ml_dinv0 + r0, di);
            vld(a.ml_x1 + r0, x1);
            vld(a.ml_wx1 + r0, wx);
#pragma unroll
            for (int e = 0; e < VN; ++e) w[e] = x1[e] + a.ml_omega * (bb[e] * di[e] - x1[e] + wx[e] * di[e]);
        } else {
            vld(a.wv + r0, w);
        }
        vld(a.rcur + r0, r);
#pragma unroll
        for (int e = 0; e < VN; ++e) {
            const bool ok = r0 + e < n && r0 + e != trim;
            w[e] = ok ? w[e] : T(0);
            acc[0] += (ok ? r[e] : T(0)) * w[e];
        }
        if (a.ml_fuse_post) vst(a.wv + r0, w);
#pragma unroll
        for (int t = 0; t < NE; ++t) {
            if (t < c) {
                T v[VN];
                vld(a.Vt + (int64_t)t * a.ldv + r0, v);
#pragma unroll
                for (int e = 0; e < VN; ++e) acc[1 + t] += (r0 + e < n && r0 + e != trim ? v[e] : T(0)) * w[e];
            }
        }
    }
    __shared__ T red[NA];
    if (block_partials_arrive<T, NA>(acc, NE > 0 ? NA : 1, a.partial, a.pstride, a.counter)) {
        last_block_sum(a.partial, a.pstride, gridDim.x, NE > 0 ? NA : 1, red, a.counter);
        if (threadIdx.x == 0) {
            // z = Pi w + Vh D h = w + Vh tv,  tv = D h - Vh^T w,  r^T z = r^T w + h^T tv
            double bb = (double)red[0];
            for (int t = 0; t < c; ++t) {
                const double h = (double)st->hv[t];
                const double tv = a.dv[t] * h - (double)red[1 + t];
                st->tv[t] = (T)tv;
                bb += h * tv;
            }
            minres_step(a, st, (T)bb, st->s_cur, init, k, cond, has_cond);
        }
    }
}

// z_{k+1} = w + Vh tv, its sum 1^T z_{k+1} (the next operator application's rank-one term) and
// g_{k+1} = Vh^T z_{k+1} (its deflation term)
template <typename T, int NC>
__global__ void __launch_bounds__(kThreads) k_ml_phase2c(InnerArgs<T> a, int init) {
    constexpr int VN = Vec<T>::N;
    constexpr int NE = Ncols<NC>::value;
    InnerState<T>* st = a.st;
    // also runs after the stop (from wv, into the slot of z_{itn+1}, which nothing reads then)
    const int k = init ? 0 : st->itn;                 // phase 2b already advanced itn to k
    T* __restrict__ zn = (k & 1) ? a.z1 : a.z0;
    const int c = st->p_c;
    __shared__ T ts[NE > 0 ? NE : 1];
    for (int t = threadIdx.x; t < c; t += blockDim.x) ts[t] = st->tv[t];
    __syncthreads();
    constexpr int NA = 1 + NE;                         // 1^T z_{k+1}, Vh^T z_{k+1}
    T acc[NA];
#pragma unroll
    for (int t = 0; t < NA; ++t) acc[t] = T(0);
    const int64_t n = a.rs.n, trim = a.trim;
    const int64_t step = (int64_t)gridDim.x * blockDim.x * VN;
    for (int64_t r0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * VN; r0 < n; r0 += step) {
        T w[VN];
        vld(a.wv + r0, w);
#pragma unroll
        for (int t = 0; t < NE; ++t) {
            if (t < c) {
                T v[VN];
                vld(a.Vt + (int64_t)t * a.ldv + r0, v);
#pragma unroll
                for (int e = 0; e < VN; ++e) w[e] += v[e] * ts[t];
            }
        }
#pragma unroll
        for (int e = 0; e < VN; ++e) {
            w[e] = (r0 + e < n && r0 + e != trim) ? w[e] : T(0);
            acc[0] += w[e];
        }
        vst(zn + r0, w);
        // Vh^T z_{k+1} for the next operator application (the columns are still in L1)
#pragma unroll
        for (int t = 0; t < NE; ++t) {
            if (t < c) {
                T v[VN];
                vld(a.Vt + (int64_t)t * a.ldv + r0, v);
#pragma unroll
                for (int e = 0; e < VN; ++e) acc[1 + t] += v[e] * w[e];
            }
        }
    }
    __shared__ T red[NA];
    if (block_partials_arrive<T, NA>(acc, NE > 0 ? NA : 1, a.partial, a.pstride, a.counter)) {
        last_block_sum(a.partial, a.pstride, gridDim.x, NE > 0 ? NA : 1, red, a.counter);
        if (threadIdx.x == 0) {
            st->s_cur = red[0];
            for (int t = 0; t < c; ++t) st->g_cur[t] = red[1 + t];
        }
    }
}

// right-hand side of a multilevel-preconditioned solve: rc = b = R / ||R|| (trimmed entry 0),
// x = w buffers = 0, state reset
template <typename T>
__global__ void __launch_bounds__(kThreads) k_ml_prep(InnerArgs<T> a, const double* R, const double* rnorm_dev) {
    const double rn = *rnorm_dev;
    const double inv = rn > 0.0 ? 1.0 / rn : 0.0;
    const int64_t n = a.rs.n;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        a.rcur[r] = (r == a.trim) ? T(0) : (T)(R[r] * inv);
        a.rprev[r] = T(0);
        a.x[r] = T(0);
        a.wb0[r] = T(0);
        a.wb1[r] = T(0);
        a.wb2[r] = T(0);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        InnerState<T>* st = a.st;
        st->p_sigma = a.sigma;
        st->p_sig_n = a.sig_n;
        st->p_c = a.c;
        st->done = 0;
        st->itn = 0;
        st->pending = 0;
        st->alpha = T(0);
        st->beta = T(1);
    }
}

// plain gather g = sum over the neighbours of x (the trimmed row gets 0); returns at once once the
// inner solve has stopped (done != null)
template <typename T, int G, int TPB>
__global__ void __launch_bounds__(TPB, TPB == kThreads ? 4 : 1) k_gather_vec(RowSched rs, const T* x, T* g,
                                                                             int64_t skip, const int* done) {
    if (done && *done) return;
    GatherStore<T> epi{g};
    for_each_row_gather<T, G>(rs, x, epi, skip);
}

// ------------------------------------------------------------------ launchers

// deflation-rank buckets: the kernels keep NC per-thread accumulators, so small buckets save registers
#define ISIRA_NC_DISPATCH(c, F) \
    do {                        \
        if ((c) == 0) { F(0); } \
        else if ((c) <= 8) { F(8); } \
        else if ((c) <= 12) { F(12); } \
        else if ((c) <= 16) { F(16); } \
        else if ((c) <= 24) { F(24); } \
        else { F(32); }         \
    } while (0)

// slices-only gathers (every row in the sliced copy): z_k of the current iteration, or a given vector
template <typename T>
__global__ void __launch_bounds__(kThreads, kSliceBlocksPerSM) k_phase1_gather_s(InnerArgs<T> a) {
    const InnerState<T>* st = a.st;
    if (st->done) return;
    const T* zc = (st->itn & 1) ? a.z1 : a.z0;
    GatherStore<T> epi{a.gsum};
    slices_only_gather<T>(a.rs, zc, epi, a.trim);
}

template <typename T>
__global__ void __launch_bounds__(kThreads, kSliceBlocksPerSM) k_gather_vec_s(RowSched rs, const T* x, T* g,
                                                                              int64_t skip, const int* done) {
    if (done && *done) return;
    GatherStore<T> epi{g};
    slices_only_gather<T>(rs, x, epi, skip);
}

inline int slice_grid(const RowSched& rs) {
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            nsm = 152;
    }
    const int64_t want = ((int64_t)rs.n_slices + kWarps - 1) / kWarps;
    const int64_t cap = (int64_t)nsm * kSliceBlocksPerSM;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

template <typename T>
void inner_gather(const InnerArgs<T>& a, int lanes, cudaStream_t s) {
    if (slices_only(a.rs)) {
        k_phase1_gather_s<T><<<slice_grid(a.rs), kThreads, 0, s>>>(a);
        return;
    }
#define LG(G, TPB) k_phase1_gather<T, G, TPB><<<a.rs.grid(), TPB, a.rs.hub_bytes, s>>>(a)
    ISIRA_GATHER_DISPATCH(lanes, a.rs.tpb, LG);
#undef LG
}

// ---- one-wave grids for the row kernels.  Their register use grows with the deflation bucket
// NC (FP64, NC = 32: over 200 registers), so the resident CTAs per SM differ per instance; a grid
// of ew_blocks CTAs could then run as one full wave plus a partial one.  Each instance is
// launched with min(ew_blocks, SMs x resident CTAs); the row loops are grid-stride.
struct WaveCache {
    std::mutex mu;
    std::unordered_map<const void*, int> per_sm;
    int nsm = 0;
};
inline WaveCache& wave_cache() {
    static WaveCache c;
    return c;
}

inline cudaError_t wave_register(const void* fn) {
    WaveCache& c = wave_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    cudaError_t e = cudaSuccess;
    if (c.nsm == 0) {
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c.nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    if (c.per_sm.count(fn)) return cudaSuccess;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kThreads, 0);
    if (e == cudaSuccess) c.per_sm[fn] = nb > 0 ? nb : 1;
    return e;
}

inline int wave_grid(const void* fn, int want) {
    WaveCache& c = wave_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    auto it = c.per_sm.find(fn);
    if (it == c.per_sm.end() || c.nsm == 0) return want;
    const int cap = c.nsm * it->second;
    return want < cap ? want : cap;
}

// Lets every gather kernel of precision T take up to `bytes` of dynamic shared memory, and
// records the resident CTAs per SM of every row-kernel instance (before any graph capture).
template <typename T>
cudaError_t inner_gather_attrs(int bytes) {
    cudaError_t e = cudaSuccess;
#define LA(G, TPB)                                                                                      \
    if (e == cudaSuccess)                                                                               \
        e = cudaFuncSetAttribute(k_phase1_gather<T, G, TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes); \
    if (e == cudaSuccess)                                                                               \
        e = cudaFuncSetAttribute(k_gather_vec<T, G, TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
    for (int tpb : {kThreads, kBigBlock})
        for (int g : {1, 2, 4, 8, 16, 32}) ISIRA_GATHER_DISPATCH(g, tpb, LA);
#undef LA
#define LW(NC)                                                                                          \
    do {                                                                                                \
        if (e == cudaSuccess) e = wave_register((const void*)k_phase1<T, NC>);                          \
        if (e == cudaSuccess) e = wave_register((const void*)k_phase2<T, NC>);                          \
        if (e == cudaSuccess) e = wave_register((const void*)k_prep<T, NC>);                            \
        if (e == cudaSuccess) e = wave_register((const void*)k_opstats<T, NC>);                         \
        if (e == cudaSuccess) e = wave_register((const void*)k_apply_rows<T, NC>);                      \
        if (e == cudaSuccess) e = wave_register((const void*)k_ml_phase1<T, NC>);                       \
        if (e == cudaSuccess) e = wave_register((const void*)k_ml_phase2a<T, NC>);                      \
        if (e == cudaSuccess) e = wave_register((const void*)k_ml_phase2b<T, NC>);                      \
        if (e == cudaSuccess) e = wave_register((const void*)k_ml_phase2c<T, NC>);                      \
        if (e == cudaSuccess) e = wave_register((const void*)k_ml_project<T, NC>);                      \
    } while (0)
    for (int nc : {0, 8, 12, 16, 24, 32}) ISIRA_NC_DISPATCH(nc, LW);
#undef LW
    return e;
}

// grid of the vectorised row kernels: one thread per Vec<T>::N rows, at most ew_blocks CTAs
template <typename T>
inline int vec_blocks(const InnerArgs<T>& a) {
    const int64_t want = (a.rs.n + (int64_t)kThreads * Vec<T>::N - 1) / ((int64_t)kThreads * Vec<T>::N);
    return (int)(want < a.ew_blocks ? (want > 0 ? want : 1) : a.ew_blocks);
}

template <typename T>
void inner_rows(const InnerArgs<T>& a, cudaStream_t s) {
#define L1(NC) k_phase1<T, NC><<<wave_grid((const void*)k_phase1<T, NC>, vec_blocks(a)), kThreads, 0, s>>>(a)
    ISIRA_NC_DISPATCH(a.c, L1);
#undef L1
}

template <typename T>
void inner_phase1(const InnerArgs<T>& a, int lanes, cudaStream_t s) {
    inner_gather<T>(a, lanes, s);
    inner_rows<T>(a, s);
}

template <typename T>
void inner_apply(const InnerArgs<T>& a, int lanes, cudaStream_t s) {
    inner_gather<T>(a, lanes, s);
#define LA(NC) k_apply_rows<T, NC><<<wave_grid((const void*)k_apply_rows<T, NC>, vec_blocks(a)), kThreads, 0, s>>>(a)
    ISIRA_NC_DISPATCH(a.c, LA);
#undef LA
}

template <typename T>
void inner_phase2(const InnerArgs<T>& a, int init, cudaStream_t s) {
#define L2(NC) k_phase2<T, NC><<<wave_grid((const void*)k_phase2<T, NC>, vec_blocks(a)), kThreads, 0, s>>>(a, init, 0, 0)
    ISIRA_NC_DISPATCH(a.c, L2);
#undef L2
}

template <typename T>
void inner_phase2_cond(const InnerArgs<T>& a, cudaGraphConditionalHandle cond, cudaStream_t s) {
#define L2C(NC) k_phase2<T, NC><<<wave_grid((const void*)k_phase2<T, NC>, vec_blocks(a)), kThreads, 0, s>>>(a, 0, cond, 1)
    ISIRA_NC_DISPATCH(a.c, L2C);
#undef L2C
}

template <typename T>
void inner_gather_vec(const InnerArgs<T>& a, const T* x, T* g, int lanes, const int* done, cudaStream_t s) {
    if (slices_only(a.rs)) {
        k_gather_vec_s<T><<<slice_grid(a.rs), kThreads, 0, s>>>(a.rs, x, g, a.trim, done);
        return;
    }
#define LGV(G, TPB) k_gather_vec<T, G, TPB><<<a.rs.grid(), TPB, a.rs.hub_bytes, s>>>(a.rs, x, g, a.trim, done)
    ISIRA_GATHER_DISPATCH(lanes, a.rs.tpb, LGV);
#undef LGV
}

template <typename T>
void ml_inner_prep(const InnerArgs<T>& a, const double* R, const double* rnorm_dev, cudaStream_t s) {
    k_ml_prep<T><<<a.ew_blocks, kThreads, 0, s>>>(a, R, rnorm_dev);
}

template <typename T>
void ml_phase1(const InnerArgs<T>& a, cudaStream_t s) {
#define L1(NC) k_ml_phase1<T, NC><<<wave_grid((const void*)k_ml_phase1<T, NC>, vec_blocks(a)), kThreads, 0, s>>>(a)
    ISIRA_NC_DISPATCH(a.c, L1);
#undef L1
}

template <typename T>
void ml_phase2a(const InnerArgs<T>& a, int init, cudaStream_t s) {
#define L2(NC) k_ml_phase2a<T, NC><<<wave_grid((const void*)k_ml_phase2a<T, NC>, vec_blocks(a)), kThreads, 0, s>>>(a, init)
    ISIRA_NC_DISPATCH(a.c, L2);
#undef L2
}

template <typename T>
void ml_project(const InnerArgs<T>& a, int init, cudaStream_t s) {
    if (a.c <= 0) return;
#define LP(NC) k_ml_project<T, NC><<<wave_grid((const void*)k_ml_project<T, NC>, vec_blocks(a)), kThreads, 0, s>>>(a, init)
    ISIRA_NC_DISPATCH(a.c, LP);
#undef LP
}

template <typename T>
void ml_phase2b(const InnerArgs<T>& a, int init, cudaGraphConditionalHandle cond, int has_cond, cudaStream_t s) {
#define L2(NC)                                                                                              \
    k_ml_phase2b<T, NC><<<wave_grid((const void*)k_ml_phase2b<T, NC>, vec_blocks(a)), kThreads, 0, s>>>(a, init, \
                                                                                                  cond, has_cond)
    ISIRA_NC_DISPATCH(a.c, L2);
#undef L2
}

template <typename T>
void ml_phase2c(const InnerArgs<T>& a, int init, cudaStream_t s) {
#define L2(NC) k_ml_phase2c<T, NC><<<wave_grid((const void*)k_ml_phase2c<T, NC>, vec_blocks(a)), kThreads, 0, s>>>(a, init)
    ISIRA_NC_DISPATCH(a.c, L2);
#undef L2
}

template <typename T>
void inner_prep_launch(const InnerArgs<T>& a, const double* R, const double* rnorm_dev, cudaStream_t s) {
#define LP(NC) k_prep<T, NC><<<wave_grid((const void*)k_prep<T, NC>, a.ew_blocks), kThreads, 0, s>>>(a, R, rnorm_dev)
    ISIRA_NC_DISPATCH(a.c, LP);
#undef LP
}

template <typename T>
void inner_finalize_to(const InnerArgs<T>& a, double* Z, cudaStream_t s) {
    k_finalize<T><<<a.ew_blocks, kThreads, 0, s>>>(a, Z);
}

template <typename T>
void inner_opstats(const InnerArgs<T>& a, const T* x, cudaStream_t s) {
#define LS(NC) k_opstats<T, NC><<<wave_grid((const void*)k_opstats<T, NC>, a.ew_blocks), kThreads, 0, s>>>(a, x)
    ISIRA_NC_DISPATCH(a.c, LS);
#undef LS
}

template <typename T>
void gram_setup(const InnerArgs<T>& a, double* G_out, double* Cinv_out, double* partial, cudaStream_t s) {
    if (a.c <= 0) return;
    const size_t smem = sizeof(double) * (size_t)a.c * (kGramTile + 1);
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_gram<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * kCMax * (kGramTile + 1)));
    });
    k_gram<T><<<a.ew_blocks, kThreads, smem, s>>>(a, G_out, Cinv_out, partial, a.pstride);
}

template <typename T>
void copy_vcol(const double* src, T* dst, int64_t n, cudaStream_t s) {
    k_copy_vcol<T><<<608, kThreads, 0, s>>>(src, dst, n);
}

#define ISIRA_INSTANTIATE_INNER(T)                                                                        \
    template void inner_phase1<T>(const InnerArgs<T>&, int, cudaStream_t);                               \
    template void inner_apply<T>(const InnerArgs<T>&, int, cudaStream_t);                                \
    template void inner_gather_vec<T>(const InnerArgs<T>&, const T*, T*, int, const int*, cudaStream_t);   \
    template void ml_inner_prep<T>(const InnerArgs<T>&, const double*, const double*, cudaStream_t);      \
    template void ml_phase1<T>(const InnerArgs<T>&, cudaStream_t);                                       \
    template void ml_phase2a<T>(const InnerArgs<T>&, int, cudaStream_t);                                 \
    template void ml_project<T>(const InnerArgs<T>&, int, cudaStream_t);                                 \
    template void ml_phase2b<T>(const InnerArgs<T>&, int, cudaGraphConditionalHandle, int, cudaStream_t); \
    template void ml_phase2c<T>(const InnerArgs<T>&, int, cudaStream_t);                                 \
    template void inner_gather<T>(const InnerArgs<T>&, int, cudaStream_t);                               \
    template void inner_rows<T>(const InnerArgs<T>&, cudaStream_t);                                      \
    template void inner_phase2<T>(const InnerArgs<T>&, int, cudaStream_t);                               \
    template void inner_phase2_cond<T>(const InnerArgs<T>&, cudaGraphConditionalHandle, cudaStream_t);   \
    template void inner_prep_launch<T>(const InnerArgs<T>&, const double*, const double*, cudaStream_t); \
    template void inner_finalize_to<T>(const InnerArgs<T>&, double*, cudaStream_t);                      \
    template void inner_opstats<T>(const InnerArgs<T>&, const T*, cudaStream_t);                         \
    template void gram_setup<T>(const InnerArgs<T>&, double*, double*, double*, cudaStream_t);           \
    template void copy_vcol<T>(const double*, T*, int64_t, cudaStream_t);                                 \
    template cudaError_t inner_gather_attrs<T>(int);

}  // namespace isira
