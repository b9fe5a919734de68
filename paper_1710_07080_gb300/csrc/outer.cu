// outer.cu -- FP64 kernels of the outer loop of Algorithm 2 and of the setup.
//
//   residual      r = W s1 - theta1 U s1, ||r||                     (Algorithm 2, residual)
//   sym_eig       all eigenpairs of H_k, one CTA, parallel Jacobi    (Rayleigh-Ritz)
//   arrow_eig     the same after one expansion of a diagonalised H:   (Rayleigh-Ritz, warm start)
//                 secular equation of the arrowhead matrix
//   cgs2          classical Gram-Schmidt, two passes, against [U V 1] (orthonormalisation)
//   expand        U(:,k) = u, W(:,k) = L u, H(:,k) = U^T W(:,k)      (expansion)
//   rotate        X <- X S(:, a:b) in place, row tiles in shared memory (restart)
//   true_residual ||L v_j - lambda_j v_j||                           (final check)
//   setup         degrees, maximum degree and its vertex, row classes (Remark 4.1)
// The tall-skinny kernels stage a tile of basis rows in shared memory once and use
// it twice (row-wise update, column-wise dot products), so U and V are read once
// per Gram-Schmidt pass.
#include <algorithm>
#include <mutex>

#include "internal.h"

namespace isira {

// ------------------------------------------------------------------ residual

__global__ void __launch_bounds__(kThreads) k_residual(OuterArgs a, int k) {
    __shared__ double s1[kMMax];
    __shared__ double red[1];
    const double th = a.theta[0];
    for (int t = threadIdx.x; t < k; t += blockDim.x) s1[t] = a.S[t];
    __syncthreads();
    double acc[1] = {0.0};
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.n; r += (int64_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int t = 0; t < k; ++t) v += (a.W[(int64_t)t * a.ld + r] - th * a.U[(int64_t)t * a.ld + r]) * s1[t];
        a.R[r] = v;
        acc[0] += v * v;
    }
    if (block_partials_arrive<double, 1>(acc, 1, a.partial, a.pstride, a.counter)) {
        last_block_sum(a.partial, a.pstride, gridDim.x, 1, red, a.counter);
        if (threadIdx.x == 0) {
            const double rn = sqrt(red[0]);
            a.dscratch[0] = rn;
            a.hs->rnorm = rn;
            a.hs->theta[0] = a.theta[0];
            a.hs->theta[1] = k > 1 ? a.theta[1] : a.theta[0];
        }
    }
}

void outer_residual(const OuterArgs& a, int k, cudaStream_t s) {
    k_residual<<<a.ew_blocks, kThreads, 0, s>>>(a, k);
}

// ------------------------------------------------------------------ symmetric eigensolver (Rayleigh-Ritz)
// All eigenpairs of the small symmetric H_k in one CTA.  One SM's FP64 pipe is slow on this
// part, so the bulk of the work runs in FP32 and FP64 only finishes it:
//   1. parallel cyclic Jacobi in FP32 (round-robin ordering: in each of K-1 rounds the K
//      indices form K/2 disjoint pairs, rotated together; K = k rounded up to even) until the
//      off-diagonal norm is ~1e-6 of the matrix norm, accumulating Q;
//   2. in FP64: Q re-orthonormalised by two Newton-Schulz steps Q <- Q (3I - Q^T Q) / 2,
//      then B = Q^T H Q;
//   3. FP64 Jacobi sweeps on the nearly diagonal B until every off-diagonal entry is
//      negligible against its diagonal entries, accumulating into Q.
// Each rotation is the symmetric 2x2 Schur rotation of Golub & Van Loan Sec. 8.5.2; a round
// applies A <- J^T A J and Q <- Q J in one pass (every new entry from at most four old ones).
// Output: eigenvalues ascending, unit eigenvectors signed so that the entry of largest
// magnitude (first index on ties) is positive.

constexpr int kEigLd = kMMax + 1;
constexpr int kEigThreads = 256;         // one CTA (more threads only add barrier cost)

template <typename T>
struct JacobiSmem {
    T* A; T* A2; T* Q; T* Q2;       // [kMMax][kEigLd] each, column-major
    int* partner; T* alpha; T* beta; int* zero_pq;   // per index
    double* red;                    // [blockDim.x / 32]
};

template <typename T>
__device__ double jacobi_off(const T* A, int K, double* red) {
    double off = 0.0;
    for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) {
        const int i = idx % K, j = idx / K;
        if (i < j) off += 2.0 * (double)A[i + j * kEigLd] * (double)A[i + j * kEigLd];
    }
    off = warp_sum(off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = off;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    __syncthreads();
    return tot;
}

template <typename T>
__device__ double jacobi_frob(const T* A, int K, double* red) {
    double f = 0.0;
    for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) {
        const int i = idx % K, j = idx / K;
        f += (double)A[i + j * kEigLd] * (double)A[i + j * kEigLd];
    }
    f = warp_sum(f);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = f;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    __syncthreads();
    return tot;
}

// Sweeps until off(A)^2 <= stop2 (or, with drop_negligible, until all entries are dropped or
// rotated to zero).  A and Q ping-pong between (A, A2) and (Q, Q2); returns the sweeps used
// (-1: no convergence) and leaves the current buffers in sm.A / sm.Q.
template <typename T>
__device__ int jacobi_sweeps(JacobiSmem<T>& sm, int K, int max_sweeps, double stop2, bool drop_negligible) {
    const int tid = threadIdx.x;
    for (int sw = 0; sw < max_sweeps; ++sw) {
        const double off = jacobi_off(sm.A, K, sm.red);
        if (off == 0.0 || off <= stop2) return sw;
        for (int rnd = 0; rnd < K - 1; ++rnd) {
            if (tid < K / 2) {
                int p, q;
                if (tid == 0) { p = K - 1; q = rnd; }
                else { p = (rnd + tid) % (K - 1); q = (rnd - tid + (K - 1)) % (K - 1); }
                if (p > q) { const int t = p; p = q; q = t; }
                T c = T(1), s = T(0);
                int zero = 0;
                const T apq = sm.A[p + q * kEigLd];
                if (apq != T(0)) {
                    const T app = sm.A[p + p * kEigLd], aqq = sm.A[q + q * kEigLd];
                    const bool negligible = drop_negligible && fabs((double)app) + 100.0 * fabs((double)apq) == fabs((double)app) &&
                                            fabs((double)aqq) + 100.0 * fabs((double)apq) == fabs((double)aqq);
                    if (negligible) {
                        zero = 1;
                    } else {
                        const T tau = (aqq - app) / (T(2) * apq);
                        const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
                        c = T(1) / sqrt(T(1) + t * t);
                        s = t * c;
                        zero = 1;
                    }
                }
                // new column p = c col_p - s col_q, new column q = s col_p + c col_q
                sm.partner[p] = q; sm.alpha[p] = c; sm.beta[p] = -s; sm.zero_pq[p] = zero;
                sm.partner[q] = p; sm.alpha[q] = c; sm.beta[q] = s; sm.zero_pq[q] = zero;
            }
            __syncthreads();
            // A2 = J^T A J (upper triangle computed, mirrored), Q2 = Q J
            for (int idx = tid; idx < K * K; idx += blockDim.x) {
                const int i = idx % K, j = idx / K;
                const int pj = sm.partner[j];
                const T aj = sm.alpha[j], bj = sm.beta[j];
                if (i <= j) {
                    const int pi = sm.partner[i];
                    const T ai = sm.alpha[i], bi = sm.beta[i];
                    T v;
                    if (pi == j && sm.zero_pq[i]) {
                        v = T(0);
                    } else {
                        v = ai * (aj * sm.A[i + j * kEigLd] + bj * sm.A[i + pj * kEigLd]) +
                            bi * (aj * sm.A[pi + j * kEigLd] + bj * sm.A[pi + pj * kEigLd]);
                    }
                    sm.A2[i + j * kEigLd] = v;
                    sm.A2[j + i * kEigLd] = v;
                }
                sm.Q2[i + j * kEigLd] = aj * sm.Q[i + j * kEigLd] + bj * sm.Q[i + pj * kEigLd];
            }
            __syncthreads();
            T* t = sm.A; sm.A = sm.A2; sm.A2 = t;
            t = sm.Q; sm.Q = sm.Q2; sm.Q2 = t;
        }
    }
    return jacobi_off(sm.A, K, sm.red) == 0.0 ? max_sweeps : -1;
}

// C = op(X) * Y for K-by-K blocks in shared memory (ld kEigLd); op = transpose if tx.
__device__ void small_gemm(const double* X, const double* Y, double* C, int K, bool tx) {
    for (int idx = threadIdx.x; idx < K * K; idx += blockDim.x) {
        const int i = idx % K, j = idx / K;
        double s = 0.0;
        if (tx) for (int r = 0; r < K; ++r) s += X[r + i * kEigLd] * Y[r + j * kEigLd];
        else for (int r = 0; r < K; ++r) s += X[i + r * kEigLd] * Y[r + j * kEigLd];
        C[i + j * kEigLd] = s;
    }
    __syncthreads();
}

// warm_w > 0: S holds, in its leading warm_w x warm_w block, eigenvectors of H's leading block
// (from the previous outer step, or set by the purge / restart).  The kernel then works on
// A = Q0^T H Q0, Q0 = S(0:w, 0:w) (+) I, which is diagonal up to the rows and columns added since
// (an arrowhead after one expansion), and returns S = Q0 times A's eigenvectors.
__global__ void __launch_bounds__(kEigThreads) k_sym_eig(const double* H, int ldh, int k, double* theta, double* S,
                                                      int lds, HostStatus* hs, int warm_w) {
    extern __shared__ double eig_sm[];
    __shared__ int partner_[kMMax], zero_[kMMax], perm[kMMax];
    __shared__ double alpha_[kMMax], beta_[kMMax], red_[kEigThreads / 32];
    __shared__ float alphaf_[kMMax], betaf_[kMMax];
    const int K = k + (k & 1);
    const int tid = threadIdx.x;
    const int blk = kMMax * kEigLd;
    double* D0 = eig_sm;            // H (kept)
    double* D1 = eig_sm + blk;
    double* D2 = eig_sm + 2 * blk;
    double* D3 = eig_sm + 3 * blk;
    // FP32 phase buffers alias D2, D3 (unused until the FP64 phase)
    double* W5 = eig_sm + 4 * blk;  // warm-start basis Q0 (kept to the end)
    float* F = reinterpret_cast<float*>(D2);
    JacobiSmem<float> fs{F, F + blk, F + 2 * blk, F + 3 * blk, partner_, alphaf_, betaf_, zero_, red_};
    const int w0 = (warm_w > 0 && warm_w <= k && k >= 2) ? warm_w : 0;
    for (int idx = tid; idx < K * K; idx += blockDim.x) {
        const int i = idx % K, j = idx / K;
        D0[i + j * kEigLd] = (i < k && j < k) ? 0.5 * (H[i + j * ldh] + H[j + i * ldh]) : 0.0;
        if (w0) W5[i + j * kEigLd] = (i < w0 && j < w0) ? S[i + j * lds] : (i == j ? 1.0 : 0.0);
    }
    __syncthreads();
    if (w0) {
        small_gemm(D0, W5, D1, K, false);                          // T = H Q0
        small_gemm(W5, D1, D3, K, true);                           // A = Q0^T T
        for (int idx = tid; idx < K * K; idx += blockDim.x) {
            const int i = idx % K, j = idx / K;
            D0[i + j * kEigLd] = 0.5 * (D3[i + j * kEigLd] + D3[j + i * kEigLd]);
        }
        __syncthreads();
    }
    for (int idx = tid; idx < K * K; idx += blockDim.x) {
        const int i = idx % K, j = idx / K;
        fs.A[i + j * kEigLd] = (float)D0[i + j * kEigLd];
        fs.Q[i + j * kEigLd] = (i == j) ? 1.0f : 0.0f;
    }
    __syncthreads();
    int sweeps32 = 0, sweeps64 = 0;
    if (K >= 2) {
        const double frob = jacobi_frob(fs.A, K, red_);
        sweeps32 = jacobi_sweeps<float>(fs, K, 40, 4e-12 * frob, false);
        // FP64: Q from the FP32 rotations, re-orthonormalised (two Newton-Schulz steps)
        for (int idx = tid; idx < K * K; idx += blockDim.x) {
            const int i = idx % K, j = idx / K;
            D1[i + j * kEigLd] = (double)fs.Q[i + j * kEigLd];
        }
        __syncthreads();
        for (int it = 0; it < 2; ++it) {
            small_gemm(D1, D1, D2, K, true);                       // G = Q^T Q
            for (int idx = tid; idx < K * K; idx += blockDim.x) {   // G <- (3I - G) / 2
                const int i = idx % K, j = idx / K;
                D2[i + j * kEigLd] = ((i == j) ? 1.5 : 0.0) - 0.5 * D2[i + j * kEigLd];
            }
            __syncthreads();
            small_gemm(D1, D2, D3, K, false);                      // Q <- Q G
            for (int idx = tid; idx < K * K; idx += blockDim.x) {
                const int i = idx % K, j = idx / K;
                D1[i + j * kEigLd] = D3[i + j * kEigLd];
            }
            __syncthreads();
        }
        small_gemm(D0, D1, D2, K, false);                          // T = H Q
        small_gemm(D1, D2, D3, K, true);                           // B = Q^T T
        JacobiSmem<double> ds{D3, D2, D1, D0, partner_, alpha_, beta_, zero_, red_};
        sweeps64 = jacobi_sweeps<double>(ds, K, 12, 0.0, true);
        // eigenvalues on the diagonal of ds.A, eigenvectors in the columns of ds.Q (of A)
        double* Af = ds.A;
        double* Qf = ds.Q;
        if (w0) {
            // eigenvectors of H: Q0 times those of A, into a buffer the sweeps left free
            double* Fr = ds.A2 != Af && ds.A2 != Qf ? ds.A2 : ds.Q2;
            small_gemm(W5, Qf, Fr, K, false);
            Qf = Fr;
        }
        if (tid == 0) {
            for (int i = 0; i < k; ++i) perm[i] = i;
            for (int i = 0; i < k; ++i) {
                int best = i;
                for (int j = i + 1; j < k; ++j)
                    if (Af[perm[j] + perm[j] * kEigLd] < Af[perm[best] + perm[best] * kEigLd]) best = j;
                const int t = perm[best];
                for (int j = best; j > i; --j) perm[j] = perm[j - 1];
                perm[i] = t;
            }
            if (hs) {
                hs->eig_sweeps = (sweeps32 < 0 || sweeps64 < 0) ? -1 : sweeps32 + sweeps64;
                hs->eig_path = 0;
            }
        }
        __syncthreads();
        if (tid < k) {
            const int src = perm[tid];
            theta[tid] = Af[src + src * kEigLd];
            int imax = 0;
            for (int r = 1; r < k; ++r)
                if (fabs(Qf[r + src * kEigLd]) > fabs(Qf[imax + src * kEigLd])) imax = r;
            const double sg = Qf[imax + src * kEigLd] < 0.0 ? -1.0 : 1.0;
            for (int r = 0; r < k; ++r) S[r + tid * lds] = sg * Qf[r + src * kEigLd];
        }
        return;
    }
    // k == 1
    if (tid == 0) {
        theta[0] = D0[0];
        S[0] = 1.0;
        if (hs) { hs->eig_sweeps = 0; hs->eig_path = 0; }
    }
}

void outer_sym_eig(const double* H, int ldh, int k, double* theta, double* S, int lds, HostStatus* hs,
                   int warm_w, cudaStream_t s) {
    const int bytes = (int)(sizeof(double) * 5 * kMMax * kEigLd);
    static std::once_flag once;
    std::call_once(once, [bytes] { cudaFuncSetAttribute(k_sym_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes); });
    k_sym_eig<<<1, kEigThreads, bytes, s>>>(H, ldh, k, theta, S, lds, hs, warm_w);
}

// ------------------------------------------------------------------ Rayleigh-Ritz after one expansion
// H = [H0 h; h^T eta] where the previous step left Q0 with Q0^T H0 Q0 diagonal.  Then
// A = diag(Q0, 1)^T H diag(Q0, 1) = [D z; z^T alpha] (D = Q0^T H0 Q0, z = Q0^T h, alpha = eta) is an
// arrowhead matrix, and by the Schur complement its eigenvalues are the roots of the secular equation
//   f(lambda) = alpha - lambda - sum_i z_i^2 / (d_i - lambda),
// one between each pair of consecutive poles d_i and one beyond each end (interlacing).  Two kinds
// of deflation come first: a pole whose z_i is negligible is an eigenvalue with eigenvector e_i,
// and of two poles closer than the tolerance a plane rotation zeroes one z (the other absorbs it)
// so that one of them deflates.  The eigenvectors follow Gu and Eisenstat (SIAM J. Matrix Anal.
// Appl. 16:172-191, 1995): a vector zhat is recomputed from the computed roots by Loewner's
// formula, so the computed roots are the exact eigenvalues of the arrowhead with zhat, and the
// vectors (zhat_i / (d_i - lambda), -1) are numerically orthogonal however close the roots lie.
// The cost is O(k^2), against the O(k^3) per sweep of Jacobi; the work of each root and of each
// zhat entry runs on its own SM, because one SM's FP64 pipe is narrow on this part.
//   setup    one CTA per column i of Q0: one Newton-Schulz step q~_i = q_i (3/2) - Q0 Q0^T q_i / 2
//            (keeps the warm-start basis orthonormal over many steps), d_i = q~_i^T H0 q~_i,
//            z_i = q~_i^T h, and the largest |q_j^T H0 q~_i|, j != i; the last CTA deflates;
//   roots    one warp per root: safeguarded Newton, in coordinates centred on the nearer pole d_o,
//            on f(lambda) times the interval's end poles, from the root of a one-pole model,
//            bisection when a step leaves the bracket;
//   zhat     one warp per undeflated pole (Loewner's formula as a product of bounded ratios);
//   vectors  one CTA per eigenpair: the vector in the arrowhead basis, its place in ascending
//            order, S(:, place) = Q~ x with the sign rule of outer_sym_eig.
// Q0 must diagonalise H0 to rounding: if the largest off-diagonal entry exceeds a few rounding
// errors (or off_cap), the setup refuses (status 1) and the caller runs the Jacobi solver.

constexpr double kEpsD = 2.220446049250313e-16;   // unit roundoff x 2 (machine epsilon, binary64)
constexpr int kArrowThreads = 64;                 // >= kMMax: one thread per row of H
constexpr int kArrowMaxIt = 200;                  // iteration limit of one root (Newton ends in 3-15; the
                                                  // bracket test ends a run of bisection steps)
constexpr int kArrowLd = kMMax + 1;

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

__device__ __forceinline__ double warp_prod(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v *= __shfl_xor_sync(kFull, v, o);
    return v;
}

// Run by the last setup CTA: refusal test, ascending order, deflation, rotations of Q~.
__device__ void arrow_deflate(int k, int w, ArrowWork* aw, HostStatus* hs, double off_cap) {
    __shared__ double d[kMMax], z[kMMax];
    __shared__ int ord[kMMax];
    __shared__ double rm[3][kArrowThreads / 32];
    __shared__ int refused, nrot_s;
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    const bool arrow = w < k;
    double dv = 0.0, zv = 0.0, ov = 0.0;
    if (tid < w) {
        dv = __ldcg(aw->d + tid);
        zv = arrow ? __ldcg(aw->z + tid) : 0.0;
        ov = __ldcg(aw->offb + tid);
        d[tid] = dv;
        z[tid] = zv;
    }
    const double alpha = arrow ? __ldcg(&aw->alpha) : 0.0;
    double a = warp_max(fmax(fabs(dv), fabs(zv)));
    double o = warp_max(ov);
    double zq = warp_sum(zv * zv);
    if (lane == 0) { rm[0][wp] = a; rm[1][wp] = o; rm[2][wp] = zq; }
    __syncthreads();
    const double scale = fmax(fmax(rm[0][0], rm[0][1]), fabs(alpha));
    const double offmax = fmax(rm[1][0], rm[1][1]);
    if (tid == 0) {
        aw->counter = 0u;
        const double lim = fmin(4.0 * k * kEpsD * scale, off_cap);
        refused = !(offmax <= lim);                       // NaN refuses too
        aw->status = refused;
        aw->znorm = sqrt(rm[2][0] + rm[2][1]);
        if (hs) hs->eig_path = refused ? -1 : 1;
    }
    __syncthreads();
    if (refused) return;
    if (tid < w) {                                        // ascending order of d, ties by index
        int r = 0;
        for (int j = 0; j < w; ++j) r += (d[j] < dv) || (d[j] == dv && j < tid);
        ord[r] = tid;
    }
    __syncthreads();
    if (tid == 0) {
        const double tol = 8.0 * kEpsD * scale;
        int m = 0, nd = 0, nrot = 0, last = -1;
        for (int r = 0; r < w; ++r) {
            const int i = ord[r];
            if (!arrow || fabs(z[i]) <= tol) {            // z_i negligible: d_i is an eigenvalue
                aw->defl[nd++] = i;
                continue;
            }
            if (last >= 0 && d[i] - d[last] <= tol) {     // two poles within tol: rotate z_last away
                const double zp = z[last], zi = z[i];
                const double rr = hypot(zp, zi);
                const double c = zi / rr, sn = -zp / rr;
                const double dp = d[last], di = d[i];
                d[last] = c * c * dp + sn * sn * di;
                d[i] = sn * sn * dp + c * c * di;
                z[last] = 0.0;
                z[i] = rr;
                aw->rot_p[nrot] = last;
                aw->rot_q[nrot] = i;
                aw->rot_c[nrot] = c;
                aw->rot_s[nrot] = sn;
                ++nrot;
                aw->defl[nd++] = last;
                aw->pole[m - 1] = i;
            } else {
                aw->pole[m++] = i;
            }
            last = i;
        }
        aw->m = m;
        aw->nd = nd;
        aw->nrot = nrot;
        nrot_s = nrot;
    }
    __syncthreads();
    if (tid < w) {
        aw->d[tid] = d[tid];
        aw->z[tid] = z[tid];
        // columns p, q of Q~ <- (c q_p + s q_q, -s q_p + c q_q), in the order the rotations were made
        for (int t = 0; t < nrot_s; ++t) {
            const int p = aw->rot_p[t], q = aw->rot_q[t];
            const double c = aw->rot_c[t], sn = aw->rot_s[t];
            const double xp = __ldcg(aw->Q + tid + p * kMMax), xq = __ldcg(aw->Q + tid + q * kMMax);
            aw->Q[tid + p * kMMax] = c * xp + sn * xq;
            aw->Q[tid + q * kMMax] = -sn * xp + c * xq;
        }
    }
}

__global__ void __launch_bounds__(kArrowThreads) k_arrow_setup(const double* H, int ldh, int k, int w,
                                                            const double* S, int lds, ArrowWork* aw,
                                                            HostStatus* hs, double off_cap) {
    extern __shared__ double arrow_sm[];
    double* Qs = arrow_sm;                    // Q0, ld kArrowLd
    double* Hs = arrow_sm + kMMax * kArrowLd; // H (symmetrised), ld kArrowLd
    __shared__ double g[kMMax], qt[kMMax], t[kMMax];
    __shared__ double red[3][kArrowThreads / 32];
    __shared__ int is_last;
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5, i = blockIdx.x;
    for (int idx = tid; idx < w * w; idx += blockDim.x) {
        const int r = idx % w, c = idx / w;
        Qs[r + c * kArrowLd] = S[r + (int64_t)c * lds];
    }
    for (int idx = tid; idx < k * k; idx += blockDim.x) {
        const int r = idx % k, c = idx / k;
        Hs[r + c * kArrowLd] = H[r + (int64_t)c * ldh];
    }
    __syncthreads();
    for (int idx = tid; idx < k * k; idx += blockDim.x) {
        const int r = idx % k, c = idx / k;
        if (r < c) {
            const double v = 0.5 * (Hs[r + c * kArrowLd] + Hs[c + r * kArrowLd]);
            Hs[r + c * kArrowLd] = v;
            Hs[c + r * kArrowLd] = v;
        }
    }
    if (tid < w) {                                        // g = Q0^T q_i
        double acc = 0.0;
        for (int r = 0; r < w; ++r) acc += Qs[r + tid * kArrowLd] * Qs[r + i * kArrowLd];
        g[tid] = acc;
    }
    __syncthreads();
    if (tid < w) {                                        // q~_i = (3/2) q_i - (1/2) Q0 g
        double acc = 0.0;
        for (int j = 0; j < w; ++j) acc += Qs[tid + j * kArrowLd] * g[j];
        qt[tid] = 1.5 * Qs[tid + i * kArrowLd] - 0.5 * acc;
    }
    __syncthreads();
    if (tid < w) {                                        // t = H0 q~_i
        double acc = 0.0;
        for (int c = 0; c < w; ++c) acc += Hs[tid + c * kArrowLd] * qt[c];
        t[tid] = acc;
    }
    __syncthreads();
    double dd = 0.0, zz = 0.0, off = 0.0;
    if (tid < w) {
        dd = qt[tid] * t[tid];
        if (w < k) zz = qt[tid] * Hs[tid + w * kArrowLd];
        if (tid != i) {
            double acc = 0.0;
            for (int r = 0; r < w; ++r) acc += Qs[r + tid * kArrowLd] * t[r];
            off = fabs(acc);
        }
    }
    dd = warp_sum(dd);
    zz = warp_sum(zz);
    off = warp_max(off);
    if (lane == 0) { red[0][wp] = dd; red[1][wp] = zz; red[2][wp] = off; }
    if (tid < k) aw->Q[tid + i * kMMax] = tid < w ? qt[tid] : 0.0;
    if (i == 0 && w < k && tid < k) aw->Q[tid + w * kMMax] = tid == w ? 1.0 : 0.0;
    __syncthreads();
    if (tid == 0) {
        aw->d[i] = red[0][0] + red[0][1];
        aw->z[i] = red[1][0] + red[1][1];
        aw->offb[i] = fmax(red[2][0], red[2][1]);
        if (i == 0) aw->alpha = w < k ? Hs[w + w * kArrowLd] : 0.0;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) is_last = atomicAdd(&aw->counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    arrow_deflate(k, w, aw, hs, off_cap);
}

// One warp per root j = blockIdx.x (0..m).  Root j lies between poles p_{j-1} and p_j (p_{-1} = -inf,
// p_m = +inf).  With o the pole nearer to the root, f the interval's other end pole (none for the
// two outer intervals) and mu = lambda - d_o:
//   g(mu) = (alpha - d_o) - mu - S1(mu) + zeta_o / mu - zeta_f / (delta_f - mu),
//   S1 = sum_{i != o, f} zeta_i / (delta_i - mu),  S2 = sum_{i != o, f} zeta_i / (delta_i - mu)^2,
// zeta_i = z_i^2, delta_i = d_i - d_o.  Newton runs on F = (-mu)(delta_f - mu) g (h = -mu g without f),
// which has no pole inside the interval:
//   F = q r + zeta_o (mu - delta_f) + zeta_f mu,  q = mu^2 - delta_f mu,  r = (alpha - d_o) - mu - S1,
//   F' = (2 mu - delta_f) r - q (1 + S2) + zeta_o + zeta_f.
// g decreases through the root, so its sign keeps a bracket; steps that leave it are replaced by
// bisection.
__global__ void __launch_bounds__(32) k_arrow_roots(ArrowWork* aw) {
    if (aw->status) return;
    const int m = aw->m, j = blockIdx.x, lane = threadIdx.x;
    if (j > m) return;
    const double alpha = aw->alpha;
    if (m == 0) {
        if (lane == 0) { aw->org[0] = -1; aw->mu[0] = alpha; }
        return;
    }
    const int i0 = lane, i1 = lane + 32;
    const double p0 = i0 < m ? aw->d[aw->pole[i0]] : 0.0, p1 = i1 < m ? aw->d[aw->pole[i1]] : 0.0;
    const double z0 = i0 < m ? aw->z[aw->pole[i0]] : 0.0, z1 = i1 < m ? aw->z[aw->pole[i1]] : 0.0;
    const double zeta0 = z0 * z0, zeta1 = z1 * z1;
    auto pole_at = [&](int i) { return __shfl_sync(kFull, i < 32 ? p0 : p1, i & 31); };
    auto zeta_at = [&](int i) { return __shfl_sync(kFull, i < 32 ? zeta0 : zeta1, i & 31); };
    // S1, S2 over the poles other than o and f, centred on d_o (one reciprocal per pole)
    auto sums = [&](int o, int f, double po, double mu, double& s1, double& s2) {
        double a1 = 0.0, a2 = 0.0;
        if (i0 < m && i0 != o && i0 != f) {
            const double inv = 1.0 / ((p0 - po) - mu), q = zeta0 * inv;
            a1 += q;
            a2 += q * inv;
        }
        if (i1 < m && i1 != o && i1 != f) {
            const double inv = 1.0 / ((p1 - po) - mu), q = zeta1 * inv;
            a1 += q;
            a2 += q * inv;
        }
        s1 = warp_sum(a1);
        s2 = warp_sum(a2);
    };
    int o;
    double a, b;                                          // bracket of mu (endpoint 0 = the pole itself)
    if (j == 0) {
        o = 0;
        const double po = pole_at(0);
        a = fmin(0.0, alpha - po) - 1.0625 * aw->znorm;
        b = 0.0;
    } else if (j == m) {
        o = m - 1;
        const double po = pole_at(m - 1);
        a = 0.0;
        b = fmax(0.0, alpha - po) + 1.0625 * aw->znorm;
    } else {
        const double pl = pole_at(j - 1), pr = pole_at(j);
        const double half = 0.5 * (pr - pl);
        double s1, s2;
        sums(j - 1, -1, pl, half, s1, s2);
        const double gm = (alpha - pl) - half - s1 + zeta_at(j - 1) / half;
        if (gm > 0.0) { o = j; a = -half; b = 0.0; }      // root in (midpoint, p_j): centre on p_j
        else { o = j - 1; a = 0.0; b = half; }            // root in (p_{j-1}, midpoint]
    }
    const double po = pole_at(o), ao = alpha - po, zo = zeta_at(o);
    // interior intervals: f is the other end pole; Newton runs on F = (-mu)(delta_f - mu) g(mu), which
    // has neither pole of the interval; the outer intervals use h = -mu g(mu)
    const int f = (j > 0 && j < m) ? (o == j - 1 ? j : j - 1) : -1;
    const double df = f >= 0 ? pole_at(f) - po : 0.0, zf = f >= 0 ? zeta_at(f) : 0.0;
    // start at the root of the model with the other poles' sum frozen at mu = 0:
    // mu^2 - C mu - zeta_o = 0, C = (alpha - d_o) - S1(0) (- zeta_f / delta_f), taken on the bracket's side
    double mu;
    {
        double s1, s2;
        sums(o, f, po, 0.0, s1, s2);
        const double cc = ao - s1 - (f >= 0 ? zf / df : 0.0), sq = sqrt(cc * cc + 4.0 * zo);
        if (b == 0.0) mu = cc <= 0.0 ? 0.5 * (cc - sq) : -2.0 * zo / (cc + sq);
        else mu = cc >= 0.0 ? 0.5 * (cc + sq) : 2.0 * zo / (sq - cc);
        if (!(mu > a && mu < b)) mu = 0.5 * (a + b);
    }
    for (int it = 0; it < kArrowMaxIt; ++it) {
        double s1, s2;
        sums(o, f, po, mu, s1, s2);
        double gv, F, Fp;
        if (f >= 0) {
            gv = ao - mu - s1 + zo / mu - zf / (df - mu);
            const double q = mu * mu - df * mu, r = ao - mu - s1;
            F = q * r + zo * (mu - df) + zf * mu;
            Fp = (2.0 * mu - df) * r - q * (1.0 + s2) + zo + zf;
        } else {
            gv = ao - mu - s1 + zo / mu;
            F = -mu * ao + mu * mu + mu * s1 - zo;
            Fp = -ao + 2.0 * mu + s1 + mu * s2;
        }
        if (gv > 0.0) a = mu;
        else if (gv < 0.0) b = mu;
        else break;
        const double nw = mu - F / Fp;
        if (fabs(nw - mu) <= 4.0 * kEpsD * fabs(mu)) {      // Newton step of a few ulps: converged
            if (nw >= a && nw <= b) mu = nw;
            break;
        }
        const double nxt = (nw > a && nw < b) ? nw : 0.5 * (a + b);   // else bisection
        mu = nxt;
        if ((b - a) <= 4.0 * kEpsD * fmax(fabs(a), fabs(b))) break;
    }
    if (lane == 0) {
        aw->org[j] = aw->pole[o];
        aw->mu[j] = mu;
    }
}

// zhat_i for undeflated pole i = blockIdx.x (ascending order), one warp:
//   zhat_i^2 = -(lambda_i - p_i)(lambda_m - p_i) prod_{j < m, j != i} (lambda_j - p_i) / (p_j - p_i),
// each ratio positive and bounded by interlacing; lambda_j - p_i = (d_{org j} - p_i) + mu_j.
__global__ void __launch_bounds__(32) k_arrow_zhat(ArrowWork* aw) {
    if (aw->status) return;
    const int m = aw->m, i = blockIdx.x, lane = threadIdx.x;
    if (i >= m) return;
    const double pi = aw->d[aw->pole[i]];
    double pr = 1.0;
    for (int j = lane; j < m; j += 32) {
        if (j == i) continue;
        const double num = (aw->d[aw->org[j]] - pi) + aw->mu[j];
        const double den = aw->d[aw->pole[j]] - pi;
        pr *= num / den;
    }
    pr = warp_prod(pr);
    if (lane == 0) {
        const double li = (aw->d[aw->org[i]] - pi) + aw->mu[i];
        const double lm = (aw->d[aw->org[m]] - pi) + aw->mu[m];
        const double z2 = -li * lm * pr;
        aw->zh[i] = copysign(sqrt(fmax(z2, 0.0)), aw->z[aw->pole[i]]);
    }
}

// Eigenpair e = blockIdx.x: e < R = (arrow ? m + 1 : 0) is root e, else deflated index defl[e - R].
__global__ void __launch_bounds__(kArrowThreads) k_arrow_vectors(int k, int w, ArrowWork* aw, double* theta,
                                                              double* S, int lds, HostStatus* hs) {
    if (aw->status) return;
    __shared__ double lam[kMMax], x[kMMax];
    __shared__ double red[kArrowThreads / 32];
    __shared__ int cnt[kArrowThreads / 32], arg[kArrowThreads / 32];
    __shared__ double amax[kArrowThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5, e = blockIdx.x;
    const bool arrow = w < k;
    const int m = aw->m, R = arrow ? m + 1 : 0;
    if (tid < k) {
        double v;
        if (tid < R) { const int og = aw->org[tid]; v = og >= 0 ? aw->d[og] + aw->mu[tid] : aw->mu[tid]; }
        else v = aw->d[aw->defl[tid - R]];
        lam[tid] = v;
        x[tid] = 0.0;
    }
    __syncthreads();
    const double le = lam[e];
    int c = 0;
    if (tid < k) c = (lam[tid] < le) || (lam[tid] == le && tid < e);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if (lane == 0) cnt[wp] = c;
    // the vector in the arrowhead basis
    double xv = 0.0;
    if (e >= R) {
        if (tid == aw->defl[e - R]) xv = 1.0;
    } else if (m == 0) {
        if (tid == w) xv = 1.0;
    } else {
        const double de = aw->d[aw->org[e]], me = aw->mu[e];
        if (tid < m) xv = aw->zh[tid] / ((aw->d[aw->pole[tid]] - de) - me);
        else if (tid == m) xv = -1.0;
    }
    double ss = warp_sum(xv * xv);
    if (lane == 0) red[wp] = ss;
    __syncthreads();
    const int pos = cnt[0] + cnt[1];
    const double inv = 1.0 / sqrt(red[0] + red[1]);
    if (e >= R || m == 0) {
        if (xv != 0.0) x[tid] = xv;
    } else {
        if (tid < m) x[aw->pole[tid]] = xv * inv;
        else if (tid == m) x[w] = -inv;
    }
    __syncthreads();
    double y = 0.0;
    if (tid < k)
        for (int cc = 0; cc < k; ++cc) y += aw->Q[tid + cc * kMMax] * x[cc];
    // sign: the largest-magnitude entry (first on ties) positive
    double av = tid < k ? fabs(y) : -1.0;
    int ai = tid;
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(kFull, av, o);
        const int oi = __shfl_xor_sync(kFull, ai, o);
        if (ov > av || (ov == av && oi < ai)) { av = ov; ai = oi; }
    }
    if (lane == 0) { amax[wp] = av; arg[wp] = ai; }
    __syncthreads();
    const int im = (amax[1] > amax[0]) ? arg[1] : arg[0];
    __shared__ double ysel;
    if (tid == im) ysel = y;
    __syncthreads();
    const double sg = ysel < 0.0 ? -1.0 : 1.0;
    if (tid < k) S[tid + (int64_t)pos * lds] = sg * y;
    if (tid == 0) {
        theta[pos] = le;
        if (hs && e == 0) hs->eig_sweeps = 0;
    }
}

void outer_arrow_eig(const double* H, int ldh, int k, int w, double* theta, double* S, int lds, ArrowWork* aw,
                     HostStatus* hs, double off_cap, int* launches, cudaStream_t s) {
    const int bytes = (int)(sizeof(double) * 2 * kMMax * kArrowLd);
    static std::once_flag once;
    std::call_once(once, [bytes] { cudaFuncSetAttribute(k_arrow_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes); });
    k_arrow_setup<<<w, kArrowThreads, bytes, s>>>(H, ldh, k, w, S, lds, aw, hs, off_cap);
    int nl = 1;
    if (w < k) {
        k_arrow_roots<<<w + 1, 32, 0, s>>>(aw);
        k_arrow_zhat<<<w, 32, 0, s>>>(aw);
        nl += 2;
    }
    k_arrow_vectors<<<k, kArrowThreads, 0, s>>>(k, w, aw, theta, S, lds, hs);
    if (launches) *launches = nl + 1;
}

// ------------------------------------------------------------------ tall-skinny passes (orthonormalisation, H column)

constexpr int kTsRows = 64;              // rows per shared-memory tile
constexpr int kTsMaxCols = kMMax + kCMax;
constexpr int kTsColsPerWarp = (kTsMaxCols + kWarps - 1) / kWarps;

// MODE 0: dots only:      out = [Q^T z, 1^T z, z^T z]
// MODE 1: update + dots:  z <- z - Q h - mu 1, written back; out = [Q^T z, 1^T z]
// MODE 2: update + norm:  as MODE 1, out = [z^T z]
// Q = [U(:, 0:k) V(:, 0:c)].  coef = [h (k + c), mu].  The last block turns the sums
// into the coefficients of the next pass (coef_next) or into the final norm.
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_tall_skinny(OuterArgs a, int k, int c, const double* z_in,
                                                          double* z_out, const double* coef, double* coef_next,
                                                          double* Hcol, int hcol) {
    extern __shared__ double tsm[];
    const int nq = k + c;
    double* Qs = tsm;                           // [nq][kTsRows]
    double* zs = tsm + (size_t)nq * kTsRows;    // [kTsRows]
    double* hs = zs + kTsRows;                  // [nq + 1]
    __shared__ double red[kTsMaxCols + 2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (MODE != 0)
        for (int j = tid; j <= nq; j += blockDim.x) hs[j] = coef[j];
    const int nv = (MODE == 0) ? nq + 2 : (MODE == 1 ? nq + 1 : 1);
    double acc[kTsColsPerWarp + 2];
#pragma unroll
    for (int i = 0; i < kTsColsPerWarp + 2; ++i) acc[i] = 0.0;
    for (int64_t r0 = (int64_t)blockIdx.x * kTsRows; r0 < a.n; r0 += (int64_t)gridDim.x * kTsRows) {
        __syncthreads();
        for (int idx = tid; idx < nq * kTsRows; idx += blockDim.x) {
            const int j = idx / kTsRows, rr = idx % kTsRows;
            const int64_t r = r0 + rr;
            const double* col = j < k ? a.U + (int64_t)j * a.ld : a.V + (int64_t)(j - k) * a.ld;
            Qs[idx] = r < a.n ? col[r] : 0.0;
        }
        for (int rr = tid; rr < kTsRows; rr += blockDim.x) {
            const int64_t r = r0 + rr;
            zs[rr] = r < a.n ? z_in[r] : 0.0;
        }
        __syncthreads();
        if (MODE != 0) {
            // four threads per row split the columns, then combine with shuffles
            const int rr = tid >> 2, part = tid & 3;
            double s = 0.0;
            for (int j = part; j < nq; j += 4) s += Qs[j * kTsRows + rr] * hs[j];
            s += __shfl_xor_sync(kFull, s, 1);
            s += __shfl_xor_sync(kFull, s, 2);
            __syncthreads();
            if (part == 0) {
                const int64_t r = r0 + rr;
                const double zn = (r < a.n) ? zs[rr] - s - hs[nq] : 0.0;
                zs[rr] = zn;
                if (r < a.n) z_out[r] = zn;
            }
            __syncthreads();
        }
        if (MODE == 2) {
            for (int rr = tid; rr < kTsRows; rr += blockDim.x) acc[0] += zs[rr] * zs[rr];
        } else {
#pragma unroll
            for (int i = 0; i < kTsColsPerWarp; ++i) {
                const int j = warp + i * kWarps;
                if (j < nq) {
                    double s = 0.0;
                    for (int rr = lane; rr < kTsRows; rr += 32) s += Qs[j * kTsRows + rr] * zs[rr];
                    acc[i] += s;
                }
            }
            if (warp == 0)
                for (int rr = lane; rr < kTsRows; rr += 32) acc[kTsColsPerWarp] += zs[rr];
            if (MODE == 0 && warp == 1)
                for (int rr = lane; rr < kTsRows; rr += 32) acc[kTsColsPerWarp + 1] += zs[rr] * zs[rr];
        }
    }
    // gather the per-warp column sums into a per-thread vector of nv slots, then reduce
    __shared__ double bsum[kTsMaxCols + 2];
    __syncthreads();
    if (MODE == 2) {
        double v = block_sum0(acc[0]);
        if (tid == 0) bsum[0] = v;
    } else {
#pragma unroll
        for (int i = 0; i < kTsColsPerWarp; ++i) {
            const int j = warp + i * kWarps;
            double v = warp_sum(acc[i]);
            if (lane == 0 && j < nq) bsum[j] = v;
        }
        double v = warp_sum(acc[kTsColsPerWarp]);
        if (warp == 0 && lane == 0) bsum[nq] = v;
        if (MODE == 0) {
            double w = warp_sum(acc[kTsColsPerWarp + 1]);
            if (warp == 1 && lane == 0) bsum[nq + 1] = w;
        }
    }
    __syncthreads();
    for (int i = tid; i < nv; i += blockDim.x) a.partial[(size_t)i * a.pstride + blockIdx.x] = bsum[i];
    __threadfence();
    __syncthreads();
    __shared__ int last;
    if (tid == 0) last = (atomicAdd(a.counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    last_block_sum(a.partial, a.pstride, gridDim.x, nv, red, a.counter);
    const double inv_n = 1.0 / (double)a.n;
    if (MODE == 0 && Hcol != nullptr) {
        // H(0:nq, hcol) and the symmetric row from the dots U^T w
        for (int j = tid; j < nq; j += blockDim.x) {
            Hcol[j + (int64_t)hcol * kMMax] = red[j];
            Hcol[hcol + (int64_t)j * kMMax] = red[j];
        }
        return;
    }
    if (MODE == 0 || MODE == 1) {
        for (int j = tid; j < nq; j += blockDim.x) coef_next[j] = red[j];
        if (tid == 0) {
            coef_next[nq] = red[nq] * inv_n;
            if (MODE == 0) {
                const double zin = sqrt(red[nq + 1]);
                a.dscratch[1] = zin;
                a.hs->cgs_in = zin;
            }
        }
    } else if (tid == 0) {
        const double nz = sqrt(red[0]);
        a.dscratch[2] = nz;
        a.hs->cgs_out = nz;
    }
}

static void ts_smem_attr() {
    static std::once_flag once;
    std::call_once(once, [] {
        const int bytes = (int)(sizeof(double) * ((size_t)kTsMaxCols * kTsRows + kTsRows + kTsMaxCols + 1));
        cudaFuncSetAttribute(k_tall_skinny<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        cudaFuncSetAttribute(k_tall_skinny<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        cudaFuncSetAttribute(k_tall_skinny<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    });
}

// One launch wave: at most SMs x resident CTAs (registers and dynamic shared memory decide the
// latter), so a tile loop never runs as a full wave plus a partial one.
static int wave_of(const void* fn, size_t smem, int want) {
    static int nsm_of[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return want;
    if (nsm_of[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return want;
        nsm_of[dev] = v;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kThreads, smem) != cudaSuccess || nb < 1) return want;
    const int cap = nb * nsm_of[dev];
    return want < cap ? want : cap;
}

static size_t ts_smem(int nq) { return sizeof(double) * ((size_t)nq * kTsRows + kTsRows + nq + 1); }

void outer_cgs2(const OuterArgs& a, int k, int c, cudaStream_t s) {
    ts_smem_attr();
    const int nq = k + c;
    double* cA = a.dscratch + 8;                 // coefficients of pass B
    double* cB = a.dscratch + 8 + kTsMaxCols + 1; // coefficients of pass C
    const size_t sm = ts_smem(nq);
    k_tall_skinny<0><<<wave_of((const void*)k_tall_skinny<0>, sm, a.ts_blocks), kThreads, sm, s>>>(
        a, k, c, a.Z, nullptr, nullptr, cA, nullptr, 0);
    k_tall_skinny<1><<<wave_of((const void*)k_tall_skinny<1>, sm, a.ts_blocks), kThreads, sm, s>>>(
        a, k, c, a.Z, a.Z, cA, cB, nullptr, 0);
    k_tall_skinny<2><<<wave_of((const void*)k_tall_skinny<2>, sm, a.ts_blocks), kThreads, sm, s>>>(
        a, k, c, a.Z, a.Z, cB, nullptr, nullptr, 0);
}

// ------------------------------------------------------------------ expand

// Plain gather g[r] = sum_{c in N(r)} x[c] over the full Laplacian (no trimmed row).
template <int G, int TPB>
__global__ void __launch_bounds__(TPB, TPB == kThreads ? 4 : 1) k_gather_plain(RowSched rs, const double* x, double* g) {
    GatherStore<double> epi{g};
    for_each_row_gather<double, G>(rs, x, epi, -1);
}

// U(:,k) = Z / ||Z||, W(:,k) = L U(:,k) from the gathered sums of Z
__global__ void __launch_bounds__(kThreads) k_expand_rows(OuterArgs a, int k) {
    const double nz = a.dscratch[2];
    const double inv = nz > 0.0 ? 1.0 / nz : 0.0;
    double* u = a.U + (int64_t)k * a.ld;
    double* w = a.W + (int64_t)k * a.ld;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.n; r += (int64_t)gridDim.x * blockDim.x) {
        const double ur = a.Z[r] * inv;
        u[r] = ur;
        w[r] = row_degree<double>(a.rs, r) * ur - a.gsum[r] * inv;
    }
}

__global__ void __launch_bounds__(kThreads) k_laplacian_rows(OuterArgs a, const double* x, double* y) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.n; r += (int64_t)gridDim.x * blockDim.x)
        y[r] = row_degree<double>(a.rs, r) * x[r] - a.gsum[r];
}

__global__ void __launch_bounds__(kThreads, kSliceBlocksPerSM) k_gather_plain_s(RowSched rs, const double* x, double* g) {
    GatherStore<double> epi{g};
    slices_only_gather<double>(rs, x, epi, -1);
}

static void outer_gather(const OuterArgs& a, const double* x, int lanes, cudaStream_t s) {
    if (slices_only(a.rs)) {
        static int nsm = 0;
        if (nsm == 0) {
            int dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                nsm = 152;
        }
        const int64_t want = ((int64_t)a.rs.n_slices + kWarps - 1) / kWarps;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)nsm * kSliceBlocksPerSM));
        k_gather_plain_s<<<grid, kThreads, 0, s>>>(a.rs, x, a.gsum);
        return;
    }
#define LG(G, TPB) k_gather_plain<G, TPB><<<a.rs.grid(), TPB, a.rs.hub_bytes, s>>>(a.rs, x, a.gsum)
    ISIRA_GATHER_DISPATCH(lanes, a.rs.tpb, LG);
#undef LG
}

cudaError_t outer_gather_attrs(int bytes) {
    cudaError_t e = cudaSuccess;
#define LA(G, TPB)                                                                                      \
    if (e == cudaSuccess)                                                                               \
        e = cudaFuncSetAttribute(k_gather_plain<G, TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
    for (int tpb : {kThreads, kBigBlock})
        for (int g : {1, 2, 4, 8, 16, 32}) ISIRA_GATHER_DISPATCH(g, tpb, LA);
#undef LA
    return e;
}

int gather_ctas_per_sm(int tpb, int hub_bytes) {
    int nb = 0;
    cudaError_t e = tpb == kBigBlock
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gather_plain<1, kBigBlock>, kBigBlock, hub_bytes)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gather_plain<1, kThreads>, kThreads, hub_bytes);
    return e == cudaSuccess ? nb : 0;
}

void outer_expand(const OuterArgs& a, int k, int lanes, cudaStream_t s) {
    ts_smem_attr();
    outer_gather(a, a.Z, lanes, s);
    k_expand_rows<<<a.ew_blocks, kThreads, 0, s>>>(a, k);
    // H(0:k+1, k) = U(:, 0:k+1)^T W(:, k)
    k_tall_skinny<0><<<wave_of((const void*)k_tall_skinny<0>, ts_smem(k + 1), a.ts_blocks), kThreads,
                       ts_smem(k + 1), s>>>(a, k + 1, 0, a.W + (int64_t)k * a.ld, nullptr,
                                                                   nullptr, nullptr, a.H, k);
}

void outer_laplacian(const OuterArgs& a, const double* x, double* y, int lanes, cudaStream_t s) {
    outer_gather(a, x, lanes, s);
    k_laplacian_rows<<<a.ew_blocks, kThreads, 0, s>>>(a, x, y);
}

// ------------------------------------------------------------------ rotate (restart, purge)

constexpr int kRotRows = 64;

__global__ void __launch_bounds__(kThreads) k_rotate(OuterArgs a, double* X, int kk, int c0, int ncol, double* vout) {
    extern __shared__ double rsm[];
    double* Xs = rsm;                           // [kk][kRotRows]
    double* Ss = rsm + (size_t)kk * kRotRows;   // [kk][ncol + 1]: S(:, c0..c0+ncol-1) then S(:, 0)
    const int tid = threadIdx.x;
    const int nsc = ncol + 1;
    for (int idx = tid; idx < kk * nsc; idx += blockDim.x) {
        const int i = idx % kk, b = idx / kk;
        const int scol = b < ncol ? c0 + b : 0;
        Ss[i + b * kk] = a.S[i + scol * kMMax];
    }
    const int nout = ncol + (vout ? 1 : 0);
    for (int64_t r0 = (int64_t)blockIdx.x * kRotRows; r0 < a.n; r0 += (int64_t)gridDim.x * kRotRows) {
        __syncthreads();
        for (int idx = tid; idx < kk * kRotRows; idx += blockDim.x) {
            const int j = idx / kRotRows, rr = idx % kRotRows;
            const int64_t r = r0 + rr;
            Xs[idx] = r < a.n ? X[(int64_t)j * a.ld + r] : 0.0;
        }
        __syncthreads();
        for (int idx = tid; idx < nout * kRotRows; idx += blockDim.x) {
            const int b = idx / kRotRows, rr = idx % kRotRows;
            const int64_t r = r0 + rr;
            if (r >= a.n) continue;
            const double* sc = Ss + (size_t)b * kk;
            double v = 0.0;
            for (int i = 0; i < kk; ++i) v += Xs[i * kRotRows + rr] * sc[i];
            if (b < ncol) X[(int64_t)b * a.ld + r] = v;
            else vout[r] = v;
        }
    }
}

void outer_rotate(const OuterArgs& a, double* X, int kk, int c0, int ncol, double* vout, cudaStream_t s) {
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_rotate, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * ((size_t)kMMax * kRotRows + (size_t)kMMax * (kMMax + 1))));
    });
    const size_t smem = sizeof(double) * ((size_t)kk * kRotRows + (size_t)kk * (ncol + 1));
    k_rotate<<<wave_of((const void*)k_rotate, smem, a.ts_blocks), kThreads, smem, s>>>(a, X, kk, c0, ncol, vout);
}

// ------------------------------------------------------------------ purge after a lock
// The purge keeps span U minus the locked Ritz direction U s1.  Any orthonormal basis of that
// space gives the same later Ritz pairs, so instead of the k x (k-1) product U S(:, 2:k) the
// solver applies the Householder reflection P = I - beta v v^T, v = s1 + sign(s1[0]) e1, which
// maps s1 to -sign(s1[0]) e1: the first column of U P is -sign(s1[0]) U s1 (the locked vector)
// and columns 2..k of U P span the rest.  Per row that is 2k FMAs instead of k(k-1).  The
// projected matrix becomes the trailing (k-1) x (k-1) block of P H P (its first row and column
// vanish because s1 is an eigenvector of H).  Scratch: beta, sign and v in dscratch[400 ..].
constexpr int kPurgeSlot = 400;

__global__ void __launch_bounds__(kThreads) k_purge_prep(OuterArgs a, int k) {
    __shared__ double Hs[kMMax][kMMax + 1];
    __shared__ double v[kMMax], w[kMMax];
    __shared__ double beta_s, gamma_s;
    const int tid = threadIdx.x;
    const double s0 = a.S[0];
    const double sgn = s0 >= 0.0 ? 1.0 : -1.0;
    for (int i = tid; i < k; i += blockDim.x) v[i] = a.S[i] + (i == 0 ? sgn : 0.0);
    for (int idx = tid; idx < k * k; idx += blockDim.x) {
        const int i = idx % k, j = idx / k;
        Hs[i][j] = 0.5 * (a.H[i + j * kMMax] + a.H[j + i * kMMax]);
    }
    if (tid == 0) beta_s = 1.0 / (1.0 + fabs(s0));       // 2 / (v^T v) for a unit s1
    __syncthreads();
    for (int i = tid; i < k; i += blockDim.x) {
        double t = 0.0;
        for (int j = 0; j < k; ++j) t += Hs[i][j] * v[j];
        w[i] = t;
    }
    __syncthreads();
    if (tid == 0) {
        double g = 0.0;
        for (int j = 0; j < k; ++j) g += v[j] * w[j];
        gamma_s = g;
        a.dscratch[kPurgeSlot] = beta_s;
        a.dscratch[kPurgeSlot + 1] = -sgn;
    }
    for (int i = tid; i < k; i += blockDim.x) a.dscratch[kPurgeSlot + 2 + i] = v[i];
    __syncthreads();
    // P H P = H - beta v w^T - beta w v^T + beta^2 gamma v v^T; keep rows/columns 1..k-1
    const double b = beta_s, bg = beta_s * beta_s * gamma_s;
    for (int idx = tid; idx < (k - 1) * (k - 1); idx += blockDim.x) {
        const int i = idx % (k - 1) + 1, j = idx / (k - 1) + 1;
        const double h = Hs[i][j] - b * (v[i] * w[j] + w[i] * v[j]) + bg * v[i] * v[j];
        a.H[(i - 1) + (j - 1) * kMMax] = h;
    }
    // eigenvectors of the new H: (P S)(1:k, 1:k), P S = S - beta v (v^T S) (warm start of the
    // next Rayleigh-Ritz step); S is read whole into shared memory before it is overwritten
    __syncthreads();
    for (int idx = tid; idx < k * k; idx += blockDim.x) {
        const int i = idx % k, j = idx / k;
        Hs[i][j] = a.S[i + j * kMMax];
    }
    __syncthreads();
    for (int j = tid; j < k; j += blockDim.x) {
        double t = 0.0;
        for (int i = 0; i < k; ++i) t += v[i] * Hs[i][j];
        w[j] = t;                                          // (v^T S)_j
    }
    __syncthreads();
    for (int idx = tid; idx < (k - 1) * (k - 1); idx += blockDim.x) {
        const int i = idx % (k - 1) + 1, j = idx / (k - 1) + 1;
        a.S[(i - 1) + (j - 1) * kMMax] = Hs[i][j] - b * v[i] * w[j];
    }
}

// X(r, 0:k) <- (X P)(r, 1:k) in place, one thread per row; vout[r] = -sign(s1[0]) (X P)(r, 0)
__global__ void __launch_bounds__(kThreads) k_purge_rows(OuterArgs a, double* X, double* Y, int k, double* vout) {
    __shared__ double v[kMMax];
    const double* ps = a.dscratch + kPurgeSlot;
    for (int i = threadIdx.x; i < k; i += blockDim.x) v[i] = ps[2 + i];
    __syncthreads();
    const double beta = ps[0], sg = ps[1];
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.n; r += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll 1
        for (int m = 0; m < 2; ++m) {
            double* Z = m == 0 ? X : Y;
            if (!Z) continue;
            double y = 0.0;
            for (int j = 0; j < k; ++j) y += Z[(int64_t)j * a.ld + r] * v[j];
            const double by = beta * y;
            if (m == 0 && vout) vout[r] = sg * (Z[r] - by * v[0]);
            for (int j = 1; j < k; ++j) Z[(int64_t)(j - 1) * a.ld + r] = Z[(int64_t)j * a.ld + r] - by * v[j];
        }
    }
}

void outer_purge(const OuterArgs& a, int k, double* vout, cudaStream_t s) {
    k_purge_prep<<<1, kThreads, 0, s>>>(a, k);
    k_purge_rows<<<wave_of((const void*)k_purge_rows, 0, a.ew_blocks), kThreads, 0, s>>>(a, a.U, a.W, k, vout);
}

// after a restart U S(:, c0 : c0+cnt) is the Ritz basis: H is diagonal and its eigenvectors
// (the warm start of the next Rayleigh-Ritz step) are the identity
__global__ void k_set_diag(double* H, const double* theta, double* S, int c0, int cnt) {
    for (int idx = threadIdx.x; idx < kMMax * kMMax; idx += blockDim.x) {
        const int i = idx % kMMax, j = idx / kMMax;
        H[idx] = (i == j && i < cnt) ? theta[c0 + i] : 0.0;
        if (i < cnt && j < cnt) S[idx] = i == j ? 1.0 : 0.0;
    }
}

void outer_set_diag(const OuterArgs& a, int c0, int cnt, cudaStream_t s) {
    k_set_diag<<<1, kThreads, 0, s>>>(a.H, a.theta, a.S, c0, cnt);
}

__global__ void k_random(double* Z, int64_t n, uint64_t seed, uint64_t blk) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        Z[r] = 2.0 * uniform_at(seed, blk * (uint64_t)n + (uint64_t)r) - 1.0;
}

void outer_random(const OuterArgs& a, uint64_t seed, uint64_t blk, cudaStream_t s) {
    k_random<<<a.ew_blocks, kThreads, 0, s>>>(a.Z, a.n, seed, blk);
}

// ------------------------------------------------------------------ true residual

// ||L v - lambda v||^2 from the gathered sums of v
__global__ void __launch_bounds__(kThreads) k_trueres_rows(OuterArgs a, const double* v, const double* lam_dev, int j,
                                                           double* out) {
    __shared__ double red[1];
    const double lam = lam_dev[j];
    double acc[1] = {0.0};
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.n; r += (int64_t)gridDim.x * blockDim.x) {
        const double d = row_degree<double>(a.rs, r) * v[r] - a.gsum[r] - lam * v[r];
        acc[0] += d * d;
    }
    if (block_partials_arrive<double, 1>(acc, 1, a.partial, a.pstride, a.counter)) {
        last_block_sum(a.partial, a.pstride, gridDim.x, 1, red, a.counter);
        if (threadIdx.x == 0) out[j] = red[0];
    }
}

void outer_true_residual(const OuterArgs& a, int d, const double* lam_dev, double* out, int lanes, cudaStream_t s) {
    for (int j = 0; j < d; ++j) {
        const double* v = a.V + (int64_t)j * a.ld;
        outer_gather(a, v, lanes, s);
        k_trueres_rows<<<a.ew_blocks, kThreads, 0, s>>>(a, v, lam_dev, j, out);
    }
}

// ------------------------------------------------------------------ setup (Remark 4.1)

constexpr int kSetupBlocks = 1024;

__device__ __forceinline__ int64_t items_of(int64_t deg, int light_deg) {
    return deg > light_deg ? (deg + kItemNnz - 1) / kItemNnz : 0;
}

// per block: max degree + smallest argmax over its row chunk, long rows and their work items
__global__ void __launch_bounds__(kThreads) k_deg_count(const int64_t* rp, int64_t n, int64_t chunk, int light_deg,
                                                        int64_t* sc) {
    const int64_t beg = (int64_t)blockIdx.x * chunk;
    const int64_t end = beg + chunk < n ? beg + chunk : n;
    int64_t best = -1, barg = 0, nl = 0, ni = 0;
    for (int64_t r = beg + threadIdx.x; r < end; r += blockDim.x) {
        const int64_t d = rp[r + 1] - rp[r];
        if (d > best) { best = d; barg = r; }
        const int64_t q = items_of(d, light_deg);
        nl += q > 0;
        ni += q;
    }
    __shared__ int64_t sb[kThreads], sa[kThreads], sl[kThreads], si[kThreads];
    sb[threadIdx.x] = best; sa[threadIdx.x] = barg; sl[threadIdx.x] = nl; si[threadIdx.x] = ni;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const int q = threadIdx.x + o;
            if (sb[q] > sb[threadIdx.x] || (sb[q] == sb[threadIdx.x] && sa[q] < sa[threadIdx.x])) {
                sb[threadIdx.x] = sb[q];
                sa[threadIdx.x] = sa[q];
            }
            sl[threadIdx.x] += sl[q];
            si[threadIdx.x] += si[q];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sc[blockIdx.x] = sb[0];
        sc[kSetupBlocks + blockIdx.x] = sa[0];
        sc[2 * kSetupBlocks + blockIdx.x] = sl[0];
        sc[3 * kSetupBlocks + blockIdx.x] = si[0];
    }
}

// one thread: totals, max/argmax (smallest id on ties), exclusive prefix of the item counts
__global__ void k_deg_scan(int64_t* sc, int nb) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t best = -1, barg = 0, nl = 0, oi = 0;
    for (int b = 0; b < nb; ++b) {
        const int64_t d = sc[b], r = sc[kSetupBlocks + b];
        if (d > best || (d == best && r < barg)) { best = d; barg = r; }
        nl += sc[2 * kSetupBlocks + b];
        const int64_t m = sc[3 * kSetupBlocks + b];
        sc[3 * kSetupBlocks + b] = oi;
        oi += m;
    }
    sc[4 * kSetupBlocks + 0] = best;
    sc[4 * kSetupBlocks + 1] = barg;
    sc[4 * kSetupBlocks + 2] = nl;
    sc[4 * kSetupBlocks + 3] = oi;
}

// ordered fill of the work items: each block walks its chunk in tiles of blockDim rows and
// places the items of a tile with a block-wide exclusive scan of the per-row item counts
__global__ void __launch_bounds__(kThreads) k_deg_fill(const int64_t* rp, int64_t n, int64_t chunk, int light_deg,
                                                       const int64_t* sc, int32_t* item_row, int32_t* item_k) {
    const int64_t beg = (int64_t)blockIdx.x * chunk;
    const int64_t end = beg + chunk < n ? beg + chunk : n;
    int64_t off = sc[3 * kSetupBlocks + blockIdx.x];
    __shared__ int64_t wsum[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t t0 = beg; t0 < end; t0 += blockDim.x) {
        const int64_t r = t0 + threadIdx.x;
        const int64_t cnt = r < end ? items_of(rp[r + 1] - rp[r], light_deg) : 0;
        int64_t v = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(kFull, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) wsum[warp] = v;
        __syncthreads();
        if (warp == 0) {
            int64_t w = lane < kWarps ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t t = __shfl_up_sync(kFull, w, o);
                if (lane >= o) w += t;
            }
            if (lane < kWarps) wsum[lane] = w;
        }
        __syncthreads();
        const int64_t excl = v - cnt + (warp > 0 ? wsum[warp - 1] : 0);
        for (int64_t q = 0; q < cnt; ++q) {
            item_row[off + excl + q] = (int32_t)r;
            item_k[off + excl + q] = (int32_t)q;
        }
        off += wsum[kWarps - 1];
        __syncthreads();
    }
}

void setup_degrees(const int64_t* rp, int64_t n, int light_deg, int32_t* item_row, int32_t* item_k, int64_t cap,
                   int64_t* scratch, DegreeInfo* out, cudaStream_t s) {
    const int64_t chunk = (n + kSetupBlocks - 1) / kSetupBlocks;
    k_deg_count<<<kSetupBlocks, kThreads, 0, s>>>(rp, n, chunk, light_deg, scratch);
    k_deg_scan<<<1, 32, 0, s>>>(scratch, kSetupBlocks);
    int64_t tot[4];
    cudaMemcpyAsync(tot, scratch + 4 * kSetupBlocks, sizeof(tot), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    out->max_degree = tot[0];
    out->argmax = tot[1];
    out->n_long = tot[2];
    out->n_items = tot[3];
    if (item_row && tot[3] <= cap)
        k_deg_fill<<<kSetupBlocks, kThreads, 0, s>>>(rp, n, chunk, light_deg, scratch, item_row, item_k);
}

// degree of every row as int32 (the row kernels read 4 bytes per row instead of two row pointers);
// rows n .. ld-1 get 0
__global__ void __launch_bounds__(kThreads) k_deg32(const int64_t* rp, int64_t n, int64_t ld, int32_t* deg) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < ld; r += (int64_t)gridDim.x * blockDim.x)
        deg[r] = r < n ? (int32_t)(rp[r + 1] - rp[r]) : 0;
}

void setup_deg32(const int64_t* rp, int64_t n, int64_t ld, int32_t* deg, cudaStream_t s) {
    k_deg32<<<1024, kThreads, 0, s>>>(rp, n, ld, deg);
}

// weighted Laplacian: degrees as weight sums (FP64 and FP32), FP32 copy of the weights
__global__ void __launch_bounds__(kThreads) k_weighted_degrees(const int64_t* rp, const double* w, int64_t n, int64_t ld,
                                                               double* dw, float* dwf) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < ld; r += (int64_t)gridDim.x * blockDim.x) {
        double sum = 0.0;
        if (r < n)
            for (int64_t e = rp[r]; e < rp[r + 1]; ++e) sum += w[e];
        dw[r] = sum;
        if (dwf) dwf[r] = (float)sum;
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_copy_cast(const double* src, T* dst, int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (T)src[i];
}

template <typename T>
void copy_cast(const double* src, T* dst, int64_t count, cudaStream_t s) {
    k_copy_cast<T><<<2048, kThreads, 0, s>>>(src, dst, count);
}
template void copy_cast<float>(const double*, float*, int64_t, cudaStream_t);
template void copy_cast<double>(const double*, double*, int64_t, cudaStream_t);

void setup_weighted(const int64_t* rp, const double* w, int64_t n, int64_t ld, int64_t nnz, double* dw, float* dwf,
                    float* wf, cudaStream_t s) {
    k_weighted_degrees<<<1024, kThreads, 0, s>>>(rp, w, n, ld, dw, dwf);
    if (wf) copy_cast<float>(w, wf, nnz, s);
}

// ------------------------------------------------------------------ balanced work partition

__global__ void __launch_bounds__(kThreads) k_unit_cost(const int64_t* rp, int64_t n, const int32_t* item_row,
                                                        const int32_t* item_k, int64_t n_items, int64_t n_units,
                                                        int light_deg, int64_t* cost) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n_units; u += (int64_t)gridDim.x * blockDim.x) {
        int64_t c;
        if (u < n_items) {
            const int64_t r = item_row[u];
            const int64_t rb = rp[r], re = rp[r + 1];
            const int64_t beg = rb + (int64_t)item_k[u] * kItemNnz;
            const int64_t end = beg + kItemNnz < re ? beg + kItemNnz : re;
            c = (end - beg) + kItemCost;
        } else {
            const int64_t t = u - n_items;
            c = 0;
            for (int64_t r = t * 32; r < t * 32 + 32 && r < n; ++r) {
                const int64_t d = rp[r + 1] - rp[r];
                c += d <= light_deg ? d + kTileRowCost : 1;
            }
        }
        cost[u] = c;
    }
}

// exclusive prefix sum of N values in one CTA: prefix[0..N]
__global__ void __launch_bounds__(kThreads) k_scan_costs(const int64_t* cost, int64_t N, int64_t* prefix) {
    __shared__ int64_t part[kThreads];
    const int64_t chunk = (N + blockDim.x - 1) / blockDim.x;
    const int64_t b = threadIdx.x * chunk;
    const int64_t e = b + chunk < N ? b + chunk : N;
    int64_t s = 0;
    for (int64_t u = b; u < e; ++u) s += cost[u];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        for (int q = 0; q < (int)blockDim.x; ++q) {
            const int64_t v = part[q];
            part[q] = acc;
            acc += v;
        }
        prefix[N] = acc;
    }
    __syncthreads();
    int64_t acc = part[threadIdx.x];
    for (int64_t u = b; u < e; ++u) {
        prefix[u] = acc;
        acc += cost[u];
    }
}

// warp w starts at the first unit whose prefix reaches w * total / W
__global__ void k_warp_starts(const int64_t* prefix, int64_t N, int W, int32_t* ws) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w > W) return;
    if (w == W) { ws[W] = (int32_t)N; return; }
    const int64_t total = prefix[N];
    const int64_t target = (int64_t)(((__int128)total * w) / W);
    int64_t lo = 0, hi = N;                                  // first u in [0, N] with prefix[u] >= target
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (prefix[mid] < target) lo = mid + 1; else hi = mid;
    }
    ws[w] = (int32_t)lo;
}

void setup_partition(const int64_t* rp, int64_t n, const int32_t* item_row, const int32_t* item_k, int64_t n_items,
                     int light_deg, int n_warps, int64_t* cost_tmp, int64_t* prefix_tmp, int32_t* warp_start,
                     cudaStream_t s) {
    const int64_t n_units = n_items + (n + 31) / 32;
    k_unit_cost<<<1024, kThreads, 0, s>>>(rp, n, item_row, item_k, n_items, n_units, light_deg, cost_tmp);
    k_scan_costs<<<1, kThreads, 0, s>>>(cost_tmp, n_units, prefix_tmp);
    k_warp_starts<<<(n_warps + 1 + kThreads - 1) / kThreads, kThreads, 0, s>>>(prefix_tmp, n_units, n_warps,
                                                                              warp_start);
}

// flag bits: 1 row_ptr not monotone / bad ends, 2 column out of range, 4 self loop,
// 8 columns not strictly increasing (duplicates), 16 asymmetric pattern
__global__ void __launch_bounds__(kThreads) k_validate(const int64_t* rp, const int32_t* ci, int64_t n, int64_t nnz,
                                                       int* flag) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = rp[r], e = rp[r + 1];
        if (b > e || b < 0 || e > nnz || (r == 0 && b != 0) || (r == n - 1 && e != nnz)) {
            atomicOr(flag, 1);
            continue;
        }
        for (int64_t q = b; q < e; ++q) {
            const int64_t col = ci[q];
            if (col < 0 || col >= n) { atomicOr(flag, 2); continue; }
            if (col == r) atomicOr(flag, 4);
            if (q > b && ci[q - 1] >= col) atomicOr(flag, 8);
            // symmetric: r must appear in row col (binary search, rows are sorted)
            int64_t lo = rp[col], hi = rp[col + 1] - 1;
            bool found = false;
            while (lo <= hi && lo >= 0 && hi < nnz) {
                const int64_t mid = (lo + hi) >> 1;
                const int64_t v = ci[mid];
                if (v == r) { found = true; break; }
                if (v < r) lo = mid + 1; else hi = mid - 1;
            }
            if (!found) atomicOr(flag, 16);
        }
    }
}

int validate_csr(const int64_t* rp, const int32_t* ci, int64_t n, int64_t nnz, int* d_flag, cudaStream_t s) {
    cudaMemsetAsync(d_flag, 0, sizeof(int), s);
    k_validate<<<1216, kThreads, 0, s>>>(rp, ci, n, nnz, d_flag);
    int h = 0;
    cudaMemcpyAsync(&h, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    return h;
}

}  // namespace isira
