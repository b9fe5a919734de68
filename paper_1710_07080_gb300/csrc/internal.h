// internal.h -- host-side interfaces between the translation units of libisira.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <vector>

#include "common.cuh"

namespace isira {

// host-side CUDA error propagation inside setup code
struct CudaFailure {
    cudaError_t e;
};
#define CUDA_OK(x)                                                   \
    do {                                                             \
        cudaError_t e_ = (x);                                        \
        if (e_ != cudaSuccess) throw ::isira::CudaFailure{e_};       \
    } while (0)

// ------------------------------------------------------------------ multilevel preconditioner (multilevel.cu)
template <typename T>
struct MlLevel {
    int64_t n = 0, nnz = 0;                   // rows; stored off-diagonal entries (levels >= 1)
    T* dinv = nullptr;                        // 1 / diagonal (0 at the trimmed vertex of level 0)
    int32_t* rp = nullptr;                    // level >= 1: CSR of the off-diagonal weights
    int32_t* ci = nullptr;
    T* w = nullptr;
    int32_t* agg = nullptr;                   // vertex -> cluster of the next level (-1: none)
    int64_t* mrp = nullptr;                   // members of each cluster of the next level
    int32_t* mem = nullptr;
    T* b = nullptr;                           // right-hand side of this level (levels >= 1)
    T* x0 = nullptr; T* x1 = nullptr; T* x = nullptr;   // work vectors
};

template <typename T>
struct MlHierarchy {
    int nlev = 0;
    int64_t n0 = 0, skip = -1, n_coarse = 0;
    std::vector<MlLevel<T>> lev;
    T* inv = nullptr;                         // dense inverse of the coarsest level
};

// g = sum over the neighbours of x (level 0), on stream s
template <typename T>
using GatherFn = std::function<void(const T* x, T* g, cudaStream_t s)>;

template <typename T>
cudaError_t ml_build(MlHierarchy<T>& H, const int64_t* d_rp, const int32_t* d_ci, const double* d_w, int64_t n,
                     int64_t ld, int64_t skip, cudaStream_t s);
template <typename T> void ml_free(MlHierarchy<T>& H);
// out = M^{-1} b, one V-cycle; kernels return at once while *done != 0 (done may be null)
template <typename T>
void ml_vcycle(MlHierarchy<T>& H, const T* b, T* out, const GatherFn<T>& gather, T omega, T alpha, const int* done,
               bool x0_ready, bool skip_post0, cudaStream_t s);
template <typename T> int ml_launches(const MlHierarchy<T>& H, bool x0_ready, bool skip_post0);

// ------------------------------------------------------------------ inner solve
// State of one preconditioned MINRES solve (Paige & Saunders 1975) kept in device
// memory: the Lanczos/Givens scalars, the c-vectors of the deflation terms, and the
// iteration counters.  Written only by the last block of a launch.
template <typename T>
struct InnerState {
    T beta;       // beta_k: v_k = z_k / beta_k
    T oldb;       // beta_{k-1}
    T alpha;      // alpha_k from phase 1
    T beta1;      // initial preconditioned residual norm
    T cs, sn, dbar, epsln, phibar;
    T w_oldeps, w_dlt, w_inv_gamma, w_phi;   // coefficients of the deferred w/x update
    T s_cur;                                 // sum(z_k)
    T g_cur[kCMax], g_prev[kCMax];           // Vh^T z_k, Vh^T z_{k-1}
    T u1[kCMax];                             // phase-1 coefficient of Vh_r (see inner_impl.cuh)
    T hv[kCMax];                             // multilevel path: Vh^T r_{k+1}
    T qv[kCMax];                             // phase-2: (alpha/beta) delta g_cur
    T tv[kCMax];                             // phase-2: SMW coefficient C^{-1} Vh^T D^{-1} y
    T p_sigma, p_sig_n;                      // shift and (sigma / n or 0) of the current solve
    int p_c;                                 // deflation rank of the current solve
    int itn, done, pending;
};

// Per-handle, per-precision buffers and parameters of the inner solve.
template <typename T>
struct InnerArgs {
    RowSched rs;
    int64_t trim;
    T sigma, sig_n, delta;      // sig_n = sigma / n, or 0 with drop_rank1
    const T* Vt;                // Vh in precision T, column-major, leading dim ldv
    int64_t ldv;
    int c;
    T* z0; T* z1; T* Y; T* wb0; T* wb1; T* wb2; T* x;
    T* dinv;                    // FP64 mode: 1/D per row, written by the prep kernel (nullptr: divide)
    T* gsum;                    // per-row neighbour sums written by the gather kernel
    const int32_t* deg;         // degree per row (ld entries, zero padding)
    T* partial; int pstride;
    unsigned* counter;
    InnerState<T>* st;
    HostStatus* hs;             // device alias of the mapped host status
    const double* Cinv;         // c-by-c inverse of C = delta^{-1} I + Vh^T D^{-1} Vh
    const double* Gm;           // c-by-c Vh^T D^{-1} Vh
    // multilevel preconditioner: stored Lanczos vectors, the projected V-cycle input, its output, and
    // D = diag(1 / (lambda_t - sigma + delta)) of the deflated directions (device, c doubles)
    T* rprev; T* rcur; T* rin; T* wv;
    T* ml_x0;                   // level 0's x0 = w D^{-1} rin, written by the projection kernel (or null)
    const T* ml_dinv0;          // level 0's 1 / diagonal
    T ml_omega;
    // level 0's post-smoothing done by phase 2b (ml_fuse_post): w = x1 + w D^{-1} (b - D x1 + W x1)
    // from the V-cycle input b, x1 and W x1
    int ml_fuse_post;
    const T* ml_b0; const T* ml_x1; const T* ml_wx1;
    const double* dv;
    double* partial_d;          // the partial-sum buffer viewed as doubles (FP64 Gram sums)
    T tau; int max_it;
    int ew_blocks;              // grid of the row-elementwise kernels
};

// Launchers (instantiated for float and double in inner_f32.cu / inner_f64.cu).
template <typename T> void inner_prep_launch(const InnerArgs<T>& a, const double* R, const double* rnorm_dev,
                                             cudaStream_t s);
template <typename T> void inner_phase1(const InnerArgs<T>& a, int lanes, cudaStream_t s);   // gather + rows
template <typename T> void inner_gather(const InnerArgs<T>& a, int lanes, cudaStream_t s);
// stand-alone operator apply: gather of z0, then Y = operator(z0) (after inner_opstats on z0)
template <typename T> void inner_apply(const InnerArgs<T>& a, int lanes, cudaStream_t s);
// every gather kernel of precision T may take up to `bytes` of dynamic shared memory
template <typename T> cudaError_t inner_gather_attrs(int bytes);
template <typename T> void inner_rows(const InnerArgs<T>& a, cudaStream_t s);
template <typename T> void inner_phase2(const InnerArgs<T>& a, int init, cudaStream_t s);
// phase 2 inside a CUDA graph whose WHILE node is driven by `cond` (set to 0 once the solve stops)
template <typename T> void inner_phase2_cond(const InnerArgs<T>& a, cudaGraphConditionalHandle cond,
                                             cudaStream_t s);
template <typename T> void inner_finalize_to(const InnerArgs<T>& a, double* Z, cudaStream_t s);
template <typename T> void inner_opstats(const InnerArgs<T>& a, const T* x, cudaStream_t s);
template <typename T> void gram_setup(const InnerArgs<T>& a, double* G_out, double* Cinv_out, double* scratch,
                                      cudaStream_t s);
template <typename T> void copy_vcol(const double* src, T* dst, int64_t n, cudaStream_t s);
// multilevel-preconditioned MINRES (inner_impl.cuh)
template <typename T> void inner_gather_vec(const InnerArgs<T>& a, const T* x, T* g, int lanes, const int* done,
                                            cudaStream_t s);
template <typename T> void ml_inner_prep(const InnerArgs<T>& a, const double* R, const double* rnorm_dev,
                                         cudaStream_t s);
template <typename T> void ml_phase1(const InnerArgs<T>& a, cudaStream_t s);
template <typename T> void ml_phase2a(const InnerArgs<T>& a, int init, cudaStream_t s);
template <typename T> void ml_project(const InnerArgs<T>& a, int init, cudaStream_t s);
template <typename T> void ml_phase2b(const InnerArgs<T>& a, int init, cudaGraphConditionalHandle cond, int has_cond,
                                      cudaStream_t s);
template <typename T> void ml_phase2c(const InnerArgs<T>& a, int init, cudaStream_t s);


// ------------------------------------------------------------------ outer loop (FP64)
struct OuterArgs {
    RowSched rs;
    double* gsum;               // per-row neighbour sums of the gather kernel
    int64_t n, ld;              // leading dimension of U, W, V
    double* U; double* W; double* V;
    double* H;                  // kMMax x kMMax, column-major, ld kMMax
    double* theta; double* S;   // Ritz values, Ritz vectors (ld kMMax)
    double* R;                  // residual n-vector
    double* Z;                  // expansion n-vector
    double* partial; int pstride;
    unsigned* counter;
    HostStatus* hs;
    double* dscratch;           // small device scratch (>= 4 * kMMax doubles)
    int ew_blocks;
    int ts_blocks;              // grid of the tall-skinny kernels
};

void outer_residual(const OuterArgs& a, int k, cudaStream_t s);
// warm_w > 0: S's leading warm_w x warm_w block holds eigenvectors of H's leading block (warm start)
void outer_sym_eig(const double* H, int ldh, int k, double* theta, double* S, int lds, HostStatus* hs, int warm_w,
                   cudaStream_t s);
// Rayleigh-Ritz after one expansion (outer.cu): with Q0 = S(0:w, 0:w) (+) 1 diagonalising H's
// leading w x w block, A = Q0^T H Q0 is an arrowhead matrix (diagonal D, last row and column z,
// corner alpha); its eigenvalues are the roots of the secular equation.  Device scratch:
struct ArrowWork {
    double d[kMMax];            // diagonal of A's leading block (after the deflating rotations)
    double z[kMMax];            // A's last column above the corner (zeroed where deflated)
    double offb[kMMax];         // per column of Q0: max |off-diagonal| of Q0^T H Q0
    double Q[kMMax * kMMax];    // Q0 with the deflating rotations applied (ld kMMax)
    double mu[kMMax + 1];       // root j = d[org[j]] + mu[j] (org[j] < 0: root j = mu[j])
    double zh[kMMax];           // z recomputed from the roots, per undeflated pole in ascending order
    double alpha, znorm;
    double rot_c[kMMax], rot_s[kMMax];
    int rot_p[kMMax], rot_q[kMMax];
    int pole[kMMax];            // undeflated indices in ascending order of d
    int defl[kMMax];            // deflated indices
    int org[kMMax + 1];
    int m, nd, nrot;
    int status;                 // 0 solved, 1 refused (Q0 does not diagonalise H's leading block)
    unsigned counter;           // arrival counter of the setup kernel (returns to 0)
};
// k >= 2 and w in {k-1, k}.  theta, S as outer_sym_eig.  On refusal (status 1, hs->eig_path -1)
// theta and S are left unspecified and the caller runs outer_sym_eig.
// off_cap: the largest off-diagonal entry of Q0^T H Q0 that may be dropped (besides the relative
// limit of a few rounding errors); launches returned in *launches.
void outer_arrow_eig(const double* H, int ldh, int k, int w, double* theta, double* S, int lds, ArrowWork* aw,
                     HostStatus* hs, double off_cap, int* launches, cudaStream_t s);
// Z <- Z - Q(Q^T Z) - mean(Z) twice, then ||Z||, for Q = [U(:,0:k) V(:,0:c)]; Z already holds the
// FP64 input.  Writes cgs_in / cgs_out to the host status.
void outer_cgs2(const OuterArgs& a, int k, int c, cudaStream_t s);
// U(:,k) = Z/||Z||, W(:,k) = L U(:,k), H(0:k, k) = U(:,0:k+1)^T W(:,k) (and the symmetric row).
void outer_expand(const OuterArgs& a, int k, int lanes, cudaStream_t s);
cudaError_t outer_gather_attrs(int bytes);
// resident gather CTAs per SM at tpb threads and hub_bytes of dynamic shared memory (0: error)
int gather_ctas_per_sm(int tpb, int hub_bytes);
// X(:, 0:ncol) <- X(:, 0:kk) S(:, c0:c0+ncol); with vout != NULL also vout = X S(:, 0).
void outer_rotate(const OuterArgs& a, double* X, int kk, int c0, int ncol, double* vout, cudaStream_t s);
// H <- diag(theta[c0 .. c0+cnt)) and S's leading cnt x cnt block <- I (after a restart)
void outer_set_diag(const OuterArgs& a, int c0, int cnt, cudaStream_t s);
// purge after a lock with a Householder reflection (U and W in place, H to P H P trimmed);
// vout receives the locked vector U s1 (S(:, 0) of the last Rayleigh-Ritz step); S's leading
// (k-1) x (k-1) block becomes the eigenvectors of the new H, (P S)(1:k, 1:k)
void outer_purge(const OuterArgs& a, int k, double* vout, cudaStream_t s);
// Z <- centred SplitMix64 vector, block `blk` of stream `seed`.
void outer_random(const OuterArgs& a, uint64_t seed, uint64_t blk, cudaStream_t s);
// out[j] = ||L V(:,j) - lam[j] V(:,j)||_2^2 for j < d (out is device, d doubles).
void outer_true_residual(const OuterArgs& a, int d, const double* lam_dev, double* out, int lanes,
                         cudaStream_t s);
// y = L x (FP64 full Laplacian), used to seed W(:,0).
void outer_laplacian(const OuterArgs& a, const double* x, double* y, int lanes, cudaStream_t s);

// setup
struct DegreeInfo { int64_t max_degree, argmax; int64_t n_long, n_items; };
// Counts (and, when item_row is given and n_items <= cap, fills) the long-row work items.
void setup_degrees(const int64_t* rp, int64_t n, int light_deg, int32_t* item_row, int32_t* item_k, int64_t cap,
                   int64_t* scratch, DegreeInfo* out, cudaStream_t s);
// deg[r] = row_ptr[r+1] - row_ptr[r] for r < n, 0 for n <= r < ld
void setup_deg32(const int64_t* rp, int64_t n, int64_t ld, int32_t* deg, cudaStream_t s);
// Equal-cost ranges of work units (items, then light tiles) for n_warps warps.
void setup_partition(const int64_t* rp, int64_t n, const int32_t* item_row, const int32_t* item_k, int64_t n_items,
                     int light_deg, int n_warps, int64_t* cost_tmp, int64_t* prefix_tmp, int32_t* warp_start,
                     cudaStream_t s);
// vertex relabelling by descending degree (reorder.cu)
// (weights w, if not null, follow their edges into w2)
cudaError_t build_reordered_graph(const int64_t* rp, const int32_t* ci, const double* w, int64_t n, int64_t nnz,
                                  int64_t maxdeg, int64_t* rp2, int32_t* ci2, double* w2, int32_t* perm, int32_t* inv,
                                  cudaStream_t s);
// sliced ELL copy of the light rows [light0, n): off (n_slices + 1 entries, caller-allocated) receives
// the slice offsets, *sci a new device array of *total entries (-1 padding)
cudaError_t build_sell(const int64_t* rp, const int32_t* ci, const double* w, int64_t n, int64_t light0,
                       int64_t n_slices, int64_t* off, int32_t** sci, double** sw, int64_t* total, cudaStream_t s);
// weighted degrees dw[r] = sum of the row's weights (r < n; 0 for n <= r < ld) and their FP32 copy;
// wf = FP32 copy of the nnz weights (either may be null)
void setup_weighted(const int64_t* rp, const double* w, int64_t n, int64_t ld, int64_t nnz, double* dw, float* dwf,
                    float* wf, cudaStream_t s);
template <typename T> void copy_cast(const double* src, T* dst, int64_t count, cudaStream_t s);
template <typename T> void to_internal(const T* src, const int32_t* perm, int64_t n, T* dst, cudaStream_t s);
template <typename T> void to_external(const T* src, const int32_t* perm, int64_t n, T* dst, cudaStream_t s);
int validate_csr(const int64_t* rp, const int32_t* ci, int64_t n, int64_t nnz, int* d_flag, cudaStream_t s);

}  // namespace isira
