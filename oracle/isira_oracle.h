/*
 * isira_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 CPU implementation of iSIRA
 * (Huang, Lin, Lu, Yau: "iSIRA: Integrated Shift-Invert Residual Arnoldi
 * Method for Graph Laplacian Matrices from Big Data", arXiv:1710.07080).
 * It exists to check the GPU library; it is not part of it.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg load it.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * Conventions: CSR adjacency pattern of a simple undirected graph,
 * row_ptr int64[n+1], col_idx int32[nnz], unit weights, no values array.
 * Dense matrices are column-major with leading dimension equal to their
 * row count.  All arithmetic is IEEE double.
 */
#ifndef ISIRA_ORACLE_H
#define ISIRA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Edge weights.  Every function below that takes `w` accepts either NULL (an unweighted graph:
 * every stored entry has weight 1, L = D - A of Eq. 1.1) or positive weights w[nnz] aligned with
 * col_idx and symmetric (w of (r, c) equals w of (c, r)): the weighted Laplacian L_w = D_w - W of
 * the Remark after Theorem 1.2, whose diagonal entry is the sum of the row's weights. */

/* y = L x with L = D - A (Eq. 1.1), or L_w x. */
void or_laplacian_apply(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* w,
                        const double* x, double* y);

/* All eigenpairs of a symmetric k-by-k matrix A by cyclic Jacobi rotations
 * (Golub & Van Loan, Matrix Computations, 4th ed., Sec. 8.5).  Eigenvalues
 * ascending in theta[k]; unit eigenvectors in the columns of S (k-by-k), each
 * signed so that its entry of largest magnitude (first one on ties) is
 * positive.  Returns the number of sweeps used, or -1 if it did not converge
 * in max_sweeps. */
int or_sym_eig(int k, const double* A, double* theta, double* S, int max_sweeps);

/* Dense definition oracle: all n eigenpairs of L (n <= a few hundred). */
int or_dense_laplacian_eig(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* w,
                           double* lam, double* X);

/* The trimmed, shifted, deflated operator of Theorem 2.6 (Eq. 2.14),
 *   yh = ((Lh - sigma*Ih) + (sigma/n) 1h 1h^T + delta Vh Vh^T) xh,
 * on (n-1)-vectors, where "h" quantities have row/column `trim` removed.
 * V is n-by-c (full rows; the trimmed row is skipped here).  drop_rank1 = 1
 * omits the (sigma/n) 1h 1h^T term (Remark 3.1). */
void or_trimmed_apply(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* w,
                      int64_t trim, double sigma, double delta, const double* V, int c, int drop_rank1,
                      const double* xh, double* yh);

/* Back-map of Theorem 2.4 (Eq. 2.5): zstar = [zh(1:i-1); 0; zh(i:n-1)] - (1h^T zh / n) 1. */
void or_backmap(int64_t n, int64_t trim, const double* zh, double* zstar);

/* Preconditioner of Remark 3.2 with a diagonal Mh_sigma ~ Lh - sigma Ih and the
 * Sherman-Morrison-Woodbury form of Eq. 3.6 when c > 0:  ph = P^{-1} xh. */
void or_precond_apply(int64_t n, const int64_t* row_ptr, const double* w, int64_t trim, double sigma,
                      double delta, const double* V, int c, const double* xh, double* ph);

/* Solve the trimmed system of Eq. 2.14 with preconditioned MINRES (Paige & Saunders 1975)
 * to relative preconditioned residual tau, then apply the back-map.  r is the
 * n-vector right-hand side; its trimmed row is dropped.  Returns iterations. */
int or_inner_solve(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* w,
                   int64_t trim, double sigma, double delta, const double* V, int c, int drop_rank1,
                   const double* r, double tau, int max_it, double* zstar, double* relres_out);

typedef struct {
    int d;              /* number of wanted eigenpairs */
    int m, q;           /* max search dimension, restart size (d <= q < m) */
    double eps;         /* convergence: ||r||_2 < eps */
    double sigma0;      /* initial shift (the paper uses 0) */
    int64_t trim;       /* trimmed index, 0-based; <0 = vertex of maximum degree (smallest id) */
    double delta;       /* deflation constant; <=0 = 2 * max degree */
    double omega;       /* shift move: sigma = theta2 - omega * (theta2 - lambda_j), kept >= 1% below theta2 */
    double tau_inner;   /* inner relative tolerance */
    int max_inner;      /* inner iteration cap */
    int max_outer;      /* outer iteration cap over all j */
    int drop_rank1;     /* 1 = Remark 3.1 variant */
    uint64_t seed;      /* seed of the breakdown-replacement vectors */
} or_params;

typedef struct {
    int status;         /* 0 ok, 1 no convergence (locked pairs kept), 2 bad argument */
    int n_locked;
    int outer_steps;
    long long inner_iters;
    int restarts;
    int breakdowns;
    int64_t trim;
    double delta;
    long long w_columns;   /* columns of W_k recomputed (W_k, H_k step), summed over outer steps */
    double sec_w;          /* wall seconds in the W_k, H_k step */
    double sec_inner;      /* wall seconds in the inner solves */
    double sec_total;      /* wall seconds of the whole call */
} or_stats;

/* Algorithm 2.  u0: unit n-vector orthogonal to 1 (the k0 = 1 start basis).
 * Outputs: lam[d] in locking order, V n-by-d (column-major). */
int or_isira(int64_t n, const int64_t* row_ptr, const int32_t* col_idx, const double* w,
             const double* u0, const or_params* p, double* lam, double* V, or_stats* st);

#ifdef __cplusplus
}
#endif
#endif
