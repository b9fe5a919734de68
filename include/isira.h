/*
 * isira.h -- C ABI of the GB300 (sm_103a) iSIRA eigensolver for graph Laplacians.
 *
 * Problem (paper Sec. 1.1 and Sec. 2, Eq. 2.1; Algorithm 2 REQUIRE/ENSURE): given a
 * simple, connected, undirected, unweighted graph with Laplacian L = D - A (Eq. 1.1),
 * find the d smallest positive eigenvalues of L and orthonormal eigenvectors, with
 * the integrated shift-invert residual Arnoldi method (Algorithm 2): an FP64 outer
 * Rayleigh-Ritz loop whose expansion vectors come from inexact solves of the
 * trimmed, shifted, deflated system of Theorem 2.6 (Eq. 2.14) followed by the
 * back-map of Theorem 2.4 (Eq. 2.5).
 *
 * Conventions shared by every entry point
 *  - Graphs are CSR adjacency patterns in DEVICE memory: row_ptr int64[n+1]
 *    (row_ptr[0] == 0, non-decreasing, row_ptr[n] == nnz), col_idx int32[nnz], each
 *    row's columns sorted ascending, the pattern symmetric, with no self loops and
 *    no duplicates.  There is no values array: every edge has weight 1 and the
 *    degree of vertex r is row_ptr[r+1] - row_ptr[r].  The caller owns the CSR; it
 *    must stay alive and unmodified until isira_destroy.
 *  - Vertex indices are 0-based.  Dense device matrices are column-major with
 *    leading dimension n.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  All
 *    work of a handle is ordered on the stream given to isira_create.  Calls that
 *    return host results (isira_solve, isira_eigpairs) synchronise that stream.
 *  - The library owns all workspace (allocated in isira_create / isira_solve, freed
 *    in isira_destroy).  No entry point throws; errors are returned as isira_status.
 *  - A handle is not thread safe: use one handle per host thread.
 */
#ifndef ISIRA_H
#define ISIRA_H

#include <stdint.h>

#if defined(__GNUC__)
#define ISIRA_API __attribute__((visibility("default")))
#else
#define ISIRA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct isira_handle_s* isira_handle;

typedef enum {
    ISIRA_OK = 0,
    ISIRA_ERR_INVALID_ARG = 1,     /* a pointer, size or option is out of range */
    ISIRA_ERR_BAD_GRAPH = 2,       /* validate=1 found a malformed CSR pattern */
    ISIRA_ERR_NOT_CONNECTED = 3,   /* a second (near) zero eigenvalue was locked */
    ISIRA_ERR_NO_CONVERGENCE = 4,  /* max_outer reached; already locked pairs are kept */
    ISIRA_ERR_CUDA = 5,            /* a CUDA runtime call failed */
    ISIRA_ERR_OOM = 6,             /* device or pinned allocation failed */
    ISIRA_ERR_NOT_SOLVED = 7,      /* eigpairs requested before a successful solve */
    ISIRA_ERR_LIMIT = 8,           /* request exceeds the fixed scratch of isira_apply_operator_noalloc */
    ISIRA_ERR_DEVICE_TIMEOUT = 9   /* a bounded wait inside a kernel ran out; the call's results are not
                                      valid (the device context stays usable) */
} isira_status;

enum { ISIRA_FP64 = 0,   /* inner solve in FP64 ("plain") */
       ISIRA_MIXED = 1   /* inner solve in FP32 with FP32 accumulation, outer loop FP64 */ };

typedef struct {
    int precision;        /* ISIRA_FP64 or ISIRA_MIXED */
    int m, q;             /* search-space limit and restart size (Algorithm 2, d <= q < m <= 64);
                             0 = m = max(20, 2d+10), q = max(d+2, m/2) */
    double tau_inner;     /* inner relative (preconditioned) residual target; <= 0: 1e-3 */
    int max_inner;        /* inner iteration cap per solve; <= 0: 5000 */
    int max_outer;        /* outer iteration cap over all eigenpairs; <= 0: 20000 */
    int64_t trim_index;   /* trimmed vertex i (Theorem 2.3); < 0: vertex of maximum degree,
                             smallest id on ties (Remark 4.1(i)) */
    double delta;         /* deflation constant (Eq. 2.6); <= 0: 2 * max degree (Remark 4.1(ii)) */
    double sigma_omega;   /* after locking lambda_j: sigma = theta2 - max(omega*(theta2 - lambda_j),
                             0.01*theta2) (Algorithm 2 "move sigma ~ theta2"); <= 0: 0.1 */
    int drop_rank1;       /* 1: omit (sigma/n) 1h 1h^T from the inner operator (Remark 3.1) */
    int validate;         /* 1: check the CSR pattern on the device in isira_create */
    uint64_t seed;        /* SplitMix64 seed of replacement vectors after an orthogonalisation
                             breakdown and of the default start vector */
    int spmv_lanes;       /* lanes per row of the light-row SpMV (1,2,4,8,16,32); <= 0: autotune */
    int inner_chunk;      /* chunked mode: inner iterations launched between convergence checks; <= 0: 16 */
    int inner_graph;      /* 1: each inner solve is one CUDA-graph launch whose WHILE node repeats the
                             iteration until the device-side stopping test fires (no host round trip);
                             0: chunked launches with a host check after each chunk */
    int reorder;          /* 1: relabel the vertices internally by descending degree (stable), which
                             packs the vectors' entries of high-degree vertices together for cache
                             reuse in the SpMV; vectors at the API stay in the caller's numbering;
                             0: use the caller's numbering (default 1) */
    int gather_block;     /* threads per CTA of the SpMV gather kernels: 256 (as many CTAs per SM as
                             registers and shared memory allow, at most 8) or 1024 (one CTA per
                             SM); 0: autotuned (timed at create on graphs with n >= 100000, cached
                             per graph-statistics bucket; else 1024 with relabelling, 256 without) */
    int hub_kb;           /* with relabelling, each gather CTA copies the vector entries of the first
                             (highest-degree) vertices into this many KB of shared memory with one
                             bulk asynchronous copy; 0: autotuned among 192 KB (1024-thread CTAs),
                             48 KB (256-thread CTAs) and none; < 0: none */
    int gather_sched;     /* 0: gather warps take work units from a device counter as they finish
                             (balanced whatever the row costs); 1: a static partition by estimated
                             cost (CSR tiles only: ignored with sell = 1).  Results are identical
                             either way. */
    int index_vec;        /* 1: with relabelling, read column indices in 128-bit chunks of the
                             solver's padded copy; 0: 32-bit loads (default) */
    int gather_chunk;     /* work units a gather warp takes at a time (1..32); 0: 2 */
    int sell;             /* 1 (default): with relabelling, the rows of degree <= 64 are gathered from a
                             sliced ELL copy (slices of 32 rows, column-major, so every index load
                             of a warp is one 128-byte line); 0: from CSR tiles with spmv_lanes
                             lanes per row.  Sums differ only by rounding order. */
    int precond;          /* preconditioner of the inner solve (Remark 3.2):
                             0: the diagonal D = diag(max(deg - sigma, deg / 2)), with the deflation
                             term by Sherman-Morrison-Woodbury (Eq. 3.6);
                             1: an aggregation multilevel preconditioner M of the trimmed Laplacian
                             (greedy aggregation, Galerkin coarse Laplacians, one symmetric V-cycle
                             with damped Jacobi smoothing), standing in for combinatorial multigrid,
                             deflated by projection: inv(P) = Pi inv(M) Pi + Vh diag(1/(lambda - sigma +
                             delta)) Vh^T, Pi = I - Vh Vh^T;
                             -1 (default): automatic: on graphs with n >= 20000 and maximum degree
                             <= 64, one timed inner solve with each at create, the faster is kept;
                             the diagonal elsewhere */
    double ml_alpha;      /* multilevel: over-correction factor of the coarse-grid correction; <= 0: 1.5 */
    int rr_arrow;         /* 1 (default): after one expansion of a diagonalised H, solve the
                             Rayleigh-Ritz step as an arrowhead eigenproblem (secular equation,
                             see isira_sym_eig_warm); 0: parallel Jacobi at every step */
    int blocking_sync;    /* 1: the calling thread sleeps while it waits for the GPU (a blocking-sync
                             event) instead of spinning, so many solver threads can share few cores
                             (the batch calls set it); 0 (default): spin, the lowest wake-up latency */
} isira_opts;

typedef struct {
    int64_t n, nnz;
    int64_t trim_index;       /* the vertex actually trimmed */
    int64_t max_degree;
    double delta;             /* the deflation constant actually used */
    double norm_L;            /* Gershgorin bound 2 * max degree, used to scale residuals */
    int spmv_lanes;           /* chosen light-row lanes per row */
    int64_t n_long_rows;      /* rows above the light-row degree threshold */
    int64_t n_work_items;     /* warp work items the long rows are cut into */
    int n_locked;             /* eigenpairs locked by the last solve */
    int outer_steps;          /* Algorithm 2 while-loop iterations */
    int restarts, breakdowns;
    long long inner_iters;    /* total MINRES iterations */
    long long inner_solves;
    long long spmv_launches;  /* launches of the inner operator's gather kernel (phase 1) */
    double solve_ms;          /* host wall time of the last isira_solve */
    double inner_phase1_ms;   /* summed device time of the phase-1 gather launches (profiling on only) */
    long long inner_phase1_timed; /* number of phase-1 gather launches timed */
    long long inner_phase1_csum;  /* sum of the deflation rank c over the timed phase-1 launches */
    long long kernel_launches;    /* kernels launched by the last isira_solve */
    int gather_block;             /* threads per gather CTA in use */
    int hub_bytes;                /* shared memory of a gather CTA holding hub vector entries */
    long long hub_timeouts;       /* gather CTAs whose staging copy missed its wait limit (the call
                                     that saw one returned ISIRA_ERR_DEVICE_TIMEOUT) */
    double inner_rows_ms;         /* summed device time of the phase-1 row kernels (profiling on only) */
    double inner_phase2_ms;       /* summed device time of the phase-2 kernels (profiling on only) */
    long long w_columns;          /* sum over outer steps of the search-space size k: the columns of
                                     W_k = (L + delta V V^T) U_k that Algorithm 2 as printed recomputes */
    long long sell_entries;       /* stored entries (with padding) of the sliced ELL copy (0: none) */
    double max_diag;              /* largest diagonal entry of L (the maximum degree; the maximum
                                     weighted degree for isira_create_weighted) */
    int precond;                  /* preconditioner in use: 0 diagonal, 1 multilevel */
    int ml_levels;                /* levels of the multilevel hierarchy in use (0: none) */
    double precond_probe_ms[2];   /* automatic choice: the timed inner solve with the diagonal and with
                                     the multilevel preconditioner (0: not probed) */
    int rr_arrow;                 /* Rayleigh-Ritz steps of the last solve done by the arrowhead path */
    int rr_jacobi;                /* ... done by parallel Jacobi (first steps, refusals, rr_arrow = 0) */
    int rr_refused;               /* arrowhead attempts refused because Q0^T H Q0 was not diagonal to
                                     rounding (each then ran Jacobi) */
    long long ml_coarse_n;        /* multilevel: vertices of the levels below the finest, summed */
    long long ml_coarse_nnz;      /* multilevel: stored off-diagonal entries of those levels, summed */
} isira_stats;

/* Fills *opts with the defaults listed above (precision = ISIRA_MIXED). */
ISIRA_API void isira_default_opts(isira_opts* opts);

/* Human-readable name of a status code (static string). */
ISIRA_API const char* isira_error_string(isira_status s);

/* Creates a solver for the graph (d_row_ptr, d_col_idx) with n vertices and nnz
 * stored adjacency entries (twice the number of edges).  Runs the setup of
 * Remark 4.1 on the device (degrees, maximum degree, trimmed index, delta) and picks
 * the SpMV layout.  opts may be NULL (defaults).  Requires n >= 3.  On success *out
 * receives a handle to release with isira_destroy; on failure *out is NULL. */
ISIRA_API isira_status isira_create(isira_handle* out, int64_t n, int64_t nnz, const int64_t* d_row_ptr,
                          const int32_t* d_col_idx, const isira_opts* opts, void* stream);

/* Same as isira_create for the weighted Laplacian L_w = D_w - W of a graph with positive edge
 * weights (paper Sec. 1.1, the Remark after Theorem 1.2): d_weights is a device double[nnz] aligned
 * with d_col_idx, symmetric (the two stored entries of an edge carry the same weight) and
 * positive; it is borrowed like the CSR.  The diagonal entry of L_w is the row's weight sum; the
 * trimmed vertex is the one with the largest such entry (smallest id on ties) and delta = 2 x that
 * entry (Remark 4.1); norm_L (stats) is 2 x that entry.  Every other call works on the handle as on
 * an unweighted one (isira_apply_operator_noalloc and the batch calls take unweighted graphs only).
 * Returns ISIRA_ERR_BAD_GRAPH if a vertex has a non-positive weight sum. */
ISIRA_API isira_status isira_create_weighted(isira_handle* out, int64_t n, int64_t nnz, const int64_t* d_row_ptr,
                                             const int32_t* d_col_idx, const double* d_weights,
                                             const isira_opts* opts, void* stream);

/* Algorithm 2: computes the k (the paper's d, 1 <= k <= min(32, n-2)) smallest positive
 * eigenpairs.  sigma: initial shift (the paper uses 0).  tol: the paper's epsilon, an
 * absolute bound on ||W s1 - theta1 U s1||_2 for unit Ritz vectors (the lock test of Algorithm 2).
 * d_u0: optional device n-vector, the k0 = 1 start basis (must be orthogonal to the
 * all-ones vector and of unit norm; NULL = a SplitMix64 vector from opts.seed).
 * Blocks until done.  Returns ISIRA_ERR_NO_CONVERGENCE if max_outer is reached (pairs
 * locked so far stay available), ISIRA_ERR_NOT_CONNECTED if a locked eigenvalue is
 * below 1e-10 * norm_L. */
ISIRA_API isira_status isira_solve(isira_handle h, int k, double sigma, double tol, const double* d_u0);

/* Results of the last solve, sorted ascending.  h_eigvals: host double[n_locked];
 * d_eigvecs: device n-by-n_locked column-major (may be NULL); h_true_resid: host
 * double[n_locked] receiving ||L v_j - lambda_j v_j||_2 / norm_L computed in FP64
 * (may be NULL).  *n_out (may be NULL) receives n_locked. */
ISIRA_API isira_status isira_eigpairs(isira_handle h, double* h_eigvals, double* d_eigvecs, double* h_true_resid,
                            int* n_out);

/* Counters of the handle (see isira_stats). */
ISIRA_API isira_status isira_get_stats(isira_handle h, isira_stats* out);

/* 1 = time every phase-1 launch with CUDA events during later solves (adds events
 * between launches; results unchanged), 0 = off. */
ISIRA_API isira_status isira_set_profiling(isira_handle h, int on);

/* Releases the handle and all its device memory.  NULL is ignored. */
ISIRA_API void isira_destroy(isira_handle h);

/* ---------------------------------------------------------------------------------
 * Component entry points: single steps of the method on the handle's graph, used by
 * tests and benchmarks.  Device pointers; results ordered on the handle's stream;
 * each call synchronises before returning.
 */

/* The implicit operator of Theorem 2.6 (Eq. 2.14) applied in n-space:
 *   y_r = (deg_r - sigma) x_r - sum_{c in N(r)} x_c + (sigma/n) sum(x) + delta sum_t V_rt (V^T x)_t
 * for r != trim, y_trim = 0, with x_trim treated as 0 (drop_rank1 from the handle's
 * options).  precision selects float (ISIRA_MIXED) or double (ISIRA_FP64) x and y.
 * d_V: n-by-c double matrix (may be NULL when c == 0), 0 <= c <= 31. */
ISIRA_API isira_status isira_apply_operator(isira_handle h, int precision, double sigma, int c, const double* d_V,
                                  const void* d_x, void* d_y);

/* One inner solve (the inner solve of Algorithm 2): preconditioned MINRES on the operator
 * above for the right-hand side d_r (double n-vector, its trim entry ignored) to
 * relative preconditioned residual tau, then the back-map of Eq. 2.5:
 * d_z (double n-vector) is orthogonal to the all-ones vector.  *iters and *relres
 * (may be NULL) receive the iteration count and the final relative residual estimate. */
ISIRA_API isira_status isira_inner_solve(isira_handle h, int precision, double sigma, int c, const double* d_V,
                               const double* d_r, double tau, int max_it, double* d_z, int* iters,
                               double* relres);

/* The multilevel preconditioner alone (opts.precond = 1; paper Sec. 3.2, where combinatorial
 * multigrid plays this role): d_y = M^{-1} d_x for one V-cycle of the aggregation hierarchy of the
 * trimmed Laplacian (Theorem 2.3), without the deflation term.  precision selects float
 * (ISIRA_MIXED) or double (ISIRA_FP64) n-vectors; the trimmed entry of x is ignored and that of y
 * is 0.  M^{-1} is symmetric and positive definite on the other entries.  Builds the hierarchy on
 * first use (for any handle).  *levels and *coarse_n (may be NULL) receive the number of levels and
 * the size of the coarsest (dense) level. */
ISIRA_API isira_status isira_precond_apply(isira_handle h, int precision, const void* d_x, void* d_y, int* levels,
                                           int64_t* coarse_n);

/* All eigenpairs of a symmetric k-by-k matrix (k <= 64), the Rayleigh-Ritz step of Algorithm 2: one CTA of
 * parallel cyclic Jacobi in FP64.  d_H: k-by-k column-major input (not modified);
 * d_theta: k ascending eigenvalues; d_S: k-by-k unit eigenvectors, each signed so that
 * its largest-magnitude entry (first on ties) is positive.  stream as above. */
ISIRA_API isira_status isira_sym_eig(int k, const double* d_H, double* d_theta, double* d_S, void* stream);

/* Convergence history of the last isira_solve: ||r||_2 of the current Ritz pair at every outer step
 * (Algorithm 2's residual, the quantity of the lock test), in step order.  Copies min(cap, steps)
 * values to h_rnorm (host array) and the number of steps to *count (may be NULL).  The paper's
 * Fig. 2 plots this kind of history. */
ISIRA_API isira_status isira_residual_history(isira_handle h, double* h_rnorm, int cap, int* count);

/* The Rayleigh-Ritz step of Algorithm 2 as isira_solve takes it after one expansion (opts.rr_arrow):
 * H = [H0 h; h^T eta] (k-by-k, column-major, 2 <= k <= 64, not modified) where d_S's leading
 * warm_w-by-warm_w block (ld k) holds orthonormal eigenvectors Q0 of H0 = H(0:warm_w, 0:warm_w);
 * warm_w = k - 1 (one new row and column) or k (no new one).  Then diag(Q0, 1)^T H diag(Q0, 1) is an
 * arrowhead matrix, whose eigenvalues are the roots of its secular equation; the eigenvectors are
 * formed as Gu and Eisenstat (1995) do, from a z recomputed from the roots, so they are numerically
 * orthogonal.  Poles with negligible z, and pairs of poles closer than 8 eps max|entry|, deflate.
 * Output as isira_sym_eig (d_theta ascending, d_S overwritten by the k eigenvectors, sign rule).
 * If Q0^T H0 Q0 is not diagonal to a few rounding errors the arrowhead path refuses and parallel
 * Jacobi (isira_sym_eig, warm-started from Q0) produces the result instead; *path (may be NULL)
 * receives 1 for the arrowhead path, 0 for Jacobi.  Allocates a small device scratch and
 * synchronises the stream. */
ISIRA_API isira_status isira_sym_eig_warm(int k, int warm_w, const double* d_H, double* d_theta, double* d_S,
                                          int* path, void* stream);

/* ---------------------------------------------------------------------------------
 * Batched solves: many independent graphs of uneven size (Algorithm 2 for each graph).
 * Every graph gets its own solver (as isira_create) and its own CUDA stream; a pool of host
 * threads drives the solvers concurrently, largest graphs first, so the kernels of different
 * graphs overlap on the GPU.  Each inner solve is one device-driven CUDA-graph launch
 * (opts->inner_graph).  The caller owns the G CSR graphs (device pointers, as in isira_create)
 * until isira_batch_destroy.
 */
typedef struct isira_batch_s* isira_batch;

/* G >= 1 graphs; h_n, h_nnz: host arrays of G sizes; d_row_ptr, d_col_idx: host arrays of G
 * device pointers.  opts as in isira_create (NULL = defaults), applied to every graph, with
 * blocking_sync forced to 1 (the pool runs more threads than the host has cores).  The graphs' streams
 * run concurrently only as far as the context has hardware queues: set CUDA_DEVICE_MAX_CONNECTIONS
 * (up to 32; default 8) in the environment before the process creates its CUDA context. */
ISIRA_API isira_status isira_batch_create(isira_batch* out, int G, const int64_t* h_n, const int64_t* h_nnz,
                                          const int64_t* const* d_row_ptr, const int32_t* const* d_col_idx,
                                          const isira_opts* opts);

/* Solves every graph for its k smallest positive eigenpairs with initial shift sigma and the
 * absolute tolerance tol_rel * (2 * max degree of that graph).  n_threads host threads
 * (<= 0: min(G, 64)).  Returns ISIRA_OK if every graph succeeded, else the first failing
 * status; per-graph statuses via isira_batch_status. */
ISIRA_API isira_status isira_batch_solve(isira_batch b, int k, double sigma, double tol_rel, int n_threads);

/* Status of graph g's last solve. */
ISIRA_API isira_status isira_batch_status(isira_batch b, int g);

/* Results of graph g, as isira_eigpairs. */
ISIRA_API isira_status isira_batch_eigpairs(isira_batch b, int g, double* h_eigvals, double* d_eigvecs,
                                            double* h_true_resid, int* n_out);

/* Counters of graph g, as isira_get_stats. */
ISIRA_API isira_status isira_batch_get_stats(isira_batch b, int g, isira_stats* out);

/* Releases every solver of the batch.  NULL is ignored. */
ISIRA_API void isira_batch_destroy(isira_batch b);

/* ---------------------------------------------------------------------------------
 * Allocation-free variant (the paper has no counterpart; it exists for callers of this
 * library that cannot allocate device memory: programs whose device memory is entirely
 * pre-reserved by their own pool allocator, latency-critical loops in which cudaMalloc and
 * cudaFree, which may synchronise the device, are not acceptable, and plug-ins whose host
 * application forbids allocations it does not make itself).
 *
 * Computes the same result as isira_apply_operator, without a handle: y_r = (deg_r - sigma) x_r
 * - sum_{c in N(r), c != trim} x_c + (sigma/n) sum_{r != trim} x_r + delta sum_t V_rt (Vh^T x)_t for
 * r != trim, y_trim = 0 (drop_rank1 = 1 omits the (sigma/n) term).  All pointers are device
 * pointers: CSR as in isira_create; d_V n-by-c column-major double (ld n, may be NULL when
 * c == 0); d_x, d_y float (ISIRA_MIXED) or double (ISIRA_FP64) n-vectors.  0 <= trim < n.
 * Calls no cudaMalloc, cudaFree or allocating routine.  Its cross-CTA partial sums live in a
 * fixed static device array of about 72 KB (held by every GPU that loads the library until the
 * process exits), which limits the deflation rank to c <= 8: larger c returns ISIRA_ERR_LIMIT.
 * All calls share that array: calls whose work overlaps on the GPU race and must be serialised.
 * The first call on each device, with that device current, looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture on the device.
 * Ordered on `stream`; synchronises it before returning. */
ISIRA_API isira_status isira_apply_operator_noalloc(int64_t n, int64_t nnz, const int64_t* d_row_ptr,
                                                    const int32_t* d_col_idx, int64_t trim, int precision,
                                                    double sigma, double delta, int drop_rank1, int c,
                                                    const double* d_V, const void* d_x, void* d_y, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ISIRA_H */
