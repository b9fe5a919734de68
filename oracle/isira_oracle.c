/*
 * isira_oracle.c -- TEST INFRASTRUCTURE ONLY (see isira_oracle.h).
 *
 * Plain FP64 CPU restatement of iSIRA, arXiv:1710.07080, written for
 * checking, not for speed: no blocking, no fusion, no reordering beyond what
 * the paper's definitions and Algorithm 2 state.  Each function names the
 * passage it follows.  Readings of points the paper leaves open:
 *   - inner solver: preconditioned MINRES (Sec. 3.2 names "PCG or MINRES";
 *     for j > 1 the shifted, deflated system is in general indefinite);
 *   - preconditioner: Mh_sigma = diag(m_r), m_r = deg_r - sigma, kept at
 *     least deg_r/2 (stands in for the CMG preconditioner of Sec. 3.2), with
 *     the deflation handled by the Sherman-Morrison-Woodbury form, Eq. 3.6;
 *   - inner stopping: preconditioned residual norm <= tau * initial;
 *   - "move sigma ~ theta2": sigma = theta2 - max(omega (theta2 - lambda_j),
 *     0.01 theta2);
 *   - orthonormalisation: classical Gram-Schmidt applied twice; if what is
 *     left is below 1e-10 of the input, a SplitMix64 random vector (centred)
 *     replaces it;
 *   - H_k is symmetrised, (H + H^T)/2, before its eigen-decomposition.
 */
#define _POSIX_C_SOURCE 199309L
#include "isira_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

static double wall_seconds(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/* ---------------------------------------------------------------- small helpers */

static double dot(int64_t n, const double* a, const double* b) {
    double s = 0.0;
    for (int64_t t = 0; t < n; ++t) s += a[t] * b[t];
    return s;
}

static double nrm2(int64_t n, const double* a) { return sqrt(dot(n, a, a)); }

static uint64_t splitmix64_at(uint64_t seed, uint64_t counter) {
    /* SplitMix64 (Vigna), output number `counter` of the stream started at seed */
    uint64_t z = seed + (counter + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double uniform_at(uint64_t seed, uint64_t counter) {
    return (double)(splitmix64_at(seed, counter) >> 11) * (1.0 / 9007199254740992.0);
}

/* Mutation testing only: tests/test_oracle_mutants.py builds separate copies of this file with
 * -DOR_PLANT=k, each planting one known, plausible mistake, and checks that the pins in
 * tests/test_oracle_pins.py catch it.  The oracle itself is built with OR_PLANT = 0. */
#ifndef OR_PLANT
#define OR_PLANT 0
#endif

/* ---------------------------------------------------------------- Eq. 1.1 and the weighted Laplacian */

/* Weight of stored entry e (1 when the graph is unweighted, w == NULL). */
static double wt(const double* w, int64_t e) { return w ? w[e] : 1.0; }

/* Diagonal entry of L (or L_w = D_w - W, the weighted Laplacian of the Remark after Theorem 1.2):
 * the sum of the weights of row r's edges. */
static double wdeg(const int64_t* rp, const double* w, int64_t r) {
    if (!w || OR_PLANT == 10) return (double)(rp[r + 1] - rp[r]);
    double s = 0.0;
    for (int64_t e = rp[r]; e < rp[r + 1]; ++e) s += w[e];
    return s;
}

void or_laplacian_apply(int64_t n, const int64_t* rp, const int32_t* ci, const double* w, const double* x,
                        double* y) {
    for (int64_t r = 0; r < n; ++r) {
        double deg = wdeg(rp, w, r);
        double s = deg * x[r];
        for (int64_t e = rp[r]; e < rp[r + 1]; ++e) s -= (OR_PLANT == 1 ? -1.0 : 1.0) * wt(w, e) * x[ci[e]];
        y[r] = s;
    }
}

/* ---------------------------------------------------------------- symmetric eigensolver */

/* Cyclic-by-row Jacobi (Golub & Van Loan Sec. 8.5.2-8.5.3): each rotation zeroes
 * A(p,q) with the symmetric 2-by-2 Schur decomposition. */
int or_sym_eig(int k, const double* Ain, double* theta, double* S, int max_sweeps) {
    double* A = (double*)malloc(sizeof(double) * (size_t)k * k);
    memcpy(A, Ain, sizeof(double) * (size_t)k * k);
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) S[a + (size_t)b * k] = (a == b) ? 1.0 : 0.0;
    int sweeps = 0, converged = 0;
    for (; sweeps < max_sweeps; ++sweeps) {
        double off = 0.0, tot = 0.0;
        for (int b = 0; b < k; ++b)
            for (int a = 0; a < k; ++a) {
                double v = A[a + (size_t)b * k];
                tot += v * v;
                if (a != b) off += v * v;
            }
        (void)tot;
        if (off == 0.0) { converged = 1; break; }
        for (int p = 0; p < k - 1; ++p)
            for (int q = p + 1; q < k; ++q) {
                double apq = A[p + (size_t)q * k];
                if (apq == 0.0) continue;
                double app = A[p + (size_t)p * k], aqq = A[q + (size_t)q * k];
                /* an entry that no longer changes either diagonal entry is set to zero */
                if (sweeps > 2 && fabs(app) + 100.0 * fabs(apq) == fabs(app) &&
                    fabs(aqq) + 100.0 * fabs(apq) == fabs(aqq)) {
                    A[p + (size_t)q * k] = A[q + (size_t)p * k] = 0.0;
                    continue;
                }
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                /* A <- J^T A J with J = [c s; -s c] in the (p,q) plane */
                for (int r = 0; r < k; ++r) {          /* columns p, q */
                    double arp = A[r + (size_t)p * k], arq = A[r + (size_t)q * k];
                    A[r + (size_t)p * k] = c * arp - s * arq;
                    A[r + (size_t)q * k] = s * arp + c * arq;
                }
                for (int r = 0; r < k; ++r) {          /* rows p, q */
                    double apr = A[p + (size_t)r * k], aqr = A[q + (size_t)r * k];
                    A[p + (size_t)r * k] = c * apr - s * aqr;
                    A[q + (size_t)r * k] = s * apr + c * aqr;
                }
                A[p + (size_t)q * k] = A[q + (size_t)p * k] = 0.0;   /* what the rotation annihilates */
                for (int r = 0; r < k; ++r) {          /* S <- S J */
                    double srp = S[r + (size_t)p * k], srq = S[r + (size_t)q * k];
                    S[r + (size_t)p * k] = c * srp - (OR_PLANT == 2 ? -s : s) * srq;
                    S[r + (size_t)q * k] = s * srp + c * srq;
                }
            }
    }
    /* ascending order (stable selection), then the sign rule */
    int* idx = (int*)malloc(sizeof(int) * (size_t)(k > 0 ? k : 1));
    for (int a = 0; a < k; ++a) idx[a] = a;
    for (int a = 0; a < k; ++a) {
        int best = a;
        for (int b = a + 1; b < k; ++b)
            if (A[idx[b] + (size_t)idx[b] * k] < A[idx[best] + (size_t)idx[best] * k]) best = b;
        int tmp = idx[best];
        for (int b = best; b > a; --b) idx[b] = idx[b - 1];
        idx[a] = tmp;
    }
    double* S2 = (double*)malloc(sizeof(double) * (size_t)k * k);
    for (int a = 0; a < k; ++a) {
        theta[a] = A[idx[a] + (size_t)idx[a] * k];
        const double* src = S + (size_t)idx[a] * k;
        int imax = 0;
        for (int r = 1; r < k; ++r)
            if (fabs(src[r]) > fabs(src[imax])) imax = r;
        double sg = src[imax] < 0.0 ? -1.0 : 1.0;
        for (int r = 0; r < k; ++r) S2[r + (size_t)a * k] = sg * src[r];
    }
    memcpy(S, S2, sizeof(double) * (size_t)k * k);
    free(S2);
    free(idx);
    free(A);
    return converged ? sweeps : -1;
}

int or_dense_laplacian_eig(int64_t n, const int64_t* rp, const int32_t* ci, const double* w, double* lam,
                           double* X) {
    double* L = (double*)calloc((size_t)n * n, sizeof(double));
    for (int64_t r = 0; r < n; ++r) {
        L[r + r * n] = wdeg(rp, w, r);
        for (int64_t e = rp[r]; e < rp[r + 1]; ++e) L[r + (int64_t)ci[e] * n] = -wt(w, e);
    }
    int sw = or_sym_eig((int)n, L, lam, X, 100);
    free(L);
    return sw;
}

/* ---------------------------------------------------------------- trimmed operator, Thm 2.6 */

static int64_t hat_of(int64_t r, int64_t trim) { return r < trim ? r : r - 1; }

void or_trimmed_apply(int64_t n, const int64_t* rp, const int32_t* ci, const double* w, int64_t trim,
                      double sigma, double delta, const double* V, int c, int drop_rank1, const double* xh,
                      double* yh) {
    int64_t nh = n - 1;
    double s1 = 0.0;
    for (int64_t t = 0; t < nh; ++t) s1 += xh[t];
    double* g = (double*)calloc((size_t)(c > 0 ? c : 1), sizeof(double));
    for (int j = 0; j < c; ++j)
        for (int64_t r = 0; r < n; ++r)
            if (r != trim) g[j] += V[r + (int64_t)j * n] * xh[hat_of(r, trim)];
    for (int64_t r = 0; r < n; ++r) {
        if (r == trim) continue;
        int64_t rh = hat_of(r, trim);
        double deg = wdeg(rp, w, r);                     /* diagonal of Lh is the full degree */
        double s = (deg - sigma) * xh[rh];
        for (int64_t e = rp[r]; e < rp[r + 1]; ++e) {
            int64_t col = ci[e];
            if (col == trim) continue;                 /* column i is deleted */
            s -= wt(w, e) * xh[hat_of(col, trim)];
        }
        if (!drop_rank1 && OR_PLANT != 3) s += (sigma / (double)n) * s1;
        for (int j = 0; j < c; ++j) s += (OR_PLANT == 4 ? -delta : delta) * V[r + (int64_t)j * n] * g[j];
        yh[rh] = s;
    }
    free(g);
}

void or_backmap(int64_t n, int64_t trim, const double* zh, double* zstar) {
    double s = 0.0;
    for (int64_t t = 0; t < n - 1; ++t) s += zh[t];
    double shift = s / (double)(OR_PLANT == 5 ? n - 1 : n);
    for (int64_t r = 0; r < n; ++r) zstar[r] = (r == trim ? 0.0 : zh[hat_of(r, trim)]) - shift;
}

/* ---------------------------------------------------------------- preconditioner, Remark 3.2 / Eq. 3.6 */

typedef struct {
    int64_t n, trim;
    const int64_t* rp;
    const int32_t* ci;
    const double* w;  /* edge weights (NULL: unit) */
    double sigma, delta;
    const double* V;
    int c, drop_rank1;
    double* mdiag;   /* (n-1) diagonal of Mh_sigma */
    double* K;       /* c-by-c LU of I_c + delta Vh^T Mh^{-1} Vh */
    int* piv;
    double* tmp;     /* (n-1) */
} op_ctx;

static void lu_factor(int c, double* K, int* piv) {
    for (int a = 0; a < c; ++a) {
        int p = a;
        for (int r = a + 1; r < c; ++r)
            if (fabs(K[r + (size_t)a * c]) > fabs(K[p + (size_t)a * c])) p = r;
        piv[a] = p;
        if (p != a)
            for (int b = 0; b < c; ++b) {
                double t = K[a + (size_t)b * c];
                K[a + (size_t)b * c] = K[p + (size_t)b * c];
                K[p + (size_t)b * c] = t;
            }
        for (int r = a + 1; r < c; ++r) {
            K[r + (size_t)a * c] /= K[a + (size_t)a * c];
            for (int b = a + 1; b < c; ++b) K[r + (size_t)b * c] -= K[r + (size_t)a * c] * K[a + (size_t)b * c];
        }
    }
}

static void lu_solve(int c, const double* K, const int* piv, double* x) {
    for (int a = 0; a < c; ++a) {
        double t = x[a]; x[a] = x[piv[a]]; x[piv[a]] = t;
    }
    for (int a = 0; a < c; ++a)
        for (int r = a + 1; r < c; ++r) x[r] -= K[r + (size_t)a * c] * x[a];
    for (int a = c - 1; a >= 0; --a) {
        for (int b = a + 1; b < c; ++b) x[a] -= K[a + (size_t)b * c] * x[b];
        x[a] /= K[a + (size_t)a * c];
    }
}

static void ctx_init(op_ctx* x, int64_t n, const int64_t* rp, const int32_t* ci, const double* w, int64_t trim,
                     double sigma, double delta, const double* V, int c, int drop_rank1) {
    x->n = n; x->rp = rp; x->ci = ci; x->w = w; x->trim = trim; x->sigma = sigma; x->delta = delta;
    x->V = V; x->c = c; x->drop_rank1 = drop_rank1;
    x->mdiag = (double*)malloc(sizeof(double) * (size_t)(n - 1));
    x->tmp = (double*)malloc(sizeof(double) * (size_t)(n - 1));
    for (int64_t r = 0; r < n; ++r) {
        if (r == trim) continue;
        double deg = wdeg(rp, w, r);
        double m = deg - sigma;
        if (m < 0.5 * deg) m = 0.5 * deg;
        x->mdiag[hat_of(r, trim)] = m;
    }
    x->K = (double*)calloc((size_t)(c > 0 ? c * c : 1), sizeof(double));
    x->piv = (int*)calloc((size_t)(c > 0 ? c : 1), sizeof(int));
    for (int a = 0; a < c; ++a)
        for (int b = 0; b < c; ++b) {
            double s = 0.0;
            for (int64_t r = 0; r < n; ++r) {
                if (r == trim) continue;
                s += V[r + (int64_t)a * n] * V[r + (int64_t)b * n] / x->mdiag[hat_of(r, trim)];
            }
            x->K[a + (size_t)b * c] = (a == b ? 1.0 : 0.0) + delta * s;
        }
    if (c > 0) lu_factor(c, x->K, x->piv);
}

static void ctx_free(op_ctx* x) {
    free(x->mdiag); free(x->tmp); free(x->K); free(x->piv);
}

/* ph = (Ih - delta M^{-1} Vh (I_c + delta Vh^T M^{-1} Vh)^{-1} Vh^T) M^{-1} xh   (Eq. 3.6) */
static void ctx_precond(const op_ctx* x, const double* xh, double* ph) {
    int64_t n = x->n, nh = n - 1;
    int c = x->c;
    for (int64_t t = 0; t < nh; ++t) ph[t] = xh[t] / x->mdiag[t];
    if (c == 0) return;
    double* b = (double*)calloc((size_t)c, sizeof(double));
    for (int a = 0; a < c; ++a)
        for (int64_t r = 0; r < n; ++r)
            if (r != x->trim) b[a] += x->V[r + (int64_t)a * n] * ph[hat_of(r, x->trim)];
    lu_solve(c, x->K, x->piv, b);
    for (int64_t r = 0; r < n; ++r) {
        if (r == x->trim) continue;
        int64_t rh = hat_of(r, x->trim);
        double s = 0.0;
        for (int a = 0; a < c; ++a) s += x->V[r + (int64_t)a * n] * b[a];
        ph[rh] -= (OR_PLANT == 7 ? -x->delta : x->delta) * s / x->mdiag[rh];
    }
    free(b);
}

void or_precond_apply(int64_t n, const int64_t* rp, const double* w, int64_t trim, double sigma, double delta,
                      const double* V, int c, const double* xh, double* ph) {
    op_ctx x;
    ctx_init(&x, n, rp, NULL, w, trim, sigma, delta, V, c, 0);
    ctx_precond(&x, xh, ph);
    ctx_free(&x);
}

/* ---------------------------------------------------------------- preconditioned MINRES */

/* Paige & Saunders (1975): Lanczos on the preconditioned operator, with the
 * tridiagonal least-squares problem solved by Givens rotations as it grows. */
static int minres(const op_ctx* cx, const double* b, double* x, double tau, int max_it, double* relres) {
    int64_t nh = cx->n - 1;
    size_t bytes = sizeof(double) * (size_t)nh;
    double *r1 = malloc(bytes), *r2 = malloc(bytes), *y = malloc(bytes), *v = malloc(bytes);
    double *w = calloc((size_t)nh, sizeof(double)), *w1 = calloc((size_t)nh, sizeof(double)),
           *w2 = calloc((size_t)nh, sizeof(double));
    memset(x, 0, bytes);
    memcpy(r1, b, bytes);
    ctx_precond(cx, r1, y);
    double beta1 = dot(nh, r1, y);
    int it = 0;
    if (!(beta1 > 0.0)) { *relres = 0.0; goto done; }
    beta1 = sqrt(beta1);
    memcpy(r2, r1, bytes);
    double beta = beta1, oldb = 0.0, dbar = 0.0, epsln = 0.0, phibar = beta1, cs = -1.0, sn = 0.0;
    while (it < max_it) {
        ++it;
        for (int64_t t = 0; t < nh; ++t) v[t] = y[t] / beta;
        or_trimmed_apply(cx->n, cx->rp, cx->ci, cx->w, cx->trim, cx->sigma, cx->delta, cx->V, cx->c, cx->drop_rank1,
                         v, y);
        if (it >= 2)
            for (int64_t t = 0; t < nh; ++t) y[t] -= (beta / oldb) * r1[t];
        double alfa = dot(nh, v, y);
        for (int64_t t = 0; t < nh; ++t) y[t] -= (alfa / beta) * r2[t];
        double* sw = r1; r1 = r2; r2 = sw;
        memcpy(r2, y, bytes);
        ctx_precond(cx, r2, y);
        oldb = beta;
        double bb = dot(nh, r2, y);
        beta = bb > 0.0 ? sqrt(bb) : 0.0;
        double oldeps = epsln;
        double dlt = cs * dbar + (OR_PLANT == 6 ? -sn : sn) * alfa;
        double gbar = sn * dbar - cs * alfa;
        epsln = sn * beta;
        dbar = -cs * beta;
        double gamma = hypot(gbar, beta);
        if (gamma == 0.0) gamma = 1e-300;
        cs = gbar / gamma;
        sn = beta / gamma;
        double phi = cs * phibar;
        phibar = sn * phibar;
        double* tw = w1; w1 = w2; w2 = w; w = tw;       /* w1 <- w2, w2 <- w */
        for (int64_t t = 0; t < nh; ++t) {
            w[t] = (v[t] - oldeps * w1[t] - dlt * w2[t]) / gamma;
            x[t] += phi * w[t];
        }
        if (phibar <= tau * beta1 || beta == 0.0) break;
    }
    *relres = phibar / beta1;
done:
    free(r1); free(r2); free(y); free(v); free(w); free(w1); free(w2);
    return it;
}

int or_inner_solve(int64_t n, const int64_t* rp, const int32_t* ci, const double* w, int64_t trim, double sigma,
                   double delta, const double* V, int c, int drop_rank1, const double* r, double tau, int max_it,
                   double* zstar, double* relres_out) {
    op_ctx cx;
    ctx_init(&cx, n, rp, ci, w, trim, sigma, delta, V, c, drop_rank1);
    double* rh = (double*)malloc(sizeof(double) * (size_t)(n - 1));
    double* zh = (double*)malloc(sizeof(double) * (size_t)(n - 1));
    for (int64_t t = 0; t < n; ++t)
        if (t != trim) rh[hat_of(t, trim)] = r[t];   /* delete row i of r (Thm 2.6) */
    double rr = 0.0;
    int it = minres(&cx, rh, zh, tau, max_it, &rr);
    or_backmap(n, trim, zh, zstar);
    if (relres_out) *relres_out = rr;
    free(rh); free(zh);
    ctx_free(&cx);
    return it;
}

/* ---------------------------------------------------------------- Algorithm 2 */

/* z <- z - Q (Q^T z) for the columns of U (k) and V (c), classical Gram-Schmidt. */
static void cgs_pass(int64_t n, const double* U, int k, const double* V, int c, double* z) {
    double* h = (double*)malloc(sizeof(double) * (size_t)(k + c + 1));
    for (int a = 0; a < k; ++a) h[a] = dot(n, U + (int64_t)a * n, z);
    for (int a = 0; a < c; ++a) h[k + a] = dot(n, V + (int64_t)a * n, z);
    for (int a = 0; a < k; ++a)
        for (int64_t t = 0; t < n; ++t) z[t] -= h[a] * U[t + (int64_t)a * n];
    for (int a = 0; a < c; ++a)
        for (int64_t t = 0; t < n; ++t) z[t] -= h[k + a] * V[t + (int64_t)a * n];
    free(h);
}

/* Orthonormalise z against U and V (Algorithm 2, orthonormalisation). Returns 1 on breakdown replacement. */
static int orthonormalize(int64_t n, const double* U, int k, const double* V, int c, double* z,
                          uint64_t seed, int* n_breakdowns) {
    int replaced = 0;
    for (int attempt = 0; attempt < 8; ++attempt) {
        double before = nrm2(n, z);
        cgs_pass(n, U, k, V, c, z);
        cgs_pass(n, U, k, V, c, z);
        double after = nrm2(n, z);
        if (after > 1e-10 * before && after > 0.0) {
            for (int64_t t = 0; t < n; ++t) z[t] /= after;
            return replaced;
        }
        /* breakdown: a centred SplitMix64 vector (stream `seed`, block n_breakdowns) */
        double mean = 0.0;
        uint64_t base = (uint64_t)(*n_breakdowns) * (uint64_t)n;
        for (int64_t t = 0; t < n; ++t) {
            z[t] = 2.0 * uniform_at(seed, base + (uint64_t)t) - 1.0;
            mean += z[t];
        }
        mean /= (double)n;
        for (int64_t t = 0; t < n; ++t) z[t] -= mean;
        ++(*n_breakdowns);
        replaced = 1;
    }
    return -1;
}

/* X(:, 0:ncol) <- X(:, 0:k) * S(:, c0:c0+ncol) for a k-by-k S (in place via a copy). */
static void rotate_basis(int64_t n, double* X, int k, const double* S, int c0, int ncol) {
    double* T = (double*)calloc((size_t)n * (size_t)ncol, sizeof(double));
    for (int b = 0; b < ncol; ++b)
        for (int a = 0; a < k; ++a) {
            double s = S[a + (size_t)(c0 + b) * k];
            const double* xa = X + (int64_t)a * n;
            double* tb = T + (int64_t)b * n;
            for (int64_t t = 0; t < n; ++t) tb[t] += xa[t] * s;
        }
    memcpy(X, T, sizeof(double) * (size_t)n * (size_t)ncol);
    free(T);
}

int or_isira(int64_t n, const int64_t* rp, const int32_t* ci, const double* w, const double* u0, const or_params* p,
             double* lam, double* Vout, or_stats* st) {
    memset(st, 0, sizeof(*st));
    const double t_start = wall_seconds();
    int d = p->d, m = p->m, q = p->q;
    if (n < 3 || d < 1 || d > n - 2 || q < d || m <= q || m < 2) { st->status = 2; return 2; }

    /* Remark 4.1: trimming index = vertex of maximum degree (diagonal entry), delta = 2 max diag(L) */
    int64_t trim = p->trim;
    double dmax = 0.0;
    int64_t argmax = 0;
    for (int64_t r = 0; r < n; ++r) {
        double dg = wdeg(rp, w, r);
        if (dg > dmax) { dmax = dg; argmax = r; }
    }
    if (trim < 0 || trim >= n) trim = argmax;
    double delta = p->delta > 0.0 ? p->delta : 2.0 * dmax;
    st->trim = trim;
    st->delta = delta;

    double* U = (double*)calloc((size_t)n * m, sizeof(double));
    double* W = (double*)calloc((size_t)n * m, sizeof(double));
    double* V = Vout;                     /* locked vectors, n-by-d */
    double* H = (double*)calloc((size_t)m * m, sizeof(double));
    double* S = (double*)calloc((size_t)m * m, sizeof(double));
    double* theta = (double*)calloc((size_t)m, sizeof(double));
    double* y = (double*)malloc(sizeof(double) * (size_t)n);
    double* r = (double*)malloc(sizeof(double) * (size_t)n);
    double* z = (double*)malloc(sizeof(double) * (size_t)n);
    double* col = (double*)malloc(sizeof(double) * (size_t)n);
    double* vtu = (double*)calloc((size_t)(d + 1), sizeof(double));

    /* start: D = [], V = [], k = k0 = 1, flag = 0 */
    memcpy(U, u0, sizeof(double) * (size_t)n);
    int k = 1, c = 0;
    double sigma = p->sigma0;
    int status = 0;

    for (int j = 1; j <= d; ++j) {                               /* for j = 1 .. d */
        int flag = 0;
        while (!flag) {                                          /* until pair j locks */
            if (st->outer_steps >= p->max_outer) { status = 1; goto finish; }
            st->outer_steps++;
            /* W_k = (L + delta V V^T) U_k,  H_k = U_k^T W_k */
            const double t_w = wall_seconds();
            st->w_columns += k;
            for (int a = 0; a < k; ++a) {
                double* ua = U + (int64_t)a * n;
                double* wa = W + (int64_t)a * n;
                or_laplacian_apply(n, rp, ci, w, ua, wa);
                for (int b = 0; b < c; ++b) vtu[b] = dot(n, V + (int64_t)b * n, ua);
                for (int b = 0; b < c; ++b)
                    for (int64_t t = 0; t < n; ++t) wa[t] += delta * V[t + (int64_t)b * n] * vtu[b];
            }
            for (int a = 0; a < k; ++a)
                for (int b = 0; b < k; ++b) H[a + (size_t)b * k] = dot(n, U + (int64_t)a * n, W + (int64_t)b * n);
            for (int a = 0; a < k; ++a)
                for (int b = a + 1; b < k; ++b) {
                    double h = 0.5 * (H[a + (size_t)b * k] + H[b + (size_t)a * k]);
                    H[a + (size_t)b * k] = H[b + (size_t)a * k] = h;
                }
            st->sec_w += wall_seconds() - t_w;
            /* Rayleigh-Ritz: all eigenpairs of H_k, ascending, unit vectors */
            or_sym_eig(k, H, theta, S, 100);
            /* residual: r = W_k s1 - theta1 U_k s1 */
            for (int64_t t = 0; t < n; ++t) { y[t] = 0.0; r[t] = 0.0; }
            for (int a = 0; a < k; ++a) {
                double s = S[a];
                for (int64_t t = 0; t < n; ++t) {
                    y[t] += U[t + (int64_t)a * n] * s;
                    r[t] += W[t + (int64_t)a * n] * s;
                }
            }
            for (int64_t t = 0; t < n; ++t) r[t] -= theta[0] * y[t];
            double rn = nrm2(n, r);
            /* the search space cannot grow past the orthogonal complement of [V 1] */
            int exhausted = (k + c >= n - 1);
            if (rn < p->eps || exhausted) {                       /* lock */
                lam[j - 1] = theta[OR_PLANT == 8 && k >= 2 ? 1 : 0];
                memcpy(V + (int64_t)c * n, y, sizeof(double) * (size_t)n);
                ++c;
                st->n_locked = c;
                flag = 1;
            } else {
                if (k == m) {                                      /* restart */
                    rotate_basis(n, U, k, S, OR_PLANT == 9 ? k - q : 0, q);
                    rotate_basis(n, W, k, S, OR_PLANT == 9 ? k - q : 0, q);
                    k = q;
                    st->restarts++;
                }
                /* inexact inner solve: trimmed solve (Eq. 2.4 / 2.14) and the back-map (Eq. 2.5) */
                double rr;
                const double t_in = wall_seconds();
                int its = or_inner_solve(n, rp, ci, w, trim, sigma, delta, V, c, p->drop_rank1, r,
                                         p->tau_inner, p->max_inner, z, &rr);
                st->inner_iters += its;
                st->sec_inner += wall_seconds() - t_in;
                /* orthonormalise against U_k and V */
                if (orthonormalize(n, U, k, V, c, z, p->seed, &st->breakdowns) < 0) { status = 1; goto finish; }
                memcpy(U + (int64_t)k * n, z, sizeof(double) * (size_t)n);   /* expand */
                ++k;
            }
        }
        if (j == d) break;
        /* purge v_j, then move sigma */
        double th2 = (k >= 2) ? theta[1] : sigma;
        if (k >= 2) {
            rotate_basis(n, U, k, S, 1, k - 1);
            rotate_basis(n, W, k, S, 1, k - 1);
            double gap = th2 - lam[j - 1];
            double move = p->omega * gap;
            if (move < 0.01 * th2) move = 0.01 * th2;
            sigma = th2 - move;
            k = k - 1;
        } else {
            /* the only basis vector was locked: restart from a fresh random direction */
            for (int64_t t = 0; t < n; ++t) col[t] = 0.0;
            k = 0;
            if (orthonormalize(n, U, 0, V, c, col, p->seed, &st->breakdowns) < 0) { status = 1; goto finish; }
            memcpy(U, col, sizeof(double) * (size_t)n);
            k = 1;
        }
    }
finish:
    st->sec_total = wall_seconds() - t_start;
    st->status = status;
    st->n_locked = c;
    free(U); free(W); free(H); free(S); free(theta); free(y); free(r); free(z); free(col); free(vtu);
    return status;
}
