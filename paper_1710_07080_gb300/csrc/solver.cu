// solver.cu -- host driver of Algorithm 2 and the C ABI declared in include/isira.h.
//
// The outer loop runs on the host, one synchronisation per outer step (to read
// ||r|| and the Ritz values written by the device into mapped pinned memory) and
// one after each orthogonalisation (breakdown test).  Everything that touches an
// n-vector runs in the kernels of inner_*.cu and outer.cu.  The inner MINRES solve
// is launched in chunks of iterations; its kernels return at once after the
// device-side stopping test has fired, so a chunk may end with a few empty launches.
#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <tuple>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/isira.h"
#include "internal.h"

using namespace isira;

namespace {

struct CudaError {
    cudaError_t e;
};

inline void ck(cudaError_t e) {
    if (e != cudaSuccess) throw CudaError{e};
}

struct StatusError {
    isira_status s;
};

template <typename T>
struct InnerBuffers {
    T* base = nullptr;
    InnerState<T>* st = nullptr;
    // multilevel preconditioner: 4 n-vectors (r_{k-1}, r_k, projected V-cycle input, V-cycle output)
    T* ml = nullptr;
    MlHierarchy<T> H;
};

}  // namespace

// NVTX range over one phase of Algorithm 2 (visible in Nsight Systems / Compute timelines; a
// no-op without a tool attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct isira_handle_s {
    int64_t n = 0, nnz = 0, ld = 0;
    const int64_t* rp = nullptr;
    const int32_t* ci = nullptr;
    cudaStream_t stream = nullptr;
    isira_opts opts{};
    int nsm = 0;
    // setup (Remark 4.1)
    int64_t max_degree = 0, trim = 0;
    double delta = 0.0, normL = 0.0;
    int32_t* item_row = nullptr;
    int32_t* item_k = nullptr;
    double* item_partial = nullptr;
    unsigned* item_count = nullptr;
    int32_t* warp_start = nullptr;
    int32_t* deg32 = nullptr;      // degree per row (solver numbering), ld entries
    // weighted Laplacian (null: unit weights): the caller's weights, the solver's relabelled copy,
    // FP32 copies, weighted degrees, and the weights of the sliced copy
    const double* w_user = nullptr;
    double* own_w = nullptr;
    float* wf = nullptr;
    double* degwd = nullptr;
    float* degwf = nullptr;
    double* sell_wd = nullptr;
    float* sell_wf = nullptr;
    int64_t* sell_off = nullptr;   // sliced ELL copy of the light rows (with relabelling)
    int32_t* sell_ci = nullptr;
    int64_t sell_total = 0;
    int smem_max = 0;
    // optional internal relabelling (opts.reorder): owned CSR, perm[new] = old, inv[old] = new
    int64_t* own_rp = nullptr;
    int32_t* own_ci = nullptr;
    int32_t* perm = nullptr;
    int32_t* inv = nullptr;
    int64_t trim_user = 0;
    int64_t n_long = 0, n_items = 0;
    RowSched rs{};
    int lanes = 8;
    int ew_blocks = 0, ts_blocks = 0;
    // FP64 outer buffers
    int m_alloc = 0, d_alloc = 0;
    double* U = nullptr;
    double* W = nullptr;
    double* V = nullptr;
    double* H = nullptr;
    double* theta = nullptr;
    double* S = nullptr;
    double* R = nullptr;
    double* Z = nullptr;
    double* dscratch = nullptr;
    ArrowWork* arrow = nullptr;   // scratch of the warm-start Rayleigh-Ritz path
    double* gsum = nullptr;       // gather output, n doubles (shared by both precisions)
    double* partial = nullptr;
    size_t partial_elems = 0;
    unsigned* counter = nullptr;
    double* Gm = nullptr;
    double* Cinv = nullptr;
    double* lam_dev = nullptr;
    double* tres_dev = nullptr;
    HostStatus* hs = nullptr;
    HostStatus* hs_dev = nullptr;
    // inner buffers (one precision per handle, plus FP64 for component calls)
    InnerBuffers<float> fb;
    InnerBuffers<double> db;
    float* Vt_f = nullptr;
    // results
    std::vector<double> lam;
    std::vector<double> rhist;    // ||r|| of every outer step of the last solve
    int n_locked = 0;
    bool solved = false;
    isira_stats stats{};
    int profiling = 0;
    std::vector<cudaEvent_t> ev;
    cudaEvent_t sync_ev = nullptr;   // blocking-sync event of sync() when opts.blocking_sync = 1
    // device-driven inner loop: one instantiated graph per deflation-rank bucket (c = 0, <=8, <=12, <=16, <=24, <=32)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t inner_graph[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaGraphExec_t ml_graph[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    double* ml_dv = nullptr;          // kCMax: 1 / (lambda_t - sigma + delta) of the deflated directions
    bool use_ml = false;              // inner solves with the multilevel preconditioner
    int pending_inner_stats = 0;
};

namespace {

template <typename T>
void alloc_inner(isira_handle h, InnerBuffers<T>& b) {
    if (b.base) return;
    // 7 MINRES vectors, plus the reciprocal preconditioner diagonal in FP64 mode
    const int nvec = sizeof(T) == sizeof(double) ? 8 : 7;
    ck(cudaMalloc(&b.base, sizeof(T) * (size_t)h->ld * nvec));
    ck(cudaMalloc(&b.st, sizeof(InnerState<T>)));
    ck(cudaMemsetAsync(b.base, 0, sizeof(T) * (size_t)h->ld * nvec, h->stream));
    ck(cudaMemsetAsync(b.st, 0, sizeof(InnerState<T>), h->stream));
}

constexpr double kMlOmega = 2.0 / 3.0;     // damping of the Jacobi smoother of the V-cycle

template <typename T>
InnerArgs<T> make_args(isira_handle h, InnerBuffers<T>& b, double sigma, int c, const T* Vt, int64_t ldv, double tau,
                       int max_it) {
    InnerArgs<T> a{};
    a.rs = h->rs;
    a.trim = h->trim;
    a.sigma = (T)sigma;
    a.sig_n = h->opts.drop_rank1 ? T(0) : (T)(sigma / (double)h->n);
    a.delta = (T)h->delta;
    a.Vt = Vt;
    a.ldv = ldv;
    a.c = c;
    T* v = b.base;
    const int64_t ld = h->ld;
    a.z0 = v; a.z1 = v + ld; a.Y = v + 2 * ld; a.wb0 = v + 3 * ld; a.wb1 = v + 4 * ld; a.wb2 = v + 5 * ld;
    a.x = v + 6 * ld;
    a.dinv = sizeof(T) == sizeof(double) ? v + 7 * ld : nullptr;
    a.gsum = reinterpret_cast<T*>(h->gsum);
    a.deg = h->deg32;
    a.partial = reinterpret_cast<T*>(h->partial);
    a.pstride = (int)(h->partial_elems / 512);
    a.counter = h->counter;
    a.st = b.st;
    a.hs = h->hs_dev;
    a.Cinv = h->Cinv;
    a.Gm = h->Gm;
    a.partial_d = h->partial;
    if (b.ml) {
        a.rprev = b.ml;
        a.rcur = b.ml + ld;
        a.rin = b.ml + 2 * ld;
        a.wv = b.ml + 3 * ld;
        a.dv = h->ml_dv;
        if (b.H.nlev >= 2) {
            a.ml_x0 = b.H.lev[0].x0;
            a.ml_dinv0 = b.H.lev[0].dinv;
            a.ml_fuse_post = 1;
            a.ml_b0 = c > 0 ? a.rin : a.rcur;
            a.ml_x1 = b.H.lev[0].x1;
            a.ml_wx1 = b.H.lev[0].x0;
        }
        a.ml_omega = (T)kMlOmega;
    }
    a.tau = (T)tau;
    a.max_it = max_it;
    a.ew_blocks = h->ew_blocks;
    return a;
}

OuterArgs make_outer(isira_handle h) {
    OuterArgs a{};
    a.rs = h->rs;
    a.n = h->n;
    a.ld = h->ld;
    a.U = h->U; a.W = h->W; a.V = h->V;
    a.H = h->H; a.theta = h->theta; a.S = h->S;
    a.R = h->R; a.Z = h->Z;
    a.gsum = h->gsum;
    a.partial = h->partial;
    a.pstride = (int)(h->partial_elems / 512);
    a.counter = h->counter;
    a.hs = h->hs_dev;
    a.dscratch = h->dscratch;
    a.ew_blocks = h->ew_blocks;
    a.ts_blocks = h->ts_blocks;
    return a;
}

void sync(isira_handle h) {
    if (h->sync_ev) {                     // the thread sleeps until the stream reaches the event
        ck(cudaEventRecord(h->sync_ev, h->stream));
        ck(cudaEventSynchronize(h->sync_ev));
    } else {
        ck(cudaStreamSynchronize(h->stream));
    }
    ck(cudaGetLastError());
    if (h->hs && (static_cast<volatile HostStatus*>(h->hs)->dev_error & 1))
        throw StatusError{ISIRA_ERR_DEVICE_TIMEOUT};
}

// start of an entry point: no device error recorded yet
void clear_dev_error(isira_handle h) {
    if (h->hs) static_cast<volatile HostStatus*>(h->hs)->dev_error = 0;
}

volatile HostStatus* hst(isira_handle h) { return h->hs; }

int nc_bucket(int c) { return c == 0 ? 0 : (c <= 8 ? 1 : (c <= 12 ? 2 : (c <= 16 ? 3 : (c <= 24 ? 4 : 5)))); }

// WHILE(cond) { phase 1; phase 2 } with phase 2's last CTA setting cond = !done.  The kernels
// read the per-solve shift and rank from device state, so one graph serves every solve of a bucket.
template <typename T>
cudaGraphExec_t build_inner_graph(isira_handle h, const InnerArgs<T>& a) {
    if (!h->cap_stream) ck(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    ck(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle hc;
    ck(cudaGraphConditionalHandleCreate(&hc, g, 1u, cudaGraphCondAssignDefault));
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = hc;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    ck(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p));
    cudaGraph_t body = p.conditional.phGraph_out[0];
    ck(cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    inner_phase1<T>(a, h->lanes, h->cap_stream);
    inner_phase2_cond<T>(a, hc, h->cap_stream);
    ck(cudaStreamEndCapture(h->cap_stream, &body));
    cudaGraphExec_t ex = nullptr;
    ck(cudaGraphInstantiate(&ex, g, 0));
    cudaGraphDestroy(g);
    return ex;
}

// One inner solve on R (right-hand side) into Z (FP64, back-mapped).  Chunked mode returns the
// iteration count; graph mode returns -1 (the count is read at the next synchronisation).
template <typename T>
int run_inner_ml(isira_handle h, InnerBuffers<T>& b, double sigma, int c, const T* Vt, int64_t ldv, double tau,
                 int max_it, bool gram_dirty, const double* R, const double* rnorm_dev, bool allow_graph,
                 const double* lam);

template <typename T>
int run_inner(isira_handle h, InnerBuffers<T>& b, double sigma, int c, const T* Vt, int64_t ldv, double tau,
              int max_it, bool gram_dirty, const double* R, const double* rnorm_dev, bool allow_graph = false,
              const double* lam = nullptr) {
    if (h->use_ml)
        return run_inner_ml<T>(h, b, sigma, c, Vt, ldv, tau, max_it, gram_dirty, R, rnorm_dev, allow_graph, lam);
    InnerArgs<T> a = make_args<T>(h, b, sigma, c, Vt, ldv, tau, max_it);
    cudaStream_t s = h->stream;
    if (gram_dirty && c > 0) {
        gram_setup<T>(a, h->Gm, h->Cinv, h->partial, s);
        h->stats.kernel_launches += 1;
    }
    inner_prep_launch<T>(a, R, rnorm_dev, s);
    inner_phase2<T>(a, 1, s);
    h->stats.kernel_launches += 2;
    if (allow_graph && h->opts.inner_graph && !h->profiling) {
        const int bkt = nc_bucket(c);
        if (!h->inner_graph[bkt]) h->inner_graph[bkt] = build_inner_graph<T>(h, a);
        ck(cudaGraphLaunch(h->inner_graph[bkt], s));
        inner_finalize_to<T>(a, h->Z, s);
        h->stats.kernel_launches += 1;
        h->stats.inner_solves += 1;
        h->pending_inner_stats = 1;
        return -1;
    }
    const int chunk = h->opts.inner_chunk > 0 ? h->opts.inner_chunk : 16;
    int launched = 0;
    while (true) {
        const bool prof = h->profiling != 0;
        for (int i = 0; i < chunk; ++i) {
            if (prof) ck(cudaEventRecord(h->ev[4 * i], s));
            inner_gather<T>(a, h->lanes, s);
            if (prof) ck(cudaEventRecord(h->ev[4 * i + 1], s));
            inner_rows<T>(a, s);
            if (prof) ck(cudaEventRecord(h->ev[4 * i + 2], s));
            inner_phase2<T>(a, 0, s);
            if (prof) ck(cudaEventRecord(h->ev[4 * i + 3], s));
        }
        h->stats.spmv_launches += chunk;
        h->stats.kernel_launches += 3 * chunk;
        sync(h);
        const int itn = hst(h)->inner_iters;
        if (prof) {
            for (int i = 0; i < chunk; ++i) {
                if (launched + i + 1 > itn) break;   // launches after the stop returned at once
                float ms = 0.f, ms_rows = 0.f, ms_p2 = 0.f;
                ck(cudaEventElapsedTime(&ms, h->ev[4 * i], h->ev[4 * i + 1]));
                ck(cudaEventElapsedTime(&ms_rows, h->ev[4 * i + 1], h->ev[4 * i + 2]));
                ck(cudaEventElapsedTime(&ms_p2, h->ev[4 * i + 2], h->ev[4 * i + 3]));
                h->stats.inner_phase1_ms += ms;
                h->stats.inner_rows_ms += ms_rows;
                h->stats.inner_phase2_ms += ms_p2;
                h->stats.inner_phase1_timed += 1;
                h->stats.inner_phase1_csum += c;
            }
        }
        launched += chunk;
        if (hst(h)->inner_done) break;
        if (launched > max_it + 2 * chunk) break;   // defensive: the device test caps at max_it
    }
    inner_finalize_to<T>(a, h->Z, s);
    h->stats.kernel_launches += 1;
    h->stats.inner_solves += 1;
    const int its = hst(h)->inner_iters;
    h->stats.inner_iters += its;
    return its;
}

// ------------------------------------------------------------------ multilevel-preconditioned inner solve

template <typename T>
void ensure_ml(isira_handle h, InnerBuffers<T>& b) {
    if (!b.ml) {
        const size_t elems = (size_t)h->ld * 4;
        ck(cudaMalloc(&b.ml, sizeof(T) * elems));
        ck(cudaMemsetAsync(b.ml, 0, sizeof(T) * elems, h->stream));
    }
    if (!h->ml_dv) ck(cudaMalloc(&h->ml_dv, sizeof(double) * kCMax));
    if (b.H.nlev == 0) ck(ml_build<T>(b.H, h->rs.rp, h->rs.ci, h->rs.wd, h->n, h->ld, h->trim, h->stream));
}

template <typename T>
T ml_alpha(isira_handle h) { return (T)(h->opts.ml_alpha > 0.0 ? h->opts.ml_alpha : 1.5); }

// body of one multilevel MINRES iteration (graph capture or chunked launches)
template <typename T>
void ml_iteration(isira_handle h, InnerBuffers<T>& b, const InnerArgs<T>& a, cudaGraphConditionalHandle cond,
                  int has_cond, cudaStream_t s) {
    const int* done = &a.st->done;
    GatherFn<T> gather = [&](const T* x, T* g, cudaStream_t st) { inner_gather_vec<T>(a, x, g, h->lanes, done, st); };
    inner_gather<T>(a, h->lanes, s);
    ml_phase1<T>(a, s);
    ml_phase2a<T>(a, 0, s);
    ml_project<T>(a, 0, s);
    ml_vcycle<T>(b.H, a.c > 0 ? a.rin : a.rcur, a.wv, gather, (T)kMlOmega, ml_alpha<T>(h), done,
                 a.c > 0 && a.ml_x0 != nullptr, a.ml_fuse_post != 0, s);
    ml_phase2b<T>(a, 0, cond, has_cond, s);
    ml_phase2c<T>(a, 0, s);
}

template <typename T>
cudaGraphExec_t build_ml_graph(isira_handle h, InnerBuffers<T>& b, const InnerArgs<T>& a) {
    if (!h->cap_stream) ck(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    ck(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle hc;
    ck(cudaGraphConditionalHandleCreate(&hc, g, 1u, cudaGraphCondAssignDefault));
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = hc;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    ck(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p));
    cudaGraph_t body = p.conditional.phGraph_out[0];
    ck(cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    ml_iteration<T>(h, b, a, hc, 1, h->cap_stream);
    ck(cudaStreamEndCapture(h->cap_stream, &body));
    cudaGraphExec_t ex = nullptr;
    ck(cudaGraphInstantiate(&ex, g, 0));
    cudaGraphDestroy(g);
    return ex;
}

template <typename T>
int ml_launches_per_iteration(const InnerBuffers<T>& b, int c) {
    return 6 + (c > 0 ? 1 : 0) + ml_launches(b.H, c > 0 && b.H.nlev >= 2, b.H.nlev >= 2);
}

// One inner solve with the multilevel preconditioner; same contract as run_inner.  lam: the
// locked eigenvalues of the deflation columns (host, c values; null: taken as 0).
template <typename T>
int run_inner_ml(isira_handle h, InnerBuffers<T>& b, double sigma, int c, const T* Vt, int64_t ldv, double tau,
                 int max_it, bool gram_dirty, const double* R, const double* rnorm_dev, bool allow_graph,
                 const double* lam) {
    ensure_ml(h, b);
    InnerArgs<T> a = make_args<T>(h, b, sigma, c, Vt, ldv, tau, max_it);
    cudaStream_t s = h->stream;
    GatherFn<T> gather0 = [&](const T* x, T* g, cudaStream_t st) { inner_gather_vec<T>(a, x, g, h->lanes, nullptr, st); };
    if (c > 0 && gram_dirty) {
        // D = diag(1 / (lambda_t - sigma + delta)) for the deflated directions (pageable copy: synchronous)
        double dv[kCMax];
        for (int t = 0; t < c; ++t) dv[t] = 1.0 / ((lam ? lam[t] : 0.0) - sigma + h->delta);
        ck(cudaMemcpyAsync(h->ml_dv, dv, sizeof(double) * c, cudaMemcpyHostToDevice, s));
    }
    ml_inner_prep<T>(a, R, rnorm_dev, s);
    ml_phase2a<T>(a, 1, s);
    ml_project<T>(a, 1, s);
    ml_vcycle<T>(b.H, c > 0 ? a.rin : a.rcur, a.wv, gather0, (T)kMlOmega, ml_alpha<T>(h), nullptr,
                 c > 0 && a.ml_x0 != nullptr, a.ml_fuse_post != 0, s);
    ml_phase2b<T>(a, 1, cudaGraphConditionalHandle{}, 0, s);
    ml_phase2c<T>(a, 1, s);
    const int per_it = ml_launches_per_iteration(b, c);
    h->stats.kernel_launches += per_it - 1;
    if (allow_graph && h->opts.inner_graph && !h->profiling) {
        const int bkt = nc_bucket(c);
        if (!h->ml_graph[bkt]) h->ml_graph[bkt] = build_ml_graph<T>(h, b, a);
        ck(cudaGraphLaunch(h->ml_graph[bkt], s));
        inner_finalize_to<T>(a, h->Z, s);
        h->stats.kernel_launches += 1;
        h->stats.inner_solves += 1;
        h->pending_inner_stats = per_it;
        return -1;
    }
    const int chunk = h->opts.inner_chunk > 0 ? h->opts.inner_chunk : 16;
    int launched = 0;
    while (true) {
        const bool prof = h->profiling != 0;
        for (int i = 0; i < chunk; ++i) {
            if (prof) ck(cudaEventRecord(h->ev[4 * i], s));
            inner_gather<T>(a, h->lanes, s);
            if (prof) ck(cudaEventRecord(h->ev[4 * i + 1], s));
            ml_phase1<T>(a, s);
            if (prof) ck(cudaEventRecord(h->ev[4 * i + 2], s));
            ml_phase2a<T>(a, 0, s);
            ml_project<T>(a, 0, s);
            ml_vcycle<T>(b.H, c > 0 ? a.rin : a.rcur, a.wv, gather0, (T)kMlOmega, ml_alpha<T>(h), &a.st->done,
                         c > 0 && a.ml_x0 != nullptr, a.ml_fuse_post != 0, s);
            ml_phase2b<T>(a, 0, cudaGraphConditionalHandle{}, 0, s);
            ml_phase2c<T>(a, 0, s);
            if (prof) ck(cudaEventRecord(h->ev[4 * i + 3], s));
        }
        h->stats.spmv_launches += chunk;
        h->stats.kernel_launches += (long long)per_it * chunk;
        sync(h);
        const int itn = hst(h)->inner_iters;
        if (prof) {
            for (int i = 0; i < chunk; ++i) {
                if (launched + i + 1 > itn) break;
                float ms = 0.f, ms_rows = 0.f, ms_p2 = 0.f;
                ck(cudaEventElapsedTime(&ms, h->ev[4 * i], h->ev[4 * i + 1]));
                ck(cudaEventElapsedTime(&ms_rows, h->ev[4 * i + 1], h->ev[4 * i + 2]));
                ck(cudaEventElapsedTime(&ms_p2, h->ev[4 * i + 2], h->ev[4 * i + 3]));
                h->stats.inner_phase1_ms += ms;
                h->stats.inner_rows_ms += ms_rows;
                h->stats.inner_phase2_ms += ms_p2;
                h->stats.inner_phase1_timed += 1;
                h->stats.inner_phase1_csum += c;
            }
        }
        launched += chunk;
        if (hst(h)->inner_done) break;
        if (launched > max_it + 2 * chunk) break;
    }
    inner_finalize_to<T>(a, h->Z, s);
    h->stats.kernel_launches += 1;
    h->stats.inner_solves += 1;
    const int its = hst(h)->inner_iters;
    h->stats.inner_iters += its;
    return its;
}

// Preconditioner of the inner solve.  precond = 0 / 1 force the diagonal / the multilevel one.
// precond = -1 (automatic): graphs with n >= 20000 and maximum degree <= 64 (mesh-like: the
// multilevel hierarchy's coarse rows stay short, and its setup is amortised) get one timed inner
// solve with each preconditioner (shift 0, no deflation, tau_inner, a seeded right-hand side) and
// keep the faster; every other graph keeps the diagonal.
template <typename T>
float time_inner(isira_handle h, InnerBuffers<T>& b, cudaEvent_t e0, cudaEvent_t e1) {
    cudaStream_t s = h->stream;
    const double tau = h->opts.tau_inner > 0.0 ? h->opts.tau_inner : 1e-3;
    const int max_it = h->opts.max_inner > 0 ? h->opts.max_inner : 5000;
    ck(cudaEventRecord(e0, s));
    run_inner<T>(h, b, 0.0, 0, nullptr, h->ld, tau, max_it, false, h->R, h->dscratch + 300, true);
    ck(cudaEventRecord(e1, s));
    sync(h);
    float ms = 0.f;
    ck(cudaEventElapsedTime(&ms, e0, e1));
    return ms;
}

void choose_preconditioner(isira_handle h) {
    const int pc = h->opts.precond;
    const bool mixed = h->opts.precision == ISIRA_MIXED;
    auto build = [&]() {
        if (mixed) ensure_ml(h, h->fb); else ensure_ml(h, h->db);
        sync(h);
    };
    h->use_ml = false;
    if (pc == 1) {
        build();
        h->use_ml = true;
    }
    if (pc != -1 || h->n < 20000 || h->max_degree > 64) return;
    build();
    OuterArgs oa = make_outer(h);
    outer_random(oa, h->opts.seed, 7777, h->stream);            // right-hand side in Z, copied to R
    ck(cudaMemcpyAsync(h->R, h->Z, sizeof(double) * (size_t)h->n, cudaMemcpyDeviceToDevice, h->stream));
    const double one = 1.0;
    ck(cudaMemcpyAsync(h->dscratch + 300, &one, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    cudaEvent_t e0, e1;
    ck(cudaEventCreate(&e0));
    ck(cudaEventCreate(&e1));
    float t[2] = {0.f, 0.f};
    for (int ml = 0; ml < 2; ++ml) {
        h->use_ml = ml == 1;
        for (int rep = 0; rep < 2; ++rep)                           // the first run builds the graph
            t[ml] = mixed ? time_inner<float>(h, h->fb, e0, e1) : time_inner<double>(h, h->db, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->use_ml = t[1] < t[0];
    h->stats.precond_probe_ms[0] = t[0];
    h->stats.precond_probe_ms[1] = t[1];
}

void ensure_outer(isira_handle h, int m, int d) {
    const size_t ld = (size_t)h->ld;
    if (m > h->m_alloc) {
        if (h->U) cudaFree(h->U);
        if (h->W) cudaFree(h->W);
        h->U = h->W = nullptr;
        ck(cudaMalloc(&h->U, sizeof(double) * ld * m));
        ck(cudaMalloc(&h->W, sizeof(double) * ld * m));
        h->m_alloc = m;
    }
    if (d > h->d_alloc) {
        if (h->V) cudaFree(h->V);
        if (h->Vt_f) cudaFree(h->Vt_f);
        h->V = nullptr;
        h->Vt_f = nullptr;
        ck(cudaMalloc(&h->V, sizeof(double) * ld * d));
        if (h->opts.precision == ISIRA_MIXED) ck(cudaMalloc(&h->Vt_f, sizeof(float) * ld * d));
        h->d_alloc = d;
    }
}

// Orthonormalise Z against [U(:,0:k) V(:,0:c) 1] and append it as column k (with W, H).
// Replaces Z by random vectors while the orthogonalisation breaks down.
bool expand_basis(isira_handle h, int k, int c) {
    OuterArgs oa = make_outer(h);
    cudaStream_t s = h->stream;
    for (int attempt = 0; attempt < 8; ++attempt) {
        outer_cgs2(oa, k, c, s);
        h->stats.kernel_launches += 3;
        sync(h);
        if (h->pending_inner_stats) {   // the graph-driven inner solve has finished by now
            const int its = hst(h)->inner_iters;
            h->stats.inner_iters += its;
            h->stats.spmv_launches += its;
            h->stats.kernel_launches += (long long)(h->pending_inner_stats > 1 ? h->pending_inner_stats : 3) * its;
            h->pending_inner_stats = 0;
        }
        const double zin = hst(h)->cgs_in, zout = hst(h)->cgs_out;
        if (zout > 1e-10 * zin && zout > 0.0 && std::isfinite(zout)) {
            outer_expand(oa, k, h->lanes, s);
            h->stats.kernel_launches += 3;
            return true;
        }
        h->stats.breakdowns += 1;
        outer_random(oa, h->opts.seed, (uint64_t)(1 + h->stats.breakdowns), s);
        h->stats.kernel_launches += 1;
    }
    return false;
}

// Gather launch shape: threads per CTA (kThreads: as many CTAs per SM as fit, at most 8;
// kBigBlock: one per SM) and the shared-memory bytes of the hub block x[0:hub) (0: none).
void apply_gather_shape(isira_handle h, int tpb, int hub_bytes) {
    RowSched& rs = h->rs;
    rs.tpb = tpb;
    rs.hub = hub_bytes > 0 ? (int)h->n : 0;
    rs.hub_bytes = hub_bytes > 0 ? hub_bytes : 0;
    const int wpb = tpb / 32;
    int ctas = gather_ctas_per_sm(tpb, rs.hub_bytes);
    if (tpb == kThreads) ctas = std::min(ctas, 8);
    if (ctas < 1) throw StatusError{ISIRA_ERR_INVALID_ARG};
    const int64_t n_units = rs.n_units();
    rs.n_warps = (int)std::max<int64_t>(wpb, std::min<int64_t>((int64_t)h->nsm * ctas * wpb,
                                                               (n_units + wpb - 1) / wpb * wpb));
}

// hub block bytes for a cap (bytes of shared memory), rounded to 128 and never above the vector
int hub_bytes_for(isira_handle h, int64_t cap) {
    cap = std::min<int64_t>(cap, h->smem_max) / 128 * 128;
    return (int)std::min<int64_t>(cap, (h->n * (int64_t)sizeof(double) + 127) / 128 * 128);
}

struct TuneKey {
    int dev, prec, sell, reorder, lanes_fixed, logn, mdeg, logmax, gb, hub_kb;
    bool operator<(const TuneKey& o) const {
        return std::tie(dev, prec, sell, reorder, lanes_fixed, logn, mdeg, logmax, gb, hub_kb) <
               std::tie(o.dev, o.prec, o.sell, o.reorder, o.lanes_fixed, o.logn, o.mdeg, o.logmax, o.gb, o.hub_kb);
    }
};
struct TuneVal { int tpb, hub_bytes, lanes; };
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;

template <typename T>
float time_gather(isira_handle h, InnerBuffers<T>& b, int lanes, cudaEvent_t e0, cudaEvent_t e1) {
    cudaStream_t s = h->stream;
    InnerArgs<T> a = make_args<T>(h, b, 0.0, 0, nullptr, h->ld, 1e-3, 1);
    inner_opstats<T>(a, a.z0, s);          // a fresh state: not done, iteration 0
    float tot = 0.f;
    for (int rep = 0; rep < 4; ++rep) {
        ck(cudaEventRecord(e0, s));
        inner_gather<T>(a, lanes, s);
        ck(cudaEventRecord(e1, s));
        sync(h);
        float ms = 0.f;
        ck(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) tot += ms;
    }
    return tot;
}

// Autotuner of the inner SpMV gather: times the gather kernel of the handle's precision on this
// graph for every candidate launch shape (and lane count of the CSR tiles, when the light rows
// are not sliced), keeps the fastest, and caches the choice per device, precision and graph-
// statistics bucket (log2 n, mean degree in half-octaves, log2 of the maximum degree), so graphs
// of the same kind (a batch) are timed once.  Small graphs (n < 100k, launch-bound) get the
// default shape without timing.
void autotune_gather(isira_handle h) {
    const isira_opts& o = h->opts;
    RowSched& rs = h->rs;
    const double mean = (double)h->nnz / (double)h->n;
    const int heur = mean <= 3.0 ? 1 : (mean <= 6.0 ? 2 : (mean <= 12.0 ? 4 : 8));
    const bool lanes_fixed = o.spmv_lanes > 0;
    int l = o.spmv_lanes;
    const int lanes0 = lanes_fixed ? ((l == 1 || l == 2 || l == 4 || l == 8 || l == 16 || l == 32) ? l : 8) : heur;
    // candidate shapes, filtered by the options the caller fixed
    std::vector<std::pair<int, int>> shapes;
    const int big_hub = (h->perm && o.hub_kb >= 0)
                            ? hub_bytes_for(h, o.hub_kb > 0 ? (int64_t)o.hub_kb * 1024 : (int64_t)kDefaultHubBytes) : 0;
    const int small_hub = (h->perm && o.hub_kb >= 0)
                              ? hub_bytes_for(h, o.hub_kb > 0 ? (int64_t)o.hub_kb * 1024 : (int64_t)48 * 1024) : 0;
    const int order_perm[2] = {kBigBlock, kThreads}, order_plain[2] = {kThreads, kBigBlock};
    for (int tpb : h->perm ? order_perm : order_plain) {
        if (o.gather_block != 0 && o.gather_block != tpb) continue;
        const int hub = tpb == kBigBlock ? big_hub : small_hub;
        if (o.hub_kb >= 0 && hub > 0) shapes.push_back({tpb, hub});
        if (o.hub_kb <= 0 || !h->perm) shapes.push_back({tpb, 0});
    }
    if (shapes.empty()) shapes.push_back({kThreads, 0});
    // default (untimed) shape: the first candidate
    apply_gather_shape(h, shapes[0].first, shapes[0].second);
    h->lanes = lanes0;
    // the slices-only kernels ignore the launch shape (their grid is one full wave of 256-thread CTAs)
    if (h->n < 100000 || slices_only(rs) || (shapes.size() == 1 && (lanes_fixed || rs.sell))) return;
    int dev = 0;
    ck(cudaGetDevice(&dev));
    auto ilog2 = [](double v) { return (int)std::floor(std::log2(std::max(1.0, v))); };
    const TuneKey key{dev, o.precision, rs.sell, o.reorder, lanes_fixed ? lanes0 : 0, ilog2((double)h->n),
                      (int)std::floor(2.0 * std::log2(std::max(1.0, mean))), ilog2((double)h->max_degree),
                      o.gather_block, o.hub_kb};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            apply_gather_shape(h, it->second.tpb, it->second.hub_bytes);
            h->lanes = it->second.lanes;
            return;
        }
    }
    std::vector<int> lane_list;
    if (lanes_fixed || rs.sell) lane_list.push_back(lanes0);
    else lane_list = {1, 2, 4, 8, 16, 32};
    cudaEvent_t e0, e1;
    ck(cudaEventCreate(&e0));
    ck(cudaEventCreate(&e1));
    float best = 1e30f;
    TuneVal bv{shapes[0].first, shapes[0].second, lanes0};
    for (const auto& sh : shapes) {
        apply_gather_shape(h, sh.first, sh.second);
        for (int ln : lane_list) {
            const float t = o.precision == ISIRA_MIXED ? time_gather<float>(h, h->fb, ln, e0, e1)
                                                       : time_gather<double>(h, h->db, ln, e0, e1);
            if (t < best) {
                best = t;
                bv = TuneVal{sh.first, sh.second, ln};
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    apply_gather_shape(h, bv.tpb, bv.hub_bytes);
    h->lanes = bv.lanes;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = bv;
}

void free_handle(isira_handle h) {
    if (!h) return;
    void* ptrs[] = {h->own_w, h->wf, h->degwd, h->degwf, h->sell_wd, h->sell_wf, h->gsum, h->deg32, h->sell_off, h->sell_ci, h->own_rp, h->own_ci, h->perm, h->inv, h->item_row, h->item_k, h->item_partial,
                    h->item_count, h->warp_start, h->U, h->W, h->V, h->H, h->theta, h->S, h->R, h->Z, h->dscratch,
                    h->arrow, h->partial, h->counter, h->Gm, h->Cinv, h->lam_dev, h->tres_dev, h->fb.base, h->fb.st,
                    h->db.base, h->db.st, h->Vt_f, h->fb.ml, h->db.ml, h->ml_dv};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    ml_free(h->fb.H);
    ml_free(h->db.H);
    for (cudaGraphExec_t g : h->ml_graph)
        if (g) cudaGraphExecDestroy(g);
    if (h->hs) cudaFreeHost(h->hs);
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    if (h->sync_ev) cudaEventDestroy(h->sync_ev);
    for (cudaGraphExec_t g : h->inner_graph)
        if (g) cudaGraphExecDestroy(g);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    delete h;
}

isira_status map_cuda(cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) return ISIRA_ERR_OOM;
    return ISIRA_ERR_CUDA;
}

}  // namespace

namespace {

// V (caller's numbering, n-by-c, ld n) into the solver's numbering, ld h->ld, precision T
template <typename T>
T* internal_V(isira_handle h, const double* d_V, int c, cudaStream_t s) {
    if (c <= 0) return nullptr;
    double* Vd = nullptr;
    ck(cudaMalloc(&Vd, sizeof(double) * (size_t)h->ld * c));
    for (int t = 0; t < c; ++t) {
        if (h->perm) to_internal<double>(d_V + (size_t)t * h->n, h->perm, h->n, Vd + (size_t)t * h->ld, s);
        else ck(cudaMemcpyAsync(Vd + (size_t)t * h->ld, d_V + (size_t)t * h->n, sizeof(double) * h->n,
                                cudaMemcpyDeviceToDevice, s));
    }
    if (sizeof(T) == sizeof(double)) return reinterpret_cast<T*>(Vd);
    float* Vf = nullptr;
    ck(cudaMalloc(&Vf, sizeof(float) * (size_t)h->ld * c));
    for (int t = 0; t < c; ++t) copy_vcol<float>(Vd + (size_t)t * h->ld, Vf + (size_t)t * h->ld, h->n, s);
    ck(cudaStreamSynchronize(s));
    cudaFree(Vd);
    return reinterpret_cast<T*>(Vf);
}

template <typename T>
void apply_operator_t(isira_handle h, InnerBuffers<T>& b, double sigma, int c, const double* d_V, const T* d_x,
                      T* d_y) {
    cudaStream_t s = h->stream;
    alloc_inner(h, b);
    T* Vt = internal_V<T>(h, d_V, c, s);
    InnerArgs<T> a = make_args<T>(h, b, sigma, c, Vt, h->ld, 1e-3, 1);
    if (h->perm) to_internal<T>(d_x, h->perm, h->n, a.z0, s);
    else ck(cudaMemcpyAsync(a.z0, d_x, sizeof(T) * h->n, cudaMemcpyDeviceToDevice, s));
    ck(cudaMemsetAsync(a.z0 + h->trim, 0, sizeof(T), s));   // x_i is treated as 0
    inner_opstats<T>(a, a.z0, s);
    inner_apply<T>(a, h->lanes, s);
    if (h->perm) to_external<T>(a.Y, h->perm, h->n, d_y, s);
    else ck(cudaMemcpyAsync(d_y, a.Y, sizeof(T) * h->n, cudaMemcpyDeviceToDevice, s));
    sync(h);
    if (Vt) cudaFree(Vt);
}

}  // namespace

namespace {
template <typename T>
void precond_apply_t(isira_handle h, InnerBuffers<T>& b, const T* d_x, T* d_y) {
    cudaStream_t s = h->stream;
    alloc_inner(h, b);
    ensure_ml(h, b);
    InnerArgs<T> a = make_args<T>(h, b, 0.0, 0, nullptr, h->ld, 1e-3, 1);
    T* xin = a.rcur;
    T* yout = a.wv;
    if (h->perm) to_internal<T>(d_x, h->perm, h->n, xin, s);
    else ck(cudaMemcpyAsync(xin, d_x, sizeof(T) * h->n, cudaMemcpyDeviceToDevice, s));
    GatherFn<T> gather = [&](const T* x, T* g, cudaStream_t st) { inner_gather_vec<T>(a, x, g, h->lanes, nullptr, st); };
    ml_vcycle<T>(b.H, xin, yout, gather, (T)kMlOmega, ml_alpha<T>(h), nullptr, false, false, s);
    if (h->perm) to_external<T>(yout, h->perm, h->n, d_y, s);
    else ck(cudaMemcpyAsync(d_y, yout, sizeof(T) * h->n, cudaMemcpyDeviceToDevice, s));
    sync(h);
}
}  // namespace

extern "C" {

void isira_default_opts(isira_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = ISIRA_MIXED;
    o->m = 0;
    o->q = 0;
    o->tau_inner = 1e-3;
    o->max_inner = 5000;
    o->max_outer = 20000;
    o->trim_index = -1;
    o->delta = 0.0;
    o->sigma_omega = 0.1;
    o->drop_rank1 = 0;
    o->validate = 0;
    o->seed = 1;
    o->spmv_lanes = 0;
    o->inner_chunk = 16;
    o->inner_graph = 1;
    o->reorder = 1;
    o->gather_block = 0;
    o->hub_kb = 0;
    o->gather_sched = 0;
    o->index_vec = 0;
    o->gather_chunk = 0;
    o->sell = 1;
    o->precond = -1;
    o->ml_alpha = 0.0;
    o->rr_arrow = 1;
    o->blocking_sync = 0;
}

const char* isira_error_string(isira_status s) {
    switch (s) {
        case ISIRA_OK: return "ok";
        case ISIRA_ERR_INVALID_ARG: return "invalid argument";
        case ISIRA_ERR_BAD_GRAPH: return "malformed CSR graph";
        case ISIRA_ERR_NOT_CONNECTED: return "graph is not connected (second zero eigenvalue)";
        case ISIRA_ERR_NO_CONVERGENCE: return "outer iteration limit reached before all eigenpairs converged";
        case ISIRA_ERR_CUDA: return "CUDA runtime error";
        case ISIRA_ERR_OOM: return "out of memory";
        case ISIRA_ERR_NOT_SOLVED: return "no successful solve on this handle";
        case ISIRA_ERR_LIMIT: return "request exceeds the fixed scratch of the allocation-free entry point (c <= 8)";
        case ISIRA_ERR_DEVICE_TIMEOUT: return "a bounded wait inside a kernel ran out (the results of the call are not valid)";
    }
    return "unknown status";
}

isira_status isira_create(isira_handle* out, int64_t n, int64_t nnz, const int64_t* d_row_ptr,
                          const int32_t* d_col_idx, const isira_opts* opts, void* stream) {
    return isira_create_weighted(out, n, nnz, d_row_ptr, d_col_idx, nullptr, opts, stream);
}

isira_status isira_create_weighted(isira_handle* out, int64_t n, int64_t nnz, const int64_t* d_row_ptr,
                                   const int32_t* d_col_idx, const double* d_weights, const isira_opts* opts,
                                   void* stream) {
    if (!out) return ISIRA_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 3 || nnz < 2 || nnz > ((int64_t)1 << 40) || !d_row_ptr || !d_col_idx || n > INT32_MAX)
        return ISIRA_ERR_INVALID_ARG;
    isira_handle h = new (std::nothrow) isira_handle_s();
    if (!h) return ISIRA_ERR_OOM;
    try {
        h->n = n;
        h->nnz = nnz;
        h->ld = (n + 31) / 32 * 32;
        h->rp = d_row_ptr;
        h->ci = d_col_idx;
        h->w_user = d_weights;
        h->stream = (cudaStream_t)stream;
        if (opts) h->opts = *opts; else isira_default_opts(&h->opts);
        const double* d_w = d_weights;
        if (h->opts.precision != ISIRA_FP64 && h->opts.precision != ISIRA_MIXED) throw StatusError{ISIRA_ERR_INVALID_ARG};
        int dev = 0;
        ck(cudaGetDevice(&dev));
        ck(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev));
        cudaStream_t s = h->stream;
        if (h->opts.validate) {
            int* flag = nullptr;
            ck(cudaMalloc(&flag, sizeof(int)));
            int f = validate_csr(d_row_ptr, d_col_idx, n, nnz, flag, s);
            cudaFree(flag);
            if (f) throw StatusError{ISIRA_ERR_BAD_GRAPH};
        }
        // Remark 4.1: degrees, maximum degree, trimmed index, delta; row classes of the scheduler
        const int light_deg = 64;
        int64_t* scratch = nullptr;
        ck(cudaMalloc(&scratch, sizeof(int64_t) * 5 * 1024));
        DegreeInfo di{};
        int64_t user_trim = -1;
        if (h->opts.reorder) {
            setup_degrees(d_row_ptr, n, light_deg, nullptr, nullptr, 0, scratch, &di, s);   // max degree
            ck(cudaMalloc(&h->own_rp, sizeof(int64_t) * (size_t)(n + 1)));
            // padded to a multiple of 4 entries: the gathers read the relabelled copy in 128-bit chunks
            const size_t nnz_pad = ((size_t)nnz + 3) / 4 * 4;
            ck(cudaMalloc(&h->own_ci, sizeof(int32_t) * nnz_pad));
            ck(cudaMemsetAsync(h->own_ci + nnz, 0, sizeof(int32_t) * (nnz_pad - (size_t)nnz), s));
            ck(cudaMalloc(&h->perm, sizeof(int32_t) * (size_t)n));
            ck(cudaMalloc(&h->inv, sizeof(int32_t) * (size_t)n));
            if (d_weights) ck(cudaMalloc(&h->own_w, sizeof(double) * (size_t)nnz));
            ck(build_reordered_graph(d_row_ptr, d_col_idx, d_weights, n, nnz, di.max_degree, h->own_rp, h->own_ci,
                                     h->own_w, h->perm, h->inv, s));
            if (h->opts.trim_index >= 0 && h->opts.trim_index < n) {
                int32_t t = 0;
                ck(cudaMemcpy(&t, h->inv + h->opts.trim_index, sizeof(int32_t), cudaMemcpyDeviceToHost));
                user_trim = h->opts.trim_index;
                h->opts.trim_index = t;
            }
            d_row_ptr = h->own_rp;
            d_col_idx = h->own_ci;
            if (d_weights) d_w = h->own_w;
            h->rp = d_row_ptr;
            h->ci = d_col_idx;
        }
        setup_degrees(d_row_ptr, n, light_deg, nullptr, nullptr, 0, scratch, &di, s);   // counts
        const size_t ni = (size_t)std::max<int64_t>(1, di.n_items);
        ck(cudaMalloc(&h->item_row, sizeof(int32_t) * ni));
        ck(cudaMalloc(&h->item_k, sizeof(int32_t) * ni));
        ck(cudaMalloc(&h->item_partial, sizeof(double) * ni));
        ck(cudaMalloc(&h->item_count, sizeof(unsigned) * ni));
        ck(cudaMemsetAsync(h->item_count, 0, sizeof(unsigned) * ni, s));
        setup_degrees(d_row_ptr, n, light_deg, h->item_row, h->item_k, di.n_items, scratch, &di, s);   // fill
        sync(h);
        cudaFree(scratch);
        h->max_degree = di.max_degree;
        if (di.max_degree < 1) throw StatusError{ISIRA_ERR_BAD_GRAPH};
        double maxdiag = (double)di.max_degree;       // largest diagonal entry of L (Remark 4.1)
        if (d_w) {
            // weighted Laplacian: diagonal = weight sums; trimmed vertex = largest diagonal entry
            // (smallest vertex id of the caller's numbering on ties)
            ck(cudaMalloc(&h->degwd, sizeof(double) * (size_t)h->ld));
            ck(cudaMalloc(&h->degwf, sizeof(float) * (size_t)h->ld));
            ck(cudaMalloc(&h->wf, sizeof(float) * (size_t)std::max<int64_t>(1, nnz)));
            setup_weighted(d_row_ptr, d_w, n, h->ld, nnz, h->degwd, h->degwf, h->wf, s);
            std::vector<double> dw((size_t)n);
            std::vector<int32_t> pm;
            ck(cudaMemcpyAsync(dw.data(), h->degwd, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, s));
            if (h->perm) {
                pm.resize((size_t)n);
                ck(cudaMemcpyAsync(pm.data(), h->perm, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
            }
            sync(h);
            int64_t best = -1, best_user = -1;
            maxdiag = 0.0;
            for (int64_t r = 0; r < n; ++r) {
                const int64_t ru = h->perm ? (int64_t)pm[(size_t)r] : r;
                if (!(dw[(size_t)r] > 0.0)) throw StatusError{ISIRA_ERR_BAD_GRAPH};
                if (dw[(size_t)r] > maxdiag || (dw[(size_t)r] == maxdiag && ru < best_user)) {
                    maxdiag = dw[(size_t)r];
                    best = r;
                    best_user = ru;
                }
            }
            di.argmax = best;
        }
        h->trim = (h->opts.trim_index >= 0 && h->opts.trim_index < n) ? h->opts.trim_index : di.argmax;
        h->trim_user = h->trim;
        if (h->perm) {
            int32_t t = 0;
            ck(cudaMemcpy(&t, h->perm + h->trim, sizeof(int32_t), cudaMemcpyDeviceToHost));
            h->trim_user = t;
            if (user_trim >= 0) h->opts.trim_index = user_trim;
        }
        h->delta = h->opts.delta > 0.0 ? h->opts.delta : 2.0 * maxdiag;
        h->normL = 2.0 * maxdiag;
        h->n_long = di.n_long;
        h->n_items = di.n_items;
        if (di.n_items > INT32_MAX) throw StatusError{ISIRA_ERR_INVALID_ARG};
        RowSched& rs = h->rs;
        rs.rp = d_row_ptr;
        rs.ci = d_col_idx;
        rs.n = n;
        rs.item_row = h->item_row;
        rs.item_k = h->item_k;
        rs.item_partial = h->item_partial;
        rs.item_count = h->item_count;
        rs.n_items = (int)di.n_items;
        rs.light_deg = light_deg;
        rs.ci_vec = h->own_ci != nullptr && h->opts.index_vec == 1 && !d_w;
        rs.wd = d_w;
        rs.wf = h->wf;
        rs.degwd = h->degwd;
        rs.degwf = h->degwf;
        rs.chunk = (h->opts.gather_chunk >= 1 && h->opts.gather_chunk <= 32) ? h->opts.gather_chunk : kUnitChunk;
        // sliced ELL copy of the light rows: the degree-descending numbering puts the long rows first
        rs.sell = 0;
        rs.n_slices = 0;
        rs.light0 = n;
        if (h->perm && h->opts.sell != 0) {
            const int64_t ns = (n - di.n_long + 31) / 32;
            if (ns > INT32_MAX / 2) throw StatusError{ISIRA_ERR_INVALID_ARG};
            ck(cudaMalloc(&h->sell_off, sizeof(int64_t) * (size_t)(ns + 1)));
            ck(build_sell(d_row_ptr, d_col_idx, d_w, n, di.n_long, ns, h->sell_off, &h->sell_ci,
                          d_w ? &h->sell_wd : nullptr, &h->sell_total, s));
            if (d_w) {
                ck(cudaMalloc(&h->sell_wf, sizeof(float) * (size_t)std::max<int64_t>(1, h->sell_total)));
                copy_cast<float>(h->sell_wd, h->sell_wf, h->sell_total, s);
                rs.swd = h->sell_wd;
                rs.swf = h->sell_wf;
            }
            rs.sell_ci = h->sell_ci;
            rs.sell_off = h->sell_off;
            rs.n_slices = (int)ns;
            rs.light0 = di.n_long;
            rs.sell = 1;
        }
        // slices are always taken dynamically; the static partition's cost model knows CSR tiles only
        rs.dyn = h->opts.gather_sched == 0 || rs.sell;
        if (rs.n_units() > INT32_MAX / 2) throw StatusError{ISIRA_ERR_INVALID_ARG};
        {
            int optin = 0;
            ck(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
            h->smem_max = std::max(0, optin - 1024);          // room for static shared memory
            ck(inner_gather_attrs<float>(h->smem_max));
            ck(inner_gather_attrs<double>(h->smem_max));
            ck(outer_gather_attrs(h->smem_max));
        }
        // the launch shape is chosen at the end of create (autotune_gather); buffers are sized for
        // every candidate: at most 8 CTAs of 8 warps per SM
        ck(cudaMalloc(&h->warp_start, sizeof(int32_t) * (size_t)(h->nsm * 64 + 1)));
        rs.warp_start = h->warp_start;
        // up to 8 CTAs per SM (a full SM of 256-thread CTAs); register-heavy row kernels are cut to
        // one wave of their resident CTAs at launch
        h->ew_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, (int64_t)h->nsm * 8));
        h->ts_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 63) / 64, (int64_t)h->nsm * 6));
        // shared scratch for block partial sums: 512 slots x the largest grid
        const int64_t maxgrid = std::max<int64_t>({(int64_t)h->nsm * 8, (int64_t)h->ew_blocks, (int64_t)h->ts_blocks});
        h->partial_elems = (size_t)512 * (size_t)maxgrid;
        ck(cudaMalloc(&h->partial, sizeof(double) * h->partial_elems));
        ck(cudaMalloc(&h->counter, sizeof(unsigned) * 8));
        ck(cudaMemsetAsync(h->counter, 0, sizeof(unsigned) * 8, s));
        rs.hub_timeouts = h->counter + 4;
        rs.sched = h->counter + 5;
        ck(cudaMalloc(&h->H, sizeof(double) * kMMax * kMMax));
        ck(cudaMalloc(&h->theta, sizeof(double) * kMMax));
        ck(cudaMalloc(&h->S, sizeof(double) * kMMax * kMMax));
        ck(cudaMalloc(&h->arrow, sizeof(ArrowWork)));
        ck(cudaMemsetAsync(h->arrow, 0, sizeof(ArrowWork), s));
        ck(cudaMalloc(&h->R, sizeof(double) * (size_t)h->ld));
        ck(cudaMalloc(&h->Z, sizeof(double) * (size_t)h->ld));
        ck(cudaMalloc(&h->gsum, sizeof(double) * (size_t)h->ld));
        ck(cudaMemsetAsync(h->gsum, 0, sizeof(double) * (size_t)h->ld, s));
        ck(cudaMalloc(&h->deg32, sizeof(int32_t) * (size_t)h->ld));
        setup_deg32(d_row_ptr, n, h->ld, h->deg32, s);
        ck(cudaMalloc(&h->dscratch, sizeof(double) * 512));
        ck(cudaMalloc(&h->Gm, sizeof(double) * kCMax * kCMax));
        ck(cudaMalloc(&h->Cinv, sizeof(double) * kCMax * kCMax));
        ck(cudaMalloc(&h->lam_dev, sizeof(double) * kCMax));
        ck(cudaMalloc(&h->tres_dev, sizeof(double) * kCMax));
        ck(cudaHostAlloc(&h->hs, sizeof(HostStatus), cudaHostAllocMapped));
        std::memset(h->hs, 0, sizeof(HostStatus));
        ck(cudaHostGetDevicePointer((void**)&h->hs_dev, h->hs, 0));
        h->rs.err = &h->hs_dev->dev_error;
        if (h->opts.precision == ISIRA_MIXED) alloc_inner(h, h->fb); else alloc_inner(h, h->db);
        if (h->opts.precond < -1 || h->opts.precond > 1) throw StatusError{ISIRA_ERR_INVALID_ARG};
        int chunk = h->opts.inner_chunk > 0 ? h->opts.inner_chunk : 16;
        h->ev.resize(4 * chunk);
        for (auto& e : h->ev) ck(cudaEventCreate(&e));
        if (h->opts.blocking_sync)
            ck(cudaEventCreateWithFlags(&h->sync_ev, cudaEventBlockingSync | cudaEventDisableTiming));
        sync(h);
        autotune_gather(h);
        choose_preconditioner(h);
        if (!rs.dyn) {   // static partition of the CSR work units for the chosen shape
            const int64_t n_units = rs.n_units();
            int64_t* cost = nullptr;
            int64_t* prefix = nullptr;
            ck(cudaMalloc(&cost, sizeof(int64_t) * (size_t)n_units));
            ck(cudaMalloc(&prefix, sizeof(int64_t) * (size_t)(n_units + 1)));
            setup_partition(d_row_ptr, n, h->item_row, h->item_k, di.n_items, light_deg, rs.n_warps, cost, prefix,
                            h->warp_start, s);
            sync(h);
            cudaFree(cost);
            cudaFree(prefix);
        }
        h->stats.n = n;
        h->stats.nnz = nnz;
        h->stats.trim_index = h->trim_user;
        h->stats.max_degree = h->max_degree;
        h->stats.delta = h->delta;
        h->stats.norm_L = h->normL;
        h->stats.spmv_lanes = h->lanes;
        h->stats.n_long_rows = h->n_long;
        h->stats.n_work_items = h->n_items;
        h->stats.gather_block = h->rs.tpb;
        h->stats.hub_bytes = h->rs.hub_bytes;
        h->stats.sell_entries = h->sell_total;
        h->stats.max_diag = maxdiag;
        h->stats.precond = h->use_ml ? 1 : 0;
        h->stats.ml_levels = h->use_ml ? (h->opts.precision == ISIRA_MIXED ? h->fb.H.nlev : h->db.H.nlev) : 0;
        h->stats.ml_coarse_n = 0;
        h->stats.ml_coarse_nnz = 0;
        if (h->use_ml) {
            auto add = [h](const auto& lev) {
                for (size_t l = 1; l < lev.size(); ++l) {
                    h->stats.ml_coarse_n += lev[l].n;
                    h->stats.ml_coarse_nnz += lev[l].nnz;
                }
            };
            if (h->opts.precision == ISIRA_MIXED) add(h->fb.H.lev);
            else add(h->db.H.lev);
        }
        h->stats.inner_iters = 0;
        h->stats.inner_solves = 0;
        h->stats.kernel_launches = 0;
        h->pending_inner_stats = 0;
    } catch (CudaError& e) {
        isira_status st = map_cuda(e.e);
        free_handle(h);
        return st;
    } catch (StatusError& e) {
        free_handle(h);
        return e.s;
    }
    *out = h;
    return ISIRA_OK;
}

void isira_destroy(isira_handle h) { free_handle(h); }

isira_status isira_set_profiling(isira_handle h, int on) {
    if (!h) return ISIRA_ERR_INVALID_ARG;
    h->profiling = on ? 1 : 0;
    return ISIRA_OK;
}

isira_status isira_get_stats(isira_handle h, isira_stats* out) {
    if (!h || !out) return ISIRA_ERR_INVALID_ARG;
    unsigned to = 0;
    if (h->counter) {
        cudaError_t e = cudaMemcpyAsync(&to, h->counter + 4, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return map_cuda(e);
    }
    h->stats.hub_timeouts = to;
    *out = h->stats;
    return ISIRA_OK;
}

isira_status isira_solve(isira_handle h, int d, double sigma, double tol, const double* d_u0) {
    if (!h) return ISIRA_ERR_INVALID_ARG;
    if (d < 1 || d > kCMax || d > h->n - 2 || !(tol >= 0.0) || !std::isfinite(sigma)) return ISIRA_ERR_INVALID_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    NvtxRange range_solve("isira_solve");
    isira_status status = ISIRA_OK;
    h->solved = false;
    h->rhist.clear();
    clear_dev_error(h);
    try {
        const isira_opts& o = h->opts;
        int m = o.m > 0 ? o.m : std::max(20, 2 * d + 10);
        int q = o.q > 0 ? o.q : std::max(d + 2, m / 2);
        m = std::min<int64_t>({(int64_t)m, (int64_t)kMMax, h->n - 1});
        q = std::min(q, m - 1);
        if (q < d || m < 2) return ISIRA_ERR_INVALID_ARG;
        const double tau = o.tau_inner > 0.0 ? o.tau_inner : 1e-3;
        const int max_inner = o.max_inner > 0 ? o.max_inner : 5000;
        const int max_outer = o.max_outer > 0 ? o.max_outer : 20000;
        const double omega = o.sigma_omega > 0.0 ? o.sigma_omega : 0.1;
        ensure_outer(h, m, d);
        cudaStream_t s = h->stream;
        // reset counters
        const isira_stats keep = h->stats;
        h->stats.n_locked = 0;
        h->stats.outer_steps = 0;
        h->stats.restarts = 0;
        h->stats.breakdowns = 0;
        h->stats.inner_iters = 0;
        h->stats.inner_solves = 0;
        h->stats.spmv_launches = 0;
        h->stats.inner_phase1_ms = 0.0;
        h->stats.inner_phase1_timed = 0;
        h->stats.inner_phase1_csum = 0;
        h->stats.inner_rows_ms = 0.0;
        h->stats.inner_phase2_ms = 0.0;
        h->stats.w_columns = 0;
        h->stats.kernel_launches = 0;
        h->stats.rr_arrow = 0;
        h->stats.rr_jacobi = 0;
        h->stats.rr_refused = 0;
        (void)keep;
        h->lam.assign(d, 0.0);
        OuterArgs oa = make_outer(h);
        ck(cudaMemsetAsync(h->H, 0, sizeof(double) * kMMax * kMMax, s));
        // start basis U_{k0}, k0 = 1 (Algorithm 2 REQUIRE): the given vector, or a SplitMix64 one
        if (d_u0 && h->perm) to_internal<double>(d_u0, h->perm, h->n, h->Z, s);
        else if (d_u0) ck(cudaMemcpyAsync(h->Z, d_u0, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, s));
        else outer_random(oa, o.seed, 0, s);
        h->stats.kernel_launches += d_u0 ? 0 : 1;
        if (!expand_basis(h, 0, 0)) throw StatusError{ISIRA_ERR_NO_CONVERGENCE};
        int k = 1, c = 0;
        double sig = sigma;
        bool gram_dirty = true;
        int warm_w = 0;   // S's leading warm_w block diagonalises H's leading block (warm start)
        // the arrowhead path may drop off-diagonal entries of Q0^T H Q0 up to 1% of tol in 2-norm
        const double off_cap = 0.01 * tol / kMMax;
        int arrow_skip = 0, arrow_backoff = 1;
        while (true) {
            if (h->stats.outer_steps >= max_outer) { status = ISIRA_ERR_NO_CONVERGENCE; break; }
            h->stats.outer_steps += 1;
            h->stats.w_columns += k;
            // Rayleigh-Ritz: the arrowhead path after one expansion of a diagonalised H, else Jacobi
            const bool try_arrow = o.rr_arrow != 0 && k >= 2 && warm_w >= k - 1 && warm_w >= 1 && arrow_skip == 0;
            if (arrow_skip > 0) --arrow_skip;
            nvtxRangePushA("rayleigh_ritz+residual");
            if (try_arrow) {
                int nl = 0;
                outer_arrow_eig(h->H, kMMax, k, warm_w, h->theta, h->S, kMMax, h->arrow, h->hs_dev, off_cap, &nl, s);
                h->stats.kernel_launches += nl;
            } else {
                outer_sym_eig(h->H, kMMax, k, h->theta, h->S, kMMax, h->hs_dev, warm_w, s);
                h->stats.kernel_launches += 1;
                h->stats.rr_jacobi += 1;
            }
            outer_residual(oa, k, s);                                              // residual
            h->stats.kernel_launches += 1;
            sync(h);
            if (try_arrow) {
                if (hst(h)->eig_path < 0) {        // Q0 no longer diagonalises H to rounding: Jacobi
                    outer_sym_eig(h->H, kMMax, k, h->theta, h->S, kMMax, h->hs_dev, warm_w, s);
                    outer_residual(oa, k, s);
                    h->stats.kernel_launches += 2;
                    h->stats.rr_jacobi += 1;
                    h->stats.rr_refused += 1;
                    arrow_skip = arrow_backoff;
                    arrow_backoff = std::min(2 * arrow_backoff, 32);
                    sync(h);
                } else {
                    h->stats.rr_arrow += 1;
                    arrow_backoff = 1;
                }
            }
            nvtxRangePop();
            warm_w = k;
            const double rn = hst(h)->rnorm, th1 = hst(h)->theta[0], th2 = hst(h)->theta[1];
            h->rhist.push_back(rn);
            const bool exhausted = (int64_t)(k + c) >= h->n - 1;
            if (rn < tol || exhausted) {                                           // lock
                NvtxRange range_lock("lock+purge");
                double* vcol = h->V + (size_t)c * h->ld;
                const bool more = (c + 1 < d);
                if (more && k >= 2) {
                    outer_purge(oa, k, vcol, s);                                   // v_j = U s1; purge
                    h->stats.kernel_launches += 2;
                } else {
                    outer_rotate(oa, h->U, k, 1, 0, vcol, s);                      // v_j = U s1
                    h->stats.kernel_launches += 1;
                }
                if (h->opts.precision == ISIRA_MIXED) {
                    copy_vcol<float>(vcol, h->Vt_f + (size_t)c * h->ld, h->n, s);
                    h->stats.kernel_launches += 1;
                }
                h->lam[c] = th1;
                ++c;
                h->stats.n_locked = c;
                if (c == d) break;
                gram_dirty = true;
                if (k >= 2) {                                                      // move sigma
                    const double move = std::max(omega * (th2 - th1), 0.01 * th2);
                    sig = th2 - move;
                    k -= 1;
                    warm_w = k;                        // the purge left S = eigenvectors of H
                } else {
                    outer_random(oa, o.seed, (uint64_t)(1000003 + c), s);
                    h->stats.kernel_launches += 1;
                    if (!expand_basis(h, 0, c)) { status = ISIRA_ERR_NO_CONVERGENCE; break; }
                    k = 1;
                    warm_w = 0;
                }
                continue;
            }
            if (k == m) {                                                          // restart
                NvtxRange range_restart("restart");
                outer_rotate(oa, h->U, k, 0, q, nullptr, s);
                outer_rotate(oa, h->W, k, 0, q, nullptr, s);
                outer_set_diag(oa, 0, q, s);
                h->stats.kernel_launches += 3;
                k = q;
                warm_w = q;
                h->stats.restarts += 1;
            }
            // inner solve of Eq. 2.14 and back-map Eq. 2.5 -> Z
            nvtxRangePushA("inner_solve");
            if (h->opts.precision == ISIRA_MIXED)
                run_inner<float>(h, h->fb, sig, c, h->Vt_f, h->ld, tau, max_inner, gram_dirty, h->R, h->dscratch,
                                 true, h->lam.data());
            else
                run_inner<double>(h, h->db, sig, c, h->V, h->ld, tau, max_inner, gram_dirty, h->R, h->dscratch,
                                  true, h->lam.data());
            gram_dirty = false;
            nvtxRangePop();
            // orthonormalise against [U V 1] and expand U, W, H
            NvtxRange range_expand("cgs2+expand");
            if (!expand_basis(h, k, c)) { status = ISIRA_ERR_NO_CONVERGENCE; break; }
            k += 1;
        }
        sync(h);
        h->n_locked = c;
        for (int j = 0; j < c; ++j)
            if (h->lam[j] < 1e-10 * h->normL) status = ISIRA_ERR_NOT_CONNECTED;
        h->solved = c > 0;
    } catch (CudaError& e) {
        status = map_cuda(e.e);
    } catch (StatusError& e) {
        status = e.s;
    }
    h->stats.solve_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return status;
}

isira_status isira_eigpairs(isira_handle h, double* h_eigvals, double* d_eigvecs, double* h_true_resid, int* n_out) {
    if (!h) return ISIRA_ERR_INVALID_ARG;
    if (!h->solved || h->n_locked < 1) return ISIRA_ERR_NOT_SOLVED;
    try {
        const int c = h->n_locked;
        std::vector<int> order(c);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return h->lam[a] < h->lam[b]; });
        cudaStream_t s = h->stream;
        if (h_eigvals)
            for (int j = 0; j < c; ++j) h_eigvals[j] = h->lam[order[j]];
        if (d_eigvecs)
            for (int j = 0; j < c; ++j) {
                if (h->perm)
                    to_external<double>(h->V + (size_t)order[j] * h->ld, h->perm, h->n, d_eigvecs + (size_t)j * h->n, s);
                else
                    ck(cudaMemcpyAsync(d_eigvecs + (size_t)j * h->n, h->V + (size_t)order[j] * h->ld,
                                       sizeof(double) * h->n, cudaMemcpyDeviceToDevice, s));
            }
        if (h_true_resid) {
            ck(cudaMemcpyAsync(h->lam_dev, h->lam.data(), sizeof(double) * c, cudaMemcpyHostToDevice, s));
            OuterArgs oa = make_outer(h);
            outer_true_residual(oa, c, h->lam_dev, h->tres_dev, h->lanes, s);
            std::vector<double> r2(c);
            ck(cudaMemcpyAsync(r2.data(), h->tres_dev, sizeof(double) * c, cudaMemcpyDeviceToHost, s));
            sync(h);
            for (int j = 0; j < c; ++j) h_true_resid[j] = std::sqrt(r2[order[j]]) / h->normL;
        }
        sync(h);
        if (n_out) *n_out = c;
    } catch (CudaError& e) {
        return map_cuda(e.e);
    } catch (StatusError& e) {
        return e.s;
    }
    return ISIRA_OK;
}

isira_status isira_apply_operator(isira_handle h, int precision, double sigma, int c, const double* d_V,
                                  const void* d_x, void* d_y) {
    if (!h || !d_x || !d_y || c < 0 || c >= kCMax || (c > 0 && !d_V) ||
        (precision != ISIRA_FP64 && precision != ISIRA_MIXED))
        return ISIRA_ERR_INVALID_ARG;
    clear_dev_error(h);
    try {
        if (precision == ISIRA_MIXED)
            apply_operator_t<float>(h, h->fb, sigma, c, d_V, static_cast<const float*>(d_x), static_cast<float*>(d_y));
        else
            apply_operator_t<double>(h, h->db, sigma, c, d_V, static_cast<const double*>(d_x),
                                     static_cast<double*>(d_y));
    } catch (CudaError& e) {
        return map_cuda(e.e);
    } catch (StatusError& e) {
        return e.s;
    }
    return ISIRA_OK;
}

isira_status isira_inner_solve(isira_handle h, int precision, double sigma, int c, const double* d_V,
                               const double* d_r, double tau, int max_it, double* d_z, int* iters, double* relres) {
    if (!h || !d_r || !d_z || c < 0 || c >= kCMax || (c > 0 && !d_V) || !(tau > 0.0) || max_it < 1 ||
        (precision != ISIRA_FP64 && precision != ISIRA_MIXED))
        return ISIRA_ERR_INVALID_ARG;
    clear_dev_error(h);
    try {
        cudaStream_t s = h->stream;
        // the right-hand side goes through the residual buffer, its norm through the scalar area
        if (h->perm) to_internal<double>(d_r, h->perm, h->n, h->R, s);
        else ck(cudaMemcpyAsync(h->R, d_r, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, s));
        const double one = 1.0;
        ck(cudaMemcpyAsync(h->dscratch + 300, &one, sizeof(double), cudaMemcpyHostToDevice, s));
        int its = 0;
        if (precision == ISIRA_MIXED) {
            alloc_inner(h, h->fb);
            float* Vt = internal_V<float>(h, d_V, c, s);
            its = run_inner<float>(h, h->fb, sigma, c, Vt, h->ld, tau, max_it, true, h->R, h->dscratch + 300);
            sync(h);
            if (Vt) cudaFree(Vt);
        } else {
            alloc_inner(h, h->db);
            double* Vt = internal_V<double>(h, d_V, c, s);
            its = run_inner<double>(h, h->db, sigma, c, Vt, h->ld, tau, max_it, true, h->R, h->dscratch + 300);
            sync(h);
            if (Vt) cudaFree(Vt);
        }
        // back-map (Eq. 2.5): remove the mean; the trimmed entry is already zero
        OuterArgs oa = make_outer(h);
        outer_cgs2(oa, 0, 0, s);   // with an empty basis the two passes only subtract the mean
        if (h->perm) to_external<double>(h->Z, h->perm, h->n, d_z, s);
        else ck(cudaMemcpyAsync(d_z, h->Z, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, s));
        sync(h);
        if (iters) *iters = its;
        if (relres) *relres = hst(h)->inner_relres;
    } catch (CudaError& e) {
        return map_cuda(e.e);
    } catch (StatusError& e) {
        return e.s;
    }
    return ISIRA_OK;
}


isira_status isira_precond_apply(isira_handle h, int precision, const void* d_x, void* d_y, int* levels,
                                 int64_t* coarse_n) {
    if (!h || !d_x || !d_y || (precision != ISIRA_FP64 && precision != ISIRA_MIXED)) return ISIRA_ERR_INVALID_ARG;
    clear_dev_error(h);
    try {
        if (precision == ISIRA_MIXED) {
            precond_apply_t<float>(h, h->fb, static_cast<const float*>(d_x), static_cast<float*>(d_y));
            if (levels) *levels = h->fb.H.nlev;
            if (coarse_n) *coarse_n = h->fb.H.n_coarse;
        } else {
            precond_apply_t<double>(h, h->db, static_cast<const double*>(d_x), static_cast<double*>(d_y));
            if (levels) *levels = h->db.H.nlev;
            if (coarse_n) *coarse_n = h->db.H.n_coarse;
        }
    } catch (CudaError& e) {
        return map_cuda(e.e);
    } catch (StatusError& e) {
        return e.s;
    }
    return ISIRA_OK;
}

isira_status isira_sym_eig(int k, const double* d_H, double* d_theta, double* d_S, void* stream) {
    if (k < 1 || k > kMMax || !d_H || !d_theta || !d_S) return ISIRA_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    outer_sym_eig(d_H, k, k, d_theta, d_S, k, nullptr, 0, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? ISIRA_OK : ISIRA_ERR_CUDA;
}

isira_status isira_residual_history(isira_handle h, double* h_rnorm, int cap, int* count) {
    if (!h || cap < 0 || (cap > 0 && !h_rnorm)) return ISIRA_ERR_INVALID_ARG;
    const int nh = (int)h->rhist.size();
    for (int i = 0; i < std::min(cap, nh); ++i) h_rnorm[i] = h->rhist[i];
    if (count) *count = nh;
    return ISIRA_OK;
}

isira_status isira_sym_eig_warm(int k, int warm_w, const double* d_H, double* d_theta, double* d_S, int* path,
                                void* stream) {
    if (k < 2 || k > kMMax || warm_w < k - 1 || warm_w > k || !d_H || !d_theta || !d_S)
        return ISIRA_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    ArrowWork* aw = nullptr;
    cudaError_t e = cudaMalloc(&aw, sizeof(ArrowWork));
    if (e != cudaSuccess) return ISIRA_ERR_OOM;
    int st = 1;
    e = cudaMemsetAsync(aw, 0, sizeof(ArrowWork), s);
    if (e == cudaSuccess) {
        outer_arrow_eig(d_H, k, k, warm_w, d_theta, d_S, k, aw, nullptr, HUGE_VAL, nullptr, s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, &aw->status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && st != 0) {
        outer_sym_eig(d_H, k, k, d_theta, d_S, k, nullptr, warm_w, s);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    cudaFree(aw);
    if (path) *path = st == 0 ? 1 : 0;
    return e == cudaSuccess ? ISIRA_OK : ISIRA_ERR_CUDA;
}

}  // extern "C"
