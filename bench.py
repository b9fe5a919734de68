#!/usr/bin/env python3
"""Benchmark: time to the k smallest positive Laplacian eigenpairs with iSIRA on one GB300.

Workload (default): 3-D 7-point grid 128^3 (n = 2,097,152), k = 20, mixed precision (FP32
inner solve with FP32 accumulation, FP64 outer loop); the plain-FP64 solve of the same graph
at the same tolerance is timed beside it.

Tolerance.  The paper's epsilon is an absolute bound on the Ritz residual (the lock test of
Algorithm 2).  The metric asks for relative residual ||L x - lambda x|| / ||L|| <= 1e-8
(||L|| := 2 * max degree) and eigenvalue relative error <= 1e-9.  Because the eigenvalue error
of a Ritz value behaves like ||r||^2 / gap, the second bar is the binding one for small,
clustered eigenvalues, so the timed solves use
    eps = min(1e-8 ||L||, sqrt(1e-10 * lambda_j * gap_j) over the wanted pairs),
with lambda_j and gap_j estimated from the Ritz values of one untimed solve at 1e-8 ||L||
(gaps below 1e-6 lambda_j are treated as one eigenvalue of higher multiplicity).

A step is one full isira_solve (all of Algorithm 2: inner solves, orthogonalisation,
Rayleigh-Ritz, restarts, locking).  Inputs are resident in HBM; the L2 is flushed (a 512 MB
write) between timed steps; each step is timed with CUDA events on the library's stream.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference] [--workload NAME]

With N > 1 (torchrun) every rank solves its own copy of the workload (replicas: the method
has no data-parallel split of one graph) and rank 0 prints the max over ranks; the batched
workload shards its graphs over the ranks instead.  ``--impl reference`` times the FP64 CPU
oracle (Algorithm 2 as written, 1 thread) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

# Hardware work queues of this process's CUDA context (read when the context is created): the batched
# workload keeps up to 64 streams busy at once, which the default of 8 queues would partly serialise.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to k eigenpairs at resid 1e-8 (mixed vs FP64); SpMV GB/s vs HBM peak"
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 512 << 20
EIG_RTOL_TARGET = 1e-10      # eigenvalue relative error aimed at (10x below the 1e-9 bar)
RESID_REL = 1e-8             # relative residual bar of the metric
CLUSTER_REL = 1e-6           # Ritz values closer than this (relative) count as one eigenvalue


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="grid128^3")
    p.add_argument("--k", type=int, default=0, help="eigenpairs (0: the workload's k)")
    p.add_argument("--eps", type=float, default=0.0,
                   help="absolute tolerance of the lock test (0: the workload's rule)")
    p.add_argument("--cmp-steps", type=int, default=2,
                   help="timed solves of the other precision (plus one untimed)")
    p.add_argument("--e2e-steps", type=int, default=3, help="timed end-to-end runs (plus one untimed)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--single-solve", choices=["fp64", "mixed"], default=None,
                   help="create one solver and run one solve, nothing else (for profiler captures)")
    p.add_argument("--opt", action="append", default=[],
                   help="solver option key=value applied to every solver (e.g. reorder=1)")
    p.add_argument("--graph-cache", default=None,
                   help="directory to keep the generated graph in (.npz), reused by later runs")
    p.add_argument("--batch-threads", type=int, default=0,
                   help="host threads of the batched solve (0: the library default, min(G, 64))")
    return p.parse_args(argv)


def solver_opts(args):
    out = {}
    for kv in args.opt:
        k, v = kv.split("=", 1)
        out[k] = float(v) if "." in v or "e" in v else int(v)
    return out


# the configurations: k, the precision of the headline value, the tolerance rule, the reference
WORKLOADS = {
    "grid128^3": dict(k=20, prec="mixed", tol="accuracy", ref="grid3d:128,128,128", desc="3-D 7-point grid 128^3"),
    "rmat20": dict(k=10, prec="fp64", tol="accuracy", ref="golden:rmat20_tight.json",
                   desc="R-MAT scale 20, edge factor 16, a,b,c,d=.57/.19/.19/.05, seed 1, symmetrised LCC"),
    "grid100x100": dict(k=5, prec="fp64", tol="abs:1e-10", ref="grid2d:100,100", desc="2-D 5-point grid 100 x 100"),
    "rgg4M": dict(k=20, prec="mixed", tol="accuracy", ref=None,
                  desc="random geometric graph, unit square, n = 4e6, r = sqrt(12/(pi n)), seed 1, LCC "
                       "(GPU cell-list generator)"),
    "rmat24": dict(k=10, prec="mixed", tol="accuracy", ref=None,
                   desc="R-MAT scale 24, edge factor 16, same a,b,c,d, seed 1, symmetrised LCC (GPU generator)"),
    "batch256": dict(k=8, prec="mixed", tol="rel:1e-8", ref=None,
                     desc="256 graphs, n log-uniform in [1e3, 2e5]: ER mean degree 8 / 2-D grid / WS k=10 p=0.1"),
}


def load_workload(args):
    import numpy as np
    import synthgraphs as sg
    if args.workload == "rmat24":
        rp, ci = sg.rmat_gpu(24)
        return sg.Graph(rp.cpu().numpy(), ci.cpu().numpy(), "rmat24")
    if args.workload == "rgg4M":
        rp, ci = sg.rgg_gpu(4_000_000, 12.0, seed=1)
        return sg.Graph(rp.cpu().numpy(), ci.cpu().numpy(), "rgg4M")
    if args.graph_cache:
        path = os.path.join(args.graph_cache, f"{args.workload}.npz")
        if os.path.exists(path):
            z = np.load(path)
            return sg.Graph(z["row_ptr"], z["col_idx"], args.workload)
        g = sg.workload(args.workload)
        os.makedirs(args.graph_cache, exist_ok=True)
        np.savez(path, row_ptr=g.row_ptr, col_idx=g.col_idx)
        return g
    return sg.workload(args.workload)


def max_over_ranks(x, dist=None, device=None):
    """Max of a per-rank scalar over all ranks (replicas: each rank solved its own copy)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_of(costs, world, rank):
    """Indices of the independent problems rank `rank` solves: greedy longest-first assignment of
    the costs to the least-loaded rank (ties: lowest rank), the same on every rank."""
    load = [0.0] * world
    mine = []
    for i in sorted(range(len(costs)), key=lambda j: (-costs[j], j)):
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += costs[i]
        if r == rank:
            mine.append(i)
    return sorted(mine)


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# --------------------------------------------------------------------------------------------- tolerance

def accuracy_eps(eig_est, norm_L, eig_rtol=EIG_RTOL_TARGET, resid_rel=RESID_REL, cluster_rel=CLUSTER_REL):
    """Absolute lock tolerance meeting both accuracy bars: min(resid_rel * ||L||,
    sqrt(eig_rtol * lambda_j * gap_j)) over the estimated eigenvalues, where gap_j is the distance
    to the nearest other estimate that differs by more than cluster_rel * lambda_j (closer ones
    are taken as copies of one multiple eigenvalue, whose eigenvectors may mix freely)."""
    lam = sorted(float(x) for x in eig_est)
    eps = resid_rel * norm_L
    for j, l in enumerate(lam):
        gaps = [abs(m - l) for i, m in enumerate(lam) if i != j and abs(m - l) > cluster_rel * abs(l)]
        if gaps and l > 0:
            eps = min(eps, math.sqrt(eig_rtol * l * min(gaps)))
    return eps


def fixed_eps(rule, norm_L):
    """Tolerance of a rule that needs no estimates ("abs:x", "rel:x"), else None."""
    if rule.startswith("abs:"):
        return float(rule[4:])
    if rule.startswith("rel:"):
        return float(rule[4:]) * norm_L
    return None


# --------------------------------------------------------------------------------------------- references

def reference_eigs(ref, k):
    """Exact or oracle eigenvalues the results are compared with: closed forms for grids (the
    Laplacian of a Cartesian product is the Kronecker sum of path Laplacians, whose spectrum is
    2 - 2 cos(pi i / N)), or the FP64 oracle's stored values (tests/golden).  None if unknown."""
    import numpy as np
    if ref is None:
        return None, None
    kind, arg = ref.split(":", 1)
    if kind in ("grid2d", "grid3d"):
        dims = [int(x) for x in arg.split(",")]
        out = np.zeros(1)
        for N in dims:
            out = (out[:, None] + (2.0 - 2.0 * np.cos(np.pi * np.arange(N) / N))[None, :]).ravel()
        return np.sort(out)[1:k + 1], "closed form (Kronecker sum of path spectra)"
    if kind == "golden":
        path = os.path.join(ROOT, "tests", "golden", arg)
        if not os.path.exists(path):
            return None, None
        g = json.load(open(path))
        lam = np.sort(np.array(g["eigvals"]))
        if lam.shape[0] < k:
            return None, None
        return lam[:k], f"FP64 oracle, eps_rel {g['eps_rel']:g} (tests/golden/{arg})"
    return None, None


def rel_eig_err(lam, ref):
    import numpy as np
    lam = np.sort(np.asarray(lam, dtype=np.float64))
    return float(np.max(np.abs(lam - ref) / np.abs(ref)))


def workload_config(name, g, k, eps, norm_L):
    spec = WORKLOADS[name]
    return {"workload": f"{name} k={k} {spec['prec']}", "graph": spec["desc"], "n": g.n, "nnz": g.nnz, "k": k,
            "eps_abs": eps, "resid_rel_bound": eps / norm_L, "norm_L": "2*max_degree", "norm_L_value": norm_L,
            "tol_rule": spec["tol"], "l2": "flushed (512 MB write) between steps",
            "start_vector": "splitmix64 seed 1, centred, unit norm"}


def config_with_opts(cfg, args):
    if args.opt:
        cfg = dict(cfg)
        cfg["solver_opts"] = solver_opts(args)
    return cfg


# --------------------------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region, for the device in use."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and self.uuid not in parts[0]:
                continue
            rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_median": statistics.median([float(r[3]) for r in rows if _isnum(r[3])]) if rows else None}


def _isnum(s):
    try:
        float(s)
        return True
    except ValueError:
        return False


# --------------------------------------------------------------------------------------------- roofline

def kernel_bytes(kind, n, Z, c, word, n_long=None, n_slices=None, ml=None):
    """Algorithmic DRAM bytes of one launch of an inner-iteration kernel (word = 4 FP32, 8 FP64):
      gather  : column indices 4Z, the gathered vector once (w n), the row sums (w n), and the row
                structure: row_ptr 8(n+1) for CSR rows, or with the sliced light rows 8(n_long+1)
                for the long rows plus 8(n_slices+1) slice offsets;
      rows    : degrees 4n; reads of the row sums, z_k, z_{k-1}, two w buffers and x (6 w n), the
                c columns of Vh (c w n); writes of Y, the new w and x (3 w n); FP64 adds the
                reciprocal preconditioner diagonal (8 n);
      phase2  : degrees 4n; reads of Y, z_k (2 w n) and Vh (c w n); write of z_{k+1} (w n); FP64
                adds 8 n.
    c is the launch's deflation rank (averaged over the timed launches)."""
    extra = 8 * n if word == 8 else 0
    if kind == "rows_ml":      # k_ml_phase1: degrees 4n, 7 vectors read (row sums, z_k, z_{k-1}, r_{k-1},
        return 4 * n + 10 * word * n   # two w buffers, x), 3 written; Vh^T z_k comes from phase 2c
    if kind == "phase2_ml":
        # one application of the projected multilevel preconditioner with MINRES phase 2:
        #   ml_phase2a (4 + c) w n, ml_project (4 + c) w n, ml_phase2c (2 + c) w n;
        #   V-cycle level 0: two gathers, restriction (2 w n + 4 n), prolongation (3 w n + 4 n);
        #   ml_phase2b with level 0's post-smoothing: b, 1/D, x1, W x1, r_{k+1}, Vh read, w written
        #   (6 + c) w n; levels below: per level two CSR sweeps 2 (4 + w) nnz_l and (16 + 5 w) n_l of
        #   vectors, cluster maps and member lists
        n_c, nnz_c = ml
        struct = 8 * (n + 1) if not n_slices else 8 * (n_long + 1) + 8 * (n_slices + 1)
        return ((25 + 4 * c) * word * n + 8 * n + 2 * (struct + 4 * Z)
                + 2 * (4 + word) * nnz_c + (16 + 5 * word) * n_c)
    if kind == "gather":
        struct = 8 * (n + 1) if not n_slices else 8 * (n_long + 1) + 8 * (n_slices + 1)
        return struct + 4 * Z + 2 * word * n
    if kind == "rows":
        return 4 * n + (9 + c) * word * n + extra
    if kind == "phase2":
        return 4 * n + (3 + c) * word * n + extra
    raise KeyError(kind)


KERNEL_NAMES = {"gather": "k_phase1_gather (trimmed-operator SpMV gather)",
                "rows": "k_phase1 (operator row epilogue + MINRES update)",
                "phase2": "k_phase2 (SMW preconditioner + MINRES reductions)"}
KERNEL_NAMES_ML = {"gather": "k_phase1_gather (trimmed-operator SpMV gather)",
                   "rows": "k_ml_phase1 (operator row epilogue + MINRES update)",
                   "phase2": "multilevel phase 2 (13 launches on the 128^3 grid in FP32): ml_phase2a, ml_project, "
                             "one V-cycle (two level-0 gathers, restriction, prolongation, fused coarse-level "
                             "sweeps), ml_phase2b with the level-0 post-smoothing, ml_phase2c"}
STAT_OF = {"gather": "inner_phase1_ms", "rows": "inner_rows_ms", "phase2": "inner_phase2_ms"}

GATHER_SOURCES = ["paper_1710_07080_gb300/csrc/common.cuh", "paper_1710_07080_gb300/csrc/inner_impl.cuh"]


def source_hash(files=GATHER_SOURCES):
    """Hash of the sources that define the inner kernels: a stored ncu traffic figure applies only
    while they are unchanged."""
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key):
    """Per-launch DRAM bytes of a kernel from the committed ncu summary, if it was taken on the
    current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    cur = source_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and parts[0] == kernel_key and parts[1] == cur:
            return float(parts[2])
    return None


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            pk = json.load(open(path))
            for key in ("hbm_gbs_sustained", "hbm_gbs"):
                if key in pk and pk[key]:
                    return float(pk[key]), f"measured ({key})"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


def kernel_rooflines(st, n, Z, word, workload, prec_tag):
    """Per-kernel achieved GB/s from one profiled solve's CUDA-event totals, and the dominant one."""
    peak, peak_src = hbm_peak()
    nl = st["inner_phase1_timed"]
    c_avg = st["inner_phase1_csum"] / max(1, nl)
    n_slices = (n - st["n_long_rows"] + 31) // 32 if st.get("sell_entries") else None
    ml = st.get("precond") == 1
    names = KERNEL_NAMES_ML if ml else KERNEL_NAMES
    out = {}
    for kind in ("gather", "rows", "phase2"):
        ms = st[STAT_OF[kind]]
        avg_s = ms / 1e3 / max(1, nl)
        bkind = kind + "_ml" if ml and kind != "gather" else kind
        b = kernel_bytes(bkind, n, Z, c_avg, word, st["n_long_rows"], n_slices,
                         (st.get("ml_coarse_n", 0), st.get("ml_coarse_nnz", 0)))
        ach = b / avg_s / 1e9 if avg_s > 0 else None
        out[kind] = {"kernel": names[kind], "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                     "frac": ach / peak if ach else None, "bytes_per_launch": b, "avg_us": avg_s * 1e6,
                     "launches_timed": nl, "total_ms": ms, "avg_deflation_rank": c_avg,
                     "traffic": ncu_traffic(f"{bkind}_{prec_tag}_{workload}")}
    dom = max(out, key=lambda q: out[q]["total_ms"])
    tot = sum(v["total_ms"] for v in out.values())
    for v in out.values():
        v["share_of_inner_kernels"] = v["total_ms"] / tot if tot > 0 else None
    return out, dom, peak_src


# --------------------------------------------------------------------------------------------- oracle leg

def oracle_counts(workload):
    """Unit counts of the FP64 oracle's own full run at the accuracy tolerance (tests/golden,
    written by tests/golden/make_golden.py, which calls only oracle/)."""
    name = {"grid128^3": "grid128_accuracy.json", "rmat20": "rmat20_accuracy.json"}.get(workload)
    if name is None:
        return None, None
    path = os.path.join(ROOT, "tests", "golden", name)
    if not os.path.exists(path):
        return None, None
    g = json.load(open(path))
    return g["oracle_stats"], {"file": f"tests/golden/{name}", "eps_abs": g.get("eps_abs"),
                               "oracle_seconds_on_build_host": g.get("oracle_seconds")}


SAMPLE_CAPS = {"grid128^3": (2, 100), "rmat20": (3, 5000), "grid100x100": (100000, 20000),
               "rgg4M": (1, 60), "rmat24": (1, 20)}


# inner iterations of the oracle timed at the workload's average deflation rank
INNER_RATE_ITERS = {"grid128^3": 24, "rmat20": 60, "grid100x100": 400, "rgg4M": 20, "rmat24": 8}


def oracle_inner_rate(g, c, iters):
    """Seconds per inner MINRES iteration of the oracle (trimmed operator, preconditioner, MINRES
    update) with a deflation basis of c orthonormal columns: the capped run below only reaches the
    first eigenpair (c = 0), while the cost of an iteration grows with c."""
    import numpy as np

    import oracle
    rng = np.random.default_rng(7)
    V = np.linalg.qr(rng.standard_normal((g.n, c)))[0] if c > 0 else None
    r = rng.standard_normal(g.n)
    r -= r.mean()
    trim = int(np.argmax(g.degrees))
    t0 = time.perf_counter()
    _, it, _ = oracle.inner_solve(g.row_ptr, g.col_idx, trim, 0.0, 2.0 * float(g.degrees.max()), V, r,
                                  tau=1e-300, max_it=iters)
    return (time.perf_counter() - t0) / max(1, it), it


def oracle_sample(g, k, eps, u0, workload, c_avg):
    """Runs the oracle on the workload with outer steps and inner iterations capped (a bounded
    sample), then times inner iterations at deflation rank round(c_avg); returns the wall seconds
    and the stats (per-phase seconds and unit counts, plus the per-iteration rate at that rank)."""
    import oracle
    max_outer, max_inner = SAMPLE_CAPS.get(workload, (2, 100))
    t0 = time.perf_counter()
    _, _, st = oracle.isira(g.row_ptr, g.col_idx, k, u0, eps=eps, tau_inner=1e-3, max_outer=max_outer,
                            max_inner=max_inner)
    c = int(round(c_avg))
    st["rate_c"] = c
    st["rate_sec_per_it"], st["rate_iters"] = oracle_inner_rate(g, c, INNER_RATE_ITERS.get(workload, 50))
    return time.perf_counter() - t0, st


def project(st_sample, counts):
    """Seconds of a full run from the sample's per-unit costs: seconds per recomputed W column (the
    W_k, H_k step of Algorithm 2), per inner MINRES iteration (its inner solve, at the average
    deflation rank) and per outer step (the rest), times the full run's counts of those units."""
    per_col = st_sample["sec_w"] / max(1, st_sample["w_columns"])
    per_it = st_sample.get("rate_sec_per_it") or st_sample["sec_inner"] / max(1, st_sample["inner_iters"])
    rest = st_sample["sec_total"] - st_sample["sec_w"] - st_sample["sec_inner"]
    per_step = rest / max(1, st_sample["outer_steps"])
    return per_col * counts["w_columns"] + per_it * counts["inner_iters"] + per_step * counts["outer_steps"]


def host_cpu():
    model = platform.processor() or platform.machine()
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "model": model, "machine": platform.machine()}


def sample_text(st, counts, src):
    return (f"Algorithm 2 by the FP64 oracle (tau_inner 1e-3, 1 thread) on the same graph at the same eps, "
            f"capped at {st['outer_steps']} outer steps and {st['inner_iters']} inner iterations (measured "
            f"{st['sec_total']:.1f} s: {st['sec_inner'] / max(1, st['inner_iters']) * 1e3:.2f} ms per inner "
            f"iteration at deflation rank 0, {st['sec_w'] / max(1, st['w_columns']) * 1e3:.2f} ms per recomputed "
            f"W column), then {st['rate_iters']} oracle inner iterations at deflation rank {st['rate_c']} (the "
            f"solve's average; {st['rate_sec_per_it'] * 1e3:.2f} ms each); scaled to "
            f"one full solve with the unit counts {counts['inner_iters']} inner iterations, {counts['w_columns']} W "
            f"columns, {counts['outer_steps']} outer steps ({src})")


def run_reference(args):
    import synthgraphs as sg
    rank, world, _ = env_rank()
    if rank != 0:
        return
    spec = WORKLOADS.get(args.workload)
    if spec is None or args.workload == "batch256":
        print(json.dumps({"impl": "reference", "unavailable": f"no oracle leg for workload {args.workload}"}))
        return
    counts, src = oracle_counts(args.workload)
    if counts is None:
        print(json.dumps({"impl": "reference",
                          "unavailable": f"no stored oracle unit counts for {args.workload} (tests/golden)"}))
        return
    k = args.k if args.k > 0 else spec["k"]
    g = load_workload(args)
    norm_L = 2.0 * float(g.degrees.max())
    eps = args.eps if args.eps > 0 else (src["eps_abs"] or fixed_eps(spec["tol"], norm_L))
    u0 = sg.start_vector(g.n, 1)
    values, walls, st = [], [], None
    t_all = time.perf_counter()
    for i in range(args.warmup + args.steps):
        # average deflation rank over the inner iterations, taken as (k - 1) / 2 (no GPU run here)
        dt, st = oracle_sample(g, k, eps, u0, args.workload, (k - 1) / 2.0)
        if i >= args.warmup:
            values.append(project(st, counts))
            walls.append(dt)
    value = statistics.mean(values)
    cpu = host_cpu()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(walls) * 1e3,
            "ms_per_step_is": "measured wall time of one bounded oracle sample (the timed region is steps x this); "
                              "value is that sample scaled to one full solve",
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.workload, g, k, eps, norm_L),
            "cpu_baseline": {"value": value, "unit": "s", "cores": 1, "kind": "oracle",
                             "sample": sample_text(st, counts, src["file"]), "host": cpu},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s_total": time.perf_counter() - t_all}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------------- batch

def run_batch(args):
    """256 graphs of uneven size solved together through isira_batch_* (one step = the whole batch)."""
    import torch

    import paper_1710_07080_gb300 as isira
    import synthgraphs as sg
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    spec = WORKLOADS["batch256"]
    k = args.k if args.k > 0 else spec["k"]
    rel = float(spec["tol"][4:])
    import torch.distributed as tdist
    dist = tdist if (world > 1 and tdist.is_initialized()) else None
    all_graphs = sg.batch_family(256, 1000, 200000, seed=1)
    # the graphs are independent problems: each rank solves its share (no data-path collective)
    mine = shard_of([g.nnz + 10 * g.n for g in all_graphs], world, rank)
    graphs = [all_graphs[i] for i in mine]
    dg = [(torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col_idx).to(dev)) for g in graphs]
    b = isira.Batch(dg, precision=isira.ISIRA_MIXED, **solver_opts(args))
    times = []
    for i in range(args.warmup + args.steps):
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = b.solve(k, rel_tol=rel, n_threads=args.batch_threads)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    per = [b.stats(g) for g in range(len(graphs))]
    iters = [p["inner_iters"] for p in per]
    solve_s = [p["solve_ms"] / 1e3 for p in per]
    res = [float(b.eigpairs(g)[2].max()) for g in range(len(graphs))]
    crit = max(range(len(graphs)), key=lambda q: solve_s[q])
    # per family (graph index mod 3: ER / 2-D grid / WS): how much sequential work each carries
    fams = {}
    for q, p in enumerate(per):
        f = ("er", "grid2d", "ws")[mine[q] % 3]
        a = fams.setdefault(f, {"graphs": 0, "sum_n": 0, "inner_iters": 0, "outer_steps": 0, "multilevel": 0,
                                "max_inner_iters": 0})
        a["graphs"] += 1
        a["sum_n"] += graphs[q].n
        a["inner_iters"] += p["inner_iters"]
        a["outer_steps"] += p["outer_steps"]
        a["multilevel"] += 1 if p["precond"] == 1 else 0
        a["max_inner_iters"] = max(a["max_inner_iters"], p["inner_iters"])
    # the graph with the most inner iterations, solved alone afterwards (not in the timed region):
    # the batch cannot finish before this chain of dependent iterations does
    longest = max(range(len(graphs)), key=lambda q: iters[q])
    alone = None
    if rank == 0:
        rp_l, ci_l = dg[longest]
        with isira.Solver(rp_l, ci_l, precision=isira.ISIRA_MIXED, **solver_opts(args)) as s1:
            tol_l = rel * s1.stats()["norm_L"]
            s1.solve(k, tol=tol_l)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s1.solve(k, tol=tol_l)
            torch.cuda.synchronize()
            alone = {"index": mine[longest], "n": graphs[longest].n, "inner_iters": s1.stats()["inner_iters"],
                     "precond": s1.stats()["precond"], "solve_alone_s": time.perf_counter() - t0}
    value = max_over_ranks(statistics.mean(times), dist, dev)
    max_res = max_over_ranks(max(res), dist, dev)
    iters_max = max_over_ranks(float(max(iters)), dist, dev)
    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
            "scaling": "strong" if world > 1 else "weak",
            "vs_baseline": None, "dtype": "f32 inner / f64 outer", "data": "synthetic",
            "config": {"workload": f"batch256 k={k} mixed", "graph": spec["desc"], "graphs": len(graphs),
                       "sum_n": int(sum(g.n for g in graphs)), "sum_nnz": int(sum(g.nnz for g in graphs)),
                       "resid_rel": rel, "host_threads": args.batch_threads or min(len(graphs), 64)},
            "batch": {"status": st, "max_true_resid_rel": max_res, "inner_iters_max": int(iters_max),
                      "graphs_on_rank0": len(graphs), "sharding": "greedy by nnz + 10 n, no collective",
                      # the batch can finish no sooner than its slowest graph's own solve (a chain of
                      # dependent inner iterations): wall time against that bound and against the sum
                      "critical_graph": {"index": mine[crit], "n": graphs[crit].n, "nnz": graphs[crit].nnz,
                                         "solve_s": solve_s[crit], "inner_iters": iters[crit]},
                      "sum_of_graph_solves_s": sum(solve_s),
                      "families": fams, "longest_chain_alone": alone,
                      "wall_over_critical": (statistics.mean(times) / solve_s[crit]) if solve_s[crit] > 0 else None}}
    b.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------------- our arm

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch

    import paper_1710_07080_gb300 as isira
    import synthgraphs as sg

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    def reduce_max(x):
        return max_over_ranks(x, dist, dev)

    if args.workload == "batch256":
        run_batch(args)
        if dist is not None:
            dist.destroy_process_group()
        return
    stages = {}
    t_stage = time.perf_counter()
    spec = WORKLOADS[args.workload]
    g = load_workload(args)
    stages["graph_build_s"] = time.perf_counter() - t_stage
    n, Z = g.n, g.nnz
    k = args.k if args.k > 0 else spec["k"]
    norm_L = 2.0 * float(g.degrees.max())
    head = spec["prec"]
    other = "fp64" if head == "mixed" else "mixed"
    P = {"fp64": isira.ISIRA_FP64, "mixed": isira.ISIRA_MIXED}
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    ci_h = torch.from_numpy(g.col_idx).pin_memory()
    u0_h = torch.from_numpy(sg.start_vector(n, 1)).pin_memory()
    rp = rp_h.to(dev)
    ci = ci_h.to(dev)
    u0 = u0_h.to(dev)
    if args.single_solve:
        eps = args.eps if args.eps > 0 else (fixed_eps(spec["tol"], norm_L) or RESID_REL * norm_L)
        with isira.Solver(rp, ci, precision=P[args.single_solve], **solver_opts(args)) as s:
            s.solve(k, tol=eps, u0=u0)
            torch.cuda.synchronize()
            print(json.dumps({"single_solve": args.single_solve, "eps": eps, **s.stats()}), flush=True)
        return
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    props = torch.cuda.get_device_properties(dev)
    uuid = str(props.uuid) if hasattr(props, "uuid") else ""

    t_stage = time.perf_counter()
    solvers = {p: isira.Solver(rp, ci, precision=P[p], **solver_opts(args)) for p in (head, other)}
    torch.cuda.synchronize()
    stages["create_both_s"] = time.perf_counter() - t_stage

    # tolerance (untimed): the workload's fixed rule, or the accuracy rule from one loose solve's Ritz values
    t_stage = time.perf_counter()
    eps = args.eps if args.eps > 0 else fixed_eps(spec["tol"], norm_L)
    calib = None
    if eps is None:
        solvers[head].solve(k, tol=RESID_REL * norm_L, u0=u0)
        lam_loose = solvers[head].eigpairs(want_vectors=False, want_resid=False)[0].numpy()
        eps = accuracy_eps(lam_loose, norm_L)
        calib = {"loose_eps_abs": RESID_REL * norm_L, "loose_eigvals": [float(x) for x in lam_loose],
                 "rule": "min(1e-8 ||L||, sqrt(1e-10 lambda_j gap_j)), clusters merged at 1e-6 relative"}
    stages["calibration_s"] = time.perf_counter() - t_stage

    def timed(solver, warm, steps, profile=False):
        for _ in range(warm):
            solver.solve(k, tol=eps, u0=u0)
        torch.cuda.synchronize()
        solver.set_profiling(profile)
        times, stats = [], []
        for _ in range(steps):
            flush.zero_()
            barrier()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solver.solve(k, tol=eps, u0=u0)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            times.append(e0.elapsed_time(e1) / 1e3)
            stats.append(solver.stats())
        solver.set_profiling(False)
        return times, stats

    clk = ClockSampler(uuid.replace("GPU-", "") if uuid else "")
    clk.start()
    t_stage = time.perf_counter()
    t_head, st_head = timed(solvers[head], args.warmup, args.steps)
    stages["timed_headline_s"] = time.perf_counter() - t_stage
    clocks = clk.stop()
    t_stage = time.perf_counter()
    t_oth, st_oth = timed(solvers[other], 1, max(1, min(args.steps, args.cmp_steps)))
    stages["timed_other_precision_s"] = time.perf_counter() - t_stage
    # kernel timing: one solve per precision with CUDA events around every inner launch (chunked launches)
    t_stage = time.perf_counter()
    prof = {p: timed(solvers[p], 0, 1, profile=True) for p in (head, other)}
    stages["profiled_solves_s"] = time.perf_counter() - t_stage

    # accuracy of the benchmarked solves against the closed form or the FP64 oracle (untimed)
    ref, ref_src = reference_eigs(spec["ref"], k)
    acc = {"reference": ref_src}
    for p in (head, other):
        lam, vec, res = solvers[p].eigpairs()
        acc[f"max_true_resid_rel_{p}"] = float(res.max())
        acc[f"n_locked_{p}"] = int(lam.numel())
        if ref is not None and lam.numel() == k:
            acc[f"max_rel_eig_err_{p}"] = rel_eig_err(lam.numpy(), ref)
        acc[f"eigvals_{p}"] = [float(x) for x in lam]
    acc["bars"] = {"max_rel_eig_err": 1e-9, "max_true_resid_rel": RESID_REL}

    # end to end through the public API, in the headline precision:
    # pinned host CSR -> device, create (with autotuning), solve, eigenpairs -> host
    t_stage = time.perf_counter()
    e2e_times = []
    h2d = rp_h.numel() * 8 + ci_h.numel() * 4 + u0_h.numel() * 8
    d2h = n * k * 8 + k * 8 * 2
    e2e_n = max(1, min(args.steps, args.e2e_steps))
    for i in range(1 + e2e_n):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rp_d = rp_h.to(dev, non_blocking=True)
        ci_d = ci_h.to(dev, non_blocking=True)
        u0_d = u0_h.to(dev, non_blocking=True)
        with isira.Solver(rp_d, ci_d, precision=P[head], **solver_opts(args)) as s:
            s.solve(k, tol=eps, u0=u0_d)
            lam_e, vec_e, res_e = s.eigpairs()
            vec_host = vec_e.cpu()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if i >= 1:
            e2e_times.append(dt)
    del vec_host
    stages["e2e_s"] = time.perf_counter() - t_stage

    value = reduce_max(statistics.mean(t_head))
    value_oth = reduce_max(statistics.mean(t_oth))
    e2e = reduce_max(statistics.mean(e2e_times))
    word = {"fp64": 8, "mixed": 4}
    kern = {}
    for p in (head, other):
        kern[p] = kernel_rooflines(prof[p][1][0], n, Z, word[p], args.workload, "f32" if p == "mixed" else "f64")
    rk, dom, peak_src = kern[head]
    roof = dict(rk[dom])
    roof.update(peak_source=peak_src, dominant_of="inner-iteration kernels (gather, rows, phase2), by total time",
                other_kernels={q: {kk: v[kk] for kk in ("kernel", "achieved", "frac", "avg_us", "share_of_inner_kernels")}
                               for q, v in rk.items() if q != dom})
    ro, dom_o, _ = kern[other]

    def summary(p, times, stats):
        s = stats[-1]
        return {"value": statistics.mean(times), "unit": "s", "steps": len(times),
                "dtype": "f64" if p == "fp64" else "f32 inner / f64 outer", "outer_steps": s["outer_steps"],
                "inner_iters": s["inner_iters"], "inner_solves": s["inner_solves"], "restarts": s["restarts"],
                "w_columns": s["w_columns"], "spmv_lanes": s["spmv_lanes"], "gather_block": s["gather_block"],
                "hub_bytes": s["hub_bytes"], "sell_entries": s["sell_entries"], "n_long_rows": s["n_long_rows"],
                "profiled_solve_s": prof[p][0][0]}

    line = {
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if head == "fp64" else "f32 inner / f64 outer", "data": "synthetic",
        "config": config_with_opts(workload_config(args.workload, g, k, eps, norm_L), args),
        head: summary(head, t_head, st_head),
        other: {**summary(other, t_oth, st_oth), "roofline": {**ro[dom_o], "dominant": dom_o}},
        "mixed_speedup_vs_fp64": (value_oth / value) if head == "mixed" else (value / value_oth),
        "accuracy": acc,
        "roofline": roof,
        "kernels": {p: {q: {kk: v[kk] for kk in ("achieved", "frac", "avg_us", "bytes_per_launch", "total_ms",
                                                  "share_of_inner_kernels")} for q, v in kern[p][0].items()}
                    for p in (head, other)},
        "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": e2e_n,
                "path": "pinned host CSR -> isira_create (autotune) -> isira_solve -> isira_eigpairs -> host"},
        "gpu_launches": int(sum(s["kernel_launches"] for s in st_head)),
        "clocks": clocks,
        "stages": stages,
    }
    if calib is not None:
        line["config"]["calibration"] = calib
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload in SAMPLE_CAPS:
        t_stage = time.perf_counter()
        counts, src = oracle_counts(args.workload)
        if counts is None:
            s64 = st_head[-1] if head == "fp64" else st_oth[-1]
            counts = {"inner_iters": s64["inner_iters"], "w_columns": s64["w_columns"],
                      "outer_steps": s64["outer_steps"]}
            src = {"file": "unit counts of the GPU FP64 solve of this run (same algorithm, same eps)"}
        c_avg = line.get("roofline", {}).get("avg_deflation_rank") or (k - 1) / 2.0
        dt, st = oracle_sample(g, k, eps, u0_h.numpy(), args.workload, c_avg)
        line["cpu_baseline"] = {"value": project(st, counts), "unit": "s", "cores": 1, "kind": "oracle",
                                "sample": sample_text(st, counts, src["file"]), "sample_seconds": dt,
                                "host": host_cpu()}
        stages["cpu_baseline_s"] = time.perf_counter() - t_stage
    if rank == 0:
        print(json.dumps(line), flush=True)
    for s in solvers.values():
        s.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
