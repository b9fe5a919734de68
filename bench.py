#!/usr/bin/env python3
"""Benchmark: time to the k smallest positive Laplacian eigenpairs with iSIRA on one GB300.

Workload (default): R-MAT scale 20 (edge factor 16, a,b,c,d = .57/.19/.19/.05, seed 1),
symmetrised, deduplicated, loop-free, largest connected component; k = 10; convergence at
relative residual ||L x - lambda x|| / ||L|| <= 1e-8 with ||L|| := 2 * max degree.  The
headline value is the plain-FP64 solve; the mixed solve (FP32 inner, FP64 outer) is timed on
the same graph and reported beside it.

A step is one full isira_solve (all of Algorithm 2: inner solves, orthogonalisation,
Rayleigh-Ritz, restarts, locking).  Inputs are resident in HBM; the L2 is flushed (a 512 MB
write) between timed steps; each step is timed with CUDA events on the library's stream.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

With N > 1 (torchrun) every rank solves its own copy of the workload (replicas: the method
has no data-parallel split of one graph) and rank 0 prints the max over ranks.
``--impl reference`` times the FP64 CPU oracle (Algorithm 2 as written, 1 thread) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to k eigenpairs at resid 1e-8 (mixed vs FP64); SpMV GB/s vs HBM peak"
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 512 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="rmat20")
    p.add_argument("--k", type=int, default=0, help="eigenpairs (0: the workload's k)")
    p.add_argument("--rel-tol", type=float, default=0.0, help="relative residual (0: the workload's)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--single-solve", choices=["fp64", "mixed"], default=None,
                   help="create one solver and run one solve, nothing else (for profiler captures)")
    p.add_argument("--opt", action="append", default=[],
                   help="solver option key=value applied to every solver (e.g. reorder=1)")
    p.add_argument("--graph-cache", default=None,
                   help="directory to keep the generated graph in (.npz), reused by later runs")
    return p.parse_args()


def solver_opts(args):
    out = {}
    for kv in args.opt:
        k, v = kv.split("=", 1)
        out[k] = float(v) if "." in v or "e" in v else int(v)
    return out


def load_workload(args):
    import numpy as np
    import synthgraphs as sg
    if args.workload == "rmat24":
        rp, ci = sg.rmat_gpu(24)
        return sg.Graph(rp.cpu().numpy(), ci.cpu().numpy(), "rmat24")
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


# the five configurations: k, the precision of the headline value, tolerance
WORKLOADS = {
    "rmat20": dict(k=10, prec="fp64", tol=("rel", 1e-8),
                   desc="R-MAT scale 20, edge factor 16, a,b,c,d=.57/.19/.19/.05, seed 1, symmetrised LCC"),
    "grid100x100": dict(k=5, prec="fp64", tol=("abs", 1e-10), desc="2-D 5-point grid 100 x 100"),
    "grid128^3": dict(k=20, prec="mixed", tol=("rel", 1e-8), desc="3-D 7-point grid 128^3"),
    "rgg4M": dict(k=20, prec="mixed", tol=("rel", 1e-8),
                  desc="random geometric graph, unit square, n = 4e6, r = sqrt(12/(pi n)), seed 1, LCC"),
    "rmat24": dict(k=10, prec="mixed", tol=("rel", 1e-8),
                   desc="R-MAT scale 24, edge factor 16, same a,b,c,d, seed 1, symmetrised LCC (GPU generator)"),
    "batch256": dict(k=8, prec="mixed", tol=("rel", 1e-8),
                     desc="256 graphs, n log-uniform in [1e3, 2e5]: ER mean degree 8 / 2-D grid / WS k=10 p=0.1"),
}


def workload_config(name, g, k, rel_tol):
    spec = WORKLOADS[name]
    kind, t = spec["tol"]
    return {"workload": f"{name} k={k} {spec['prec']}", "graph": spec["desc"], "n": g.n, "nnz": g.nnz,
            "k": k, ("resid_rel" if kind == "rel" else "tol_abs"): t, "norm_L": "2*max_degree",
            "l2": "flushed (512 MB write) between steps", "start_vector": "splitmix64 seed 1, centred, unit norm"}


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

def phase1_bytes(n, Z, c_avg, word):
    """Algorithmic DRAM bytes of one launch of the phase-1 gather kernel (the dominant kernel):
    row_ptr 8(n+1), col_idx 4Z, the gathered vector once (word*n) and the per-row sums written
    (word*n).  c_avg is unused: the deflation terms live in the row-epilogue kernel."""
    return 8 * (n + 1) + 4 * Z + 2 * word * n


def phase1_fp64_ops(n, Z, c_avg):
    """FP64 lane operations of one FP64 gather launch: one add per stored entry."""
    return Z


def fp64_peak_ops(sm_max_mhz):
    """FP64 lane operations per second: 152 SMs x 2 lanes per clock (the FP64 pipe issues one warp
    instruction per 16 cycles per SM on this part; 1.25 TFLOP/s nominal counts an FMA as 2) x clock."""
    mhz = sm_max_mhz or 2070.0
    return 152 * 2 * mhz * 1e6


GATHER_SOURCES = ["paper_1710_07080_gb300/csrc/common.cuh", "paper_1710_07080_gb300/csrc/inner_impl.cuh"]


def source_hash(files=GATHER_SOURCES):
    """Hash of the sources that define the gather kernel: a stored ncu traffic figure applies only
    while they are unchanged."""
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key):
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
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


# --------------------------------------------------------------------------------------------- oracle leg

def oracle_sample(g, k, tol_abs, u0, max_outer):
    import oracle
    t0 = time.perf_counter()
    lam, V, st = oracle.isira(g.row_ptr, g.col_idx, k, u0, eps=tol_abs, tau_inner=1e-3, max_outer=max_outer)
    return time.perf_counter() - t0, st


def oracle_full_counts(name):
    """Work counts of the oracle's full run on this workload (written by tests/golden/make_golden.py)."""
    path = os.path.join(ROOT, "tests", "golden", f"{name}_bench.json")
    if os.path.exists(path):
        return json.load(open(path))["oracle_stats"]
    return None


def project_oracle(st_sample, full):
    """Seconds of the oracle's full run, projected from a sample's per-unit costs: seconds per
    recomputed W column (the W_k, H_k step of Algorithm 2), per inner MINRES iteration (its inner solve) and per outer step (the
    rest), times the full run's counts of those units."""
    per_col = st_sample["sec_w"] / max(1, st_sample["w_columns"])
    per_it = st_sample["sec_inner"] / max(1, st_sample["inner_iters"])
    rest = st_sample["sec_total"] - st_sample["sec_w"] - st_sample["sec_inner"]
    per_step = rest / max(1, st_sample["outer_steps"])
    return per_col * full["w_columns"] + per_it * full["inner_iters"] + per_step * full["outer_steps"]


SAMPLE_STEPS = 6


def sample_text(st, full):
    return (f"first {st['outer_steps']} outer steps of Algorithm 2 (FP64 oracle, tau_inner 1e-3, 1 thread) on the "
            f"same graph: {st['sec_w'] / max(1, st['w_columns']) * 1e3:.1f} ms per recomputed W column, "
            f"{st['sec_inner'] / max(1, st['inner_iters']) * 1e3:.1f} ms per inner iteration; projected with the "
            f"unit counts of the oracle's full run ({full['w_columns']} W columns, {full['inner_iters']} inner "
            f"iterations, {full['outer_steps']} outer steps; tests/golden)")


def run_reference(args):
    import synthgraphs as sg
    rank, world, _ = env_rank()
    if rank != 0:
        return
    if args.workload not in ("rmat20",):
        print(json.dumps({"impl": "reference", "unavailable": "oracle work counts exist only for rmat20"}))
        return
    spec = WORKLOADS[args.workload]
    k = args.k if args.k > 0 else spec["k"]
    g = load_workload(args)
    normL = 2.0 * float(g.degrees.max())
    tol = (args.rel_tol if args.rel_tol > 0 else spec["tol"][1]) * normL
    u0 = sg.start_vector(g.n, 1)
    full = oracle_full_counts(args.workload)
    if full is None:
        print(json.dumps({"impl": "reference", "unavailable": "no oracle work counts for this workload"}))
        return
    values, st = [], None
    for i in range(args.warmup + args.steps):
        _, st = oracle_sample(g, k, tol, u0, SAMPLE_STEPS)
        if i >= args.warmup:
            values.append(project_oracle(st, full))
    value = statistics.mean(values)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.workload, g, k, tol / normL),
            "cpu_baseline": {"value": value, "unit": "s", "cores": 1, "kind": "oracle",
                             "sample": sample_text(st, full)},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------------- batch

def run_batch(args):
    """256 graphs of uneven size solved together through isira_batch_* (one step = the whole batch)."""
    import numpy as np
    import torch

    import paper_1710_07080_gb300 as isira
    import synthgraphs as sg
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    spec = WORKLOADS["batch256"]
    k = args.k if args.k > 0 else spec["k"]
    rel = args.rel_tol if args.rel_tol > 0 else spec["tol"][1]
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
        st = b.solve(k, rel_tol=rel)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    iters = [b.stats(g)["inner_iters"] for g in range(len(graphs))]
    res = [float(b.eigpairs(g)[2].max()) for g in range(len(graphs))]
    value = max_over_ranks(statistics.mean(times), dist, dev)
    max_res = max_over_ranks(max(res), dist, dev)
    iters_max = max_over_ranks(float(max(iters)), dist, dev)
    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
            "scaling": "strong" if world > 1 else "weak",
            "vs_baseline": None, "dtype": "f32 inner / f64 outer", "data": "synthetic",
            "config": {"workload": f"batch256 k={k} mixed", "graph": spec["desc"], "graphs": len(graphs),
                       "sum_n": int(sum(g.n for g in graphs)), "sum_nnz": int(sum(g.nnz for g in graphs)),
                       "resid_rel": rel},
            "batch": {"status": st, "max_true_resid_rel": max_res, "inner_iters_max": int(iters_max),
                      "graphs_on_rank0": len(graphs), "sharding": "greedy by nnz + 10 n, no collective"}}
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
    spec = WORKLOADS[args.workload]
    g = load_workload(args)
    n, Z = g.n, g.nnz
    k = args.k if args.k > 0 else spec["k"]
    normL = 2.0 * float(g.degrees.max())
    kind, tv = spec["tol"]
    tol = (args.rel_tol if args.rel_tol > 0 else tv) * normL if kind == "rel" else tv
    rel_for_cfg = tol / normL
    if args.single_solve:
        prec = isira.ISIRA_FP64 if args.single_solve == "fp64" else isira.ISIRA_MIXED
        with isira.Solver(torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col_idx).to(dev),
                          precision=prec, **solver_opts(args)) as s:
            s.solve(k, tol=tol, u0=torch.from_numpy(sg.start_vector(n, 1)).to(dev))
            torch.cuda.synchronize()
            print(json.dumps({"single_solve": args.single_solve, **s.stats()}), flush=True)
        return
    rp_h = torch.from_numpy(g.row_ptr).pin_memory()
    ci_h = torch.from_numpy(g.col_idx).pin_memory()
    u0_h = torch.from_numpy(sg.start_vector(n, 1)).pin_memory()
    rp = rp_h.to(dev)
    ci = ci_h.to(dev)
    u0 = u0_h.to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    uuid = str(torch.cuda.get_device_properties(dev).uuid) if hasattr(torch.cuda.get_device_properties(dev), "uuid") else ""

    def timed_solves(solver, profile):
        for _ in range(args.warmup):
            solver.solve(k, tol=tol, u0=u0)
        torch.cuda.synchronize()
        solver.set_profiling(profile)
        times, stats = [], []
        for _ in range(args.steps):
            flush.zero_()
            barrier()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solver.solve(k, tol=tol, u0=u0)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            times.append(e0.elapsed_time(e1) / 1e3)
            stats.append(solver.stats())
        solver.set_profiling(False)
        return times, stats

    clk = ClockSampler(uuid.replace("GPU-", "") if uuid else "")
    s64 = isira.Solver(rp, ci, precision=isira.ISIRA_FP64, **solver_opts(args))
    smx = isira.Solver(rp, ci, precision=isira.ISIRA_MIXED, **solver_opts(args))
    clk.start()
    # headline: the default device-driven inner loop (one CUDA-graph launch per inner solve)
    t64, st64 = timed_solves(s64, False)
    tmx, stmx = timed_solves(smx, False)
    # kernel timing: the same solves with CUDA events around every phase-1 launch (chunked launches)
    tp64, sp64 = timed_solves(s64, True)
    tpmx, spmx = timed_solves(smx, True)
    clocks = clk.stop()
    lam64, vec64, res64 = s64.eigpairs()
    lammx, vecmx, resmx = smx.eigpairs()

    # accuracy of the benchmarked solves against a tight FP64 solve (untimed)
    ref = isira.solve(rp, ci, k, tol=1e-12 * normL, u0=u0, precision=isira.ISIRA_FP64, **solver_opts(args))
    lam_ref = ref.eigvals.numpy()

    def relerr(a):
        return float(np.max(np.abs(a.numpy() - lam_ref) / np.abs(lam_ref)))

    # end to end through the public API, in the precision the configuration names:
    # pinned host CSR -> device, create, solve, eigenpairs -> host
    e2e_times = []
    h2d = rp_h.numel() * 8 + ci_h.numel() * 4 + u0_h.numel() * 8
    d2h = n * k * 8 + k * 8 * 2
    for i in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rp_d = rp_h.to(dev, non_blocking=True)
        ci_d = ci_h.to(dev, non_blocking=True)
        u0_d = u0_h.to(dev, non_blocking=True)
        e2e_prec = isira.ISIRA_MIXED if spec["prec"] == "mixed" else isira.ISIRA_FP64
        with isira.Solver(rp_d, ci_d, precision=e2e_prec, **solver_opts(args)) as s:
            s.solve(k, tol=tol, u0=u0_d)
            lam_e, vec_e, res_e = s.eigpairs()
            vec_host = vec_e.cpu()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            e2e_times.append(dt)
    del vec_host

    value = reduce_max(statistics.mean(t64))
    value_mx = reduce_max(statistics.mean(tmx))
    e2e = reduce_max(statistics.mean(e2e_times))

    # roofline of the dominant kernel (phase 1 of the FP64 inner solve), from the live events
    p1_ms = sum(s["inner_phase1_ms"] for s in sp64)
    p1_n = sum(s["inner_phase1_timed"] for s in sp64)
    p1_c = sum(s["inner_phase1_csum"] for s in sp64) / max(1, p1_n)
    avg_s = p1_ms / 1e3 / max(1, p1_n)
    bytes_launch = phase1_bytes(n, Z, p1_c, 8)
    peak, peak_src = hbm_peak()
    achieved = bytes_launch / avg_s / 1e9 if avg_s > 0 else None
    p1mx_ms = sum(s["inner_phase1_ms"] for s in spmx)
    p1mx_n = sum(s["inner_phase1_timed"] for s in spmx)
    p1mx_c = sum(s["inner_phase1_csum"] for s in spmx) / max(1, p1mx_n)
    avgmx_s = p1mx_ms / 1e3 / max(1, p1mx_n)
    achieved_mx = phase1_bytes(n, Z, p1mx_c, 4) / avgmx_s / 1e9 if avgmx_s > 0 else None
    traffic = ncu_traffic(f"phase1_fp64_{args.workload}")
    ops_peak = fp64_peak_ops(clocks.get("sm_max_mhz"))
    ops_achieved = phase1_fp64_ops(n, Z, p1_c) / avg_s if avg_s > 0 else None

    line = {
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": config_with_opts(workload_config(args.workload, g, k, rel_for_cfg), args),
        "mixed": {"value": value_mx, "unit": "s", "dtype": "f32 inner / f64 outer",
                  "speedup_vs_fp64": value / value_mx if value_mx else None,
                  "roofline": {"kernel": "k_phase1_gather<float>", "bound": "hbm", "achieved": achieved_mx, "peak": peak,
                               "unit": "GB/s", "frac": (achieved_mx / peak) if achieved_mx else None,
                               "bytes_per_launch": phase1_bytes(n, Z, p1mx_c, 4), "avg_deflation_rank": p1mx_c},
                  "outer_steps": stmx[-1]["outer_steps"], "inner_iters": stmx[-1]["inner_iters"],
                  "phase1_avg_us": avgmx_s * 1e6, "phase1_GBps": achieved_mx},
        "fp64": {"outer_steps": st64[-1]["outer_steps"], "inner_iters": st64[-1]["inner_iters"],
                 "restarts": st64[-1]["restarts"], "spmv_lanes": st64[-1]["spmv_lanes"],
                 "phase1_avg_us": avg_s * 1e6, "phase1_launches_timed": p1_n,
                 "timed_with_events_s": statistics.mean(tp64)},
        "accuracy": {"max_rel_eig_err_fp64_vs_tight": relerr(lam64), "max_rel_eig_err_mixed_vs_tight": relerr(lammx),
                     "max_true_resid_rel_fp64": float(res64.max()), "max_true_resid_rel_mixed": float(resmx.max()),
                     "tight_tol_rel": 1e-12, "eigvals": [float(x) for x in lam_ref]},
        "roofline": {"kernel": "k_phase1_gather<double> (trimmed operator SpMV gather)", "bound": "alu",
                     "achieved": ops_achieved / 1e9 if ops_achieved else None, "peak": ops_peak / 1e9,
                     "unit": "G FP64 lane-ops/s", "frac": (ops_achieved / ops_peak) if ops_achieved else None,
                     "peak_source": "derived: 152 SMs x 2 FP64 lanes/clk x max SM clock (1.25 TFLOP/s nominal)",
                     "ops_per_launch": phase1_fp64_ops(n, Z, p1_c), "hbm_achieved_GBps": achieved,
                     "hbm_frac": (achieved / peak) if achieved else None, "hbm_peak": peak, "hbm_peak_source": peak_src,
                     "bytes_per_launch": bytes_launch, "avg_deflation_rank": p1_c, "traffic": traffic},
        "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "path": "pinned host CSR -> isira_create -> isira_solve -> isira_eigpairs -> host"},
        "gpu_launches": int(sum(s["kernel_launches"] for s in (stmx if spec["prec"] == "mixed" else st64))),
        "clocks": clocks,
    }
    if spec["prec"] == "mixed":
        # the configuration names the mixed form: it is the headline, FP64 is reported beside it
        fp64_part = {"value": line["value"], "unit": "s", "dtype": "f64", "roofline": line["roofline"],
                     **line["fp64"]}
        mixed = line.pop("mixed")
        mroof = mixed.pop("roofline")
        line.update(value=mixed["value"], ms_per_step=mixed["value"] * 1e3, dtype="f32 inner / f64 outer",
                    roofline={**mroof, "peak_source": peak_src, "hbm_frac": mroof["frac"],
                              "traffic": ncu_traffic(f"phase1_f32_{args.workload}")})
        line["fp64"] = fp64_part
        line["mixed"] = mixed
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "rmat20":
        full = oracle_full_counts(args.workload)
        dt, st = oracle_sample(g, k, tol, u0_h.numpy(), SAMPLE_STEPS)
        if full is not None:
            line["cpu_baseline"] = {"value": project_oracle(st, full), "unit": "s", "cores": 1, "kind": "oracle",
                                    "sample": sample_text(st, full), "sample_seconds": dt}
    if rank == 0:
        print(json.dumps(line), flush=True)
    s64.close()
    smx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
