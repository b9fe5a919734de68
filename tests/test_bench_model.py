"""CPU checks of bench.py's host-side arithmetic: the accuracy-driven lock tolerance
min(1e-8 ||L||, sqrt(1e-10 lambda_j gap_j)) reproduces the tolerance the oracle's golden 128^3-grid
run was made at, from the grid's closed-form spectrum; the byte models and the CPU-baseline
projection are the stated sums."""
import json
import math
import os

import numpy as np

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _grid_spectrum(dims, k):
    lam = np.zeros(1)
    for N in dims:
        lam = (lam[:, None] + (2.0 - 2.0 * np.cos(np.pi * np.arange(N) / N))[None, :]).ravel()
    return np.sort(lam)[1:k + 1]


def test_accuracy_tolerance_of_the_128_grid_matches_the_golden_run():
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "grid128_accuracy.json")))
    eps = bench.accuracy_eps(_grid_spectrum([128, 128, 128], 20), 12.0)
    # the golden run took its estimates from a loose GPU solve; the closed form gives the same
    # tolerance to the accuracy of those estimates
    assert math.isclose(eps, g["eps_abs"], rel_tol=1e-6)
    assert eps < 1e-8 * 12.0


def test_accuracy_tolerance_merges_clusters_and_caps_at_the_residual_bar():
    # a triple eigenvalue and a well separated one: only the gap to the other cluster counts
    lam = [1.0, 1.0 + 1e-9, 1.0 - 1e-9, 2.0]
    assert math.isclose(bench.accuracy_eps(lam, 1e4), math.sqrt(1e-10 * (1.0 - 1e-9) * (1.0 + 1e-9)))
    # wide gaps: the residual bar 1e-8 ||L|| binds
    assert bench.accuracy_eps([1.0, 3.0], 1e-3) == 1e-8 * 1e-3


def test_byte_models():
    n, Z, w = 1000, 6000, 4
    assert bench.kernel_bytes("gather", n, Z, 0, w) == 8 * (n + 1) + 4 * Z + 2 * w * n
    assert bench.kernel_bytes("gather", n, Z, 0, w, n_long=10, n_slices=32) == 8 * 11 + 8 * 33 + 4 * Z + 2 * w * n
    assert bench.kernel_bytes("rows", n, Z, 3, 8) == 4 * n + 12 * 8 * n + 8 * n
    assert bench.kernel_bytes("rows_ml", n, Z, 3, w) == 4 * n + 10 * w * n
    c, nc, nnzc = 5, 300, 2000
    expect = (25 + 4 * c) * w * n + 8 * n + 2 * (8 * (n + 1) + 4 * Z) + 2 * (4 + w) * nnzc + (16 + 5 * w) * nc
    assert bench.kernel_bytes("phase2_ml", n, Z, c, w, ml=(nc, nnzc)) == expect


def test_cpu_baseline_projection_is_the_per_unit_sum():
    st = {"sec_w": 2.0, "w_columns": 4, "sec_inner": 3.0, "inner_iters": 30, "sec_total": 6.0, "outer_steps": 2}
    counts = {"w_columns": 100, "inner_iters": 1000, "outer_steps": 10}
    # 0.5 s per column, 0.1 s per iteration, 0.5 s per outer step for the rest
    assert math.isclose(bench.project(st, counts), 50.0 + 100.0 + 5.0)
    st["rate_sec_per_it"] = 0.2              # measured at the solve's average deflation rank
    assert math.isclose(bench.project(st, counts), 50.0 + 200.0 + 5.0)
