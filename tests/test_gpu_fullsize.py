"""Full-size parity on the benchmark workload (R-MAT scale 20 LCC, n = 646,379, nnz = 31.4 M,
k = 10), in the launch configuration bench.py times, against stored eigenvalues of the FP64
oracle's full run (tests/golden/, written by tests/golden/make_golden.py from oracle/ only) and
against residuals the oracle recomputes from the GPU eigenvectors."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synthgraphs as sg
from tests.gpu_util import dev_graph, need_gpu, torch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def rmat20():
    need_gpu()
    return sg.workload("rmat20")


def golden(name):
    return json.load(open(os.path.join(HERE, "golden", name)))


def solve(g, prec, eps_rel):
    import paper_1710_07080_gb300 as isira
    rp, ci = dev_graph(g)
    u0 = torch.from_numpy(sg.start_vector(g.n, 1)).cuda()
    p = isira.ISIRA_FP64 if prec == "fp64" else isira.ISIRA_MIXED
    return isira.solve(rp, ci, 10, tol=eps_rel * 2.0 * g.degrees.max(), u0=u0, precision=p)


def oracle_residuals(g, lam, V):
    normL = 2.0 * g.degrees.max()
    return np.array([np.linalg.norm(oracle.laplacian_apply(g.row_ptr, g.col_idx, V[:, j]) - lam[j] * V[:, j])
                     for j in range(lam.shape[0])]) / normL


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rmat20_tight_matches_oracle_eigenvalues(rmat20, prec):
    g = rmat20
    gold = golden("rmat20_tight.json")
    assert (gold["n"], gold["nnz"]) == (g.n, g.nnz)
    res = solve(g, prec, 1e-12)
    assert res.status == 0
    lam = res.eigvals.numpy()
    V = res.eigvecs.cpu().numpy()
    np.testing.assert_allclose(lam, gold["eigvals"], rtol=1e-9)
    r = oracle_residuals(g, lam, V)
    assert r.max() <= 1e-11
    np.testing.assert_allclose(res.true_resid.numpy(), r, rtol=1e-3, atol=1e-15)
    np.testing.assert_allclose(V.T @ V, np.eye(10), atol=1e-10)
    assert np.abs(V.sum(axis=0)).max() <= 1e-9 * math.sqrt(g.n)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rmat20_benchmark_tolerance(rmat20, prec):
    """At the benchmark's residual 1e-8 (relative to 2 d_max): every pair meets it (checked by the
    oracle), and each eigenvalue lies within its residual norm of a true eigenvalue
    (Bauer-Fike for symmetric matrices), here the oracle's tight values."""
    g = rmat20
    gold = golden("rmat20_tight.json")
    res = solve(g, prec, 1e-8)
    assert res.status == 0
    lam = res.eigvals.numpy()
    V = res.eigvecs.cpu().numpy()
    r = oracle_residuals(g, lam, V)
    assert r.max() <= 1e-8
    normL = 2.0 * g.degrees.max()
    ref = np.array(gold["eigvals"])
    for j in range(10):
        assert np.min(np.abs(ref - lam[j])) <= r[j] * normL * (1 + 1e-6) + 1e-14
    if prec == "fp64":
        # same algorithm, same readings: the FP64 oracle's run at this tolerance took as many steps
        st = golden("rmat20_bench.json")["oracle_stats"]
        assert abs(res.stats["outer_steps"] - st["outer_steps"]) <= 3
