"""Weighted graph Laplacian L_w = D_w - W (paper Sec. 1.1, the Remark after Theorem 1.2) on the GPU:
the trimmed operator against the oracle's on the same weights, the Remark 4.1 choices on the
weighted diagonal, and whole solves against uniform-weight closed forms, the dense definition
and the oracle's Algorithm 2."""
import numpy as np
import pytest

import oracle
import synthgraphs as sg
from tests import closed_forms as cf
from tests.gpu_util import dev_graph, need_gpu, orthonormal_columns, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def isira():
    need_gpu()
    import paper_1710_07080_gb300 as m
    return m


def graphs():
    return {"grid31x33": sg.grid2d(31, 33), "rmat12": sg.rmat(12), "er3000": sg.erdos_renyi(3000, 8.0, seed=5),
            "star5000": sg.star(5000)}


def _wdense(g, w):
    import scipy.sparse as sp
    W = sp.csr_matrix((w, g.col_idx, g.row_ptr), shape=(g.n, g.n))
    return (sp.diags(np.asarray(W.sum(axis=1)).ravel()) - W).toarray()


@pytest.mark.parametrize("name", list(graphs().keys()))
@pytest.mark.parametrize("reorder", [0, 1])
@pytest.mark.parametrize("sigma,c", [(0.0, 0), (0.3, 3)])
def test_weighted_operator_fp64_matches_oracle(isira, name, reorder, sigma, c):
    g = graphs()[name]
    w = sg.edge_weights(g, seed=3)
    rp, ci = dev_graph(g)
    tw = torch.from_numpy(w).cuda()
    with isira.Solver(rp, ci, weights=tw, precision=isira.ISIRA_FP64, reorder=reorder) as s:
        st = s.stats()
        trim, delta = st["trim_index"], st["delta"]
        dw = np.zeros(g.n)
        np.add.at(dw, np.repeat(np.arange(g.n), g.degrees), w)
        assert trim == int(np.argmax(dw))                      # Remark 4.1(i) on the weighted diagonal
        np.testing.assert_allclose([delta, st["norm_L"], st["max_diag"]], [2 * dw.max()] * 2 + [dw.max()])
        rng = np.random.default_rng(c + reorder)
        x = rng.standard_normal(g.n)
        V = orthonormal_columns(g.n, c, 4) if c else None
        y = s.apply_operator(torch.from_numpy(x).cuda(), sigma=sigma,
                             V=torch.from_numpy(V).cuda() if c else None).cpu().numpy()
        x0 = x.copy()
        x0[trim] = 0.0
        ref = np.insert(oracle.trimmed_apply(g.row_ptr, g.col_idx, trim, sigma, delta, V, np.delete(x0, trim),
                                             weights=w), trim, 0.0)
        np.testing.assert_allclose(y, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("name", ["grid31x33", "rmat12"])
def test_weighted_operator_fp32_within_rounding_bound(isira, name):
    g = graphs()[name]
    w = sg.edge_weights(g, seed=8)
    rp, ci = dev_graph(g)
    with isira.Solver(rp, ci, weights=torch.from_numpy(w).cuda(), precision=isira.ISIRA_MIXED) as s:
        st = s.stats()
        trim, delta = st["trim_index"], st["delta"]
        sigma = 0.2
        rng = np.random.default_rng(1)
        x = rng.standard_normal(g.n).astype(np.float32).astype(np.float64)
        y = s.apply_operator(torch.from_numpy(x).float().cuda(), sigma=sigma).double().cpu().numpy()
        x[trim] = 0.0
        ref = np.insert(oracle.trimmed_apply(g.row_ptr, g.col_idx, trim, sigma, delta, None, np.delete(x, trim),
                                             weights=w), trim, 0.0)
        import scipy.sparse as sp
        W = sp.csr_matrix((w, g.col_idx, g.row_ptr), shape=(g.n, g.n))
        dw = np.asarray(W.sum(axis=1)).ravel()
        # terms: weights and weighted degrees rounded to FP32, products and sums in FP32
        local = (dw + sigma) * np.abs(x) + W @ np.abs(x) + sigma / g.n * np.abs(x).sum()
        bound = (g.degrees + 8) * 2.0 ** -24 * local + sigma / g.n * np.abs(x).sum() * g.n * 2.0 ** -24
        assert np.all(np.abs(y - ref) <= 2 * bound + 1e-30), float(np.max(np.abs(y - ref) / bound))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("precond", [0, 1])
def test_weighted_solves(isira, prec, precond):
    from tests.test_gpu_solve import _prec
    p = _prec(isira, prec)
    # uniform weight 2.5 scales the closed form
    g = sg.grid2d(40, 37)
    rp, ci = dev_graph(g)
    u0 = torch.from_numpy(sg.start_vector(g.n, 1)).cuda()
    res = isira.solve(rp, ci, 5, tol=1e-10, u0=u0, precision=p, precond=precond,
                      weights=torch.full((g.nnz,), 2.5, dtype=torch.float64, device="cuda"))
    assert res.status == isira.ISIRA_OK
    np.testing.assert_allclose(res.eigvals.numpy(), 2.5 * cf.grid2d(40, 37)[1:6], rtol=1e-9)
    # random weights: the dense definition and the oracle's Algorithm 2
    g = sg.erdos_renyi(1200, 8.0, seed=2)
    w = sg.edge_weights(g, seed=6)
    rp, ci = dev_graph(g)
    u0 = torch.from_numpy(sg.start_vector(g.n, 1)).cuda()
    res = isira.solve(rp, ci, 6, tol=1e-10, u0=u0, precision=p, precond=precond,
                      weights=torch.from_numpy(w).cuda())
    assert res.status == isira.ISIRA_OK
    lam = res.eigvals.numpy()
    V = res.eigvecs.cpu().numpy()
    L = _wdense(g, w)
    np.testing.assert_allclose(lam, np.linalg.eigvalsh(L)[1:7], rtol=1e-9)
    normL = 2.0 * np.diag(L).max()
    R = L @ V - V * lam[None, :]
    assert np.linalg.norm(R, axis=0).max() / normL <= 1e-8
    np.testing.assert_allclose(res.true_resid.numpy(), np.linalg.norm(R, axis=0) / normL, rtol=1e-5, atol=1e-15)
    lam_or, _, st = oracle.isira(g.row_ptr, g.col_idx, 6, sg.start_vector(g.n, 1), eps=1e-10, tau_inner=1e-3,
                                 weights=w)
    assert st["status"] == 0
    np.testing.assert_allclose(lam, np.sort(lam_or), rtol=1e-9)
