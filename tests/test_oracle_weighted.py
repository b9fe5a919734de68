"""Pins for the oracle on weighted graphs: the weighted Laplacian L_w = D_w - W of the Remark after
Theorem 1.2 (D_w = diagonal of the weighted degrees).  The method's theory carries over unchanged
(L_w is a symmetric, singular, irreducible M-matrix with null space span{1}), so the checks are
the unweighted ones with weights: brute force on the edge list, uniform weights scaling closed
forms, LAPACK on the assembled matrix, Theorems 2.4/2.6 by dense solves, and Algorithm 2 against
the dense definition."""
import numpy as np
import pytest

import oracle
import synthgraphs as sg
from tests import closed_forms as cf


def weighted_dense(g, w):
    """L_w assembled entry by entry from the edge list."""
    L = np.zeros((g.n, g.n))
    for r in range(g.n):
        for e in range(g.row_ptr[r], g.row_ptr[r + 1]):
            c = g.col_idx[e]
            L[r, c] -= w[e]
            L[r, r] += w[e]
    return L


def graphs():
    return [sg.path(9), sg.grid2d(4, 5), sg.erdos_renyi(60, 5.0, seed=3), sg.rmat(7)]


@pytest.mark.parametrize("g", graphs(), ids=lambda g: g.name)
def test_weighted_laplacian_definition(g):
    w = sg.edge_weights(g, seed=4)
    L = weighted_dense(g, w)
    np.testing.assert_allclose(L, L.T, atol=0)                       # symmetric weights
    I = np.eye(g.n)
    Lo = oracle.laplacian_apply(g.row_ptr, g.col_idx, I, weights=w)
    np.testing.assert_allclose(Lo, L, rtol=0, atol=1e-14 * np.abs(L).max())
    np.testing.assert_allclose(oracle.laplacian_apply(g.row_ptr, g.col_idx, np.ones(g.n), weights=w), 0.0,
                               atol=1e-13 * np.abs(L).max())
    rng = np.random.default_rng(2)
    x = rng.standard_normal(g.n)
    quad = 0.0
    for r in range(g.n):                                              # x^T L_w x = sum_edges w (x_u - x_v)^2
        for e in range(g.row_ptr[r], g.row_ptr[r + 1]):
            c = g.col_idx[e]
            if r < c:
                quad += w[e] * (x[r] - x[c]) ** 2
    np.testing.assert_allclose(x @ oracle.laplacian_apply(g.row_ptr, g.col_idx, x, weights=w), quad, rtol=1e-12)


@pytest.mark.parametrize("g,ref", [(sg.path(30), cf.path(30)), (sg.grid2d(5, 6), cf.grid2d(5, 6))],
                         ids=["path30", "grid5x6"])
def test_uniform_weight_scales_closed_forms(g, ref):
    w = np.full(g.nnz, 2.5)
    lam, _ = oracle.dense_laplacian_eig(g.row_ptr, g.col_idx, weights=w)
    np.testing.assert_allclose(lam, 2.5 * ref, atol=1e-12 * 2.5 * ref.max())
    lam4, V, st = oracle.isira(g.row_ptr, g.col_idx, 4, sg.start_vector(g.n, 1), eps=1e-10, tau_inner=1e-3,
                               weights=w)
    assert st["status"] == 0
    np.testing.assert_allclose(np.sort(lam4), 2.5 * ref[1:5], rtol=1e-9)


def test_weighted_dense_matches_lapack():
    g = sg.erdos_renyi(60, 5.0, seed=3)
    w = sg.edge_weights(g, seed=9)
    lam, X = oracle.dense_laplacian_eig(g.row_ptr, g.col_idx, weights=w)
    L = weighted_dense(g, w)
    np.testing.assert_allclose(lam, np.linalg.eigvalsh(L), atol=1e-12 * np.abs(L).max())
    np.testing.assert_allclose(L @ X, X * lam[None, :], atol=1e-11 * np.abs(L).max())


@pytest.mark.parametrize("trim,c,sigma", [(0, 0, 0.0), (5, 2, 0.3), (17, 3, 0.9)])
def test_weighted_trimmed_solution_solves_singular_system(trim, c, sigma):
    """Theorems 2.4/2.6 with L_w: the back-mapped solution of the trimmed system solves
    (L_w + delta V V^T - sigma I) z = r with 1^T z = 0."""
    g = sg.erdos_renyi(30, 6.0, seed=11)
    w = sg.edge_weights(g, seed=5)
    L = weighted_dense(g, w)
    lam, X = np.linalg.eigh(L)
    V = X[:, 1:1 + c] if c else None
    delta = 2.0 * np.diag(L).max()
    nh = g.n - 1
    M = np.stack([oracle.trimmed_apply(g.row_ptr, g.col_idx, trim, sigma, delta, V, np.eye(nh)[:, j], weights=w)
                  for j in range(nh)], axis=1)
    np.testing.assert_allclose(M, M.T, atol=1e-12 * np.abs(M).max())
    rng = np.random.default_rng(trim + c)
    r = rng.standard_normal(g.n)
    r -= r.mean()
    z = oracle.backmap(g.n, trim, np.linalg.solve(M, np.delete(r, trim)))
    assert abs(z.sum()) <= 1e-11 * np.abs(z).sum()
    Vd = V if c else np.zeros((g.n, 0))
    np.testing.assert_allclose((L + delta * Vd @ Vd.T - sigma * np.eye(g.n)) @ z, r, atol=1e-9 * np.abs(r).max())
    # the oracle's own inner solve reaches the same vector
    zo, _, _ = oracle.inner_solve(g.row_ptr, g.col_idx, trim, sigma, delta, V, r, tau=1e-13, max_it=5000, weights=w)
    np.testing.assert_allclose(zo, z, atol=1e-8 * np.abs(z).max())


@pytest.mark.parametrize("g,d", [(sg.erdos_renyi(150, 6.0, seed=9), 6), (sg.grid2d(12, 13), 5)],
                         ids=["er150", "grid12x13"])
def test_weighted_isira_matches_dense_definition(g, d):
    w = sg.edge_weights(g, seed=2)
    lam, V, st = oracle.isira(g.row_ptr, g.col_idx, d, sg.start_vector(g.n, 1), eps=1e-10, tau_inner=1e-3,
                              weights=w)
    assert st["status"] == 0 and st["n_locked"] == d
    L = weighted_dense(g, w)
    ref = np.linalg.eigvalsh(L)[1:1 + d]
    order = np.argsort(lam)
    np.testing.assert_allclose(lam[order], ref, rtol=1e-9)
    R = L @ V - V * lam[None, :]
    assert np.abs(R).max() <= 1e-9
    assert st["trim"] == int(np.argmax(np.diag(L)))                   # Remark 4.1(i): largest diagonal entry
    np.testing.assert_allclose(st["delta"], 2.0 * np.diag(L).max())   # Remark 4.1(ii)
