"""Pins for the FP64 oracle: each test checks it against something other than itself
(closed forms, LAPACK as a library routine, brute force on tiny inputs, and the
theorems of the paper), chosen so that a dropped term, a wrong sign or index or a
transposed operand in the oracle fails at least one of them."""
import math

import numpy as np
import pytest

import oracle
import synthgraphs as sg
from tests import closed_forms as cf


def dense_laplacian_bruteforce(g):
    """L = D - A written out entry by entry from the edge list (Eq. 1.1)."""
    n = g.n
    L = np.zeros((n, n))
    for r in range(n):
        for e in range(g.row_ptr[r], g.row_ptr[r + 1]):
            c = g.col_idx[e]
            L[r, c] -= 1.0
            L[r, r] += 1.0
    return L


def small_graphs():
    return [sg.path(7), sg.cycle(9), sg.complete(6), sg.star(8), sg.hypercube(3), sg.grid2d(4, 5),
            sg.erdos_renyi(60, 5.0, seed=3), sg.rmat(7), sg.watts_strogatz(50, 6, 0.2, seed=5)]


# ----------------------------------------------------------------------------- Jacobi eigensolver

@pytest.mark.parametrize("k", [1, 2, 3, 7, 20, 31, 64])
def test_sym_eig_matches_lapack(k):
    rng = np.random.default_rng(k)
    B = rng.standard_normal((k, k))
    A = B + B.T
    th, S, sweeps = oracle.sym_eig(A)
    assert sweeps >= 0
    ref = np.linalg.eigvalsh(A)
    scale = np.abs(ref).max()
    assert np.all(np.diff(th) >= 0)
    np.testing.assert_allclose(th, ref, atol=1e-13 * scale * k)
    np.testing.assert_allclose(A @ S, S * th[None, :], atol=1e-12 * scale * k)
    np.testing.assert_allclose(S.T @ S, np.eye(k), atol=1e-13 * k)
    for t in range(k):  # sign rule: largest-magnitude entry (first on ties) is positive
        col = S[:, t]
        assert col[np.argmax(np.abs(col))] > 0


def test_sym_eig_special_cases():
    th, S, _ = oracle.sym_eig(np.diag([3.0, -1.0, 2.0]))
    np.testing.assert_array_equal(th, [-1.0, 2.0, 3.0])
    np.testing.assert_array_equal(np.abs(S), np.eye(3)[:, [1, 2, 0]])
    # 2x2 closed form: [[a, b], [b, c]] has (a+c)/2 -+ sqrt(((a-c)/2)^2 + b^2)
    a, b, c = 2.0, 3.0, -1.0
    th, S, _ = oracle.sym_eig(np.array([[a, b], [b, c]]))
    rad = math.sqrt(((a - c) / 2) ** 2 + b * b)
    np.testing.assert_allclose(th, [(a + c) / 2 - rad, (a + c) / 2 + rad], rtol=1e-15)
    th, S, _ = oracle.sym_eig(np.eye(5) * 4.0)
    np.testing.assert_array_equal(th, [4.0] * 5)


# ----------------------------------------------------------------------------- definition oracle

@pytest.mark.parametrize("g,ref", [
    (sg.path(12), cf.path(12)),
    (sg.cycle(11), cf.cycle(11)),
    (sg.complete(9), cf.complete(9)),
    (sg.star(10), cf.star(10)),
    (sg.hypercube(5), cf.hypercube(5)),
    (sg.grid2d(6, 7), cf.grid2d(6, 7)),
    (sg.grid3d(3, 4, 5), cf.grid3d(3, 4, 5)),
], ids=lambda x: getattr(x, "name", ""))
def test_dense_eig_closed_forms(g, ref):
    lam, X = oracle.dense_laplacian_eig(g.row_ptr, g.col_idx)
    np.testing.assert_allclose(lam, ref, atol=1e-12 * max(1.0, ref.max()))
    L = dense_laplacian_bruteforce(g)
    np.testing.assert_allclose(L @ X, X * lam[None, :], atol=1e-11 * ref.max())


@pytest.mark.parametrize("g", small_graphs(), ids=lambda g: g.name)
def test_laplacian_apply_and_invariants(g):
    """Theorem 1.2: L 1 = 0, L symmetric, x^T L x = sum over edges (x_u - x_v)^2 >= 0."""
    rng = np.random.default_rng(0)
    n = g.n
    L = dense_laplacian_bruteforce(g)
    x, y = rng.standard_normal(n), rng.standard_normal(n)
    Lx = oracle.laplacian_apply(g.row_ptr, g.col_idx, x)
    np.testing.assert_allclose(Lx, L @ x, atol=1e-12 * n)
    np.testing.assert_allclose(oracle.laplacian_apply(g.row_ptr, g.col_idx, np.ones(n)), 0.0, atol=0)
    Ly = oracle.laplacian_apply(g.row_ptr, g.col_idx, y)
    assert abs(x @ Ly - y @ Lx) <= 1e-10 * n
    quad = sum((x[u] - x[g.col_idx[e]]) ** 2 for u in range(n)
               for e in range(g.row_ptr[u], g.row_ptr[u + 1])) / 2.0
    assert abs(x @ Lx - quad) <= 1e-10 * abs(quad)
    lam, _ = oracle.dense_laplacian_eig(g.row_ptr, g.col_idx)
    np.testing.assert_allclose(lam, np.linalg.eigvalsh(L), atol=1e-11 * lam.max())
    assert lam[0] > -1e-12 and lam[1] > 1e-8   # connected: one zero eigenvalue (Thm 1.2 ii)


def test_laplacian_apply_integer_exact():
    """On integer-valued x every term is an exactly representable integer."""
    g = sg.rmat(8)
    x = np.arange(g.n, dtype=np.float64) % 17 - 8
    L = dense_laplacian_bruteforce(g)
    np.testing.assert_array_equal(oracle.laplacian_apply(g.row_ptr, g.col_idx, x), L @ x)


# ----------------------------------------------------------------------------- trimming + deflation

def _trimmed_matrix(g, trim, sigma, delta, V, drop_rank1=False):
    n = g.n
    M = np.zeros((n - 1, n - 1))
    for t in range(n - 1):
        e = np.zeros(n - 1)
        e[t] = 1.0
        M[:, t] = oracle.trimmed_apply(g.row_ptr, g.col_idx, trim, sigma, delta, V, e, drop_rank1)
    return M


@pytest.mark.parametrize("trim", [0, 5, 29])
@pytest.mark.parametrize("c,sigma", [(0, 0.0), (0, 0.35), (2, 0.0), (3, 0.8)])
def test_theorem_2_6_trimmed_solution_solves_singular_system(trim, c, sigma):
    """Theorems 2.4/2.6: if zh solves the trimmed system, the back-mapped z* satisfies
    (L + delta V V^T - sigma I) z* = r and 1^T z* = 0, for r orthogonal to 1 and V made of
    eigenvectors of L orthogonal to 1."""
    g = sg.erdos_renyi(30, 6.0, seed=11)
    assert g.n == 30
    L = dense_laplacian_bruteforce(g)
    lam, X = np.linalg.eigh(L)
    V = X[:, 1:1 + c]
    delta = 2.0 * g.degrees.max()
    rng = np.random.default_rng(trim + 7 * c)
    r = rng.standard_normal(g.n)
    r -= r.mean()
    rh = np.delete(r, trim)
    M = _trimmed_matrix(g, trim, sigma, delta, V)
    np.testing.assert_allclose(M, M.T, atol=1e-12)        # symmetric operator
    zh = np.linalg.solve(M, rh)
    z = oracle.backmap(g.n, trim, zh)
    assert abs(z.sum()) <= 1e-11 * np.abs(z).sum()
    Ltil = L + delta * V @ V.T - sigma * np.eye(g.n)
    np.testing.assert_allclose(Ltil @ z, r, atol=1e-9 * np.abs(r).max())
    if sigma != 0.0:   # Remark 3.1: dropping the rank-one term loses exactness
        Md = _trimmed_matrix(g, trim, sigma, delta, V, drop_rank1=True)
        zd = oracle.backmap(g.n, trim, np.linalg.solve(Md, rh))
        assert np.abs(Ltil @ zd - r).max() > 1e-6 * np.abs(r).max()


def test_trimmed_matrix_is_spd_at_zero_shift():
    """Theorem 2.3: the trimmed Laplacian is a nonsingular M-matrix (SPD)."""
    g = sg.rmat(7)
    for trim in [0, g.n // 2, g.n - 1]:
        M = _trimmed_matrix(g, trim, 0.0, 1.0, None)
        off = M - np.diag(np.diag(M))
        assert off.max() <= 0.0
        assert np.linalg.eigvalsh(M).min() > 0.0


def test_trimmed_inertia_matches_deflated_operator():
    """Inertia of the trimmed operator equals that of (L + delta V V^T - sigma I) on 1-perp:
    the congruence used in the proof of Theorem 2.6."""
    g = sg.erdos_renyi(40, 5.0, seed=4)
    L = dense_laplacian_bruteforce(g)
    lam, X = np.linalg.eigh(L)
    delta = 2.0 * g.degrees.max()
    V = X[:, 1:3]
    for sigma in [0.0, 0.5 * (lam[3] + lam[4]), 0.5 * (lam[5] + lam[6])]:
        M = _trimmed_matrix(g, 3, sigma, delta, V)
        ev = np.linalg.eigvalsh(M)
        full = np.linalg.eigvalsh(L + delta * V @ V.T - sigma * np.eye(g.n))
        # drop the eigenvalue -sigma that belongs to the direction 1
        full = np.delete(full, np.argmin(np.abs(full + sigma)))
        assert (ev < 0).sum() == (full < 0).sum()


def test_backmap_is_orthogonal_to_ones_and_places_zero():
    zh = np.arange(1.0, 10.0)
    z = oracle.backmap(10, 4, zh)
    shift = zh.sum() / 10
    np.testing.assert_allclose(z, np.concatenate([zh[:4], [0.0], zh[4:]]) - shift, rtol=0, atol=1e-15)
    assert abs(z.sum()) < 1e-12


def test_preconditioner_smw_inverts_its_matrix():
    """Eq. 3.6: the SMW form applies (Mh + delta Vh Vh^T)^{-1} with Mh = diag(deg - sigma)."""
    g = sg.erdos_renyi(50, 6.0, seed=2)
    L = dense_laplacian_bruteforce(g)
    _, X = np.linalg.eigh(L)
    trim, sigma, delta = 7, 0.2, 2.0 * g.degrees.max()
    for c in [0, 1, 4]:
        V = X[:, 1:1 + c]
        Vh = np.delete(V, trim, axis=0)
        deg = np.delete(g.degrees.astype(float), trim)
        P = np.diag(deg - sigma) + delta * Vh @ Vh.T
        x = np.random.default_rng(c).standard_normal(g.n - 1)
        p = oracle.precond_apply(g.row_ptr, trim, sigma, delta, V if c else None, x)
        np.testing.assert_allclose(P @ p, x, atol=1e-11 * np.abs(x).max())


@pytest.mark.parametrize("case", ["spd", "indefinite"])
def test_minres_matches_direct_solve(case):
    g = sg.rmat(7)
    L = dense_laplacian_bruteforce(g)
    lam, X = np.linalg.eigh(L)
    delta = 2.0 * g.degrees.max()
    trim = int(np.argmax(g.degrees))
    if case == "spd":
        V, sigma = None, 0.0
    else:
        V, sigma = X[:, 1:3], 0.5 * (lam[4] + lam[5])
    r = np.random.default_rng(1).standard_normal(g.n)
    r -= r.mean()
    z, its, rel = oracle.inner_solve(g.row_ptr, g.col_idx, trim, sigma, delta, V, r, tau=1e-13, max_it=5000)
    M = _trimmed_matrix(g, trim, sigma, delta, V)
    zref = oracle.backmap(g.n, trim, np.linalg.solve(M, np.delete(r, trim)))
    np.testing.assert_allclose(z, zref, atol=1e-8 * np.abs(zref).max())
    assert rel <= 1e-13


def test_deflation_moves_locked_eigenvalues():
    """Theorem 2.5: spectrum of L + delta V V^T is {lambda_j + delta} plus the rest unchanged."""
    g = sg.grid2d(5, 6)
    L = dense_laplacian_bruteforce(g)
    lam, X = oracle.dense_laplacian_eig(g.row_ptr, g.col_idx)
    delta = 2.0 * g.degrees.max()
    V = X[:, 1:4]
    ev = np.linalg.eigvalsh(L + delta * V @ V.T)
    expect = np.sort(np.concatenate([lam[[0]], lam[4:], lam[1:4] + delta]))
    np.testing.assert_allclose(ev, expect, atol=1e-11 * delta)


# ----------------------------------------------------------------------------- Algorithm 2

def _check_pairs(g, lam, V, eps, ref=None, rtol=1e-9):
    L = dense_laplacian_bruteforce(g) if g.n <= 3000 else None
    order = np.argsort(lam)
    lam, V = lam[order], V[:, order]
    for j in range(lam.shape[0]):
        Lv = oracle.laplacian_apply(g.row_ptr, g.col_idx, V[:, j])
        assert np.linalg.norm(Lv - lam[j] * V[:, j]) <= 2 * eps
    np.testing.assert_allclose(V.T @ V, np.eye(V.shape[1]), atol=1e-10)
    np.testing.assert_allclose(V.sum(axis=0), 0.0, atol=1e-9 * math.sqrt(g.n))
    if ref is not None:
        np.testing.assert_allclose(lam, ref, rtol=rtol, atol=1e-13)
    return lam


@pytest.mark.parametrize("g,ref,d", [
    (sg.path(40), cf.path(40), 6),
    (sg.cycle(40), cf.cycle(40), 7),
    (sg.grid2d(20, 20), cf.grid2d(20, 20), 8),
    (sg.grid2d(100, 100), cf.grid2d(100, 100), 5),
    (sg.grid3d(8, 8, 8), cf.grid3d(8, 8, 8), 6),
    (sg.hypercube(6), cf.hypercube(6), 3),
    (sg.star(30), cf.star(30), 1),
    (sg.complete(25), cf.complete(25), 4),
], ids=lambda x: getattr(x, "name", "") if hasattr(x, "name") else "")
def test_isira_closed_forms(g, ref, d):
    eps = 1e-10
    u0 = sg.start_vector(g.n, 1)
    lam, V, st = oracle.isira(g.row_ptr, g.col_idx, d, u0, eps=eps, tau_inner=1e-3)
    assert st["status"] == 0 and st["n_locked"] == d
    _check_pairs(g, lam, V, eps, ref[1:1 + d])


@pytest.mark.parametrize("g,d", [(sg.rmat(9), 10), (sg.erdos_renyi(150, 6.0, seed=9), 8),
                                 (sg.watts_strogatz(180, 6, 0.1, seed=3), 6)], ids=lambda x: getattr(x, "name", ""))
def test_isira_matches_dense_definition(g, d):
    eps = 1e-9
    u0 = sg.start_vector(g.n, 1)
    lam, V, st = oracle.isira(g.row_ptr, g.col_idx, d, u0, eps=eps, tau_inner=1e-3)
    assert st["status"] == 0
    dl, _ = oracle.dense_laplacian_eig(g.row_ptr, g.col_idx)
    lam = _check_pairs(g, lam, V, eps, dl[1:1 + d], rtol=1e-9)
    # Rayleigh-quotient bound |lambda - theta| <= ||r||^2 / gap, with the gap to the rest of the spectrum
    gap = np.min(np.abs(dl[1 + d:1 + d + 1] - lam[-1]))
    if gap > 1e-6:
        assert abs(lam[-1] - dl[d]) <= (2 * eps) ** 2 / gap + 1e-13 * dl[d]


def test_isira_drop_rank1_and_explicit_trim_reach_same_pairs():
    g = sg.grid2d(12, 13)
    u0 = sg.start_vector(g.n, 1)
    base, _, _ = oracle.isira(g.row_ptr, g.col_idx, 5, u0, eps=1e-10, tau_inner=1e-3)
    for kw in [dict(drop_rank1=True), dict(trim=0), dict(trim=g.n - 1)]:
        lam, V, st = oracle.isira(g.row_ptr, g.col_idx, 5, u0, eps=1e-10, tau_inner=1e-3, **kw)
        assert st["status"] == 0
        np.testing.assert_allclose(np.sort(lam), np.sort(base), rtol=1e-9)


def test_isira_reports_no_convergence_and_keeps_locked():
    g = sg.grid2d(10, 10)
    u0 = sg.start_vector(g.n, 1)
    lam, V, st = oracle.isira(g.row_ptr, g.col_idx, 5, u0, eps=1e-10, tau_inner=1e-3, max_outer=12)
    assert st["status"] == 1 and st["n_locked"] < 5


def test_isira_rejects_bad_arguments():
    g = sg.path(5)
    u0 = sg.start_vector(g.n, 1)
    _, _, st = oracle.isira(g.row_ptr, g.col_idx, 4, u0)
    assert st["status"] == 2


def test_isira_restart_branch_keeps_the_closed_form_pairs():
    """A small search space (m = 6, q = 4 for d = 4) forces restarts (U <- U S(:, 1:q)); the locked
    pairs are still the path graph's closed-form eigenpairs."""
    g = sg.path(40)
    eps = 1e-10
    lam, V, st = oracle.isira(g.row_ptr, g.col_idx, 4, sg.start_vector(g.n, 1), eps=eps, tau_inner=1e-3,
                              m=6, q=4)
    assert st["status"] == 0 and st["n_locked"] == 4
    assert st["restarts"] > 0
    _check_pairs(g, lam, V, eps, cf.path(40)[1:5])
