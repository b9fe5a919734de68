"""Parity of the single GPU kernels with the FP64 oracle: the trimmed operator (every
lane count, every row class), the Rayleigh-Ritz eigensolver, and the inner solve."""
import numpy as np
import pytest

import oracle
import synthgraphs as sg
from tests.gpu_util import abs_adjacency_apply, dev_graph, need_gpu, orthonormal_columns, torch

pytestmark = pytest.mark.gpu

LANES = [1, 2, 4, 8, 16, 32]


def graphs():
    return {
        "grid31x33": sg.grid2d(31, 33),        # ragged tail: n = 1023
        "rmat12": sg.rmat(12),                 # light + medium rows
        "star5000": sg.star(5000),             # one heavy row (degree 4999 > 4096)
        "er3000": sg.erdos_renyi(3000, 8.0, seed=5),
        "path997": sg.path(997),
    }


@pytest.fixture(scope="module")
def isira():
    need_gpu()
    import paper_1710_07080_gb300 as m
    return m


def _oracle_op(g, trim, sigma, delta, V, x, drop=False):
    xh = np.delete(x, trim)
    yh = oracle.trimmed_apply(g.row_ptr, g.col_idx, trim, sigma, delta, V, xh, drop)
    return np.insert(yh, trim, 0.0)


@pytest.mark.parametrize("name", list(graphs().keys()))
@pytest.mark.parametrize("lanes", LANES)
def test_operator_fp64_integer_inputs_bit_exact(isira, name, lanes):
    g = graphs()[name]
    rp, ci = dev_graph(g)
    with isira.Solver(rp, ci, precision=isira.ISIRA_FP64, spmv_lanes=lanes) as s:
        st = s.stats()
        assert st["spmv_lanes"] == lanes
        x = (np.arange(g.n) * 7919 % 23 - 11).astype(np.float64)
        y = s.apply_operator(torch.from_numpy(x).cuda(), sigma=0.0).cpu().numpy()
        ref = _oracle_op(g, st["trim_index"], 0.0, st["delta"], None, np.where(np.arange(g.n) == st["trim_index"], 0, x))
        np.testing.assert_array_equal(y, ref)


@pytest.mark.parametrize("name", list(graphs().keys()))
@pytest.mark.parametrize("lanes,reorder", [(1, 0), (4, 0), (32, 0), (4, 1)])
@pytest.mark.parametrize("sigma,c", [(0.0, 0), (0.37, 0), (0.21, 3), (1.7, 9)])
def test_operator_fp64_matches_oracle(isira, name, lanes, reorder, sigma, c):
    g = graphs()[name]
    rp, ci = dev_graph(g)
    rng = np.random.default_rng(lanes + c)
    with isira.Solver(rp, ci, precision=isira.ISIRA_FP64, spmv_lanes=lanes, reorder=reorder) as s:
        st = s.stats()
        trim, delta = st["trim_index"], st["delta"]
        x = rng.standard_normal(g.n)
        V = orthonormal_columns(g.n, c, 3) if c else None
        Vt = torch.from_numpy(V).cuda() if c else None
        y = s.apply_operator(torch.from_numpy(x).cuda(), sigma=sigma, V=Vt).cpu().numpy()
        x0 = x.copy()
        x0[trim] = 0.0
        ref = _oracle_op(g, trim, sigma, delta, V, x0)
        scale = np.abs(ref).max()
        np.testing.assert_allclose(y, ref, rtol=0, atol=1e-12 * scale)
        assert y[trim] == 0.0


@pytest.mark.parametrize("name", list(graphs().keys()))
@pytest.mark.parametrize("lanes", LANES)
def test_operator_fp32_within_rounding_bound(isira, name, lanes):
    g = graphs()[name]
    rp, ci = dev_graph(g)
    rng = np.random.default_rng(7)
    with isira.Solver(rp, ci, precision=isira.ISIRA_MIXED, spmv_lanes=lanes) as s:
        st = s.stats()
        trim, delta = st["trim_index"], st["delta"]
        sigma, c = 0.3, 2
        x = rng.standard_normal(g.n).astype(np.float32).astype(np.float64)
        V = orthonormal_columns(g.n, c, 11).astype(np.float32).astype(np.float64)
        y = s.apply_operator(torch.from_numpy(x).float().cuda(), sigma=sigma,
                             V=torch.from_numpy(V).cuda()).cpu().numpy().astype(np.float64)
        x[trim] = 0.0
        ref = _oracle_op(g, trim, sigma, delta, V, x)
        deg = g.degrees.astype(np.float64)
        # first-order FP32 rounding bound: gamma_m * (sum of |terms| of the row), m = deg + c + 6, plus the
        # rounding of the two global reductions (1^T x and V^T x), bounded by n * 2^-24 times their magnitude
        local = (deg + abs(sigma)) * np.abs(x) + abs_adjacency_apply(g, x) + abs(sigma) / g.n * np.abs(x).sum() \
            + delta * np.abs(V) @ np.abs(V.T @ x)
        glob = (abs(sigma) / g.n * np.abs(x).sum() + delta * np.abs(V) @ (np.abs(V).T @ np.abs(x))) * g.n * 2.0 ** -24
        gam = (deg + c + 6) * 2.0 ** -24
        mag = gam * local + glob
        err = np.abs(y - ref)
        assert np.all(err <= 2 * mag + 1e-30), float(np.max(err / (mag + 1e-300)))


@pytest.mark.parametrize("name", ["rmat12", "star5000", "grid31x33"])
@pytest.mark.parametrize("dtype", ["fp32", "fp64"])
@pytest.mark.parametrize("index_vec", [0, 1])
def test_operator_independent_of_gather_launch_shape(isira, name, dtype, index_vec):
    """The gather's summation order is fixed by the row and its work items, not by the launch
    shape: 256- and 1024-thread CTAs, dynamic or static work distribution, with the hub block of
    x staged in shared memory by a bulk copy (whole vector, a part of it) or not at all, give
    bit-identical operator values."""
    g = graphs()[name]
    rp, ci = dev_graph(g)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(g.n)
    V = orthonormal_columns(g.n, 2, 9)
    tx = torch.from_numpy(x).cuda()
    tV = torch.from_numpy(V).cuda()
    if dtype == "fp32":
        tx = tx.float()                 # the deflation vectors stay float64 (the C ABI's type)
    prec = isira.ISIRA_MIXED if dtype == "fp32" else isira.ISIRA_FP64
    outs = []
    for block, hub, sched in [(256, -1, 1), (256, 16, 0), (1024, -1, 0), (1024, 1, 1), (1024, 0, 0), (256, 0, 1)]:
        with isira.Solver(rp, ci, precision=prec, spmv_lanes=2, gather_block=block, hub_kb=hub, gather_sched=sched,
                          index_vec=index_vec) as s:
            st = s.stats()
            assert st["gather_block"] == block
            assert (st["hub_bytes"] > 0) == (hub >= 0)
            outs.append(s.apply_operator(tx, sigma=0.3, V=tV).cpu().numpy())
            # a second launch on the same handle: the work counter was reset by the first
            np.testing.assert_array_equal(s.apply_operator(tx, sigma=0.3, V=tV).cpu().numpy(), outs[-1])
            assert s.stats()["hub_timeouts"] == 0
    for y in outs[1:]:
        np.testing.assert_array_equal(y, outs[0])


@pytest.mark.parametrize("k", [1, 2, 3, 7, 17, 30, 50, 64])
def test_sym_eig_matches_oracle_and_lapack(isira, k):
    rng = np.random.default_rng(100 + k)
    B = rng.standard_normal((k, k))
    A = B + B.T
    th, S = isira.sym_eig(torch.from_numpy(A).cuda())
    th, S = th.cpu().numpy(), S.cpu().numpy()
    th_or, S_or, _ = oracle.sym_eig(A)
    scale = max(1.0, np.abs(th_or).max())
    np.testing.assert_allclose(th, th_or, atol=1e-13 * scale * k)
    np.testing.assert_allclose(th, np.linalg.eigvalsh(A), atol=1e-13 * scale * k)
    np.testing.assert_allclose(A @ S, S * th[None, :], atol=1e-12 * scale * k)
    np.testing.assert_allclose(S.T @ S, np.eye(k), atol=1e-13 * k)
    # simple spectrum here: eigenvectors are unique up to sign, and the sign rule fixes it
    np.testing.assert_allclose(S, S_or, atol=1e-10 * k)


def test_sym_eig_degenerate_and_diagonal(isira):
    D = np.diag([3.0, -1.0, 2.0, 2.0, 0.0])
    th, S = isira.sym_eig(torch.from_numpy(D).cuda())
    np.testing.assert_array_equal(th.cpu().numpy(), [-1.0, 0.0, 2.0, 2.0, 3.0])
    k = 12
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    lam = np.array([1.0] * 5 + [2.0] * 4 + [5.0, 6.0, 7.0])
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    th, S = isira.sym_eig(torch.from_numpy(A).cuda())
    th, S = th.cpu().numpy(), S.cpu().numpy()
    np.testing.assert_allclose(th, lam, atol=1e-13 * 7 * k)
    np.testing.assert_allclose(A @ S, S * th[None, :], atol=1e-12 * k)
    np.testing.assert_allclose(S.T @ S, np.eye(k), atol=1e-13 * k)


def _warm_case(k, kind, rng):
    """A symmetric k x k H and orthonormal eigenvectors Q0 of its leading w x w block (w = k - 1, or k
    for kind 'diag'), shaped to exercise each deflation of the arrowhead path."""
    w = k if kind == "diag" else k - 1
    B = rng.standard_normal((k, k))
    H = B + B.T
    if kind == "repeated":            # H0 with eigenvalues of multiplicity > 1 (rotation deflation)
        Q, _ = np.linalg.qr(rng.standard_normal((w, w)))
        lam0 = np.round(rng.standard_normal(w) * 2.0) / 2.0
        H0 = (Q * lam0) @ Q.T
        H[:w, :w] = 0.5 * (H0 + H0.T)
    th0, Q0, _ = oracle.sym_eig(H[:w, :w])
    if kind == "orthogonal" and w >= 2:   # new column orthogonal to half of Q0 (z_i = 0 deflation)
        col = Q0[:, : w // 2] @ rng.standard_normal(w // 2)
        H[:w, w] = col
        H[w, :w] = col
    if kind == "zero":                # new column zero: alpha is an eigenvalue as it stands
        H[:w, w] = 0.0
        H[w, :w] = 0.0
    return H, Q0


@pytest.mark.parametrize("k", [2, 3, 7, 17, 30, 50, 64])
@pytest.mark.parametrize("kind", ["plain", "repeated", "orthogonal", "zero", "diag"])
def test_sym_eig_warm_arrowhead_matches_oracle(isira, k, kind):
    """Rayleigh-Ritz after one expansion (secular equation of the arrowhead matrix, Gu-Eisenstat
    vectors) against the oracle's Jacobi eigensolver and LAPACK."""
    rng = np.random.default_rng(1000 * k + len(kind))
    H, Q0 = _warm_case(k, kind, rng)
    th, S, path = isira.sym_eig_warm(torch.from_numpy(H).cuda(), torch.from_numpy(Q0).cuda())
    th, S = th.cpu().numpy(), S.cpu().numpy()
    assert path == 1
    th_or, S_or, _ = oracle.sym_eig(H)
    scale = max(1.0, np.abs(th_or).max())
    np.testing.assert_allclose(th, th_or, atol=1e-13 * scale * k)
    np.testing.assert_allclose(th, np.linalg.eigvalsh(H), atol=1e-13 * scale * k)
    np.testing.assert_allclose(H @ S, S * th[None, :], atol=1e-12 * scale * k)
    np.testing.assert_allclose(S.T @ S, np.eye(k), atol=1e-13 * k)
    gaps = np.diff(th_or)
    if kind == "plain" and gaps.min() > 1e-6 * scale:    # simple spectrum: unique up to the sign rule
        np.testing.assert_allclose(S, S_or, atol=1e-9 * k)


def test_sym_eig_warm_refuses_a_basis_that_does_not_diagonalise(isira):
    rng = np.random.default_rng(7)
    k = 20
    B = rng.standard_normal((k, k))
    H = B + B.T
    Q0, _ = np.linalg.qr(rng.standard_normal((k - 1, k - 1)))     # orthonormal, not eigenvectors
    th, S, path = isira.sym_eig_warm(torch.from_numpy(H).cuda(), torch.from_numpy(Q0).cuda())
    th, S = th.cpu().numpy(), S.cpu().numpy()
    assert path == 0
    th_or, _, _ = oracle.sym_eig(H)
    np.testing.assert_allclose(th, th_or, atol=1e-13 * np.abs(th_or).max() * k)
    np.testing.assert_allclose(S.T @ S, np.eye(k), atol=1e-13 * k)


@pytest.mark.parametrize("name", ["grid31x33", "rmat12", "er3000"])
@pytest.mark.parametrize("sigma,c,reorder", [(0.0, 0, 0), (0.15, 2, 0), (0.15, 2, 1)])
def test_inner_solve_fp64_matches_oracle(isira, name, sigma, c, reorder):
    g = graphs()[name]
    rp, ci = dev_graph(g)
    with isira.Solver(rp, ci, precision=isira.ISIRA_FP64, reorder=reorder) as s:
        st = s.stats()
        trim, delta = st["trim_index"], st["delta"]
        rng = np.random.default_rng(1)
        r = rng.standard_normal(g.n)
        r -= r.mean()
        V = orthonormal_columns(g.n, c, 5) if c else None
        z, its, rel = s.inner_solve(torch.from_numpy(r).cuda(), sigma=sigma,
                                    V=torch.from_numpy(V).cuda() if c else None, tau=1e-11, max_it=20000,
                                    precision=isira.ISIRA_FP64)
        z = z.cpu().numpy()
        zr, its_or, rel_or = oracle.inner_solve(g.row_ptr, g.col_idx, trim, sigma, delta, V, r, tau=1e-12,
                                                max_it=40000)
        assert rel <= 1e-11 and its > 0
        assert abs(z.sum()) <= 1e-10 * np.abs(z).sum()
        np.testing.assert_allclose(z, zr, atol=1e-8 * np.abs(zr).max())


@pytest.mark.parametrize("name", ["grid31x33", "rmat12", "star5000"])
def test_inner_solve_mixed_reaches_tau(isira, name):
    g = graphs()[name]
    rp, ci = dev_graph(g)
    with isira.Solver(rp, ci, precision=isira.ISIRA_MIXED) as s:
        st = s.stats()
        trim, delta = st["trim_index"], st["delta"]
        rng = np.random.default_rng(2)
        r = rng.standard_normal(g.n)
        r -= r.mean()
        tau = 1e-3
        z, its, rel = s.inner_solve(torch.from_numpy(r).cuda(), sigma=0.0, tau=tau, max_it=5000,
                                    precision=isira.ISIRA_MIXED)
        z = z.cpu().numpy()
        assert rel <= tau
        assert abs(z.sum()) <= 1e-6 * np.abs(z).sum()
        # the back-mapped vector solves the singular system L z = r (Thm 2.4) to the inner accuracy,
        # measured in the 2-norm: the preconditioned criterion loses at most sqrt(cond(D)), and the true
        # residual of an FP32 MINRES solve separates from its recursive estimate by a few tens of
        # u * cond(Lh) (rounding in the three-term w recurrence)
        Lz = oracle.laplacian_apply(g.row_ptr, g.col_idx, z)
        deg = g.degrees.astype(float)
        import scipy.sparse as sp
        from scipy.sparse.linalg import eigsh
        A = sp.csr_matrix((np.ones(g.nnz), g.col_idx, g.row_ptr), shape=(g.n, g.n))
        Lh = (sp.diags(deg) - A).tocsr()
        keep = np.delete(np.arange(g.n), trim)
        Lh = Lh[keep][:, keep]
        lmax = eigsh(Lh, k=1, which="LA", return_eigenvectors=False)[0]
        lmin = eigsh(Lh, k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
        bound = 4 * tau * np.sqrt(deg.max() / deg.min()) + 30 * 2.0 ** -24 * lmax / lmin
        assert np.linalg.norm(Lz - r) <= bound * np.linalg.norm(r)
