"""The aggregation multilevel preconditioner (opts.precond = 1, standing in for the combinatorial
multigrid of the paper's Sec. 3.2): one V-cycle is a symmetric positive definite operator, it is
spectrally much closer to the trimmed Laplacian (Theorem 2.3) than the diagonal, the inner solve
with it reaches the oracle's solution of the trimmed, shifted, deflated system (Theorem 2.6), and
whole solves give the same eigenpairs as closed forms and the oracle."""
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
            "grid3d_20": sg.grid3d(20, 20, 20)}


def _trimmed_laplacian(g, trim):
    import scipy.sparse as sp
    A = sp.csr_matrix((np.ones(g.nnz), g.col_idx, g.row_ptr), shape=(g.n, g.n))
    L = (sp.diags(g.degrees.astype(float)) - A).tocsr()
    keep = np.delete(np.arange(g.n), trim)
    return L[keep][:, keep], keep


@pytest.mark.parametrize("name", list(graphs().keys()))
def test_vcycle_is_symmetric_positive_definite(isira, name):
    g = graphs()[name]
    rp, ci = dev_graph(g)
    with isira.Solver(rp, ci, precision=isira.ISIRA_FP64, precond=1) as s:
        trim = s.stats()["trim_index"]
        rng = np.random.default_rng(3)
        X = rng.standard_normal((g.n, 4))
        X[trim] = 0.0
        Y = []
        for j in range(4):
            y, levels, nc = s.precond_apply(torch.from_numpy(X[:, j].copy()).cuda())
            Y.append(y.cpu().numpy())
        Y = np.stack(Y, axis=1)
        assert levels >= (1 if g.n <= 512 else 2) and nc <= 512
        assert np.all(Y[trim] == 0.0)
        G = X.T @ Y
        np.testing.assert_allclose(G, G.T, rtol=0, atol=1e-12 * np.abs(G).max())
        assert np.all(np.linalg.eigvalsh(0.5 * (G + G.T)) > 0)
        # mixed precision: the same operator within FP32 rounding
        yf, _, _ = s.precond_apply(torch.from_numpy(X[:, 0].copy()).float().cuda())
        np.testing.assert_allclose(yf.double().cpu().numpy(), Y[:, 0], rtol=0, atol=1e-4 * np.abs(Y[:, 0]).max())


@pytest.mark.parametrize("g", [sg.grid2d(31, 33), sg.grid3d(10, 11, 12), sg.erdos_renyi(1200, 8.0, seed=4)],
                         ids=["grid31x33", "grid10x11x12", "er1200"])
def test_vcycle_is_spectrally_close_to_the_trimmed_laplacian(isira, g):
    """kappa(M^{-1} Lh) of the V-cycle (M^{-1} formed column by column on the GPU, then the dense
    generalized eigenproblem), against kappa(D^{-1} Lh) of the diagonal preconditioner."""
    import scipy.linalg as sl
    rp, ci = dev_graph(g)
    with isira.Solver(rp, ci, precision=isira.ISIRA_FP64, precond=1) as s:
        trim = s.stats()["trim_index"]
        Lh, keep = _trimmed_laplacian(g, trim)
        Lh = Lh.toarray()
        m = Lh.shape[0]
        B = np.empty((m, m))
        for j in range(m):
            x = np.zeros(g.n)
            x[keep[j]] = 1.0
            B[:, j] = s.precond_apply(torch.from_numpy(x).cuda())[0].cpu().numpy()[keep]
    B = 0.5 * (B + B.T)                      # M^{-1} (symmetric to rounding)
    assert np.linalg.eigvalsh(B).min() > 0
    ev = sl.eigh(Lh, np.linalg.inv(B), eigvals_only=True)      # spectrum of M^{-1} Lh
    kappa_ml = ev.max() / ev.min()
    d = np.diag(Lh)
    evj = sl.eigh(Lh, np.diag(d), eigvals_only=True)
    kappa_j = evj.max() / evj.min()
    assert kappa_ml < 0.2 * kappa_j, (kappa_ml, kappa_j)


@pytest.mark.parametrize("name", ["grid31x33", "rmat12", "er3000"])
@pytest.mark.parametrize("sigma,c", [(0.0, 0), (0.15, 2)])
def test_inner_solve_multilevel_fp64_matches_oracle(isira, name, sigma, c):
    g = graphs()[name]
    rp, ci = dev_graph(g)
    with isira.Solver(rp, ci, precision=isira.ISIRA_FP64, precond=1) as s:
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
        zr, _, _ = oracle.inner_solve(g.row_ptr, g.col_idx, trim, sigma, delta, V, r, tau=1e-12, max_it=40000)
        assert rel <= 1e-11 and its > 0
        np.testing.assert_allclose(z, zr, atol=1e-8 * np.abs(zr).max())


def test_inner_iterations_drop_on_a_3d_grid(isira):
    g = sg.grid3d(32, 32, 32)
    rp, ci = dev_graph(g)
    rng = np.random.default_rng(2)
    r = rng.standard_normal(g.n)
    r -= r.mean()
    its = {}
    for pc in (0, 1):
        with isira.Solver(rp, ci, precision=isira.ISIRA_MIXED, precond=pc) as s:
            _, its[pc], rel = s.inner_solve(torch.from_numpy(r).cuda(), sigma=0.0, tau=1e-3, max_it=5000,
                                            precision=isira.ISIRA_MIXED)
            assert rel <= 1e-3
    assert its[1] * 4 <= its[0], its


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_with_multilevel_matches_closed_form_and_oracle(isira, prec):
    from tests.test_gpu_solve import check_pairs, run
    g = sg.grid2d(40, 37)
    res = run(isira, g, 6, prec, tol=1e-10, precond=1)
    assert res.status == isira.ISIRA_OK
    lam, _ = check_pairs(g, res, 6)
    np.testing.assert_allclose(lam, cf.grid2d(40, 37)[1:7], rtol=1e-9)
    g2 = sg.rmat(12)
    res2 = run(isira, g2, 5, prec, tol=1e-10, precond=1)
    assert res2.status == isira.ISIRA_OK
    lam2, _ = check_pairs(g2, res2, 5)
    lam_or, _, st = oracle.isira(g2.row_ptr, g2.col_idx, 5, sg.start_vector(g2.n, 1), eps=1e-10, tau_inner=1e-3)
    np.testing.assert_allclose(lam2, np.sort(lam_or), rtol=1e-9)
