"""Independent witness for the oracle's full-size R-MAT scale-20 eigenvalues (no missed eigenvalue):
SciPy's ARPACK (a library eigensolver, used only as a witness) computes the 11 smallest
eigenvalues of B = L + (1/n) 1 1^T live, in shift-invert mode around 0 with conjugate-gradient
solves of B.  B is SPD with the same eigenpairs as L except that 0 (eigenvector 1) moves to 1, so
its smallest eigenvalues are the smallest positive ones of L.  No value is stored: the check
compares the live result with tests/golden (written by the oracle alone).

Slow (about ten minutes on one core): runs only with ISIRA_RUN_SLOW=1."""
import json
import os

import numpy as np
import pytest

import synthgraphs as sg

pytestmark = pytest.mark.slow

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.skipif(os.environ.get("ISIRA_RUN_SLOW") != "1", reason="slow witness: set ISIRA_RUN_SLOW=1")
def test_arpack_witness_confirms_golden_rmat20():
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla
    g = sg.rmat(20)
    gold = json.load(open(os.path.join(HERE, "golden", "rmat20_tight.json")))
    assert (g.n, g.nnz) == (gold["n"], gold["nnz"])
    n = g.n
    A = sp.csr_matrix((np.ones(g.nnz), g.col_idx, g.row_ptr), shape=(n, n))
    deg = np.asarray(A.sum(axis=1)).ravel()
    L = (sp.diags(deg) - A).tocsr()
    one = np.ones(n) / np.sqrt(n)
    B = sla.LinearOperator((n, n), matvec=lambda x: L @ x + one * (one @ x), dtype=np.float64)
    Minv = sla.LinearOperator((n, n), matvec=lambda x: x / deg, dtype=np.float64)

    def solve(x):
        y, info = sla.cg(B, x, rtol=1e-13, atol=0.0, M=Minv, maxiter=10000)
        assert info == 0
        return y

    OPinv = sla.LinearOperator((n, n), matvec=solve, dtype=np.float64)
    v0 = (np.arange(n) % 7 - 3.0)
    w = np.sort(sla.eigsh(B, k=11, sigma=0.0, which="LM", OPinv=OPinv, tol=1e-12, v0=v0,
                          return_eigenvectors=False))
    ref = np.array(gold["eigvals"])
    # the ten golden values are the ten smallest positive eigenvalues of L: none is missed
    np.testing.assert_allclose(w[:10], ref, rtol=1e-9)
    assert w[10] >= ref[-1] * (1 - 1e-9)
