"""CPU-only checks of the Python binding's argument validation: every tensor is checked for dtype,
shape, layout and device before its raw pointer reaches the library (a float32 buffer passed
where the C ABI expects float64 would be read past its end)."""
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def isira():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1710_07080_gb300 as m
    return m


def _csr(n=6):
    # path graph on n vertices
    rp = torch.tensor([0] + [1] + [3 + 2 * i for i in range(n - 2)] + [2 * (n - 1)], dtype=torch.int64)
    cols = []
    for v in range(n):
        cols += [u for u in (v - 1, v + 1) if 0 <= u < n]
    return rp, torch.tensor(cols, dtype=torch.int32)


def test_noalloc_rejections(isira):
    rp, ci = _csr()
    x = torch.zeros(6, dtype=torch.float64)
    cases = [
        (dict(row_ptr=rp.int()), "row_ptr must have dtype"),
        (dict(col_idx=ci.long()), "col_idx must have dtype"),
        (dict(x=x.half()), "x must have dtype"),
        (dict(x=torch.zeros(7, dtype=torch.float64)), "x must have shape"),
        (dict(x=torch.zeros(12, dtype=torch.float64)[::2]), "x must be contiguous"),
        (dict(y=torch.zeros(6, dtype=torch.float32)), "y must have dtype"),
        (dict(y=torch.zeros(5, dtype=torch.float64)), "y must have shape"),
        (dict(V=torch.zeros(6, 2, dtype=torch.float32)), "V must have dtype"),
        (dict(V=torch.zeros(5, 2, dtype=torch.float64)), "V must have shape"),
        (dict(V=torch.zeros(6, 32, dtype=torch.float64)), "at most 31 columns"),
        (dict(), "must be a CUDA tensor"),
    ]
    for over, msg in cases:
        kw = dict(row_ptr=rp, col_idx=ci, x=x, y=None, V=None)
        kw.update(over)
        with pytest.raises(ValueError, match=msg):
            isira.apply_operator_noalloc(kw["row_ptr"], kw["col_idx"], kw["x"], trim=0, V=kw["V"], y=kw["y"])


def test_solver_and_sym_eig_rejections(isira):
    rp, ci = _csr()
    with pytest.raises(ValueError, match="row_ptr must have dtype"):
        isira.Solver(rp.int(), ci)
    with pytest.raises(ValueError, match="col_idx must have dtype"):
        isira.Solver(rp, ci.long())
    with pytest.raises(ValueError, match="must be a CUDA tensor"):
        isira.Solver(rp, ci)
    with pytest.raises(ValueError, match="must have dtype"):
        isira.sym_eig(torch.eye(3, dtype=torch.float32))
    with pytest.raises(ValueError, match="square matrix"):
        isira.sym_eig(torch.zeros(3, 4, dtype=torch.float64))
    with pytest.raises(ValueError, match="must be a CUDA tensor"):
        isira.sym_eig(torch.eye(3, dtype=torch.float64))
    with pytest.raises(ValueError, match="must be a CUDA tensor"):
        isira.Batch([(rp, ci)])


def test_vector_checks(isira):
    x = torch.zeros(4, dtype=torch.float32)
    with pytest.raises(ValueError, match="must be a CUDA tensor"):
        isira._check_x(x, 4)
    with pytest.raises(ValueError, match="shape"):
        isira._check_x(x, 5)
    with pytest.raises(ValueError, match="dtype"):
        isira._check_x(x.int(), 4)
    assert isira._check_V(None, 4) == 0


def test_sym_eig_warm_rejections(isira):
    H = torch.eye(4, dtype=torch.float64)
    with pytest.raises(ValueError, match="order 2..64"):
        isira.sym_eig_warm(torch.eye(1, dtype=torch.float64), torch.eye(1, dtype=torch.float64))
    with pytest.raises(ValueError, match="order k-1 or k"):
        isira.sym_eig_warm(H, torch.eye(2, dtype=torch.float64))
    with pytest.raises(ValueError, match="must have dtype"):
        isira.sym_eig_warm(H.float(), torch.eye(3, dtype=torch.float64))
    with pytest.raises(ValueError, match="must be a CUDA tensor"):
        isira.sym_eig_warm(H, torch.eye(3, dtype=torch.float64))


def test_abi_rejects_bad_warm_start_sizes(isira):
    lib = isira.lib
    assert lib.isira_sym_eig_warm(1, 0, None, None, None, None, None) == isira.ISIRA_ERR_INVALID_ARG
    assert lib.isira_sym_eig_warm(8, 5, 8, 8, 8, None, None) == isira.ISIRA_ERR_INVALID_ARG     # warm_w < k - 1
    assert lib.isira_sym_eig_warm(65, 64, 8, 8, 8, None, None) == isira.ISIRA_ERR_INVALID_ARG   # k > 64
    assert lib.isira_residual_history(None, None, 0, None) == isira.ISIRA_ERR_INVALID_ARG
