"""Helpers shared by the GPU tests: move synthetic graphs to the device, numpy views."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev_graph(g, device="cuda:0"):
    return (torch.from_numpy(g.row_ptr).to(device), torch.from_numpy(g.col_idx).to(device))


def abs_adjacency_apply(g, x):
    """sum over neighbours of |x_c| for every row (a magnitude bound helper)."""
    import scipy.sparse as sp
    A = sp.csr_matrix((np.ones(g.nnz), g.col_idx, g.row_ptr), shape=(g.n, g.n))
    return A @ np.abs(x)


def orthonormal_columns(n, c, seed, exclude_ones=True):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, c + 1))
    if exclude_ones:
        M[:, 0] = 1.0
    Q, _ = np.linalg.qr(M)
    return np.ascontiguousarray(Q[:, 1:] if exclude_ones else Q[:, :c])
