"""The GPU-oriented random geometric graph generator (cell lists, torch) builds exactly the graph
of the k-d-tree reference generator: same points, same pairs, same component and labels.  Run
with torch on the CPU here; the benchmark runs the same code on the GPU."""
import numpy as np
import pytest

import synthgraphs as sg

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("n", [2000, 20000])
def test_rgg_cell_list_matches_kdtree(n):
    g = sg.rgg(n, 12.0, seed=1)
    rp, ci = sg.rgg_gpu(n, 12.0, seed=1, device="cpu")
    np.testing.assert_array_equal(rp.numpy(), g.row_ptr)
    np.testing.assert_array_equal(ci.numpy(), g.col_idx)
    assert abs(g.nnz / g.n - 12.0) < 1.0           # mean degree near the target (boundary loses a little)
