"""The GPU R-MAT generator (used for the scale-24 workload) reproduces the numpy generator."""
import numpy as np
import pytest

import synthgraphs as sg
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scale", [10, 14])
def test_rmat_gpu_matches_numpy(scale):
    need_gpu()
    g = sg.rmat(scale)
    rp, ci = sg.rmat_gpu(scale)
    np.testing.assert_array_equal(rp.cpu().numpy(), g.row_ptr)
    np.testing.assert_array_equal(ci.cpu().numpy(), g.col_idx)
