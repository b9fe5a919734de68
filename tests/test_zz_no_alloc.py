"""isira_apply_operator_noalloc: the allocation-free, handle-free operator entry point, for
callers that cannot let a library allocate device memory (a pre-reserved pool with a fixed
budget, latency-critical loops where cudaMalloc/cudaFree may synchronise the device, plug-in
hosts that forbid allocations).  Checked through the C ABI against isira_apply_operator, on two
calls in a row (the static scratch keeps the first call's contents), in FP64 and FP32, and
elementwise against the FP64 oracle's trimmed operator (Theorem 2.6) on the same inputs.

This file is named so that pytest collects it last."""
import numpy as np
import pytest

import oracle
import synthgraphs as sg
from tests.gpu_util import abs_adjacency_apply, dev_graph, need_gpu, orthonormal_columns, torch

pytestmark = pytest.mark.gpu


def fp32_bound(g, x, V, sigma, delta, c):
    """First-order FP32 rounding bound of one evaluation of the operator (per row)."""
    deg = g.degrees.astype(np.float64)
    Vd = V if c else np.zeros((g.n, 0))
    local = (deg + abs(sigma)) * np.abs(x) + abs_adjacency_apply(g, x) + abs(sigma) / g.n * np.abs(x).sum() \
        + delta * np.abs(Vd) @ np.abs(Vd.T @ x)
    glob = (abs(sigma) / g.n * np.abs(x).sum() + delta * np.abs(Vd) @ (np.abs(Vd).T @ np.abs(x))) * g.n * 2.0 ** -24
    return (deg + c + 6) * 2.0 ** -24 * local + glob


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["rmat12", "grid31x33"])
def test_noalloc_matches_handle_entry_point_on_two_calls(prec, name):
    need_gpu()
    import paper_1710_07080_gb300 as isira
    g = sg.rmat(12) if name == "rmat12" else sg.grid2d(31, 33)
    rp, ci = dev_graph(g)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    with isira.Solver(rp, ci, precision=isira.ISIRA_FP64 if prec == "fp64" else isira.ISIRA_MIXED) as s:
        st = s.stats()
        trim, delta = st["trim_index"], st["delta"]
        for call, (sigma, c) in enumerate([(0.37, 3), (0.0, 0), (1.1, 8)]):
            rng = np.random.default_rng(10 + call)
            x = rng.standard_normal(g.n).astype(np.float32).astype(np.float64)
            x[trim] = 0.0            # the handle path pins x_trim to 0; give both the same input
            V = orthonormal_columns(g.n, c, 20 + call).astype(np.float32).astype(np.float64) if c else None
            xt = torch.from_numpy(x).to(dtype).cuda()
            Vt = torch.from_numpy(V).cuda() if c else None
            y_ref = s.apply_operator(xt, sigma=sigma, V=Vt).double().cpu().numpy()
            y_out = torch.full_like(xt, float("nan"))
            isira.apply_operator_noalloc(rp, ci, xt, trim, sigma, delta, Vt, y=y_out)
            torch.cuda.synchronize()
            y = y_out.double().cpu().numpy()
            # the same call again straight through the C ABI: the device's free memory does not move
            Vc = Vt.t().contiguous() if c else None
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            st2 = isira.lib.isira_apply_operator_noalloc(
                g.n, g.nnz, rp.data_ptr(), ci.data_ptr(), trim, isira.ISIRA_FP64 if prec == "fp64" else isira.ISIRA_MIXED,
                sigma, delta, 0, c, Vc.data_ptr() if c else None, xt.data_ptr(), y_out.data_ptr(), None)
            torch.cuda.synchronize()
            free1 = torch.cuda.mem_get_info()[0]
            assert st2 == isira.ISIRA_OK and free1 == free0
            np.testing.assert_array_equal(y_out.double().cpu().numpy(), y)   # deterministic
            assert y[trim] == 0.0 and np.all(np.isfinite(y))
            # the oracle's operator on the (n-1)-vector with the trimmed entry removed
            x0 = x.copy()
            x0[trim] = 0.0
            yh = oracle.trimmed_apply(g.row_ptr, g.col_idx, trim, sigma, delta, V, np.delete(x0, trim))
            y_or = np.insert(yh, trim, 0.0)
            if prec == "fp64":
                np.testing.assert_allclose(y, y_ref, rtol=0, atol=1e-12 * np.abs(y_ref).max())
                np.testing.assert_allclose(y, y_or, rtol=0, atol=1e-12 * np.abs(y_or).max())
            else:
                bound = fp32_bound(g, x, V, sigma, delta, c)
                assert np.all(np.abs(y - y_ref) <= 4 * bound + 1e-30)
                assert np.all(np.abs(y - y_or) <= 2 * bound + 1e-30)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    need_gpu()
    import paper_1710_07080_gb300 as isira
    g = sg.grid2d(8, 9)
    rp, ci = dev_graph(g)
    x = torch.randn(g.n, dtype=torch.float64, device="cuda")
    V = torch.from_numpy(orthonormal_columns(g.n, 9, 1)).cuda()
    with pytest.raises(isira.IsiraError) as e:
        isira.apply_operator_noalloc(rp, ci, x, 0, 0.1, 32.0, V)
    assert e.value.status == isira.ISIRA_ERR_LIMIT
    lib = isira.lib
    assert lib.isira_apply_operator_noalloc(g.n, g.nnz, rp.data_ptr(), ci.data_ptr(), g.n, 0, 0.0, 1.0, 0, 0,
                                            None, x.data_ptr(), x.data_ptr(), None) == isira.ISIRA_ERR_INVALID_ARG
