"""Thin Python binding of libisira (GB300 / sm_103a iSIRA eigensolver, arXiv:1710.07080).

Argument marshalling only: every step of the method runs in the CUDA kernels of
``libisira.so``.  PyTorch provides device memory and the current CUDA stream.
The C entry points keep their names (``isira_create``, ``isira_solve``, ...);
:func:`solve` is the one-call convenience wrapper.  There is no CPU fallback:
if the library is missing, importing the binding raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libisira.so")

ISIRA_OK = 0
ISIRA_ERR_INVALID_ARG = 1
ISIRA_ERR_BAD_GRAPH = 2
ISIRA_ERR_NOT_CONNECTED = 3
ISIRA_ERR_NO_CONVERGENCE = 4
ISIRA_ERR_CUDA = 5
ISIRA_ERR_OOM = 6
ISIRA_ERR_NOT_SOLVED = 7
ISIRA_ERR_LIMIT = 8
ISIRA_ERR_DEVICE_TIMEOUT = 9

ISIRA_FP64 = 0
ISIRA_MIXED = 1

EXPORTED = ["isira_default_opts", "isira_error_string", "isira_create", "isira_create_weighted", "isira_solve",
            "isira_eigpairs",
            "isira_get_stats", "isira_set_profiling", "isira_destroy", "isira_apply_operator",
            "isira_inner_solve", "isira_sym_eig", "isira_sym_eig_warm", "isira_residual_history", "isira_apply_operator_noalloc", "isira_batch_create",
            "isira_precond_apply",
            "isira_batch_solve", "isira_batch_status", "isira_batch_eigpairs", "isira_batch_get_stats",
            "isira_batch_destroy"]


class isira_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("m", C.c_int), ("q", C.c_int), ("tau_inner", C.c_double),
                ("max_inner", C.c_int), ("max_outer", C.c_int), ("trim_index", C.c_int64), ("delta", C.c_double),
                ("sigma_omega", C.c_double), ("drop_rank1", C.c_int), ("validate", C.c_int), ("seed", C.c_uint64),
                ("spmv_lanes", C.c_int), ("inner_chunk", C.c_int), ("inner_graph", C.c_int),
                ("reorder", C.c_int), ("gather_block", C.c_int), ("hub_kb", C.c_int),
                ("gather_sched", C.c_int), ("index_vec", C.c_int), ("gather_chunk", C.c_int), ("sell", C.c_int),
                ("precond", C.c_int), ("ml_alpha", C.c_double), ("rr_arrow", C.c_int),
                ("blocking_sync", C.c_int)]


class isira_stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("trim_index", C.c_int64), ("max_degree", C.c_int64),
                ("delta", C.c_double), ("norm_L", C.c_double), ("spmv_lanes", C.c_int),
                ("n_long_rows", C.c_int64), ("n_work_items", C.c_int64), ("n_locked", C.c_int),
                ("outer_steps", C.c_int), ("restarts", C.c_int), ("breakdowns", C.c_int),
                ("inner_iters", C.c_longlong), ("inner_solves", C.c_longlong), ("spmv_launches", C.c_longlong),
                ("solve_ms", C.c_double), ("inner_phase1_ms", C.c_double), ("inner_phase1_timed", C.c_longlong),
                ("inner_phase1_csum", C.c_longlong), ("kernel_launches", C.c_longlong),
                ("gather_block", C.c_int), ("hub_bytes", C.c_int), ("hub_timeouts", C.c_longlong),
                ("inner_rows_ms", C.c_double), ("inner_phase2_ms", C.c_double), ("w_columns", C.c_longlong),
                ("sell_entries", C.c_longlong), ("max_diag", C.c_double), ("precond", C.c_int),
                ("ml_levels", C.c_int), ("precond_probe_ms", C.c_double * 2), ("rr_arrow", C.c_int),
                ("rr_jacobi", C.c_int), ("rr_refused", C.c_int), ("ml_coarse_n", C.c_longlong),
                ("ml_coarse_nnz", C.c_longlong)]

    def as_dict(self) -> dict:
        out = {}
        for f, _ in self._fields_:
            v = getattr(self, f)
            out[f] = list(v) if hasattr(v, "__len__") else v
        return out


def _load() -> C.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libisira.so is not built ({LIB_PATH}); run __graft_entry__.build() or "
                          "python paper_1710_07080_gb300/_build.py")
    lib = C.CDLL(LIB_PATH)
    P, I, D, I64 = C.c_void_p, C.c_int, C.c_double, C.c_int64
    lib.isira_default_opts.argtypes = [C.POINTER(isira_opts)]
    lib.isira_default_opts.restype = None
    lib.isira_error_string.argtypes = [I]
    lib.isira_error_string.restype = C.c_char_p
    lib.isira_create.argtypes = [C.POINTER(P), I64, I64, P, P, C.POINTER(isira_opts), P]
    lib.isira_create.restype = I
    lib.isira_create_weighted.argtypes = [C.POINTER(P), I64, I64, P, P, P, C.POINTER(isira_opts), P]
    lib.isira_create_weighted.restype = I
    lib.isira_solve.argtypes = [P, I, D, D, P]
    lib.isira_solve.restype = I
    lib.isira_eigpairs.argtypes = [P, P, P, P, C.POINTER(I)]
    lib.isira_eigpairs.restype = I
    lib.isira_get_stats.argtypes = [P, C.POINTER(isira_stats)]
    lib.isira_get_stats.restype = I
    lib.isira_set_profiling.argtypes = [P, I]
    lib.isira_set_profiling.restype = I
    lib.isira_destroy.argtypes = [P]
    lib.isira_destroy.restype = None
    lib.isira_apply_operator.argtypes = [P, I, D, I, P, P, P]
    lib.isira_apply_operator.restype = I
    lib.isira_inner_solve.argtypes = [P, I, D, I, P, P, D, I, P, C.POINTER(I), C.POINTER(D)]
    lib.isira_inner_solve.restype = I
    lib.isira_precond_apply.argtypes = [P, I, P, P, C.POINTER(I), C.POINTER(I64)]
    lib.isira_precond_apply.restype = I
    lib.isira_sym_eig.argtypes = [I, P, P, P, P]
    lib.isira_sym_eig.restype = I
    lib.isira_sym_eig_warm.argtypes = [I, I, P, P, P, C.POINTER(C.c_int), P]
    lib.isira_sym_eig_warm.restype = I
    lib.isira_residual_history.argtypes = [P, P, I, C.POINTER(C.c_int)]
    lib.isira_residual_history.restype = I
    lib.isira_apply_operator_noalloc.argtypes = [I64, I64, P, P, I64, I, D, D, I, I, P, P, P, P]
    lib.isira_apply_operator_noalloc.restype = I
    lib.isira_batch_create.argtypes = [C.POINTER(P), I, P, P, P, P, C.POINTER(isira_opts)]
    lib.isira_batch_create.restype = I
    lib.isira_batch_solve.argtypes = [P, I, D, D, I]
    lib.isira_batch_solve.restype = I
    lib.isira_batch_status.argtypes = [P, I]
    lib.isira_batch_status.restype = I
    lib.isira_batch_eigpairs.argtypes = [P, I, P, P, P, C.POINTER(I)]
    lib.isira_batch_eigpairs.restype = I
    lib.isira_batch_get_stats.argtypes = [P, I, C.POINTER(isira_stats)]
    lib.isira_batch_get_stats.restype = I
    lib.isira_batch_destroy.argtypes = [P]
    lib.isira_batch_destroy.restype = None
    return lib


lib = _load()


class IsiraError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {lib.isira_error_string(status).decode()} (status {status})")


def check(status: int, where: str) -> int:
    if status != ISIRA_OK:
        raise IsiraError(status, where)
    return status


def default_opts(**kw) -> isira_opts:
    o = isira_opts()
    lib.isira_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k!r}")
        setattr(o, k, v)
    return o


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


# ------------------------------------------------------------------ argument checks
# Every tensor handed to the library is checked here first (dtype, shape, layout, then device):
# the C entry points take raw pointers and cannot tell a float32 buffer from a float64 one.

def _check_tensor(t, name: str, dtypes: tuple, shape: tuple, cuda: bool = True):
    """Raises ValueError unless t has one of `dtypes`, exactly `shape` (None = any extent in that
    dimension), is contiguous and (with cuda) lives on a CUDA device."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name} must be a torch.Tensor")
    if t.dtype not in dtypes:
        raise ValueError(f"{name} must have dtype {' or '.join(str(d) for d in dtypes)}, not {t.dtype}")
    if t.dim() != len(shape) or any(want is not None and got != want for got, want in zip(t.shape, shape)):
        raise ValueError(f"{name} must have shape {tuple('*' if w is None else w for w in shape)}, "
                         f"not {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if cuda:
        _check_cuda(**{name: t})


def _check_cuda(**tensors):
    """Raises ValueError unless every given tensor (None skipped) is on one and the same CUDA device."""
    dev = None
    for name, t in tensors.items():
        if t is None:
            continue
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if dev is not None and t.device != dev:
            raise ValueError(f"{name} must be on the same device as the other arguments")
        dev = t.device


def _check_csr(row_ptr, col_idx, cuda: bool = True):
    import torch
    _check_tensor(row_ptr, "row_ptr", (torch.int64,), (None,), cuda=False)
    _check_tensor(col_idx, "col_idx", (torch.int32,), (None,), cuda=False)
    if row_ptr.numel() < 2:
        raise ValueError("row_ptr must have n + 1 >= 2 entries")
    if cuda:
        _check_cuda(row_ptr=row_ptr, col_idx=col_idx)


def _check_x(x, n: int, name: str = "x", cuda: bool = True):
    """An operator input: float32 (ISIRA_MIXED) or float64 (ISIRA_FP64) n-vector; returns the precision."""
    import torch
    _check_tensor(x, name, (torch.float32, torch.float64), (n,), cuda=cuda)
    return ISIRA_MIXED if x.dtype == torch.float32 else ISIRA_FP64


def _check_y(y, x, name: str = "y", cuda: bool = True):
    _check_tensor(y, name, (x.dtype,), (x.numel(),), cuda=cuda)


def _check_V(V, n: int, cmax: int = 31, cuda: bool = True):
    """Deflation vectors: float64 n-by-c with c <= cmax (None = no deflation)."""
    import torch
    if V is None:
        return 0
    _check_tensor(V.contiguous() if isinstance(V, torch.Tensor) else V, "V", (torch.float64,), (n, None),
                  cuda=cuda)
    if V.shape[1] > cmax:
        raise ValueError(f"V may have at most {cmax} columns, not {V.shape[1]}")
    return int(V.shape[1])


def _stream_ptr(stream=None) -> int | None:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


@dataclass
class Result:
    eigvals: "object"        # torch.float64 [k] on the CPU, ascending
    eigvecs: "object"        # torch.float64 [n, k] on the GPU
    true_resid: "object"     # torch.float64 [k]: ||L v - lambda v|| / (2 max degree)
    stats: dict
    status: int


class Solver:
    """Owns an isira handle for one graph (CSR on the GPU, kept alive by this object)."""

    def __init__(self, row_ptr, col_idx, stream=None, weights=None, **opts):
        """weights: optional float64 CUDA tensor [nnz] of positive, symmetric edge weights (the
        weighted Laplacian, isira_create_weighted)."""
        import torch
        _check_csr(row_ptr, col_idx, cuda=False)
        if weights is not None:
            _check_tensor(weights, "weights", (torch.float64,), (col_idx.numel(),), cuda=False)
        _check_cuda(row_ptr=row_ptr, col_idx=col_idx, weights=weights)
        self.row_ptr = row_ptr
        self.col_idx = col_idx
        self.weights = weights
        self.n = self.row_ptr.numel() - 1
        self.nnz = self.col_idx.numel()
        self.opts = default_opts(**opts)
        self.stream = _stream_ptr(stream)
        h = C.c_void_p()
        if weights is None:
            check(lib.isira_create(C.byref(h), self.n, self.nnz, _ptr(self.row_ptr), _ptr(self.col_idx),
                                   C.byref(self.opts), self.stream), "isira_create")
        else:
            check(lib.isira_create_weighted(C.byref(h), self.n, self.nnz, _ptr(self.row_ptr), _ptr(self.col_idx),
                                            _ptr(weights), C.byref(self.opts), self.stream), "isira_create_weighted")
        self.h = h
        self._last_status = None

    def close(self):
        if getattr(self, "h", None):
            lib.isira_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def stats(self) -> dict:
        st = isira_stats()
        check(lib.isira_get_stats(self.h, C.byref(st)), "isira_get_stats")
        return st.as_dict()

    def set_profiling(self, on: bool):
        check(lib.isira_set_profiling(self.h, int(bool(on))), "isira_set_profiling")

    def residual_history(self) -> list:
        """||r||_2 of the Ritz pair at every outer step of the last solve (isira_residual_history)."""
        cnt = C.c_int(0)
        check(lib.isira_residual_history(self.h, None, 0, C.byref(cnt)), "isira_residual_history")
        buf = (C.c_double * max(1, cnt.value))()
        check(lib.isira_residual_history(self.h, buf, cnt.value, C.byref(cnt)), "isira_residual_history")
        return list(buf[:cnt.value])

    def solve(self, k: int, sigma: float = 0.0, tol: float | None = None, u0=None, rel_tol: float = 1e-8,
              raise_on_error: bool = True) -> int:
        """Algorithm 2.  tol: absolute bound on ||r||_2 (the paper's epsilon); default rel_tol * 2 max degree."""
        if tol is None:
            tol = rel_tol * self.stats()["norm_L"]
        if u0 is not None:
            import torch
            _check_tensor(u0, "u0", (torch.float64,), (self.n,))
        st = lib.isira_solve(self.h, int(k), float(sigma), float(tol), _ptr(u0))
        self._last_status = st
        if raise_on_error and st not in (ISIRA_OK,):
            raise IsiraError(st, "isira_solve")
        return st

    def eigpairs(self, want_vectors: bool = True, want_resid: bool = True):
        import torch
        st = self.stats()
        k = st["n_locked"]
        if k == 0 and self._last_status == ISIRA_ERR_NO_CONVERGENCE:
            empty = torch.empty(0, dtype=torch.float64)
            vec = torch.empty((self.n, 0), dtype=torch.float64, device=self.row_ptr.device)
            return empty, (vec if want_vectors else None), (empty if want_resid else None)
        lam = torch.empty(k, dtype=torch.float64)
        vec = torch.empty((k, self.n), dtype=torch.float64, device=self.row_ptr.device) if want_vectors else None
        res = torch.empty(k, dtype=torch.float64) if want_resid else None
        nout = C.c_int(0)
        check(lib.isira_eigpairs(self.h, _ptr(lam), _ptr(vec), _ptr(res), C.byref(nout)), "isira_eigpairs")
        return lam, (vec.t() if vec is not None else None), res

    def apply_operator(self, x, sigma: float = 0.0, V=None):
        """y = trimmed, shifted, deflated operator (Eq. 2.14) applied in n-space."""
        import torch
        prec = _check_x(x, self.n)
        c = _check_V(V, self.n)
        y = torch.empty_like(x)
        Vc = None if V is None else V.t().contiguous()   # column-major n-by-c
        check(lib.isira_apply_operator(self.h, prec, float(sigma), c, _ptr(Vc), _ptr(x), _ptr(y)),
              "isira_apply_operator")
        return y

    def precond_apply(self, x):
        """y = M^{-1} x, one V-cycle of the multilevel preconditioner (isira_precond_apply); returns
        (y, levels, coarsest size)."""
        import torch
        prec = _check_x(x, self.n, cuda=False)
        _check_cuda(x=x, row_ptr=self.row_ptr)
        y = torch.empty_like(x)
        lv = C.c_int(0)
        nc = C.c_int64(0)
        check(lib.isira_precond_apply(self.h, prec, _ptr(x), _ptr(y), C.byref(lv), C.byref(nc)),
              "isira_precond_apply")
        return y, lv.value, nc.value

    def inner_solve(self, r, sigma: float = 0.0, V=None, tau: float = 1e-3, max_it: int = 5000,
                    precision: int = ISIRA_MIXED):
        import torch
        _check_tensor(r, "r", (torch.float64,), (self.n,), cuda=False)
        c = _check_V(V, self.n, cuda=False)
        _check_cuda(r=r, V=V, row_ptr=self.row_ptr)
        z = torch.empty_like(r)
        Vc = None if V is None else V.t().contiguous()
        its = C.c_int(0)
        rel = C.c_double(0.0)
        check(lib.isira_inner_solve(self.h, precision, float(sigma), c, _ptr(Vc), _ptr(r), float(tau),
                                    int(max_it), _ptr(z), C.byref(its), C.byref(rel)), "isira_inner_solve")
        return z, its.value, rel.value


def sym_eig(H):
    """All eigenpairs of a symmetric k-by-k CUDA float64 matrix on the GPU (k <= 64)."""
    import torch
    if not isinstance(H, torch.Tensor) or H.dim() != 2 or H.shape[0] != H.shape[1] or not 1 <= H.shape[0] <= 64:
        raise ValueError("H must be a square matrix of order 1..64")
    _check_tensor(H.contiguous(), "H", (torch.float64,), (H.shape[0], H.shape[0]))   # includes the device
    k = H.shape[0]
    Hc = H.t().contiguous()          # column-major
    th = torch.empty(k, dtype=torch.float64, device=H.device)
    S = torch.empty((k, k), dtype=torch.float64, device=H.device)
    check(lib.isira_sym_eig(k, _ptr(Hc), _ptr(th), _ptr(S), _stream_ptr()), "isira_sym_eig")
    return th, S.t()                 # S was written column-major


def sym_eig_warm(H, S0):
    """Rayleigh-Ritz after one expansion (see isira_sym_eig_warm in include/isira.h): H is a symmetric
    k-by-k CUDA float64 matrix (2 <= k <= 64) and S0 a w-by-w matrix (w = k - 1 or k) of orthonormal
    eigenvectors of H[:w, :w].  Returns (theta, S, path), path 1 = arrowhead, 0 = Jacobi."""
    import torch
    if not isinstance(H, torch.Tensor) or H.dim() != 2 or H.shape[0] != H.shape[1] or not 2 <= H.shape[0] <= 64:
        raise ValueError("H must be a square matrix of order 2..64")
    k = H.shape[0]
    if not isinstance(S0, torch.Tensor) or S0.dim() != 2 or S0.shape[0] != S0.shape[1] or S0.shape[0] not in (k - 1, k):
        raise ValueError("S0 must be square of order k-1 or k")
    _check_tensor(H.contiguous(), "H", (torch.float64,), (k, k))
    _check_tensor(S0.contiguous(), "S0", (torch.float64,), tuple(S0.shape))
    _check_cuda(H=H, S0=S0)
    w = S0.shape[0]
    Hc = H.t().contiguous()
    S = torch.zeros((k, k), dtype=torch.float64, device=H.device)
    S[:w, :w] = S0.t()                    # column-major, ld k
    th = torch.empty(k, dtype=torch.float64, device=H.device)
    path = C.c_int(-1)
    check(lib.isira_sym_eig_warm(k, w, _ptr(Hc), _ptr(th), _ptr(S), C.byref(path), _stream_ptr()),
          "isira_sym_eig_warm")
    return th, S.t(), path.value


def apply_operator_noalloc(row_ptr, col_idx, x, trim: int, sigma: float = 0.0, delta: float = 0.0, V=None,
                           drop_rank1: bool = False, y=None, stream=None):
    """Handle-free operator apply that allocates no device memory inside the library (see
    isira_apply_operator_noalloc in include/isira.h).  Pass y to avoid the output allocation here too."""
    import torch
    _check_csr(row_ptr, col_idx, cuda=False)
    n = row_ptr.numel() - 1
    prec = _check_x(x, n, cuda=False)
    c = _check_V(V, n, cuda=False)          # the scratch limit (c <= 8) is the library's to report
    if y is not None:
        _check_y(y, x, cuda=False)
    _check_cuda(row_ptr=row_ptr, col_idx=col_idx, x=x, y=y, V=V)
    if y is None:
        y = torch.empty_like(x)
    Vc = None if V is None else V.t().contiguous()
    check(lib.isira_apply_operator_noalloc(row_ptr.numel() - 1, col_idx.numel(), _ptr(row_ptr), _ptr(col_idx),
                                           int(trim), prec, float(sigma), float(delta), int(bool(drop_rank1)), c,
                                           _ptr(Vc), _ptr(x), _ptr(y), _stream_ptr(stream)),
          "isira_apply_operator_noalloc")
    return y


class Batch:
    """Many independent graphs solved concurrently (isira_batch_*): one solver and one CUDA stream
    per graph, driven by a pool of host threads inside the library."""

    def __init__(self, graphs, **opts):
        """graphs: list of (row_ptr int64 CUDA tensor, col_idx int32 CUDA tensor)."""
        import numpy as np
        for rp, ci in graphs:
            _check_csr(rp, ci)
        self.graphs = list(graphs)
        G = len(self.graphs)
        self.n = [rp.numel() - 1 for rp, _ in self.graphs]
        n = np.array(self.n, dtype=np.int64)
        nnz = np.array([ci.numel() for _, ci in self.graphs], dtype=np.int64)
        rps = (C.c_void_p * G)(*[rp.data_ptr() for rp, _ in self.graphs])
        cis = (C.c_void_p * G)(*[ci.data_ptr() for _, ci in self.graphs])
        self.opts = default_opts(**opts)
        h = C.c_void_p()
        check(lib.isira_batch_create(C.byref(h), G, n.ctypes.data, nnz.ctypes.data, C.cast(rps, C.c_void_p),
                                     C.cast(cis, C.c_void_p), C.byref(self.opts)), "isira_batch_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib.isira_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, k: int, sigma: float = 0.0, rel_tol: float = 1e-8, n_threads: int = 0) -> int:
        return lib.isira_batch_solve(self.h, int(k), float(sigma), float(rel_tol), int(n_threads))

    def status(self, g: int) -> int:
        return lib.isira_batch_status(self.h, g)

    def stats(self, g: int) -> dict:
        st = isira_stats()
        check(lib.isira_batch_get_stats(self.h, g, C.byref(st)), "isira_batch_get_stats")
        return st.as_dict()

    def eigpairs(self, g: int):
        import torch
        k = self.stats(g)["n_locked"]
        lam = torch.empty(k, dtype=torch.float64)
        vec = torch.empty((k, self.n[g]), dtype=torch.float64, device=self.graphs[g][0].device)
        res = torch.empty(k, dtype=torch.float64)
        nout = C.c_int(0)
        check(lib.isira_batch_eigpairs(self.h, g, _ptr(lam), _ptr(vec), _ptr(res), C.byref(nout)),
              "isira_batch_eigpairs")
        return lam, vec.t(), res


def solve(row_ptr, col_idx, k: int, sigma: float = 0.0, tol: float | None = None, rel_tol: float = 1e-8, u0=None,
          weights=None, **opts) -> Result:
    """Computes the k smallest positive eigenpairs of the Laplacian (weighted, with weights) of the graph
    (row_ptr, col_idx)."""
    with Solver(row_ptr, col_idx, weights=weights, **opts) as s:
        status = s.solve(k, sigma, tol, u0=u0, rel_tol=rel_tol, raise_on_error=False)
        if status not in (ISIRA_OK, ISIRA_ERR_NO_CONVERGENCE, ISIRA_ERR_NOT_CONNECTED):
            raise IsiraError(status, "isira_solve")
        lam, vec, res = s.eigpairs()
        return Result(lam, vec, res, s.stats(), status)
