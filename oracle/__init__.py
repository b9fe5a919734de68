"""FP64 CPU oracle for iSIRA (arXiv:1710.07080) -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously-correct restatement of the paper's method, used to
check the GPU library.  Only the test suite, ``__graft_entry__.smoke()`` and
the benchmark's ``cpu_baseline`` leg may import it; the GPU library never
does, and this package never imports the GPU library.

The numerical core lives in ``isira_oracle.c`` (single-threaded C, IEEE
double); this module compiles it with gcc on first use and calls it through
ctypes with numpy arrays.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "isira_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain -O2, no architecture-specific flags)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
                os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "isira_oracle.h"))):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("d", C.c_int), ("m", C.c_int), ("q", C.c_int), ("eps", C.c_double),
                ("sigma0", C.c_double), ("trim", C.c_int64), ("delta", C.c_double),
                ("omega", C.c_double), ("tau_inner", C.c_double), ("max_inner", C.c_int),
                ("max_outer", C.c_int), ("drop_rank1", C.c_int), ("seed", C.c_uint64)]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int), ("n_locked", C.c_int), ("outer_steps", C.c_int),
                ("inner_iters", C.c_longlong), ("restarts", C.c_int), ("breakdowns", C.c_int),
                ("trim", C.c_int64), ("delta", C.c_double), ("w_columns", C.c_longlong),
                ("sec_w", C.c_double), ("sec_inner", C.c_double), ("sec_total", C.c_double)]


def build_variant(out_path: str, plant: int) -> str:
    """Mutation testing only: compile a separate copy of the oracle with one planted mistake
    (-DOR_PLANT=plant, see isira_oracle.c) to check that the pins catch it."""
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", f"-DOR_PLANT={int(plant)}",
                           "-Wl,-Bsymbolic", "-o", out_path, _SRC, "-lm"])
    return out_path


@contextlib.contextmanager
def using_library(path: str):
    """Mutation testing only: route every oracle call through the library at `path`."""
    global _lib
    saved = _lib
    _lib = _bind(C.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(C.CDLL(build()))
    return _lib


def _bind(lib):
    """Declares the C signatures on a loaded oracle library."""
    P = C.c_void_p
    lib.or_laplacian_apply.argtypes = [C.c_int64, P, P, P, P, P]
    lib.or_sym_eig.argtypes = [C.c_int, P, P, P, C.c_int]
    lib.or_sym_eig.restype = C.c_int
    lib.or_dense_laplacian_eig.argtypes = [C.c_int64, P, P, P, P, P]
    lib.or_trimmed_apply.argtypes = [C.c_int64, P, P, P, C.c_int64, C.c_double, C.c_double, P, C.c_int,
                                     C.c_int, P, P]
    lib.or_backmap.argtypes = [C.c_int64, C.c_int64, P, P]
    lib.or_precond_apply.argtypes = [C.c_int64, P, P, C.c_int64, C.c_double, C.c_double, P, C.c_int, P, P]
    lib.or_inner_solve.argtypes = [C.c_int64, P, P, P, C.c_int64, C.c_double, C.c_double, P, C.c_int,
                                   C.c_int, P, C.c_double, C.c_int, P, P]
    lib.or_inner_solve.restype = C.c_int
    lib.or_isira.argtypes = [C.c_int64, P, P, P, P, C.POINTER(Params), P, P, C.POINTER(Stats)]
    lib.or_isira.restype = C.c_int
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _csr(row_ptr, col_idx):
    return (np.ascontiguousarray(row_ptr, dtype=np.int64), np.ascontiguousarray(col_idx, dtype=np.int32))


def _w(weights, nnz):
    """Edge weights as a contiguous float64 array aligned with col_idx (None: unit weights)."""
    if weights is None:
        return None, None
    w = np.ascontiguousarray(weights, dtype=np.float64)
    if w.shape != (nnz,):
        raise ValueError(f"weights must have shape ({nnz},)")
    return w, _p(w)


def laplacian_apply(row_ptr, col_idx, x, weights=None) -> np.ndarray:
    """y = L x, L = D - A (paper Eq. 1.1), or the weighted L_w x. x may be (n,) or (n, b)."""
    rp, ci = _csr(row_ptr, col_idx)
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 2:
        return np.stack([laplacian_apply(rp, ci, x[:, t], weights) for t in range(x.shape[1])], axis=1)
    x = np.ascontiguousarray(x)
    y = np.empty_like(x)
    w, wp = _w(weights, ci.shape[0])
    _load().or_laplacian_apply(rp.shape[0] - 1, _p(rp), _p(ci), wp, _p(x), _p(y))
    return y


def sym_eig(A, max_sweeps: int = 100):
    """Cyclic Jacobi eigen-decomposition of a symmetric matrix: (theta ascending, S, sweeps)."""
    A = np.asfortranarray(np.asarray(A, dtype=np.float64))
    k = A.shape[0]
    th = np.empty(k)
    S = np.empty((k, k), order="F")
    sw = _load().or_sym_eig(k, _p(A), _p(th), _p(S), max_sweeps)
    return th, S, sw


def dense_laplacian_eig(row_ptr, col_idx, weights=None):
    """All eigenpairs of L (or L_w) by dense Jacobi (definition oracle, small n)."""
    rp, ci = _csr(row_ptr, col_idx)
    n = rp.shape[0] - 1
    lam = np.empty(n)
    X = np.empty((n, n), order="F")
    w, wp = _w(weights, ci.shape[0])
    _load().or_dense_laplacian_eig(n, _p(rp), _p(ci), wp, _p(lam), _p(X))
    return lam, X


def _vmat(V, n):
    if V is None:
        return np.zeros((n, 0), order="F"), 0
    V = np.asfortranarray(np.asarray(V, dtype=np.float64).reshape(n, -1))
    return V, V.shape[1]


def trimmed_apply(row_ptr, col_idx, trim, sigma, delta, V, xh, drop_rank1=False, weights=None) -> np.ndarray:
    """Theorem 2.6 operator on an (n-1)-vector."""
    rp, ci = _csr(row_ptr, col_idx)
    n = rp.shape[0] - 1
    V, c = _vmat(V, n)
    xh = np.ascontiguousarray(xh, dtype=np.float64)
    yh = np.empty(n - 1)
    w, wp = _w(weights, ci.shape[0])
    _load().or_trimmed_apply(n, _p(rp), _p(ci), wp, int(trim), float(sigma), float(delta), _p(V), c,
                             int(bool(drop_rank1)), _p(xh), _p(yh))
    return yh


def backmap(n, trim, zh) -> np.ndarray:
    """Theorem 2.4 back-map (Eq. 2.5) from an (n-1)-vector to an n-vector orthogonal to 1."""
    zh = np.ascontiguousarray(zh, dtype=np.float64)
    z = np.empty(n)
    _load().or_backmap(int(n), int(trim), _p(zh), _p(z))
    return z


def precond_apply(row_ptr, trim, sigma, delta, V, xh, weights=None) -> np.ndarray:
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    n = rp.shape[0] - 1
    V, c = _vmat(V, n)
    xh = np.ascontiguousarray(xh, dtype=np.float64)
    ph = np.empty(n - 1)
    w, wp = _w(weights, int(rp[-1]))
    _load().or_precond_apply(n, _p(rp), wp, int(trim), float(sigma), float(delta), _p(V), c, _p(xh), _p(ph))
    return ph


def inner_solve(row_ptr, col_idx, trim, sigma, delta, V, r, tau=1e-10, max_it=100000, drop_rank1=False,
                weights=None):
    """Trimmed MINRES solve + back-map: returns (zstar, iterations, relative residual estimate)."""
    rp, ci = _csr(row_ptr, col_idx)
    n = rp.shape[0] - 1
    V, c = _vmat(V, n)
    r = np.ascontiguousarray(r, dtype=np.float64)
    z = np.empty(n)
    rr = C.c_double(0.0)
    w, wp = _w(weights, ci.shape[0])
    it = _load().or_inner_solve(n, _p(rp), _p(ci), wp, int(trim), float(sigma), float(delta), _p(V), c,
                                int(bool(drop_rank1)), _p(r), float(tau), int(max_it), _p(z), C.byref(rr))
    return z, it, rr.value


def default_mq(d: int) -> tuple[int, int]:
    """Search-space size m and restart size q used when the caller gives none."""
    m = max(20, 2 * d + 10)
    q = max(d + 2, m // 2)
    return m, q


def isira(row_ptr, col_idx, d, u0, eps=1e-10, sigma0=0.0, m=None, q=None, trim=-1, delta=0.0,
          omega=0.1, tau_inner=1e-10, max_inner=20000, max_outer=100000, drop_rank1=False, seed=2, weights=None):
    """Algorithm 2 (on L, or on the weighted L_w when weights are given).  Returns (lam[d] in locking
    order, V n-by-d, stats dict)."""
    rp, ci = _csr(row_ptr, col_idx)
    n = rp.shape[0] - 1
    dm, dq = default_mq(d)
    m = dm if m is None else m
    q = dq if q is None else q
    m = min(m, n - 1)
    q = min(q, m - 1)
    p = Params(d, m, q, eps, sigma0, trim, delta, omega, tau_inner, max_inner, max_outer, int(bool(drop_rank1)),
               seed)
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    lam = np.zeros(d)
    V = np.zeros((n, d), order="F")
    st = Stats()
    w, wp = _w(weights, ci.shape[0])
    _load().or_isira(n, _p(rp), _p(ci), wp, _p(u0), C.byref(p), _p(lam), _p(V), C.byref(st))
    stats = {f: getattr(st, f) for f, _ in Stats._fields_}
    stats.update(m=m, q=q)
    return lam, V, stats
