"""Python face of the CPU oracle (TEST INFRASTRUCTURE ONLY).

* ``d_iteration``  - the sequential FP64 D-iteration of ``diter.c``
  (Eqs. defF/defH, pseudo-code of Sec. 2.1, threshold sweep of Sec. 2.4).
* ``residual``     - F = B + P H - H in FP64 (the invariant that follows
  from Eqs. defF/defH: F_n + H_n - P H_n is the same for every n).
* ``power_iteration`` - the textbook Jacobi/power iteration X <- P X + B,
  an independent route to X (its error after n steps is at most
  d^n |B|_1 / (1-d)), used to pin the D-iteration.
* ``dense_p``      - P as a dense matrix (Sec. 2.2: p_kj = d / #out_j per
  edge j -> k, zero column for a dangling j, or d/N in every row with the
  optional 1/N completion), for small-N direct solves.
"""
from __future__ import annotations

import ctypes
import threading
from dataclasses import dataclass

import numpy as np

from . import _build

_LOCK = threading.Lock()
_LIB = None


class _Stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int64), ("node_diffusions", ctypes.c_int64),
                ("edge_diffusions", ctypes.c_int64), ("resid_l1", ctypes.c_double),
                ("threshold", ctypes.c_double)]


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(_build.build())
            vp, i64, dbl, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
            lib.oracle_diter.restype = ci
            lib.oracle_diter.argtypes = [i64, vp, vp, vp, dbl, dbl, dbl, i64, ci, vp, vp,
                                         ctypes.POINTER(_Stats), vp, i64, vp, ci]
            lib.oracle_residual.restype = dbl
            lib.oracle_residual.argtypes = [i64, vp, vp, vp, dbl, vp, vp, ci]
            _LIB = lib
    return _LIB


@dataclass
class OracleResult:
    H: np.ndarray
    F: np.ndarray
    status: int              # 0 converged, 4 level cap reached
    levels: int
    node_diffusions: int
    edge_diffusions: int
    resid_l1: float
    threshold: float
    trace: np.ndarray | None = None


def _csr(row_ptr, col):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    if len(cl) == 0:
        cl = np.zeros(1, dtype=np.int32)
    return rp, cl


def selection_weights(row_ptr, col) -> np.ndarray:
    """w_i = 1 / ((#in_i + 1)(#out_i + 1)): the weight of the selection score
    F_i / ((#in_i + 1)(#out_i + 1)) of Sec. 2.4 (edges counted with multiplicity)."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    n = len(rp) - 1
    indeg = np.bincount(np.asarray(col, dtype=np.int64), minlength=n)
    outdeg = np.diff(rp)
    return 1.0 / ((indeg + 1.0) * (outdeg + 1.0))


def d_iteration(row_ptr, col, B, d: float = 0.85, tol: float = 1e-14, alpha: float = 1.5,
                max_levels: int = 100_000, H0=None, trace: bool = False,
                weighted: bool = False, dangling: bool = False) -> OracleResult:
    """Sequential cyclic-threshold D-iteration in FP64 until sum|F| <= tol.
    weighted: select on |F_i| / ((#in_i + 1)(#out_i + 1)) (Sec. 2.4).
    dangling: complete the columns of nodes without out-edges by 1/N
    (Sec. 2.2), so that a dangling diffusion adds d F_j / N to every node."""
    rp, cl = _csr(row_ptr, col)
    n = len(rp) - 1
    w = np.ascontiguousarray(selection_weights(row_ptr, col)) if weighted else None
    B = np.ascontiguousarray(B, dtype=np.float64)
    assert B.shape == (n,)
    H = np.zeros(n, dtype=np.float64) if H0 is None else np.array(H0, dtype=np.float64, copy=True)
    F = np.empty(n, dtype=np.float64)
    st = _Stats()
    tr = np.zeros(max_levels if trace else 1, dtype=np.float64)
    status = _lib().oracle_diter(n, rp.ctypes.data, cl.ctypes.data, B.ctypes.data, d, tol, alpha,
                                 max_levels, 0 if H0 is None else 1, H.ctypes.data, F.ctypes.data,
                                 ctypes.byref(st), tr.ctypes.data if trace else None,
                                 len(tr) if trace else 0, w.ctypes.data if weighted else None,
                                 1 if dangling else 0)
    if status == 1:
        raise ValueError("oracle rejected its arguments")
    return OracleResult(H=H, F=F, status=status, levels=st.levels,
                        node_diffusions=st.node_diffusions, edge_diffusions=st.edge_diffusions,
                        resid_l1=st.resid_l1, threshold=st.threshold,
                        trace=tr[:st.levels].copy() if trace else None)


def residual(row_ptr, col, B, d: float, H, dangling: bool = False) -> tuple[np.ndarray, float]:
    """(F, sum|F|) with F = B + P H - H, in FP64 (dangling: P with the 1/N
    completion of its dangling columns)."""
    rp, cl = _csr(row_ptr, col)
    n = len(rp) - 1
    B = np.ascontiguousarray(B, dtype=np.float64)
    H = np.ascontiguousarray(H, dtype=np.float64)
    F = np.empty(n, dtype=np.float64)
    r = _lib().oracle_residual(n, rp.ctypes.data, cl.ctypes.data, B.ctypes.data, d,
                               H.ctypes.data, F.ctypes.data, 1 if dangling else 0)
    return F, float(r)


def p_times(row_ptr, col, d: float, x, dangling: bool = False) -> np.ndarray:
    """P x with numpy (gather per edge, then a bincount over targets); with
    dangling, plus d/N times the sum of x over the dangling nodes in every row."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    n = len(row_ptr) - 1
    deg = np.diff(row_ptr)
    src = np.repeat(np.arange(n), deg)
    w = np.zeros(n)
    nz = deg > 0
    w[nz] = d / deg[nz]
    x = np.asarray(x, dtype=np.float64)
    y = np.bincount(col, weights=(w * x)[src], minlength=n)
    if dangling:
        y += d / n * x[~nz].sum()
    return y


def power_iteration(row_ptr, col, B, d: float = 0.85, tol: float = 1e-14,
                    max_iter: int = 100_000, dangling: bool = False) -> tuple[np.ndarray, int]:
    """X <- P X + B from X = B until |X_new - X|_1 <= tol."""
    B = np.asarray(B, dtype=np.float64)
    x = B.copy()
    for it in range(1, max_iter + 1):
        nx = p_times(row_ptr, col, d, x, dangling) + B
        delta = np.abs(nx - x).sum()
        x = nx
        if delta <= tol:
            return x, it
    raise RuntimeError("power iteration did not converge")


def dense_p(row_ptr, col, d: float = 0.85, dangling: bool = False) -> np.ndarray:
    """P with p_kj = d * (number of entries j -> k) / #out_j; with dangling,
    a column without out-edges is d/N in every row."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    n = len(row_ptr) - 1
    P = np.zeros((n, n))
    for j in range(n):
        deg = row_ptr[j + 1] - row_ptr[j]
        if deg == 0 and dangling:
            P[:, j] = d / n
        for e in range(row_ptr[j], row_ptr[j + 1]):
            P[col[e], j] += d / deg
    return P
