"""K-PID asynchronous D-iteration of Secs. 2.3-2.6 (TEST INFRASTRUCTURE ONLY).

* ``uniform_bounds`` / ``cb_bounds`` - the two partitions of Sec. 2.3:
  Omega_k = [w_k, w_{k+1}) with w_k = floor(k N / K), or cost balanced so that
  every range holds about L / K out-edges.
* ``kpid`` - the sequential emulation of K PIDs in ``diter.c``: lock-step
  rounds of one threshold sweep per PID, local diffusion only (algorithm (*)),
  transmission of P (H - H_old) to external nodes when s_k > r_k / K
  (Eq. send), threshold rescaling on reception (Sec. 2.6); with ``dangling``
  the columns of nodes without out-edges are completed by d/N (Sec. 2.2), their
  own range's part local and the rest owed like external edges.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import diter as _d


def uniform_bounds(n: int, k: int) -> np.ndarray:
    """w_k = floor(k N / K), k = 0..K (Sec. 2.3, uniform partition)."""
    if k < 1:
        raise ValueError("K must be >= 1")
    return np.array([(i * n) // k for i in range(k + 1)], dtype=np.int64)


def cb_bounds(row_ptr, k: int) -> np.ndarray:
    """Cost-balanced partition (Sec. 2.3): w_k is the first node index at which
    the out-edge prefix sum reaches k L / K, so that every range holds about
    L / K out-edges (exactly, up to one row)."""
    if k < 1:
        raise ValueError("K must be >= 1")
    rp = np.asarray(row_ptr, dtype=np.int64)
    n = len(rp) - 1
    L = int(rp[-1])
    b = [0]
    for i in range(1, k):
        target = i * L / k
        w = int(np.searchsorted(rp, target, side="left"))   # first j with rp[j] >= target
        b.append(min(max(w, b[-1]), n))
    b.append(n)
    return np.array(b, dtype=np.int64)


@dataclass
class KpidResult:
    H: np.ndarray
    F: np.ndarray
    H_old: np.ndarray
    status: int              # 0 converged, 4 round cap reached
    rounds: int
    ops: np.ndarray          # elementary diffusions per PID
    sends: np.ndarray        # transmissions per PID
    resid_l1: float          # exact |B + P H - H|_1 at return
    trace: np.ndarray | None  # rounds x K: r_k after every round
    T: np.ndarray            # every PID's threshold at return


def _lib():
    lib = _d._lib()
    if not getattr(lib, "_kpid_ready", False):
        vp, i64, dbl, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        lib.oracle_kpid.restype = ci
        lib.oracle_kpid.argtypes = [i64, vp, vp, vp, dbl, dbl, dbl, ci, vp, i64, vp, vp, vp, vp, vp,
                                    ctypes.POINTER(i64), ctypes.POINTER(dbl), vp, i64, vp, ci]
        lib._kpid_ready = True
    return lib


def kpid(row_ptr, col, B, d: float = 0.85, tol: float = 1e-14, alpha: float = 1.5, bounds=None,
         K: int = 1, max_rounds: int = 100_000, trace: bool = False, dangling: bool = False) -> KpidResult:
    rp, cl = _d._csr(row_ptr, col)
    n = len(rp) - 1
    bnd = np.ascontiguousarray(uniform_bounds(n, K) if bounds is None else bounds, dtype=np.int64)
    K = len(bnd) - 1
    B = np.ascontiguousarray(B, dtype=np.float64)
    H = np.zeros(n)
    F = np.zeros(n)
    Ho = np.zeros(n)
    ops = np.zeros(K, dtype=np.int64)
    sends = np.zeros(K, dtype=np.int64)
    rounds = ctypes.c_int64(0)
    resid = ctypes.c_double(0.0)
    tr = np.zeros((max_rounds if trace else 1, K))
    T = np.zeros(K)
    status = _lib().oracle_kpid(n, rp.ctypes.data, cl.ctypes.data, B.ctypes.data, d, tol, alpha, K,
                                bnd.ctypes.data, max_rounds, H.ctypes.data, F.ctypes.data, Ho.ctypes.data,
                                ops.ctypes.data, sends.ctypes.data, ctypes.byref(rounds), ctypes.byref(resid),
                                tr.ctypes.data if trace else None, max_rounds if trace else 0, T.ctypes.data,
                                1 if dangling else 0)
    if status == 1:
        raise ValueError("oracle rejected its arguments")
    if status == 2:
        raise MemoryError("oracle scratch allocation failed")
    return KpidResult(H=H, F=F, H_old=Ho, status=status, rounds=rounds.value, ops=ops, sends=sends,
                      resid_l1=resid.value, trace=tr[:rounds.value].copy() if trace else None, T=T)
