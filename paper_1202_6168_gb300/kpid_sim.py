"""Time-stepped simulation of K asynchronous PIDs (Secs. 2.3-2.6; the PID
model of Sec. 2.4 and the evaluation of Sec. 3), on the host cores.

* ``uniform_bounds`` / ``cb_bounds`` - the partitions of Sec. 2.3: contiguous
  ranges of N/K nodes, or cost balanced so that every range holds about L/K
  out-edges.
* ``simulate`` - K PIDs that each spend PID_Speed elementary operations per
  time step on cyclic threshold sweeps of their own nodes (local diffusion
  only, algorithm (*)), transmit P (H - H_old) to the other ranges when
  s_k > r_k / K (Eq. send) with a geometric delay of parameter Delay_Proba
  (Sec. 3), and rescale their thresholds on reception (Sec. 2.6).  It
  reports the time in normalised iterations (steps x PID_Speed / L), each
  PID's elementary operations and idle capacity, and the idle proportion
  idle / (cost + idle) of Sec. 3.

The simulation itself is ``sim/kpid_sim.c`` (libdisim.so).
"""
from __future__ import annotations

import ctypes
import threading
from dataclasses import dataclass

import numpy as np

from . import _build

_LOCK = threading.Lock()
_LIB = None


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(_build.build_sim())
            vp, i64, dbl, ci, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int, ctypes.c_uint64
            lib.ks_run.restype = ci
            lib.ks_run.argtypes = [i64, vp, vp, vp, dbl, dbl, dbl, ci, vp, dbl, ci, dbl, u64, dbl, i64, ci,
                                   vp, vp, vp, vp, vp, vp, ctypes.POINTER(i64), ctypes.POINTER(dbl),
                                   ctypes.POINTER(i64), vp, i64]
            lib.ks_delay_steps.restype = i64
            lib.ks_delay_steps.argtypes = [dbl, u64, u64]
            _LIB = lib
    return _LIB


def uniform_bounds(n: int, k: int) -> np.ndarray:
    """Omega_k = [floor(k N / K), floor((k + 1) N / K)) (Sec. 2.3)."""
    if k < 1:
        raise ValueError("K must be >= 1")
    return np.array([(i * n) // k for i in range(k + 1)], dtype=np.int64)


def cb_bounds(row_ptr, k: int) -> np.ndarray:
    """Cost-balanced ranges (Sec. 2.3): the k-th boundary is the first node at
    which the prefix sum of out-degrees reaches k L / K."""
    if k < 1:
        raise ValueError("K must be >= 1")
    rp = np.asarray(row_ptr, dtype=np.int64)
    n, L = len(rp) - 1, int(rp[-1])
    out = np.empty(k + 1, dtype=np.int64)
    out[0], out[k] = 0, n
    for i in range(1, k):
        out[i] = min(max(int(np.searchsorted(rp, i * L / k, side="left")), out[i - 1]), n)
    return out


@dataclass
class SimResult:
    H: np.ndarray
    F: np.ndarray
    status: int              # 0 converged, 4 step cap, 3 stalled above tol
    steps: int
    speed: float             # operations per PID per step (inf: unbounded)
    ops: np.ndarray          # elementary operations per PID (local diffusions + transmitted edges)
    idle: np.ndarray         # unused capacity per PID, in operations (bounded speed)
    sleep_steps: np.ndarray  # steps each PID spent asleep
    sends: np.ndarray        # transmissions per PID
    resid_l1: float          # exact |B + P H - H|_1 at return
    in_transit: int          # transmissions not yet delivered at return
    L: int
    trace: np.ndarray | None  # steps x K: r_k + s_k at the end of each step

    @property
    def normalised_time(self) -> float:
        """Elapsed time in normalised iterations: steps x PID_Speed / L."""
        return self.steps * self.speed / self.L

    @property
    def idle_share(self) -> float:
        """idle / (elementary cost + idle), over all PIDs (Sec. 3)."""
        tot = float(self.ops.sum()) + float(self.idle.sum())
        return float(self.idle.sum()) / tot if tot > 0 else 0.0


def delay_steps(delay_proba: float, seed: int, message: int) -> int:
    """Steps a transmission waits under the delay model (for its tests)."""
    return int(_lib().ks_delay_steps(delay_proba, seed, message))


def simulate(row_ptr, col, B, d: float = 0.85, tol: float = 1e-10, alpha: float = 1.5, bounds=None, K: int = 1,
             speed: float | None = None, sweeps_per_step: int = 0, delay_proba: float = 0.0, seed: int = 0,
             sleep_tol: float | None = None, max_steps: int = 100_000, threads: int = 0,
             trace: bool = False) -> SimResult:
    """K PIDs on the ranges ``bounds`` (default uniform).  speed: elementary
    operations per PID per step, default L / K (Sec. 2.4); float('inf') for an
    unbounded speed, which needs a sweep limit.  sweeps_per_step: cyclic
    sweeps a PID may start per step (0: no limit).  delay_proba: Sec. 3's
    Delay_Proba.  sleep_tol: a PID whose residual r_k is at most this sleeps
    until it receives fluid (Sec. 2.4); default tol / (2K): with every PID
    asleep and nothing in transit the exact residual is then at most
    sum r_k + sum s_k <= tol / 2 + tol / (2K) <= tol (a PID that does not
    transmit owes s_k <= r_k / K), so the run cannot stall above tol."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    n = len(rp) - 1
    L = int(rp[-1])
    bnd = np.ascontiguousarray(uniform_bounds(n, K) if bounds is None else bounds, dtype=np.int64)
    K = len(bnd) - 1
    if speed is None:
        speed = max(L / K, 1.0)
    if sleep_tol is None:
        sleep_tol = tol / (2 * K)
    B = np.ascontiguousarray(B, dtype=np.float64)
    H, F = np.zeros(n), np.zeros(n)
    ops = np.zeros(K, dtype=np.int64)
    idle = np.zeros(K)
    sleep = np.zeros(K, dtype=np.int64)
    sends = np.zeros(K, dtype=np.int64)
    steps, resid, transit = ctypes.c_int64(0), ctypes.c_double(0.0), ctypes.c_int64(0)
    tr = np.zeros((max_steps if trace else 1, K))
    status = _lib().ks_run(n, rp.ctypes.data, cl.ctypes.data if L else None, B.ctypes.data, d, tol, alpha, K,
                           bnd.ctypes.data, -1.0 if np.isinf(speed) else float(speed), sweeps_per_step,
                           delay_proba, seed, sleep_tol, max_steps, threads, H.ctypes.data, F.ctypes.data,
                           ops.ctypes.data, idle.ctypes.data, sleep.ctypes.data, sends.ctypes.data,
                           ctypes.byref(steps), ctypes.byref(resid), ctypes.byref(transit),
                           tr.ctypes.data if trace else None, max_steps if trace else 0)
    if status == 1:
        raise ValueError("simulator rejected its arguments")
    if status == 2:
        raise MemoryError("simulator allocation failed")
    return SimResult(H=H, F=F, status=status, steps=steps.value, speed=float(speed), ops=ops, idle=idle,
                     sleep_steps=sleep, sends=sends, resid_l1=resid.value, in_transit=transit.value, L=L,
                     trace=tr[:steps.value].copy() if trace else None)
