"""Seeded synthetic inputs: directed graphs shaped like the paper's web graphs
(Sec. 3, Table 1) and right-hand sides B of the PageRank form (Eq. 3).

This module is the one piece shared by the CPU oracle and the CUDA path.  It
generates inputs only; it holds no step of the D-iteration method.  The
graph recipe is documented in ``gen/graphgen.c``.

Graphs come back as a CSR of out-edges: ``row_ptr`` (int64, N+1) and ``col``
(int32, L); row j lists the targets k of the edges j -> k, i.e. the non-zero
rows of column j of P (p_kj = d / outdeg_j).
"""
from __future__ import annotations

import ctypes
import math
import os
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
            path = _build.build_gen()
            lib = ctypes.CDLL(path)
            c_i64, c_dbl, c_u64, c_int = ctypes.c_int64, ctypes.c_double, ctypes.c_uint64, ctypes.c_int
            vp = ctypes.c_void_p
            lib.dg_new.restype = vp
            lib.dg_new.argtypes = [c_i64, c_dbl, c_i64, c_dbl, c_dbl, c_dbl, c_int, c_dbl, c_u64]
            lib.dg_free.argtypes = [vp]
            lib.dg_row_ptr.restype = c_i64
            lib.dg_row_ptr.argtypes = [vp, vp]
            lib.dg_fill.restype = c_int
            lib.dg_fill.argtypes = [vp, vp, vp]
            lib.dg_hash.restype = c_u64
            lib.dg_hash.argtypes = [c_i64, vp, vp]
            lib.dg_zipf_mean.restype = c_dbl
            lib.dg_zipf_mean.argtypes = [vp]
            lib.dg_max_degree.restype = c_i64
            lib.dg_max_degree.argtypes = [vp]
            for name in ("dg_det_pow",):
                getattr(lib, name).restype = c_dbl
                getattr(lib, name).argtypes = [c_dbl, c_dbl]
            for name in ("dg_det_log", "dg_det_exp"):
                getattr(lib, name).restype = c_dbl
                getattr(lib, name).argtypes = [c_dbl]
            _LIB = lib
    return _LIB


@dataclass(frozen=True)
class GraphSpec:
    """Parameters of one synthetic graph (defaults: the web-graph recipe)."""
    n: int
    mean_deg: float = 8.0
    window: int = 64
    seed: int = 0
    p_local: float = 0.3
    p_dangling: float = 0.1
    zipf_exp: float = 2.1
    zipf_max: int = 1000
    rank_exp: float = 0.9


# Workload presets, named by what they are.
SMALL_10K = GraphSpec(n=10_000, mean_deg=8.0, window=64, seed=0)            # N=1e4, m=8
WEB_1M = GraphSpec(n=1_000_000, mean_deg=10.0, window=64, seed=0)           # N=1e6, m=10
STRESS_16M = GraphSpec(n=1 << 24, mean_deg=16.0, window=256, seed=0)        # N=2^24, m=16
MID_4M = GraphSpec(n=1 << 22, mean_deg=16.0, window=256, seed=0)            # N=2^22, m=16 (profiling size)

PAGERANK_D = 0.85


def generate(spec: GraphSpec) -> tuple[np.ndarray, np.ndarray]:
    """CSR (row_ptr int64[N+1], col int32[L]) of the graph ``spec`` describes."""
    lib = _lib()
    ctx = lib.dg_new(spec.n, spec.mean_deg, spec.window, spec.p_local, spec.p_dangling,
                     spec.zipf_exp, spec.zipf_max, spec.rank_exp, spec.seed & 0xFFFFFFFFFFFFFFFF)
    if not ctx:
        raise ValueError(f"invalid graph spec {spec}")
    try:
        row_ptr = np.empty(spec.n + 1, dtype=np.int64)
        nnz = lib.dg_row_ptr(ctx, row_ptr.ctypes.data)
        if nnz < 0:
            raise MemoryError("generator pass 1 failed")
        col = np.empty(max(nnz, 1), dtype=np.int32)[:nnz]
        if lib.dg_fill(ctx, row_ptr.ctypes.data, col.ctypes.data if nnz else None) != 0:
            raise RuntimeError("generator pass 2 disagreed with pass 1")
    finally:
        lib.dg_free(ctx)
    return row_ptr, col


def csr_hash(row_ptr: np.ndarray, col: np.ndarray) -> int:
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    return int(_lib().dg_hash(len(rp) - 1, rp.ctypes.data, cl.ctypes.data if len(cl) else rp.ctypes.data))


def zipf_mean(zipf_exp: float = 2.1, zipf_max: int = 1000) -> float:
    lib = _lib()
    ctx = lib.dg_new(2, 1.0, 0, 0.3, 0.1, zipf_exp, zipf_max, 0.9, 0)
    try:
        return float(lib.dg_zipf_mean(ctx))
    finally:
        lib.dg_free(ctx)


def uniform_b(n: int, d: float = PAGERANK_D) -> np.ndarray:
    """B = (1-d) V with V the uniform probability vector (Eq. 3)."""
    return np.full(n, (1.0 - d) / n, dtype=np.float64)


def personalised_b(n: int, source: int, d: float = PAGERANK_D) -> np.ndarray:
    """B = (1-d) e_s: the personalised right-hand side (Eq. 3 with V = e_s)."""
    b = np.zeros(n, dtype=np.float64)
    b[source] = 1.0 - d
    return b


def batch_specs(count: int = 64, seed: int = 0, n_lo: float = 1e4, n_hi: float = 2e6,
                deg_lo: float = 6.0, deg_hi: float = 14.0) -> list[GraphSpec]:
    """Uneven batch of graphs: N log-uniform in [n_lo, n_hi], mean out-degree
    uniform in [deg_lo, deg_hi], graph g seeded with seed*1000 + g."""
    rng = np.random.default_rng(seed)
    out = []
    for g in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        m = float(rng.uniform(deg_lo, deg_hi))
        out.append(GraphSpec(n=n, mean_deg=m, window=64, seed=seed * 1000 + g))
    return out


def batch_sources(n: int, count: int, seed: int) -> np.ndarray:
    """``count`` seeded random source nodes of a graph with ``n`` nodes."""
    rng = np.random.default_rng(0xB5 + seed)
    return rng.integers(0, n, size=count, dtype=np.int64)


def warmstart_specs(kind: str, count: int | None = None) -> list[GraphSpec]:
    """Graphs of the learned-warm-start study: 'train' (N log-uniform in
    [1e5, 1e6], seeds 1000...) or 'eval' (N = 3e6, seeds 2000...); m = 10."""
    if kind == "train":
        count = 200 if count is None else count
        rng = np.random.default_rng(1000)
        return [GraphSpec(n=int(round(math.exp(rng.uniform(math.log(1e5), math.log(1e6))))),
                          mean_deg=10.0, window=64, seed=1000 + g) for g in range(count)]
    if kind == "eval":
        count = 32 if count is None else count
        return [GraphSpec(n=3_000_000, mean_deg=10.0, window=64, seed=2000 + g) for g in range(count)]
    raise ValueError(kind)


def det_pow(a: float, b: float) -> float:
    return float(_lib().dg_det_pow(a, b))


def det_log(a: float) -> float:
    return float(_lib().dg_det_log(a))


def det_exp(a: float) -> float:
    return float(_lib().dg_det_exp(a))
