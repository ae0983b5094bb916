"""Thin ctypes binding of the C ABI in ``include/di.h`` (libdi.so).

Argument marshalling only: every step of the D-iteration runs in the CUDA
library.  There is no CPU fallback; if ``libdi.so`` has not been built the
first call raises.  Device buffers are passed as raw pointers (for example
``tensor.data_ptr()`` of a CUDA ``torch.Tensor``); streams as the
``cudaStream_t`` value (``torch.cuda.current_stream().cuda_stream``).
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

c_i32, c_i64, c_dbl, c_int, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_int, ctypes.c_void_p

DI_OK, DI_EINVAL, DI_ENOMEM, DI_ECUDA, DI_ENOCONV, DI_ETIMEOUT, DI_ENONFINITE = range(7)
STATUS_NAMES = {0: "DI_OK", 1: "DI_EINVAL", 2: "DI_ENOMEM", 3: "DI_ECUDA", 4: "DI_ENOCONV",
                5: "DI_ETIMEOUT", 6: "DI_ENONFINITE"}


class di_opts(ctypes.Structure):
    _fields_ = [("alpha", c_dbl), ("fluid_fp64", c_int), ("recompute_every", c_int),
                ("max_levels", c_int), ("warm_start", c_int), ("warm_fallback", c_int),
                ("l2_window", c_int), ("timing", c_int), ("propagation", c_int), ("push_ratio", c_int), ("exact_residual", c_int), ("selection", c_int),
                ("dangling", c_int), ("recompute_drop", c_dbl), ("spin_limit", ctypes.c_longlong),
                ("stream", c_vp), ("resweeps", c_int), ("slice_sweeps", c_int)]


class di_train_opts(ctypes.Structure):
    _fields_ = [("epochs", c_int), ("batch", c_int), ("lr", c_dbl), ("beta1", c_dbl), ("beta2", c_dbl),
                ("eps", c_dbl), ("seed", ctypes.c_uint64), ("stream", c_vp)]


class di_tune(ctypes.Structure):
    _fields_ = [("thread_max_deg", c_i32), ("warp_max_deg", c_i32), ("push_ctas_per_sm", c_i32),
                ("push_window", c_i32)]

    def as_dict(self) -> dict:
        return {"thread_max_deg": self.thread_max_deg, "warp_max_deg": self.warp_max_deg,
                "push_ctas_per_sm": self.push_ctas_per_sm, "push_window": self.push_window}


class di_stats(ctypes.Structure):
    _fields_ = [("levels", c_i32), ("recomputes", c_i32), ("node_diffusions", c_i64),
                ("edge_diffusions", c_i64), ("resid_l1", c_dbl), ("err_bound", c_dbl),
                ("b_l1", c_dbl), ("f0_l1", c_dbl), ("seconds", c_dbl), ("warm_used", c_i32),
                ("status", c_i32), ("gpu_launches", c_i64), ("level_seconds", c_dbl),
                ("recompute_seconds", c_dbl), ("level_launches", c_i32), ("recompute_launches", c_i32),
                ("body_iterations", c_i32), ("slice_sweeps", c_i32), ("select_seconds", c_dbl),
                ("red_ops", c_i64), ("slice_nodes", c_i64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class DiError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_LOCK = threading.Lock()
_LIB = None

# name -> (restype, argtypes); every function declared in include/di.h
SIGNATURES = {
    "di_version": (ctypes.c_char_p, []),
    "di_last_error": (ctypes.c_char_p, []),
    "di_opts_default": (c_int, [ctypes.POINTER(di_opts)]),
    "di_graph_create": (c_int, [c_i64, c_i64, c_vp, c_vp, c_int, c_vp, ctypes.POINTER(c_vp)]),
    "di_graph_destroy": (None, [c_vp]),
    "di_graph_info": (c_int, [c_vp] + [ctypes.POINTER(c_i64)] * 6),
    "di_solve": (c_int, [c_vp, c_vp, c_dbl, c_dbl, c_vp, c_vp, ctypes.POINTER(di_opts),
                         ctypes.POINTER(di_stats)]),
    "di_solve_host": (c_int, [c_vp, c_vp, c_dbl, c_dbl, c_vp, c_vp, ctypes.POINTER(di_opts),
                              ctypes.POINTER(di_stats)]),
    "di_residual": (c_int, [c_vp, c_vp, c_dbl, c_vp, c_vp, ctypes.POINTER(c_dbl), c_vp]),
    "di_frontier": (c_int, [c_vp, c_vp, c_int, c_dbl, c_vp, ctypes.POINTER(c_i64),
                            ctypes.POINTER(c_dbl), ctypes.POINTER(c_dbl), c_vp]),
    "di_residual_noalloc": (c_int, [c_vp, c_vp, c_dbl, c_vp, c_vp, ctypes.POINTER(c_dbl), c_vp]),
    "di_solve_partitioned": (c_int, [c_vp, c_vp, c_dbl, c_dbl, c_vp, c_vp, ctypes.POINTER(di_opts), c_i32, c_i32,
                                     c_vp, c_vp, ctypes.POINTER(di_stats)]),
    "di_train_opts_default": (c_int, [ctypes.POINTER(di_train_opts)]),
    "di_model_create": (c_int, [ctypes.c_uint64, ctypes.POINTER(c_vp)]),
    "di_model_destroy": (None, [c_vp]),
    "di_model_get": (c_int, [c_vp, c_vp]),
    "di_model_set": (c_int, [c_vp, c_vp]),
    "di_features": (c_int, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    "di_mlp_forward": (c_int, [c_vp, c_vp, c_i64, c_vp, c_vp]),
    "di_mlp_grad": (c_int, [c_vp, c_vp, c_vp, c_i64, c_vp, ctypes.POINTER(c_dbl), c_vp]),
    "di_model_adam": (c_int, [c_vp, c_vp, ctypes.POINTER(di_train_opts)]),
    "di_warmstart_train": (c_int, [c_vp, c_vp, c_int, c_vp, c_vp, ctypes.POINTER(di_train_opts),
                                   ctypes.POINTER(c_dbl)]),
    "di_warmstart_infer": (c_int, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    "di_warmstart_save": (c_int, [c_vp, ctypes.c_char_p]),
    "di_warmstart_load": (c_int, [ctypes.c_char_p, ctypes.POINTER(c_vp)]),
    "di_tune_default": (c_int, [ctypes.POINTER(di_tune)]),
    "di_graph_set_tune": (c_int, [c_vp, ctypes.POINTER(di_tune)]),
    "di_graph_get_tune": (c_int, [c_vp, ctypes.POINTER(di_tune)]),
    "di_batch_set_tune": (c_int, [c_vp, ctypes.POINTER(di_tune)]),
    "di_batch_get_tune": (c_int, [c_vp, ctypes.POINTER(di_tune)]),
    "di_autotune": (c_int, [c_vp, c_vp, c_dbl, c_dbl, ctypes.POINTER(di_opts), ctypes.c_char_p,
                            ctypes.POINTER(di_tune), ctypes.POINTER(c_dbl)]),
    "di_batch_autotune": (c_int, [c_vp, c_vp, c_dbl, c_vp, c_vp, ctypes.POINTER(di_opts), ctypes.c_char_p,
                                  ctypes.POINTER(di_tune), ctypes.POINTER(c_dbl)]),
    "di_batch_create": (c_int, [c_vp, c_int, c_vp, c_vp, ctypes.POINTER(c_vp)]),
    "di_batch_destroy": (None, [c_vp]),
    "di_batch_info": (c_int, [c_vp, ctypes.POINTER(c_int), ctypes.POINTER(c_i64), ctypes.POINTER(c_i64)]),
    "di_solve_batched": (c_int, [c_vp, c_vp, c_dbl, c_vp, c_vp, ctypes.POINTER(di_opts),
                                 ctypes.POINTER(di_stats), ctypes.POINTER(di_stats)]),
    "di_probe_l2": (c_int, [c_int, c_i64, c_i64, ctypes.POINTER(c_dbl), ctypes.POINTER(c_dbl), c_vp]),
}


def library_path() -> str:
    return _build.DI_SO


def lib():
    """The loaded libdi.so (raises if it has not been built)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libdi.so not found at {path}: build it first "
                                   "(python -c 'import __graft_entry__ as g; g.build()')")
            handle = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = handle
    return _LIB


def last_error() -> str:
    return lib().di_last_error().decode()


def check(status: int, allow=(DI_OK,)) -> int:
    if status not in allow:
        raise DiError(status, last_error())
    return status


def opts_default(**overrides) -> di_opts:
    o = di_opts()
    check(lib().di_opts_default(ctypes.byref(o)))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def opts_copy(o: di_opts, **overrides) -> di_opts:
    """A copy of an options struct (raw bytes: the stream pointer included),
    with fields overridden."""
    c = di_opts.from_buffer_copy(o)
    for k, v in overrides.items():
        setattr(c, k, v)
    return c


def _ptr(x) -> int | None:
    """Raw address of a torch tensor, numpy array, int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Graph:
    """Owner of a ``di_graph`` handle (freed by ``close`` or garbage collection)."""

    def __init__(self, handle: int, n: int, nnz: int):
        self.handle = handle
        self.n = n
        self.nnz = nnz

    @classmethod
    def create(cls, row_ptr, col, on_device: bool = False, stream=None) -> "Graph":
        n = len(row_ptr) - 1
        nnz = len(col)
        h = c_vp()
        check(lib().di_graph_create(n, nnz, _ptr(row_ptr), _ptr(col) if nnz else None,
                                    1 if on_device else 0, _stream(stream), ctypes.byref(h)))
        return cls(h.value, n, nnz)

    def info(self) -> dict:
        vals = [c_i64() for _ in range(6)]
        check(lib().di_graph_info(self.handle, *[ctypes.byref(v) for v in vals]))
        keys = ["n", "nnz", "n_dangling", "max_outdeg", "max_indeg", "n_hot"]
        return {k: v.value for k, v in zip(keys, vals)}

    def close(self) -> None:
        if self.handle:
            lib().di_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def di_solve(graph: Graph, B, d: float, tol: float, H, F=None, opts: di_opts | None = None,
             allow=(DI_OK,)) -> tuple[int, di_stats]:
    st = di_stats()
    rc = lib().di_solve(graph.handle, _ptr(B), d, tol, _ptr(H), _ptr(F),
                        ctypes.byref(opts) if opts is not None else None, ctypes.byref(st))
    check(rc, allow)
    return rc, st


def di_solve_host(graph: Graph, B, d: float, tol: float, H, F=None, opts: di_opts | None = None,
                  allow=(DI_OK,)) -> tuple[int, di_stats]:
    st = di_stats()
    rc = lib().di_solve_host(graph.handle, _ptr(B), d, tol, _ptr(H), _ptr(F),
                             ctypes.byref(opts) if opts is not None else None, ctypes.byref(st))
    check(rc, allow)
    return rc, st


def di_residual(graph: Graph, B, d: float, H, F, stream=None) -> float:
    r = c_dbl()
    check(lib().di_residual(graph.handle, _ptr(B), d, _ptr(H), _ptr(F), ctypes.byref(r), _stream(stream)))
    return r.value


def di_residual_noalloc(graph: Graph, B, d: float, H, F, stream=None) -> float:
    """di_residual for callers that cannot allocate device memory: scratch in
    a fixed static array of the library (graphs up to 2^20 nodes)."""
    r = c_dbl()
    check(lib().di_residual_noalloc(graph.handle, _ptr(B), d, _ptr(H), _ptr(F), ctypes.byref(r),
                                    _stream(stream)))
    return r.value


def di_solve_partitioned(graph: Graph, B, d: float, tol: float, H, K: int, kind: int = 0, F=None,
                         opts: di_opts | None = None, allow=(DI_OK,)):
    """K-PID asynchronous D-iteration (Secs. 2.3-2.6); kind 0 uniform, 1 cost-balanced
    ranges.  Returns (status, di_stats, per-PID elementary diffusions, per-PID transmissions)."""
    import numpy as np
    st = di_stats()
    ops = np.zeros(K, dtype=np.int64)
    sends = np.zeros(K, dtype=np.int64)
    rc = lib().di_solve_partitioned(graph.handle, _ptr(B), d, tol, _ptr(H), _ptr(F),
                                    ctypes.byref(opts) if opts is not None else None, K, kind,
                                    ops.ctypes.data, sends.ctypes.data, ctypes.byref(st))
    check(rc, allow)
    return rc, st, ops, sends


class Batch:
    """Owner of a ``di_batch`` handle: work item t is right-hand side r of
    graph g, numbered graph-major (all items of graphs[0] first)."""

    def __init__(self, graphs, nrhs, stream=None):
        self.graphs = list(graphs)
        self.nrhs = [int(r) for r in nrhs]
        if len(self.graphs) != len(self.nrhs):
            raise ValueError("one nrhs per graph")
        handles = (c_vp * len(self.graphs))(*[g.handle for g in self.graphs])
        counts = (c_int * len(self.nrhs))(*self.nrhs)
        h = c_vp()
        check(lib().di_batch_create(handles, len(self.graphs), counts, _stream(stream), ctypes.byref(h)))
        self.handle = h.value
        self.sizes = [g.n for g, r in zip(self.graphs, self.nrhs) for _ in range(r)]

    def info(self) -> dict:
        ni, nu, eu = c_int(), c_i64(), c_i64()
        check(lib().di_batch_info(self.handle, ctypes.byref(ni), ctypes.byref(nu), ctypes.byref(eu)))
        return {"n_items": ni.value, "n_union": nu.value, "nnz_union": eu.value}

    def close(self) -> None:
        if self.handle:
            lib().di_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def di_solve_batched(batch: Batch, B: list, d: float, tol, H: list, opts: di_opts | None = None,
                     allow=(DI_OK,)) -> tuple[int, list, di_stats]:
    """Solves every item; B and H are lists of device buffers (one per item),
    tol a scalar or one tolerance per item.  Returns (status, per-item
    stats, total stats)."""
    ni = len(batch.sizes)
    if len(B) != ni or len(H) != ni:
        raise ValueError(f"need {ni} B and H buffers")
    tols = [float(tol)] * ni if isinstance(tol, (int, float)) else [float(t) for t in tol]
    bp = (c_vp * ni)(*[_ptr(x) for x in B])
    hp = (c_vp * ni)(*[_ptr(x) for x in H])
    tp = (c_dbl * ni)(*tols)
    items = (di_stats * ni)()
    tot = di_stats()
    rc = lib().di_solve_batched(batch.handle, bp, d, tp, hp,
                                ctypes.byref(opts) if opts is not None else None, items, ctypes.byref(tot))
    check(rc, allow)
    return rc, list(items), tot


MODEL_NFEAT = 9
MODEL_NPARAM = 5313
MODEL_STATE = 2 * MODEL_NFEAT + MODEL_NPARAM


def train_opts_default(**overrides) -> di_train_opts:
    o = di_train_opts()
    check(lib().di_train_opts_default(ctypes.byref(o)))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


class Model:
    """Owner of a ``di_model`` handle (the learned warm start)."""

    def __init__(self, handle: int):
        self.handle = handle

    @classmethod
    def create(cls, seed: int = 1) -> "Model":
        h = c_vp()
        check(lib().di_model_create(seed, ctypes.byref(h)))
        return cls(h.value)

    @classmethod
    def load(cls, path: str) -> "Model":
        h = c_vp()
        check(lib().di_warmstart_load(path.encode(), ctypes.byref(h)))
        return cls(h.value)

    def save(self, path: str) -> None:
        check(lib().di_warmstart_save(self.handle, path.encode()))

    def get_state(self):
        import numpy as np
        st = np.zeros(MODEL_STATE, dtype=np.float32)
        check(lib().di_model_get(self.handle, st.ctypes.data))
        return st

    def set_state(self, state) -> None:
        import numpy as np
        st = np.ascontiguousarray(state, dtype=np.float32)
        if st.shape != (MODEL_STATE,):
            raise ValueError(f"state must have {MODEL_STATE} floats")
        check(lib().di_model_set(self.handle, st.ctypes.data))

    def features(self, graph: "Graph", B, feat, stream=None) -> None:
        check(lib().di_features(self.handle, graph.handle, _ptr(B), _ptr(feat), _stream(stream)))

    def forward(self, feat, n: int, y, stream=None) -> None:
        check(lib().di_mlp_forward(self.handle, _ptr(feat), n, _ptr(y), _stream(stream)))

    def grad(self, feat, target, n: int, stream=None):
        import numpy as np
        g = np.zeros(MODEL_NPARAM, dtype=np.float32)
        loss = c_dbl()
        check(lib().di_mlp_grad(self.handle, _ptr(feat), _ptr(target), n, g.ctypes.data, ctypes.byref(loss),
                                _stream(stream)))
        return loss.value, g

    def adam(self, grad, opts: di_train_opts | None = None) -> None:
        import numpy as np
        g = np.ascontiguousarray(grad, dtype=np.float32)
        check(lib().di_model_adam(self.handle, g.ctypes.data, ctypes.byref(opts) if opts is not None else None))

    def train(self, graphs: list, B: list, X: list, opts: di_train_opts | None = None) -> float:
        ng = len(graphs)
        gp = (c_vp * ng)(*[g.handle for g in graphs])
        bp = (c_vp * ng)(*[_ptr(b) for b in B])
        xp = (c_vp * ng)(*[_ptr(x) for x in X])
        loss = c_dbl()
        check(lib().di_warmstart_train(self.handle, gp, ng, bp, xp,
                                       ctypes.byref(opts) if opts is not None else None, ctypes.byref(loss)))
        return loss.value

    def infer(self, graph: "Graph", B, H0, stream=None) -> None:
        check(lib().di_warmstart_infer(self.handle, graph.handle, _ptr(B), _ptr(H0), _stream(stream)))

    def close(self) -> None:
        if self.handle:
            lib().di_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tune_default() -> di_tune:
    t = di_tune()
    check(lib().di_tune_default(ctypes.byref(t)))
    return t


def autotune(graph: Graph, B, d: float, tol: float, opts: di_opts | None = None,
             cache_path: str | None = None) -> tuple[di_tune, float]:
    """Times solves for candidate push shapes, keeps the fastest in the graph."""
    t, secs = di_tune(), c_dbl()
    check(lib().di_autotune(graph.handle, _ptr(B), d, tol, ctypes.byref(opts) if opts is not None else None,
                            cache_path.encode() if cache_path else None, ctypes.byref(t), ctypes.byref(secs)))
    return t, secs.value


def batch_autotune(batch: "Batch", B: list, d: float, tol, H: list, opts: di_opts | None = None,
                   cache_path: str | None = None) -> tuple[di_tune, float]:
    """Times batched solves for candidate push shapes, keeps the fastest in the batch."""
    ni = len(batch.sizes)
    tols = [float(tol)] * ni if isinstance(tol, (int, float)) else [float(x) for x in tol]
    bp = (c_vp * ni)(*[_ptr(x) for x in B])
    hp = (c_vp * ni)(*[_ptr(x) for x in H])
    tp = (c_dbl * ni)(*tols)
    t, secs = di_tune(), c_dbl()
    check(lib().di_batch_autotune(batch.handle, bp, d, tp, hp, ctypes.byref(opts) if opts is not None else None,
                                  cache_path.encode() if cache_path else None, ctypes.byref(t),
                                  ctypes.byref(secs)))
    return t, secs.value


def set_tune(obj, tune: di_tune) -> None:
    fn = lib().di_batch_set_tune if isinstance(obj, Batch) else lib().di_graph_set_tune
    check(fn(obj.handle, ctypes.byref(tune)))


def get_tune(obj) -> di_tune:
    t = di_tune()
    fn = lib().di_batch_get_tune if isinstance(obj, Batch) else lib().di_graph_get_tune
    check(fn(obj.handle, ctypes.byref(t)))
    return t


def di_frontier(graph: Graph, F, fluid_fp64: bool, T: float, out_list, stream=None) -> tuple[int, float, float]:
    cnt, r, mx = c_i64(), c_dbl(), c_dbl()
    check(lib().di_frontier(graph.handle, _ptr(F), 1 if fluid_fp64 else 0, T, _ptr(out_list),
                            ctypes.byref(cnt), ctypes.byref(r), ctypes.byref(mx), _stream(stream)))
    return cnt.value, r.value, mx.value


def version() -> str:
    return lib().di_version().decode()


PROBE_MODES = {"red_f32": 0, "red_f64": 1, "gather_f32": 2, "red_f32_coalesced": 3, "atom_f32": 4}


def probe_l2(mode: str, slots: int, ops: int, stream=None) -> tuple[float, float]:
    """(operations per second, seconds of the best launch) of one scattered
    operation kind over a device array of `slots` words (di_probe_l2)."""
    rate, secs = c_dbl(), c_dbl()
    check(lib().di_probe_l2(PROBE_MODES[mode], slots, ops, ctypes.byref(rate), ctypes.byref(secs),
                            _stream(stream)))
    return rate.value, secs.value
