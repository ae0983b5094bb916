"""The C-ABI library loads and exports every symbol ``include/*.h`` declares.
No GPU work: only calls that validate arguments before touching a device."""
import ctypes
import glob
import os
import re

import pytest

from paper_1202_6168_gb300 import _build, binding

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for h in glob.glob(os.path.join(REPO, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"DI_API\s+[^;(]*?\b(di_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    _build.build_di()
    return binding.lib()


def test_header_declares_the_entry_points():
    names = declared_symbols()
    for required in ("di_graph_create", "di_graph_destroy", "di_solve", "di_solve_host",
                     "di_residual", "di_frontier", "di_last_error", "di_opts_default"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert name in binding.SIGNATURES, f"binding lacks {name}"


def test_only_abi_symbols_are_exported(lib):
    # the library is built with hidden visibility: nothing but di_* leaks
    out = os.popen(f"nm -D --defined-only {binding.library_path()}").read()
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert exported and all(s.startswith("di_") for s in exported), exported


def test_version_and_defaults(lib):
    assert "sm_103a" in binding.version()
    o = binding.opts_default()
    assert o.alpha == 1.5 and o.fluid_fp64 == 0 and o.recompute_every == 0 and o.recompute_drop == 1024.0
    assert o.warm_fallback == 1 and o.max_levels == 100000
    # the fields after the double keep their place in the C layout
    assert o.propagation == 3 and o.push_ratio == 8 and o.selection == 0 and o.spin_limit == 1 << 20
    assert o.resweeps == 0 and o.slice_sweeps == -1   # the last fields, after the stream pointer
    # the C side writes every field the binding declares: start from all-ones bytes
    raw = binding.di_opts()
    ctypes.memset(ctypes.byref(raw), 0xFF, ctypes.sizeof(raw))
    assert lib.di_opts_default(ctypes.byref(raw)) == binding.DI_OK
    assert raw.resweeps == 0 and raw.slice_sweeps == -1 and raw.stream is None and raw.alpha == 1.5


def test_invalid_arguments_are_rejected_before_gpu_work(lib):
    h = ctypes.c_void_p()
    rc = lib.di_graph_create(0, 0, None, None, 0, None, ctypes.byref(h))
    assert rc == binding.DI_EINVAL and "n = 0" in binding.last_error()
    rc = lib.di_graph_create(1 << 32, 0, None, None, 0, None, ctypes.byref(h))
    assert rc == binding.DI_EINVAL
    assert lib.di_opts_default(None) == binding.DI_EINVAL
    assert lib.di_solve(None, None, 0.85, 1e-8, None, None, None, None) == binding.DI_EINVAL
    assert lib.di_residual(None, None, 0.85, None, None, None, None) == binding.DI_EINVAL


def test_opts_copy_keeps_every_field(lib):
    o = binding.opts_default(alpha=2.0, resweeps=3, stream=12345)
    c = binding.opts_copy(o, propagation=7)
    assert c.alpha == 2.0 and c.resweeps == 3 and c.stream == 12345 and c.propagation == 7
    assert o.propagation == 3   # the original is untouched
