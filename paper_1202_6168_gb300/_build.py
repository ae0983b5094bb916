"""In-tree build of the native libraries of the package.

* ``libdigen.so``  - the seeded input generator (plain C, gcc).
* ``libdi.so``     - the D-iteration CUDA library behind the C ABI declared in
  ``include/di.h`` (nvcc, sm_103a only).

Both land in ``paper_1202_6168_gb300/_lib``.  Nothing is installed into
site-packages, so the loaded ``.so`` files are the in-tree ones.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
REPO_DIR = os.path.dirname(PKG_DIR)
LIB_DIR = os.path.join(PKG_DIR, "_lib")
CSRC_DIR = os.path.join(PKG_DIR, "csrc")
GEN_SRC = os.path.join(PKG_DIR, "gen", "graphgen.c")
INCLUDE_DIR = os.path.join(REPO_DIR, "include")

GEN_SO = os.path.join(LIB_DIR, "libdigen.so")
SIM_SRC = os.path.join(PKG_DIR, "sim", "kpid_sim.c")
SIM_SO = os.path.join(LIB_DIR, "libdisim.so")
DI_SO = os.path.join(LIB_DIR, "libdi.so")

CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]

# translation units of libdi.so, compiled in parallel then linked
CU_SOURCES = [
    "abi.cu",
    "graph.cu",
    "solve.cu",
    "residual.cu",
    "noalloc.cu",
    "batch.cu",
    "warmstart.cu",
    "tune.cu",
    "partition.cu",
    "probe.cu",
]


def _run(cmd: list[str]) -> None:
    res = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if res.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + res.stdout)


def _newer(target: str, sources: list[str]) -> bool:
    if not os.path.exists(target):
        return False
    t = os.path.getmtime(target)
    return all(os.path.getmtime(s) <= t for s in sources if os.path.exists(s))


def build_gen(force: bool = False) -> str:
    os.makedirs(LIB_DIR, exist_ok=True)
    if not force and _newer(GEN_SO, [GEN_SRC]):
        return GEN_SO
    tmp = GEN_SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", "-ffp-contract=off",
            "-fno-fast-math", GEN_SRC, "-o", tmp, "-lm"]
    try:
        _run(base[:1] + ["-fopenmp"] + base[1:])
    except RuntimeError:
        _run(base)
    os.replace(tmp, GEN_SO)
    return GEN_SO


def build_sim(force: bool = False) -> str:
    """The time-stepped K-PID simulator (plain C, OpenMP over the PIDs)."""
    os.makedirs(LIB_DIR, exist_ok=True)
    if not force and _newer(SIM_SO, [SIM_SRC]):
        return SIM_SO
    tmp = SIM_SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", "-ffp-contract=off",
            "-fno-fast-math", SIM_SRC, "-o", tmp, "-lm"]
    try:
        _run(base[:1] + ["-fopenmp"] + base[1:])
    except RuntimeError:
        _run(base)
    os.replace(tmp, SIM_SO)
    return SIM_SO


def _cu_objects() -> list[tuple[str, str]]:
    obj_dir = os.path.join(LIB_DIR, "obj")
    os.makedirs(obj_dir, exist_ok=True)
    return [(os.path.join(CSRC_DIR, s), os.path.join(obj_dir, s.replace(".cu", ".o")))
            for s in CU_SOURCES]


def build_di(force: bool = False, extra_flags: list[str] | None = None) -> str:
    """Compile every CUDA translation unit for sm_103a and link libdi.so."""
    os.makedirs(LIB_DIR, exist_ok=True)
    headers = [os.path.join(CSRC_DIR, f) for f in os.listdir(CSRC_DIR) if f.endswith((".cuh", ".h"))]
    headers += [os.path.join(INCLUDE_DIR, f) for f in os.listdir(INCLUDE_DIR) if f.endswith(".h")]
    pairs = _cu_objects()
    all_src = [p[0] for p in pairs] + headers
    if not force and _newer(DI_SO, all_src):
        return DI_SO
    if not os.path.exists(NVCC) and shutil.which("nvcc") is None:
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    nvcc = NVCC if os.path.exists(NVCC) else shutil.which("nvcc")
    flags = ARCH_FLAGS + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                          "-Xcompiler", "-fvisibility=hidden", "-I", INCLUDE_DIR, "-I", CSRC_DIR,
                          "--expt-relaxed-constexpr"]
    if extra_flags:
        flags += list(extra_flags)

    def compile_one(p):
        src, obj = p
        if not force and _newer(obj, [src] + headers):
            return
        _run([nvcc] + flags + ["-c", src, "-o", obj])

    with ThreadPoolExecutor(max_workers=min(len(pairs), os.cpu_count() or 4)) as ex:
        list(ex.map(compile_one, pairs))
    tmp = DI_SO + f".tmp{os.getpid()}"
    _run([nvcc] + ARCH_FLAGS + ["-shared", "-o", tmp] + [p[1] for p in pairs] +
         ["-lcudart", "-lcuda"])
    os.replace(tmp, DI_SO)
    return DI_SO


def build_all(force: bool = False) -> None:
    build_gen(force)
    build_sim(force)
    build_di(force)
