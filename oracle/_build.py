"""Builds the oracle's C part (``liboracle.so``) with gcc, in-tree.
TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``)."""
from __future__ import annotations

import os
import subprocess

ORACLE_DIR = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(ORACLE_DIR, "diter.c")
SO = os.path.join(ORACLE_DIR, "_lib", "liboracle.so")


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(SO), exist_ok=True)
    if not force and os.path.exists(SO) and os.path.getmtime(SO) >= os.path.getmtime(SRC):
        return SO
    tmp = SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", "-ffp-contract=off",
           "-fno-fast-math", SRC, "-o", tmp, "-lm"]
    res = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if res.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + " ".join(cmd) + "\n" + res.stdout)
    os.replace(tmp, SO)
    return SO
