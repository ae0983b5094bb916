"""Small hand-built graphs for tests (CSR of out-edges, int64 row_ptr, int32 col)."""
import numpy as np


def csr_from_edges(n, edges):
    """CSR of out-edges from a list of (src, dst); keeps duplicates/self-loops."""
    rows = [[] for _ in range(n)]
    for s, t in edges:
        rows[s].append(t)
    rp = np.zeros(n + 1, dtype=np.int64)
    col = []
    for j in range(n):
        col.extend(rows[j])
        rp[j + 1] = len(col)
    return rp, np.array(col, dtype=np.int32)


def random_graph(n, rng, p_dangling=0.15, max_deg=6, self_loops=True, dups=True):
    edges = []
    for j in range(n):
        if rng.random() < p_dangling:
            continue
        deg = int(rng.integers(1, max_deg + 1))
        for _ in range(deg):
            t = int(rng.integers(0, n))
            if t == j and not self_loops:
                continue
            edges.append((j, t))
            if dups and rng.random() < 0.1:
                edges.append((j, t))
    return csr_from_edges(n, edges)


def transpose(rp, col):
    n = len(rp) - 1
    src = np.repeat(np.arange(n), np.diff(rp))
    order = np.argsort(col, kind="stable")
    rpt = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rpt, col.astype(np.int64) + 1, 1)
    return np.cumsum(rpt), src[order].astype(np.int32)
