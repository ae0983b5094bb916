"""di_residual_noalloc: the exact residual for callers that cannot allocate
device memory on their hot path (a serving loop with memory reserved at
start-up, code running while another component owns the allocator).  Its
scratch is a fixed static array inside libdi.so instead of library
allocations, which caps it at 2^20 nodes.

On a freshly created graph, two calls in a row - the second with other
inputs, so that the first call's leftovers in the shared array cannot leak
into it - must
  * leave the free device memory unchanged (nothing is allocated; the
    kernels were loaded by a warm-up call on another graph beforehand);
  * give the residual of the CPU oracle, elementwise within the FP64
    summation bound 2 (m_k + 2) eps (|B_k| + (P|H|)_k + |H_k|) for in-degree
    m_k (the two sum each in-row in a different order), and its L1 norm to
    1e-13 relative;
  * give what the allocating entry point di_residual gives, within the same
    bound (di_residual is called after the allocation-free calls, since it
    allocates the graph's workspace).
This file is collected last; it passes alone in a fresh process and after
the other tests.
"""
import numpy as np
import pytest
import torch

from oracle import diter as od
from paper_1202_6168_gb300 import binding as di
from paper_1202_6168_gb300 import graphgen as gg

from graphs_util import csr_from_edges

pytestmark = pytest.mark.gpu
D = 0.85


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def graphs():
    rp, col = gg.generate(gg.GraphSpec(n=200_000, mean_deg=10, seed=7))
    yield "web-200k", rp, col
    # a star whose centre has in-degree 99,999: its in-row is cut into segments
    n = 100_000
    rp, col = csr_from_edges(n, [(j, 0) for j in range(1, n)] + [(0, 1), (1, 2)])
    yield "star-100k", rp, col


def summation_bound(rp, col, b, h):
    eps = np.finfo(np.float64).eps
    indeg = np.bincount(col, minlength=len(b))
    return 2 * (indeg + 2) * eps * (np.abs(b) + od.p_times(rp, col, D, np.abs(h)) + np.abs(h))


def warm_up():
    # loads the allocation-free kernels (module loading may take device memory
    # once) and resolves the static array's address on this device
    rp, col = csr_from_edges(3, [(0, 1), (1, 2), (2, 0)])
    g = di.Graph.create(rp, col)
    x = dev(np.ones(3))
    di.di_residual_noalloc(g, x, D, x, torch.zeros_like(x))
    torch.cuda.synchronize()
    g.close()


@pytest.mark.parametrize("name,rp,col", list(graphs()), ids=lambda v: v if isinstance(v, str) else "")
def test_noalloc_residual_allocates_nothing_and_matches_twice(name, rp, col):
    n = len(rp) - 1
    warm_up()
    g = di.Graph.create(rp, col)
    rng = np.random.default_rng(42)
    calls = []
    for call in range(2):
        h = rng.standard_normal(n) * 10.0 ** (-3 - call)
        b = rng.random(n) * 1e-5
        calls.append((b, h, dev(b), dev(h)))
    F_new = [torch.full((n,), float("nan"), dtype=torch.float64, device="cuda") for _ in calls]
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    r_new = [di.di_residual_noalloc(g, B, D, H, F) for (_, _, B, H), F in zip(calls, F_new)]
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before, (name, free_before - free_after)
    for call, ((b, h, B, H), F, r) in enumerate(zip(calls, F_new, r_new)):
        bound = summation_bound(rp, col, b, h)
        f_new = F.cpu().numpy()
        assert np.all(np.isfinite(f_new))
        # against the oracle's F = B + P H - H
        f_cpu, r_cpu = od.residual(rp, col, b, D, h)
        err = np.abs(f_new - f_cpu)
        assert np.all(err <= bound), (name, call, float(np.max(err - bound)))
        assert r == pytest.approx(r_cpu, rel=1e-13), (name, call)
        # against the allocating entry point
        F_ref = torch.zeros(n, dtype=torch.float64, device="cuda")
        r_ref = di.di_residual(g, B, D, H, F_ref)
        err = np.abs(f_new - F_ref.cpu().numpy())
        assert np.all(err <= bound), (name, call, float(np.max(err - bound)))
        assert r == pytest.approx(r_ref, rel=1e-13), (name, call)
    g.close()


def test_noalloc_rejects_graphs_beyond_its_capacity():
    n = (1 << 20) + 1
    g = di.Graph.create(np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32))
    B = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(di.DiError) as e:
        di.di_residual_noalloc(g, B, D, B, torch.zeros_like(B))
    assert e.value.status == di.DI_EINVAL
    assert "capacity" in str(e.value)
    g.close()
