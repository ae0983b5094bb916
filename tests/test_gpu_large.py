"""Parity above 2^22 nodes: the graph spans three source blocks of the exact
residual (blocks of 2^22 sources, the last one ragged), and its fluid vector
(34 MB) and CSR (0.5 GB) exceed what the smaller parity cases exercise.

The graph is the web-like generator's (mean out-degree 16, +-256 window) at
N = 2^23 + 4093.  X is the oracle's sequential D-iteration run to
1e-12 |B|_1; its own distance to the limit is then at most
1e-12 |B|_1 / (1 - d) <= 6.7e-12 |X|_1 (Sec. 2 error bound, |X|_1 >= |B|_1),
far below the 1e-6 |X|_1 allowed for the FP32-fluid path.  The solves use
the N = 2^24 workload's schedule (exact FP64 residual every 8 levels) as well
as the library's default drop rule.
"""
import numpy as np
import pytest
import torch

from oracle import diter as od
from paper_1202_6168_gb300 import binding as di
from paper_1202_6168_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu
D = 0.85
N = (1 << 23) + 4093


@pytest.fixture(scope="module")
def web8m():
    spec = gg.GraphSpec(n=N, mean_deg=16.0, window=256, seed=5)
    rp, col = gg.generate(spec)
    b = gg.uniform_b(N, D)
    r = od.d_iteration(rp, col, b, D, tol=1e-12 * b.sum())
    assert r.status == 0
    g = di.Graph.create(rp, col)
    yield rp, col, b, r.H, g
    g.close()


def check(rp, col, b, x, h, st, tol):
    assert np.all(np.isfinite(h))
    err = np.abs(h - x).sum() / np.abs(x).sum()
    assert err <= 1e-6, f"relative L1 error {err:.3e} > 1e-6"
    # the stop: the oracle's FP64 residual of the returned H meets tol and
    # equals the reported one (floor: two summation orders of |F|_1)
    _, r_cpu = od.residual(rp, col, b, D, h)
    floor = 64 * np.finfo(np.float64).eps * (np.abs(b).sum() + 2 * np.abs(h).sum())
    assert r_cpu <= tol * (1 + 1e-9) + floor
    assert abs(st.resid_l1 - r_cpu) <= 1e-9 * max(r_cpu, tol) + floor
    return err


@pytest.mark.parametrize("prop", [3, 4, 5, 6, 7])
@pytest.mark.parametrize("every", [8, 0])
def test_three_source_blocks_match_the_oracle(web8m, prop, every):
    rp, col, b, x, g = web8m
    assert g.info()["n"] > 2 * (1 << 22)          # three source blocks, the last ragged
    tol = 1e-8 * b.sum()
    H = torch.zeros(N, dtype=torch.float64, device="cuda")
    o = di.opts_default(propagation=prop, recompute_every=every, recompute_drop=0.0 if every else 1024.0)
    _, st = di.di_solve(g, torch.from_numpy(b).cuda(), D, tol, H, None, o)
    torch.cuda.synchronize()
    check(rp, col, b, x, H.cpu().numpy(), st, tol)
    assert st.recomputes >= 1
