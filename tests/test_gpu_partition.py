"""K-PID asynchronous D-iteration (di_solve_partitioned, Secs. 2.3-2.6)
against the CPU oracle.

The ranges change the diffusion order only (any order with every node
diffused infinitely often converges, Sec. 2), so every K and both partitions
must reach the oracle's X within the FP32 tolerance and stop on an exact
residual below tol.  The per-PID costs follow the paper's observation (each
PID pays about 1/K of the one-PID cost) loosely, as the K-PID oracle does.
"""
import numpy as np
import pytest
import torch

from oracle import diter as od
from oracle import kpid as ok
from paper_1202_6168_gb300 import binding as di
from paper_1202_6168_gb300 import graphgen as gg

from graphs_util import csr_from_edges

pytestmark = pytest.mark.gpu
D = 0.85


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(rp, col, b, tol, K, kind=0, **opt):
    g = di.Graph.create(rp, col)
    H = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    F = torch.zeros_like(H)
    opt.setdefault("max_levels", 20000)          # bounds a run that would not converge
    rc, st, ops, sends = di.di_solve_partitioned(g, dev(b), D, tol, H, K, kind, F, di.opts_default(**opt))
    torch.cuda.synchronize()
    out = H.cpu().numpy(), st, ops, sends, F.cpu().numpy()
    g.close()
    return out


def check_stop(rp, col, b, h, st, tol):
    _, r_cpu = od.residual(rp, col, b, D, h)
    floor = 64 * np.finfo(np.float64).eps * (np.abs(b).sum() + 2 * np.abs(h).sum())
    assert r_cpu <= tol * (1 + 1e-9) + floor
    assert abs(st.resid_l1 - r_cpu) <= 1e-9 * max(r_cpu, tol) + floor


@pytest.fixture(scope="module")
def web10k():
    rp, col = gg.generate(gg.SMALL_10K)
    b = gg.uniform_b(gg.SMALL_10K.n, D)
    return rp, col, b, od.d_iteration(rp, col, b, D, tol=1e-14 * b.sum()).H


@pytest.mark.parametrize("K", [1, 2, 4, 8, 64])
@pytest.mark.parametrize("kind", [0, 1])
def test_every_partition_reaches_x(web10k, K, kind):
    rp, col, b, x = web10k
    tol = 1e-8 * b.sum()
    h, st, ops, sends, f = run(rp, col, b, tol, K, kind)
    assert st.status == di.DI_OK
    assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()
    check_stop(rp, col, b, h, st, tol)
    assert ops.sum() == st.edge_diffusions
    if K == 1:
        assert sends.sum() == 0
    else:
        assert sends.min() >= 1


def test_personalised_rhs_and_crossing_edges():
    # every edge joins the two halves: only transmissions move fluid across
    n = 4000
    rng = np.random.default_rng(3)
    edges = [(j, int(2000 + rng.integers(0, 2000))) for j in range(2000) for _ in range(3)]
    edges += [(j, int(rng.integers(0, 2000))) for j in range(2000, 4000) for _ in range(2)]
    rp, col = csr_from_edges(n, edges)
    b = gg.personalised_b(n, 17)
    x = od.d_iteration(rp, col, b, D, tol=1e-14 * b.sum()).H
    tol = 1e-8 * b.sum()
    h, st, ops, sends, _ = run(rp, col, b, tol, 2)
    assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()
    check_stop(rp, col, b, h, st, tol)
    assert sends.min() >= 3


def test_more_ranges_than_nodes():
    rp, col = csr_from_edges(3, [(0, 1), (1, 2), (2, 0)])
    b = np.array([0.1, 0.0, 0.05])
    x = od.d_iteration(rp, col, b, D, tol=1e-15).H
    h, st, _, _, _ = run(rp, col, b, 1e-12, 8)
    assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()


@pytest.mark.parametrize("K,bound", [(2, 0.65), (4, 0.4), (8, 0.27)])
def test_each_pid_costs_about_one_kth(K, bound):
    rp, col = gg.generate(gg.GraphSpec(n=20000, mean_deg=10.0, seed=3))
    b = gg.uniform_b(20000, D)
    tol = 1e-10 * b.sum()
    _, _, one, _, _ = run(rp, col, b, tol, 1)
    for kind in (0, 1):
        h, st, ops, _, _ = run(rp, col, b, tol, K, kind)
        assert st.status == di.DI_OK
        assert ops.max() <= bound * one[0]
    # the oracle's emulation of the same K PIDs shows the same split
    r = ok.kpid(rp, col, b, D, tol=tol, K=K)
    assert r.ops.max() <= bound * ok.kpid(rp, col, b, D, tol=tol, K=1).ops[0]


def test_rejects_unsupported_arguments(web10k):
    rp, col, b, _ = web10k
    g = di.Graph.create(rp, col)
    B = dev(b)
    H = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    for K, kind, opt in ((0, 0, {}), (65, 0, {}), (2, 2, {}), (2, 0, dict(fluid_fp64=1)),
                         (2, 0, dict(warm_start=1)), (2, 0, dict(dangling=2)), (2, 0, dict(selection=1))):
        with pytest.raises(di.DiError) as e:
            di.di_solve_partitioned(g, B, D, 1e-8, H, K, kind, None, di.opts_default(**opt))
        assert e.value.status == di.DI_EINVAL
    g.close()


def test_repeated_calls_on_one_graph_switch_ranges(web10k):
    # the ranges, buffers and round graph stay on the graph between calls:
    # changing K or the partition kind reloads the tables, and a plain solve
    # in between (another exact-residual form) rebuilds the round graph
    rp, col, b, x = web10k
    tol = 1e-8 * b.sum()
    g = di.Graph.create(rp, col)
    B = dev(b)
    for K, kind, plain in ((4, 0, False), (4, 1, False), (2, 0, False), (2, 0, True), (64, 1, False),
                           (4, 0, False), (4, 0, False)):
        if plain:
            Hp = torch.zeros(len(b), dtype=torch.float64, device="cuda")
            di.di_solve(g, B, D, tol, Hp, None, di.opts_default(exact_residual=1))
        H = torch.zeros(len(b), dtype=torch.float64, device="cuda")
        rc, st, ops, sends = di.di_solve_partitioned(g, B, D, tol, H, K, kind, None, di.opts_default())
        h = H.cpu().numpy()
        assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum(), (K, kind, plain)
        check_stop(rp, col, b, h, st, tol)
        assert len(ops) == K and all(o > 0 for o in ops)
    g.close()


@pytest.mark.parametrize("K", [1, 4])
def test_host_driven_rounds_match_and_time_the_kernels(web10k, K):
    rp, col, b, x = web10k
    tol = 1e-8 * b.sum()
    h, st, ops, sends, f = run(rp, col, b, tol, K, 0, timing=1)
    assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()
    check_stop(rp, col, b, h, st, tol)
    assert 0 < st.select_seconds < st.level_seconds
    assert st.recompute_seconds > 0 and st.level_launches >= st.body_iterations
    assert st.recompute_launches == st.recomputes >= 1


# ---------------------------------------------------------------- 1/N completion of dangling columns (Sec. 2.2)

@pytest.fixture(scope="module")
def web10k_completed():
    rp, col = gg.generate(gg.SMALL_10K)
    b = gg.uniform_b(gg.SMALL_10K.n, D)
    r = od.d_iteration(rp, col, b, D, tol=1e-14 * b.sum(), dangling=True)
    assert r.status == 0
    return rp, col, b, r.H


def check_stop_completed(rp, col, b, h, st, tol):
    """check_stop for the completed P: the one sum over the dangling nodes that
    every row shares adds 2 d n_dangling eps sum_dangling |H_j| to the
    rounding allowance of |F|_1."""
    _, r_cpu = od.residual(rp, col, b, D, h, dangling=True)
    eps = np.finfo(np.float64).eps
    dang = np.diff(rp) == 0
    floor = 64 * eps * (np.abs(b).sum() + 2 * np.abs(h).sum())
    floor += 2 * D * dang.sum() * eps * np.abs(h[dang]).sum()
    assert r_cpu <= tol * (1 + 1e-9) + floor
    assert abs(st.resid_l1 - r_cpu) <= 1e-9 * max(r_cpu, tol) + floor


@pytest.mark.parametrize("K", [1, 2, 4, 8, 64])
@pytest.mark.parametrize("kind", [0, 1])
def test_dangling_completion_every_partition(web10k_completed, K, kind):
    # a completed column has n_k rows in its PID's range (local) and N - n_k
    # outside (transmitted from H - H_old): every K reaches the completed X
    rp, col, b, x = web10k_completed
    assert np.sum(np.diff(rp) == 0) > 500
    tol = 1e-8 * b.sum()
    h, st, ops, sends, f = run(rp, col, b, tol, K, kind, dangling=1)
    assert st.status == di.DI_OK
    assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()
    check_stop_completed(rp, col, b, h, st, tol)
    # the completed columns are stochastic: 1'H is within the error bound of 1'X = 1
    assert abs(h.sum() - 1.0) <= st.resid_l1 / (1 - D) * 1.001 + 1e-12
    # the completed rows are elementary diffusions too (n_k local + N - n_k sent)
    assert ops.sum() > st.edge_diffusions
    if K > 1:
        assert sends.min() >= 1


def test_dangling_completion_matches_kpid_oracle():
    # all of one half's fluid leaves through dangling nodes: only the completed
    # columns' transmissions reach the other half
    n = 3000
    rng = np.random.default_rng(11)
    edges = [(j, int(rng.integers(1500, 3000))) for j in range(1500) for _ in range(2)]
    edges += [(j, int(rng.integers(1500, 3000))) for j in range(1500, 2500) for _ in range(3)]
    rp, col = csr_from_edges(n, edges)               # nodes 2500..2999 dangling
    b = gg.personalised_b(n, 5)
    tol = 1e-9 * b.sum()
    ref = ok.kpid(rp, col, b, D, tol=1e-13 * b.sum(), K=2, dangling=True)
    assert ref.status == 0
    for kind in (0, 1):
        h, st, ops, sends, _ = run(rp, col, b, tol, 2, kind, dangling=1)
        assert st.status == di.DI_OK
        assert np.abs(h - ref.H).sum() <= 1e-6 * np.abs(ref.H).sum()
        check_stop_completed(rp, col, b, h, st, tol)
        assert h[:1500].min() > 0                    # reached only by the 1/N rows
        assert sends.min() >= 1


def test_dangling_completion_all_dangling_and_tiny():
    # no edges at all: X = B + d (1'X / N) 1, so 1'X = 1'B / (1 - d)
    n = 37
    rp = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(0, dtype=np.int32)
    b = np.linspace(0.01, 0.05, n)
    x = b + D / n * b.sum() / (1 - D)
    for K in (1, 3, 8):
        h, st, _, _, _ = run(rp, col, b, 1e-13, K, dangling=1)
        assert st.status == di.DI_OK
        assert np.abs(h - x).max() <= 1e-6 * np.abs(x).max()


@pytest.mark.parametrize("K", [1, 4])
def test_dangling_completion_host_driven_rounds(web10k_completed, K):
    # the same kernels launched one round at a time: the pending uniform
    # shares survive between launches and the completed X is reached
    rp, col, b, x = web10k_completed
    tol = 1e-8 * b.sum()
    h, st, ops, sends, _ = run(rp, col, b, tol, K, 1, dangling=1, timing=1)
    assert st.status == di.DI_OK
    assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()
    check_stop_completed(rp, col, b, h, st, tol)
    assert 0 < st.select_seconds < st.level_seconds
