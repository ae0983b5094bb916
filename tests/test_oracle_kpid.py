"""Pins of the K-PID oracle (Secs. 2.3-2.6): the sequential emulation of K
PIDs that diffuse locally and exchange fluid through H - H_old.

What pins it besides itself:
* one PID is the plain cyclic sweep, bit for bit;
* any K and either partition reaches the exact rational solution of
  (I - P) X = B;
* after every round the fluid plus the fluid still owed to other PIDs,
  F + P_ext (H - H_old), equals B + P H - H (an independent dense P);
* a partition that no edge crosses never transmits; one that every edge
  crosses converges only through transmissions;
* the partitions of Sec. 2.3 have their defining properties;
* the cost of each PID for the same accuracy is about 1/K of one PID's
  (the paper's observation on its web graph; its figures are lost, so this
  is a loose, qualitative bound: parity of the curves is unpinned).
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import diter as od
from oracle import kpid as ok
from paper_1202_6168_gb300 import graphgen as gg

from graphs_util import csr_from_edges, random_graph
from test_oracle_pins import exact_solve

D = 0.85


def dense(rp, col, n):
    P = np.zeros((n, n))
    for j in range(n):
        deg = rp[j + 1] - rp[j]
        for e in range(rp[j], rp[j + 1]):
            P[col[e], j] += D / deg
    return P


@pytest.mark.parametrize("rounds", [1, 4, 11])
def test_one_pid_is_the_plain_sweep(rounds):
    rp, col = gg.generate(gg.GraphSpec(n=3000, mean_deg=7.0, seed=5))
    b = np.random.default_rng(1).random(3000)
    plain = od.d_iteration(rp, col, b, D, tol=0.0, max_levels=rounds)
    r = ok.kpid(rp, col, b, D, tol=0.0, K=1, max_rounds=rounds)
    assert r.status == 4 and r.rounds == rounds
    assert np.array_equal(r.H, plain.H) and np.array_equal(r.F, plain.F)
    assert r.ops[0] == plain.edge_diffusions and r.sends[0] == 0


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("K,kind", [(2, "uniform"), (3, "cb"), (5, "uniform"), (4, "cb")])
def test_any_partition_reaches_the_exact_solution(seed, K, kind):
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(K + 2, 14))
    rp, col = random_graph(n, rng)
    b = [Fraction(int(rng.integers(0, 7)), 100) for _ in range(n)]
    b[0] += Fraction(1, 50)
    x = np.array([float(v) for v in exact_solve(rp, col, b)])
    bounds = ok.uniform_bounds(n, K) if kind == "uniform" else ok.cb_bounds(rp, K)
    bf = np.array([float(v) for v in b])
    # the stop test is the exact residual, whose rounding floor is ~eps |H|_1:
    # stop at 1e-14 |B|_1, so |H - X|_1 <= 1e-14 |B|_1 / (1 - d) < 1e-13 |X|_1
    r = ok.kpid(rp, col, bf, D, tol=1e-14 * bf.sum(), bounds=bounds)
    assert r.status == 0
    assert np.abs(r.H - x).sum() <= 1e-13 * np.abs(x).sum()


@pytest.mark.parametrize("rounds", [1, 2, 5, 9])
def test_pending_fluid_invariant(rounds):
    rng = np.random.default_rng(77)
    rp, col = random_graph(80, rng)
    b = rng.random(80)
    bounds = ok.uniform_bounds(80, 3)
    part = np.repeat(np.arange(3), np.diff(bounds))
    P = dense(rp, col, 80)
    ext = P * (part[:, None] != part[None, :])       # p_ji across partitions
    r = ok.kpid(rp, col, b, D, tol=0.0, bounds=bounds, max_rounds=rounds)
    np.testing.assert_allclose(r.F + ext @ (r.H - r.H_old), b + P @ r.H - r.H, atol=1e-13)


def test_partitions_have_their_defining_properties():
    rp, col = gg.generate(gg.GraphSpec(n=5000, mean_deg=9.0, seed=6))
    assert list(ok.uniform_bounds(10, 3)) == [0, 3, 6, 10]
    L, maxdeg = int(rp[-1]), int(np.diff(rp).max())
    for K in (2, 5, 16):
        bnd = ok.cb_bounds(rp, K)
        assert bnd[0] == 0 and bnd[-1] == 5000 and np.all(np.diff(bnd) >= 0)
        cost = np.diff(rp[bnd])
        assert np.all(np.abs(cost - L / K) <= maxdeg + 1)


def test_separate_components_never_transmit():
    # two components aligned with the partition: no edge crosses it
    rng = np.random.default_rng(9)
    rp1, col1 = random_graph(50, rng, p_dangling=0.0)
    edges = [(j, int(c)) for j in range(50) for c in col1[rp1[j]:rp1[j + 1]]]
    edges += [(j + 50, c + 50) for j, c in edges]
    rp, col = csr_from_edges(100, edges)
    b = rng.random(100)
    r = ok.kpid(rp, col, b, D, tol=1e-13 * b.sum(), K=2)
    assert r.status == 0 and r.sends.sum() == 0
    x = od.d_iteration(rp, col, b, D, tol=1e-15 * b.sum()).H
    assert np.abs(r.H - x).sum() <= 1e-12 * np.abs(x).sum()


def test_crossing_edges_converge_through_transmissions():
    # every edge joins the two halves: no PID can diffuse locally at all
    n = 40
    edges = [(j, (j + 20 + k) % 40) for j in range(20) for k in range(3)]
    edges += [(j, (j - 20 + k) % 20) for j in range(20, 40) for k in range(2)]
    rp, col = csr_from_edges(n, edges)
    b = np.full(n, 0.15 / n)
    r = ok.kpid(rp, col, b, D, tol=1e-13 * b.sum(), K=2)
    x = od.d_iteration(rp, col, b, D, tol=1e-15 * b.sum()).H
    assert r.status == 0 and r.sends.min() > 5
    assert np.abs(r.H - x).sum() <= 1e-11 * np.abs(x).sum()


@pytest.mark.parametrize("K,bound", [(2, 0.6), (4, 0.35), (8, 0.22)])
def test_each_pid_costs_about_one_kth(K, bound):
    rp, col = gg.generate(gg.GraphSpec(n=20000, mean_deg=10.0, seed=3))
    b = gg.uniform_b(20000, D)
    tol = 1e-10 * b.sum()
    one = ok.kpid(rp, col, b, D, tol=tol, K=1)
    for bounds in (ok.uniform_bounds(20000, K), ok.cb_bounds(rp, K)):
        r = ok.kpid(rp, col, b, D, tol=tol, bounds=bounds)
        assert r.status == 0
        assert r.ops.max() <= bound * one.ops[0]
        assert np.abs(r.H - one.H).sum() <= 2 * tol / (1 - D)


def test_hand_trace_idle_send_and_restart():
    # 0 <-> 1, each node its own range, B = (1, 0).  Round 1: PID 0 diffuses
    # node 0 (its child is external, so nothing moves locally), owes 0.85 and
    # sends it (s_0 = 0.85 > r_0 / 2 = 0); PID 1 idles, receives 0.85 with no
    # fluid of its own and takes T_1 = received = 0.85 (Sec. 2.6).  Round 2
    # mirrors it: PID 1 diffuses node 1 and sends 0.85^2 back; PID 0 takes
    # T_0 = 0.7225.
    rp, col = csr_from_edges(2, [(0, 1), (1, 0)])
    b = np.array([1.0, 0.0])
    r1 = ok.kpid(rp, col, b, D, tol=0.0, K=2, max_rounds=1)
    np.testing.assert_array_equal(r1.H, [1.0, 0.0])
    np.testing.assert_allclose(r1.F, [0.0, 0.85], rtol=1e-15)
    np.testing.assert_array_equal(r1.H_old, [1.0, 0.0])
    np.testing.assert_allclose(r1.T, [1.0 / 1.5, 0.85], rtol=1e-15)
    assert list(r1.ops) == [1, 0] and list(r1.sends) == [1, 0]
    r2 = ok.kpid(rp, col, b, D, tol=0.0, K=2, max_rounds=2)
    np.testing.assert_allclose(r2.H, [1.0, 0.85], rtol=1e-15)
    np.testing.assert_allclose(r2.F, [0.85 ** 2, 0.0], rtol=1e-15)
    np.testing.assert_allclose(r2.T, [0.85 ** 2, 0.85 / 1.5], rtol=1e-15)
    assert list(r2.ops) == [1, 1] and list(r2.sends) == [1, 1]


def test_hand_trace_rescale_on_reception():
    # ranges {0} and {1, 2}; edges 0 -> 2 (external), 1 -> 2 and 2 -> 1 (local);
    # B = (1, 0.4, 0).  Round 1: PID 0 diffuses node 0 and sends 0.85 to node 2;
    # PID 1 starts at T_1 = 0.4, diffuses node 1 (0.34 reaches node 2 locally,
    # below T_1), ends the sweep at T_1 = 0.4 / 1.5 holding r_1 = 0.34, then
    # receives 0.85: T_1 <- T_1 (r_1 + 0.85) / r_1 (Sec. 2.6 reading).
    rp, col = csr_from_edges(3, [(0, 2), (1, 2), (2, 1)])
    b = np.array([1.0, 0.4, 0.0])
    r = ok.kpid(rp, col, b, D, tol=0.0, bounds=np.array([0, 1, 3]), max_rounds=1)
    np.testing.assert_allclose(r.H, [1.0, 0.4, 0.0], rtol=1e-15)
    np.testing.assert_allclose(r.F, [0.0, 0.0, 0.4 * 0.85 + 0.85], rtol=1e-15)
    np.testing.assert_allclose(r.T, [1.0 / 1.5, (0.4 / 1.5) * (0.34 + 0.85) / 0.34], rtol=1e-14)
    assert list(r.ops) == [1, 1] and list(r.sends) == [1, 0]


def test_hand_trace_empty_receiver_takes_the_received_amount():
    # ranges {0} and {1, 2}; edges 0 -> 1 and 0 -> 2 (both external); B = (1, 0, 0).
    # Round 1: PID 0 diffuses node 0 and owes 0.425 to each of nodes 1 and 2
    # (s_0 = 0.85 > r_0 / 2 = 0: it sends); PID 1 holds no fluid (r_1 = 0), so
    # on reception T_1 is set to received = 0.85 (Sec. 2.6), not to the largest
    # fluid of its range (0.425).  Round 2: PID 1 lowers T_1 past its empty
    # sweeps, 0.85 -> 0.85/1.5 -> 0.85/1.5^2 <= 0.425, diffuses both nodes (no
    # children) and ends at T_1 = 0.85 / 1.5^3.
    rp, col = csr_from_edges(3, [(0, 1), (0, 2)])
    b = np.array([1.0, 0.0, 0.0])
    bounds = np.array([0, 1, 3])
    r1 = ok.kpid(rp, col, b, D, tol=0.0, bounds=bounds, max_rounds=1)
    np.testing.assert_array_equal(r1.H, [1.0, 0.0, 0.0])
    np.testing.assert_allclose(r1.F, [0.0, 0.425, 0.425], rtol=1e-15)
    np.testing.assert_allclose(r1.T, [1.0 / 1.5, 0.85], rtol=1e-15)
    assert list(r1.ops) == [2, 0] and list(r1.sends) == [1, 0]
    r2 = ok.kpid(rp, col, b, D, tol=0.0, bounds=bounds, max_rounds=2)
    np.testing.assert_allclose(r2.H, [1.0, 0.425, 0.425], rtol=1e-15)
    np.testing.assert_array_equal(r2.F, [0.0, 0.0, 0.0])
    np.testing.assert_allclose(r2.T, [1.0 / 1.5, 0.85 / 1.5 ** 3], rtol=1e-15)
    assert list(r2.ops) == [2, 0] and list(r2.sends) == [1, 0]


# ---------------------------------------------------------------- 1/N completion (Sec. 2.2)

from test_oracle_pins import exact_solve_completed


def dense_completed(rp, col, n):
    """P with every column without out-edges completed by d/N."""
    P = dense(rp, col, n)
    for j in range(n):
        if rp[j + 1] == rp[j]:
            P[:, j] = D / n
    return P


@pytest.mark.parametrize("rounds", [1, 4, 11])
def test_one_pid_with_completion_is_the_plain_completed_sweep(rounds):
    # one range holds every node: a completed column is all local, so the
    # rounds are the plain sweeps of the completed D-iteration, bit for bit
    rp, col = gg.generate(gg.GraphSpec(n=1500, mean_deg=6.0, seed=7, p_dangling=0.1))
    assert np.sum(np.diff(rp) == 0) > 50
    b = np.random.default_rng(2).random(1500)
    plain = od.d_iteration(rp, col, b, D, tol=0.0, max_levels=rounds, dangling=True)
    r = ok.kpid(rp, col, b, D, tol=0.0, K=1, max_rounds=rounds, dangling=True)
    assert r.status == 4 and r.rounds == rounds
    assert np.array_equal(r.H, plain.H) and np.array_equal(r.F, plain.F)
    assert r.sends[0] == 0


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("K,kind", [(2, "uniform"), (3, "cb"), (5, "uniform")])
def test_any_partition_reaches_the_exact_completed_solution(seed, K, kind):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(K + 3, 14))
    rp, col = random_graph(n, rng, p_dangling=0.3)
    b = [Fraction(int(rng.integers(0, 7)), 100) for _ in range(n)]
    b[0] += Fraction(1, 50)
    x = np.array([float(v) for v in exact_solve_completed(rp, col, b)])
    bounds = ok.uniform_bounds(n, K) if kind == "uniform" else ok.cb_bounds(rp, K)
    bf = np.array([float(v) for v in b])
    r = ok.kpid(rp, col, bf, D, tol=1e-14 * bf.sum(), bounds=bounds, dangling=True)
    assert r.status == 0
    assert np.abs(r.H - x).sum() <= 1e-13 * np.abs(x).sum()


@pytest.mark.parametrize("rounds", [1, 2, 5, 9])
def test_pending_fluid_invariant_with_completion(rounds):
    # F plus the fluid still owed to other ranges - including the completed
    # columns' rows outside the owner's range - is the residual of the
    # completed P after every round
    rng = np.random.default_rng(78)
    rp, col = random_graph(80, rng, p_dangling=0.25)
    b = rng.random(80)
    bounds = ok.uniform_bounds(80, 3)
    part = np.repeat(np.arange(3), np.diff(bounds))
    P = dense_completed(rp, col, 80)
    ext = P * (part[:, None] != part[None, :])
    r = ok.kpid(rp, col, b, D, tol=0.0, bounds=bounds, max_rounds=rounds, dangling=True)
    np.testing.assert_allclose(r.F + ext @ (r.H - r.H_old), b + P @ r.H - r.H, atol=1e-13)


def test_hand_trace_dangling_node_transmits_to_every_other_range():
    # nodes 0..3, ranges {0, 1} and {2, 3}; node 0 is dangling and holds the
    # only fluid.  Round 1: PID 0 diffuses node 0 (H_0 = 1); its completed
    # column adds d/4 to nodes 0 and 1 (local) and owes d/4 to each of 2, 3:
    # s_0 = d/2 > r_0 / 2 = d/4, so it transmits d/4 to nodes 2 and 3
    rp, col = csr_from_edges(4, [(1, 0), (2, 3), (3, 2)])
    b = np.array([1.0, 0.0, 0.0, 0.0])
    r = ok.kpid(rp, col, b, D, tol=0.0, bounds=np.array([0, 2, 4]), max_rounds=1, dangling=True)
    q = D / 4
    assert r.H[0] == 1.0
    np.testing.assert_array_equal(r.F, [q, q, q, q])
    np.testing.assert_array_equal(r.H_old, [1.0, 0.0, 0.0, 0.0])
    assert r.sends.tolist() == [1, 0]
    assert r.ops.tolist() == [2 + 2, 0]   # two local rows, two transmitted rows
