"""The time-stepped K-PID simulator (Secs. 2.3-2.6, the PID model of Sec. 2.4
and the delay and idle measures of Sec. 3), pinned against the CPU oracle:

* with an unbounded speed, one sweep per step, no delay and no sleeping, a
  step is one lock-step round of the oracle's sequential emulation of the
  scheme - H, F, every PID's operations and transmissions, the round count
  and the residual must be the same bit for bit;
* at any speed and delay the limit is the oracle's X (within the error bound
  tol / (1 - d) of the stop rule);
* the delay of a transmission is geometric with mean p / (1 - p) steps;
* the idle share idle / (cost + idle) is zero for one PID and grows with K;
* the two partitions of Sec. 2.3 equal the oracle's.
"""
import numpy as np
import pytest

from oracle import diter as od
from oracle import kpid as ok
from paper_1202_6168_gb300 import graphgen as gg
from paper_1202_6168_gb300 import kpid_sim as ks

from graphs_util import csr_from_edges, random_graph

D = 0.85


def small_graphs():
    rp, col = gg.generate(gg.GraphSpec(n=3000, mean_deg=8.0, seed=4))
    yield "web-3k", rp, col, gg.uniform_b(3000, D)
    rng = np.random.default_rng(9)
    rp, col = random_graph(800, rng)          # dangling nodes, self-loops, duplicates
    yield "random-800", rp, col, rng.random(800)


@pytest.mark.parametrize("name,rp,col,b", list(small_graphs()), ids=lambda v: v if isinstance(v, str) else "")
@pytest.mark.parametrize("K", [1, 2, 4, 8])
@pytest.mark.parametrize("kind", ["uniform", "cb"])
def test_unbounded_speed_is_the_lock_step_emulation_bit_for_bit(name, rp, col, b, K, kind):
    n = len(rp) - 1
    bounds = ks.uniform_bounds(n, K) if kind == "uniform" else ks.cb_bounds(rp, K)
    tol = 1e-11 * b.sum()
    o = ok.kpid(rp, col, b, D, tol=tol, bounds=bounds)
    s = ks.simulate(rp, col, b, D, tol=tol, bounds=bounds, speed=float("inf"), sweeps_per_step=1, sleep_tol=0.0)
    assert o.status == 0 and s.status == 0
    assert s.steps == o.rounds
    np.testing.assert_array_equal(s.H, o.H)
    np.testing.assert_array_equal(s.F, o.F)
    assert list(s.ops) == list(o.ops) and list(s.sends) == list(o.sends)
    assert s.resid_l1 == o.resid_l1


def test_partitions_equal_the_oracles():
    rp, col = gg.generate(gg.GraphSpec(n=5000, mean_deg=9.0, seed=2))
    for K in (1, 2, 3, 7, 64, 6000):
        np.testing.assert_array_equal(ks.uniform_bounds(5000, K), ok.uniform_bounds(5000, K))
        np.testing.assert_array_equal(ks.cb_bounds(rp, K), ok.cb_bounds(rp, K))


@pytest.fixture(scope="module")
def web20k():
    rp, col = gg.generate(gg.GraphSpec(n=20_000, mean_deg=10.0, seed=3))
    b = gg.uniform_b(20_000, D)
    x = od.d_iteration(rp, col, b, D, tol=1e-14 * b.sum()).H
    return rp, col, b, x


@pytest.mark.parametrize("K", [2, 8])
@pytest.mark.parametrize("p", [0.0, 0.5, 0.8])
@pytest.mark.parametrize("kind", ["uniform", "cb"])
def test_bounded_speed_and_delays_reach_the_oracles_x(web20k, K, p, kind):
    rp, col, b, x = web20k
    bounds = ks.uniform_bounds(len(b), K) if kind == "uniform" else ks.cb_bounds(rp, K)
    tol = 1e-9 * b.sum()
    s = ks.simulate(rp, col, b, D, tol=tol, bounds=bounds, delay_proba=p, seed=11)
    assert s.status == 0 and s.resid_l1 <= tol
    # |X - H|_1 <= |B + P H - H|_1 / (1 - d), the residual counting the fluid in transit
    assert np.abs(s.H - x).sum() <= tol / (1 - D) * (1 + 1e-6)
    _, r = od.residual(rp, col, b, D, s.H)
    assert r == pytest.approx(s.resid_l1, rel=1e-12)


def test_delays_are_geometric_with_the_papers_mean():
    for p in (0.2, 0.5, 0.8):
        t = np.array([ks.delay_steps(p, 5, m) for m in range(20000)])
        mean = p / (1 - p)
        sd = np.sqrt(p) / (1 - p) / np.sqrt(len(t))          # standard error of a geometric mean
        assert abs(t.mean() - mean) <= 5 * sd, (p, t.mean(), mean)
        assert abs((t == 0).mean() - (1 - p)) <= 5 * np.sqrt(p * (1 - p) / len(t))


def test_delay_slows_the_run_and_no_delay_is_deterministic(web20k):
    rp, col, b, _ = web20k
    tol = 1e-9 * b.sum()
    a = ks.simulate(rp, col, b, D, tol=tol, K=8)
    a2 = ks.simulate(rp, col, b, D, tol=tol, K=8, threads=1)
    np.testing.assert_array_equal(a.H, a2.H)                # the PIDs' parallel work is deterministic
    slow = ks.simulate(rp, col, b, D, tol=tol, K=8, delay_proba=0.8, seed=1)
    assert slow.normalised_time > a.normalised_time


def test_idle_share_is_zero_for_one_pid_and_grows_with_k(web20k):
    rp, col, b, _ = web20k
    tol = 1e-9 * b.sum()
    shares = {}
    for K in (1, 2, 16):
        s = ks.simulate(rp, col, b, D, tol=tol, K=K)
        assert s.status == 0
        shares[K] = s.idle_share
        # the capacity of every step is either used or idle (debts carry over)
        assert s.ops.sum() + s.idle.sum() >= s.steps * s.speed * K - K * s.speed - s.L
    assert shares[1] == 0.0
    assert shares[2] < shares[16]


def test_more_pids_cost_less_time(web20k):
    # the paper's observation: with K PIDs the time to a given error falls
    # close to 1/K while N/K stays large
    rp, col, b, _ = web20k
    tol = 1e-9 * b.sum()
    one = ks.simulate(rp, col, b, D, tol=tol, K=1).normalised_time
    eight = ks.simulate(rp, col, b, D, tol=tol, K=8).normalised_time
    assert eight <= 0.5 * one


def test_edge_cases():
    # more ranges than nodes, a graph without edges, and a sleep threshold too
    # large for the tolerance (the run stops as stalled instead of spinning)
    rng = np.random.default_rng(3)
    rp, col = random_graph(30, rng)
    b = rng.random(30)
    x = od.d_iteration(rp, col, b, D, tol=1e-15 * b.sum()).H
    s = ks.simulate(rp, col, b, D, tol=1e-12 * b.sum(), K=40)
    assert s.status == 0 and np.abs(s.H - x).sum() <= 1e-12 * b.sum() / (1 - D) * 1.001
    rp0, col0 = csr_from_edges(5, [])
    s = ks.simulate(rp0, col0, np.ones(5), D, tol=1e-12, K=2)
    assert s.status == 0 and np.allclose(s.H, 1.0)
    s = ks.simulate(rp, col, b, D, tol=1e-12 * b.sum(), K=4, sleep_tol=1.0)
    assert s.status == 3
    with pytest.raises(ValueError):
        ks.simulate(rp, col, b, D, K=2, speed=float("inf"))     # unbounded speed needs a sweep limit
