"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each check is independent of the oracle's own code: exact rational solves,
a library dense solve, the textbook power iteration, closed forms, the
invariants implied by Eqs. defF/defH, brute force over random diffusion
orders, and hand-derived traces of the threshold schedule (Sec. 2.4).
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import diter as od
from paper_1202_6168_gb300 import graphgen as gg

from graphs_util import csr_from_edges, random_graph, transpose

D = 0.85


def exact_solve(rp, col, b, d=Fraction(17, 20)):
    """(I - P) X = B over the rationals by Gauss-Jordan elimination."""
    n = len(rp) - 1
    A = [[Fraction(int(i == k)) for k in range(n)] for i in range(n)]
    for j in range(n):
        deg = int(rp[j + 1] - rp[j])
        for e in range(rp[j], rp[j + 1]):
            A[int(col[e])][j] -= d / deg
    rhs = [Fraction(x) for x in b]
    for c in range(n):
        piv = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        rhs[c], rhs[piv] = rhs[piv], rhs[c]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c] / A[c][c]
                A[r] = [a - f * p for a, p in zip(A[r], A[c])]
                rhs[r] -= f * rhs[c]
    return [rhs[i] / A[i][i] for i in range(n)]


# ---------------------------------------------------------------- exact X

@pytest.mark.parametrize("seed", range(6))
def test_matches_exact_rational_solution(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 11))
    rp, col = random_graph(n, rng)
    b = [Fraction(int(rng.integers(0, 7)), 100) for _ in range(n)]
    b[0] += Fraction(1, 50)
    x = exact_solve(rp, col, b)
    res = od.d_iteration(rp, col, np.array([float(v) for v in b]), D, tol=1e-17)
    assert res.status == 0
    xf = np.array([float(v) for v in x])
    assert np.abs(res.H - xf).sum() <= 1e-14 * np.abs(xf).sum()


@pytest.mark.parametrize("seed", range(8))
def test_matches_dense_solve_n200(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(20, 201))
    rp, col = random_graph(n, rng, max_deg=12)
    b = rng.random(n) * 0.01
    x = np.linalg.solve(np.eye(n) - od.dense_p(rp, col, D), b)
    res = od.d_iteration(rp, col, b, D, tol=1e-16 * b.sum())
    assert res.status == 0
    assert np.abs(res.H - x).sum() <= 1e-13 * np.abs(x).sum()


def test_matches_power_iteration_on_10k_web_graph():
    rp, col = gg.generate(gg.SMALL_10K)
    b = gg.uniform_b(gg.SMALL_10K.n, D)
    x_pi, iters = od.power_iteration(rp, col, b, D, tol=1e-14)
    assert iters > 100
    res = od.d_iteration(rp, col, b, D, tol=1e-15)
    assert res.status == 0
    assert np.abs(res.H - x_pi).sum() <= 1e-12 * np.abs(x_pi).sum()
    # the D-iteration needed fewer elementary diffusions than power iteration
    # needs edge visits (Sec. 1: the motivation of the method)
    assert res.edge_diffusions < iters * len(col)


# ---------------------------------------------------------------- closed forms

def test_isolated_dangling_node_keeps_its_b():
    rp, col = csr_from_edges(3, [(0, 1), (1, 0)])
    b = np.array([0.1, 0.2, 0.3])
    res = od.d_iteration(rp, col, b, D, tol=1e-16)
    assert res.H[2] == pytest.approx(0.3, abs=0)


def test_two_cycle():
    rp, col = csr_from_edges(2, [(0, 1), (1, 0)])
    b = np.array([0.15, 0.15])
    res = od.d_iteration(rp, col, b, D, tol=1e-16)
    np.testing.assert_allclose(res.H, 0.15 / (1 - D), rtol=1e-14)


def test_directed_path():
    n = 12
    rp, col = csr_from_edges(n, [(k, k + 1) for k in range(n - 1)])
    b = np.full(n, 0.01)
    res = od.d_iteration(rp, col, b, D, tol=1e-17)
    x = np.empty(n)
    x[0] = 0.01
    for k in range(1, n):
        x[k] = 0.01 + D * x[k - 1]
    np.testing.assert_allclose(res.H, x, rtol=1e-14)


def test_complete_digraph():
    n = 9
    rp, col = csr_from_edges(n, [(i, j) for i in range(n) for j in range(n) if i != j])
    res = od.d_iteration(rp, col, np.full(n, (1 - D) / n), D, tol=1e-16)
    np.testing.assert_allclose(res.H, 1.0 / n, rtol=1e-13)


def test_pagerank_mass_is_one_without_dangling_nodes():
    rng = np.random.default_rng(7)
    rp, col = random_graph(150, rng, p_dangling=0.0)
    res = od.d_iteration(rp, col, np.full(150, (1 - D) / 150), D, tol=1e-16)
    assert res.H.sum() == pytest.approx(1.0, abs=1e-13)


# ---------------------------------------------------------------- invariants

def test_invariants_after_every_sweep():
    rng = np.random.default_rng(11)
    rp, col = random_graph(60, rng, p_dangling=0.2)
    b = rng.random(60) * 0.01
    x = np.linalg.solve(np.eye(60) - od.dense_p(rp, col, D), b)
    deg = np.diff(rp)
    prev_h = np.zeros(60)
    full = od.d_iteration(rp, col, b, D, tol=1e-15)
    for k in range(1, full.levels + 1):
        r = od.d_iteration(rp, col, b, D, tol=1e-15, max_levels=k)
        # F_n = B + P H_n - H_n (from Eqs. defF and defH)
        f_ref = b + od.p_times(rp, col, D, r.H) - r.H
        scale = max(np.abs(b).max(), np.abs(r.H).max())
        assert np.abs(r.F - f_ref).max() <= 1e-14 * scale
        # mass: sum F = sum B - sum H + d sum_{non-dangling j} H_j
        mass = b.sum() - r.H.sum() + D * r.H[deg > 0].sum()
        assert r.F.sum() == pytest.approx(mass, abs=1e-15)
        # H is non-decreasing and below X for non-negative P and B (Sec. 2)
        assert np.all(r.H >= prev_h)
        assert np.all(r.H <= x * (1 + 1e-12))
        # error bound |X - H|_1 <= |F|_1 / (1 - d)
        assert np.abs(x - r.H).sum() <= np.abs(r.F).sum() / (1 - D) * (1 + 1e-12) + 1e-18
        prev_h = r.H


def test_residual_helper_equals_independent_matvec():
    rng = np.random.default_rng(3)
    rp, col = random_graph(40, rng)
    h = rng.standard_normal(40)
    b = rng.random(40)
    f, r = od.residual(rp, col, b, D, h)
    f_dense = b + od.dense_p(rp, col, D) @ h - h
    np.testing.assert_allclose(f, f_dense, rtol=0, atol=1e-14)
    assert r == pytest.approx(np.abs(f_dense).sum(), rel=1e-14)


# ---------------------------------------------------------------- any order converges

def brute_force_random_order(P, b, rng, tol=1e-15):
    """Eqs. defF/defH applied literally with a uniformly random sequence i_n."""
    n = len(b)
    F, H = b.copy(), np.zeros(n)
    eye = np.eye(n)
    for _ in range(200_000):
        i = int(rng.integers(0, n))
        J = np.zeros((n, n))
        J[i, i] = 1.0
        H = H + J @ F
        F = (eye - J + P @ J) @ F
        if np.abs(F).sum() <= tol:
            break
    return H


@pytest.mark.parametrize("seed", range(4))
def test_random_orders_reach_the_same_x(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(3, 9))
    rp, col = random_graph(n, rng)
    P = od.dense_p(rp, col, D)
    b = rng.random(n) * 0.1
    ref = od.d_iteration(rp, col, b, D, tol=1e-15)
    for _ in range(3):
        h = brute_force_random_order(P, b, rng)
        assert np.abs(h - ref.H).sum() <= 1e-13


# ---------------------------------------------------------------- threshold schedule

def test_threshold_schedule_on_isolated_nodes():
    rp, col = csr_from_edges(3, [])
    b = np.array([1.0, 0.5, 0.25])
    r = od.d_iteration(rp, col, b, D, tol=0.0, alpha=2.0)
    assert (r.levels, r.node_diffusions, r.edge_diffusions) == (3, 3, 0)
    assert r.threshold == pytest.approx(0.125)
    # alpha = 1.5: T = 1 -> {0}; 2/3 and 4/9 skipped as empty... T = 4/9 -> {1};
    # 8/27 empty; T = 16/81 -> {2}
    r = od.d_iteration(rp, col, b, D, tol=0.0, alpha=1.5)
    assert (r.levels, r.node_diffusions) == (3, 3)
    assert r.threshold == pytest.approx(16 / 81 / 1.5)
    np.testing.assert_array_equal(r.H, b)


def test_fluid_received_earlier_in_a_sweep_counts():
    rp, col = csr_from_edges(2, [(0, 1)])
    # T0 = 1: node 0 sends 0.85 to node 1, whose fluid 0.9 + 0.85 >= 1 is then
    # diffused in the same sweep (cyclic scan in index order)
    r = od.d_iteration(rp, col, np.array([1.0, 0.9]), D, tol=0.0)
    assert (r.levels, r.node_diffusions, r.edge_diffusions) == (1, 2, 1)
    # with node 1 first in index order it waits for the next level
    rp2, col2 = csr_from_edges(2, [(1, 0)])
    r2 = od.d_iteration(rp2, col2, np.array([0.9, 1.0]), D, tol=0.0)
    assert (r2.levels, r2.node_diffusions) == (2, 2)


def test_stop_rule_uses_fresh_l1_residual():
    rng = np.random.default_rng(5)
    rp, col = random_graph(80, rng)
    b = rng.random(80) * 0.01
    tol = 1e-9 * b.sum()
    r = od.d_iteration(rp, col, b, D, tol=tol, trace=True)
    assert r.resid_l1 <= tol
    assert np.all(r.trace[:-1] > tol) and r.trace[-1] <= tol
    f, rr = od.residual(rp, col, b, D, r.H)
    assert rr == pytest.approx(r.resid_l1, rel=1e-9)


def test_level_cap_reports_no_convergence():
    rp, col = csr_from_edges(2, [(0, 1), (1, 0)])
    r = od.d_iteration(rp, col, np.array([0.1, 0.2]), D, tol=1e-15, max_levels=3)
    assert r.status == 4 and r.levels == 3


# ---------------------------------------------------------------- warm start

def test_warm_start_at_the_solution_does_no_work():
    rng = np.random.default_rng(9)
    rp, col = random_graph(50, rng)
    b = rng.random(50) * 0.01
    x = np.linalg.solve(np.eye(50) - od.dense_p(rp, col, D), b)
    r = od.d_iteration(rp, col, b, D, tol=1e-14 * b.sum(), H0=x)
    assert r.node_diffusions == 0 and r.status == 0


def test_warm_start_from_zero_is_the_plain_solve():
    rng = np.random.default_rng(10)
    rp, col = random_graph(50, rng)
    b = rng.random(50) * 0.01
    a = od.d_iteration(rp, col, b, D, tol=1e-12)
    w = od.d_iteration(rp, col, b, D, tol=1e-12, H0=np.zeros(50))
    np.testing.assert_array_equal(a.H, w.H)
    assert a.node_diffusions == w.node_diffusions


def test_signed_warm_start_converges_to_x():
    rng = np.random.default_rng(12)
    rp, col = random_graph(70, rng)
    b = rng.random(70) * 0.01
    x = np.linalg.solve(np.eye(70) - od.dense_p(rp, col, D), b)
    h0 = x * (1 + 0.5 * rng.standard_normal(70))
    r = od.d_iteration(rp, col, b, D, tol=1e-15, H0=h0)
    assert r.status == 0
    assert np.abs(r.H - x).sum() <= 1e-15 / (1 - D) * 1.01 + 1e-13 * np.abs(x).sum()


# ---------------------------------------------------------------- the pins catch mistakes

def test_pin_detects_a_transposed_operand():
    rng = np.random.default_rng(21)
    rp, col = random_graph(30, rng, p_dangling=0.1)
    b = rng.random(30) * 0.01
    x = np.linalg.solve(np.eye(30) - od.dense_p(rp, col, D), b)
    # the transposed graph (in-edges taken as out-edges) gives another X
    rpt, colt = transpose(rp, col)
    wrong = od.d_iteration(rpt, colt, b, D, tol=1e-15)
    assert np.abs(wrong.H - x).sum() > 1e-6 * np.abs(x).sum()


def test_pin_detects_a_wrong_damping():
    rng = np.random.default_rng(22)
    rp, col = random_graph(30, rng)
    b = rng.random(30) * 0.01
    x = np.linalg.solve(np.eye(30) - od.dense_p(rp, col, D), b)
    wrong = od.d_iteration(rp, col, b, 0.8, tol=1e-15)
    assert np.abs(wrong.H - x).sum() > 1e-6 * np.abs(x).sum()


# ---------------------------------------------------------------- weighted selection (Sec. 2.4 score)

def weighted_sweep_by_loops(rp, col, b, tol, alpha=1.5, max_levels=10_000):
    """The weighted cyclic threshold sweep with plain Python loops:
    select |F_i| / ((#in_i + 1)(#out_i + 1)) >= T, T0 = the largest score."""
    n = len(rp) - 1
    indeg = [0] * n
    for e in range(len(col)):
        indeg[int(col[e])] += 1
    w = [1.0 / ((indeg[i] + 1.0) * (rp[i + 1] - rp[i] + 1.0)) for i in range(n)]
    F = [float(x) for x in b]
    H = [0.0] * n
    T = max(abs(F[i]) * w[i] for i in range(n))
    nodes = edges = levels = 0
    while True:
        r = sum(abs(x) for x in F)
        if r <= tol or levels >= max_levels:
            break
        mx = max(abs(F[i]) * w[i] for i in range(n))
        while T > mx:
            T /= alpha
        for i in range(n):
            sent = F[i]
            if abs(sent) * w[i] < T or sent == 0.0:
                continue
            H[i] += sent
            F[i] = 0.0
            nodes += 1
            deg = int(rp[i + 1] - rp[i])
            if deg == 0:
                continue
            p = D / deg
            for e in range(rp[i], rp[i + 1]):
                F[int(col[e])] += sent * p
            edges += deg
        levels += 1
        T /= alpha
    return np.array(H), nodes, edges, levels


@pytest.mark.parametrize("seed", range(3))
def test_weighted_selection_matches_a_loop_restatement(seed):
    rng = np.random.default_rng(300 + seed)
    rp, col = random_graph(40, rng, p_dangling=0.2, max_deg=8)
    b = rng.random(40) * 0.02
    tol = 1e-10
    h_ref, nodes, edges, levels = weighted_sweep_by_loops(rp, col, b, tol)
    r = od.d_iteration(rp, col, b, D, tol=tol, weighted=True)
    assert (r.node_diffusions, r.edge_diffusions, r.levels) == (nodes, edges, levels)
    np.testing.assert_allclose(r.H, h_ref, rtol=1e-14, atol=1e-18)


def test_weighted_selection_reaches_x():
    rng = np.random.default_rng(310)
    rp, col = random_graph(150, rng, max_deg=10)
    b = rng.random(150) * 0.01
    x = np.linalg.solve(np.eye(150) - od.dense_p(rp, col, D), b)
    r = od.d_iteration(rp, col, b, D, tol=1e-16 * b.sum(), weighted=True)
    assert r.status == 0
    assert np.abs(r.H - x).sum() <= 1e-13 * np.abs(x).sum()


def test_weighted_equals_raw_when_every_node_has_the_same_degrees():
    # a directed cycle: every score is |F_i| / 4, so both rules select the same sets
    n = 64
    rp, col = csr_from_edges(n, [(k, (k + 1) % n) for k in range(n)])
    rng = np.random.default_rng(311)
    b = rng.random(n)
    a = od.d_iteration(rp, col, b, D, tol=1e-12)
    w = od.d_iteration(rp, col, b, D, tol=1e-12, weighted=True)
    assert (a.levels, a.node_diffusions, a.edge_diffusions) == (w.levels, w.node_diffusions, w.edge_diffusions)
    np.testing.assert_array_equal(a.H, w.H)


# ---------------------------------------------------------------- 1/N completion of dangling columns (Sec. 2.2)

def exact_solve_completed(rp, col, b, d=Fraction(17, 20)):
    """(I - P) X = B over the rationals when every column without out-edges
    is d/N in every row (Sec. 2.2's completion), by Gauss-Jordan elimination."""
    n = len(rp) - 1
    A = [[Fraction(int(i == k)) for k in range(n)] for i in range(n)]
    for j in range(n):
        deg = int(rp[j + 1] - rp[j])
        if deg == 0:
            for i in range(n):
                A[i][j] -= d / n
        for e in range(rp[j], rp[j + 1]):
            A[int(col[e])][j] -= d / deg
    rhs = [Fraction(x) for x in b]
    for c in range(n):
        piv = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        rhs[c], rhs[piv] = rhs[piv], rhs[c]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c] / A[c][c]
                A[r] = [a - f * p for a, p in zip(A[r], A[c])]
                rhs[r] -= f * rhs[c]
    return [rhs[i] / A[i][i] for i in range(n)]


@pytest.mark.parametrize("seed", range(5))
def test_completion_matches_exact_rational_solution(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(3, 10))
    rp, col = random_graph(n, rng, p_dangling=0.4)
    b = [Fraction(int(rng.integers(0, 7)), 100) for _ in range(n)]
    b[0] += Fraction(1, 50)
    x = np.array([float(v) for v in exact_solve_completed(rp, col, b)])
    res = od.d_iteration(rp, col, np.array([float(v) for v in b]), D, tol=1e-17, dangling=True)
    assert res.status == 0
    assert np.abs(res.H - x).sum() <= 1e-14 * np.abs(x).sum()


def test_completion_makes_the_pagerank_mass_one():
    # completed columns sum to d, so 1'X = 1'B / (1 - d) = 1 for B = (1-d)/N,
    # whatever the share of dangling nodes (without the completion it is < 1)
    rp, col = gg.generate(gg.GraphSpec(n=3000, mean_deg=6.0, seed=21, p_dangling=0.3))
    assert np.sum(np.diff(rp) == 0) > 500
    b = gg.uniform_b(3000, D)
    res = od.d_iteration(rp, col, b, D, tol=1e-14, dangling=True)
    assert res.H.sum() == pytest.approx(1.0, abs=1e-12)
    plain = od.d_iteration(rp, col, b, D, tol=1e-14)
    assert plain.H.sum() < 0.9


def test_completion_on_a_graph_without_edges():
    # every column is d/N everywhere: X_k = B_k + d * sum(B) / ((1 - d) N)
    n = 7
    rp, col = csr_from_edges(n, [])
    b = np.array([0.1, 0.0, 0.3, 0.05, 0.0, 0.2, 0.01])
    res = od.d_iteration(rp, col, b, D, tol=1e-16, dangling=True)
    want = b + D * b.sum() / ((1 - D) * n)
    np.testing.assert_allclose(res.H, want, rtol=1e-13)


def test_completion_residual_and_invariant():
    # F_n = B + P H_n - H_n with the completed P after any number of sweeps,
    # and the residual helper equals an independent dense matvec
    rng = np.random.default_rng(33)
    rp, col = random_graph(60, rng, p_dangling=0.3)
    b = rng.random(60)
    P = np.zeros((60, 60))
    for j in range(60):
        deg = rp[j + 1] - rp[j]
        if deg == 0:
            P[:, j] = D / 60
        for e in range(rp[j], rp[j + 1]):
            P[col[e], j] += D / deg
    for levels in (1, 3, 7):
        res = od.d_iteration(rp, col, b, D, tol=0.0, max_levels=levels, dangling=True)
        np.testing.assert_allclose(res.F, b + P @ res.H - res.H, atol=1e-14)
        f, r = od.residual(rp, col, b, D, res.H, dangling=True)
        np.testing.assert_allclose(f, res.F, atol=1e-14)
        assert r == pytest.approx(np.abs(res.F).sum(), rel=1e-12)


def test_completion_power_iteration_agrees():
    rp, col = gg.generate(gg.GraphSpec(n=2000, mean_deg=5.0, seed=22, p_dangling=0.25))
    b = gg.uniform_b(2000, D)
    x, _ = od.power_iteration(rp, col, b, D, dangling=True)
    res = od.d_iteration(rp, col, b, D, tol=1e-14, dangling=True)
    assert np.abs(res.H - x).sum() <= 1e-12
