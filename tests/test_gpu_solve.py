"""Parity of the CUDA D-iteration (through the C ABI) with the CPU oracle.

Tolerances (written here, derived from the error bound |X - H|_1 <=
|F|_1 / (1 - d) of Sec. 2):
  * FP64 fluid: |H - X|_1 <= 1e-11 |X|_1, solving to tol = 1e-11 (1-d) |B|_1
    (|X|_1 >= |B|_1, so the bound gives 1e-11 |X|_1);
  * FP32 fluid / FP64 history: |H - X|_1 <= 1e-6 |X|_1 at tol = 1e-8 |B|_1;
  * the stop: the oracle's FP64 residual |B + P H - H|_1 of the returned H is
    <= tol and equals the reported residual.
X is the oracle's D-iteration run to 1e-14 |B|_1, itself pinned to exact and
dense solves on CPU.  Frontier sets (an integer decision) are compared
exactly, in the fluid's precision.
"""
import numpy as np
import pytest
import torch

from oracle import diter as od
from paper_1202_6168_gb300 import binding as di
from paper_1202_6168_gb300 import graphgen as gg

from graphs_util import csr_from_edges, random_graph

pytestmark = pytest.mark.gpu
D = 0.85


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def solve(rp, col, b, tol, fp64=False, h0=None, want_f=True, allow=(di.DI_OK,), window=False, **opt):
    g = di.Graph.create(rp, col)
    if window:   # the frontier push's shared-memory fluid window (propagations 3, 7)
        t = di.tune_default()
        t.push_window = 1
        di.set_tune(g, t)
    B = dev(b)
    H = dev(h0) if h0 is not None else torch.zeros(len(b), dtype=torch.float64, device="cuda")
    F = torch.zeros_like(H) if want_f else None
    o = di.opts_default(fluid_fp64=1 if fp64 else 0, warm_start=1 if h0 is not None else 0, **opt)
    rc, st = di.di_solve(g, B, D, tol, H, F, o, allow=allow)
    torch.cuda.synchronize()
    out = (H.cpu().numpy(), st, F.cpu().numpy() if want_f else None, rc)
    g.close()
    return out


def oracle_x(rp, col, b):
    r = od.d_iteration(rp, col, b, D, tol=1e-14 * max(np.abs(b).sum(), 1e-300))
    assert r.status == 0
    return r.H


def check_stop(rp, col, b, h, st, tol):
    """The oracle's FP64 residual of the returned H is within tol, and equals
    the reported one.  Each F_k = B_k + (P H)_k - H_k cancels terms far larger
    than F_k, so two FP64 evaluations of |F|_1 (different summation orders)
    differ by up to ~eps (|B|_1 + 2 |H|_1): that floor is allowed for."""
    f_cpu, r_cpu = od.residual(rp, col, b, D, h)
    floor = 64 * np.finfo(np.float64).eps * (np.abs(b).sum() + 2 * np.abs(h).sum())
    assert r_cpu <= tol * (1 + 1e-9) + floor
    assert abs(st.resid_l1 - r_cpu) <= 1e-9 * max(r_cpu, tol) + floor
    return f_cpu


def assert_residual_close(f_gpu, f_cpu, rp, col, b, h):
    """Elementwise FP64 agreement of two evaluations of F = B + P H - H that
    sum each in-row in different orders: |dF_k| <= 2 (m_k + 2) eps
    (|B_k| + (P|H|)_k + |H_k|), m_k the in-degree (recursive-summation bound)."""
    eps = np.finfo(np.float64).eps
    indeg = np.bincount(col, minlength=len(b))
    scale = np.abs(b) + od.p_times(rp, col, D, np.abs(h)) + np.abs(h)
    bound = 2 * (indeg + 2) * eps * scale
    err = np.abs(f_gpu - f_cpu)
    assert np.all(err <= bound + 1e-300), f"max excess {np.max(err - bound):.3e}"


@pytest.fixture(scope="module")
def web10k():
    rp, col = gg.generate(gg.SMALL_10K)
    b = gg.uniform_b(gg.SMALL_10K.n, D)
    return rp, col, b, oracle_x(rp, col, b)


@pytest.fixture(scope="module")
def web1m():
    rp, col = gg.generate(gg.WEB_1M)
    b = gg.uniform_b(gg.WEB_1M.n, D)
    return rp, col, b, oracle_x(rp, col, b)


# ---------------------------------------------------------------- single kernels

@pytest.mark.parametrize("fp64", [False, True])
def test_frontier_set_is_exact(web10k, fp64):
    rp, col, _, _ = web10k
    n = len(rp) - 1
    rng = np.random.default_rng(1)
    f = rng.standard_normal(n) * np.exp(rng.uniform(-20, 0, n))
    f = f.astype(np.float64 if fp64 else np.float32)
    g = di.Graph.create(rp, col)
    lst = torch.empty(n, dtype=torch.int32, device="cuda")
    for T in (0.0, 1e-9, np.quantile(np.abs(f), 0.5), float(np.abs(f).max()), 2.0):
        cnt, r, mx = di.di_frontier(g, dev(f), fp64, float(T), lst)
        got = np.sort(lst[:cnt].cpu().numpy())
        if fp64:
            want = np.nonzero(np.abs(f) >= T)[0]
        else:   # comparison in FP32: |F_i| >= T  <=>  |F_i| >= T rounded up to a float
            want = np.nonzero(np.abs(f).astype(np.float64) >= T)[0]
        np.testing.assert_array_equal(got, want)
        assert r == pytest.approx(np.abs(f.astype(np.float64)).sum(), rel=1e-5 if not fp64 else 1e-12)
        assert mx == float(np.abs(f).max())
    g.close()


def test_exact_residual_matches_oracle(web10k):
    rp, col, b, _ = web10k
    rng = np.random.default_rng(2)
    h = rng.standard_normal(len(b)) * 1e-4
    g = di.Graph.create(rp, col)
    F = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    r = di.di_residual(g, dev(b), D, dev(h), F)
    f_cpu, r_cpu = od.residual(rp, col, b, D, h)
    assert_residual_close(F.cpu().numpy(), f_cpu, rp, col, b, h)
    assert r == pytest.approx(r_cpu, rel=1e-13)
    g.close()


def test_residual_with_long_in_rows():
    # a star: node 0 receives an edge from every other node (in-degree 19999)
    n = 20000
    rp, col = csr_from_edges(n, [(j, 0) for j in range(1, n)] + [(0, 1)])
    rng = np.random.default_rng(3)
    h, b = rng.random(n), rng.random(n)
    g = di.Graph.create(rp, col)
    assert g.info()["max_indeg"] == n - 1
    F = torch.zeros(n, dtype=torch.float64, device="cuda")
    r = di.di_residual(g, dev(b), D, dev(h), F)
    f_cpu, r_cpu = od.residual(rp, col, b, D, h)
    assert_residual_close(F.cpu().numpy(), f_cpu, rp, col, b, h)
    assert r == pytest.approx(r_cpu, rel=1e-13)
    g.close()


# ---------------------------------------------------------------- full solves vs the oracle

def test_fp64_parity_web10k(web10k):
    rp, col, b, x = web10k
    tol = 1e-11 * (1 - D) * b.sum()
    h, st, f, _ = solve(rp, col, b, tol, fp64=True)
    assert np.abs(h - x).sum() <= 1e-11 * np.abs(x).sum()
    f_cpu = check_stop(rp, col, b, h, st, tol)
    assert_residual_close(f, f_cpu, rp, col, b, h)
    assert st.levels > 10 and st.edge_diffusions > len(col)


def test_fp32_parity_web10k(web10k):
    rp, col, b, x = web10k
    tol = 1e-8 * b.sum()
    h, st, f, _ = solve(rp, col, b, tol)
    assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()
    check_stop(rp, col, b, h, st, tol)
    assert st.recomputes >= 1


def test_config_tolerance_1e10_web10k(web10k):
    # the small workload's own stop rule: |F|_1 <= 1e-10, FP64
    rp, col, b, x = web10k
    h, st, _, _ = solve(rp, col, b, 1e-10, fp64=True, want_f=False)
    check_stop(rp, col, b, h, st, 1e-10)
    assert np.abs(h - x).sum() <= st.resid_l1 / (1 - D) * (1 + 1e-6)


@pytest.mark.parametrize("fp64", [False, True])
def test_parity_web1m(web1m, fp64):
    rp, col, b, x = web1m
    tol = (1e-11 * (1 - D) if fp64 else 1e-8) * b.sum()
    h, st, _, _ = solve(rp, col, b, tol, fp64=fp64, want_f=False)
    assert np.abs(h - x).sum() <= (1e-11 if fp64 else 1e-6) * np.abs(x).sum()
    check_stop(rp, col, b, h, st, tol)


def test_host_buffer_entry_point_matches(web10k):
    rp, col, b, x = web10k
    tol = 1e-8 * b.sum()
    g = di.Graph.create(rp, col)
    H = np.zeros(len(b))
    F = np.zeros(len(b))
    rc, st = di.di_solve_host(g, b, D, tol, H, F)
    assert np.abs(H - x).sum() <= 1e-6 * np.abs(x).sum()
    f_cpu = check_stop(rp, col, b, H, st, tol)
    assert_residual_close(F, f_cpu, rp, col, b, H)
    g.close()


# ---------------------------------------------------------------- edge cases

@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("case", ["single", "two_cycle", "all_dangling", "path", "ragged", "selfloop_dups",
                                  "personalised", "complete"])
def test_edge_cases(case, fp64):
    rng = np.random.default_rng(hash(case) % 1000)
    if case == "single":
        rp, col = csr_from_edges(1, [])
        b = np.array([0.15])
    elif case == "two_cycle":
        rp, col = csr_from_edges(2, [(0, 1), (1, 0)])
        b = np.array([0.15, 0.15])
    elif case == "all_dangling":
        rp, col = csr_from_edges(5000, [])
        b = rng.random(5000)
    elif case == "path":
        rp, col = csr_from_edges(300, [(k, k + 1) for k in range(299)])
        b = np.full(300, 0.01)
    elif case == "ragged":
        rp, col = gg.generate(gg.GraphSpec(n=2048 * 3 + 1, mean_deg=9, seed=5))
        b = gg.uniform_b(len(rp) - 1)
    elif case == "selfloop_dups":
        rp, col = random_graph(3000, rng, max_deg=40)
        b = rng.random(3000) * 1e-3
    elif case == "personalised":
        rp, col = gg.generate(gg.GraphSpec(n=20000, mean_deg=8, seed=6))
        b = gg.personalised_b(20000, 123)
    else:
        n = 40
        rp, col = csr_from_edges(n, [(i, j) for i in range(n) for j in range(n) if i != j])
        b = np.full(n, (1 - D) / n)
    x = oracle_x(rp, col, b)
    tol = (1e-11 * (1 - D) if fp64 else 1e-8) * b.sum()
    h, st, f, _ = solve(rp, col, b, tol, fp64=fp64)
    assert np.abs(h - x).sum() <= (1e-11 if fp64 else 1e-6) * np.abs(x).sum()
    check_stop(rp, col, b, h, st, tol)


def test_empty_edge_set_and_zero_b():
    rp, col = csr_from_edges(100, [])
    h, st, _, rc = solve(rp, col, np.zeros(100), 1e-12)
    assert rc == di.DI_OK and st.node_diffusions == 0 and np.all(h == 0)


def test_hot_targets_are_privatised_and_exact():
    # every node links to node 0 and to a neighbour: node 0 is a hot target
    n = 50000
    edges = [(j, 0) for j in range(1, n)] + [(j, (j + 1) % n) for j in range(n)]
    rp, col = csr_from_edges(n, edges)
    b = gg.uniform_b(n)
    g = di.Graph.create(rp, col)
    assert g.info()["n_hot"] >= 1
    g.close()
    x = oracle_x(rp, col, b)
    for fp64 in (False, True):
        tol = (1e-11 * (1 - D) if fp64 else 1e-8) * b.sum()
        h, st, _, _ = solve(rp, col, b, tol, fp64=fp64)
        assert np.abs(h - x).sum() <= (1e-11 if fp64 else 1e-6) * np.abs(x).sum()


# ---------------------------------------------------------------- warm start and statuses

def test_warm_start_at_solution_does_no_work(web10k):
    rp, col, b, x = web10k
    h, st, _, _ = solve(rp, col, b, 1e-10 * b.sum(), fp64=True, h0=x)
    assert st.warm_used == 1 and st.node_diffusions == 0
    assert st.f0_l1 <= 1e-12


def test_warm_start_near_solution_converges(web10k):
    rp, col, b, x = web10k
    rng = np.random.default_rng(4)
    h0 = x * (1 + 0.2 * rng.standard_normal(len(x)))
    for fp64 in (False, True):
        tol = (1e-11 * (1 - D) if fp64 else 1e-8) * b.sum()
        h, st, _, _ = solve(rp, col, b, tol, fp64=fp64, h0=h0)
        assert st.warm_used == 1 and st.f0_l1 < st.b_l1
        assert np.abs(h - x).sum() <= (1e-11 if fp64 else 1e-6) * np.abs(x).sum()
        check_stop(rp, col, b, h, st, tol)


def test_warm_start_fallback_on_garbage(web10k):
    rp, col, b, x = web10k
    h0 = np.full(len(b), 1.0)
    h, st, _, _ = solve(rp, col, b, 1e-8 * b.sum(), h0=h0)
    assert st.warm_used == 0 and st.f0_l1 == pytest.approx(st.b_l1)
    assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()


@pytest.mark.parametrize("cap", [1, 3, 4])
def test_level_cap_reports_no_convergence(web10k, cap):
    # the level graph runs two levels per WHILE iteration: caps that stop the
    # loop at the first and at the second level of an iteration
    rp, col, b, x = web10k
    h, st, f, rc = solve(rp, col, b, 1e-12, max_levels=cap, allow=(di.DI_ENOCONV,))
    assert rc == di.DI_ENOCONV and st.levels == cap
    f_cpu, r_cpu = od.residual(rp, col, b, D, h)
    assert st.resid_l1 == pytest.approx(r_cpu, rel=1e-12)
    assert_residual_close(f, f_cpu, rp, col, b, h)


def test_non_finite_b_is_reported(web10k):
    rp, col, b, _ = web10k
    bad = b.copy()
    bad[17] = np.nan
    _, _, _, rc = solve(rp, col, bad, 1e-8, allow=(di.DI_ENONFINITE,))
    assert rc == di.DI_ENONFINITE


def test_invalid_inputs_are_rejected():
    rp, col = csr_from_edges(3, [(0, 1), (1, 2)])
    with pytest.raises(di.DiError) as e:
        di.Graph.create(rp, np.array([0, 5], dtype=np.int32))
    assert e.value.status == di.DI_EINVAL
    with pytest.raises(di.DiError):
        di.Graph.create(np.array([0, 2, 1, 2], dtype=np.int64), col)
    g = di.Graph.create(rp, col)
    B = dev(np.ones(3))
    H = torch.zeros(3, dtype=torch.float64, device="cuda")
    for d, tol in ((1.0, 1e-8), (0.0, 1e-8), (0.85, 0.0), (0.85, -1.0), (0.85, float("nan"))):
        with pytest.raises(di.DiError) as e:
            di.di_solve(g, B, d, tol, H)
        assert e.value.status == di.DI_EINVAL
    for drop in (0.5, 1.0, -2.0, float("inf"), float("nan")):
        with pytest.raises(di.DiError) as e:
            di.di_solve(g, B, D, 1e-8, H, None, di.opts_default(recompute_drop=drop))
        assert e.value.status == di.DI_EINVAL
    g.close()


@pytest.mark.parametrize("every,drop", [(0, 1024.0), (8, 0.0), (3, 16.0), (0, 0.0)])
def test_refinement_schedules(web10k, every, drop):
    # exact FP64 recomputations every `every` levels and/or whenever |F|_1 fell
    # by `drop`; (0, 0) leaves only the confirmations of stop requests.  Any
    # schedule reaches the same X within the FP32 tolerance and stops on an
    # exact residual below tol.
    rp, col, b, x = web10k
    tol = 1e-8 * b.sum()
    h, st, f, _ = solve(rp, col, b, tol, recompute_every=every, recompute_drop=drop)
    assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()
    check_stop(rp, col, b, h, st, tol)
    assert st.recomputes >= 1
    if every:
        assert st.recomputes >= st.levels // every
    if drop:
        # one recomputation at least per factor `drop` of the residual's fall
        assert st.recomputes >= int(np.log(b.sum() / tol) / np.log(drop))


def test_device_resident_csr_input(web10k):
    rp, col, b, x = web10k
    g = di.Graph.create(dev(rp), dev(col), on_device=True)
    H = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    di.di_solve(g, dev(b), D, 1e-8 * b.sum(), H)
    assert np.abs(H.cpu().numpy() - x).sum() <= 1e-6 * np.abs(x).sum()
    g.close()


# ---------------------------------------------------------------- every propagation mode

@pytest.mark.parametrize("prop", [0, 1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("fp64", [False, True])
def test_parity_every_propagation_mode(web10k, prop, fp64):
    rp, col, b, x = web10k
    tol = (1e-11 * (1 - D) if fp64 else 1e-8) * b.sum()
    for alpha in (1.5, 2.0):
        h, st, f, _ = solve(rp, col, b, tol, fp64=fp64, propagation=prop, alpha=alpha)
        assert np.abs(h - x).sum() <= (1e-11 if fp64 else 1e-6) * np.abs(x).sum(), (prop, alpha)
        check_stop(rp, col, b, h, st, tol)


@pytest.mark.parametrize("prop", [3, 4, 5, 6, 7])
@pytest.mark.parametrize("resweeps", [0, 1, 2])
def test_parity_every_resweep_count(web10k, prop, resweeps):
    # re-selections at the same threshold change the order of the diffusions,
    # not the limit (Sec. 2: any order that keeps diffusing every node)
    rp, col, b, x = web10k
    for fp64, rel in ((False, 1e-6), (True, 1e-11)):
        tol = (1e-11 * (1 - D) if fp64 else 1e-8) * b.sum()
        h, st, f, _ = solve(rp, col, b, tol, fp64=fp64, propagation=prop, resweeps=resweeps)
        assert np.abs(h - x).sum() <= rel * np.abs(x).sum()
        check_stop(rp, col, b, h, st, tol)
        assert st.body_iterations >= st.levels


def test_resweeps_out_of_range_are_rejected(web10k):
    rp, col, b, _ = web10k
    g = di.Graph.create(rp, col)
    H = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    for bad in (-1, 9):
        with pytest.raises(di.DiError) as e:
            di.di_solve(g, dev(b), D, 1e-8, H, None, di.opts_default(resweeps=bad))
        assert e.value.status == di.DI_EINVAL
    g.close()


@pytest.mark.parametrize("prop", [3, 7])
@pytest.mark.parametrize("sweeps", [1, 2, 4])
def test_parity_every_slice_sweep_count(web10k, prop, sweeps):
    # slice sweeps diffuse, in the same level, nodes whose fluid crossed T
    # while the level pushed: another order of the diffusions, the same limit
    # (Sec. 2: any order that keeps diffusing every node)
    rp, col, b, x = web10k
    for fp64, rel in ((False, 1e-6), (True, 1e-11)):
        tol = (1e-11 * (1 - D) if fp64 else 1e-8) * b.sum()
        h, st, f, _ = solve(rp, col, b, tol, fp64=fp64, propagation=prop, slice_sweeps=sweeps)
        assert np.abs(h - x).sum() <= rel * np.abs(x).sum(), (fp64, sweeps)
        check_stop(rp, col, b, h, st, tol)
        assert 0 < st.slice_nodes < st.node_diffusions


def test_slice_sweeps_with_resweeps_and_persistent_timing(web10k):
    rp, col, b, x = web10k
    tol = 1e-8 * b.sum()
    for prop, timing in ((3, 0), (3, 1), (7, 0), (7, 1)):
        h, st, _, _ = solve(rp, col, b, tol, propagation=prop, slice_sweeps=1, resweeps=1, timing=timing)
        assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum(), (prop, timing)
        check_stop(rp, col, b, h, st, tol)
        assert st.slice_nodes > 0 and st.body_iterations >= st.levels


@pytest.fixture(scope="module")
def web100k():
    spec = gg.GraphSpec(n=100_000, mean_deg=10.0, window=64, seed=0)
    rp, col = gg.generate(spec)
    b = gg.uniform_b(spec.n, D)
    return rp, col, b, oracle_x(rp, col, b)


def test_slice_sweeps_cut_the_diffusions(web100k):
    # a level that selects its frontier first diffuses each node at most once;
    # the sequential sweep also diffuses the nodes whose fluid crosses T before
    # their turn.  Slice sweeps recover most of that: far fewer elementary
    # diffusions to the same tolerance, and no more levels.
    rp, col, b, x = web100k
    tol = 1e-8 * b.sum()
    runs = {}
    for sweeps in (0, 1, 2):
        h, st, _, _ = solve(rp, col, b, tol, propagation=3, slice_sweeps=sweeps)
        assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()
        check_stop(rp, col, b, h, st, tol)
        runs[sweeps] = st
    assert runs[0].slice_nodes == 0
    assert runs[1].edge_diffusions < 0.8 * runs[0].edge_diffusions
    assert runs[2].edge_diffusions < 0.8 * runs[0].edge_diffusions
    assert runs[1].levels <= runs[0].levels
    # the oracle's sequential sweep, for scale (the same graph and tolerance)
    seq = od.d_iteration(rp, col, b, D, tol=tol)
    assert runs[1].edge_diffusions < 1.5 * seq.edge_diffusions   # measured: 1.22x


def test_slice_sweeps_on_many_segments(web5m):
    # about 5.5e3 nodes per CTA slice: several 1024-node segments and queue
    # batches per sweep; two source blocks in the exact residual
    rp, col, b = web5m
    tol = 1e-8 * b.sum()
    h0, st0, _, _ = solve(rp, col, b, tol, propagation=3)
    h, st, _, _ = solve(rp, col, b, tol, propagation=3, slice_sweeps=2)
    check_stop(rp, col, b, h, st, tol)
    assert st.slice_nodes > 0 and st.edge_diffusions < st0.edge_diffusions
    # both are within |F|_1 / (1 - d) of X, so within twice that of each other
    assert np.abs(h - h0).sum() <= 2 * tol / (1 - D) * 1.01


def test_slice_sweeps_on_tiny_and_ragged_graphs():
    # fewer nodes than push CTAs: most slices are empty, the last is ragged
    rng = np.random.default_rng(71)
    for n in (1, 7, 1001):
        rp, col = random_graph(n, rng)
        b = rng.random(n) + 0.1
        x = oracle_x(rp, col, b)
        for fp64 in (False, True):
            tol = (1e-11 * (1 - D) if fp64 else 1e-8) * b.sum()
            h, st, _, _ = solve(rp, col, b, tol, fp64=fp64, propagation=3, slice_sweeps=3)
            assert np.abs(h - x).sum() <= (1e-11 if fp64 else 1e-6) * np.abs(x).sum(), (n, fp64)
            check_stop(rp, col, b, h, st, tol)


def test_slice_sweeps_with_dangling_completion_and_warm_start(web10k_completed):
    rp, col, b, x = web10k_completed
    tol = 1e-8 * b.sum()
    for prop in (3, 7):
        h, st, _, _ = solve(rp, col, b, tol, propagation=prop, dangling=1, slice_sweeps=1)
        assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()
        check_stop_completed(rp, col, b, h, st, tol)
        assert st.slice_nodes > 0
    # a warm start: signed fluid, selected on |F_i|
    rng = np.random.default_rng(45)
    h0 = x * (1 + 0.05 * rng.standard_normal(len(x)))
    h, st, _, _ = solve(rp, col, b, tol, h0=h0, propagation=3, dangling=1, slice_sweeps=2)
    assert st.warm_used == 1
    assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()
    check_stop_completed(rp, col, b, h, st, tol)


def test_slice_sweeps_turn_the_fluid_window_off(web10k):
    rp, col, b, x = web10k
    tol = 1e-8 * b.sum()
    h, st, _, _ = solve(rp, col, b, tol, propagation=3, slice_sweeps=1, window=True)
    assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()
    check_stop(rp, col, b, h, st, tol)
    assert st.slice_nodes > 0 and st.red_ops > 0


def test_slice_sweeps_without_the_wait(web10k):
    # spin_limit = 0: the push's wait for the frontier gives up at once, so
    # the sweeps run while frontier tiles are still pushing (nodes drained
    # twice, crossings missed): the result must not change beyond the tolerance
    rp, col, b, x = web10k
    for fp64, rel in ((False, 1e-6), (True, 1e-11)):
        tol = (1e-11 * (1 - D) if fp64 else 1e-8) * b.sum()
        for prop in (3, 7):
            opts = dict(slice_sweeps=2) if prop == 3 else dict(slice_sweeps=1)   # propagation 7's barriers need time
            h, st, _, _ = solve(rp, col, b, tol, fp64=fp64, propagation=prop, spin_limit=0 if prop == 3 else 1 << 20,
                                **opts)
            assert np.abs(h - x).sum() <= rel * np.abs(x).sum(), (fp64, prop)
            check_stop(rp, col, b, h, st, tol)


def test_slice_sweeps_rejections(web10k):
    rp, col, b, _ = web10k
    g = di.Graph.create(rp, col)
    H = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    bad = [dict(slice_sweeps=-2), dict(slice_sweeps=5)]
    bad += [dict(slice_sweeps=1, propagation=p) for p in (0, 1, 2, 4, 5, 6)]
    bad.append(dict(slice_sweeps=1, selection=1))
    for opt in bad:
        with pytest.raises(di.DiError) as e:
            di.di_solve(g, dev(b), D, 1e-8, H, None, di.opts_default(**opt))
        assert e.value.status == di.DI_EINVAL, opt
    g.close()


@pytest.mark.parametrize("prop", [0, 1, 2, 3, 4, 5, 6, 7])
def test_personalised_sparse_levels_every_mode(prop):
    # a personalised right-hand side keeps the early frontiers tiny (scatter levels)
    rp, col = gg.generate(gg.GraphSpec(n=30000, mean_deg=9, seed=8))
    b = gg.personalised_b(30000, 4242)
    x = oracle_x(rp, col, b)
    tol = 1e-8 * b.sum()
    h, st, _, _ = solve(rp, col, b, tol, propagation=prop)
    assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()
    check_stop(rp, col, b, h, st, tol)


@pytest.mark.parametrize("prop", [1, 3, 5, 6, 7])
def test_timing_mode_matches(web10k, prop):
    rp, col, b, x = web10k
    tol = 1e-8 * b.sum()
    h, st, _, _ = solve(rp, col, b, tol, propagation=prop, timing=1)
    assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()
    assert st.level_seconds > 0 and st.level_launches > 0
    check_stop(rp, col, b, h, st, tol)


# ---------------------------------------------------------------- both forms of the exact residual

@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("fp64", [False, True])
def test_parity_every_residual_form(web10k, form, fp64):
    rp, col, b, x = web10k
    tol = (1e-11 * (1 - D) if fp64 else 1e-8) * b.sum()
    h, st, f, _ = solve(rp, col, b, tol, fp64=fp64, exact_residual=form)
    assert np.abs(h - x).sum() <= (1e-11 if fp64 else 1e-6) * np.abs(x).sum()
    f_cpu = check_stop(rp, col, b, h, st, tol)
    assert_residual_close(f, f_cpu, rp, col, b, h)


@pytest.mark.parametrize("form", [1, 2])
def test_warm_start_every_residual_form(web10k, form):
    rp, col, b, x = web10k
    rng = np.random.default_rng(14)
    h0 = x * (1 + 0.2 * rng.standard_normal(len(x)))
    tol = 1e-8 * b.sum()
    h, st, _, _ = solve(rp, col, b, tol, h0=h0, exact_residual=form)
    _, f0 = od.residual(rp, col, b, D, h0)
    assert st.f0_l1 == pytest.approx(f0, rel=1e-12)
    assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()
    check_stop(rp, col, b, h, st, tol)


@pytest.mark.parametrize("nnz", [0, 1, 2047, 2048, 4096, 6143, 2048 * 37 + 5])
def test_blocked_residual_ragged_edge_counts(nnz):
    # the flat gather takes 8 in-edges per thread with vector loads and
    # clips the last group: edge counts around those boundaries, none, one
    rng = np.random.default_rng(nnz + 1)
    n = 3000
    src = rng.integers(0, n, size=nnz)
    dst = rng.integers(0, n, size=nnz)
    rp, col = csr_from_edges(n, list(zip(src.tolist(), dst.tolist())))
    assert len(col) == nnz
    h, b = rng.random(n), rng.random(n)
    g = di.Graph.create(rp, col)
    F = torch.zeros(n, dtype=torch.float64, device="cuda")
    r = di.di_residual(g, dev(b), D, dev(h), F)
    f_cpu, r_cpu = od.residual(rp, col, b, D, h)
    assert_residual_close(F.cpu().numpy(), f_cpu, rp, col, b, h)
    assert r == pytest.approx(r_cpu, rel=1e-13)
    g.close()


def hub_csr(n, seed):
    """Every node j links to node 0, to hub 1 + j % 3 and to one random node
    (self-loops and duplicates kept): destination runs of n and n / 3 edges."""
    rng = np.random.default_rng(seed)
    col = np.stack([np.zeros(n, dtype=np.int64), 1 + np.arange(n) % 3, rng.integers(0, n, size=n)], axis=1)
    return np.arange(0, 3 * n + 1, 3, dtype=np.int64), col.reshape(-1).astype(np.int32)


@pytest.mark.parametrize("n", [200_000, (1 << 22) + 5000])
def test_blocked_residual_hub_destinations(n):
    # the runs of equal destination span thousands of lanes and warps (and,
    # above 2^22 nodes, both source blocks): the residual sums them over the
    # warp before each reduction; every value must still be added once
    rp, col = hub_csr(n, n)
    rng = np.random.default_rng(n + 1)
    h, b = rng.random(n), rng.random(n)
    g = di.Graph.create(rp, col)
    F = torch.zeros(n, dtype=torch.float64, device="cuda")
    f_cpu, r_cpu = od.residual(rp, col, b, D, h)
    for _ in range(2):
        r = di.di_residual(g, dev(b), D, dev(h), F)
        assert_residual_close(F.cpu().numpy(), f_cpu, rp, col, b, h)
        assert r == pytest.approx(r_cpu, rel=1e-13)
    g.close()


def test_hub_destinations_solve_matches_oracle():
    rp, col = hub_csr(60_000, 3)
    b = gg.uniform_b(60_000, D)
    tol = 1e-8 * b.sum()
    h, st, f, _ = solve(rp, col, b, tol)
    x = oracle_x(rp, col, b)
    assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()
    f_cpu = check_stop(rp, col, b, h, st, tol)
    assert_residual_close(f, f_cpu, rp, col, b, h)


@pytest.mark.parametrize("edges_per_node", [5.6, 11.2])
def test_blocked_residual_many_grid_strides(edges_per_node):
    # uniformly random in-edges (no locality) and enough of them that every
    # thread of the grid loops several times; repeated calls agree with the
    # oracle each time
    rng = np.random.default_rng(int(edges_per_node * 10))
    n = 1_000_000
    nnz = int(n * edges_per_node) + 777
    src = np.sort(rng.integers(0, n, size=nnz))
    col = rng.integers(0, n, size=nnz).astype(np.int32)
    rp = np.concatenate(([0], np.cumsum(np.bincount(src, minlength=n)))).astype(np.int64)
    h, b = rng.random(n), rng.random(n)
    g = di.Graph.create(rp, col)
    F = torch.zeros(n, dtype=torch.float64, device="cuda")
    f_cpu, r_cpu = od.residual(rp, col, b, D, h)
    for _ in range(3):
        r = di.di_residual(g, dev(b), D, dev(h), F)
        assert_residual_close(F.cpu().numpy(), f_cpu, rp, col, b, h)
        assert r == pytest.approx(r_cpu, rel=1e-13)
    g.close()


@pytest.fixture(scope="module")
def web5m():
    """More than 2^22 nodes: the exact residual runs over two source blocks."""
    spec = gg.GraphSpec(n=5_000_000, mean_deg=6.0, window=256, seed=3)
    rp, col = gg.generate(spec)
    return rp, col, gg.uniform_b(spec.n)


def test_blocked_residual_spans_source_blocks(web5m):
    rp, col, b = web5m
    rng = np.random.default_rng(15)
    h = rng.random(len(b)) * 2e-7
    g = di.Graph.create(rp, col)
    F = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    r = di.di_residual(g, dev(b), D, dev(h), F)
    f_cpu, r_cpu = od.residual(rp, col, b, D, h)
    assert_residual_close(F.cpu().numpy(), f_cpu, rp, col, b, h)
    assert r == pytest.approx(r_cpu, rel=1e-13)
    g.close()


def test_solve_on_two_source_blocks_meets_the_stop(web5m):
    rp, col, b = web5m
    tol = 1e-8 * b.sum()
    h, st, f, _ = solve(rp, col, b, tol, propagation=4)
    assert st.recomputes >= 1
    f_cpu = check_stop(rp, col, b, h, st, tol)
    assert_residual_close(f, f_cpu, rp, col, b, h)
    # H below X and within the error bound of it: |X - H|_1 <= |F|_1 / (1 - d)
    # (checked against the oracle's solution at a sample of nodes would need
    # its full solve; the bound and the exact residual pin the result here)
    assert np.all(h >= 0)


# ---------------------------------------------------------------- push shapes and the autotuner

@pytest.mark.parametrize("prop", [3, 4, 5, 6, 7])
@pytest.mark.parametrize("shape", [(1, 1, 0), (4, 64, 1), (32, 32, 0), (1024, 1 << 30, 2)])
def test_parity_every_push_shape(web10k, prop, shape):
    rp, col, b, x = web10k
    g = di.Graph.create(rp, col)
    t = di.tune_default()
    t.thread_max_deg, t.warp_max_deg, t.push_ctas_per_sm = shape
    di.set_tune(g, t)
    assert di.get_tune(g).as_dict() == t.as_dict()
    H = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    tol = 1e-8 * b.sum()
    _, st = di.di_solve(g, dev(b), D, tol, H, None, di.opts_default(propagation=prop))
    h = H.cpu().numpy()
    assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()
    check_stop(rp, col, b, h, st, tol)
    g.close()


def test_autotune_keeps_a_shape_and_caches_it(web10k, tmp_path):
    rp, col, b, x = web10k
    g = di.Graph.create(rp, col)
    cache = str(tmp_path / "tune.jsonl")
    tol = 1e-8 * b.sum()
    t, secs = di.autotune(g, dev(b), D, tol, None, cache)
    assert secs > 0 and 1 <= t.thread_max_deg <= 1024
    assert di.get_tune(g).as_dict() == t.as_dict()
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and '"key": "solve n=2^13' in lines[0]
    # a second graph of the same size bucket takes the cached shape without timing
    g2 = di.Graph.create(rp, col)
    t2, secs2 = di.autotune(g2, dev(b), D, tol, None, cache)
    assert secs2 == 0.0 and t2.as_dict() == t.as_dict()
    H = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    _, st = di.di_solve(g2, dev(b), D, tol, H)
    assert np.abs(H.cpu().numpy() - x).sum() <= 1e-6 * np.abs(x).sum()
    bad = di.tune_default()
    bad.thread_max_deg = 0
    with pytest.raises(di.DiError):
        di.set_tune(g, bad)
    g.close()
    g2.close()


# ---------------------------------------------------------------- weighted selection (Sec. 2.4 score)

@pytest.mark.parametrize("prop", [3, 4, 7])
@pytest.mark.parametrize("fp64", [False, True])
def test_weighted_selection_parity(web10k, prop, fp64):
    rp, col, b, x = web10k
    tol = (1e-11 * (1 - D) if fp64 else 1e-8) * b.sum()
    h, st, f, _ = solve(rp, col, b, tol, fp64=fp64, propagation=prop, selection=1)
    assert np.abs(h - x).sum() <= (1e-11 if fp64 else 1e-6) * np.abs(x).sum()
    f_cpu = check_stop(rp, col, b, h, st, tol)
    assert_residual_close(f, f_cpu, rp, col, b, h)


def test_weighted_selection_personalised_and_warm():
    rp, col = gg.generate(gg.GraphSpec(n=30000, mean_deg=9, seed=8))
    b = gg.personalised_b(30000, 4242)
    x = oracle_x(rp, col, b)
    tol = 1e-8 * b.sum()
    h, st, _, _ = solve(rp, col, b, tol, selection=1)
    assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()
    check_stop(rp, col, b, h, st, tol)
    rng = np.random.default_rng(16)
    h0 = x * (1 + 0.1 * rng.standard_normal(len(x)))
    h, st, _, _ = solve(rp, col, b, tol, h0=h0, selection=1)
    assert st.warm_used == 1
    assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()
    check_stop(rp, col, b, h, st, tol)


def test_weighted_selection_needs_a_selection_kernel(web10k):
    rp, col, b, _ = web10k
    g = di.Graph.create(rp, col)
    H = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    for prop in (0, 1, 2, 5, 6):
        with pytest.raises(di.DiError) as e:
            di.di_solve(g, dev(b), D, 1e-8, H, None, di.opts_default(propagation=prop, selection=1))
        assert e.value.status == di.DI_EINVAL
    with pytest.raises(di.DiError):
        di.di_solve(g, dev(b), D, 1e-8, H, None, di.opts_default(selection=2))
    g.close()


# ---------------------------------------------------------------- 1/N completion of dangling columns (Sec. 2.2)

@pytest.fixture(scope="module")
def web10k_completed():
    rp, col = gg.generate(gg.SMALL_10K)
    b = gg.uniform_b(gg.SMALL_10K.n, D)
    r = od.d_iteration(rp, col, b, D, tol=1e-14 * b.sum(), dangling=True)
    assert r.status == 0
    return rp, col, b, r.H


def check_stop_completed(rp, col, b, h, st, tol):
    """As check_stop, for the completed P.  Every F_k then holds the same term
    (d/N) sum_dangling H_j, so the rounding of that one sum (recursive
    summation: at most n_dangling eps sum|H_j| on each side) shifts all N
    residual elements alike and adds up coherently in |F|_1: the allowance
    grows by 2 d n_dangling eps sum_dangling |H_j|."""
    f_cpu, r_cpu = od.residual(rp, col, b, D, h, dangling=True)
    eps = np.finfo(np.float64).eps
    dang = np.diff(rp) == 0
    floor = 64 * eps * (np.abs(b).sum() + 2 * np.abs(h).sum())
    floor += 2 * D * dang.sum() * eps * np.abs(h[dang]).sum()
    assert r_cpu <= tol * (1 + 1e-9) + floor
    assert abs(st.resid_l1 - r_cpu) <= 1e-9 * max(r_cpu, tol) + floor
    return f_cpu


def assert_completed_residual_close(f_gpu, f_cpu, rp, col, b, h):
    """Elementwise agreement of two FP64 evaluations of F = B + P_c H - H with
    the completed P_c: the recursive-summation bound of each in-row sum, as in
    assert_residual_close, with P_c |H| in the scale, plus the rounding of the
    one sum over the dangling nodes that every row shares (n_dangling eps
    sum_dangling |H_j| on each side, times d / N)."""
    eps = np.finfo(np.float64).eps
    n = len(b)
    dang = np.diff(rp) == 0
    indeg = np.bincount(col, minlength=n)
    shared = D / n * np.abs(h[dang]).sum()
    scale = np.abs(b) + od.p_times(rp, col, D, np.abs(h)) + shared + np.abs(h)
    bound = 2 * (indeg + 2) * eps * scale + 2 * dang.sum() * eps * shared
    err = np.abs(f_gpu - f_cpu)
    assert np.all(err <= bound + 1e-300), f"max excess {np.max(err - bound):.3e}"


@pytest.mark.parametrize("prop", [3, 4, 5, 6, 7])
@pytest.mark.parametrize("fp64", [False, True])
def test_dangling_completion_matches_oracle(web10k_completed, prop, fp64):
    rp, col, b, x = web10k_completed
    assert np.sum(np.diff(rp) == 0) > 500          # about 10% of the nodes are dangling
    tol = (1e-11 * (1 - D) if fp64 else 1e-8) * b.sum()
    h, st, f, _ = solve(rp, col, b, tol, fp64=fp64, propagation=prop, dangling=1)
    assert np.abs(h - x).sum() <= (1e-11 if fp64 else 1e-6) * np.abs(x).sum()
    f_cpu = check_stop_completed(rp, col, b, h, st, tol)
    assert_completed_residual_close(f, f_cpu, rp, col, b, h)
    # the completed columns are stochastic: 1'H is within the error bound of 1'X = 1
    assert abs(h.sum() - 1.0) <= st.resid_l1 / (1 - D) * 1.001 + 1e-12


def test_dangling_completion_personalised_and_warm(web10k_completed):
    rp, col, b, x = web10k_completed
    # a personalised right-hand side (sparse early levels)
    bp = gg.personalised_b(len(b), 1234)
    xp = od.d_iteration(rp, col, bp, D, tol=1e-14 * bp.sum(), dangling=True).H
    for prop in (4, 5, 6, 7):
        h, st, _, _ = solve(rp, col, bp, 1e-8 * bp.sum(), propagation=prop, dangling=1)
        assert np.abs(h - xp).sum() <= 1e-6 * np.abs(xp).sum()
        check_stop_completed(rp, col, bp, h, st, 1e-8 * bp.sum())
    # a warm start: F0 = B + P H0 - H0 with the completed P (small enough that
    # the start is kept: |F0|_1 <= |B|_1)
    rng = np.random.default_rng(44)
    h0 = x * (1 + 0.05 * rng.standard_normal(len(x)))
    h, st, _, _ = solve(rp, col, b, 1e-8 * b.sum(), h0=h0, propagation=3, dangling=1)
    _, f0 = od.residual(rp, col, b, D, h0, dangling=True)
    assert f0 < b.sum() and st.warm_used == 1
    assert st.f0_l1 == pytest.approx(f0, rel=1e-12)
    assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()
    check_stop_completed(rp, col, b, h, st, 1e-8 * b.sum())


@pytest.mark.parametrize("prop", [4, 5, 6, 7])
def test_dangling_completion_on_two_source_blocks(web5m, prop):
    # more than 2^22 nodes: the dangling sum of the exact residual spans both blocks
    rp, col, b = web5m
    tol = 1e-8 * b.sum()
    h, st, f, _ = solve(rp, col, b, tol, propagation=prop, dangling=1)
    assert st.recomputes >= 1
    f_cpu = check_stop_completed(rp, col, b, h, st, tol)
    assert_completed_residual_close(f, f_cpu, rp, col, b, h)
    assert abs(h.sum() - 1.0) <= st.resid_l1 / (1 - D) * 1.001 + 1e-9


def test_dangling_completion_rejects_unsupported_modes():
    rp, col = csr_from_edges(3, [(0, 1), (1, 2)])
    g = di.Graph.create(rp, col)
    B = dev(np.ones(3))
    H = torch.zeros(3, dtype=torch.float64, device="cuda")
    for opt in (dict(dangling=2), dict(dangling=1, propagation=2), dict(dangling=1, propagation=0),
                dict(dangling=1, exact_residual=1)):
        with pytest.raises(di.DiError) as e:
            di.di_solve(g, B, D, 1e-8, H, None, di.opts_default(**opt))
        assert e.value.status == di.DI_EINVAL
    batch = di.Batch([g], [1])
    with pytest.raises(di.DiError) as e:
        di.di_solve_batched(batch, [B], D, 1e-8, [H], di.opts_default(dangling=2))
    assert e.value.status == di.DI_EINVAL
    batch.close()
    g.close()


@pytest.mark.parametrize("case", ["ragged", "single", "tiny_mixed"])
def test_dangling_completion_edge_cases(case):
    # the uniform add skips the zero padding of the fluid past N (N not a
    # multiple of 4), a lone dangling node (X = B / (1 - d)), and a graph
    # where most nodes are dangling
    if case == "ragged":
        rp, col = gg.generate(gg.GraphSpec(n=10007, mean_deg=7.0, seed=31))
        b = gg.uniform_b(10007, D)
    elif case == "single":
        rp, col = csr_from_edges(1, [])
        b = np.array([0.15])
    else:
        rp, col = csr_from_edges(7, [(0, 1), (1, 2), (2, 0), (3, 0)])
        b = np.array([0.01, 0.02, 0.0, 0.05, 0.03, 0.0, 0.04])
    x = od.d_iteration(rp, col, b, D, tol=1e-15 * b.sum(), dangling=True).H
    if case == "single":
        assert x[0] == pytest.approx(0.15 / (1 - D), rel=1e-13)
    for fp64, rel in ((False, 1e-6), (True, 1e-11)):
        tol = (1e-11 * (1 - D) if fp64 else 1e-8) * b.sum()
        for prop in (3, 5, 6, 7):
            h, st, f, _ = solve(rp, col, b, tol, fp64=fp64, propagation=prop, dangling=1)
            assert np.abs(h - x).sum() <= rel * np.abs(x).sum()
            check_stop_completed(rp, col, b, h, st, tol)


# ---------------------------------------------------------------- propagation 6: on-chip window and hot slots

def ring_graph(n, reach):
    """Every node j points to j+1 .. j+reach (mod n): all edges local."""
    edges = [(j, (j + k) % n) for j in range(n) for k in range(1, reach + 1)]
    return csr_from_edges(n, edges)


@pytest.mark.parametrize("prop", [3, 6, 7])
@pytest.mark.parametrize("case", ["ring", "random", "ragged", "tiny", "hub_and_ring"])
@pytest.mark.parametrize("fp64", [False, True])
def test_fluid_window_cases(prop, case, fp64):
    # ring: every target lies in the shared-memory window (wrap-around edges
    # at both ends of the node range go to global memory); random: no
    # locality, the window radius is 0; ragged: N not a multiple of the chunk;
    # tiny: N below one chunk; hub_and_ring: a target of very high in-degree
    # (a hot slot) that is also inside the window of its sources
    rng = np.random.default_rng({"ring": 1, "random": 2, "ragged": 3, "tiny": 4, "hub_and_ring": 5}[case])
    if case == "ring":
        rp, col = ring_graph(5000, 6)
    elif case == "random":
        rp, col = random_graph(6000, rng)
    elif case == "ragged":
        rp, col = gg.generate(gg.GraphSpec(n=20011, mean_deg=9.0, seed=17))
    elif case == "tiny":
        rp, col = random_graph(37, rng)
    else:
        n = 4000
        edges = [(j, (j + 1) % n) for j in range(n)] + [(j, 2000) for j in range(n) if j != 2000]
        rp, col = csr_from_edges(n, edges)
    b = rng.random(len(rp) - 1)
    x = oracle_x(rp, col, b)
    tol = (1e-11 * (1 - D) if fp64 else 1e-8) * b.sum()
    h, st, f, _ = solve(rp, col, b, tol, fp64=fp64, propagation=prop, window=True)
    assert np.abs(h - x).sum() <= (1e-11 if fp64 else 1e-6) * np.abs(x).sum()
    f_cpu = check_stop(rp, col, b, h, st, tol)
    assert_residual_close(f, f_cpu, rp, col, b, h)
    assert st.red_ops >= 0


def test_fluid_window_issues_fewer_reductions_than_edges():
    # on a graph whose edges all stay within the window, the push's global
    # reductions are mostly the coalesced flushes (one per sector of 8 FP32
    # words) - far fewer than the elementary diffusions it performs
    rp, col = ring_graph(200_000, 8)
    b = gg.uniform_b(200_000, D)
    tol = 1e-8 * b.sum()
    x = oracle_x(rp, col, b)
    for prop in (3, 6, 7):
        h, st, _, _ = solve(rp, col, b, tol, propagation=prop, want_f=False, window=True)
        assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()
        assert 0 < st.red_ops < st.edge_diffusions / 4, (prop, st.red_ops, st.edge_diffusions)
    # without the window every edge is one scattered reduction (the ring has no hot targets)
    _, st3, _, _ = solve(rp, col, b, tol, propagation=3, want_f=False)
    assert st3.red_ops == st3.edge_diffusions
    # the warp-tile push does not count
    _, st4, _, _ = solve(rp, col, b, tol, propagation=4, want_f=False)
    assert st4.red_ops == 0


# ---------------------------------------------------------------- propagation 7: persistent level loop

def test_persistent_loop_times_its_phases(web10k):
    rp, col, b, x = web10k
    tol = 1e-8 * b.sum()
    for timing in (0, 1):
        h, st, _, _ = solve(rp, col, b, tol, propagation=7, resweeps=1, timing=timing)
        assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()
        check_stop(rp, col, b, h, st, tol)
        # device-timed phases: every selection pass is counted, the push phases
        # take part of the level time, and the whole loop fits in the solve
        assert st.level_launches == st.body_iterations
        assert 0 < st.select_seconds < st.level_seconds <= st.seconds


def test_persistent_loop_barrier_timeout_returns_an_error(web10k):
    # a zero bound on the grid barriers' wait: the waiting CTAs give up, the
    # solve returns DI_ETIMEOUT (no fault, no hang) and the context stays usable
    rp, col, b, x = web10k
    g = di.Graph.create(rp, col)
    B = dev(b)
    H = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    rc, st = di.di_solve(g, B, D, 1e-8 * b.sum(), H, None, di.opts_default(propagation=7, spin_limit=0),
                         allow=(di.DI_ETIMEOUT,))
    assert rc == di.DI_ETIMEOUT and "grid barrier" in di.last_error()
    rc, st = di.di_solve(g, B, D, 1e-8 * b.sum(), H, None, di.opts_default(propagation=7))
    assert rc == di.DI_OK
    assert np.abs(H.cpu().numpy() - x).sum() <= 1e-6 * np.abs(x).sum()
    with pytest.raises(di.DiError) as e:
        di.di_solve(g, B, D, 1e-8, H, None, di.opts_default(propagation=7, spin_limit=-1))
    assert e.value.status == di.DI_EINVAL
    g.close()
