"""Batched solves (di_solve_batched) against the CPU oracle, item by item.

Every work item (right-hand side r of graph g) is an independent D-iteration;
the batch must return, for each item, an H within the single-solve
tolerances of the oracle's X (FP32 fluid: |H - X|_1 <= 1e-6 |X|_1 at tol =
1e-8 |B|_1; FP64 fluid: 1e-11 |X|_1 at tol = 1e-11 (1-d) |B|_1), with the
oracle's FP64 residual of that H below the item's own tolerance.
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


def oracle_x(rp, col, b):
    r = od.d_iteration(rp, col, b, D, tol=1e-14 * max(np.abs(b).sum(), 1e-300))
    assert r.status == 0
    return r.H


def stop_ok(rp, col, b, h, tol, reported):
    _, r_cpu = od.residual(rp, col, b, D, h)
    floor = 64 * np.finfo(np.float64).eps * (np.abs(b).sum() + 2 * np.abs(h).sum())
    assert r_cpu <= tol * (1 + 1e-9) + floor
    assert abs(reported - r_cpu) <= 1e-9 * max(r_cpu, tol) + floor


@pytest.fixture(scope="module")
def mixed_graphs():
    """Uneven sizes (none a multiple of the 2048-node alignment but one),
    degrees, a single node, an all-dangling graph, duplicates and self-loops."""
    rng = np.random.default_rng(31)
    out = [gg.generate(gg.GraphSpec(n=n, mean_deg=m, seed=s))
           for n, m, s in ((5000, 6.0, 1), (23457, 12.0, 2), (2048, 8.0, 3), (61001, 9.0, 4))]
    out.append(csr_from_edges(1, []))
    out.append(csr_from_edges(3000, []))
    out.append(random_graph(4000, rng, max_deg=30))
    return out


def rhs_for(n, k, rng):
    if k == 0:
        return gg.uniform_b(n)
    if k == 1:
        return gg.personalised_b(n, int(rng.integers(0, n)))
    return rng.random(n) * (0.15 / n) * 2.0


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("sweeps", [-1, 0, 2])
def test_batch_matches_oracle_item_by_item(mixed_graphs, fp64, sweeps):
    rng = np.random.default_rng(5)
    graphs = [di.Graph.create(rp, col) for rp, col in mixed_graphs]
    nrhs = [3, 2, 1, 3, 1, 2, 3]
    batch = di.Batch(graphs, nrhs)
    info = batch.info()
    assert info["n_items"] == sum(nrhs)
    assert info["n_union"] % 2048 == 0
    items = []
    for (rp, col), r in zip(mixed_graphs, nrhs):
        for k in range(r):
            items.append((rp, col, rhs_for(len(rp) - 1, k, rng)))
    tols = [(1e-11 * (1 - D) if fp64 else 1e-8) * b.sum() for _, _, b in items]
    B = [dev(b) for _, _, b in items]
    H = [torch.full((len(b),), float("nan"), dtype=torch.float64, device="cuda") for _, _, b in items]
    # slice sweeps (-1: the default, one) change the order of the diffusions, not the limit
    rc, st, tot = di.di_solve_batched(batch, B, D, tols, H,
                                      di.opts_default(fluid_fp64=1 if fp64 else 0, slice_sweeps=sweeps))
    torch.cuda.synchronize()
    rel = 1e-11 if fp64 else 1e-6
    for t, ((rp, col, b), h, s, tol) in enumerate(zip(items, H, st, tols)):
        hn = h.cpu().numpy()
        x = oracle_x(rp, col, b)
        assert np.abs(hn - x).sum() <= rel * np.abs(x).sum() + 1e-300, t
        stop_ok(rp, col, b, hn, tol, s.resid_l1)
        assert s.status == di.DI_OK
    assert tot.edge_diffusions == sum(s.edge_diffusions for s in st)
    assert tot.gpu_launches > 0
    batch.close()
    for g in graphs:
        g.close()


def test_batch_agrees_with_single_solves():
    specs = [gg.GraphSpec(n=n, mean_deg=m, seed=40 + i) for i, (n, m) in enumerate(((12000, 7.0), (70000, 11.0)))]
    csrs = [gg.generate(s) for s in specs]
    graphs = [di.Graph.create(rp, col) for rp, col in csrs]
    batch = di.Batch(graphs, [2, 2])
    bs, singles = [], []
    for (rp, col), g in zip(csrs, graphs):
        n = len(rp) - 1
        for src in gg.batch_sources(n, 2, seed=n):
            b = gg.personalised_b(n, int(src))
            bs.append(b)
            Hs = torch.zeros(n, dtype=torch.float64, device="cuda")
            di.di_solve(g, dev(b), D, 1e-8 * b.sum(), Hs)
            singles.append(Hs.cpu().numpy())
    H = [torch.zeros(len(b), dtype=torch.float64, device="cuda") for b in bs]
    di.di_solve_batched(batch, [dev(b) for b in bs], D, [1e-8 * b.sum() for b in bs], H)
    for h, s, b in zip(H, singles, bs):
        # both are within 1e-8 |B|_1 / (1 - d) of X
        assert np.abs(h.cpu().numpy() - s).sum() <= 2 * 1e-8 * b.sum() / (1 - D) * 1.001
    batch.close()
    for g in graphs:
        g.close()


def test_batch_hub_destinations_match_oracle():
    # items whose in-edges funnel into a few hubs: the batched residual's runs
    # of equal destination span many warps, summed over the warp before each
    # reduction, and an item's range starts mid-chunk
    csrs = []
    for n, seed in ((50_001, 1), (120_003, 2)):
        rng = np.random.default_rng(seed)
        col = np.stack([np.zeros(n, dtype=np.int64), 1 + np.arange(n) % 3, rng.integers(0, n, size=n)], axis=1)
        csrs.append((np.arange(0, 3 * n + 1, 3, dtype=np.int64), col.reshape(-1).astype(np.int32)))
    graphs = [di.Graph.create(rp, col) for rp, col in csrs]
    batch = di.Batch(graphs, [2, 2])
    bs, xs, gi = [], [], []
    for k, (rp, col) in enumerate(csrs):
        n = len(rp) - 1
        for src in gg.batch_sources(n, 2, seed=n):
            b = gg.personalised_b(n, int(src))
            bs.append(b)
            xs.append(oracle_x(rp, col, b))
            gi.append(k)
    H = [torch.zeros(len(b), dtype=torch.float64, device="cuda") for b in bs]
    _, st, _ = di.di_solve_batched(batch, [dev(b) for b in bs], D, [1e-8 * b.sum() for b in bs], H)
    for t, (h, x, b, k) in enumerate(zip(H, xs, bs, gi)):
        h = h.cpu().numpy()
        assert np.abs(h - x).sum() <= 1e-6 * np.abs(x).sum()
        stop_ok(*csrs[k], b, h, 1e-8 * b.sum(), st[t].resid_l1)
    batch.close()
    for g in graphs:
        g.close()


def test_batch_level_cap_and_zero_rhs():
    rp, col = gg.generate(gg.GraphSpec(n=9000, mean_deg=8.0, seed=9))
    g = di.Graph.create(rp, col)
    batch = di.Batch([g], [2])
    b = gg.uniform_b(9000)
    B = [dev(b), dev(np.zeros(9000))]
    H = [torch.zeros(9000, dtype=torch.float64, device="cuda") for _ in range(2)]
    rc, st, _ = di.di_solve_batched(batch, B, D, 1e-12, H, di.opts_default(max_levels=3),
                                    allow=(di.DI_ENOCONV,))
    assert rc == di.DI_ENOCONV
    assert st[0].status == di.DI_ENOCONV and st[0].levels == 3
    _, r_cpu = od.residual(rp, col, b, D, H[0].cpu().numpy())
    assert st[0].resid_l1 == pytest.approx(r_cpu, rel=1e-12)
    assert st[1].status == di.DI_OK and st[1].node_diffusions == 0
    assert torch.all(H[1] == 0)
    batch.close()
    g.close()


def test_batch_timing_mode_matches():
    rp, col = gg.generate(gg.GraphSpec(n=15000, mean_deg=9.0, seed=12))
    g = di.Graph.create(rp, col)
    batch = di.Batch([g], [2])
    bs = [gg.uniform_b(15000), gg.personalised_b(15000, 77)]
    H = [torch.zeros(15000, dtype=torch.float64, device="cuda") for _ in bs]
    tols = [1e-8 * b.sum() for b in bs]
    rc, st, tot = di.di_solve_batched(batch, [dev(b) for b in bs], D, tols, H, di.opts_default(timing=1))
    for b, h, s, tol in zip(bs, H, st, tols):
        x = oracle_x(rp, col, b)
        assert np.abs(h.cpu().numpy() - x).sum() <= 1e-6 * np.abs(x).sum()
        stop_ok(rp, col, b, h.cpu().numpy(), tol, s.resid_l1)
    batch.close()
    g.close()


@pytest.mark.parametrize("every,drop", [(8, 0.0), (0, 64.0)])
def test_batch_refinement_schedules(mixed_graphs, every, drop):
    rng = np.random.default_rng(every + 1)
    graphs = [di.Graph.create(rp, col) for rp, col in mixed_graphs[:4]]
    batch = di.Batch(graphs, [1, 2, 1, 1])
    items = []
    for (rp, col), r in zip(mixed_graphs[:4], [1, 2, 1, 1]):
        for k in range(r):
            items.append((rp, col, rhs_for(len(rp) - 1, k, rng)))
    tols = [1e-8 * b.sum() for _, _, b in items]
    H = [torch.zeros(len(b), dtype=torch.float64, device="cuda") for _, _, b in items]
    rc, st, _ = di.di_solve_batched(batch, [dev(b) for _, _, b in items], D, tols, H,
                                    di.opts_default(recompute_every=every, recompute_drop=drop))
    for (rp, col, b), h, s, tol in zip(items, H, st, tols):
        x = oracle_x(rp, col, b)
        assert np.abs(h.cpu().numpy() - x).sum() <= 1e-6 * np.abs(x).sum()
        stop_ok(rp, col, b, h.cpu().numpy(), tol, s.resid_l1)
        if every:
            assert s.recomputes >= s.levels // every
    batch.close()
    for g in graphs:
        g.close()


def test_batch_rejects_bad_arguments():
    rp, col = csr_from_edges(3, [(0, 1), (1, 2)])
    g = di.Graph.create(rp, col)
    with pytest.raises(di.DiError):
        di.Batch([g], [0])
    batch = di.Batch([g], [1])
    B = [dev(np.ones(3))]
    H = [torch.zeros(3, dtype=torch.float64, device="cuda")]
    for d, tol in ((1.0, 1e-8), (0.85, 0.0), (0.85, float("inf"))):
        with pytest.raises(di.DiError) as e:
            di.di_solve_batched(batch, B, d, tol, H)
        assert e.value.status == di.DI_EINVAL
    with pytest.raises(di.DiError) as e:
        di.di_solve_batched(batch, B, D, 1e-8, H, di.opts_default(warm_start=1))
    assert e.value.status == di.DI_EINVAL
    with pytest.raises(di.DiError) as e:
        di.di_solve_batched(batch, B, D, 1e-8, H, di.opts_default(recompute_drop=0.9))
    assert e.value.status == di.DI_EINVAL
    batch.close()
    g.close()


def test_batch_autotune_then_parity(mixed_graphs, tmp_path):
    rng = np.random.default_rng(21)
    graphs = [di.Graph.create(rp, col) for rp, col in mixed_graphs[:4]]
    batch = di.Batch(graphs, [2, 1, 1, 2])
    items = []
    for (rp, col), r in zip(mixed_graphs[:4], [2, 1, 1, 2]):
        for k in range(r):
            items.append((rp, col, rhs_for(len(rp) - 1, k, rng)))
    tols = [1e-8 * b.sum() for _, _, b in items]
    B = [dev(b) for _, _, b in items]
    H = [torch.zeros(len(b), dtype=torch.float64, device="cuda") for _, _, b in items]
    cache = str(tmp_path / "tune.jsonl")
    t, secs = di.batch_autotune(batch, B, D, tols, H, None, cache)
    assert secs > 0 and di.get_tune(batch).as_dict() == t.as_dict()
    assert '"key": "batch items=6' in open(cache).read()
    H = [torch.zeros_like(h) for h in H]
    rc, st, _ = di.di_solve_batched(batch, B, D, tols, H)
    for (rp, col, b), h, s, tol in zip(items, H, st, tols):
        x = oracle_x(rp, col, b)
        assert np.abs(h.cpu().numpy() - x).sum() <= 1e-6 * np.abs(x).sum()
        stop_ok(rp, col, b, h.cpu().numpy(), tol, s.resid_l1)
    batch.close()
    for g in graphs:
        g.close()


# ---------------------------------------------------------------- 1/N completion of the dangling columns (Sec. 2.2)

@pytest.mark.parametrize("fp64", [False, True])
def test_batch_dangling_completion_matches_the_completed_oracle(fp64):
    # every item completes the dangling columns of its own graph by 1/n_g;
    # the chunk padding between items (union nodes past n_g) takes no part
    rng = np.random.default_rng(77)
    graphs = [gg.generate(gg.GraphSpec(n=n, mean_deg=m, seed=s)) for n, m, s in ((2000, 6.0, 5), (4999, 9.0, 6))]
    graphs += [csr_from_edges(1, []), csr_from_edges(700, []), random_graph(800, rng, max_deg=12)]
    nrhs = [2, 1, 1, 1, 2]
    gs = [di.Graph.create(rp, col) for rp, col in graphs]
    batch = di.Batch(gs, nrhs)
    items, Bs, Hs, tols = [], [], [], []
    for (rp, col), k in zip(graphs, nrhs):
        n = len(rp) - 1
        for r in range(k):
            b = rhs_for(n, r, rng)
            items.append((rp, col, b))
            Bs.append(dev(b))
            Hs.append(torch.zeros(n, dtype=torch.float64, device="cuda"))
            tols.append((1e-11 * (1 - D) if fp64 else 1e-8) * b.sum())
    rc, st, _ = di.di_solve_batched(batch, Bs, D, tols, Hs, di.opts_default(fluid_fp64=1 if fp64 else 0, dangling=1))
    eps = np.finfo(np.float64).eps
    for (rp, col, b), h, tol, s in zip(items, Hs, tols, st):
        h = h.cpu().numpy()
        x = od.d_iteration(rp, col, b, D, tol=1e-14 * b.sum(), dangling=True).H
        assert np.abs(h - x).sum() <= (1e-11 if fp64 else 1e-6) * np.abs(x).sum()
        # the stop, with the allowance for the one dangling sum every residual element shares
        _, r_cpu = od.residual(rp, col, b, D, h, dangling=True)
        dang = np.diff(rp) == 0
        floor = 64 * eps * (np.abs(b).sum() + 2 * np.abs(h).sum()) + 2 * D * dang.sum() * eps * np.abs(h[dang]).sum()
        assert r_cpu <= tol * (1 + 1e-9) + floor
        assert abs(s.resid_l1 - r_cpu) <= 1e-9 * max(r_cpu, tol) + floor
    batch.close()
    for g in gs:
        g.close()


def test_batch_slice_sweeps_cut_the_diffusions(mixed_graphs):
    # the batched push sweeps its CTA slices at each item's threshold after
    # the frontier, as the single-graph push does: fewer elementary
    # diffusions to the same tolerances, and the per-item counts add up
    rng = np.random.default_rng(9)
    graphs = [di.Graph.create(rp, col) for rp, col in mixed_graphs]
    nrhs = [2] * len(graphs)
    batch = di.Batch(graphs, nrhs)
    items = []
    for (rp, col), r in zip(mixed_graphs, nrhs):
        for k in range(r):
            items.append((rp, col, rhs_for(len(rp) - 1, k, rng)))
    tols = [1e-8 * b.sum() for _, _, b in items]
    B = [dev(b) for _, _, b in items]
    edges = {}
    for sweeps in (0, 1):
        H = [torch.zeros(len(b), dtype=torch.float64, device="cuda") for _, _, b in items]
        rc, st, tot = di.di_solve_batched(batch, B, D, tols, H, di.opts_default(slice_sweeps=sweeps))
        for (rp, col, b), h, s, tol in zip(items, H, st, tols):
            stop_ok(rp, col, b, h.cpu().numpy(), tol, s.resid_l1)
            assert s.node_diffusions > 0   # (a source at a dangling node diffuses no edge)
        assert tot.edge_diffusions == sum(s.edge_diffusions for s in st)
        edges[sweeps] = tot.edge_diffusions
    assert edges[1] < 0.85 * edges[0], edges
    # the wait for the frontier given up at once (spin_limit = 0): still exact to tol
    H = [torch.zeros(len(b), dtype=torch.float64, device="cuda") for _, _, b in items]
    rc, st, tot = di.di_solve_batched(batch, B, D, tols, H, di.opts_default(slice_sweeps=2, spin_limit=0))
    for (rp, col, b), h, s, tol in zip(items, H, st, tols):
        stop_ok(rp, col, b, h.cpu().numpy(), tol, s.resid_l1)
    for bad in (-2, 5):
        H = [torch.zeros(len(b), dtype=torch.float64, device="cuda") for _, _, b in items]
        with pytest.raises(di.DiError) as e:
            di.di_solve_batched(batch, B, D, tols, H, di.opts_default(slice_sweeps=bad))
        assert e.value.status == di.DI_EINVAL
    batch.close()
    for g in graphs:
        g.close()
