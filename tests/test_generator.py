"""The seeded input generator: determinism, structure and shape statistics."""
import json
import math
import os

import numpy as np
import pytest

from paper_1202_6168_gb300 import graphgen as gg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "graph_hashes.json")


def test_deterministic_elementary_functions():
    for a in (0.3, 1.0, 2.0, 10.0, 1e6 + 1):
        assert gg.det_log(a) == pytest.approx(math.log(a), rel=2e-15, abs=1e-16)
    for y in (-20.0, -1.0, 0.0, 0.5, 3.0, 30.0):
        assert gg.det_exp(y) == pytest.approx(math.exp(y), rel=2e-15)
    assert gg.det_pow(1000.0, -2.1) == pytest.approx(1000.0 ** -2.1, rel=1e-14)


def test_zipf_mean():
    k = np.arange(1, 1001, dtype=np.float64)
    w = k ** -2.1
    assert gg.zipf_mean() == pytest.approx((k * w).sum() / w.sum(), rel=1e-13)


def test_same_seed_same_graph_other_seed_other_graph():
    a = gg.generate(gg.GraphSpec(n=5000, mean_deg=8, seed=3))
    b = gg.generate(gg.GraphSpec(n=5000, mean_deg=8, seed=3))
    c = gg.generate(gg.GraphSpec(n=5000, mean_deg=8, seed=4))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert gg.csr_hash(*a) != gg.csr_hash(*c)


def test_rows_sorted_unique_in_range_no_self_loops():
    rp, col = gg.generate(gg.SMALL_10K)
    n = gg.SMALL_10K.n
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == len(col)
    assert col.min() >= 0 and col.max() < n
    src = np.repeat(np.arange(n), np.diff(rp))
    assert not np.any(src == col)
    # strictly increasing inside each row
    same_row = src[1:] == src[:-1]
    assert np.all(col[1:][same_row] > col[:-1][same_row])


@pytest.mark.parametrize("spec", [gg.SMALL_10K, gg.WEB_1M], ids=["10k", "1m"])
def test_shape_statistics(spec):
    rp, col = gg.generate(spec)
    deg = np.diff(rp)
    assert abs((deg == 0).mean() - 0.1) < 0.01          # dangling share
    nd = deg[deg > 0].mean()
    assert 0.8 * spec.mean_deg < nd < 1.1 * spec.mean_deg
    src = np.repeat(np.arange(spec.n), deg)
    dist = np.abs(col.astype(np.int64) - src)
    dist = np.minimum(dist, spec.n - dist)
    local = (dist <= spec.window).mean()
    assert 0.25 < local < 0.40       # 30% drawn local, less self-loops and window dups
    indeg = np.bincount(col, minlength=spec.n)
    assert indeg.max() > 50 * indeg.mean()               # heavy-tailed in-degree


def test_golden_hashes():
    gold = json.load(open(GOLDEN))
    for name, spec in [("web_10k_m8", gg.SMALL_10K), ("web_1m_m10", gg.WEB_1M)]:
        rp, col = gg.generate(spec)
        assert int(rp[-1]) == gold[name]["nnz"]
        assert hex(gg.csr_hash(rp, col)) == gold[name]["fnv1a64"]


def test_right_hand_sides():
    b = gg.uniform_b(1000)
    assert b.sum() == pytest.approx(0.15)
    p = gg.personalised_b(1000, 17)
    assert p[17] == pytest.approx(0.15) and p.sum() == pytest.approx(0.15)
    specs = gg.batch_specs(64, seed=0)
    ns = np.array([s.n for s in specs])
    assert ns.min() >= 1e4 and ns.max() <= 2e6
    assert all(6 <= s.mean_deg <= 14 for s in specs)
