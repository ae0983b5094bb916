"""The learned warm start on the GPU against the warm-start oracle.

Tolerances, derived from the arithmetic:
  * features: the device evaluates log1p and 1/outdeg in FP32 (within 1
    unit in the last place each) and sums with compensated FP32 sums (within
    2 units of the exact sum of its terms); along the longest chain (x7:
    reciprocal, first-hop sum, product, second-hop sum, log1p, each rounding)
    these add up to under 8 FP32 units in the last place, so the test allows
    relative 1e-6 against the oracle's FP64 values rounded to FP32;
  * network output: both sides round the same operands to BF16 (the
    standardised features are chosen BF16-exact), then the device
    accumulates in FP32 where the oracle uses FP64; a first-layer activation
    whose FP32 and FP64 values straddle a BF16 rounding boundary may round
    one BF16 unit (2^-8 relative) apart, so the bound per row is
    2^-7 sum_j |w3_j| sum_k |W2_jk| |h1_k| + 1e-5 (1 + |y|), and 99% of the
    rows must agree to 1e-5 (1 + |y|);
  * gradient: FP32 sums over the rows; each component within 2e-4 of the
    largest component (and the loss to 1e-5 relative);
  * Adam: FP32 against FP64, 1e-6 relative on the updated parameters.
"""
import os
import tempfile

import numpy as np
import pytest
import torch

from oracle import diter as od
from oracle import warmstart as ow
from paper_1202_6168_gb300 import binding as di
from paper_1202_6168_gb300 import graphgen as gg

from graphs_util import csr_from_edges, random_graph

pytestmark = pytest.mark.gpu
D = 0.85


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def model_with(theta, mu=None, sd=None):
    m = di.Model.create(3)
    st = np.zeros(di.MODEL_STATE, dtype=np.float32)
    st[:9] = 0.0 if mu is None else mu
    st[9:18] = 1.0 if sd is None else sd
    st[18:] = theta
    m.set_state(st)
    return m


def random_theta(rng, scale=0.25):
    th = (rng.standard_normal(ow.N_PARAM) * scale).astype(np.float32)
    p = ow.unpack(th.astype(np.float64))
    p["W1"][:, 9:] = 0.0
    return ow.pack(p).astype(np.float32)


# ---------------------------------------------------------------- features

@pytest.mark.parametrize("case", ["web", "dups_selfloops", "star", "single", "ragged", "hubs_mid_group"])
def test_features_match_oracle(case):
    rng = np.random.default_rng(1)
    if case == "web":
        rp, col = gg.generate(gg.GraphSpec(n=20000, mean_deg=9.0, seed=4))
    elif case == "dups_selfloops":
        rp, col = random_graph(3000, rng, max_deg=50)
    elif case == "star":   # in-rows far longer than a warp
        n = 5000
        rp, col = csr_from_edges(n, [(j, 0) for j in range(1, n)] + [(j, 1) for j in range(2, 200)] + [(0, 2)])
    elif case == "single":
        rp, col = csr_from_edges(1, [])
    elif case == "hubs_mid_group":
        # two rows longer than 4096 inside one 32-row group (5 and 17), one of
        # several hundred (40), empty rows and random short rows around them
        n = 12000
        edges = [(j, 5) for j in range(100, 5200)] + [(j, 17) for j in range(200, 4500)]
        edges += [(j, 40) for j in range(0, 300)]
        src = rng.integers(0, n, size=30000)
        dst = rng.integers(0, n, size=30000)
        edges += [(int(a), int(t)) for a, t in zip(src, dst) if t % 7]
        rp, col = csr_from_edges(n, edges)
    else:
        rp, col = gg.generate(gg.GraphSpec(n=32 * 97 + 13, mean_deg=6.0, seed=5))
    n = len(rp) - 1
    b = rng.random(n) / n
    g = di.Graph.create(rp, col)
    m = di.Model.create(1)
    feat = torch.zeros((n, 9), dtype=torch.float32, device="cuda")
    m.features(g, dev(b), feat)
    torch.cuda.synchronize()
    want = ow.features(rp, col, b).astype(np.float32)
    got = feat.cpu().numpy()
    np.testing.assert_allclose(got, want, rtol=1e-6, atol=0)
    g.close()
    m.close()


# ---------------------------------------------------------------- network

def bf16_exact_features(rng, n):
    return ow.round_bf16(rng.standard_normal((n, 9)) * 1.5).astype(np.float32)


def test_forward_matches_oracle():
    rng = np.random.default_rng(2)
    th = random_theta(rng)
    m = model_with(th)
    n = 5000                                   # 312 tiles of 16 rows and a ragged tail of 8
    x = bf16_exact_features(rng, n)
    y = torch.zeros(n, dtype=torch.float32, device="cuda")
    m.forward(dev(x), n, y)
    torch.cuda.synchronize()
    xs = np.hstack([x.astype(np.float64), np.zeros((n, 7))])
    a = ow.forward(th.astype(np.float64), xs, bf16=True)
    got = y.cpu().numpy().astype(np.float64)
    err = np.abs(got - a["y"])
    scale = np.abs(a["h1"]) @ np.abs(a["W2"]).T @ np.abs(a["w3"])
    assert np.all(err <= 2.0 ** -7 * scale + 1e-5 * (1 + np.abs(a["y"])))
    assert np.mean(err <= 1e-5 * (1 + np.abs(a["y"]))) >= 0.99
    m.close()


def test_forward_standardises_with_the_model_statistics():
    rng = np.random.default_rng(3)
    th = random_theta(rng)
    mu = rng.standard_normal(9).astype(np.float32)
    sd = (rng.random(9) + 0.5).astype(np.float32)
    m = model_with(th, mu, sd)
    n = 2000
    x = (rng.standard_normal((n, 9)) * 2).astype(np.float32)
    y = torch.zeros(n, dtype=torch.float32, device="cuda")
    m.forward(dev(x), n, y)
    xs = ow.standardise(x.astype(np.float64), mu.astype(np.float64), sd.astype(np.float64))
    a = ow.forward(th.astype(np.float64), xs, bf16=True)
    err = np.abs(y.cpu().numpy() - a["y"])
    # the standardised value is formed in FP32 on the device: it may round to
    # the neighbouring BF16 value (2^-8 relative) on any input column, and a
    # first-layer activation may then round one BF16 unit apart as well
    d1 = 2.0 ** -8 * (np.abs(a["x"]) @ np.abs(a["W1"]).T) + 2.0 ** -8 * np.abs(a["h1"])
    scale = d1 @ np.abs(a["W2"]).T @ np.abs(a["w3"])
    assert np.all(err <= 2 * scale + 1e-5 * (1 + np.abs(a["y"])))
    assert np.median(err) <= 1e-5 * (1 + np.median(np.abs(a["y"])))
    m.close()


def test_gradient_matches_oracle():
    rng = np.random.default_rng(4)
    th = random_theta(rng)
    m = model_with(th)
    n = 3000
    x = bf16_exact_features(rng, n)
    t = rng.standard_normal(n).astype(np.float32)
    loss, g = m.grad(dev(x), dev(t), n)
    xs = np.hstack([x.astype(np.float64), np.zeros((n, 7))])
    loss_o, g_o = ow.backward(th.astype(np.float64), xs, t.astype(np.float64), bf16=True)
    assert loss == pytest.approx(loss_o, rel=1e-5)
    assert np.max(np.abs(g - g_o)) <= 2e-4 * np.max(np.abs(g_o))
    pad = ow.unpack(g.astype(np.float64))["W1"][:, 9:]
    assert np.all(pad == 0)
    m.close()


def test_adam_matches_oracle():
    rng = np.random.default_rng(5)
    th = random_theta(rng)
    m = model_with(th)
    mo = vo = np.zeros(ow.N_PARAM)
    tho = th.astype(np.float64)
    opts = di.train_opts_default(lr=1e-2)
    moved = np.zeros(ow.N_PARAM)          # sum over steps of |step update|
    for step in range(1, 4):
        grad = (rng.standard_normal(ow.N_PARAM) * 0.1).astype(np.float32)
        m.adam(grad, opts)
        prev = tho
        tho, mo, vo = ow.adam_step(tho, grad.astype(np.float64), mo, vo, step, lr=1e-2)
        moved += np.abs(tho - prev)
    got = m.get_state()[18:].astype(np.float64)
    # the device keeps FP32 weights: each of the 3 steps rounds theta to FP32
    # (half a unit in the last place), and each step's update is formed in
    # FP32 (relative 1e-5 covers its few roundings, taken on the sum of the
    # step magnitudes since steps of opposite sign may cancel)
    upd_gpu, upd_o = got - th, tho - th
    ulp = np.spacing(np.abs(th).astype(np.float32) + moved.astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(upd_gpu - upd_o) <= 1e-5 * moved + 2.0 * ulp)
    m.close()


# ---------------------------------------------------------------- training and the gain

def solved(rp, col, b):
    g = di.Graph.create(rp, col)
    H = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    di.di_solve(g, dev(b), D, 1e-11 * (1 - D) * b.sum(), H, None, di.opts_default(fluid_fp64=1))
    return g, H


def test_training_learns_and_the_warm_start_pays():
    specs = [gg.GraphSpec(n=n, mean_deg=10.0, seed=700 + i) for i, n in enumerate((20000, 35000, 50000, 28000))]
    graphs, Bs, Xs = [], [], []
    for sp in specs:
        rp, col = gg.generate(sp)
        b = gg.uniform_b(sp.n)
        g, H = solved(rp, col, b)
        graphs.append(g)
        Bs.append(dev(b))
        Xs.append(H)
    m = di.Model.create(11)
    loss = m.train(graphs, Bs, Xs, di.train_opts_default(epochs=30, batch=8192, lr=3e-3))
    # the target log(N x) has variance ~0.5 on these graphs; the network explains most of it
    y_all = np.concatenate([ow.target(X.cpu().numpy(), len(X)) for X in Xs])
    assert loss < 0.25 * y_all.var()
    # held-out graph: H0 from the network, its fluid F0 = B + P H0 - H0
    rp, col = gg.generate(gg.GraphSpec(n=60000, mean_deg=10.0, seed=799))
    b = gg.uniform_b(60000)
    x = od.d_iteration(rp, col, b, D, tol=1e-14 * b.sum()).H
    g = di.Graph.create(rp, col)
    H0 = torch.zeros(60000, dtype=torch.float64, device="cuda")
    m.infer(g, dev(b), H0)
    f0 = di.di_residual(g, dev(b), D, H0, torch.zeros_like(H0))
    _, f0_oracle = od.residual(rp, col, b, D, H0.cpu().numpy())
    assert f0 == pytest.approx(f0_oracle, rel=1e-12)
    assert f0 < b.sum()                       # the warm start holds less fluid than B
    tol = 1e-8 * b.sum()
    H = H0.clone()
    _, st_w = di.di_solve(g, dev(b), D, tol, H, None, di.opts_default(warm_start=1))
    assert st_w.warm_used == 1
    assert np.abs(H.cpu().numpy() - x).sum() <= 1e-6 * np.abs(x).sum()
    Hc = torch.zeros_like(H0)
    _, st_c = di.di_solve(g, dev(b), D, tol, Hc, None, di.opts_default())
    assert np.abs(Hc.cpu().numpy() - x).sum() <= 1e-6 * np.abs(x).sum()
    assert st_c.warm_used == 0
    # the gain, at equal accuracy: both solves stop on an exact residual below the
    # same tol (so |X - H|_1 <= tol / (1 - d) for both), and the warm start gets
    # there with fewer elementary diffusions (Sec. 2.4 cost) and no more levels
    for h, st in ((H, st_w), (Hc, st_c)):
        _, r = od.residual(rp, col, b, D, h.cpu().numpy())
        assert r <= tol * (1 + 1e-9) + 64 * np.finfo(np.float64).eps * (b.sum() + 2 * x.sum())
    print(f"warm start: {st_w.edge_diffusions} vs {st_c.edge_diffusions} edge diffusions "
          f"({st_w.edge_diffusions / st_c.edge_diffusions:.3f}), {st_w.levels} vs {st_c.levels} levels, "
          f"|F0|_1 / |B|_1 = {st_w.f0_l1 / st_w.b_l1:.3f}")
    assert st_w.edge_diffusions < st_c.edge_diffusions
    assert st_w.levels <= st_c.levels
    g.close()
    for gg_ in graphs:
        gg_.close()
    m.close()


def test_infer_is_exp_of_forward_over_n():
    rng = np.random.default_rng(6)
    m = model_with(random_theta(rng, 0.1))
    rp, col = gg.generate(gg.GraphSpec(n=7000, mean_deg=8.0, seed=9))
    g = di.Graph.create(rp, col)
    b = dev(gg.uniform_b(7000))
    feat = torch.zeros((7000, 9), dtype=torch.float32, device="cuda")
    y = torch.zeros(7000, dtype=torch.float32, device="cuda")
    H0 = torch.zeros(7000, dtype=torch.float64, device="cuda")
    m.features(g, b, feat)
    m.forward(feat, 7000, y)
    m.infer(g, b, H0)
    # H0 = expf(y) / N: CUDA's expf is within 2 ulp (relative 2 * 2^-23), and
    # the FP64 product with 1/N adds one FP64 rounding
    np.testing.assert_allclose(H0.cpu().numpy(), np.exp(y.cpu().numpy().astype(np.float64)) / 7000,
                               rtol=2 * 2.0 ** -23 + 4e-16)
    g.close()
    m.close()


def test_save_load_roundtrip():
    rng = np.random.default_rng(7)
    m = model_with(random_theta(rng), rng.standard_normal(9).astype(np.float32),
                   (rng.random(9) + 0.5).astype(np.float32))
    m.adam((rng.standard_normal(ow.N_PARAM) * 0.1).astype(np.float32))
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ws.bin")
        m.save(path)
        m2 = di.Model.load(path)
        np.testing.assert_array_equal(m.get_state(), m2.get_state())
        # the Adam moments travel too: one more identical step stays identical
        grad = (rng.standard_normal(ow.N_PARAM) * 0.1).astype(np.float32)
        m.adam(grad)
        m2.adam(grad)
        np.testing.assert_array_equal(m.get_state(), m2.get_state())
        with open(path, "r+b") as f:
            f.write(b"XXXX")
        with pytest.raises(di.DiError):
            di.Model.load(path)
        m2.close()
    m.close()


def test_model_rejects_bad_state():
    m = di.Model.create(1)
    st = m.get_state()
    st[9] = 0.0
    with pytest.raises(di.DiError):
        m.set_state(st)
    m.close()
