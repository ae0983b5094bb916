"""Pins of the warm-start oracle (features, network, gradient, Adam).

Each check uses something other than the oracle's own formula: hand-derived
values on small graphs, a pure-Python loop over the edges, dense matrix
powers of Q, the bfloat16 conversion of a library, hand-evaluated networks,
central finite differences, and the closed form of Adam's first steps.
"""
import math

import numpy as np
import pytest
import torch

from oracle import diter as od
from oracle import warmstart as ow

from graphs_util import csr_from_edges, random_graph


# ---------------------------------------------------------------- bfloat16 rounding

def test_bf16_rounding_hand_values():
    one = 1.0
    assert ow.round_bf16([one])[0] == 1.0
    assert ow.round_bf16([1 + 2 ** -8])[0] == 1.0                  # tie -> even (1.0)
    assert ow.round_bf16([1 + 3 * 2 ** -8])[0] == 1 + 2 ** -6       # tie -> even (mantissa 2)
    assert ow.round_bf16([1 + 2 ** -8 + 2 ** -12])[0] == 1 + 2 ** -7
    assert ow.round_bf16([-3.0])[0] == -3.0


def test_bf16_rounding_matches_a_library_conversion():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    lib = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(ow.round_bf16(x), lib)


# ---------------------------------------------------------------- features

def test_features_on_a_path_by_hand():
    rp, col = csr_from_edges(3, [(0, 1), (1, 2)])
    x = ow.features(rp, col, np.array([0.05, 0.05, 0.05]))
    l2 = math.log(2.0)
    want = np.array([
        # x0   x1    x2   x3   x4   x5  x6          x7          x8
        [0.0, l2, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.15],
        [l2, l2, 0.0, 0.0, 0.0, 0.0, math.log(2.0), 0.0, 0.15],
        [l2, 0.0, l2, l2, 0.0, 0.0, math.log(2.0), math.log(2.0), 0.15],
    ])
    np.testing.assert_allclose(x, want, rtol=0, atol=1e-15)


def test_features_with_duplicates_and_self_loops_by_hand():
    # 1 -> 0 twice, 2 -> 0, 0 -> 0 (self-loop), 0 -> 1
    rp, col = csr_from_edges(3, [(0, 0), (0, 1), (1, 0), (1, 0), (2, 0)])
    x = ow.features(rp, col, np.zeros(3))
    ld = [math.log(5.0), math.log(2.0), 0.0]       # in-degrees 4, 1, 0
    # in-edges of 0: from 0, 1, 1, 2
    assert x[0, 2] == pytest.approx((ld[0] + 2 * ld[1] + ld[2]) / 4)
    assert x[0, 3] == pytest.approx(ld[0])
    s = [1 / 2, 1 / 2, 1.0]                        # out-degrees 2, 2, 1
    a1_0 = s[0] + 2 * s[1] + s[2]
    a1_1 = s[0]
    assert x[0, 6] == pytest.approx(math.log1p(a1_0))
    assert x[1, 6] == pytest.approx(math.log1p(a1_1))
    assert x[0, 7] == pytest.approx(math.log1p(s[0] * a1_0 + 2 * s[1] * a1_1 + s[2] * 0.0))
    assert x[2, 2:8].tolist() == [0.0] * 6            # no in-edge


def features_by_loops(rp, col, b):
    """The same definitions with plain Python loops over the edges."""
    n = len(rp) - 1
    ins = [[] for _ in range(n)]
    for j in range(n):
        for e in range(rp[j], rp[j + 1]):
            ins[int(col[e])].append(j)
    outd = [int(rp[j + 1] - rp[j]) for j in range(n)]
    ld = [math.log(1 + len(ins[i])) for i in range(n)]
    s = [1.0 / o if o else 0.0 for o in outd]
    x = [[0.0] * 9 for _ in range(n)]
    for i in range(n):
        x[i][0] = ld[i]
        x[i][1] = math.log(1 + outd[i])
        if ins[i]:
            x[i][2] = sum(ld[j] for j in ins[i]) / len(ins[i])
            x[i][3] = max(ld[j] for j in ins[i])
    a1 = [sum(s[j] for j in ins[i]) for i in range(n)]
    a2 = [sum(s[j] * a1[j] for j in ins[i]) for i in range(n)]
    for i in range(n):
        if ins[i]:
            x[i][4] = sum(x[j][2] for j in ins[i]) / len(ins[i])
            x[i][5] = max(x[j][3] for j in ins[i])
        x[i][6] = math.log(1 + a1[i])
        x[i][7] = math.log(1 + a2[i])
        x[i][8] = n * b[i]
    return np.array(x)


@pytest.mark.parametrize("seed", range(3))
def test_features_match_edge_loops(seed):
    rng = np.random.default_rng(seed)
    rp, col = random_graph(300, rng, max_deg=9)
    b = rng.random(300)
    np.testing.assert_allclose(ow.features(rp, col, b), features_by_loops(rp, col, b), rtol=1e-13, atol=1e-14)


def test_one_and_two_hop_sums_are_powers_of_q():
    rng = np.random.default_rng(4)
    rp, col = random_graph(120, rng, p_dangling=0.2)
    q = od.dense_p(rp, col, 1.0)                      # Q: q_kj = 1/#out_j
    x = ow.features(rp, col, np.zeros(120))
    ones = np.ones(120)
    np.testing.assert_allclose(np.expm1(x[:, 6]), q @ ones, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(np.expm1(x[:, 7]), q @ (q @ ones), rtol=1e-12, atol=1e-14)


def test_standardise():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((500, 9)) * 3 + 7
    x[:, 8] = 0.15
    mu, sd = ow.norm_stats(x)
    z = ow.standardise(x, mu, sd)
    assert z.shape == (500, ow.K1)
    np.testing.assert_allclose(z[:, :8].mean(axis=0), 0, atol=1e-12)
    np.testing.assert_allclose(z[:, :8].std(axis=0), 1, atol=1e-12)
    assert np.all(np.abs(z[:, 8]) < 1e-15)      # constant column: sigma 1, centred to ~0
    assert np.all(z[:, 9:] == 0)


# ---------------------------------------------------------------- the network

def hand_params():
    p = {name: np.zeros(shape) for name, shape in ow.SHAPES}
    p["W1"][0, 0] = 2.0
    p["b1"][0] = -1.0
    p["W2"][0, 0] = 3.0
    p["w3"][0] = 0.5
    p["b3"][0] = 0.25
    return ow.pack(p)


def test_forward_hand_values():
    th = hand_params()
    xs = np.zeros((3, ow.K1))
    xs[0, 0] = 1.0            # z1 = 1, h1 = 1, z2 = 3, y = 1.75
    xs[1, 0] = 0.25           # z1 = -0.5 -> relu 0 -> y = b3
    xs[2, 0] = 1 + 2 ** -8    # bf16 rounds the input to 1.0
    y = ow.forward(th, xs, bf16=True)["y"]
    np.testing.assert_array_equal(y, [1.75, 0.25, 1.75])
    y64 = ow.forward(th, xs, bf16=False)["y"]
    assert y64[2] == pytest.approx(0.25 + 0.5 * 3 * (2 * (1 + 2 ** -8) - 1), rel=1e-15)


def random_params(rng, scale=0.3):
    return rng.standard_normal(ow.N_PARAM) * scale


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(6)
    th = random_params(rng)
    xs = np.hstack([rng.standard_normal((40, 9)), np.zeros((40, 7))])
    t = rng.standard_normal(40)
    _, g = ow.backward(th, xs, t, bf16=False)
    idx = list(range(0, ow.N_PARAM, 37)) + [ow.N_PARAM - 1, ow.N_PARAM - 2]
    h = 1e-6
    for k in idx:
        e = np.zeros(ow.N_PARAM)
        e[k] = h
        fd = (ow.loss(th + e, xs, t, bf16=False) - ow.loss(th - e, xs, t, bf16=False)) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-6, abs=1e-9), k


def test_gradient_of_padding_columns_is_zero():
    rng = np.random.default_rng(7)
    th = random_params(rng)
    xs = np.hstack([rng.standard_normal((30, 9)), np.zeros((30, 7))])
    _, g = ow.backward(th, xs, rng.standard_normal(30))
    gw1 = ow.unpack(g)["W1"]
    assert np.all(gw1[:, 9:] == 0)


# ---------------------------------------------------------------- Adam

def test_adam_first_steps_closed_form():
    th0 = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m = v = np.zeros(3)
    th = th0
    for step in range(1, 4):
        th, m, v = ow.adam_step(th, g, m, v, step, lr=1e-3)
        # a constant gradient gives m_hat = g and v_hat = g^2 at every step
        np.testing.assert_allclose(th, th0 - step * 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-13)
    assert np.allclose(m, (1 - 0.9 ** 3) * g) and np.allclose(v, (1 - 0.999 ** 3) * g * g)


def test_adam_fits_a_toy_target():
    rng = np.random.default_rng(8)
    xs = np.hstack([rng.standard_normal((256, 9)), np.zeros((256, 7))])
    t = xs[:, 0] * 0.7 - xs[:, 3] * 0.2 + 0.1 * np.maximum(xs[:, 1], 0)
    th = random_params(rng, 0.2)
    m = v = np.zeros_like(th)
    l0 = ow.loss(th, xs, t, bf16=False)
    for step in range(1, 401):
        _, g = ow.backward(th, xs, t, bf16=False)
        th, m, v = ow.adam_step(th, g, m, v, step, lr=3e-3)
    assert ow.loss(th, xs, t, bf16=False) < 0.05 * l0


def test_warm_h0_inverts_the_target():
    x = np.array([1e-7, 3e-6, 0.2])
    np.testing.assert_allclose(ow.warm_h0(ow.target(x, 1000), 1000), x, rtol=1e-14)
