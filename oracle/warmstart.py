"""CPU oracle of the learned warm start (TEST INFRASTRUCTURE ONLY).

The paper has no learned component; what is restated here is the plain
definition of each step the CUDA warm-start path computes, in FP64 numpy,
so that a reader can check it by eye:

* ``features``  - per-node structural features from degree aggregates over
  the in-edges (one and two hops) and from B;
* ``standardise`` - (x - mu) / sigma with the training statistics;
* ``forward``   - the 3-layer ReLU network 9 -> 64 -> 64 -> 1;
* ``backward``  - the gradient of the mean squared error of that network
  (the chain rule written out layer by layer);
* ``adam_step`` - one Adam update with bias correction (Kingma & Ba, 2015);
* ``warm_h0``   - H0_i = exp(y_i) / N from a prediction of y_i = log(N x_i).

Where the CUDA path rounds to bfloat16 (the tensor-core operands: the
standardised features, W1, W2 and the first hidden layer), ``forward`` and
``backward`` take ``bf16=True`` and apply the same round-to-nearest-even at
the same points, then compute in FP64; with ``bf16=False`` they are the plain
FP64 function, which the finite-difference pins check.

Only ``tests/`` may import this module.  It shares no code with the CUDA
library.
"""
from __future__ import annotations

import numpy as np

N_FEAT = 9          # raw features per node
K1 = 16             # first-layer input width (features padded with zeros)
HID = 64            # hidden width

# flat parameter layout (float32 on the device, float64 here)
SHAPES = [("W1", (HID, K1)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("w3", (HID,)), ("b3", (1,))]
N_PARAM = sum(int(np.prod(s)) for _, s in SHAPES)   # 5313


def unpack(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + size], dtype=np.float64).reshape(shape)
        o += size
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def round_bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64.

    bfloat16 keeps the top 16 bits of an IEEE float32: round the float32 bit
    pattern at bit 16 with ties to even (values here are finite)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


# ---------------------------------------------------------------- features

def features(row_ptr, col, B) -> np.ndarray:
    """Per-node features (N x 9) of the graph with out-edge CSR (row_ptr, col).

    For node i with in-degree m_i and out-degree o_i (edges counted with
    multiplicity), ld_i = log(1 + m_i), s_i = 1/o_i (0 for a dangling node):
      x0 = ld_i                         x1 = log(1 + o_i)
      x2 = mean of ld_j over in-edges   x3 = max of ld_j over in-edges
      x4 = mean of x2_j over in-edges   x5 = max of x3_j over in-edges
      x6 = log(1 + a1_i),  a1_i = sum of s_j over in-edges j -> i
      x7 = log(1 + a2_i),  a2_i = sum of s_j a1_j over in-edges j -> i
      x8 = N B_i
    A node without in-edges has x2 .. x7 = 0 (empty mean, max and sums).
    a1 and a2 are N (Q u)_i and N (Q^2 u)_i for u uniform: the first terms of
    the series X = sum_n d^n Q^n B (Eq. 1 with P = d Q)."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    cl = np.asarray(col, dtype=np.int64)
    n = len(rp) - 1
    out = np.diff(rp)
    src = np.repeat(np.arange(n), out)          # edge e: src[e] -> cl[e]
    indeg = np.bincount(cl, minlength=n)
    ld = np.log1p(indeg.astype(np.float64))
    s = np.where(out > 0, 1.0 / np.maximum(out, 1), 0.0)

    def mean_in(v):
        tot = np.bincount(cl, weights=v[src], minlength=n)
        return np.where(indeg > 0, tot / np.maximum(indeg, 1), 0.0)

    def max_in(v):
        m = np.full(n, -np.inf)
        np.maximum.at(m, cl, v[src])
        return np.where(indeg > 0, m, 0.0)

    def sum_in(v):
        return np.bincount(cl, weights=v[src], minlength=n)

    x = np.zeros((n, N_FEAT))
    x[:, 0] = ld
    x[:, 1] = np.log1p(out.astype(np.float64))
    x[:, 2] = mean_in(ld)
    x[:, 3] = max_in(ld)
    x[:, 4] = mean_in(x[:, 2])
    x[:, 5] = max_in(x[:, 3])
    a1 = sum_in(s)
    a2 = sum_in(s * a1)
    x[:, 6] = np.log1p(a1)
    x[:, 7] = np.log1p(a2)
    x[:, 8] = n * np.asarray(B, dtype=np.float64)
    return x


def norm_stats(x: np.ndarray):
    """Mean and standard deviation of every feature column (population form);
    a constant column gets sigma = 1 so that it standardises to zero."""
    mu = x.mean(axis=0)
    sd = x.std(axis=0)
    sd = np.where(sd > 1e-12, sd, 1.0)
    return mu, sd


def standardise(x, mu, sd) -> np.ndarray:
    """(x - mu) / sd, padded with zero columns to the first layer's width."""
    z = (np.asarray(x, dtype=np.float64) - mu) / sd
    return np.hstack([z, np.zeros((z.shape[0], K1 - N_FEAT))])


# ---------------------------------------------------------------- the network

def forward(theta, xs, bf16: bool = True) -> dict:
    """y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 for every row of xs (N x 16).

    Returns the prediction and the activations the gradient needs."""
    p = unpack(theta)
    rnd = round_bf16 if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    x = rnd(xs)
    z1 = x @ rnd(p["W1"]).T + p["b1"]
    h1 = rnd(np.maximum(z1, 0.0))
    z2 = h1 @ rnd(p["W2"]).T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["w3"] + p["b3"][0]
    return {"x": x, "z1": z1, "h1": h1, "z2": z2, "h2": h2, "y": y,
            "W1": rnd(p["W1"]), "W2": rnd(p["W2"]), "w3": p["w3"]}


def loss(theta, xs, target, bf16: bool = True) -> float:
    """Mean squared error (1/M) sum_i (y_i - target_i)^2."""
    y = forward(theta, xs, bf16)["y"]
    return float(np.mean((y - np.asarray(target, dtype=np.float64)) ** 2))


def backward(theta, xs, target, bf16: bool = True):
    """(loss, gradient) of the mean squared error by the chain rule.

    With bf16=True the rounding points of the forward pass are taken as
    constants (their derivative is the identity), i.e. this is the gradient
    the device computes from the activations it stored."""
    a = forward(theta, xs, bf16)
    t = np.asarray(target, dtype=np.float64)
    m = len(t)
    dy = 2.0 * (a["y"] - t) / m                         # d loss / d y
    g = {}
    g["w3"] = a["h2"].T @ dy
    g["b3"] = np.array([dy.sum()])
    dz2 = np.outer(dy, a["w3"]) * (a["z2"] > 0)        # through relu
    g["W2"] = dz2.T @ a["h1"]
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ a["W2"]
    dz1 = dh1 * (a["z1"] > 0)
    g["W1"] = dz1.T @ a["x"]
    g["b1"] = dz1.sum(axis=0)
    return float(np.mean((a["y"] - t) ** 2)), pack(g)


def adam_step(theta, grad, m, v, step: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update; step counts from 1.  Returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def warm_h0(y, n: int) -> np.ndarray:
    """H0_i = exp(y_i) / N (y predicts log(N x_i))."""
    return np.exp(np.asarray(y, dtype=np.float64)) / n


def target(x_solution, n: int) -> np.ndarray:
    """Training target log(N x_i) of a converged solution."""
    return np.log(n * np.maximum(np.asarray(x_solution, dtype=np.float64), 1e-300))
