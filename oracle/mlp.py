"""CPU reference of the learned-priority MLP (test infrastructure).

Plain numpy in float64: the feature transform, BF16 round-to-nearest-even
(from the format's definition: keep the top 16 bits of the IEEE-754 single,
rounding the dropped 16 bits to nearest, ties to even), the forward pass with
the roundings the tensor-core inference applies (inputs, W1, W2 and the
first hidden layer in BF16; everything else exact), the mean-squared-error
gradient by backpropagation (roundings treated as identity), and Adam.
Parameters are one flat vector in the library's layout: W1[12][64], b1[64],
W2[64][64], b2[64], W3[64], b3.
"""
from __future__ import annotations

import numpy as np

NIN, NH = 12, 64
NPARAM = NIN * NH + NH + NH * NH + NH + NH + 1


def split(w):
    w = np.asarray(w, dtype=np.float64)
    i = 0
    W1 = w[i:i + NIN * NH].reshape(NIN, NH); i += NIN * NH
    b1 = w[i:i + NH]; i += NH
    W2 = w[i:i + NH * NH].reshape(NH, NH); i += NH * NH
    b2 = w[i:i + NH]; i += NH
    W3 = w[i:i + NH]; i += NH
    b3 = w[i]
    return W1, b1, W2, b2, W3, b3


def join(W1, b1, W2, b2, W3, b3):
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3, [b3]])


def transform(f):
    """sign(f) * log2(1 + |f|) of integer features, rounded to float32."""
    f = np.asarray(f, dtype=np.float64)
    return (np.sign(f) * np.log2(1.0 + np.abs(f))).astype(np.float32).astype(np.float64)


def targets(rows):
    """Training target of trace rows (round, vertex, 12 features): the
    transformed score x = edge difference + 2 * hierarchy depth, features 4
    and 6 of the row (the learned-priority label reading), float64 of the
    float32 value."""
    r = np.asarray(rows, dtype=np.int64)
    return transform(r[:, 2 + 4] + 2 * r[:, 2 + 6])


def bf16(x):
    """Round to the nearest bfloat16 value (ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float32)
    bits = a.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    rounded = ((bits + 0x7FFF + lsb) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(w, X, quantise=True):
    """Outputs and activations for inputs X [n, 12] (already transformed)."""
    W1, b1, W2, b2, W3, b3 = split(w)
    q = bf16 if quantise else (lambda v: np.asarray(v, dtype=np.float64))
    x = q(X)
    h1 = q(np.maximum(x @ q(W1) + b1, 0.0))
    h2 = np.maximum(h1 @ q(W2) + b2, 0.0)
    y = h2 @ W3 + b3
    return y, (x, h1, h2)


def loss_and_grad(w, X, labels, quantise=True):
    """Mean squared error over the rows and its gradient (flat vector)."""
    W1, b1, W2, b2, W3, b3 = split(w)
    q = bf16 if quantise else (lambda v: np.asarray(v, dtype=np.float64))
    y, (x, h1, h2) = forward(w, X, quantise)
    n = X.shape[0]
    diff = y - labels
    dy = 2.0 * diff / n
    gW3 = h2.T @ dy
    gb3 = dy.sum()
    g2 = np.outer(dy, W3) * (h2 > 0)
    gW2 = h1.T @ g2
    gb2 = g2.sum(0)
    g1 = (g2 @ q(W2).T) * (h1 > 0)
    gW1 = x.T @ g1
    gb1 = g1.sum(0)
    return float(np.mean(diff * diff)), join(gW1, gb1, gW2, gb2, gW3, gb3)


def init_weights(seed=0, scale=0.3):
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, scale / np.sqrt(NIN), (NIN, NH))
    W2 = rng.normal(0, scale / np.sqrt(NH), (NH, NH))
    W3 = rng.normal(0, scale / np.sqrt(NH), NH)
    return join(W1, np.zeros(NH), W2, np.zeros(NH), W3, 0.0).astype(np.float32)
