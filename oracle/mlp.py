"""Plain FP64 CPU reference of the surrogate network (oracle; test infrastructure only).

The surrogate maps Hamiltonian parameters to electronic population trajectories.  The
paper motivates its method with advances in machine learning (Introduction) but gives
no network; this is the plain definition of the network this library trains:

    h_0 = x                                   (batch x n_in)
    a_l = h_{l-1} W_l + b_l,  h_l = tanh(a_l)  for the hidden layers l = 1 .. L-1
    y   = h_{L-1} W_L + b_L                   (linear output layer)
    loss = sum over batch and outputs of (y - t)^2 / (2 * batch)

with W_l of shape (n_{l-1}, n_l), row-major.  Backpropagation (chain rule):

    dy = (y - t) / batch
    dW_L = h_{L-1}^T dy,  db_L = sum_rows dy,  dh_{L-1} = dy W_L^T
    da_l = dh_l * (1 - h_l^2),  dW_l = h_{l-1}^T da_l,  db_l = sum_rows da_l,
    dh_{l-1} = da_l W_l^T

Adam (Kingma & Ba 2015), step t >= 1, for every parameter p with gradient g:

    m <- beta1 m + (1 - beta1) g,  v <- beta2 v + (1 - beta2) g^2,
    p <- p - lr * (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps)

Pins (tests/test_oracle_mlp.py): the analytic gradient against central finite
differences of the loss; one Adam step against the update written out for a single
scalar; the forward pass against an explicit per-sample loop.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np


def init_params(widths: List[int], seed: int) -> List[Tuple[np.ndarray, np.ndarray]]:
    """Weights uniform in +-sqrt(6 / (fan_in + fan_out)) (Glorot), biases zero."""
    rng = np.random.default_rng(seed)
    params = []
    for a, b in zip(widths[:-1], widths[1:]):
        lim = np.sqrt(6.0 / (a + b))
        params.append((rng.uniform(-lim, lim, size=(a, b)), np.zeros(b)))
    return params


def forward(params, x: np.ndarray):
    """Returns the output and the list of layer outputs h_0 .. h_{L-1} (for backward)."""
    h = np.asarray(x, dtype=np.float64)
    hs = [h]
    L = len(params)
    for l, (W, b) in enumerate(params):
        a = h @ W + b
        h = a if l == L - 1 else np.tanh(a)
        if l < L - 1:
            hs.append(h)
    return h, hs


def loss(params, x, t) -> float:
    y, _ = forward(params, x)
    return float(np.sum((y - t) ** 2) / (2.0 * x.shape[0]))


def backward(params, x, t):
    """Gradients [(dW_l, db_l)] of the loss, in layer order."""
    y, hs = forward(params, x)
    B = x.shape[0]
    L = len(params)
    grads = [None] * L
    d = (y - t) / B                      # d loss / d a_L (linear output)
    for l in range(L - 1, -1, -1):
        W, _ = params[l]
        h_prev = hs[l]
        grads[l] = (h_prev.T @ d, d.sum(axis=0))
        if l > 0:
            dh = d @ W.T
            d = dh * (1.0 - hs[l] ** 2)  # tanh'(a) = 1 - tanh(a)^2
    return grads


class Adam:
    def __init__(self, params, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.m = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
        self.v = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
        self.t = 0

    def step(self, params, grads):
        """New parameters after one step (the moments are updated in place)."""
        self.t += 1
        c1 = 1.0 - self.b1 ** self.t
        c2 = 1.0 - self.b2 ** self.t
        out = []
        for k, (layer, glayer) in enumerate(zip(params, grads)):
            new = []
            for j in range(2):
                p, g = layer[j], glayer[j]
                self.m[k][j] = self.b1 * self.m[k][j] + (1.0 - self.b1) * g
                self.v[k][j] = self.b2 * self.v[k][j] + (1.0 - self.b2) * g * g
                new.append(p - self.lr * (self.m[k][j] / c1) / (np.sqrt(self.v[k][j] / c2) + self.eps))
            out.append((new[0], new[1]))
        return out
