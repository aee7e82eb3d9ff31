"""Pins of the FP64 surrogate-network oracle (oracle/mlp.py) that do not depend on it:
central finite differences of the loss for the analytic gradient, a per-sample loop for
the forward pass, and one Adam step written out for single scalars."""
import numpy as np

from oracle import mlp


def _setup(seed=0, widths=(6, 9, 7, 5), B=4):
    rng = np.random.default_rng(seed)
    params = mlp.init_params(list(widths), seed)
    params = [(W, rng.normal(scale=0.3, size=b.shape)) for W, b in params]  # nonzero biases
    x = rng.normal(size=(B, widths[0]))
    t = rng.normal(size=(B, widths[-1]))
    return params, x, t


def test_forward_equals_a_per_sample_loop():
    params, x, t = _setup()
    y, _ = mlp.forward(params, x)
    for n in range(x.shape[0]):
        h = x[n]
        for l, (W, b) in enumerate(params):
            a = np.array([sum(h[i] * W[i, j] for i in range(W.shape[0])) + b[j] for j in range(W.shape[1])])
            h = a if l == len(params) - 1 else np.tanh(a)
        np.testing.assert_allclose(y[n], h, rtol=1e-13, atol=1e-14)


def test_gradient_equals_central_finite_differences():
    params, x, t = _setup(seed=3)
    grads = mlp.backward(params, x, t)
    eps = 1e-6
    rng = np.random.default_rng(7)
    for l, (W, b) in enumerate(params):
        for arr, g in ((W, grads[l][0]), (b, grads[l][1])):
            for _ in range(6):
                idx = tuple(rng.integers(0, s) for s in arr.shape)
                old = arr[idx]
                arr[idx] = old + eps
                lp = mlp.loss(params, x, t)
                arr[idx] = old - eps
                lm = mlp.loss(params, x, t)
                arr[idx] = old
                fd = (lp - lm) / (2 * eps)
                assert abs(fd - g[idx]) <= 1e-8 + 1e-6 * abs(fd), (l, idx, fd, g[idx])


def test_one_adam_step_by_hand():
    W = np.array([[0.5]])
    b = np.array([-0.25])
    gW = np.array([[0.2]])
    gb = np.array([-4.0])
    opt = mlp.Adam([(W, b)], lr=0.01, beta1=0.8, beta2=0.9, eps=1e-7)
    (W1, b1), = opt.step([(W, b)], [(gW, gb)])
    for p, g, p1 in ((0.5, 0.2, W1[0, 0]), (-0.25, -4.0, b1[0])):
        m = 0.2 * g
        v = 0.1 * g * g
        mh, vh = m / 0.2, v / 0.1
        assert abs(p1 - (p - 0.01 * mh / (np.sqrt(vh) + 1e-7))) < 1e-15
    # the first step moves every parameter by lr * sign(g) (up to eps)
    assert abs((W1[0, 0] - 0.5) + 0.01) < 1e-6 and abs((b1[0] + 0.25) - 0.01) < 1e-6
