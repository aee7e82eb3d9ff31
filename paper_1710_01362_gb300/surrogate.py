"""Surrogate of the TTNS sweep: a multilayer perceptron from 30 Hamiltonian parameters to the
electronic population trajectory, trained on batched TTNS runs, with the plain TTNS sweep as
its fallback and the judge of its error.

Network (widths 30 -> 256 -> 256 -> 256 -> 5 * n_points, tanh hidden layers, linear
output): FP32 weights trained with Adam on the squared loss, every layer product on the
tensor cores through ttns_mlp_gemm (3xTF32 for training, one BF16 product for inference),
gradients by backpropagation through the library's kernels.  This module only sequences
those calls and holds the weights in torch device tensors; no arithmetic of the network
runs here.

Fallback: two networks trained from different initialisations form an ensemble; their
disagreement, scaled by a factor calibrated on a validation split, is the predicted error
of a prediction.  Parameter sets whose predicted error exceeds the threshold (1e-3) are
run through the TTNS sweep instead.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import time
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import ttns
from . import workloads as W

N_STATES = 5
WIDTHS_HIDDEN = [256, 256, 256]
KIND_TRAIN = 1   # 3xTF32
KIND_INFER = 3   # one BF16 product


def _check(code: int) -> None:
    if code != 0:
        raise ttns.TTNSError(code, ttns.lib().ttns_last_error().decode())


def _p(t) -> int:
    return t.data_ptr()


# ------------------------------------------------------------------ training data
def generate(seeds: Sequence[int], n_points: int = 200, L: int = 8, d: int = 6, D: int = 8, dt: float = 1.0,
             precision: int = ttns.TTNS_TF32X3, chunk: int = 2048, cluster_ctas: int = 1,
             stream: Optional[int] = None):
    """TTNS population trajectories of the surrogate workload, batched: returns X (n x 30),
    Y (n x n_points * 5, populations after every step, step-major) and the device seconds."""
    X = np.stack([W.surrogate_params(s) for s in seeds])
    Y = np.zeros((len(seeds), n_points * N_STATES))
    secs = 0.0
    for c0 in range(0, len(seeds), chunk):
        probs = [W.surrogate_problem(X[k], L=L, d=d, D=D, dt=dt, n_steps=n_points)
                 for k in range(c0, min(len(seeds), c0 + chunk))]
        t0 = time.perf_counter()
        tree = ttns.Tree(probs, precision=precision, record=True, max_record=n_points, cluster_ctas=cluster_ctas,
                         stream=stream)
        tree.step(dt, n_points)
        tree.sync()
        secs += time.perf_counter() - t0
        for k in range(len(probs)):
            tr = tree.trajectory(k, max_steps=n_points)
            Y[c0 + k] = np.real(np.einsum("kii->ki", tr)).reshape(-1)
        tree.close()
    return X, Y, secs


# ------------------------------------------------------------------ the network
class Net:
    """Weights W_l (n_{l-1} x n_l, row-major) and biases b_l as torch float32 device tensors."""

    def __init__(self, widths: List[int], seed: int, device="cuda"):
        import torch
        self.torch = torch
        self.widths = list(widths)
        self.device = device
        rng = np.random.default_rng(seed)
        self.W, self.b = [], []
        for a, c in zip(widths[:-1], widths[1:]):
            lim = math.sqrt(6.0 / (a + c))
            self.W.append(torch.tensor(rng.uniform(-lim, lim, size=(a, c)), dtype=torch.float32, device=device))
            self.b.append(torch.zeros(c, dtype=torch.float32, device=device))
        self.mW = [torch.zeros_like(w) for w in self.W]
        self.vW = [torch.zeros_like(w) for w in self.W]
        self.mb = [torch.zeros_like(b) for b in self.b]
        self.vb = [torch.zeros_like(b) for b in self.b]
        self.step_count = 0
        self.x_mean = None
        self.x_std = None

    @property
    def n_layers(self) -> int:
        return len(self.W)

    def set_params(self, params) -> None:
        """Weights from host arrays [(W, b)] (float64 or float32)."""
        torch = self.torch
        for l, (Wl, bl) in enumerate(params):
            self.W[l] = torch.tensor(np.asarray(Wl), dtype=torch.float32, device=self.device).contiguous()
            self.b[l] = torch.tensor(np.asarray(bl), dtype=torch.float32, device=self.device).contiguous()

    def forward(self, x, kind: int = KIND_TRAIN, stream: Optional[int] = None):
        """Returns the output and the layer outputs [h_0 = x, h_1, .., h_{L-1}]."""
        torch = self.torch
        hs = [x]
        h = x
        L = self.n_layers
        lib = ttns.lib()
        for l in range(L):
            M, K = h.shape
            N = self.widths[l + 1]
            out = torch.empty((M, N), dtype=torch.float32, device=self.device)
            _check(lib.ttns_mlp_gemm(kind, M, N, K, _p(h), K, 0, _p(self.W[l]), N, 0, _p(out), N,
                                     1 if l == L - 1 else 2, _p(self.b[l]), stream))
            h = out
            if l < L - 1:
                hs.append(h)
        return h, hs

    def backward(self, hs, y, t, stream: Optional[int] = None):
        """Gradients [(dW_l, db_l)] of sum (y - t)^2 / (2 batch)."""
        torch = self.torch
        lib = ttns.lib()
        B = y.shape[0]
        d = torch.empty_like(y)
        _check(lib.ttns_mlp_diff(_p(y), _p(t), _p(d), y.numel(), 1.0 / B, stream))
        grads = [None] * self.n_layers
        for l in range(self.n_layers - 1, -1, -1):
            h_prev = hs[l]
            K_in, N_out = self.W[l].shape
            dW = torch.empty_like(self.W[l])
            db = torch.empty_like(self.b[l])
            # dW = h_prev^T d  (n_in x n_out, inner dimension = batch)
            _check(lib.ttns_mlp_gemm(KIND_TRAIN, K_in, N_out, B, _p(h_prev), K_in, 1, _p(d), N_out, 0, _p(dW), N_out,
                                     0, None, stream))
            _check(lib.ttns_mlp_colsum(_p(d), B, N_out, N_out, _p(db), stream))
            grads[l] = (dW, db)
            if l > 0:
                # d_prev = (d W^T) * (1 - h_prev^2)
                dn = torch.empty((B, K_in), dtype=torch.float32, device=self.device)
                _check(lib.ttns_mlp_gemm(KIND_TRAIN, B, K_in, N_out, _p(d), N_out, 0, _p(self.W[l]), N_out, 1, _p(dn),
                                         K_in, 3, _p(h_prev), stream))
                d = dn
        return grads

    def adam(self, grads, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, stream: Optional[int] = None) -> None:
        lib = ttns.lib()
        self.step_count += 1
        for l, (dW, db) in enumerate(grads):
            _check(lib.ttns_mlp_adam(_p(self.W[l]), _p(dW), _p(self.mW[l]), _p(self.vW[l]), self.W[l].numel(), lr,
                                     beta1, beta2, eps, self.step_count, stream))
            _check(lib.ttns_mlp_adam(_p(self.b[l]), _p(db), _p(self.mb[l]), _p(self.vb[l]), self.b[l].numel(), lr,
                                     beta1, beta2, eps, self.step_count, stream))

    # ---------------------------------------------------------------- training / inference
    def fit(self, X: np.ndarray, Y: np.ndarray, epochs: int = 200, batch: int = 256, lr: float = 1e-3,
            lr_final: float = 1e-5, seed: int = 0, log_every: int = 0):
        """Adam on standardised inputs; the learning rate decays geometrically to lr_final."""
        torch = self.torch
        self.x_mean = X.mean(axis=0)
        self.x_std = X.std(axis=0) + 1e-12
        Xd = torch.tensor((X - self.x_mean) / self.x_std, dtype=torch.float32, device=self.device)
        Yd = torch.tensor(Y, dtype=torch.float32, device=self.device)
        n = X.shape[0]
        rng = np.random.default_rng(seed)
        steps = epochs * max(1, n // batch)
        gamma = (lr_final / lr) ** (1.0 / max(1, steps))
        rate = lr
        losses = []
        for ep in range(epochs):
            perm = torch.tensor(rng.permutation(n), device=self.device)
            tot = 0.0
            for k in range(0, n - batch + 1, batch):
                idx = perm[k:k + batch]
                xb, yb = Xd[idx].contiguous(), Yd[idx].contiguous()
                y, hs = self.forward(xb)
                grads = self.backward(hs, y, yb)
                self.adam(grads, rate)
                rate *= gamma
                if log_every and ep % log_every == 0:
                    tot += float(((y - yb) ** 2).sum()) / (2 * batch)
            if log_every and ep % log_every == 0:
                losses.append((ep, tot))
        return losses

    def predict(self, X: np.ndarray, kind: int = KIND_INFER) -> np.ndarray:
        torch = self.torch
        Xd = torch.tensor((X - self.x_mean) / self.x_std, dtype=torch.float32, device=self.device)
        y, _ = self.forward(Xd, kind=kind)
        torch.cuda.synchronize()
        return y.double().cpu().numpy()


class Surrogate:
    """Ensemble of two networks with a calibrated predicted error and the TTNS fallback."""

    def __init__(self, n_points: int = 200, seed: int = 0, device="cuda"):
        self.n_points = n_points
        widths = [W.SURROGATE_N_PARAMS] + WIDTHS_HIDDEN + [N_STATES * n_points]
        self.nets = [Net(widths, seed + 101 * k, device) for k in range(2)]
        self.scale = 1.0

    def fit(self, X, Y, X_cal, Y_cal, quantile: float = 0.95, seed: int = 0, **kw):
        for k, net in enumerate(self.nets):
            net.fit(X, Y, seed=seed + k, **kw)
        # calibration: the scale that makes the disagreement bound the true error on the
        # calibration split for the given fraction of its samples
        mean, dis = self.predict_raw(X_cal)
        err = np.abs(mean - Y_cal).max(axis=1)
        ratio = err / np.maximum(dis, 1e-12)
        self.scale = float(np.quantile(ratio, quantile))
        return self

    def predict_raw(self, X, kind: int = KIND_INFER):
        ys = [net.predict(X, kind) for net in self.nets]
        mean = 0.5 * (ys[0] + ys[1])
        dis = np.abs(ys[0] - ys[1]).max(axis=1)
        return mean, dis

    def predict(self, X, threshold: float = 1e-3, kind: int = KIND_INFER, fallback=None):
        """Predictions with their predicted errors; rows above the threshold are replaced by
        fallback(rows) (the TTNS runs) when a fallback is given.  Returns (Y, predicted
        error, mask of rows that fell back)."""
        mean, dis = self.predict_raw(X, kind)
        pred_err = self.scale * dis
        back = pred_err > threshold
        Y = mean.copy()
        if fallback is not None and back.any():
            Y[back] = fallback(np.nonzero(back)[0])
        return Y, pred_err, back


# ------------------------------------------------------------------ end-to-end run
def run(n_train: int, n_cal: int, n_test: int, n_points: int = 200, epochs: int = 200, batch: int = 256,
        threshold: float = 1e-3, seed0: int = 100000, cluster_ctas: int = 1, out: Optional[str] = None,
        data: Optional[str] = None, lr: float = 1e-3, lr_final: float = 1e-5) -> dict:
    """Data from batched TTNS runs (training seeds seed0.., then calibration, then held-out),
    the ensemble trained on the GPU, its held-out error in BF16 inference, and what it gains:
    the held-out parameter sets answered by the network within the threshold, the rest by the
    sweep, against the sweep alone."""
    import json
    import torch
    seeds = list(range(seed0, seed0 + n_train + n_cal + n_test))
    if data and os.path.exists(data):
        # a dataset written by an earlier run (the same seeds and workload)
        z = np.load(data)
        if list(z["seeds"]) != seeds or int(z["n_points"]) != n_points:
            raise ValueError(f"{data} holds other seeds or trajectory lengths")
        X, Y, gen_s = z["X"].astype(np.float64), z["Y"].astype(np.float64), float(z["generation_seconds"])
    else:
        X, Y, gen_s = generate(seeds, n_points=n_points, cluster_ctas=cluster_ctas)
        if data:
            np.savez_compressed(data, X=X, Y=Y.astype(np.float32), seeds=np.array(seeds), n_points=n_points,
                                generation_seconds=gen_s)
    tr = slice(0, n_train)
    ca = slice(n_train, n_train + n_cal)
    te = slice(n_train + n_cal, n_train + n_cal + n_test)
    sur = Surrogate(n_points=n_points, seed=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sur.fit(X[tr], Y[tr], X[ca], Y[ca], epochs=epochs, batch=batch, lr=lr, lr_final=lr_final)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    Yp, perr, back = sur.predict(X[te], threshold=threshold)
    infer_s = time.perf_counter() - t0
    err = np.abs(Yp - Y[te]).max(axis=1)
    ttns_per_run = gen_s / len(seeds)
    accepted = ~back
    res = {
        "n_train": n_train, "n_cal": n_cal, "n_test": n_test, "n_points": n_points, "epochs": epochs,
        "tree": "ER tree, 5 states, 8 chains x 8 sites, d 6, D 8, dt 1 fs",
        "ttns_seconds_per_run_batched": ttns_per_run, "generation_seconds": gen_s, "train_seconds": train_s,
        "inference_seconds": infer_s,
        "heldout_max_error": {"median": float(np.median(err)), "p90": float(np.quantile(err, 0.9)),
                              "p99": float(np.quantile(err, 0.99)), "max": float(err.max())},
        "heldout_rms_error": float(np.sqrt(np.mean((Yp - Y[te]) ** 2))),
        "predicted_error_scale": sur.scale,
        "threshold": threshold,
        "accepted_fraction": float(accepted.mean()),
        "accepted_max_error": float(err[accepted].max()) if accepted.any() else None,
        "accepted_within_threshold": float((err[accepted] <= threshold).mean()) if accepted.any() else None,
        "time_ttns_only": ttns_per_run * n_test,
        "time_with_surrogate": infer_s + ttns_per_run * int(back.sum()),
    }
    if out:
        with open(out, "w") as f:
            json.dump(res, f, indent=1)
    return res


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="train and evaluate the TTNS surrogate on the GPU")
    ap.add_argument("--n-train", type=int, default=20000)
    ap.add_argument("--n-cal", type=int, default=1000)
    ap.add_argument("--n-test", type=int, default=1000)
    ap.add_argument("--n-points", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--threshold", type=float, default=1e-3)
    ap.add_argument("--cluster-ctas", type=int, default=1)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-final", type=float, default=1e-5)
    ap.add_argument("--data", default="", help=".npz dataset: read if present, else written")
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    print(json.dumps(run(a.n_train, a.n_cal, a.n_test, a.n_points, a.epochs, batch=a.batch, threshold=a.threshold,
                         cluster_ctas=a.cluster_ctas, out=a.out or None, data=a.data or None, lr=a.lr,
                         lr_final=a.lr_final), indent=1))
