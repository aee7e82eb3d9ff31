"""Grouping of vibrational modes into environments by weighted k-means (oracle; test
infrastructure only).

The paper's Hamiltonian couples every mode n through its own electronic pattern W_n
(Eq. 1); the chain transformation needs modes that share one pattern, W_n = lambda_n
Wbar_n.  The paper groups modes with similar normalised patterns by k-means clustering
with k-means++ seeding (Results, "Interface to TTNS"), and each cluster becomes one
environment i with a pattern Wbar_i (Eq. 2).  Readings:

  * pattern and strength of a mode: lambda_n = ||W_n||_F and Wbar_n = W_n / lambda_n; W and
    -W describe the same coupling direction (the sign goes into lambda), so the clustering
    is sign-invariant: a mode is compared with a centre c after the sign s = sign(<x, c>)
    (+1 at zero) that aligns it, at the distance ||x||^2 + ||c||^2 - 2 |<x, c>|;
  * features: the real and imaginary parts of Wbar_n, flattened (2 n_el^2 reals); weights
    w_n = lambda_n^2 (the mode's coupling strength);
  * Lloyd iterations from given initial centres (the k-means++ draw is an input, so that the
    random numbers stay outside the algorithm): assign every mode to the nearest centre (ties
    to the lower index), move every centre to the weighted mean of its modes, each aligned by
    its sign (an empty cluster keeps its centre), until no assignment changes;
  * environment i: Wbar_i = centre_i / ||centre_i||_F, and each of its modes couples with
    lambda_{n,i} = Re <Wbar_i, W_n>_F (the least-squares strength along the pattern).
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np


def pattern_and_strength(W: np.ndarray) -> Tuple[np.ndarray, float]:
    W = np.asarray(W, dtype=complex)
    lam = float(np.sqrt(np.sum(np.abs(W) ** 2)))
    if lam == 0.0:
        return np.zeros_like(W), 0.0
    return W / lam, lam


def features(Wb: np.ndarray) -> np.ndarray:
    return np.concatenate([Wb.real.reshape(-1), Wb.imag.reshape(-1)])


def weighted_kmeans(X: np.ndarray, w: np.ndarray, centers0: np.ndarray, max_iter: int = 100):
    """Sign-invariant Lloyd iterations; returns (assignment, centres, iterations)."""
    C = np.array(centers0, dtype=float)
    k = C.shape[0]
    assign = np.full(X.shape[0], -1)
    xx = (X ** 2).sum(axis=1)
    it = 0
    for it in range(1, max_iter + 1):
        dots = X @ C.T
        d = xx[:, None] + (C ** 2).sum(axis=1)[None, :] - 2.0 * np.abs(dots)
        new = np.argmin(d, axis=1)           # first minimum: ties go to the lower index
        changed = np.any(new != assign)
        assign = new
        sgn = np.where(dots[np.arange(len(X)), assign] >= 0.0, 1.0, -1.0)
        for c in range(k):
            m = assign == c
            if m.any():
                C[c] = ((w[m] * sgn[m])[:, None] * X[m]).sum(axis=0) / w[m].sum()
        if not changed:
            break
    return assign, C, it


def cluster_modes(W: np.ndarray, k: int, init: List[int], max_iter: int = 100):
    """W: (n_modes, n_el, n_el) coupling matrices.  Returns (assignment, Wbar_i (k, n_el,
    n_el), lambda_{n, i(n)} (n_modes,), iterations)."""
    n_modes, n_el, _ = W.shape
    pats, lams = zip(*[pattern_and_strength(W[n]) for n in range(n_modes)])
    X = np.array([features(p) for p in pats])
    w = np.array(lams) ** 2
    assign, C, it = weighted_kmeans(X, w, X[list(init)], max_iter)
    Wbar = np.zeros((k, n_el, n_el), dtype=complex)
    for c in range(k):
        M = C[c, : n_el * n_el].reshape(n_el, n_el) + 1j * C[c, n_el * n_el:].reshape(n_el, n_el)
        nrm = np.sqrt(np.sum(np.abs(M) ** 2))
        Wbar[c] = M / nrm if nrm > 0 else M
    lam = np.array([np.real(np.vdot(Wbar[assign[n]], W[n])) for n in range(n_modes)])
    return assign, Wbar, lam, it
