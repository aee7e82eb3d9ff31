"""Orthogonal-polynomial chain maps (oracle; test infrastructure only).

The paper maps each environment (a set of harmonic modes that share one coupling
pattern Wbar_i, with strengths lambda_k) unitarily onto a 1D chain whose first
site is the reaction coordinate (Results, "Interface to TTNS", and Methods,
"Tensor Network States"; Eq. 2).  The chain Hamiltonian H_c,i is not written out
in the paper; the reading used here is the nearest-neighbour tight-binding chain

    H_c = sum_n omega_n a_n^+ a_n + sum_n t_n (a_n^+ a_{n+1} + h.c.),

with the system coupled through Wbar ||lambda|| (a_0 + a_0^+) / sqrt(2).
"""
from __future__ import annotations

import numpy as np


def chain_from_modes(omega: np.ndarray, lam: np.ndarray, L: int):
    """Chain map of discrete modes by the Lanczos tridiagonalisation of diag(omega)
    started from lam / ||lam||, with full re-orthogonalisation.

    Returns (rc, onsite[L], hop[L-1]) where rc = ||lam|| (Eq. 2), onsite = the
    Lanczos alphas and hop = the Lanczos betas.  L may not exceed the number of modes.
    """
    omega = np.asarray(omega, dtype=float)
    lam = np.asarray(lam, dtype=float)
    K = omega.size
    if L > K:
        raise ValueError("chain longer than the number of modes")
    rc = float(np.linalg.norm(lam))
    if rc == 0.0:
        # no coupling: any orthonormal chain basis works; take the modes themselves
        # in increasing frequency with zero hopping
        return 0.0, np.sort(omega)[:L].copy(), np.zeros(max(L - 1, 0))
    V = np.zeros((K, L))
    alpha = np.zeros(L)
    beta = np.zeros(max(L - 1, 0))
    V[:, 0] = lam / rc
    for n in range(L):
        w = omega * V[:, n]
        alpha[n] = V[:, n] @ w
        w = w - alpha[n] * V[:, n]
        if n > 0:
            w = w - beta[n - 1] * V[:, n - 1]
        for _ in range(2):  # full re-orthogonalisation, twice
            w = w - V[:, : n + 1] @ (V[:, : n + 1].T @ w)
        if n + 1 < L:
            b = np.linalg.norm(w)
            beta[n] = b
            V[:, n + 1] = w / b
    return rc, alpha, beta


def chain_ohmic(alpha: float, omega_c: float, L: int):
    """Closed-form chain of the Ohmic density J(w) = 2 pi alpha w exp(-w / omega_c).

    With J(w) = pi sum_k g_k^2 delta(w - w_k) and g_k = lambda_k / sqrt(2), the
    measure is J(w)/pi dw = 2 alpha w exp(-w/omega_c) dw, i.e. generalised Laguerre
    weight x exp(-x) (parameter 1) in x = w / omega_c.  Its monic recurrence has
    a_n = 2n + 2 and b_n = n (n + 1), so

        ||lambda|| = sqrt(2) * sqrt(2 alpha) omega_c = 2 omega_c sqrt(alpha),
        omega_n    = omega_c (2n + 2),
        t_n        = omega_c sqrt((n + 1)(n + 2)).
    """
    n = np.arange(L, dtype=float)
    rc = 2.0 * omega_c * np.sqrt(alpha)
    onsite = omega_c * (2.0 * n + 2.0)
    hop = omega_c * np.sqrt((n[:-1] + 1.0) * (n[:-1] + 2.0))
    return float(rc), onsite, hop


def chain_of(env_spectral, L: int):
    kind = env_spectral[0]
    if kind == "ohmic":
        return chain_ohmic(env_spectral[1], env_spectral[2], L)
    if kind == "modes":
        return chain_from_modes(env_spectral[1], env_spectral[2], L)
    raise ValueError(kind)
