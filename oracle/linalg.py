"""Householder QR with a fixed completion rule, and the Lanczos matrix exponential
(oracle; test infrastructure only).

The paper re-gauges the tree between local updates with a matrix factorisation
("the SVD is a central element in the numerical algorithm for updating and
normalising the TTNS", Results, energy-surface section) and evolves every tensor
with its local effective Hamiltonian (Results, "TDVP for TTNS").  The
Supplement that fixes the algorithm is not part of the paper, so the readings
below are used (they are the same on the CUDA side):

QR  (complex Householder, column by column)
    For column j the remaining sub-column x = M[j:, j] is reflected onto
    alpha e_0 with alpha = -exp(i arg x_0) ||x||.  If ||x|| <= cutoff ||M||_F the
    reflector is the identity, R_jj = 0 and the sub-column is dropped.
    Q = H_0 ... H_{n-1} I[:, :n].  Every column j is re-phased so that R_jj is real
    and >= 0, and R is rescaled to ||R||_F = ||M||_F (the dropped weight is returned to
    the kept content; at cutoff 1e-8 the factor is 1 to ~1e-16).
    The cutoff is a truncation parameter of the run, like the bond dimension: 1e-8
    (four orders above the Krylov tolerance) keeps the step exact at full bond
    dimension and suffices where bonds are well filled; 1e-3 is used for trees whose
    bonds fill up during the run (long spin-boson chains, the ER tree), where kept
    columns between 1e-8 and 1e-3 of the norm amplify rounding-level differences by
    ~10-30 per step (measured: two oracle runs with Krylov tolerances 1e-12 and 1e-14
    drift 1e-3 apart within 30 steps at 1e-8, stay within 1e-9 over 40-60 steps at 1e-3
    with the rescale).

Krylov exponential  y = exp(-i s H) v  (s = time / hbar, any sign)
    Lanczos with classical Gram-Schmidt run twice against all previous vectors
    (full re-orthogonalisation).  After step j the tridiagonal T is
    exponentiated through its eigen-decomposition; the step stops when
    beta_{j+1} |e_j^T exp(-i s T) e_0| <= tol (Saad's estimate).  If mmax steps
    do not reach tol, the time is split: the largest s / 2^k whose estimate on
    the same Krylov space reaches tol is taken, and a new space is built from the
    result for the remaining time (long chains whose onsite energies grow along
    the chain have local Hamiltonians too wide for one space of dimension 30).
"""
from __future__ import annotations

import numpy as np

QR_NULL_REL = 1e-8
KRYLOV_TOL = 1e-12
KRYLOV_MMAX = 30


def householder_qr(M: np.ndarray, cutoff: float | None = None):
    """QR of an m x n complex matrix (m >= n) with the completion rule above.

    Returns Q (m x n, orthonormal columns) and R (n x n, upper triangular with a
    real non-negative diagonal) such that M = Q R up to the dropped sub-columns (norm at
    most cutoff * ||M||_F each, default QR_NULL_REL); R is then rescaled so that
    ||R||_F = ||M||_F, which keeps the norm of the state that the dropped content carried.
    """
    M = np.array(M, dtype=complex)
    m, n = M.shape
    if m < n:
        raise ValueError("householder_qr needs rows >= cols")
    fro = np.sqrt(np.sum(np.abs(M) ** 2))
    thr = (QR_NULL_REL if cutoff is None else cutoff) * fro
    W = M.copy()
    vs = []
    for j in range(n):
        x = W[j:, j]
        sigma = np.sqrt(np.sum(np.abs(x) ** 2))
        if sigma <= thr or sigma == 0.0:
            vs.append(None)
            # the identity reflector leaves column j as it is below the diagonal;
            # only its diagonal entry is kept in R, set to zero
            W[j, j] = 0.0
            W[j + 1:, j] = 0.0
            continue
        x0 = x[0]
        # a head below 1e-280 (far below any amplitude that matters; its reciprocal would
        # overflow) is treated as zero: phase 1
        phase = x0 / abs(x0) if abs(x0) > 1e-280 else 1.0 + 0.0j
        alpha = -phase * sigma
        v = x.copy()
        v[0] -= alpha
        vnorm2 = np.real(np.vdot(v, v))
        # apply H = I - 2 v v^H / (v^H v) to the trailing block
        sub = W[j:, j:]
        coef = (2.0 / vnorm2) * (v.conj() @ sub)
        sub -= np.outer(v, coef)
        W[j:, j:] = sub
        W[j, j] = alpha
        W[j + 1:, j] = 0.0
        vs.append(v)
    R = np.triu(W[:n, :n])
    # Q = H_0 H_1 ... H_{n-1} applied to the first n columns of the identity
    Q = np.zeros((m, n), dtype=complex)
    Q[np.arange(n), np.arange(n)] = 1.0
    for j in range(n - 1, -1, -1):
        v = vs[j]
        if v is None:
            continue
        vnorm2 = np.real(np.vdot(v, v))
        sub = Q[j:, :]
        coef = (2.0 / vnorm2) * (v.conj() @ sub)
        Q[j:, :] = sub - np.outer(v, coef)
    # make the diagonal of R real and non-negative
    for j in range(n):
        r = R[j, j]
        if abs(r) > 0.0:
            ph = r / abs(r)
            Q[:, j] *= ph
            R[j, :] *= np.conj(ph)
            R[j, j] = abs(r)
    nr = np.sqrt(np.sum(np.abs(R) ** 2))
    if nr > 0.0:
        R *= fro / nr
    return Q, R


def expm_tridiag_e0(alpha: np.ndarray, beta: np.ndarray, s: float) -> np.ndarray:
    """exp(-i s T) e_0 for the real symmetric tridiagonal T (diagonal alpha,
    off-diagonal beta), through T = S diag(w) S^T."""
    m = alpha.size
    T = np.diag(alpha)
    if m > 1:
        T += np.diag(beta[: m - 1], 1) + np.diag(beta[: m - 1], -1)
    w, S = np.linalg.eigh(T)
    return S @ (np.exp(-1j * s * w) * S[0, :])


def _lanczos_chunk(apply_H, v: np.ndarray, shape, s: float, tol: float, mmax: int, stats):
    """One Krylov space from v.  Returns (y, s_done): y = exp(-i s_done H) v with
    s_done = s when the estimate reaches tol within mmax steps, else the largest
    s / 2^k whose estimate on the same space reaches tol."""
    beta0 = np.linalg.norm(v)
    n = v.size
    mmax = min(mmax, n)
    Qk = np.zeros((mmax, n), dtype=complex)
    alpha = np.zeros(mmax)
    beta = np.zeros(mmax)
    Qk[0] = v / beta0
    u = None
    m = 0
    err = 0.0
    b = 0.0
    for j in range(mmax):
        w = np.asarray(apply_H(Qk[j].reshape(shape)), dtype=complex).reshape(-1)
        alpha[j] = np.real(np.vdot(Qk[j], w))
        w = w - alpha[j] * Qk[j]
        if j > 0:
            w = w - beta[j - 1] * Qk[j - 1]
        for _ in range(2):
            w = w - Qk[: j + 1].T @ (Qk[: j + 1].conj() @ w)
        b = np.linalg.norm(w)
        beta[j] = b
        u = expm_tridiag_e0(alpha[: j + 1], beta[:j], s)
        m = j + 1
        err = b * abs(u[j])
        if err <= tol or j + 1 == mmax:
            break
        Qk[j + 1] = w / b
    if stats is not None:
        stats["krylov_iters"] = stats.get("krylov_iters", 0) + m
        stats["applies"] = stats.get("applies", 0) + m
    s_done = s
    if err > tol and m < n:
        # time-substep on the same Krylov space: the largest s / 2^k that converges
        s_done = s
        for _ in range(30):
            s_done = 0.5 * s_done
            u = expm_tridiag_e0(alpha[:m], beta[: m - 1], s_done)
            if b * abs(u[m - 1]) <= tol:
                break
    return beta0 * (u @ Qk[:m]), s_done


def expm_lanczos(apply_H, v: np.ndarray, s: float, tol: float = KRYLOV_TOL,
                 mmax: int = KRYLOV_MMAX, stats: dict | None = None) -> np.ndarray:
    """y = exp(-i s H) v for Hermitian H given as a matrix-free apply_H(x).

    When mmax Lanczos steps do not reach the tolerance for the whole time s, the
    step is split: the largest s / 2^k that converges on the current Krylov
    space is taken, and a new space is built from the result for the rest."""
    shape = v.shape
    y = np.asarray(v, dtype=complex).reshape(-1)
    if np.linalg.norm(y) == 0.0:
        return y.reshape(shape).copy()
    remaining = s
    for chunk in range(64):
        y, done = _lanczos_chunk(apply_H, y, shape, remaining, tol, mmax, stats)
        if done == remaining:
            break
        remaining = remaining - done
        if stats is not None:
            stats["substeps"] = stats.get("substeps", 0) + 1
    else:
        if stats is not None:
            stats["not_converged"] = stats.get("not_converged", 0) + 1
    return y.reshape(shape)
