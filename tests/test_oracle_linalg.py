"""Pins of the oracle's QR and Krylov exponential against numpy / scipy."""
import numpy as np
import pytest
import scipy.linalg

from oracle.linalg import expm_lanczos, expm_tridiag_e0, householder_qr


def _rand(rng, m, n):
    return rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))


@pytest.mark.parametrize("m,n", [(8, 8), (40, 6), (200, 20)])
def test_qr_matches_numpy_up_to_phases(m, n):
    rng = np.random.default_rng(m * 100 + n)
    M = _rand(rng, m, n)
    Q, R = householder_qr(M)
    Qn, Rn = np.linalg.qr(M)
    ph = np.diag(Rn) / np.abs(np.diag(Rn))
    Qn = Qn * ph
    Rn = np.conj(ph)[:, None] * Rn
    np.testing.assert_allclose(Q, Qn, atol=1e-12)
    np.testing.assert_allclose(R, Rn, atol=1e-12)
    assert np.all(np.abs(np.imag(np.diag(R))) == 0) and np.all(np.real(np.diag(R)) >= 0)
    np.testing.assert_allclose(Q @ R, M, atol=1e-12)
    np.testing.assert_allclose(Q.conj().T @ Q, np.eye(n), atol=1e-12)


def test_qr_rank_deficient_completion_rule():
    # columns 1 and 3 are zero: identity reflectors, R_jj = 0, Q still orthonormal,
    # and the completion column j is H_0 ... H_{j-1} e_j
    rng = np.random.default_rng(5)
    M = _rand(rng, 10, 4)
    M[:, 1] = 0.0
    M[:, 3] = 0.0
    Q, R = householder_qr(M)
    np.testing.assert_allclose(Q @ R, M, atol=1e-12)
    np.testing.assert_allclose(Q.conj().T @ Q, np.eye(4), atol=1e-12)
    assert R[1, 1] == 0 and R[3, 3] == 0
    # column 1 of Q: the first reflector applied to e_1 (phase of column 1 untouched)
    x = M[:, 0]
    sigma = np.linalg.norm(x)
    alpha = -x[0] / abs(x[0]) * sigma
    v = x.copy()
    v[0] -= alpha
    H0 = np.eye(10) - 2.0 * np.outer(v, v.conj()) / np.vdot(v, v).real
    np.testing.assert_allclose(Q[:, 1], H0[:, 1], atol=1e-12)


def test_qr_all_zero_matrix_gives_identity_columns():
    Q, R = householder_qr(np.zeros((6, 3), dtype=complex))
    np.testing.assert_allclose(Q, np.eye(6)[:, :3])
    assert np.all(R == 0)


@pytest.mark.parametrize("s", [0.3, 2.0, -1.5])
def test_tridiagonal_exponential(s):
    rng = np.random.default_rng(2)
    a = rng.standard_normal(9)
    b = rng.uniform(0.1, 1.0, 8)
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    ref = scipy.linalg.expm(-1j * s * T)[:, 0]
    np.testing.assert_allclose(expm_tridiag_e0(a, b, s), ref, atol=1e-13)


@pytest.mark.parametrize("s", [0.2, 1.0, -0.7])
def test_lanczos_exponential_matches_expm(s):
    rng = np.random.default_rng(7)
    n = 120
    X = _rand(rng, n, n)
    H = 0.5 * (X + X.conj().T) / np.sqrt(n)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = scipy.linalg.expm(-1j * s * H) @ v
    y = expm_lanczos(lambda x: H @ x, v, s)
    assert np.linalg.norm(y - ref) <= 1e-11 * np.linalg.norm(v)
    assert abs(np.linalg.norm(y) - np.linalg.norm(v)) <= 1e-12 * np.linalg.norm(v)


def test_lanczos_invariant_subspace_is_exact():
    # v in a 3-dimensional invariant subspace: exact after 3 steps (beta -> 0)
    n = 30
    H = np.diag(np.linspace(-1, 1, n)).astype(complex)
    v = np.zeros(n, dtype=complex)
    v[[2, 10, 20]] = [1.0, 2.0j, -1.0]
    stats = {}
    y = expm_lanczos(lambda x: H @ x, v, 3.0, stats=stats)
    ref = np.exp(-3.0j * np.diag(H)) * v
    np.testing.assert_allclose(y, ref, atol=1e-13)
    assert stats["krylov_iters"] <= 4


def test_lanczos_substeps_when_the_space_is_too_small():
    # a wide spectrum and a long time: 10 Krylov vectors cannot reach 1e-12 in one go,
    # the step is split and the result still matches expm
    rng = np.random.default_rng(4)
    n = 200
    X = _rand(rng, n, n)
    H = 2.0 * (X + X.conj().T) / np.sqrt(n)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = scipy.linalg.expm(-1j * 1.0 * H) @ v
    stats = {}
    y = expm_lanczos(lambda x: H @ x, v, 1.0, mmax=10, stats=stats)
    assert stats.get("substeps", 0) > 0 and stats.get("not_converged", 0) == 0
    assert np.linalg.norm(y - ref) <= 1e-9 * np.linalg.norm(v)
