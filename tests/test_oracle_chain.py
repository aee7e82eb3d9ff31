"""Pins of the oracle's chain maps (Eq. 2; Methods, orthogonal-polynomial chain map)."""
import numpy as np
import pytest
from scipy.special import roots_genlaguerre

from oracle.chain import chain_from_modes, chain_ohmic


@pytest.mark.parametrize("alpha,omega_c", [(0.1, 0.2), (0.3, 0.15)])
def test_ohmic_closed_form_matches_quadrature(alpha, omega_c):
    # Discretise J(w)/pi = 2 alpha w exp(-w/omega_c) with Gauss quadrature for the
    # weight x exp(-x) (x = w/omega_c), then chain-map the discrete modes by Lanczos.
    # The quadrature is exact for polynomials up to degree 2K-1, so the first
    # chain coefficients equal the continuous ones.
    K = 120
    x, wq = roots_genlaguerre(K, 1.0)
    omega = omega_c * x
    g2 = 2.0 * alpha * omega_c ** 2 * wq       # g_k^2, with sum g_k^2 = int J/pi
    lam = np.sqrt(2.0 * g2)                     # lambda_k = sqrt(2) g_k
    L = 8
    rc_q, on_q, hop_q = chain_from_modes(omega, lam, L)
    rc, on, hop = chain_ohmic(alpha, omega_c, L)
    assert abs(rc_q - rc) <= 1e-12 * rc
    np.testing.assert_allclose(on_q[:6], on[:6], rtol=1e-10)
    np.testing.assert_allclose(hop_q[:6], hop[:6], rtol=1e-10)
    # closed-form values spelled out for the first sites
    assert np.isclose(rc, 2 * omega_c * np.sqrt(alpha))
    assert np.isclose(on[0], 2 * omega_c) and np.isclose(on[1], 4 * omega_c)
    assert np.isclose(hop[0], omega_c * np.sqrt(2)) and np.isclose(hop[1], omega_c * np.sqrt(6))


def test_chain_from_modes_inverse_spectral_problem():
    # With as many sites as modes the chain is a unitary rotation of the star:
    # its spectrum is the mode set and its reaction-coordinate weights are lambda_k^2.
    rng = np.random.default_rng(11)
    K = 15
    omega = np.sort(rng.uniform(0.01, 0.2, K))
    lam = rng.uniform(0.001, 0.05, K)
    rc, on, hop = chain_from_modes(omega, lam, K)
    T = np.diag(on) + np.diag(hop, 1) + np.diag(hop, -1)
    w, S = np.linalg.eigh(T)
    np.testing.assert_allclose(w, omega, atol=1e-12)
    np.testing.assert_allclose((rc * S[0, :]) ** 2, lam ** 2, rtol=1e-9, atol=1e-16)
    assert np.isclose(rc ** 2, np.sum(lam ** 2))


def test_chain_from_modes_truncation_keeps_leading_coefficients():
    rng = np.random.default_rng(3)
    omega = np.sort(rng.uniform(0.01, 0.2, 40))
    lam = rng.uniform(0.001, 0.05, 40)
    full = chain_from_modes(omega, lam, 40)
    short = chain_from_modes(omega, lam, 10)
    np.testing.assert_allclose(short[1], full[1][:10], rtol=1e-12)
    np.testing.assert_allclose(short[2], full[2][:9], rtol=1e-12)
