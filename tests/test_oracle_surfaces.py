"""Pins of the oracle's energy surfaces (Eq. 3-4): at full bond dimension they must equal
the surfaces computed from the dense state vector (its SVD, the dense Hamiltonian of Eq. 2
and the dense kinetic energy built term by term, none of it through the tree); with zero
system-bath coupling the state stays a product with the vacuum, so the total surfaces are
the eigenvalues of H_S (shifted by -tr H_S / n_el) and the potential surfaces those minus
the chains' zero-point kinetic energy sum_m w_m / 4."""
import numpy as np

from paper_1710_01362_gb300 import workloads as W
from oracle.chain import chain_of
from oracle.statevector import Exact, dense_kinetic, energy_surfaces
from oracle.ttns import TTNS


def _compare(p, steps, tol):
    st, ex = TTNS(p), Exact(p)
    T = dense_kinetic(p)
    for k in range(steps):
        st.step(p.dt)
        if k % 2 == 1:
            e_h, e_v, sig, _, _ = st.energy_surfaces()
            d_h, d_v, dsig = energy_surfaces(p, ex.H, T, st.to_dense())
            assert len(e_h) == len(d_h), (k, sig, dsig)
            np.testing.assert_allclose(sig, dsig, atol=tol)
            np.testing.assert_allclose(e_h, d_h, atol=tol)
            np.testing.assert_allclose(e_v, d_v, atol=tol)


def test_surfaces_equal_the_dense_state_vector_star_tree():
    _compare(W.sf_small(seed=11, n_env=2, L=2, d=3, D=64, n_modes=4, dt=0.5), 6, 1e-9)


def test_surfaces_equal_the_dense_state_vector_er_tree():
    _compare(W.sf_small(seed=5, n_env=2, L=2, d=3, D=64, n_modes=4, dt=0.5, er_tree=True, D_er=64), 6, 1e-9)


def test_surfaces_of_a_truncated_tree_equal_the_dense_matrix_elements_of_its_state():
    # at truncated bond dimension the TTNS state is still a definite vector: its surfaces
    # from the environment blocks must equal those of that vector with the dense operators
    _compare(W.sf_small(seed=11, n_env=2, L=3, d=3, D=3, n_modes=4, dt=0.5), 4, 1e-9)


def test_zero_coupling_surfaces_are_the_system_spectrum():
    p = W.rabi(eps=0.1, V=0.05, L=3, d=3, D=3)
    st = TTNS(p)
    for _ in range(5):
        st.step(p.dt)
    e_h, e_v, sig, _, _ = st.energy_surfaces()
    H_S = np.array(p.H_S) - np.trace(p.H_S).real / 2 * np.eye(2)
    lam = np.linalg.eigvalsh(H_S)
    assert len(sig) == 1 and abs(sig[0] - 1) < 1e-12
    np.testing.assert_allclose(e_h, lam, atol=1e-12)
    _, om, _ = chain_of(p.envs[0].spectral, p.envs[0].L)
    np.testing.assert_allclose(e_v, lam - 0.25 * om.sum(), atol=1e-12)


def test_kinetic_energy_of_one_quantum_in_a_normal_mode():
    # a chain of L = K sites is an exact orthogonal transform of K modes; one quantum in
    # normal mode n (sum_m U_mn a_m^+ |0>, U the eigenvectors of the chain's tridiagonal
    # matrix) has the harmonic-oscillator kinetic energy 3 w_n / 4 in that mode and w_k / 4
    # in the others: <T> = sum_k w_k / 4 + w_n / 2.  The hopping part of T enters through
    # the products U_mn U_(m+1)n, so a wrong sign or factor there fails this.
    w = np.array([0.11, 0.17, 0.26])
    lam = np.array([0.02, 0.03, 0.01])
    p = W.pure_dephasing(omega=w, lam=lam, L=3, d=4, D=64)
    _, om, hop = chain_of(p.envs[0].spectral, 3)
    h = np.diag(om) + np.diag(hop, 1) + np.diag(hop, -1)
    wn, U = np.linalg.eigh(h)
    np.testing.assert_allclose(wn, np.sort(w), atol=1e-12)
    T = dense_kinetic(p)
    d = 4
    for n in range(3):
        vec = np.zeros((p.n_el,) + (d,) * 3, dtype=complex)
        for m in range(3):
            idx = [0, 0, 0, 0]
            idx[1 + m] = 1
            vec[tuple(idx)] = U[m, n]
        v = vec.reshape(-1)
        assert abs(np.vdot(v, T @ v).real - (w.sum() / 4 + wn[n] / 2)) < 1e-12
