"""Pins of the oracle's adaptive bond dimension (the bonds are raised until the dynamics
converge; Methods, tensor network states), against results that do not depend on it:

* growing leaves the state unchanged (its dense vector) and every non-root tensor an
  isometry toward its parent;
* growing every bond to the full Hilbert-space dimension makes the one-site integrator exact
  (every tangent-space projector is the identity): from t = 0 the run equals the dense state
  vector of Eq. 2, and from a later time it equals the exact evolution of the tree's own
  state at that time;
* the adaptive rule grows exactly the bonds whose smallest Schmidt weight exceeds eps.
"""
import numpy as np

from paper_1710_01362_gb300 import workloads as W
from oracle.statevector import Exact, dense_hamiltonian
from oracle.ttns import HBAR, TTNS


def isometry_error(st):
    tr = st.tree
    worst = 0.0
    for v in range(1, tr.n):
        A = st.A[v]
        M = A.reshape(A.shape[0], -1)  # the parent leg first
        worst = max(worst, np.abs(M @ M.conj().T - np.eye(A.shape[0])).max())
    return worst


def small(D, L=3):
    return W.sf_small(seed=11, n_env=2, L=L, d=3, D=D, n_modes=4, dt=0.5)


def test_growth_keeps_the_state_and_the_gauge():
    for p in (small(2), W.sf_small(seed=9, n_env=4, L=2, d=3, D=2, n_modes=6, n_steps=30, er_tree=True, D_er=2)):
        st = TTNS(p)
        for _ in range(6):
            st.step(p.dt)
        psi, pops, bonds = st.to_dense(), st.populations(), list(st.tree.bond)
        grown = st.grow_bonds([0] + [5] * (st.tree.n - 1))
        assert grown and all(st.tree.bond[v] > bonds[v] for v in grown)
        assert all(st.tree.bond[v] == bonds[v] for v in range(1, st.tree.n) if v not in grown)
        assert np.abs(st.to_dense() - psi).max() < 1e-13
        assert np.abs(st.populations() - pops).max() < 1e-13
        assert isometry_error(st) < 1e-13
        if not p.er_tree:
            # the environments were rebuilt from the new tensors: the energy is the dense one
            H, _ = dense_hamiltonian(p)
            psi = st.to_dense()
            assert abs(st.energy() - float(np.real(np.vdot(psi, H @ psi)))) < 1e-12


def test_growth_requests_below_the_current_dimension_change_nothing():
    p = small(3)
    st = TTNS(p)
    st.step(p.dt)
    A = [a.copy() for a in st.A]
    assert st.grow_bonds([0] * st.tree.n) == []
    assert st.grow_bonds([0] + [1] * (st.tree.n - 1)) == []
    assert all(np.array_equal(a, b) for a, b in zip(A, st.A))


def test_growth_to_full_dimension_at_t0_is_exact():
    p = small(1, L=2)
    st, ex = TTNS(p), Exact(p)
    st.grow_bonds([0] + [1 << 20] * (st.tree.n - 1))
    assert st.tree.bond == TTNS(small(1 << 20, L=2)).tree.bond
    for _ in range(16):
        st.step(p.dt)
    psi = ex.state(st.t)
    assert np.abs(st.to_dense() - psi).max() < 5e-8
    np.testing.assert_allclose(st.rho_el(), ex.rho_el(psi), atol=1e-8)


def test_growth_to_full_dimension_later_continues_exactly_from_the_tree_state():
    p = small(2, L=2)
    st, ex = TTNS(p), Exact(p)
    for _ in range(8):
        st.step(p.dt)
    st.grow_bonds([0] + [1 << 20] * (st.tree.n - 1))
    psi0, t0 = st.to_dense(), st.t
    for _ in range(10):
        st.step(p.dt)
    # exact evolution of the truncated run's own state from t0
    c0 = ex.S.conj().T @ psi0
    psi = ex.S @ (np.exp(-1j * ex.w * (st.t - t0) / HBAR) * c0)
    assert np.abs(st.to_dense() - psi).max() < 5e-8


def test_adaptive_rule_grows_the_bonds_with_large_smallest_weights():
    p = small(2)
    st = TTNS(p)
    for _ in range(10):
        st.step(p.dt)
    spec = st.bond_spectra()
    eps = float(np.median([w[0] for w in spec.values()]))
    expect = [v for v, w in spec.items() if w[0] > eps and st.tree.bond[v] < 6]
    ref = TTNS(p)
    for _ in range(10):
        ref.step(p.dt)
    req = [0] * st.tree.n
    for v in expect:
        req[v] = min(st.tree.bond[v] + 2, 6)
    grown = st.adapt_bonds(eps, 2, 6)
    assert grown == ref.grow_bonds(req)
    assert np.abs(st.to_dense() - ref.to_dense()).max() < 1e-13
    # nothing exceeds eps = 1 (weights are at most 1 and the smallest below 1 / D)
    assert st.adapt_bonds(1.0, 2, 6) == []


def test_growth_of_an_er_tree_to_full_dimension_is_exact():
    # ER nodes carry no physical leg: their bonds are clamped by products of child bonds only
    p = W.sf_small(seed=5, n_env=2, L=2, d=3, D=1, n_modes=4, dt=0.5, er_tree=True, D_er=1)
    st, ex = TTNS(p), Exact(p)
    assert st.tree.kind[1] == "er"
    st.grow_bonds([0] + [1 << 20] * (st.tree.n - 1))
    full = TTNS(W.sf_small(seed=5, n_env=2, L=2, d=3, D=64, n_modes=4, dt=0.5, er_tree=True, D_er=64))
    assert st.tree.bond == full.tree.bond
    for _ in range(10):
        st.step(p.dt)
    psi = ex.state(st.t)
    assert np.abs(st.to_dense() - psi).max() < 5e-8
