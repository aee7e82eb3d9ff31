"""Pins of the optimised-boson-basis trees (every chain site joined to a leaf holding its
Fock leg): with the OBB dimension equal to the Fock dimension and full bond dimensions
every tangent projector is the identity and the sweep must equal the dense state vector;
with a smaller OBB it is a truncation whose error against the exact state falls to zero as
the OBB dimension grows to the Fock dimension."""
import numpy as np

from paper_1710_01362_gb300 import workloads as W
from oracle.statevector import Exact
from oracle.ttns import TTNS


def _obb_problem(obb, D=64, seed=11):
    p = W.sf_small(seed=seed, n_env=2, L=2, d=3, D=D, n_modes=4, dt=0.5)
    for e in p.envs:
        e.obb = obb
    return p


def test_obb_tree_shape():
    st = TTNS(_obb_problem(2, D=4))
    tr = st.tree
    for nodes in tr.chain_nodes:
        for v in nodes:
            assert tr.kind[v] == "obb" and tr.phys[v] == 3 and tr.bond[v] == 2
            assert tr.kind[tr.parent[v]] == "site" and tr.phys[tr.parent[v]] == 0


def test_full_obb_and_bonds_are_exact():
    p = _obb_problem(3)
    st, ex = TTNS(p), Exact(p)
    for _ in range(8):
        st.step(p.dt)
    psi = ex.state(st.t)
    assert np.abs(st.to_dense() - psi).max() < 5e-8
    np.testing.assert_allclose(st.occupations(), ex.occupations(psi), atol=5e-9)


def test_obb_error_falls_to_zero_with_the_obb_dimension():
    errs = []
    for obb in (1, 2, 3):
        p = _obb_problem(obb)
        st, ex = TTNS(p), Exact(p)
        for _ in range(10):
            st.step(p.dt)
        errs.append(np.abs(st.populations() - np.real(np.diag(ex.rho_el(ex.state(st.t))))).max())
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-8 and errs[0] > 1e-6
