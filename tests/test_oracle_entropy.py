"""Pins of the oracle's entanglement entropies: at full bond dimension the entropy of the
bond between node v and its parent must equal the entanglement entropy of the dense state
vector for the bipartition (physical sites of v's subtree) | (the rest), computed by an
SVD of the regrouped vector; S(rho_S) is the electronic one; a product state has zero
entropy everywhere."""
import numpy as np

from paper_1710_01362_gb300 import workloads as W
from oracle.ttns import TTNS


def _dense_entropy(psi, dims, part):
    """Entanglement entropy of psi (legs of sizes dims) for the legs in `part` vs the rest."""
    rest = [k for k in range(len(dims)) if k not in part]
    T = psi.reshape(dims).transpose(list(part) + rest)
    M = T.reshape(int(np.prod([dims[k] for k in part])), -1)
    s = np.linalg.svd(M, compute_uv=False)
    p = s ** 2
    p = p[p > 1e-300]
    return float(-np.sum(p * np.log(p)))


def _phys_order(st):
    """Dense basis order of to_dense (electronic first, then chain sites in node order) and
    each physical node's position in it."""
    tr = st.tree
    owners = [v for v in range(tr.n) if tr.phys[v] > 0]
    owners.sort()
    return owners, [tr.phys[v] for v in owners]


def test_entropies_equal_the_dense_state_at_full_bond_dimension():
    for p in (W.sf_small(seed=11, n_env=2, L=2, d=3, D=64, n_modes=4, dt=0.5),
              W.sf_small(seed=5, n_env=2, L=2, d=3, D=64, n_modes=4, dt=0.5, er_tree=True, D_er=64)):
        st = TTNS(p)
        for _ in range(4):
            st.step(p.dt)
        S = st.bond_entropies()
        psi = st.to_dense()
        owners, dims = _phys_order(st)
        pos = {v: i for i, v in enumerate(owners)}
        assert abs(S[0] - _dense_entropy(psi, dims, [pos[0]])) < 1e-10
        for v in range(1, st.tree.n):
            part = sorted(pos[x] for x in st.sub[v] if x in pos)
            assert abs(S[v] - _dense_entropy(psi, dims, part)) < 1e-9, (p.name, v)
        assert S.max() > 1e-3          # the state is entangled


def test_product_state_has_zero_entropy():
    st = TTNS(W.sf_small(seed=7))
    assert np.abs(st.bond_entropies()).max() < 1e-14
