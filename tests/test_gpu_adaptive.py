"""GPU parity of the adaptive bond dimension (ttns_grow_bonds / ttns_adapt_bonds) with the
oracle's, through the C ABI: the same growth schedule on both sides, every population
afterwards at the stated tolerance; growth keeps the state; growth to the full bond
dimension at t = 0 equals the dense state vector of Eq. 2 (a closed form independent of both).
"""
import numpy as np
import pytest

from paper_1710_01362_gb300 import build, ttns
from paper_1710_01362_gb300 import workloads as W
from oracle.statevector import Exact
from oracle.ttns import TTNS

pytestmark = pytest.mark.gpu

TOL = {ttns.TTNS_FP64: 1e-7, ttns.TTNS_MIXED: 1e-6}
PRECS = [ttns.TTNS_FP64, ttns.TTNS_MIXED]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def small(D, L=3):
    return W.sf_small(seed=11, n_env=2, L=L, d=3, D=D, n_modes=4, dt=0.5)


@pytest.mark.parametrize("prec", PRECS)
def test_growth_schedule_matches_oracle(prec):
    """D = 2 for 6 steps, every bond grown to 5, 8 more steps, then to 8 and 6 more steps:
    every population of every step against the oracle doing the same."""
    p = small(2)
    st = TTNS(p)
    g = ttns.Tree(p, precision=prec)
    ref, got = [], []
    for n_steps, target in ((6, 5), (8, 8), (6, None)):
        for _ in range(n_steps):
            st.step(p.dt)
            g.step(p.dt, 1)
            ref.append(st.populations())
            got.append(g.populations())
        if target is not None:
            before = g.populations()
            grown_o = st.grow_bonds([0] + [target] * (st.tree.n - 1))
            n = g.grow_bonds([0] + [target] * (st.tree.n - 1))
            assert n == len(grown_o) > 0
            assert g.bonds() == st.tree.bond
            # growth keeps the state
            assert np.abs(g.populations() - before).max() < 1e-12
    err = np.abs(np.array(got) - np.array(ref)).max()
    print(f"max population error {err:.3e}")
    assert err < TOL[prec]
    g.close()


def test_growth_to_full_dimension_at_t0_is_exact():
    p = small(1, L=2)
    ex = Exact(p)
    g = ttns.Tree(p, precision=ttns.TTNS_FP64)
    g.grow_bonds([0] + [1 << 20] * (g.n_nodes() - 1))
    assert g.bonds() == TTNS(small(1 << 20, L=2)).tree.bond
    g.step(p.dt, 16)
    psi = ex.state(16 * p.dt)
    np.testing.assert_allclose(g.rho(), ex.rho_el(psi), atol=1e-8)
    g.close()


def test_adaptive_rule_matches_oracle():
    p = small(2)
    st = TTNS(p)
    g = ttns.Tree(p, precision=ttns.TTNS_FP64)
    for _ in range(10):
        st.step(p.dt)
    g.step(p.dt, 10)
    # eps in the widest gap between the bonds' smallest Schmidt weights (a decision that
    # rounding cannot flip)
    lows = np.sort([w[0] for w in st.bond_spectra().values()])
    k = int(np.argmax(np.diff(np.log(np.maximum(lows, 1e-300)))))
    eps = float(np.sqrt(max(lows[k], 1e-300) * lows[k + 1]))
    grown_o = st.adapt_bonds(eps, 2, 6)
    assert g.adapt_bonds(eps, 2, 6) == len(grown_o) > 0
    assert g.bonds() == st.tree.bond
    for _ in range(6):
        st.step(p.dt)
        g.step(p.dt, 1)
        assert np.abs(g.populations() - st.populations()).max() < TOL[ttns.TTNS_FP64]
    g.close()


def test_checkpoint_of_a_grown_tree(tmp_path):
    p = small(2)
    g = ttns.Tree(p, precision=ttns.TTNS_FP64)
    g.step(p.dt, 4)
    g.grow_bonds([0] + [5] * (g.n_nodes() - 1))
    g.step(p.dt, 2)
    path = str(tmp_path / "grown.ckpt")
    g.save(path)
    h = ttns.Tree.load(path, p, precision=ttns.TTNS_FP64)
    assert h.bonds() == g.bonds()
    g.step(p.dt, 3)
    h.step(p.dt, 3)
    assert np.array_equal(g.rho(), h.rho())
    g.close()
    h.close()


def test_growth_rejects_batches_and_bad_sizes():
    ps = [small(2), small(2)]
    g = ttns.Tree(ps, precision=ttns.TTNS_FP64)
    with pytest.raises(ttns.TTNSError):
        g.grow_bonds([0] + [4] * (g.n_nodes() - 1))
    g.close()
    g = ttns.Tree(small(2), precision=ttns.TTNS_FP64)
    with pytest.raises(ttns.TTNSError):
        lib = ttns.lib()
        import ctypes as C
        req = (C.c_int * 3)(0, 4, 4)
        ttns._check(lib.ttns_grow_bonds(g.h, req, 3, None))
    with pytest.raises(ttns.TTNSError):
        g.adapt_bonds(-1.0, 2, 6)
    g.close()


def test_er_tree_growth_to_full_dimension_at_t0_is_exact():
    # ER tensors have three bond legs and no physical leg
    p = W.sf_small(seed=5, n_env=2, L=2, d=3, D=1, n_modes=4, dt=0.5, er_tree=True, D_er=1)
    ex = Exact(p)
    g = ttns.Tree(p, precision=ttns.TTNS_FP64)
    g.grow_bonds([0] + [1 << 20] * (g.n_nodes() - 1))
    full = TTNS(W.sf_small(seed=5, n_env=2, L=2, d=3, D=64, n_modes=4, dt=0.5, er_tree=True, D_er=64))
    assert g.bonds() == full.tree.bond
    g.step(p.dt, 10)
    np.testing.assert_allclose(g.rho(), ex.rho_el(ex.state(10 * p.dt)), atol=1e-8)
    g.close()
