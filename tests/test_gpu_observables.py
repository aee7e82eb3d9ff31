"""Energy surfaces (Eq. 3-4) and entanglement entropies on the GPU against the FP64 oracle
(and a closed form), through the C ABI.

The surfaces are eigenvalues of 25 x 25 Hermitian matrices built from the state, so they
inherit its difference from the oracle (1e-7 of the populations' scale in FP64 at these
lengths, ~1e-6 in split precision) times the operator's scale (~1 eV): bounds 1e-6 eV (FP64)
and 2e-5 eV (mixed).  Entropies: 1e-6 (FP64) and 2e-5 (mixed)."""
import numpy as np
import pytest

from paper_1710_01362_gb300 import build, ttns
from paper_1710_01362_gb300 import workloads as W
from oracle.chain import chain_of
from oracle.ttns import TTNS

pytestmark = pytest.mark.gpu
TOL = {ttns.TTNS_FP64: 1e-6, ttns.TTNS_MIXED: 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


CASES = {
    "star": lambda: W.sf_small(seed=7, n_env=3, L=4, d=4, D=6, n_modes=12, n_steps=10),
    "er": lambda: W.sf_small(seed=9, n_env=4, L=3, d=3, D=5, n_modes=6, n_steps=10, er_tree=True, D_er=7),
}


@pytest.mark.parametrize("prec", [ttns.TTNS_FP64, ttns.TTNS_MIXED])
@pytest.mark.parametrize("name", list(CASES))
def test_energy_surfaces_and_entropies_match_the_oracle(name, prec):
    p = CASES[name]()
    g = ttns.Tree(p, precision=prec)
    o = TTNS(p)
    for step in range(1, 7):
        g.step(p.dt, 1)
        o.step(p.dt)
        if step % 3:
            continue
        tes, pes, sig = g.energy_surfaces()
        e_h, e_v, osig, _, _ = o.energy_surfaces()
        assert len(tes) == len(e_h), (len(sig), len(osig))
        np.testing.assert_allclose(sig, osig, atol=TOL[prec])
        np.testing.assert_allclose(tes, e_h, atol=TOL[prec])
        np.testing.assert_allclose(pes, e_v, atol=TOL[prec])
        np.testing.assert_allclose(g.bond_entropies(), o.bond_entropies(), atol=TOL[prec])
    g.close()


def test_zero_coupling_surfaces_are_the_system_spectrum():
    p = W.rabi(eps=0.1, V=0.05, L=3, d=3, D=3)
    g = ttns.Tree(p, precision=ttns.TTNS_FP64)
    g.step(p.dt, 5)
    tes, pes, sig = g.energy_surfaces()
    lam = np.linalg.eigvalsh(np.array(p.H_S) - np.trace(p.H_S).real / 2 * np.eye(2))
    _, om, _ = chain_of(p.envs[0].spectral, p.envs[0].L)
    assert len(sig) == 1 and abs(sig[0] - 1) < 1e-12
    np.testing.assert_allclose(tes, lam, atol=1e-12)
    np.testing.assert_allclose(pes, lam - 0.25 * om.sum(), atol=1e-12)
    assert np.abs(g.bond_entropies()).max() < 1e-12          # a product state
    g.close()


def test_energy_surfaces_in_batched_mode_and_on_the_large_root():
    # every tree of a batch has its own surfaces; the 4 x 20 star root (800 000 elements) goes
    # through the same projections (only the mixed path's consistency with the FP64 path is
    # checked there: both from the same initial state, a few steps)
    ps = [W.sf_small(seed=s, n_env=2, L=3, d=3, D=4, n_modes=6, n_steps=4) for s in (31, 32, 33)]
    g = ttns.Tree(ps, precision=ttns.TTNS_FP64)
    g.step(0.5, 4)
    for k, p in enumerate(ps):
        o = TTNS(p)
        for _ in range(4):
            o.step(p.dt)
        tes, pes, _ = g.energy_surfaces(k)
        e_h, e_v, _, _, _ = o.energy_surfaces()
        np.testing.assert_allclose(tes, e_h, atol=1e-6)
        np.testing.assert_allclose(pes, e_v, atol=1e-6)
    g.close()
    p = W.sf_5state_4x20()
    a = ttns.Tree(p, precision=ttns.TTNS_FP64)
    b = ttns.Tree(p, precision=ttns.TTNS_MIXED)
    a.step(p.dt, 3)
    b.step(p.dt, 3)
    ta, pa, sa = a.energy_surfaces()
    tb, pb, sb = b.energy_surfaces()
    assert len(ta) == len(tb) and np.abs(ta - tb).max() < 1e-4 and np.abs(pa - pb).max() < 1e-4
    a.close()
    b.close()
