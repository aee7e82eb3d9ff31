"""Host-side checks of the C-ABI library (no GPU): it loads, exports every symbol
include/ttns.h declares, and its host logic (argument validation, chain maps,
tree construction with the bond clamp, table checks) agrees with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1710_01362_gb300 import build, ttns
from paper_1710_01362_gb300 import workloads as W
from oracle.chain import chain_from_modes as o_chain_modes
from oracle.chain import chain_ohmic as o_chain_ohmic
from oracle.model import build_tree as o_build_tree

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ttns.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ttns_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert "ttns_build_tree" in names and "ttns_step" in names and len(names) >= 18
    L = ctypes.CDLL(ttns.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(ttns.EXPORTS)


def test_chain_maps_match_oracle():
    rc, on, hop = ttns.chain_ohmic(0.1, 0.2, 12)
    orc, oon, ohop = o_chain_ohmic(0.1, 0.2, 12)
    assert rc == pytest.approx(orc, rel=1e-15)
    np.testing.assert_allclose(on, oon, rtol=1e-15)
    np.testing.assert_allclose(hop, ohop, rtol=1e-15)
    p = W.sf_5state_4x20()
    for env in p.envs:
        a = ttns.chain_from_modes(env.spectral[1], env.spectral[2], env.L)
        b = o_chain_modes(env.spectral[1], env.spectral[2], env.L)
        assert abs(a[0] - b[0]) < 1e-14
        np.testing.assert_allclose(a[1], b[1], atol=1e-13)
        np.testing.assert_allclose(a[2], b[2], atol=1e-13)


@pytest.mark.parametrize("factory", [
    lambda: W.ohmic_2state_L4(False),
    lambda: W.ohmic_2state_L4(True),
    lambda: W.sf_small(seed=7),
    lambda: W.sf_small(seed=9, n_env=4, L=3, d=3, D=5, n_modes=6, er_tree=True, D_er=7),
    W.sf_5state_4x20,
    lambda: W.sf_er_5state_8x60(L=12, n_steps=40),
])
def test_plan_builds_the_oracle_tree(factory):
    p = factory()
    info = ttns.plan(p)
    t = o_build_tree(p)
    assert info["n_nodes"] == t.n
    assert info["bonds"] == t.bond
    sizes = [int(np.prod(t.legs(v))) for v in range(t.n)]
    assert info["max_node"] == max(sizes)
    # one step: each node is evolved twice, each edge twice
    assert info["exponentials_per_step"] == 2 * t.n + 2 * (t.n - 1)


def test_plan_of_the_headline_workload():
    info = ttns.plan(W.sf_5state_4x20())
    assert info["max_node"] == 5 * 20 ** 4          # the electronic root
    assert info["n_nodes"] == 81


def test_batched_plan():
    ps = [W.batched_spin_boson(s) for s in range(1000, 1010)]
    info = ttns.plan(ps)
    assert info["n_nodes"] == sum(1 + p.envs[0].L for p in ps)


def _problem_with(**kw):
    p = W.sf_small(seed=7)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_invalid_arguments_are_rejected_before_any_allocation():
    p = W.sf_small(seed=7)
    bad = p.H_S.copy()
    bad[0, 1] += 0.01
    with pytest.raises(ttns.TTNSError) as e:
        ttns.plan(_problem_with(H_S=bad))
    assert e.value.code == 1 and "Hermitian" in str(e.value)
    p2 = W.sf_small(seed=7)
    p2.envs[0].d = 1
    with pytest.raises(ttns.TTNSError) as e:
        ttns.plan(p2)
    assert e.value.code == 1
    p3 = W.sf_small(seed=7, n_env=3)
    p3.er_tree = True
    p3.D_er = 4
    with pytest.raises(ttns.TTNSError) as e:   # 3 environments: no balanced binary ER tree
        ttns.plan(p3)
    assert e.value.code == 1
    with pytest.raises(ttns.TTNSError):
        ttns.chain_from_modes([0.1, 0.2], [0.01, 0.02], 3)
    # the autotuner checks its arguments before it builds anything
    for cand, dt in (([0], 0.5), ([17], 0.5), ([8], 0.0), ([8], float("nan"))):
        with pytest.raises(ttns.TTNSError) as e:
            ttns.autotune(p, dt, candidates=cand, stream=0)
        assert e.value.code == 1


def test_flop_accounting_of_the_root_apply():
    # H_eff of the 5-state root: H_S on the physical leg, four H blocks on the bond legs and
    # four (Wbar, X) products: 8 flops per complex MAC
    p = W.sf_5state_4x20()
    info = ttns.plan(p)
    root = 5 * 20 ** 4
    per_apply_root = 8.0 * root * (5 + 4 * 20 + 4 * (20 + 5))
    assert info["apply_flops_per_step"] > 2 * per_apply_root
