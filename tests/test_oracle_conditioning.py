"""The oracle's own conditioning on the workloads whose GPU parity is checked over long
horizons: the stored trajectories at Krylov tolerance 1e-12 and 1e-14 (both written by
tests/golden/make_golden.py from oracle/) must agree to 1e-9 at every step, so that a
1e-6 / 1e-7 parity bound means something at every step.  Reads stored files only."""
import json
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("name", ["sf_er_5state_8x12_d20_D40"] + [f"batched_spin_boson_{s}" for s in range(1000, 1004)])
def test_krylov_tolerance_envelope_is_tiny(name):
    paths = [os.path.join(GOLD, name + ".json"), os.path.join(GOLD, name + "_tol14.json")]
    if not all(os.path.exists(p) for p in paths):
        pytest.skip("golden trajectories not generated")
    a, b = [np.array(json.load(open(p))["populations"]) for p in paths]
    assert np.abs(a - b).max() < 1e-9
    # populations of a normalised state
    assert np.abs(a.sum(axis=1) - 1).max() < 1e-10
