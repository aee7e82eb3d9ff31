"""Writes the oracle's trajectories used as expected values by the GPU parity tests.

Every number written here comes from the FP64 CPU oracle (``oracle/``) run on
the seeded synthetic workloads of ``paper_1710_01362_gb300.workloads``; nothing
comes from the CUDA path.  Usage:

    python tests/golden/make_golden.py <name> [<name> ...]

Names: see CASES below.  Each case writes tests/golden/<name>.json with the
electronic populations after every step, the chain occupations every
``occ_every`` steps, and the run's Krylov statistics.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from paper_1710_01362_gb300 import workloads as W  # noqa: E402
from oracle.ttns import TTNS  # noqa: E402

CASES = {
    # name: (problem factory, steps, occupation stride)
    "ohmic_2state_L4_D4": (lambda: W.ohmic_2state_L4(False), 200, 10),
    "ohmic_2state_L4_fullD": (lambda: W.ohmic_2state_L4(True), 200, 10),
    "sf_5state_4x20_d10_D20": (W.sf_5state_4x20, 400, 20),
    "sf_er_5state_8x12_d20_D40": (lambda: W.sf_er_5state_8x60(L=12, n_steps=40), 40, 10),
    "sf_small_s7": (lambda: W.sf_small(seed=7, n_env=3, L=5, d=4, D=6, n_modes=12, n_steps=60), 60, 10),
    "sf_small_er_s9": (lambda: W.sf_small(seed=9, n_env=4, L=3, d=3, D=5, n_modes=6, n_steps=30,
                                          er_tree=True, D_er=7), 30, 10),
}
for s in range(1000, 1016):
    CASES[f"batched_spin_boson_{s}"] = ((lambda s=s: W.batched_spin_boson(s)), 60, 10)

# Sensitivity envelopes of the trajectories themselves, from the oracle alone:
#   *_tol14:  the same run with the Krylov tolerance 1e-14 instead of 1e-12 (differences at
#             the FP64 rounding level: what an FP64 implementation can be held to);
#   *_noise7: the same run with relative Gaussian noise of 1e-7 added to every H v and
#             environment application (seeded; the FP32 level of the mixed-precision
#             contractions).
# A well-conditioned trajectory keeps both small; where the trajectory amplifies them (a
# kept sub-column near the QR cutoff steers the one-site tangent space), two correct runs
# differ by the envelope, and parity is judged against it.
TIGHT = {f"batched_spin_boson_{s}_tol14": (f"batched_spin_boson_{s}", 1e-14) for s in range(1000, 1016)}
TIGHT["sf_er_5state_8x12_d20_D40_tol14"] = ("sf_er_5state_8x12_d20_D40", 1e-14)
TIGHT["sf_5state_4x20_d10_D20_tol14"] = ("sf_5state_4x20_d10_D20", 1e-14)
NOISY = {f"batched_spin_boson_{s}_noise7": (f"batched_spin_boson_{s}", 1e-7) for s in range(1000, 1016)}
NOISY["sf_er_5state_8x12_d20_D40_noise7"] = ("sf_er_5state_8x12_d20_D40", 1e-7)
NOISY["sf_5state_4x20_d10_D20_noise7"] = ("sf_5state_4x20_d10_D20", 1e-7)


def _noisy_apply(level: float, seed: int = 123):
    """TTNS.apply_terms with relative Gaussian noise of the given level on every result."""
    rng = np.random.default_rng(seed)
    plain = TTNS.apply_terms

    def noisy(A, terms):
        y = plain(A, terms)
        s = np.sqrt(np.mean(np.abs(y) ** 2)) if y.size else 0.0
        return y + level * s * (rng.standard_normal(y.shape) + 1j * rng.standard_normal(y.shape)) / np.sqrt(2)
    return plain, noisy


def run_case(name: str) -> None:
    tol = None
    noise = 0.0
    if name in TIGHT:
        base, tol = TIGHT[name]
        factory, n_steps, occ_every = CASES[base]
    elif name in NOISY:
        base, noise = NOISY[name]
        factory, n_steps, occ_every = CASES[base]
    else:
        factory, n_steps, occ_every = CASES[name]
    p = factory()
    st = TTNS(p) if tol is None else TTNS(p, tol=tol)
    plain = None
    if noise > 0.0:
        plain, noisy = _noisy_apply(noise)
        TTNS.apply_terms = staticmethod(noisy)
    pops = [st.populations().tolist()]
    occ = {0: st.occupations().tolist()}
    t0 = time.time()
    for k in range(n_steps):
        st.step(p.dt)
        pops.append(st.populations().tolist())
        if (k + 1) % occ_every == 0 or k + 1 == n_steps:
            occ[k + 1] = st.occupations().tolist()
    out = {
        "name": name,
        "problem": p.name,
        "dt": p.dt,
        "n_steps": n_steps,
        "bonds": st.tree.bond,
        "populations": pops,
        "occupations": {str(k): v for k, v in occ.items()},
        "norm": st.norm(),
        "energy": st.energy(),
        "stats": st.stats,
        "oracle_seconds": time.time() - t0,
    }
    if plain is not None:
        TTNS.apply_terms = staticmethod(plain)
        out["noise"] = noise
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print(name, "done in", round(time.time() - t0, 1), "s", flush=True)


if __name__ == "__main__":
    for name in sys.argv[1:]:
        run_case(name)
