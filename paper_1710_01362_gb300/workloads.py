"""Seeded synthetic workloads for the TTNS sweep.

This module only draws numbers: electronic Hamiltonians, coupling patterns and
bath spectral densities with the shapes of the paper's singlet-fission model
(five diabatic states, several bosonic environments; Eq. 1-2).  It holds none of
the method's arithmetic: the chain mapping, the tree, the bond-dimension clamp,
the energy shift and the sweep are done by the code that consumes a
``Problem`` (the CUDA library, or the test oracle), each on its own.

Units: energies in eV, times in fs.  Mode frequencies are drawn in cm^-1 and
converted with 1 cm^-1 = 1.239841984e-4 eV.

A discrete mode k with frequency w_k and Huang-Rhys factor S_k has the coupling
strength lambda_k = w_k * sqrt(2 S_k) in the convention of Eq. 1, where the
coupling operator is lambda_k * Wbar * (b + b^dagger) / sqrt(2).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

CM1_TO_EV = 1.239841984e-4


@dataclass
class Environment:
    """One bosonic environment i of Eq. 2: pattern Wbar_i and its spectral density.

    ``spectral`` is either ("ohmic", alpha, omega_c) for J(w) = 2 pi alpha w exp(-w/omega_c)
    or ("modes", omega[K], lam[K]) for a discrete set of modes.
    """

    W_bar: np.ndarray                 # (n_el, n_el) complex Hermitian
    spectral: Tuple
    L: int                            # chain length (sites)
    d: int                            # local Fock dimension per chain site
    D: int                            # requested bond dimension along this chain
    obb: int = 0                      # optimised boson basis dimension per site (0: none)


@dataclass
class Problem:
    name: str
    H_S: np.ndarray                   # (n_el, n_el) complex Hermitian, eV
    envs: List[Environment]
    dt: float                         # fs
    n_steps: int
    er_tree: bool = False             # balanced binary entanglement-renormalisation tree
    D_er: int = 0                     # bond dimension between ER nodes (er_tree only)
    init_state: int = 0               # initially occupied electronic state
    psi_el: Optional[np.ndarray] = None  # optional initial electronic amplitudes (n_el complex)
    seed: Optional[int] = None
    notes: str = ""
    qr_cutoff: Optional[float] = None   # QR null/truncation cutoff (relative); None: 1e-8

    @property
    def n_el(self) -> int:
        return self.H_S.shape[0]


def _herm(a: np.ndarray) -> np.ndarray:
    return 0.5 * (a + a.conj().T)


# ---------------------------------------------------------------------------
# Two-state spin-boson problems (Ohmic bath)
# ---------------------------------------------------------------------------

def spin_boson(eps: float = 0.1, V: float = 0.05, alpha: float = 0.1, omega_c: float = 0.2,
               L: int = 4, d: int = 4, D: int = 4, dt: float = 0.5, n_steps: int = 200,
               name: str = "spin_boson_ohmic") -> Problem:
    """Two electronic states at +eps/-eps with coupling V, one Ohmic chain.

    The coupling pattern is sigma_z / 2 (the spin-boson convention of the Ohmic
    spectral density J(w) = 2 pi alpha w exp(-w / omega_c)).
    """
    H_S = np.array([[eps, V], [V, -eps]], dtype=complex)
    W = np.diag([0.5, -0.5]).astype(complex)
    env = Environment(W_bar=W, spectral=("ohmic", alpha, omega_c), L=L, d=d, D=D)
    return Problem(name=name, H_S=H_S, envs=[env], dt=dt, n_steps=n_steps)


def ohmic_2state_L4(full_bond: bool = False) -> Problem:
    """2 states (+-0.1 eV, coupling 0.05 eV), Ohmic chain alpha 0.1 / cutoff 0.2 eV,
    4 sites, local dim 4, bond dim 4 (or the full Hilbert-space bond dims)."""
    p = spin_boson(D=(1 << 20) if full_bond else 4,
                   name="ohmic_2state_L4_" + ("fullD" if full_bond else "D4"))
    return p


def batched_spin_boson(seed: int, L: Optional[int] = None, D: Optional[int] = None,
                       d: int = 4, dt: float = 0.5, n_steps: int = 400) -> Problem:
    """One parameter set of the batched workload: Delta in U[0.1,0.3] eV,
    V in U[0.02,0.08] eV, alpha in U[0.05,0.3], omega_c in U[0.1,0.3] eV,
    chain length in 10..40, bond dim in 12..24, local dim 4."""
    rng = np.random.default_rng(seed)
    delta = rng.uniform(0.1, 0.3)
    V = rng.uniform(0.02, 0.08)
    alpha = rng.uniform(0.05, 0.3)
    omega_c = rng.uniform(0.1, 0.3)
    Ls = int(rng.integers(10, 41)) if L is None else L
    Ds = int(rng.integers(12, 25)) if D is None else D
    p = spin_boson(eps=delta / 2, V=V, alpha=alpha, omega_c=omega_c, L=Ls, d=d, D=Ds,
                   dt=dt, n_steps=n_steps, name=f"batched_spin_boson_{seed}")
    p.seed = seed
    p.qr_cutoff = 1e-3
    return p


# ---------------------------------------------------------------------------
# Singlet-fission-shaped problems (5 states, several environments)
# ---------------------------------------------------------------------------

def _sf_system(rng: np.random.Generator, n_el: int) -> np.ndarray:
    """Energies U[1.5, 2.5] eV; every off-diagonal pair coupled with |V| in
    U[0.02, 0.10] eV and a random sign.  State order LE+, LE-, CT+, CT-, TT."""
    H = np.zeros((n_el, n_el), dtype=complex)
    H[np.diag_indices(n_el)] = rng.uniform(1.5, 2.5, size=n_el)
    for i in range(n_el):
        for j in range(i + 1, n_el):
            v = rng.uniform(0.02, 0.10) * (1.0 if rng.random() < 0.5 else -1.0)
            H[i, j] = H[j, i] = v
    return H


def _pattern(rng: np.random.Generator, n_el: int, diagonal: bool) -> np.ndarray:
    """A coupling pattern at spectral norm 1: a diagonal tuning pattern, or a real
    symmetric off-diagonal pattern on a random mask of 2-4 state pairs."""
    W = np.zeros((n_el, n_el))
    if diagonal:
        W[np.diag_indices(n_el)] = rng.normal(size=n_el)
    else:
        pairs = [(i, j) for i in range(n_el) for j in range(i + 1, n_el)]
        k = int(rng.integers(2, 5))
        sel = rng.choice(len(pairs), size=k, replace=False)
        for s in sel:
            i, j = pairs[s]
            W[i, j] = W[j, i] = rng.normal()
    W /= np.abs(np.linalg.eigvalsh(W)).max()
    return W.astype(complex)


def _modes(rng: np.random.Generator, K: int) -> Tuple[np.ndarray, np.ndarray]:
    """K modes: frequency U[50, 1700] cm^-1, Huang-Rhys factor log-uniform in
    [1e-3, 0.5]; lambda_k = w_k sqrt(2 S_k)."""
    w = rng.uniform(50.0, 1700.0, size=K) * CM1_TO_EV
    S = np.exp(rng.uniform(np.log(1e-3), np.log(0.5), size=K))
    lam = w * np.sqrt(2.0 * S)
    order = np.argsort(w)
    return w[order], lam[order]


def singlet_fission(seed: int, n_env: int, L: int, d: int, D: int, n_modes: int,
                    dt: float, n_steps: int, er_tree: bool = False, D_er: int = 0,
                    n_el: int = 5, name: str = "singlet_fission") -> Problem:
    rng = np.random.default_rng(seed)
    H_S = _sf_system(rng, n_el)
    envs = []
    for i in range(n_env):
        W = _pattern(rng, n_el, diagonal=(i < (n_env + 1) // 2))
        w, lam = _modes(rng, n_modes)
        envs.append(Environment(W_bar=W, spectral=("modes", w, lam), L=L, d=d, D=D))
    return Problem(name=name, H_S=H_S, envs=envs, dt=dt, n_steps=n_steps, er_tree=er_tree,
                   D_er=D_er, seed=seed)


def sf_5state_4x20() -> Problem:
    """5 states, root with 4 chains of 20 sites (40 modes each), local dim 10, bond dim 20,
    dt 0.5 fs, 400 steps (the headline single-tree workload)."""
    return singlet_fission(seed=2, n_env=4, L=20, d=10, D=20, n_modes=40, dt=0.5, n_steps=400,
                           name="sf_5state_4x20_d10_D20")


def sf_er_5state_8x60(L: int = 60, n_steps: int = 800) -> Problem:
    """5 states, balanced binary ER tree over 8 chains of 60 sites (120 modes each),
    local dim 20, bond dim 40, dt 0.25 fs."""
    p = singlet_fission(seed=3, n_env=8, L=L, d=20, D=40, n_modes=120, dt=0.25,
                        n_steps=n_steps, er_tree=True, D_er=40,
                        name=f"sf_er_5state_8x{L}_d20_D40")
    p.qr_cutoff = 1e-3
    return p


def sf_small(seed: int = 7, n_env: int = 3, L: int = 5, d: int = 4, D: int = 6,
             n_modes: int = 12, dt: float = 0.5, n_steps: int = 10, er_tree: bool = False,
             D_er: int = 8) -> Problem:
    """A small singlet-fission-shaped tree for quick parity checks."""
    return singlet_fission(seed=seed, n_env=n_env, L=L, d=d, D=D, n_modes=n_modes, dt=dt,
                           n_steps=n_steps, er_tree=er_tree, D_er=D_er,
                           name=f"sf_small_s{seed}_{n_env}x{L}_d{d}_D{D}" + ("_er" if er_tree else ""))


def pure_dephasing(kappa=(0.5, -0.5), eps=(0.05, -0.05), omega=None, lam=None, L: int = 4,
                   d: int = 8, D: int = 1 << 20, dt: float = 0.5, n_steps: int = 40) -> Problem:
    """Two uncoupled states with diagonal coupling pattern diag(kappa) to one chain
    built from a few discrete modes: the independent-boson model.  The initial
    state is the equal superposition (|0> + |1>)/sqrt(2) on the electronic node."""
    if omega is None:
        omega = np.array([0.10, 0.17, 0.23, 0.31])
    if lam is None:
        lam = np.array([0.02, 0.015, 0.01, 0.012])
    H_S = np.diag(np.asarray(eps, dtype=float)).astype(complex)
    W = np.diag(np.asarray(kappa, dtype=float)).astype(complex)
    env = Environment(W_bar=W, spectral=("modes", np.asarray(omega), np.asarray(lam)), L=L, d=d, D=D)
    return Problem(name="pure_dephasing", H_S=H_S, envs=[env], dt=dt, n_steps=n_steps,
                   psi_el=np.array([1.0, 1.0], dtype=complex) / np.sqrt(2.0))


def rabi(eps: float = 0.1, V: float = 0.05, L: int = 3, d: int = 3, D: int = 3,
         dt: float = 0.5, n_steps: int = 60) -> Problem:
    """Zero system-bath coupling: the electronic node oscillates as a two-level system."""
    p = spin_boson(eps=eps, V=V, alpha=0.0, omega_c=0.2, L=L, d=d, D=D, dt=dt,
                   n_steps=n_steps, name="rabi_zero_coupling")
    return p


def all_named():
    return {
        "ohmic_2state_L4_D4": lambda: ohmic_2state_L4(False),
        "ohmic_2state_L4_fullD": lambda: ohmic_2state_L4(True),
        "sf_5state_4x20_d10_D20": sf_5state_4x20,
        "sf_er_5state_8x60_d20_D40": sf_er_5state_8x60,
    }


# ---------------------------------------------------------------------------
# Surrogate workload: the singlet-fission ER tree at reduced fidelity, parameterised by 30
# numbers (the surrogate network's inputs)
# ---------------------------------------------------------------------------

SURROGATE_N_PARAMS = 30
_SURROGATE_PATTERN_SEED = 777


def surrogate_params(seed: int) -> np.ndarray:
    """The 30 inputs: energies of LE+, LE-, CT+, CT- relative to TT (U[-0.2, 0.2] eV); the 10
    electronic couplings (|V| in U[0.02, 0.10] eV, random sign, pairs in row order); per-chain
    reorganisation energies (U[0.005, 0.08] eV, 8 chains); per-chain mean mode frequencies
    (U[400, 1500] cm^-1, in eV)."""
    rng = np.random.default_rng(seed)
    e = rng.uniform(-0.2, 0.2, size=4)
    v = rng.uniform(0.02, 0.10, size=10) * np.where(rng.random(10) < 0.5, -1.0, 1.0)
    lam = rng.uniform(0.005, 0.08, size=8)
    wbar = rng.uniform(400.0, 1500.0, size=8) * CM1_TO_EV
    return np.concatenate([e, v, lam, wbar])


def surrogate_problem(x: np.ndarray, L: int = 8, d: int = 6, D: int = 8, dt: float = 1.0, n_steps: int = 200,
                      n_modes: int = 12, name: str = "surrogate") -> Problem:
    """The ER tree (5 states, 7 ER nodes, 8 chains of L sites) for one parameter vector.  The
    coupling pattern of each chain is fixed (drawn once); chain i has n_modes modes at
    wbar_i (0.5 + k / (n_modes - 1)), k = 0 .. n_modes - 1, with equal Huang-Rhys factors
    whose reorganisation energy sum_k S_k w_k is lam_i."""
    x = np.asarray(x, dtype=float)
    n_el = 5
    H_S = np.zeros((n_el, n_el), dtype=complex)
    H_S[np.arange(4), np.arange(4)] = x[:4]
    k = 4
    for i in range(n_el):
        for j in range(i + 1, n_el):
            H_S[i, j] = H_S[j, i] = x[k]
            k += 1
    lam, wbar = x[14:22], x[22:30]
    prng = np.random.default_rng(_SURROGATE_PATTERN_SEED)
    envs = []
    for i in range(8):
        W = _pattern(prng, n_el, diagonal=(i < 4))
        w = wbar[i] * (0.5 + np.arange(n_modes) / (n_modes - 1))
        S = np.full(n_modes, lam[i] / w.sum())
        envs.append(Environment(W_bar=W, spectral=("modes", w, w * np.sqrt(2.0 * S)), L=L, d=d, D=D))
    return Problem(name=name, H_S=H_S, envs=envs, dt=dt, n_steps=n_steps, er_tree=True, D_er=D)
