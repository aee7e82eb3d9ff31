"""Dense state-vector reference for tiny problems (oracle; test infrastructure only).

Builds the star Hamiltonian of Eq. 2 directly from a Problem, as a dense matrix on
electronic (x) chain-site Fock spaces, without the tree, and propagates exactly
through its eigen-decomposition.  Basis order: electronic index first, then the
chain sites of environment 0 in site order, then environment 1, and so on.
"""
from __future__ import annotations

import numpy as np

from .chain import chain_of

HBAR = 0.6582119569  # eV fs


def _kron_all(mats):
    out = np.array([[1.0 + 0.0j]])
    for m in mats:
        out = np.kron(out, m)
    return out


def dense_hamiltonian(problem):
    n_el = problem.n_el
    H_S = np.array(problem.H_S, dtype=complex)
    H_S = H_S - (np.trace(H_S).real / n_el) * np.eye(n_el)
    dims = [n_el]
    sites = []
    for i, env in enumerate(problem.envs):
        for n in range(env.L):
            dims.append(env.d)
            sites.append((i, n))
    eye = [np.eye(d, dtype=complex) for d in dims]

    def embed(ops):
        mats = list(eye)
        for pos, op in ops:
            mats[pos] = op
        return _kron_all(mats)

    H = embed([(0, H_S)])
    pos = 1
    for i, env in enumerate(problem.envs):
        rc, om, hop = chain_of(env.spectral, env.L)
        d = env.d
        a = np.diag(np.sqrt(np.arange(1, d, dtype=float)), 1).astype(complex)
        ad = a.conj().T
        num = ad @ a
        H = H + embed([(0, np.array(env.W_bar, dtype=complex) * rc / np.sqrt(2.0)), (pos, a + ad)])
        for n in range(env.L):
            H = H + om[n] * embed([(pos + n, num)])
        for n in range(env.L - 1):
            H = H + hop[n] * (embed([(pos + n, ad), (pos + n + 1, a)]) +
                              embed([(pos + n, a), (pos + n + 1, ad)]))
        pos += env.L
    return H, dims


def initial_vector(problem, dims):
    psi_el = np.zeros(problem.n_el, dtype=complex)
    if problem.psi_el is not None:
        psi_el[:] = problem.psi_el
    else:
        psi_el[problem.init_state] = 1.0
    rest = int(np.prod(dims[1:]))
    vac = np.zeros(rest, dtype=complex)
    vac[0] = 1.0
    return np.kron(psi_el, vac)


class Exact:
    """Exact propagation psi(t) = exp(-i H t / hbar) psi(0)."""

    def __init__(self, problem):
        self.problem = problem
        self.H, self.dims = dense_hamiltonian(problem)
        self.w, self.S = np.linalg.eigh(self.H)
        self.psi0 = initial_vector(problem, self.dims)
        self.c0 = self.S.conj().T @ self.psi0

    def state(self, t: float) -> np.ndarray:
        return self.S @ (np.exp(-1j * self.w * t / HBAR) * self.c0)

    def rho_el(self, psi: np.ndarray) -> np.ndarray:
        n_el = self.dims[0]
        M = psi.reshape(n_el, -1)
        return M @ M.conj().T

    def occupations(self, psi: np.ndarray) -> np.ndarray:
        dims = self.dims
        T = psi.reshape(dims)
        out = []
        for k in range(1, len(dims)):
            p = np.sum(np.abs(np.moveaxis(T, k, 0).reshape(dims[k], -1)) ** 2, axis=1)
            out.append(float(np.sum(np.arange(dims[k]) * p)))
        return np.array(out)

    def energy(self, psi: np.ndarray) -> float:
        return float(np.real(np.vdot(psi, self.H @ psi)))


def dense_kinetic(problem):
    """The chains' nuclear kinetic energy as a dense matrix, built term by term:
    T = -(1/4) sum_m w_m (a^+ - a)_m^2 - (1/2) sum_m t_m (a^+ - a)_m (a^+ - a)_{m+1}
    per chain (w_m onsite energies, t_m hoppings of the chain map)."""
    n_el = problem.n_el
    dims = [n_el]
    for env in problem.envs:
        dims += [env.d] * env.L
    eye = [np.eye(d, dtype=complex) for d in dims]

    def embed(ops):
        mats = list(eye)
        for pos, op in ops:
            mats[pos] = op
        return _kron_all(mats)

    T = np.zeros((int(np.prod(dims)),) * 2, dtype=complex)
    pos = 1
    for env in problem.envs:
        _, om, hop = chain_of(env.spectral, env.L)
        d = env.d
        a = np.diag(np.sqrt(np.arange(1, d, dtype=float)), 1).astype(complex)
        P = a.conj().T - a
        for n in range(env.L):
            T = T - 0.25 * om[n] * embed([(pos + n, P @ P)])
        for n in range(env.L - 1):
            T = T - 0.5 * hop[n] * embed([(pos + n, P), (pos + n + 1, P)])
        pos += env.L
    return T


def energy_surfaces(problem, H, T, psi, sigma_tol: float = 1e-7):
    """Eq. 3-4 from a dense state: the Schmidt decomposition of psi for electronic | rest,
    then <phi_i, j| H |phi_k, l> and the same with H - T, in the basis ordered bath-major.
    Returns the ascending eigenvalues of H_eff and V_eff and the Schmidt values."""
    n_el = problem.n_el
    M = psi.reshape(n_el, -1)                       # electronic x rest
    Uu, sv, Vh = np.linalg.svd(M, full_matrices=False)
    keep = [k for k in range(len(sv)) if sv[k] > sigma_tol]
    vecs = []
    for k in keep:
        phi = Vh[k]                                 # rest-space Schmidt vector
        for l in range(n_el):
            e = np.zeros(n_el, dtype=complex)
            e[l] = 1.0
            vecs.append(np.kron(e, phi))
    B = np.array(vecs).T
    Heff = B.conj().T @ H @ B
    Veff = B.conj().T @ (H - T) @ B
    return np.linalg.eigvalsh(Heff), np.linalg.eigvalsh(Veff), sv[keep]
