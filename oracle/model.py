"""Star Hamiltonian, tree topology, bond-dimension clamp and initial state
(oracle; test infrastructure only).

Hamiltonian (Eq. 2):
    H = H_S + sum_i [ Wbar_i ||lambda_i|| (a_i0 + a_i0^+) / sqrt(2) + H_c,i ],
    H_c,i = sum_n omega_in n_in + sum_n t_in (a_in^+ a_i,n+1 + h.c.)
with bosons truncated to Fock states 0..d-1.  Readings:
  * H_S is shifted by -tr(H_S)/n_el (a global phase; populations unchanged).
  * Every term is an on-site operator or a product of two single-node operators;
    the coefficient of a two-node term sits on its first factor.

Tree (Results, "TTNS for vibronic quantum dynamics"; Methods, "Tensor Network States"):
  * star form: the electronic node is the root and the first site of every chain
    is one of its children (chain i, site n+1 is the child of site n);
  * ER form: the electronic node has one child, the top of a balanced binary tree
    of entanglement-renormalisation nodes (third-order tensors, no physical leg);
    each lowest ER node carries two chains;
  * optimised boson basis (Methods: Fock states compressed to a smaller basis per
    mode): every chain site gets a leaf that holds its Fock leg, joined to the site
    tensor by a bond of the OBB dimension; the site tensor keeps the chain bonds.
Each node's legs are ordered [parent bond] + [child bonds, in child order] +
[physical leg]; tensors are stored row-major in that order.

Bond dimensions: every bond e = (u, parent) asks for D_e and is then clamped to
the greatest values with D_e <= (product of the other leg dimensions) at both of
its end nodes (so every tensor can be an isometry toward any neighbour).

Initial state (zero temperature, no environmental excitation, the optically bright
state populated; Results, end of "TDVP for TTNS"): every non-root tensor is the
isometry that maps parent index k to the k-th combination of its other legs in
row-major order (k = 0 is the vacuum times the children's k = 0); the root holds
psi_el on its physical leg and index 0 on every bond.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np

from .chain import chain_of


def lowering(d: int) -> np.ndarray:
    a = np.zeros((d, d), dtype=complex)
    for s in range(1, d):
        a[s - 1, s] = np.sqrt(s)
    return a


@dataclass
class Coupling:
    va: int
    opa: np.ndarray
    vb: int
    opb: np.ndarray


@dataclass
class Tree:
    parent: List[int]
    children: List[List[int]]
    phys: List[int]                   # 0 = no physical leg
    kind: List[str]                   # "el", "er", "site", "obb" (the Fock leaf of a site)
    site_index: List[Optional[Tuple[int, int]]]   # (env, n) for chain sites
    bond: List[int]                   # bond dim to parent (root: 0)
    onsite: List[Optional[np.ndarray]]
    couplings: List[Coupling]
    n_el: int
    chain_nodes: List[List[int]]      # node ids holding chain i's Fock legs, site order
    psi_el: np.ndarray = None

    @property
    def n(self) -> int:
        return len(self.parent)

    def has_parent(self, v: int) -> bool:
        return self.parent[v] >= 0

    def legs(self, v: int) -> List[int]:
        """Leg dimensions of node v in storage order."""
        dims = []
        if self.parent[v] >= 0:
            dims.append(self.bond[v])
        for c in self.children[v]:
            dims.append(self.bond[c])
        if self.phys[v] > 0:
            dims.append(self.phys[v])
        return dims

    def leg_of(self, v: int, u: int) -> int:
        """Index of v's leg that points to its neighbour u."""
        if self.parent[v] == u:
            return 0
        off = 1 if self.parent[v] >= 0 else 0
        return off + self.children[v].index(u)

    def phys_leg(self, v: int) -> int:
        return len(self.legs(v)) - 1

    def neighbours(self, v: int) -> List[int]:
        nb = [self.parent[v]] if self.parent[v] >= 0 else []
        return nb + list(self.children[v])


def _clamp_bonds(tree: Tree, requested: List[int]) -> List[int]:
    n = tree.n
    D = list(requested)
    phys = [max(p, 1) for p in tree.phys]
    changed = True
    while changed:
        changed = False
        for u in range(n):
            if tree.parent[u] < 0:
                continue
            v = tree.parent[u]
            # at the child end u: its other legs are its children and its phys leg
            lim_u = phys[u]
            for c in tree.children[u]:
                lim_u *= D[c]
            # at the parent end v: its parent bond, its other children, its phys leg
            lim_v = phys[v]
            if tree.parent[v] >= 0:
                lim_v *= D[v]
            for c in tree.children[v]:
                if c != u:
                    lim_v *= D[c]
            new = min(D[u], lim_u, lim_v)
            if new != D[u]:
                D[u] = new
                changed = True
    return D


def build_tree(problem) -> Tree:
    """Builds the tree, the term list and the clamped bond dimensions of a Problem."""
    n_el = problem.n_el
    H_S = np.array(problem.H_S, dtype=complex)
    H_S = H_S - (np.trace(H_S).real / n_el) * np.eye(n_el)
    envs = problem.envs
    n_env = len(envs)

    parent: List[int] = []
    children: List[List[int]] = []
    phys: List[int] = []
    kind: List[str] = []
    site_index: List[Optional[Tuple[int, int]]] = []
    req: List[int] = []

    def add(p: int, ph: int, k: str, si, D: int) -> int:
        v = len(parent)
        parent.append(p)
        children.append([])
        phys.append(ph)
        kind.append(k)
        site_index.append(si)
        req.append(D)
        if p >= 0:
            children[p].append(v)
        return v

    root = add(-1, n_el, "el", None, 0)
    attach: List[int] = []            # parent node of chain i's first site
    if problem.er_tree:
        if n_env < 2 or (n_env & (n_env - 1)) != 0:
            raise ValueError("the ER tree needs a power-of-two number of environments >= 2")
        top = add(root, 0, "er", None, problem.D_er)
        level = [top]
        while 2 * len(level) < n_env:
            nxt = []
            for p in level:
                nxt.append(add(p, 0, "er", None, problem.D_er))
                nxt.append(add(p, 0, "er", None, problem.D_er))
            level = nxt
        for p in level:
            attach += [p, p]
    else:
        attach = [root] * n_env

    chain_nodes: List[List[int]] = []
    chains = []
    for i, env in enumerate(envs):
        rc, om, hop = chain_of(env.spectral, env.L)
        chains.append((rc, om, hop))
        nodes = []
        p = attach[i]
        obb = getattr(env, "obb", 0) or 0
        for nn in range(env.L):
            if obb > 0:
                # optimised boson basis: the site tensor keeps the chain bonds and a bond of
                # dimension obb to a leaf that holds the Fock leg (the site's operators act
                # on the leaf)
                v = add(p, 0, "site", (i, nn), env.D)
                leaf = add(v, env.d, "obb", (i, nn), obb)
                nodes.append(leaf)
            else:
                v = add(p, env.d, "site", (i, nn), env.D)
                nodes.append(v)
            p = v
        chain_nodes.append(nodes)

    tree = Tree(parent=parent, children=children, phys=phys, kind=kind, site_index=site_index,
                bond=[0] * len(parent), onsite=[None] * len(parent), couplings=[], n_el=n_el,
                chain_nodes=chain_nodes)
    tree.bond = _clamp_bonds(tree, req)
    tree.bond[root] = 0

    tree.onsite[root] = H_S
    for i, env in enumerate(envs):
        rc, om, hop = chains[i]
        d = env.d
        a = lowering(d)
        ad = a.conj().T
        num = np.diag(np.arange(d, dtype=float)).astype(complex)
        nodes = chain_nodes[i]
        for nn, v in enumerate(nodes):
            tree.onsite[v] = om[nn] * num
        W = np.array(env.W_bar, dtype=complex)
        tree.couplings.append(Coupling(root, W * (rc / np.sqrt(2.0)), nodes[0], a + ad))
        for nn in range(env.L - 1):
            tree.couplings.append(Coupling(nodes[nn], hop[nn] * ad, nodes[nn + 1], a))
            tree.couplings.append(Coupling(nodes[nn], hop[nn] * a, nodes[nn + 1], ad))

    psi = np.zeros(n_el, dtype=complex)
    if problem.psi_el is not None:
        psi[:] = np.asarray(problem.psi_el, dtype=complex)
    else:
        psi[problem.init_state] = 1.0
    tree.psi_el = psi
    return tree


def initial_tensors(tree: Tree) -> List[np.ndarray]:
    """Isometric product initial state (see the module docstring)."""
    A = []
    for v in range(tree.n):
        dims = tree.legs(v)
        if tree.parent[v] < 0:
            T = np.zeros(dims, dtype=complex)
            idx = tuple([0] * (len(dims) - 1))
            T[idx] = tree.psi_el  # the physical leg is the last one
            A.append(T)
        else:
            Dp = dims[0]
            rest = int(np.prod(dims[1:]))
            M = np.zeros((Dp, rest), dtype=complex)
            M[np.arange(Dp), np.arange(Dp)] = 1.0
            A.append(M.reshape(dims))
    return A
