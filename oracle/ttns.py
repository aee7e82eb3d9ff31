"""One-site TDVP for a tree tensor network state (oracle; test infrastructure only).

The paper propagates its TTNS with the time-dependent variational principle: the
tensors are updated one after another, each under a local effective Hamiltonian
H_eff(t) that is rebuilt at every step from the current state of the whole tree
(Results, section on TTNS for vibronic dynamics, last paragraph; Methods, section on
tensor network states).  The algorithm
itself sits in the paper's Supplement, which is not part of the paper text; the
reading used here is the one-site projector-splitting integrator on a tree:

  S(tau) = visit(root) with
    visit(v):  A_v <- exp(-i tau H_eff(v)) A_v
               for each child c, in order:
                   QR of A_v toward c (A_v <- Q, bond matrix C <- R); env(v -> c)
                   C <- exp(+i tau H_bond(v, c)) C;  A_c <- C A_c (on A_c's parent leg)
                   visit(c)
                   QR of A_c toward v; env(c -> v); A_v <- R A_v (no evolution)
  S*(tau) = the same operations in reverse order:
    visit*(v): for each child c, in reverse order:
                   QR of A_v toward c; env(v -> c); A_c <- R A_c (no evolution)
                   visit*(c)
                   QR of A_c toward v; env(c -> v)
                   C <- exp(+i tau H_bond(c, v)) C;  A_v <- C A_v
               A_v <- exp(-i tau H_eff(v)) A_v
  one step of length dt = S(dt/2) followed by S*(dt/2).

Environment blocks.  For a directed edge (u -> v), env(u -> v) describes the part
of the tree on u's side of the edge, projected on the bond basis given by u's
tensor when u is an isometry toward v:
  'H'  the sum of all terms that lie entirely on u's side,
  t    for every two-node term t with one end on each side, the projected
       factor of its end on u's side.
H_eff(v) is the sum of v's on-site term, every neighbour's 'H' block on the leg
toward it, and every two-node term whose two ends lie in different slots of v
(its physical leg, or the subtrees behind two different legs).
"""
from __future__ import annotations

from typing import Dict, List, Optional, Tuple

import numpy as np

from .linalg import expm_lanczos, householder_qr, KRYLOV_TOL, KRYLOV_MMAX
from .model import Coupling, Tree, _clamp_bonds, build_tree, initial_tensors, lowering

HBAR = 0.6582119569  # eV fs


def apply_factor(A: np.ndarray, leg: int, M: np.ndarray) -> np.ndarray:
    """y[..., i, ...] = sum_k M[i, k] A[..., k, ...] on the given leg."""
    return np.moveaxis(np.tensordot(M, A, axes=([1], [leg])), 0, leg)


class TTNS:
    def __init__(self, problem, tol: float = KRYLOV_TOL, mmax: int = KRYLOV_MMAX):
        self.problem = problem
        self.tree: Tree = build_tree(problem)
        self.A: List[np.ndarray] = initial_tensors(self.tree)
        self.tol = tol
        self.mmax = mmax
        self.qr_cutoff = getattr(problem, "qr_cutoff", None)
        self.stats: Dict[str, int] = {}
        self.t = 0.0
        t = self.tree
        n = t.n
        # subtree membership
        self.sub = [set() for _ in range(n)]
        for v in reversed(range(n)):
            self.sub[v].add(v)
            for c in t.children[v]:
                self.sub[v] |= self.sub[c]
        self.env: Dict[Tuple[int, int], Dict] = {}
        self._init_envs()

    # ------------------------------------------------------------------ tree helpers
    def piece(self, u: int, v: int) -> set:
        """Nodes on u's side of the edge (u, v)."""
        t = self.tree
        if t.parent[u] == v:
            return self.sub[u]
        return set(range(t.n)) - self.sub[v]

    def toward(self, v: int, x: int) -> int:
        """The neighbour of v on the path to node x (x != v)."""
        t = self.tree
        for c in t.children[v]:
            if x in self.sub[c]:
                return c
        return t.parent[v]

    def end_factor(self, u: int, e: int, op: np.ndarray, t_idx: int):
        """(leg, matrix) of a term's end e seen from node u."""
        tr = self.tree
        if e == u:
            return tr.phys_leg(u), op
        w = self.toward(u, e)
        return tr.leg_of(u, w), self.env[(w, u)][t_idx]

    def crossing(self, u: int, v: int) -> List[Tuple[int, int]]:
        """Terms crossing edge (u, v): list of (term index, end node on u's side)."""
        P = self.piece(u, v)
        out = []
        for ti, c in enumerate(self.tree.couplings):
            ina, inb = c.va in P, c.vb in P
            if ina != inb:
                out.append((ti, c.va if ina else c.vb))
        return out

    def node_terms(self, v: int, exclude: Optional[int] = None):
        """Terms of H restricted to the slots of v (all neighbours but `exclude`).

        Returns a list of terms, each a list of (leg, matrix) factors."""
        tr = self.tree
        terms = []
        if tr.onsite[v] is not None:
            terms.append([(tr.phys_leg(v), tr.onsite[v])])
        for w in tr.neighbours(v):
            if w == exclude:
                continue
            terms.append([(tr.leg_of(v, w), self.env[(w, v)]["H"])])
        P = self.piece(v, exclude) if exclude is not None else set(range(tr.n))
        for ti, c in enumerate(tr.couplings):
            if c.va not in P or c.vb not in P:
                continue
            sa = "p" if c.va == v else self.toward(v, c.va)
            sb = "p" if c.vb == v else self.toward(v, c.vb)
            if sa == sb:
                continue
            fa = self.end_factor(v, c.va, c.opa, ti)
            fb = self.end_factor(v, c.vb, c.opb, ti)
            terms.append([fa, fb])
        return terms

    @staticmethod
    def apply_terms(A: np.ndarray, terms) -> np.ndarray:
        y = np.zeros_like(A)
        for term in terms:
            x = A
            for leg, M in term:
                x = apply_factor(x, leg, M)
            y += x
        return y

    # ------------------------------------------------------------------ environments
    def update_env(self, u: int, v: int) -> None:
        """env(u -> v) from A_u, which must be an isometry toward v."""
        tr = self.tree
        Q = self.A[u]
        lv = tr.leg_of(u, v)
        others = [k for k in range(Q.ndim) if k != lv]
        Qc = Q.conj()

        def project(X):
            return np.tensordot(Qc, X, axes=(others, others))

        blocks = {"H": project(self.apply_terms(Q, self.node_terms(u, exclude=v)))}
        for ti, e in self.crossing(u, v):
            c = tr.couplings[ti]
            op = c.opa if e == c.va else c.opb
            leg, M = self.end_factor(u, e, op, ti)
            blocks[ti] = project(apply_factor(Q, leg, M))
        self.env[(u, v)] = blocks

    def _init_envs(self) -> None:
        tr = self.tree
        order = []

        def post(v):
            for c in tr.children[v]:
                post(c)
            order.append(v)

        post(0)
        for v in order:
            if tr.parent[v] >= 0:
                self.update_env(v, tr.parent[v])

    # ------------------------------------------------------------------ local maps
    def heff(self, v: int, x: np.ndarray) -> np.ndarray:
        return self.apply_terms(x, self.node_terms(v))

    def hbond(self, u: int, w: int, X: np.ndarray) -> np.ndarray:
        """H_bond(u, w) X for the bond matrix X[i_u, i_w]."""
        Eu = self.env[(u, w)]
        Ew = self.env[(w, u)]
        y = Eu["H"] @ X + X @ Ew["H"].T
        for ti, _ in self.crossing(u, w):
            y = y + Eu[ti] @ X @ Ew[ti].T
        return y

    def qr_toward(self, v: int, u: int) -> np.ndarray:
        """A_v <- Q (isometry toward u); returns R with R[i_v, i_u-old]."""
        tr = self.tree
        A = self.A[v]
        l = tr.leg_of(v, u)
        Am = np.moveaxis(A, l, -1)
        shp = Am.shape
        Q, R = householder_qr(Am.reshape(-1, shp[-1]), self.qr_cutoff)
        self.A[v] = np.moveaxis(Q.reshape(shp), -1, l)
        return R

    def absorb(self, R: np.ndarray, u: int, v: int) -> None:
        """A_u <- R on u's leg toward v."""
        self.A[u] = apply_factor(self.A[u], self.tree.leg_of(u, v), R)

    def forward(self, v: int, tau: float) -> None:
        self.A[v] = expm_lanczos(lambda x: self.heff(v, x), self.A[v], tau / HBAR,
                                 self.tol, self.mmax, self.stats)
        self.stats["forward"] = self.stats.get("forward", 0) + 1

    def backward(self, u: int, w: int, R: np.ndarray, tau: float) -> np.ndarray:
        self.stats["backward"] = self.stats.get("backward", 0) + 1
        return expm_lanczos(lambda X: self.hbond(u, w, X), R, -tau / HBAR,
                            self.tol, self.mmax, self.stats)

    # ------------------------------------------------------------------ sweeps
    def _visit(self, v: int, tau: float) -> None:
        tr = self.tree
        self.forward(v, tau)
        for c in tr.children[v]:
            R = self.qr_toward(v, c)
            self.update_env(v, c)
            R = self.backward(v, c, R, tau)
            self.absorb(R, c, v)
            self._visit(c, tau)
            R = self.qr_toward(c, v)
            self.update_env(c, v)
            self.absorb(R, v, c)

    def _visit_adj(self, v: int, tau: float) -> None:
        tr = self.tree
        for c in reversed(tr.children[v]):
            R = self.qr_toward(v, c)
            self.update_env(v, c)
            self.absorb(R, c, v)
            self._visit_adj(c, tau)
            R = self.qr_toward(c, v)
            self.update_env(c, v)
            R = self.backward(c, v, R, tau)
            self.absorb(R, v, c)
        self.forward(v, tau)

    def step(self, dt: float) -> None:
        self._visit(0, 0.5 * dt)
        self._visit_adj(0, 0.5 * dt)
        self.t += dt

    # ------------------------------------------------------------------ adaptive bond dimension
    def grow_bonds(self, new_bond) -> List[int]:
        """Raises bond dimensions during the run (the paper raises them until the dynamics
        converge; Methods, tensor network states).  new_bond[v] is the requested dimension of
        node v's parent bond; the root's entry and requests not above the current dimension
        leave a bond as it is, and the requests go through the build's clamp.  The state is
        unchanged:
          * both tensors of a grown bond get zero slices on it;
          * grown bonds are taken children first: the child's tensor is made an isometry
            toward its parent again by this module's QR, whose zero columns get the identity
            reflector (the completion rule), and R (the identity on the old indices, zero on
            the new ones) is absorbed into the parent;
          * every environment is rebuilt.
        Taking children first leaves each parent's completion for later, so no absorb acts on
        a completed tensor.  The new bond directions are the completion vectors, which the
        one-site integrator can then populate.  Returns the grown nodes."""
        tr = self.tree
        req = [0] + [max(tr.bond[v], int(new_bond[v])) for v in range(1, tr.n)]
        nb = _clamp_bonds(tr, req)
        nb[0] = 0
        grown = [v for v in range(1, tr.n) if nb[v] > tr.bond[v]]
        if not grown:
            return []
        tr.bond = nb
        for v in range(tr.n):
            shape = tuple(tr.legs(v))
            if shape != self.A[v].shape:
                B = np.zeros(shape, dtype=complex)
                B[tuple(slice(0, k) for k in self.A[v].shape)] = self.A[v]
                self.A[v] = B
        for v in sorted(grown, reverse=True):
            p = tr.parent[v]
            R = self.qr_toward(v, p)
            self.absorb(R, p, v)
        self.env = {}
        self._init_envs()
        return grown

    def bond_spectra(self) -> Dict[int, np.ndarray]:
        """Ascending eigenvalues (Schmidt weights) of every parent bond's density matrix."""
        return {v: np.linalg.eigvalsh(0.5 * (rho + rho.conj().T)) for v, rho in self.bond_densities().items()}

    def adapt_bonds(self, eps: float, step: int, d_max: int) -> List[int]:
        """Adaptive rule: a parent bond below d_max whose smallest Schmidt weight exceeds eps
        uses all of its dimension; it grows by `step`, up to d_max (then the build's clamp)."""
        new = [0] * self.tree.n
        for v, w in self.bond_spectra().items():
            if self.tree.bond[v] < d_max and w[0] > eps:
                new[v] = min(self.tree.bond[v] + step, d_max)
        return self.grow_bonds(new)

    # ------------------------------------------------------------------ observables
    def norm(self) -> float:
        return float(np.sqrt(np.sum(np.abs(self.A[0]) ** 2)))

    def energy(self) -> float:
        A = self.A[0]
        return float(np.real(np.vdot(A, self.heff(0, A))) / np.real(np.vdot(A, A)))

    def rho_el(self) -> np.ndarray:
        """Reduced density matrix of the electronic node (the centre is at the root)."""
        A = self.A[0]
        pl = self.tree.phys_leg(0)
        others = [k for k in range(A.ndim) if k != pl]
        return np.tensordot(A, A.conj(), axes=(others, others))

    def site_densities(self) -> Dict[int, np.ndarray]:
        """Local reduced density matrices of every node with a physical leg,
        by the downward pass of bond density matrices from the root."""
        tr = self.tree
        out = {0: self.rho_el()}
        stack = []
        A = self.A[0]
        for c in tr.children[0]:
            l = tr.leg_of(0, c)
            others = [k for k in range(A.ndim) if k != l]
            stack.append((c, np.tensordot(A, A.conj(), axes=(others, others))))
        while stack:
            v, rho_in = stack.pop()
            Q = self.A[v]
            # X[a, ...] = sum_a' rho_in[a', a] Q[a', ...]; contracting X with conj(Q)
            # over a gives sum rho_in[a', a] Q[a', ...] conj(Q[a, ...])
            X = apply_factor(Q, 0, rho_in.T)
            if tr.phys[v] > 0:
                pl = tr.phys_leg(v)
                others = [k for k in range(Q.ndim) if k != pl]
                out[v] = np.tensordot(X, Q.conj(), axes=(others, others))
            for c in tr.children[v]:
                l = tr.leg_of(v, c)
                others = [k for k in range(Q.ndim) if k != l]
                stack.append((c, np.tensordot(X, Q.conj(), axes=(others, others))))
        return out

    def bond_densities(self) -> Dict[int, np.ndarray]:
        """Density matrix of every non-root node's parent bond, by the downward pass from the
        root (the centre): rho_in(v)[b, b'] in the bond basis of v's tensor."""
        tr = self.tree
        out = {}
        A = self.A[0]
        stack = []
        for c in tr.children[0]:
            l = tr.leg_of(0, c)
            others = [k for k in range(A.ndim) if k != l]
            stack.append((c, np.tensordot(A, A.conj(), axes=(others, others))))
        while stack:
            v, rho_in = stack.pop()
            out[v] = rho_in
            Q = self.A[v]
            X = apply_factor(Q, 0, rho_in.T)
            for c in tr.children[v]:
                l = tr.leg_of(v, c)
                others = [k for k in range(Q.ndim) if k != l]
                stack.append((c, np.tensordot(X, Q.conj(), axes=(others, others))))
        return out

    def bond_entropies(self) -> np.ndarray:
        """[S(rho_S), S(bond of node 1), ...]: von Neumann entropies -sum l ln l of the
        electronic reduced density matrix and of every bond's density matrix (Results, the
        entanglement entropy that guides the tree's design)."""
        def ent(rho):
            w = np.linalg.eigvalsh(0.5 * (rho + rho.conj().T))
            w = w[w > 1e-300]
            return float(-np.sum(w * np.log(w)))
        dens = self.bond_densities()
        S = np.zeros(self.tree.n)
        S[0] = ent(self.rho_el())
        for v, rho in dens.items():
            S[v] = ent(rho)
        return S

    def occupations(self) -> np.ndarray:
        """<a^+ a> of every chain site, chains in order, sites in chain order."""
        tr = self.tree
        dens = self.site_densities()
        occ = []
        for nodes in tr.chain_nodes:
            for v in nodes:
                d = tr.phys[v]
                occ.append(float(np.real(np.sum(np.arange(d) * np.diag(dens[v])))))
        return np.array(occ)

    def populations(self) -> np.ndarray:
        return np.real(np.diag(self.rho_el())).copy()

    # ------------------------------------------------------------------ energy surfaces
    def kinetic_tree(self) -> Tree:
        """The tree with the nuclear kinetic energy T of the chains as its operator.

        A chain is an orthogonal transform a_m = sum_n U_mn b_n of normal modes with
        dimensionless momenta p_n = i (b_n^+ - b_n) / sqrt(2) and kinetic energy
        w_n p_n^2 / 2, so T = (1/2) sum_mm' h_mm' P_m P_m' with h = U diag(w) U^T the chain's
        tridiagonal matrix (onsite w_m, hoppings t_m) and P_m = i (a_m^+ - a_m) / sqrt(2):
            T = -(1/4) sum_m w_m (a^+ - a)_m^2 - (1/2) sum_m t_m (a^+ - a)_m (a^+ - a)_{m+1},
        with the operators truncated to the Fock states 0 .. d-1 (products of the truncated
        matrices)."""
        from .chain import chain_of
        tr = self.tree
        onsite = [None] * tr.n
        coups = []
        for i, env in enumerate(self.problem.envs):
            _, om, hop = chain_of(env.spectral, env.L)
            a = lowering(env.d)
            P = a.conj().T - a
            nodes = tr.chain_nodes[i]
            for nn, v in enumerate(nodes):
                onsite[v] = -0.25 * om[nn] * (P @ P)
            for nn in range(env.L - 1):
                coups.append(Coupling(nodes[nn], -0.5 * hop[nn] * P, nodes[nn + 1], P.copy()))
        return Tree(parent=tr.parent, children=tr.children, phys=tr.phys, kind=tr.kind,
                    site_index=tr.site_index, bond=tr.bond, onsite=onsite, couplings=coups, n_el=tr.n_el,
                    chain_nodes=tr.chain_nodes, psi_el=tr.psi_el)

    def _projected(self, op_tree: Tree):
        """The root's local operator for op_tree (its environment blocks computed from the
        current tensors, which are isometries toward the root after a step), as a
        function on root-shaped tensors."""
        other = object.__new__(TTNS)
        other.__dict__.update(self.__dict__)
        other.tree = op_tree
        other.env = {}
        other._init_envs()
        return lambda x: other.heff(0, x)

    def energy_surfaces(self, sigma_tol: float = 1e-7):
        """Energy surfaces of Eq. 3-4 at the current time (the centre at the root).

        The bath states phi_k are the environment Schmidt vectors of the state for the
        bipartition electronic | everything else (the SVD of the root tensor matricised as
        other legs x electronic leg), kept where the Schmidt value exceeds sigma_tol.  With
        the basis |k, l> = |phi_k> |l> (bath-major),
            H_eff[(i j), (k l)] = <phi_i| <j| H |phi_k> |l>,   V_eff = H_eff - T_eff,
        T the chains' nuclear kinetic energy (kinetic_tree).  Returns the ascending
        eigenvalues of H_eff (total energy surfaces) and of V_eff (potential energy
        surfaces), the Schmidt values, and both matrices."""
        tr = self.tree
        A = self.A[0]
        n_el = tr.n_el
        M = A.reshape(-1, n_el)                       # (other legs) x electronic
        rho = M.T @ M.conj()                          # rho[s, s'] = sum_r M[r, s] conj(M[r, s'])
        w, U = np.linalg.eigh(rho)
        order = np.argsort(w)[::-1]
        w, U = w[order], U[:, order]
        sig = np.sqrt(np.clip(w, 0.0, None))
        keep = [k for k in range(n_el) if sig[k] > sigma_tol]
        phis = [(M @ U[:, k].conj()) / sig[k] for k in keep]
        basis = []
        for ph in phis:
            for l in range(n_el):
                X = np.zeros_like(M)
                X[:, l] = ph
                basis.append(X.reshape(A.shape))
        H = self._projected(tr)
        T = self._projected(self.kinetic_tree())
        nb = len(basis)
        Heff = np.zeros((nb, nb), dtype=complex)
        Teff = np.zeros((nb, nb), dtype=complex)
        for c, X in enumerate(basis):
            hx, tx = H(X), T(X)
            for r, Y in enumerate(basis):
                Heff[r, c] = np.vdot(Y, hx)
                Teff[r, c] = np.vdot(Y, tx)
        Veff = Heff - Teff
        return np.linalg.eigvalsh(Heff), np.linalg.eigvalsh(Veff), sig[keep], Heff, Veff

    # ------------------------------------------------------------------ dense state
    def to_dense(self) -> np.ndarray:
        """The full state vector; basis order: electronic index, then the chain
        sites in node order (only for tiny trees)."""
        tr = self.tree

        def contract(v):
            # returns tensor with legs [parent bond?] + [phys of subtree nodes in node order]
            T = self.A[v]
            legs_nodes = []  # node id owning each physical leg currently in T (after bonds)
            # children bond legs sit at positions (1 if parent) .. ; contract them one by one
            off = 1 if tr.parent[v] >= 0 else 0
            nchild = len(tr.children[v])
            # move own phys leg to the end first
            cur = T
            phys_owner = []
            if tr.phys[v] > 0:
                phys_owner = [v]
            for k, c in enumerate(tr.children[v]):
                S, owners = contract(c)
                # the child's bond leg is at position off (we consume children in order)
                cur = np.tensordot(cur, S, axes=([off], [0]))
                # now legs: [parent?] + remaining children + own phys(es) + child's phys legs
                phys_owner = phys_owner + owners
            return cur, phys_owner

        T, owners = contract(0)
        # T legs: own phys of root then all others in the order they were appended
        order = np.argsort(owners, kind="stable")
        T = np.transpose(T, order)
        return T.reshape(-1)


def run(problem, n_steps: Optional[int] = None, record_every: int = 1, occupations: bool = True):
    """Runs the sweep and returns the populations (and chain occupations) after
    every `record_every` steps, starting with t = 0."""
    st = TTNS(problem)
    n = problem.n_steps if n_steps is None else n_steps
    pops = [st.populations()]
    occs = [st.occupations()] if occupations else []
    for k in range(n):
        st.step(problem.dt)
        if (k + 1) % record_every == 0:
            pops.append(st.populations())
            if occupations:
                occs.append(st.occupations())
    return st, np.array(pops), (np.array(occs) if occupations else None)
