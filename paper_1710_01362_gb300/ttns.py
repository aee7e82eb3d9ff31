"""Thin ctypes binding of libttns.so (argument marshalling only).

Every call maps one-to-one onto an entry point of include/ttns.h.  The library
must be built (``paper_1710_01362_gb300.build.build()``); importing this module
without it raises, and there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libttns.so")

TTNS_FP64 = 0
TTNS_TF32X3 = 1
TTNS_MIXED = 1
TTNS_BF16X3 = 2
TTNS_FP32 = 3

STATUS = {0: "ok", 1: "invalid", 2: "oom", 3: "cuda", 4: "not converged", 5: "timeout", 6: "nonfinite", 7: "io"}

EXPORTS = [
    "ttns_build_tree", "ttns_build_batch", "ttns_step", "ttns_sync", "ttns_reduced_density_matrix",
    "ttns_occupations", "ttns_observables", "ttns_trajectory", "ttns_populations_device", "ttns_get_counters",
    "ttns_node_info", "ttns_get_node", "ttns_save", "ttns_load", "ttns_load_state", "ttns_last_error", "ttns_free",
    "ttns_chain_ohmic", "ttns_chain_from_modes", "ttns_plan", "ttns_selftest_wait_timeout",
    "ttns_rho_from_root_noalloc", "ttns_autotune", "ttns_selftest_tc_gemm", "ttns_mlp_gemm", "ttns_mlp_colsum",
    "ttns_mlp_diff", "ttns_mlp_adam", "ttns_mlp_status", "ttns_energy_surfaces", "ttns_bond_entropies",
    "ttns_cluster_modes", "ttns_grow_bonds", "ttns_adapt_bonds",
]


class TTNSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Options(C.Structure):
    _fields_ = [
        ("precision", C.c_int), ("krylov_tol", C.c_double), ("krylov_mmax", C.c_int),
        ("cuda_stream", C.c_void_p), ("er_tree", C.c_int), ("D_er", C.c_int), ("init_state", C.c_int),
        ("psi_el", C.POINTER(C.c_double)), ("record", C.c_int), ("max_record", C.c_int),
        ("cluster_ctas", C.c_int), ("grid_ctas", C.c_int), ("grid_threshold", C.c_int),
        ("spin_limit", C.c_longlong), ("profile", C.c_int), ("launch_flags", C.c_int),
        ("qr_grid_threshold", C.c_int), ("qr_cutoff", C.c_double),
    ]


class ProblemC(C.Structure):
    _fields_ = [
        ("n_el", C.c_int), ("H_S", C.POINTER(C.c_double)), ("n_env", C.c_int), ("W_bar", C.POINTER(C.c_double)),
        ("rc_coupling", C.POINTER(C.c_double)), ("chain_len", C.POINTER(C.c_int)),
        ("chain_omega", C.POINTER(C.POINTER(C.c_double))), ("chain_hop", C.POINTER(C.POINTER(C.c_double))),
        ("local_dim", C.POINTER(C.c_int)), ("bond_dim", C.POINTER(C.c_int)), ("obb_dim", C.POINTER(C.c_int)),
    ]


class PlanInfo(C.Structure):
    _fields_ = [("n_nodes", C.c_int), ("pool_complex", C.c_longlong), ("max_node", C.c_int), ("max_bond", C.c_int),
                ("instructions_per_step", C.c_int), ("work_complex_per_worker", C.c_longlong),
                ("apply_flops_per_step", C.c_double), ("env_flops_per_step", C.c_double),
                ("exponentials_per_step", C.c_int), ("env_updates_per_step", C.c_int),
                ("n_bonds_written", C.c_int), ("bonds", C.c_int * 4096)]


class Counters(C.Structure):
    _fields_ = [("krylov_iters", C.c_longlong), ("applies", C.c_longlong), ("contraction_flops", C.c_double),
                ("not_converged", C.c_longlong), ("steps", C.c_longlong), ("op_seconds", (C.c_double * 2) * 6),
                ("op_count", (C.c_longlong * 2) * 6), ("expm_phase_seconds", C.c_double * 8),
                ("qr_phase_seconds", C.c_double * 8), ("expm_phase_seconds_grid", C.c_double * 8),
                ("qr_phase_seconds_grid", C.c_double * 8), ("launch_fallbacks", C.c_longlong),
                ("env_phase_seconds", (C.c_double * 4) * 2), ("tc_phase_seconds", C.c_double * 4)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_1710_01362_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        dp = C.POINTER(C.c_double)
        L.ttns_last_error.restype = C.c_char_p
        L.ttns_build_tree.argtypes = [C.POINTER(ProblemC), C.POINTER(Options), C.POINTER(C.c_void_p)]
        L.ttns_build_batch.argtypes = [C.c_int, C.POINTER(ProblemC), C.POINTER(Options), C.POINTER(C.c_void_p)]
        L.ttns_step.argtypes = [C.c_void_p, C.c_double, C.c_int]
        L.ttns_autotune.argtypes = [C.c_int, C.POINTER(ProblemC), C.POINTER(Options), C.c_double, C.c_int,
                                    C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double)]
        L.ttns_sync.argtypes = [C.c_void_p]
        L.ttns_reduced_density_matrix.argtypes = [C.c_void_p, C.c_int, dp]
        L.ttns_occupations.argtypes = [C.c_void_p, C.c_int, dp]
        L.ttns_observables.argtypes = [C.c_void_p, C.c_int, dp, dp]
        L.ttns_trajectory.argtypes = [C.c_void_p, C.c_int, dp, C.c_int, C.POINTER(C.c_int)]
        L.ttns_energy_surfaces.argtypes = [C.c_void_p, C.c_int, C.c_double, dp, dp, dp, C.POINTER(C.c_int)]
        L.ttns_bond_entropies.argtypes = [C.c_void_p, C.c_int, dp]
        L.ttns_grow_bonds.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int)]
        L.ttns_adapt_bonds.argtypes = [C.c_void_p, C.c_double, C.c_int, C.c_int, C.POINTER(C.c_int)]
        ip = C.POINTER(C.c_int)
        L.ttns_cluster_modes.argtypes = [C.c_int, C.c_int, dp, C.c_int, ip, C.c_int, ip, dp, dp, ip]
        L.ttns_populations_device.argtypes = [C.c_void_p, C.c_void_p]
        L.ttns_get_counters.argtypes = [C.c_void_p, C.POINTER(Counters)]
        L.ttns_node_info.argtypes = [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                     C.POINTER(C.c_int)]
        L.ttns_get_node.argtypes = [C.c_void_p, C.c_int, C.c_int, dp, C.c_size_t]
        L.ttns_save.argtypes = [C.c_void_p, C.c_char_p]
        L.ttns_load_state.argtypes = [C.c_void_p, C.c_char_p]
        L.ttns_load.argtypes = [C.c_char_p, C.POINTER(Options), C.POINTER(C.c_void_p)]
        L.ttns_free.argtypes = [C.c_void_p]
        L.ttns_free.restype = None
        L.ttns_plan.argtypes = [C.c_int, C.POINTER(ProblemC), C.POINTER(Options), C.POINTER(PlanInfo)]
        L.ttns_selftest_wait_timeout.argtypes = [C.c_longlong, C.POINTER(C.c_int)]
        L.ttns_selftest_tc_gemm.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, dp, dp, dp, C.POINTER(C.c_int)]
        vp = C.c_void_p
        L.ttns_mlp_gemm.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, vp, C.c_int, C.c_int, vp, C.c_int, C.c_int,
                                    vp, C.c_int, C.c_int, vp, vp]
        L.ttns_mlp_colsum.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp, vp]
        L.ttns_mlp_diff.argtypes = [vp, vp, vp, C.c_longlong, C.c_float, vp]
        L.ttns_mlp_adam.argtypes = [vp, vp, vp, vp, C.c_longlong, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int,
                                    vp]
        L.ttns_mlp_status.argtypes = [C.POINTER(C.c_int), C.c_int]
        L.ttns_rho_from_root_noalloc.argtypes = [C.c_void_p, C.c_longlong, C.c_int, C.c_void_p, C.c_void_p]
        L.ttns_chain_ohmic.argtypes = [C.c_double, C.c_double, C.c_int, dp, dp, dp]
        L.ttns_chain_from_modes.argtypes = [C.c_int, dp, dp, C.c_int, dp, dp, dp]
        _lib = L
    return _lib


def _check(code: int) -> None:
    if code != 0:
        raise TTNSError(code, lib().ttns_last_error().decode())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def selftest_wait_timeout(spin_limit: int) -> int:
    st = C.c_int(-1)
    _check(lib().ttns_selftest_wait_timeout(spin_limit, C.byref(st)))
    return st.value


def selftest_tc_gemm(kind: int, Z: np.ndarray, Mt: np.ndarray):
    """Y = Z Mt^T on the tensor cores (kind 1: TF32X3, 2: BF16X3); returns (Y, device status)."""
    Zc = np.ascontiguousarray(Z, dtype=np.complex128)
    Mc = np.ascontiguousarray(Mt, dtype=np.complex128)
    M, K = Zc.shape
    N = Mc.shape[0]
    Y = np.zeros((M, N), dtype=np.complex128)
    st = C.c_int(-1)
    _check(lib().ttns_selftest_tc_gemm(kind, M, K, N, _dptr(Zc.view(np.float64)), _dptr(Mc.view(np.float64)),
                                        _dptr(Y.view(np.float64)), C.byref(st)))
    return Y, st.value


def rho_from_root_noalloc(d_root: int, rows: int, n_el: int, d_rho: int, stream: Optional[int] = None) -> None:
    """Allocation-free electronic density matrix from a root tensor in device memory
    (device pointers given as integers); enqueued on `stream`."""
    _check(lib().ttns_rho_from_root_noalloc(C.c_void_p(d_root), rows, n_el, C.c_void_p(d_rho), C.c_void_p(stream)))


def cluster_modes(W: np.ndarray, k: int, init, max_iter: int = 100):
    """Weighted k-means of the modes' coupling patterns (ttns_cluster_modes): returns
    (assignment, Wbar (k, n_el, n_el), lambda per mode, iterations)."""
    Wc = np.ascontiguousarray(W, dtype=np.complex128)
    n_modes, n_el, _ = Wc.shape
    ini = np.ascontiguousarray(init, dtype=np.int32)
    assign = np.zeros(n_modes, dtype=np.int32)
    Wbar = np.zeros((k, n_el, n_el), dtype=np.complex128)
    lam = np.zeros(n_modes)
    it = C.c_int()
    ip = C.POINTER(C.c_int)
    _check(lib().ttns_cluster_modes(n_modes, n_el, _dptr(Wc.view(np.float64)), k, ini.ctypes.data_as(ip), max_iter,
                                    assign.ctypes.data_as(ip), _dptr(Wbar.view(np.float64)), _dptr(lam), C.byref(it)))
    return assign, Wbar, lam, it.value


def chain_ohmic(alpha: float, omega_c: float, L: int):
    rc = np.zeros(1)
    on = np.zeros(L)
    hop = np.zeros(max(L - 1, 1))
    _check(lib().ttns_chain_ohmic(alpha, omega_c, L, _dptr(rc), _dptr(on), _dptr(hop)))
    return float(rc[0]), on, hop[: L - 1]


def chain_from_modes(omega, lam, L: int):
    om = np.ascontiguousarray(omega, dtype=float)
    la = np.ascontiguousarray(lam, dtype=float)
    rc = np.zeros(1)
    on = np.zeros(L)
    hop = np.zeros(max(L - 1, 1))
    _check(lib().ttns_chain_from_modes(om.size, _dptr(om), _dptr(la), L, _dptr(rc), _dptr(on), _dptr(hop)))
    return float(rc[0]), on, hop[: L - 1]


def chain_of(spectral, L: int):
    if spectral[0] == "ohmic":
        return chain_ohmic(spectral[1], spectral[2], L)
    return chain_from_modes(spectral[1], spectral[2], L)


def _cplx(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    return np.ascontiguousarray(a.view(np.float64).reshape(-1))


class _ProblemKeep:
    """Holds the numpy buffers a ProblemC points into."""

    def __init__(self, problem):
        p = problem
        ne = p.n_el
        self.H = _cplx(p.H_S)
        self.W = _cplx(np.stack([e.W_bar for e in p.envs]))
        chains = [chain_of(e.spectral, e.L) for e in p.envs]
        self.rc = np.array([c[0] for c in chains], dtype=float)
        self.L = np.array([e.L for e in p.envs], dtype=np.int32)
        self.om = [np.ascontiguousarray(c[1], dtype=float) for c in chains]
        self.hop = [np.ascontiguousarray(c[2] if len(c[2]) else np.zeros(1), dtype=float) for c in chains]
        self.om_ptrs = (C.POINTER(C.c_double) * len(self.om))(*[_dptr(x) for x in self.om])
        self.hop_ptrs = (C.POINTER(C.c_double) * len(self.hop))(*[_dptr(x) for x in self.hop])
        self.d = np.array([e.d for e in p.envs], dtype=np.int32)
        self.D = np.array([e.D for e in p.envs], dtype=np.int32)
        self.obb = np.array([getattr(e, "obb", 0) or 0 for e in p.envs], dtype=np.int32)
        self.c = ProblemC(ne, _dptr(self.H), len(p.envs), _dptr(self.W), _dptr(self.rc),
                          self.L.ctypes.data_as(C.POINTER(C.c_int)), self.om_ptrs, self.hop_ptrs,
                          self.d.ctypes.data_as(C.POINTER(C.c_int)), self.D.ctypes.data_as(C.POINTER(C.c_int)),
                          self.obb.ctypes.data_as(C.POINTER(C.c_int)))


def current_stream() -> Optional[int]:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def _options(p0, precision, record=False, max_record=0, stream=None, cluster_ctas=0, grid_ctas=0,
             krylov_tol=0.0, krylov_mmax=0, keep=None, grid_threshold=0, spin_limit=0, profile=0,
             launch_flags=0, qr_grid_threshold=0, qr_cutoff=0.0):
    psi = None
    if p0.psi_el is not None:
        arr = _cplx(p0.psi_el)
        if keep is not None:
            keep.append(arr)
        psi = _dptr(arr)
    if not qr_cutoff and getattr(p0, "qr_cutoff", None):
        qr_cutoff = float(p0.qr_cutoff)
    return Options(precision, krylov_tol, krylov_mmax, stream, int(p0.er_tree), int(p0.D_er),
                   int(p0.init_state), psi, int(record), int(max_record), cluster_ctas, grid_ctas,
                   grid_threshold, spin_limit, profile, launch_flags, qr_grid_threshold, qr_cutoff)


def plan(problems, precision: int = TTNS_MIXED, krylov_mmax: int = 0, **kw) -> dict:
    """Host-only compile and table check; no GPU needed."""
    probs = list(problems) if isinstance(problems, (list, tuple)) else [problems]
    keep = [_ProblemKeep(p) for p in probs]
    hold = []
    opt = _options(probs[0], precision, keep=hold, krylov_mmax=krylov_mmax, **kw)
    arr = (ProblemC * len(probs))(*[k.c for k in keep])
    info = PlanInfo()
    _check(lib().ttns_plan(len(probs), arr, C.byref(opt), C.byref(info)))
    return {"n_nodes": info.n_nodes, "pool_complex": info.pool_complex, "max_node": info.max_node,
            "max_bond": info.max_bond, "instructions_per_step": info.instructions_per_step,
            "work_complex_per_worker": info.work_complex_per_worker,
            "apply_flops_per_step": info.apply_flops_per_step, "env_flops_per_step": info.env_flops_per_step,
            "exponentials_per_step": info.exponentials_per_step, "env_updates_per_step": info.env_updates_per_step,
            "bonds": [info.bonds[i] for i in range(info.n_bonds_written)]}


def autotune(problems, dt: float, precision: int = TTNS_MIXED, candidates=None, stream: Optional[int] = None, **kw):
    """Fastest number of CTAs per cluster team for this tree set (ttns_autotune); returns
    (cluster_ctas, seconds_per_step)."""
    probs = list(problems) if isinstance(problems, (list, tuple)) else [problems]
    keep = [_ProblemKeep(p) for p in probs]
    hold = []
    if stream is None:
        stream = current_stream()
    opt = _options(probs[0], precision, stream=stream, keep=hold, **kw)
    arr = (ProblemC * len(probs))(*[k.c for k in keep])
    cand = list(candidates or [])
    carr = (C.c_int * max(1, len(cand)))(*cand) if cand else None
    best = C.c_int(0)
    secs = C.c_double(0.0)
    _check(lib().ttns_autotune(len(probs), arr, C.byref(opt), C.c_double(dt), len(cand), carr, C.byref(best),
                               C.byref(secs)))
    return best.value, secs.value


class Tree:
    """A set of trees on the device (one tree, or a batch advanced together)."""

    def __init__(self, problems, precision: int = TTNS_MIXED, record: bool = False, max_record: int = 0,
                 stream: Optional[int] = None, cluster_ctas: int = 0, grid_ctas: int = 0,
                 krylov_tol: float = 0.0, krylov_mmax: int = 0, grid_threshold: int = 0, spin_limit: int = 0,
                 profile: bool = False, launch_flags: int = 0, qr_grid_threshold: int = 0, qr_cutoff: float = 0.0):
        single = not isinstance(problems, (list, tuple))
        probs = [problems] if single else list(problems)
        self.problems = probs
        self._keep = [_ProblemKeep(p) for p in probs]
        self._hold = []
        if stream is None:
            stream = current_stream()
        self.opt = _options(probs[0], precision, record, max_record, stream, cluster_ctas, grid_ctas, krylov_tol,
                            krylov_mmax, keep=self._hold, grid_threshold=grid_threshold, spin_limit=spin_limit,
                            profile=int(profile), launch_flags=int(launch_flags),
                            qr_grid_threshold=qr_grid_threshold, qr_cutoff=qr_cutoff)
        h = C.c_void_p()
        arr = (ProblemC * len(probs))(*[k.c for k in self._keep])
        if len(probs) == 1:
            _check(lib().ttns_build_tree(arr, C.byref(self.opt), C.byref(h)))
        else:
            _check(lib().ttns_build_batch(len(probs), arr, C.byref(self.opt), C.byref(h)))
        self.h = h
        self.n_trees = len(probs)

    def close(self) -> None:
        if self.h:
            lib().ttns_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, dt: float, n: int = 1) -> None:
        _check(lib().ttns_step(self.h, dt, n))

    def sync(self) -> None:
        _check(lib().ttns_sync(self.h))

    def rho(self, k: int = 0) -> np.ndarray:
        ne = self.problems[k].n_el
        out = np.zeros(2 * ne * ne)
        _check(lib().ttns_reduced_density_matrix(self.h, k, _dptr(out)))
        return out.view(np.complex128).reshape(ne, ne)

    def populations(self, k: int = 0) -> np.ndarray:
        return np.real(np.diag(self.rho(k))).copy()

    def occupations(self, k: int = 0) -> np.ndarray:
        n = sum(e.L for e in self.problems[k].envs)
        out = np.zeros(n)
        _check(lib().ttns_occupations(self.h, k, _dptr(out)))
        return out

    def observables(self, k: int = 0):
        nrm = C.c_double()
        en = C.c_double()
        _check(lib().ttns_observables(self.h, k, C.byref(nrm), C.byref(en)))
        return nrm.value, en.value

    def trajectory(self, k: int = 0, max_steps: int = 100000) -> np.ndarray:
        ne = self.problems[k].n_el
        out = np.zeros(2 * max_steps * ne * ne)
        n = C.c_int()
        _check(lib().ttns_trajectory(self.h, k, _dptr(out), max_steps, C.byref(n)))
        return out[: 2 * n.value * ne * ne].view(np.complex128).reshape(n.value, ne, ne)

    def energy_surfaces(self, k: int = 0, sigma_tol: float = 1e-7):
        """(total energy surfaces, potential energy surfaces, Schmidt values): the ascending
        eigenvalues of H_eff and V_eff in the basis of the kept bath states (Eq. 3-4)."""
        ne = self.problems[k].n_el
        tes = np.zeros(32)
        pes = np.zeros(32)
        sig = np.zeros(ne)
        nb = C.c_int()
        _check(lib().ttns_energy_surfaces(self.h, k, sigma_tol, _dptr(tes), _dptr(pes), _dptr(sig), C.byref(nb)))
        nv = nb.value * ne
        return tes[:nv].copy(), pes[:nv].copy(), sig[: nb.value].copy()

    def bond_entropies(self, k: int = 0) -> np.ndarray:
        """[S(rho_S), S(bond of node 1), ..]: von Neumann entropies (natural log)."""
        out = np.zeros(self.n_nodes(k))
        _check(lib().ttns_bond_entropies(self.h, k, _dptr(out)))
        return out

    def bonds(self, k: int = 0) -> list:
        """Parent-bond dimension of every node (the root's entry 0)."""
        out = [0]
        for v in range(1, self.n_nodes(k)):
            nl = C.c_int()
            dims = (C.c_int * 8)()
            _check(lib().ttns_node_info(self.h, k, v, C.byref(nl), dims, None))
            out.append(dims[0])
        return out

    def grow_bonds(self, new_bond) -> int:
        """Raises parent-bond dimensions (new_bond[v] for node v; see ttns_grow_bonds); returns
        the number of grown bonds."""
        n = self.n_nodes(0)
        req = (C.c_int * n)(*[int(x) for x in new_bond])
        g = C.c_int()
        _check(lib().ttns_grow_bonds(self.h, req, n, C.byref(g)))
        return g.value

    def adapt_bonds(self, eps: float, step: int, d_max: int) -> int:
        """The adaptive rule (ttns_adapt_bonds); returns the number of grown bonds."""
        g = C.c_int()
        _check(lib().ttns_adapt_bonds(self.h, eps, step, d_max, C.byref(g)))
        return g.value

    def populations_device(self, dev_ptr: int) -> None:
        _check(lib().ttns_populations_device(self.h, C.c_void_p(dev_ptr)))

    def counters(self) -> dict:
        c = Counters()
        _check(lib().ttns_get_counters(self.h, C.byref(c)))
        names = ["fwd", "qr", "env", "bond", "absorb", "record"]
        prof = {}
        for op in range(6):
            for k, team in enumerate(["grid", "cluster"]):
                if c.op_count[op][k]:
                    prof[f"{names[op]}_{team}"] = (c.op_seconds[op][k], c.op_count[op][k])
        phases = dict(zip(["staging", "stage1", "apply_alpha", "recurrence_beta", "small_expm", "combine", "norm", "tc_tasks"],
                          [c.expm_phase_seconds[k] for k in range(8)]))
        qr_names = ["copy_norm", "columns", "gram", "T_Z", "write_Q", "col_reflector", "col_update", "col_dots"]
        qr = dict(zip(qr_names, [c.qr_phase_seconds[k] for k in range(8)]))
        phases_g = dict(zip(["staging", "stage1", "apply_alpha", "recurrence_beta", "small_expm", "combine", "norm", "tc_tasks"],
                            [c.expm_phase_seconds_grid[k] for k in range(8)]))
        qr_g = dict(zip(qr_names, [c.qr_phase_seconds_grid[k] for k in range(8)]))
        env_names = ["staging", "apply", "projection", "team_sum"]
        return {"krylov_iters": c.krylov_iters, "applies": c.applies, "contraction_flops": c.contraction_flops,
                "not_converged": c.not_converged, "steps": c.steps, "profile": prof, "expm_phases": phases,
                "qr_phases": qr, "expm_phases_grid": phases_g, "qr_phases_grid": qr_g,
                "env_phases": dict(zip(env_names, [c.env_phase_seconds[0][k] for k in range(4)])),
                "env_phases_grid": dict(zip(env_names, [c.env_phase_seconds[1][k] for k in range(4)])),
                "tc_phases": dict(zip(["staging", "mma", "readback", "write"], [c.tc_phase_seconds[k] for k in range(4)])),
                "launch_fallbacks": c.launch_fallbacks}

    def n_nodes(self, k: int = 0) -> int:
        n = C.c_int()
        _check(lib().ttns_node_info(self.h, k, -1, None, None, C.byref(n)))
        return n.value

    def node(self, v: int, k: int = 0) -> np.ndarray:
        nl = C.c_int()
        dims = (C.c_int * 8)()
        _check(lib().ttns_node_info(self.h, k, v, C.byref(nl), dims, None))
        shape = tuple(dims[i] for i in range(nl.value))
        n = int(np.prod(shape))
        out = np.zeros(2 * n)
        _check(lib().ttns_get_node(self.h, k, v, _dptr(out), n))
        return out.view(np.complex128).reshape(shape)

    def save(self, path: str) -> None:
        _check(lib().ttns_save(self.h, path.encode()))

    def load_state(self, path: str) -> None:
        _check(lib().ttns_load_state(self.h, path.encode()))

    @classmethod
    def load(cls, path: str, problems, precision: int = TTNS_MIXED, stream: Optional[int] = None,
             **kw) -> "Tree":
        """A new tree set built by ttns_load from a checkpoint file alone (problem, recording
        settings and state come from the file).  `problems` gives the binding its host-side
        shapes (electronic states and chain lengths) only."""
        self = cls.__new__(cls)
        probs = [problems] if not isinstance(problems, (list, tuple)) else list(problems)
        self.problems = probs
        self._keep = []
        self._hold = []
        if stream is None:
            stream = current_stream()
        self.opt = _options(probs[0], precision, stream=stream, keep=self._hold, **kw)
        h = C.c_void_p()
        self.h = None
        _check(lib().ttns_load(path.encode(), C.byref(self.opt), C.byref(h)))
        self.h = h
        self.n_trees = len(probs)
        return self
