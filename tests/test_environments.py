"""Weighted k-means grouping of modes into environments (Results, "Interface to TTNS"): the
oracle against what fixes it (a well-separated mixture whose generating groups must come
back, brute force over all partitions of a tiny set, sign invariance), and the library's
host implementation against the oracle bit for bit in the assignments."""
import itertools

import numpy as np
import pytest

from oracle.environments import cluster_modes, features, pattern_and_strength


def _mixture(seed, n_el=4, groups=3, per=8, noise=0.02):
    rng = np.random.default_rng(seed)
    base = []
    for g in range(groups):
        A = rng.normal(size=(n_el, n_el)) + 1j * rng.normal(size=(n_el, n_el))
        A = A + A.conj().T
        base.append(A / np.linalg.norm(A))
    W, labels = [], []
    for g in range(groups):
        for _ in range(per):
            E = rng.normal(size=(n_el, n_el)) + 1j * rng.normal(size=(n_el, n_el))
            E = (E + E.conj().T) * noise
            lam = rng.uniform(0.01, 0.1) * (1 if rng.random() < 0.5 else -1)
            W.append(lam * (base[g] + E))
            labels.append(g)
    order = rng.permutation(len(W))
    return np.array(W)[order], np.array(labels)[order]


def _same_partition(a, b):
    pairs = {}
    for x, y in zip(a, b):
        if pairs.setdefault(x, y) != y:
            return False
    return len(set(pairs.values())) == len(pairs)


def test_well_separated_groups_are_recovered():
    W, labels = _mixture(1, noise=0.005)   # residual per mode ~4% of its norm
    init = [int(np.nonzero(labels == g)[0][0]) for g in range(3)]   # one seed in each group
    assign, Wbar, lam, it = cluster_modes(W, 3, init)
    assert _same_partition(assign, labels) and it < 10
    # the mode's coupling is recovered along its environment's pattern
    for n in range(len(W)):
        approx = lam[n] * Wbar[assign[n]]
        assert np.linalg.norm(W[n] - approx) < 0.1 * np.linalg.norm(W[n])


def test_sign_of_a_mode_does_not_change_its_group():
    W, labels = _mixture(2)
    init = [int(np.nonzero(labels == g)[0][0]) for g in range(3)]
    a1, _, lam1, _ = cluster_modes(W, 3, init)
    W2 = W.copy()
    W2[::3] *= -1
    a2, _, lam2, _ = cluster_modes(W2, 3, init)
    assert np.array_equal(a1, a2)
    np.testing.assert_allclose(np.abs(lam1), np.abs(lam2), rtol=1e-12)


def test_lloyd_reaches_the_brute_force_optimum_on_a_tiny_set():
    W, labels = _mixture(3, groups=2, per=4, noise=0.05)
    pats, lams = zip(*[pattern_and_strength(x) for x in W])
    X = np.array([features(p) for p in pats])
    w = np.array(lams) ** 2

    # the generating patterns are all aligned with the first mode of their group: align
    # every mode by the sign of its overlap with that mode, then cluster plainly
    ref = [X[int(np.nonzero(labels == g)[0][0])] for g in (0, 1)]
    Xa = np.array([x * (1.0 if np.dot(x, ref[labels[n]]) >= 0 else -1.0) for n, x in enumerate(X)])

    def cost(part):
        c = 0.0
        for g in (0, 1):
            m = np.array(part) == g
            if m.any():
                mu = (w[m, None] * Xa[m]).sum(0) / w[m].sum()
                c += float((w[m] * ((Xa[m] - mu) ** 2).sum(1)).sum())
        return c

    best = min(cost(p) for p in itertools.product((0, 1), repeat=len(W)))  # sign-aligned below
    assign, _, _, _ = cluster_modes(W, 2, [0, int(np.nonzero(labels != labels[0])[0][0])])
    assert _same_partition(assign, labels) and cost(assign) <= best + 1e-12


def test_library_matches_the_oracle():
    from paper_1710_01362_gb300 import build, ttns
    build.build()
    for seed in range(4):
        W, labels = _mixture(10 + seed, n_el=5, groups=4, per=10, noise=0.3)
        rng = np.random.default_rng(seed)
        init = list(rng.choice(len(W), size=4, replace=False))
        a_o, Wb_o, lam_o, it_o = cluster_modes(W, 4, init)
        a_l, Wb_l, lam_l, it_l = ttns.cluster_modes(W, 4, init)
        assert np.array_equal(a_o, a_l) and it_o == it_l
        np.testing.assert_allclose(Wb_l, Wb_o, atol=1e-12)
        np.testing.assert_allclose(lam_l, lam_o, atol=1e-12)
