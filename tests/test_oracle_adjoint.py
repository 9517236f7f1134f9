"""Pins for the oracle adjoint: finite differences, energy from density matrices,
homogeneity of the Hubbard energy, electron count, and the transposed recursion."""

import itertools
import math

import numpy as np
import pytest

from oracle import adjoint, fci, mbe as omb
from workloads import hubbard_ring_momentum, random_system


def _sym_orbit(p, q, r, s):
    """The 8-fold permutational symmetry orbit of (pq|rs)."""
    return {(p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r),
            (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)}


@pytest.mark.parametrize("A,seed", [((1, 2, 3), 1), ((0, 2, 4), 2), ((0, 1, 2, 3, 4), 3), ((), 4)])
def test_cas_gradient_reproduces_energy_and_electron_count(A, seed):
    h1, eri, occ = random_system(5, 3, seed=seed)
    e, g, G = adjoint.cas_gradient(h1, eri, occ, A)
    assert abs(np.einsum("pq,pq", h1, g) + np.einsum("pqrs,pqrs", eri, G) - e) < 1e-11
    assert abs(np.trace(g) - 2 * occ.sum()) < 1e-12
    if len(A) == 0:
        assert abs(e - omb.phi_energy(h1, eri, occ)) < 1e-13


@pytest.mark.parametrize("A", [(1, 2, 3), (0, 3, 4)])
def test_cas_gradient_matches_finite_differences(A):
    h1, eri, occ = random_system(5, 3, seed=8)
    _, g, G = adjoint.cas_gradient(h1, eri, occ, A)
    d = 1e-5
    rng = np.random.default_rng(0)
    for _ in range(6):
        p, q = rng.integers(0, 5, size=2)
        hp, hm = h1.copy(), h1.copy()
        for (a, b) in {(p, q), (q, p)}:
            hp[a, b] += d
            hm[a, b] -= d
        fd = (omb.casci_energy(hp, eri, occ, A) - omb.casci_energy(hm, eri, occ, A)) / (2 * d)
        want = g[p, q] + (g[q, p] if p != q else 0.0)
        assert abs(fd - want) < 1e-7, (p, q, fd, want)
    for _ in range(6):
        idx = tuple(int(x) for x in rng.integers(0, 5, size=4))
        orbit = _sym_orbit(*idx)
        ep, em = eri.copy(), eri.copy()
        for o in orbit:
            ep[o] += d
            em[o] -= d
        fd = (omb.casci_energy(h1, ep, occ, A) - omb.casci_energy(h1, em, occ, A)) / (2 * d)
        want = sum(G[o] for o in orbit)
        assert abs(fd - want) < 1e-7, (idx, fd, want)


def test_mbe_gradient_matches_finite_differences():
    h1, eri, occ = random_system(6, 3, seed=12)
    ref, exp, orders = [2, 3], [0, 1, 4, 5], [1, 2, 3]
    E, gh, ge = adjoint.mbe_gradient(h1, eri, occ, ref, exp, orders, skip=False)
    assert abs(E - omb.run_mbe(h1, eri, occ, ref, exp, orders, False)["e_tot"]) < 1e-10
    d = 1e-5
    rng = np.random.default_rng(1)

    def energy(h, e):
        return omb.run_mbe(h, e, occ, ref, exp, orders, False)["e_tot"]

    for _ in range(4):
        p, q = (int(x) for x in rng.integers(0, 6, size=2))
        hp, hm = h1.copy(), h1.copy()
        for (a, b) in {(p, q), (q, p)}:
            hp[a, b] += d
            hm[a, b] -= d
        fd = (energy(hp, eri) - energy(hm, eri)) / (2 * d)
        want = gh[p, q] + (gh[q, p] if p != q else 0.0)
        assert abs(fd - want) < 1e-6 * max(1.0, abs(want)), (p, q, fd, want)
    for _ in range(4):
        idx = tuple(int(x) for x in rng.integers(0, 6, size=4))
        orbit = _sym_orbit(*idx)
        ep, em = eri.copy(), eri.copy()
        for o in orbit:
            ep[o] += d
            em[o] -= d
        fd = (energy(h1, ep) - energy(h1, em)) / (2 * d)
        want = sum(ge[o] for o in orbit)
        assert abs(fd - want) < 1e-6 * max(1.0, abs(want)), (idx, fd, want)


def test_hubbard_homogeneity_and_fd_in_t_and_u():
    L, t, U = 6, 1.0, 3.0
    h1, eri, occ, _ = hubbard_ring_momentum(L, t, U)
    orders = [1, 2, 3]
    E, gh, ge = adjoint.mbe_gradient(h1, eri, occ, [], list(range(L)), orders, skip=True)
    dEdt = float(np.sum(gh * h1)) / t
    dEdU = float(np.sum(ge * eri)) / U
    assert abs(t * dEdt + U * dEdU - E) < 1e-10
    assert abs(np.trace(gh) - L) < 1e-10
    d = 1e-4

    def energy(tt, uu):
        a, b, o, _ = hubbard_ring_momentum(L, tt, uu)
        return omb.run_mbe(a, b, o, [], list(range(L)), orders, True)["e_tot"]

    assert abs((energy(t + d, U) - energy(t - d, U)) / (2 * d) - dEdt) < 1e-6
    assert abs((energy(t, U + d) - energy(t, U - d)) / (2 * d) - dEdU) < 1e-6


def test_transposed_recursion_weights():
    # E_MBE - E_CAS(R) = sum_S w(S) eps(S) for arbitrary eps, with skipped tuples absent.
    occ = np.array([1, 1, 1, 0, 0, 0], dtype=np.uint8)
    orders = [1, 2, 3, 4]
    tup = {n: omb.tuples(list(range(6)), [], occ, n, True) for n in orders}
    w = adjoint.adjoint_weights(tup)
    rng = np.random.default_rng(3)
    eps = {n: {t: float(rng.normal()) for t in tup[n]} for n in orders}
    inc = omb.increments(eps)
    lhs = math.fsum(inc.values())
    rhs = math.fsum(w[t] * eps[n][t] for n in orders for t in tup[n])
    assert abs(lhs - rhs) < 1e-12
    # with no skipping and all orders up to m, w(S) = sum_j (-1)^j C(M-|S|, j)
    full = {n: list(itertools.combinations(range(5), n)) for n in (1, 2, 3)}
    wf = adjoint.adjoint_weights(full)
    for S, v in wf.items():
        want = sum((-1) ** j * math.comb(5 - len(S), j) for j in range(0, 3 - len(S) + 1))
        assert v == want
