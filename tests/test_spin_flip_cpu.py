"""The spin-flip symmetry the CASCI solvers use, checked on the oracle's
Hamiltonian (CPU only).

Exchanging the alpha and beta strings of every determinant, (P c)[Ia][Ib] =
c[Ib][Ia], commutes with the determinant-basis Hamiltonian of the oracle, so its
eigenvectors split into P = +1 and P = -1 sectors; the closed-shell
determinants lie in P = +1. The counts of tuple spaces whose lowest state is
odd, quoted for the seeded 8-orbital test system and the Hubbard ring, are
recomputed here.
"""

import itertools
import math

import numpy as np
import pytest

from oracle import fci, mbe as omb
from workloads import hubbard_ring_momentum, random_system


def _swap(ns):
    N = ns * ns
    p = np.empty(N, dtype=np.int64)
    for ia in range(ns):
        for ib in range(ns):
            p[ia * ns + ib] = ib * ns + ia
    return p


@pytest.mark.parametrize("n,k,seed", [(4, 2, 1), (5, 2, 2), (6, 3, 3), (6, 2, 4)])
def test_string_exchange_commutes_with_h(n, k, seed):
    h1, eri, _ = random_system(n, k, seed=seed)
    H = fci.h_dense(h1, eri, k, k)
    p = _swap(math.comb(n, k))
    assert np.abs(H[np.ix_(p, p)] - H).max() < 1e-12


def _lowest_parity(h1, eri, occ, A):
    k = omb.n_active_electrons(occ, A)
    _, he, ea = omb.frozen_core(h1, eri, occ, A)
    w, v = np.linalg.eigh(fci.h_dense(he, ea, k, k))
    ns = math.comb(len(A), k)
    c = v[:, 0].reshape(ns, ns)
    return float(np.vdot(c.ravel(), c.T.ravel())), w[1] - w[0]


def test_odd_ground_states_in_the_seeded_test_system():
    h1, eri, occ = random_system(8, 4, seed=33)
    odd = 0
    total = 0
    for n in range(2, 8):
        for t in itertools.combinations(range(8), n):
            if not omb.keep_tuple(t, [], occ):
                continue
            total += 1
            par, gap = _lowest_parity(h1, eri, occ, t)
            assert gap < 1e-8 or abs(abs(par) - 1.0) < 1e-8
            if gap > 1e-8 and par < 0:
                odd += 1
    assert (odd, total) == (13, 224)


def test_hubbard_tuple_ground_states_are_even():
    h1, eri, occ, _ = hubbard_ring_momentum(10, 1.0, 4.0)
    for n in (2, 3, 4):
        for t in omb.tuples(list(range(10)), [], occ, n, True)[::7]:
            par, gap = _lowest_parity(h1, eri, occ, t)
            if gap > 1e-8:
                assert par > 0.999, t


def test_even_sector_eigenvalue_pins():
    from oracle import fci as f
    h1, eri, occ = random_system(8, 4, seed=33)
    # the odd-ground tuple: the even-sector value is the lowest full eigenvalue
    # whose eigenvector is even, found here by classifying all eigenvectors
    A = [0, 1, 2, 3, 4, 6, 7]
    k = omb.n_active_electrons(occ, A)
    _, he, ea = omb.frozen_core(h1, eri, occ, A)
    H = fci.h_dense(he, ea, k, k)
    w, v = np.linalg.eigh(H)
    ns = math.comb(len(A), k)
    par = [float(np.vdot(v[:, i], v[:, i].reshape(ns, ns).T.ravel())) for i in range(len(w))]
    first_even = next(w[i] for i in range(len(w)) if par[i] > 0.5)
    assert abs(f.lowest_eigenvalue_even(he, ea, k) - first_even) < 1e-12
    assert f.lowest_eigenvalue_even(he, ea, k) > w[0] + 1e-3
    # the basis: orthonormal, spans exactly the even vectors (dimension Ns(Ns+1)/2)
    for n, ne in ((4, 2), (6, 3), (5, 1)):
        Q = f.even_sector_basis(n, ne).toarray()
        nsn = math.comb(n, ne)
        assert Q.shape == (nsn * nsn, nsn * (nsn + 1) // 2)
        assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() < 1e-15
        p = _swap(nsn)
        assert np.abs(Q[p] - Q).max() < 1e-15
    # an even-ground space: both readings agree (dense and sparse paths)
    h1, eri, occ, _ = hubbard_ring_momentum(8, 1.0, 4.0)
    for A in ([0, 1, 2, 3, 4, 5], list(range(8))):
        k = omb.n_active_electrons(occ, A)
        _, he, ea = omb.frozen_core(h1, eri, occ, A)
        assert abs(f.lowest_eigenvalue_even(he, ea, k) - f.lowest_eigenvalue(he, ea, k, k)) < 1e-9
