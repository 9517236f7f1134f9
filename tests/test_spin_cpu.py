"""Pins of the oracle's total-spin operator S^2 and of its spin-targeted energies.

State targeting (the paper converges its Cr2 expansion onto the 1Sigma_g+
ground state) rests on oracle.fci.s2_dense and lowest_eigenvalue_spin.  They are
pinned against things other than themselves:
  * S^2 built from Jordan-Wigner fermion matrices (tests/fock_space.py), which
    involves no sign bookkeeping, element by element, also for n_alpha != n_beta;
  * the spectrum: S(S+1) with the multiplicities of Weyl's dimension formula for
    N electrons in n spatial orbitals (one M_S = 0 state per spin multiplet);
  * [H, S^2] = 0 for the oracle's Hamiltonian with random integrals;
  * two electrons in two orbitals: the triplet energy in closed form, and the
    singlet ground state from the textbook 3x3 singlet block.
"""

import math

import numpy as np
import pytest

from fock_space import annihilators, sector_words
from oracle import fci
from workloads import random_system


def weyl_dimension(n: int, ne_total: int, spin: int) -> int:
    """Number of spin-`spin` multiplets of ne_total electrons in n spatial orbitals."""
    half = ne_total // 2
    if half - spin < 0:
        return 0
    return (2 * spin + 1) * math.comb(n + 1, half - spin) * math.comb(n + 1, half + spin + 1) // (n + 1)


@pytest.mark.parametrize("n,ne", [(2, 1), (3, 1), (4, 2), (5, 2), (6, 3), (5, 3)])
def test_s2_spectrum_is_weyl(n, ne):
    w = np.linalg.eigvalsh(fci.s2_dense(n, ne, ne))
    total = 0
    for spin in range(ne + 1):
        mult = int(np.sum(np.abs(w - spin * (spin + 1)) < 1e-9))
        assert mult == weyl_dimension(n, 2 * ne, spin), (n, ne, spin)
        total += mult
    assert total == len(w)


@pytest.mark.parametrize("n,na,nb", [(3, 1, 1), (4, 2, 2), (4, 2, 1), (3, 2, 1)])
def test_s2_equals_jordan_wigner(n, na, nb):
    a = annihilators(2 * n)
    ad = [x.T for x in a]
    dim = 2 ** (2 * n)
    import scipy.sparse as sp
    Sp = sp.csr_matrix((dim, dim))
    Sm = sp.csr_matrix((dim, dim))
    Sz = sp.csr_matrix((dim, dim))
    for p in range(n):
        Sp = Sp + ad[p] @ a[n + p]
        Sm = Sm + ad[n + p] @ a[p]
        Sz = Sz + 0.5 * (ad[p] @ a[p] - ad[n + p] @ a[n + p])
    S2 = (Sm @ Sp + Sz @ Sz + Sz).tocsr()
    w = sector_words(n, na, nb)
    want = S2[w][:, w].toarray()
    got = fci.s2_dense(n, na, nb)
    np.testing.assert_allclose(got, want, atol=1e-14)


@pytest.mark.parametrize("n,ne,seed", [(4, 2, 1), (5, 2, 2), (5, 3, 3)])
def test_s2_commutes_with_hamiltonian(n, ne, seed):
    h, eri, _ = random_system(n, ne, seed=seed)
    H = fci.h_dense(h, eri, ne, ne)
    S2 = fci.s2_dense(n, ne, ne)
    assert np.abs(H @ S2 - S2 @ H).max() <= 1e-12 * np.abs(H).max()


def test_two_electrons_singlet_and_triplet_closed_forms():
    h, eri, _ = random_system(2, 1, seed=7)
    g = lambda p, q, r, s: eri[p, q, r, s]
    triplet = h[0, 0] + h[1, 1] + g(0, 0, 1, 1) - g(0, 1, 1, 0)
    a = math.sqrt(2.0) * (h[0, 1] + g(0, 0, 0, 1))
    b = math.sqrt(2.0) * (h[0, 1] + g(1, 1, 0, 1))
    S = np.array([[2 * h[0, 0] + g(0, 0, 0, 0), a, g(0, 1, 0, 1)],
                  [a, h[0, 0] + h[1, 1] + g(0, 0, 1, 1) + g(0, 1, 1, 0), b],
                  [g(0, 1, 0, 1), b, 2 * h[1, 1] + g(1, 1, 1, 1)]])
    assert abs(fci.lowest_eigenvalue_spin(h, eri, 1, 1.0) - triplet) < 1e-12
    assert abs(fci.lowest_eigenvalue_spin(h, eri, 1, 0.0) - np.linalg.eigvalsh(S)[0]) < 1e-12


def test_singlet_energy_ignores_a_lower_triplet():
    """Tuple spaces of the seeded 8-orbital test system whose ground state is a
    triplet (S^2 = 2, found by brute force): the spin-0 energy lies above the
    lowest eigenvalue and equals the lowest eigenvalue among the eigenvectors of
    H with S^2 = 0."""
    from oracle import mbe as omb
    h1, eri, occ = random_system(8, 4, seed=33)
    for A in ((2, 3, 4), (0, 2, 3, 4), (2, 3, 4, 5), (2, 3, 4, 5, 7)):
        k = omb.n_active_electrons(occ, list(A))
        _, he, ea = omb.frozen_core(h1, eri, occ, list(A))
        H = fci.h_dense(he, ea, k, k)
        S2 = fci.s2_dense(len(A), k, k)
        w, v = np.linalg.eigh(H)
        spins = np.einsum("di,de,ei->i", v, S2, v)
        assert abs(spins[0] - 2.0) < 1e-8, A
        e0 = fci.lowest_eigenvalue_spin(he, ea, k, 0.0)
        assert e0 > w[0] + 1e-3
        assert abs(e0 - w[np.abs(spins) < 1e-8].min()) < 1e-10
