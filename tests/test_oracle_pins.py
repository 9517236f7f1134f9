"""Pins for the oracle: facts fixed by the mathematics or by the paper, not by the oracle.

Each test ties an oracle function to something outside it:
* string enumeration and addressing  -> combinatorial number system, brute force;
* Slater-Condon matrix elements       -> Fock-space Hamiltonian from fermion
                                         operator matrices (tests/fock_space.py);
* CASCI lowest eigenvalue             -> Hubbard dimer closed form, U = 0 band
                                         filling, two-electron/two-orbital
                                         textbook blocks, dense vs sparse solvers;
* frozen core / effective Hamiltonian -> full-space FCI restricted to the
                                         determinants with the core filled;
* tuple enumeration                   -> closed-form counts, itertools brute force;
* increment recursion (Eq. 2)         -> Moebius inversion on the subset lattice,
                                         full-order MBE == FCI, decoupled blocks,
                                         vanishing occupied-only / virtual-only tuples.
"""

import itertools
import math
import os

import numpy as np
import pytest

from fock_space import annihilators, hamiltonian, sector_matrix, sector_words
from oracle import fci, mbe
from workloads import (block_decoupled_system, hubbard_open_dimer, hubbard_ring_momentum,
                       random_system, workload)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- strings

@pytest.mark.parametrize("n,k", [(1, 0), (1, 1), (4, 2), (6, 3), (7, 2), (8, 4), (10, 5)])
def test_strings_are_all_k_subsets_ascending(n, k):
    s = fci.strings(n, k)
    brute = sorted(sum(1 << c for c in comb) for comb in itertools.combinations(range(n), k))
    assert s.tolist() == brute
    assert len(s) == math.comb(n, k)


@pytest.mark.parametrize("n,k", [(6, 3), (8, 4), (10, 3), (12, 6)])
def test_string_rank_is_combinatorial_number_system(n, k):
    # rank of the string with set bits c_1 < ... < c_k is sum_i C(c_i, i)
    s = fci.strings(n, k)
    for idx, w in enumerate(s.tolist()):
        bits = [b for b in range(n) if (w >> b) & 1]
        assert sum(math.comb(c, i + 1) for i, c in enumerate(bits)) == idx


def test_paper_determinant_counts():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "paper_det_counts.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 2
    for r in rows:
        printed, digits, n, k = float(r[1]), int(r[2]), int(r[3]), int(r[4])
        ndet = fci.binom(n, k) ** 2
        assert float(f"{ndet:.{digits - 1}e}") == printed
        assert len(fci.dets(n, k, k)) == ndet if n <= 12 else True


# ----------------------------------------------------------------------------- operators

def test_fock_operators_satisfy_car():
    a = annihilators(6)
    eye = np.eye(64)
    for i in range(6):
        for j in range(6):
            assert np.allclose((a[i] @ a[j].T + a[j].T @ a[i]).toarray(), eye * (i == j))
            assert np.allclose((a[i] @ a[j] + a[j] @ a[i]).toarray(), 0.0)


@pytest.mark.parametrize("n,na,nb,seed", [(2, 1, 1, 0), (3, 1, 2, 1), (3, 2, 1, 2), (4, 2, 2, 3),
                                          (4, 1, 3, 4), (4, 3, 3, 5), (5, 2, 2, 6)])
def test_slater_condon_matrix_equals_fock_space(n, na, nb, seed):
    h, eri, _ = random_system(n, na, seed=seed)
    H_ref, words = sector_matrix(h, eri, na, nb)
    assert fci.dets(n, na, nb).tolist() == words
    H = fci.h_dense(h, eri, na, nb)
    np.testing.assert_allclose(H, H_ref, atol=1e-12, rtol=0)


def test_sigma_and_diagonal_match_dense():
    h, eri, _ = random_system(6, 3, seed=11)
    H = fci.h_dense(h, eri, 3, 2)
    c = np.random.default_rng(0).normal(size=H.shape[0])
    np.testing.assert_allclose(fci.sigma(h, eri, 3, 2, c), H @ c, atol=1e-12)
    np.testing.assert_allclose(fci.hdiag(h, eri, 3, 2), np.diag(H), atol=1e-13)
    assert np.allclose(H, H.T, atol=1e-14)


# sigma_rows is the only checker of the GPU sigma above 50k determinants, so it is
# pinned here twice: against H c from the Fock-space Hamiltonian (fermion operator
# matrices, no Slater-Condon case analysis, no determinant addressing of the oracle),
# and against the column-driven oracle sigma on larger sectors.  Sectors include
# na != nb, empty and full spin strings, and every row as well as random subsets
# (a wrong row-to-determinant mapping or a dropped connection class fails).
@pytest.mark.parametrize("n,na,nb,seed", [(2, 1, 1, 0), (3, 1, 2, 1), (4, 2, 2, 2), (4, 0, 2, 3),
                                          (4, 4, 1, 4), (5, 2, 3, 5), (5, 3, 3, 6), (5, 5, 0, 7)])
def test_sigma_rows_equals_fock_space_h_times_c(n, na, nb, seed):
    h, eri, _ = random_system(n, max(na, nb), seed=seed)
    H_ref, words = sector_matrix(h, eri, na, nb)
    c = np.random.default_rng(seed).normal(size=len(words))
    want = H_ref @ c
    rows = np.arange(len(words))
    got = fci.sigma_rows(h, eri, na, nb, c, rows)
    np.testing.assert_allclose(got, want, atol=1e-12 * max(1.0, np.abs(want).max()), rtol=0)
    sub = np.random.default_rng(seed + 100).permutation(len(words))[: max(1, len(words) // 3)]
    got_sub = fci.sigma_rows(h, eri, na, nb, c, sub)
    np.testing.assert_allclose(got_sub, want[sub], atol=1e-12 * max(1.0, np.abs(want).max()), rtol=0)


@pytest.mark.parametrize("n,na,nb,seed", [(6, 3, 3, 11), (7, 2, 4, 12), (8, 4, 4, 13), (8, 1, 7, 14),
                                          (8, 3, 2, 15)])
def test_sigma_rows_equals_oracle_sigma(n, na, nb, seed):
    h, eri, _ = random_system(n, max(na, nb), seed=seed)
    N = fci.binom(n, na) * fci.binom(n, nb)
    c = np.random.default_rng(seed).normal(size=N)
    want = fci.sigma(h, eri, na, nb, c)
    got = fci.sigma_rows(h, eri, na, nb, c, np.arange(N))
    scale = np.abs(want).max()
    np.testing.assert_allclose(got, want, atol=1e-12 * scale, rtol=0)
    rows = np.random.default_rng(seed + 1).choice(N, size=min(N, 97), replace=False)
    np.testing.assert_allclose(fci.sigma_rows(h, eri, na, nb, c, rows), want[rows], atol=1e-12 * scale,
                               rtol=0)
    # a single unit vector: column j of H, against the dense Slater-Condon matrix of another route
    if N <= 1500:
        H = fci.h_dense(h, eri, na, nb)
        j = int(np.argmax(np.abs(c)))
        e = np.zeros(N)
        e[j] = 1.0
        np.testing.assert_allclose(fci.sigma_rows(h, eri, na, nb, e, np.arange(N)), H[:, j], atol=1e-13,
                                   rtol=0)


# ----------------------------------------------------------------------------- closed forms

@pytest.mark.parametrize("t,U", [(1.0, 0.0), (1.0, 2.0), (1.0, 4.0), (0.5, 3.0), (2.0, 1.0)])
def test_hubbard_dimer_closed_form(t, U):
    h, eri, _ = hubbard_open_dimer(t, U)
    e = fci.lowest_eigenvalue(h, eri, 1, 1)
    assert abs(e - (U - math.sqrt(U * U + 16 * t * t)) / 2) < 1e-12


@pytest.mark.parametrize("L", [4, 6, 8])
def test_hubbard_u0_is_band_filling(L):
    h, eri, occ, _ = hubbard_ring_momentum(L, 1.0, 0.0)
    levels = sorted(-2.0 * math.cos(2 * math.pi * k / L) for k in range(L))
    exact = 2.0 * sum(levels[: L // 2])
    e = fci.lowest_eigenvalue(h, eri, L // 2, L // 2)
    assert abs(e - exact) < 1e-10
    assert abs(mbe.phi_energy(h, eri, occ) - exact) < 1e-12


def test_two_electrons_in_two_orbitals_textbook_blocks():
    h, eri, _ = random_system(2, 1, seed=7)
    H = fci.h_dense(h, eri, 1, 1)
    w = np.linalg.eigvalsh(H)
    g = lambda p, q, r, s: eri[p, q, r, s]
    triplet = h[0, 0] + h[1, 1] + g(0, 0, 1, 1) - g(0, 1, 1, 0)
    a = math.sqrt(2.0) * (h[0, 1] + g(0, 0, 0, 1))
    b = math.sqrt(2.0) * (h[0, 1] + g(1, 1, 0, 1))
    S = np.array([[2 * h[0, 0] + g(0, 0, 0, 0), a, g(0, 1, 0, 1)],
                  [a, h[0, 0] + h[1, 1] + g(0, 0, 1, 1) + g(0, 1, 1, 0), b],
                  [g(0, 1, 0, 1), b, 2 * h[1, 1] + g(1, 1, 1, 1)]])
    expect = np.sort(np.concatenate([np.linalg.eigvalsh(S), [triplet]]))
    np.testing.assert_allclose(w, expect, atol=1e-12)


def test_dense_and_sparse_eigensolvers_agree(monkeypatch):
    h, eri, _ = random_system(8, 3, seed=5)
    e_dense = fci.lowest_eigenvalue(h, eri, 3, 3)  # 3136 dets -> sparse path by default
    monkeypatch.setattr(fci, "DENSE_MAX", 10 ** 6)
    e_full = fci.lowest_eigenvalue(h, eri, 3, 3)
    monkeypatch.setattr(fci, "DENSE_MAX", 10)
    monkeypatch.setattr(fci, "SPARSE_MAX_ENTRIES", 0)
    e_op = fci.lowest_eigenvalue(h, eri, 3, 3)
    assert abs(e_dense - e_full) < 1e-10 and abs(e_op - e_full) < 1e-10


# ----------------------------------------------------------------------------- frozen core

@pytest.mark.parametrize("A,seed", [((1, 2, 3), 1), ((0, 3, 4), 2), ((2, 4), 3), ((1, 3), 4),
                                    ((0, 1, 2, 3, 4), 5)])
def test_frozen_core_casci_equals_restricted_full_space_fci(A, seed):
    n, nocc = 5, 3
    h, eri, occ = random_system(n, nocc, seed=seed)
    core = [c for c in range(n) if occ[c] and c not in A]
    deleted = [v for v in range(n) if not occ[v] and v not in A]
    ne = nocc  # all electrons, core ones included
    Hs, _ = sector_matrix(h, eri, ne, ne, must_occ=core, must_empty=deleted)
    exact = np.linalg.eigvalsh(Hs)[0]
    assert abs(mbe.casci_energy(h, eri, occ, A) - exact) < 1e-11


def test_phi_energy_is_fock_space_expectation():
    h, eri, occ = random_system(4, 2, seed=9)
    H = hamiltonian(h, eri)
    w = 0b0011 | (0b0011 << 4)
    assert abs(H[w, w] - mbe.phi_energy(h, eri, occ)) < 1e-12


# ----------------------------------------------------------------------------- tuples

def test_tuple_enumeration_is_lexicographic_and_filtered():
    occ = np.array([1, 1, 1, 0, 0, 0, 0], dtype=np.uint8)
    exp = list(range(7))
    for n in range(1, 8):
        got = mbe.tuples(exp, [], occ, n, skip=True)
        brute = [t for t in itertools.combinations(exp, n)
                 if any(occ[p] for p in t) and not all(occ[p] for p in t)]
        assert got == brute
        assert len(got) == mbe.tuple_count_closed_form(3, 4, False, False, n, True)


@pytest.mark.parametrize("name,counts", [
    ("hubbard8", [8, 28, 56, 70, 56, 28, 8, 1]),
    ("hubbard22", [0, 121, 1210, 6655, 25410, 73689]),
    ("molecule40", [34, 561, 5984, 46376]),
    ("hubbard46", [0, 529, 11638, 145475]),
])
def test_workload_tuple_counts(name, counts):
    w = workload(name)
    m_occ = int(sum(w.occ[p] for p in w.exp))
    m_vir = len(w.exp) - m_occ
    r_occ = any(w.occ[p] for p in w.ref)
    r_vir = any(not w.occ[p] for p in w.ref)
    closed = [mbe.tuple_count_closed_form(m_occ, m_vir, r_occ, r_vir, n, w.skip) for n in w.orders]
    assert closed == counts
    for n in w.orders:
        if math.comb(len(w.exp), n) <= 100_000:
            assert len(mbe.tuples(w.exp, w.ref, w.occ, n, w.skip)) == counts[n - 1]


# ----------------------------------------------------------------------------- recursion

def test_recursion_moebius_constant_and_additive():
    X = list(range(6))
    eps1 = {n: {t: 1.0 for t in itertools.combinations(X, n)} for n in range(1, 7)}
    inc = mbe.increments(eps1)
    for t, v in inc.items():
        assert v == (-1.0) ** (len(t) + 1)
    f = {p: 0.1 * p - 0.3 for p in X}
    eps2 = {n: {t: sum(f[p] for p in t) for t in itertools.combinations(X, n)}
            for n in range(1, 7)}
    inc = mbe.increments(eps2)
    for t, v in inc.items():
        assert abs(v - (f[t[0]] if len(t) == 1 else 0.0)) < 1e-14


def test_occupied_only_and_virtual_only_tuples_vanish():
    h, eri, occ, _ = hubbard_ring_momentum(6, 1.0, 3.0)
    e_phi = mbe.phi_energy(h, eri, occ)
    for t in [(0,), (1, 2), (0, 1, 2), (3,), (4, 5), (3, 4, 5)]:
        assert abs(mbe.tuple_energy(h, eri, occ, [], t, e_phi, 0.0)) < 1e-12


@pytest.mark.parametrize("L,U", [(4, 4.0), (6, 2.0)])
def test_full_order_mbe_equals_fci_hubbard(L, U):
    h, eri, occ, _ = hubbard_ring_momentum(L, 1.0, U)
    res = mbe.run_mbe(h, eri, occ, [], list(range(L)), list(range(1, L + 1)), skip=False)
    fci_e = fci.lowest_eigenvalue(h, eri, L // 2, L // 2)
    assert abs(res["e_tot"] - fci_e) < 1e-9


def test_full_order_mbe_equals_fci_hubbard8():
    w = workload("hubbard8")
    res = mbe.run_mbe(w.h1, w.eri, w.occ, w.ref, w.exp, w.orders, w.skip)
    fci_e = fci.lowest_eigenvalue(w.h1, w.eri, 4, 4)
    assert abs(res["e_tot"] - fci_e) < 1e-9
    assert len(res["inc"]) == 255


def test_full_order_mbe_equals_fci_with_reference_space():
    h, eri, occ = random_system(6, 3, seed=21)
    ref, exp = [1, 3], [0, 2, 4, 5]
    res = mbe.run_mbe(h, eri, occ, ref, exp, list(range(1, 5)), skip=False)
    fci_e = fci.lowest_eigenvalue(h, eri, 3, 3)
    assert abs(res["e_tot"] - fci_e) < 1e-9
    assert abs(res["e_ref_corr"] - (mbe.casci_energy(h, eri, occ, ref) - res["e_phi"])) < 1e-14


def test_u0_increments_vanish():
    h, eri, occ, _ = hubbard_ring_momentum(6, 1.0, 0.0)
    res = mbe.run_mbe(h, eri, occ, [], list(range(6)), [1, 2, 3], skip=True)
    assert max(abs(v) for v in res["inc"].values()) < 1e-10


def test_decoupled_blocks_cross_increments_vanish():
    h, eri, occ, block = block_decoupled_system(3, 1, 3, 2, seed=4)
    res = mbe.run_mbe(h, eri, occ, [], list(range(6)), [1, 2, 3, 4], skip=True)
    cross = [v for t, v in res["inc"].items() if len({int(block[p]) for p in t}) == 2]
    inner = [v for t, v in res["inc"].items() if len({int(block[p]) for p in t}) == 1]
    assert len(cross) > 20 and max(abs(v) for v in cross) < 1e-10
    assert max(abs(v) for v in inner) > 1e-4
