"""Type-1 and Type-2 expansions (Sec. 1, Fig. 1): the host-side choice of the
reference and expansion spaces, and the oracle on those spaces pinned against
facts outside it.

* Type-1 puts every virtual orbital in the reference space and expands in the
  occupied ones: an order-k tuple correlates 2k electrons.  Type-2 puts every
  occupied orbital (plus optional active virtuals) in the reference space and
  expands in the virtuals: every tuple correlates all electrons.
* Pins: a reference space of only virtuals, or of only occupied orbitals, has a
  single determinant, so E_ref,corr = 0; every tuple energy equals the full-space
  Hamiltonian (built from fermion operator matrices) restricted to the
  determinants with the core filled and the deleted orbitals empty; an order-1
  Type-1 tuple is a two-electron problem whose opposite-spin sector is the
  tensor product of the orbital spaces (first quantisation, no strings); the
  full-order expansion equals FCI.
"""

import math

import numpy as np
import pytest

from fock_space import sector_matrix
from oracle import fci, mbe
from paper_1910_03527_gb300.binding import expansion_spaces
from workloads import hubbard_ring_momentum, random_system


def test_expansion_spaces_follow_the_three_definitions():
    occ = [1, 1, 1, 0, 0, 0, 0]
    assert expansion_spaces(occ, "type1") == ([3, 4, 5, 6], [0, 1, 2])
    assert expansion_spaces(occ, "type2") == ([0, 1, 2], [3, 4, 5, 6])
    assert expansion_spaces(occ, "type2", active=[5, 3]) == ([0, 1, 2, 3, 5], [4, 6])
    assert expansion_spaces(occ, "type3") == ([], [0, 1, 2, 3, 4, 5, 6])
    assert expansion_spaces(occ, "type3", active=[3, 2]) == ([2, 3], [0, 1, 4, 5, 6])
    # occupation need not be a leading block
    assert expansion_spaces([0, 1, 0, 1], "type1") == ([0, 2], [1, 3])
    assert expansion_spaces([0, 1, 0, 1], "type2") == ([1, 3], [0, 2])
    for kind, active in (("type4", ()), ("type1", (4,)), ("type2", (1,)), ("type3", (7,)),
                         ("type3", (2, 2)), ("type2", (-1,))):
        with pytest.raises(ValueError):
            expansion_spaces(occ, kind, active)


@pytest.mark.parametrize("seed", [1, 2])
def test_pure_reference_spaces_carry_no_correlation(seed):
    h, eri, occ = random_system(7, 3, seed=seed)
    for kind in ("type1", "type2"):
        ref, _ = expansion_spaces(occ, kind)
        assert abs(mbe.ref_corr_energy(h, eri, occ, ref)) < 1e-12


def test_electrons_and_tuple_counts_per_order():
    occ = np.array([1] * 4 + [0] * 5, dtype=np.uint8)
    r1, x1 = expansion_spaces(occ, "type1")
    r2, x2 = expansion_spaces(occ, "type2")
    for k in range(1, 5):
        t1 = mbe.tuples(x1, r1, occ, k, True)
        assert len(t1) == math.comb(4, k)
        # n_active_electrons counts one spin; both spins give the electrons correlated
        assert all(2 * mbe.n_active_electrons(occ, sorted(r1 + list(t))) == 2 * k for t in t1)
        assert len(t1) == mbe.tuple_count_closed_form(4, 0, False, True, k, True)
    for k in range(1, 6):
        t2 = mbe.tuples(x2, r2, occ, k, True)
        assert len(t2) == math.comb(5, k)
        assert all(2 * mbe.n_active_electrons(occ, sorted(r2 + list(t))) == 8 for t in t2)
        assert len(t2) == mbe.tuple_count_closed_form(0, 5, True, False, k, True)


@pytest.mark.parametrize("kind,seed", [("type1", 3), ("type2", 4), ("type2a", 5)])
def test_tuple_energies_equal_restricted_full_space_fci(kind, seed):
    n, nocc = 5, 2
    h, eri, occ = random_system(n, nocc, seed=seed)
    ref, exp = (expansion_spaces(occ, "type2", active=[4]) if kind == "type2a"
                else expansion_spaces(occ, kind))
    e_phi = mbe.phi_energy(h, eri, occ)
    e_ref = mbe.ref_corr_energy(h, eri, occ, ref)
    if kind == "type2a":
        Hs, _ = sector_matrix(h, eri, nocc, nocc, must_empty=[p for p in range(n) if p not in ref])
        assert abs(e_ref - (np.linalg.eigvalsh(Hs)[0] - e_phi)) < 1e-11
    for k in range(1, len(exp) + 1):
        for t in mbe.tuples(exp, ref, occ, k, True):
            A = set(ref) | set(t)
            core = [p for p in range(n) if occ[p] and p not in A]
            deleted = [p for p in range(n) if not occ[p] and p not in A]
            Hs, _ = sector_matrix(h, eri, nocc, nocc, must_occ=core, must_empty=deleted)
            exact = np.linalg.eigvalsh(Hs)[0] - e_phi - e_ref
            assert abs(mbe.tuple_energy(h, eri, occ, ref, t, e_phi, e_ref) - exact) < 1e-11, t


def test_type1_order1_is_a_two_electron_tensor_product_problem():
    # One alpha and one beta electron: |p_a q_b> <-> phi_p(1) phi_q(2), and H acts as
    # h x 1 + 1 x h + V with V[(p'q'),(pq)] = (p'p|q'q) on the n^2 product space.
    n, nocc = 10, 3
    h, eri, occ = random_system(n, nocc, seed=6)
    ref, exp = expansion_spaces(occ, "type1")
    e_phi = mbe.phi_energy(h, eri, occ)
    for i in exp:
        A = sorted(ref + [i])
        e_core, h_a, eri_a = mbe.frozen_core(h, eri, occ, A)
        m = len(A)
        one = np.eye(m)
        H2 = np.kron(h_a, one) + np.kron(one, h_a) + eri_a.transpose(0, 2, 1, 3).reshape(m * m, m * m)
        exact = np.linalg.eigvalsh(H2)[0] + e_core - e_phi
        assert abs(mbe.tuple_energy(h, eri, occ, ref, (i,), e_phi, 0.0) - exact) < 1e-11


@pytest.mark.parametrize("kind", ["type1", "type2", "type2a"])
def test_full_order_expansion_equals_fci(kind):
    h, eri, occ = random_system(7, 3, seed=7)
    ref, exp = (expansion_spaces(occ, "type2", active=[3]) if kind == "type2a"
                else expansion_spaces(occ, kind))
    res = mbe.run_mbe(h, eri, occ, ref, exp, list(range(1, len(exp) + 1)), skip=True)
    assert abs(res["e_tot"] - fci.lowest_eigenvalue(h, eri, 3, 3)) < 1e-9
    # truncated one order short of full, the expansion is not exact
    short = sum(res["e_order"][k] for k in range(1, len(exp)))
    assert abs(res["e_phi"] + res["e_ref_corr"] + short - res["e_tot"]) > 1e-8


def test_hubbard_type1_and_type2_reach_fci():
    # momentum basis: both inversions of the expansion recover the ring's FCI energy
    h, eri, occ, _ = hubbard_ring_momentum(6, 1.0, 2.0)
    fci_e = fci.lowest_eigenvalue(h, eri, 3, 3)
    for kind in ("type1", "type2"):
        ref, exp = expansion_spaces(occ, kind)
        res = mbe.run_mbe(h, eri, occ, ref, exp, list(range(1, 4)), skip=True)
        assert abs(res["e_tot"] - fci_e) < 1e-9
        assert all(len(t) <= 3 for t in res["inc"])
        assert len(res["inc"]) == sum(math.comb(3, k) for k in range(1, 4))


def test_decoupled_blocks_cas_energy_is_the_sum_over_blocks():
    # The reading the large-active-space GPU test takes its expected values from:
    # with h and (pq|rs) zero across two blocks (and a gap that keeps each block's
    # electron count), E_CAS(A) - E_Phi is the sum over the blocks of the CASCI of
    # A's part in that block, the other block frozen.
    from workloads import block_decoupled_system

    h, eri, occ, block = block_decoupled_system(4, 2, 4, 2, seed=8)
    e_phi = mbe.phi_energy(h, eri, occ)
    ref, exp = expansion_spaces(occ, "type2", active=[4, 5])
    for A in (ref, sorted(ref + [6]), sorted(ref + [7]), list(range(8))):
        direct = mbe.casci_energy(h, eri, occ, A) - e_phi
        split = sum(mbe.casci_energy(h, eri, occ, [p for p in A if block[p] == b]) - e_phi for b in (0, 1))
        assert abs(direct - split) < 1e-10


@pytest.mark.parametrize("L,U", [(6, 2.0), (10, 4.0)])
def test_particle_hole_symmetry_makes_type1_equal_type2_on_the_half_filled_ring(L, U):
    # An even ring is bipartite, so at half filling the particle-hole map (which
    # sends the momentum orbital k to k + pi, occupied to virtual) is a symmetry of
    # H: the Type-1 and Type-2 expansions are mirror images and agree at every
    # truncation order.
    h, eri, occ, _ = hubbard_ring_momentum(L, 1.0, U)
    for kmax in (1, 2):
        e = [mbe.run_mbe(h, eri, occ, *expansion_spaces(occ, kind), list(range(1, kmax + 1)), True)["e_tot"]
             for kind in ("type1", "type2")]
        assert abs(e[0] - e[1]) < 1e-12


def test_run_mbe_routes_large_active_spaces():
    # host-side choice between casci_batch and casci_batch_routed (no GPU: a fake
    # context records which entry point each order would call)
    from paper_1910_03527_gb300.binding import _order_casci

    class Fake:
        def __init__(self):
            self.calls = []

        def casci_batch(self, h1, eri, occ, ref, e_ref, order, tup, opts):
            self.calls.append(("batch", len(ref) + order))

        def casci_batch_routed(self, h1, eri, occ, ref, e_ref, order, tup, opts, large_ndet):
            self.calls.append(("routed", len(ref) + order, large_ndet))

    f = Fake()
    ref = list(range(11))
    for order in (0, 1, 2, 5):
        _order_casci(f, None, None, None, ref, 0.0, order, None, None, None)
    _order_casci(f, None, None, None, ref[:4], 0.0, 2, None, None, 5000)
    assert f.calls == [("batch", 11), ("batch", 12), ("routed", 13, 0), ("routed", 16, 0),
                       ("routed", 6, 5000)]
