"""Pins for the oracle's screened expansion (Eq. 4 thresholds, child spawning).

Each pin fixes the screening against something other than the oracle's own
code: the complete tuple sets and energies (zero thresholds), an expansion that
must stop (an unreachable threshold), a four-orbital example worked by hand,
Eq. 4 at hand-computed points, monotonicity in the relaxation factor a, and a
second, parent-driven enumeration of the children written here.
"""

import itertools

import numpy as np
import pytest

from oracle import mbe as omb
from workloads import random_system


def test_eq4_thresholds_at_hand_computed_points():
    occ = np.array([1, 1, 1, 1, 0, 0, 0, 0, 0, 0], dtype=np.uint8)
    # the paper's parameters: T_init = 1e-10, M_init = 3, a = 5
    assert omb.tuple_threshold((0, 4), occ, 1e-10, 3, 5.0) == 0.0          # M_tup = 1
    assert omb.tuple_threshold((0, 1, 4, 5), occ, 1e-10, 3, 5.0) == 0.0    # M_tup = 2
    assert omb.tuple_threshold((0, 1, 2, 4), occ, 1e-10, 3, 5.0) == 1e-10  # M_tup = 3 (occupied)
    assert omb.tuple_threshold((0, 4, 5, 6), occ, 1e-10, 3, 5.0) == 1e-10  # M_tup = 3 (virtual)
    assert omb.tuple_threshold((0, 1, 2, 3, 4), occ, 1e-10, 3, 5.0) == pytest.approx(5e-10, rel=1e-15)
    assert omb.tuple_threshold((0, 4, 5, 6, 7, 8), occ, 1e-10, 3, 5.0) == pytest.approx(2.5e-9, rel=1e-15)
    assert omb.tuple_threshold((0, 1, 4, 5, 6, 7, 8, 9), occ, 1e-10, 3, 5.0) == pytest.approx(1.25e-8, rel=1e-15)  # M_tup = 6


def test_hand_worked_four_orbital_example():
    # X = {0, 1, 2, 3}, O = {0, 1}, empty reference, skip rule; order-2 increments by hand
    occ = np.array([1, 1, 0, 0], dtype=np.uint8)
    inc2 = {(0, 2): 1e-3, (0, 3): 0.0, (1, 2): -0.0, (1, 3): -2e-11}
    # every 3-subset holds 2 of one kind and 1 of the other: M_tup = 2, threshold 1e-10 at M_init = 2
    got = omb.spawn([0, 1, 2, 3], [], occ, 2, inc2, True, 1e-10, 2, 10.0)
    # {0,1,2}: |inc(0,2)| = 1e-3 spawns; {0,1,3}: at most 2e-11, no; {0,2,3}: 1e-3, yes;
    # {1,2,3}: at most 2e-11, no
    assert got == [(0, 1, 2), (0, 2, 3)]
    # order 4 from the two spawned triples; {0,1,2,3} has M_tup = 2
    assert omb.spawn([0, 1, 2, 3], [], occ, 3, {(0, 1, 2): 5e-11, (0, 2, 3): -3e-10}, True,
                     1e-10, 2, 10.0) == [(0, 1, 2, 3)]
    assert omb.spawn([0, 1, 2, 3], [], occ, 3, {(0, 1, 2): 5e-11, (0, 2, 3): 5e-11}, True,
                     1e-10, 2, 10.0) == []
    # M_init = 1 raises the order-4 threshold to 1e-10 * 10
    assert omb.spawn([0, 1, 2, 3], [], occ, 3, {(0, 1, 2): 5e-11, (0, 2, 3): -3e-10}, True,
                     1e-10, 1, 10.0) == []
    # without the skip rule the all-virtual and all-occupied children are tested too
    assert omb.spawn([0, 1, 2, 3], [], occ, 2, {(0, 1): 1.0}, False, 0.0, 3, 5.0) == [(0, 1, 2), (0, 1, 3)]


def test_zero_thresholds_give_the_complete_expansion():
    h1, eri, occ = random_system(6, 3, seed=21)
    exp = list(range(6))
    scr = omb.run_mbe_screened(h1, eri, occ, [], exp, 6, True, t_init=0.0, m_init=0, a=5.0)
    assert scr["orders"] == [2, 3, 4, 5, 6]
    for n in scr["orders"]:
        assert len(scr["tuples"][n]) == omb.tuple_count_closed_form(3, 3, False, False, n, True)
        assert scr["tuples"][n] == omb.tuples(exp, [], occ, n, True)
    full = omb.run_mbe(h1, eri, occ, [], exp, [2, 3, 4, 5, 6], True)
    assert abs(scr["e_tot"] - full["e_tot"]) < 1e-12


def test_unreachable_threshold_stops_after_the_first_order():
    h1, eri, occ = random_system(6, 3, seed=22)
    scr = omb.run_mbe_screened(h1, eri, occ, [], list(range(6)), 6, True, t_init=1e10, m_init=0, a=1.0)
    assert scr["orders"] == [2]
    assert len(scr["tuples"][2]) == 9
    # a non-empty reference space starts at order 1
    scr = omb.run_mbe_screened(h1, eri, occ, [2, 3], [0, 1, 4, 5], 4, True, t_init=1e10, m_init=0, a=1.0)
    assert scr["orders"] == [1] and len(scr["tuples"][1]) == 4


def test_screening_is_monotone_in_a_and_children_have_a_computed_parent():
    h1, eri, occ = random_system(7, 3, seed=23)
    exp = list(range(7))
    runs = {a: omb.run_mbe_screened(h1, eri, occ, [], exp, 5, True, t_init=1e-4, m_init=2, a=a)
            for a in (1.0, 10.0, 100.0)}
    for lo, hi in ((1.0, 10.0), (10.0, 100.0)):
        for n, tups in runs[hi]["tuples"].items():
            assert set(tups) <= set(runs[lo]["tuples"].get(n, []))
    # parent-driven enumeration: every child is a computed parent plus one orbital
    r = runs[10.0]
    for n in r["orders"][1:]:
        parents = r["tuples"][n - 1]
        inc = {t: r["inc"][t] for t in parents}
        gen = set()
        for P in parents:
            for c in exp:
                if c in P:
                    continue
                child = tuple(sorted(P + (c,)))
                if not omb.keep_tuple(child, [], occ):
                    continue
                best = max(abs(inc.get(s, 0.0)) for s in itertools.combinations(child, n - 1))
                if best > omb.tuple_threshold(child, occ, 1e-4, 2, 10.0):
                    gen.add(child)
        assert sorted(gen) == r["tuples"][n]
    # screening removed tuples at a = 10 and more at a = 100
    count = {a: sum(len(v) for v in runs[a]["tuples"].values()) for a in runs}
    full = sum(omb.tuple_count_closed_form(3, 4, False, False, n, True) for n in (2, 3, 4, 5))
    assert count[100.0] < count[10.0] < full


def test_first_order_rule():
    assert omb.first_order([], True) == 2
    assert omb.first_order([], False) == 1
    assert omb.first_order([3, 4], True) == 1
