"""Host arithmetic of bench.py's roofline, checked on CPU.

The algorithmic flops per sigma element use R = k(n-k+1), the length of a
string's replacement list (every E_pq that maps a k-electron string of n
orbitals to a string, the diagonal E_pp included).  Here R is counted by brute
force over the strings, and the solver-class choice is checked against its
definition: the warp solver, with the smallest determinants-per-lane class that
holds the space, up to the tuned determinant limit; the block solver above it.
"""

import itertools
import math

import pytest

import bench


def brute_force_list_length(n: int, k: int) -> int:
    lengths = set()
    for occ in itertools.combinations(range(n), k):
        occ = set(occ)
        lengths.add(sum(1 for p in range(n) for q in occ if p == q or p not in occ))
    assert len(lengths) == 1  # every string has the same number of replacements
    return lengths.pop()


@pytest.mark.parametrize("n,k", [(1, 1), (2, 1), (4, 2), (6, 3), (6, 1), (9, 4), (10, 5), (12, 6)])
def test_sigma_flops_use_the_replacement_list_length(n, k):
    r = brute_force_list_length(n, k)
    assert r == k * (n - k + 1)
    assert bench.sigma_flops_per_det(n, k) == 2 * (2 * math.comb(n, k) + r * r)


@pytest.mark.parametrize("warp_max", [100, 225, 416])
def test_solver_class_choice(warp_max):
    for n in range(1, 13):
        for k in range(0, n + 1):
            ndet = math.comb(n, k) ** 2
            solver, dpl = bench.solver_bucket(n, k, warp_max)
            if n <= 8 and ndet <= warp_max:
                assert solver == 0
                assert dpl * 32 >= ndet
                smaller = [d for d in (1, 2, 4, 8, 13) if d < dpl]
                assert all(d * 32 < ndet for d in smaller)
            else:
                assert (solver, dpl) == (1, 0)


def test_recorded_traffic_is_gated_by_the_kernel_source(monkeypatch):
    # the committed DRAM counters count only while the solver sources are the ones
    # they were taken on; any other source hash reports no traffic
    key = "k_casci_warp_mixed<13>:order6"
    got = bench.recorded_traffic(key)
    assert got is None or (isinstance(got, int) and got > 0)
    monkeypatch.setattr(bench, "source_hash", lambda: "0000000000000000")
    assert bench.recorded_traffic(key) is None
    assert bench.recorded_traffic("no such kernel") is None
