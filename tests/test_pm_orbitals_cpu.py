"""Pipek-Mezey orbitals of the Hubbard ring (the paper's orbital basis for its
Hubbard results), as an input generator: checked against the definition of a
Pipek-Mezey maximum and against invariants of the reference determinant."""

import numpy as np
import pytest

from oracle import mbe as omb
from workloads import hubbard_ring_momentum, hubbard_ring_pm, pm_functional


@pytest.mark.parametrize("L", [10, 22])
def test_pm_orbitals(L):
    h1, eri, occ, C = hubbard_ring_pm(L, 1.0, 4.0)
    h1m, erim, occm, Cm = hubbard_ring_momentum(L, 1.0, 4.0)
    no = int(occ.sum())
    # orthonormal, and each space spans the same subspace as before
    assert np.abs(C.T @ C - np.eye(L)).max() < 1e-12
    Po, Pm = C[:, :no] @ C[:, :no].T, Cm[:, :no] @ Cm[:, :no].T
    assert np.abs(Po - Pm).max() < 1e-12
    # the reference determinant and its energy are unchanged
    assert abs(omb.phi_energy(h1, eri, occ) - omb.phi_energy(h1m, erim, occm)) < 1e-10
    # localised: the functional grew, and every pair sits at its optimal angle 0
    for sl in (slice(0, no), slice(no, L)):
        assert pm_functional(C[:, sl]) > pm_functional(Cm[:, sl]) + 0.1
        X = C[:, sl]
        n = X.shape[1]
        for p in range(n):
            for q in range(p + 1, n):
                qpq, qpp, qqq = X[:, p] * X[:, q], X[:, p] ** 2, X[:, q] ** 2
                A = np.sum(qpq * qpq - 0.25 * (qpp - qqq) ** 2)
                B = np.sum(qpq * (qpp - qqq))
                assert abs(B) < 1e-9 and A <= 1e-9
    # integrals transform as the site Hamiltonian does
    assert abs(np.trace(h1) - np.trace(h1m)) < 1e-12
