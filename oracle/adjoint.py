"""Oracle for the adjoint of the MBE-FCI energy (gradients by Hellmann-Feynman).

TEST INFRASTRUCTURE ONLY.  Only tests/ (and the smoke check) use this module;
the CUDA product path never imports it.

The paper defines the energy, not its derivatives; the gradient follows from
the definitions used by `oracle.mbe`:

* every CASCI energy E_CAS(A) is the lowest eigenvalue of the Hamiltonian
  restricted to determinants with the core C = O \\ A doubly occupied, so by
  Hellmann-Feynman its derivatives are expectation values in the full orbital
  space of the state |core> x |Psi_A>:
      dE/dh_pq       = gamma_pq,
      dE/d(pq|rs)    = 1/2 Gamma_pqrs,
  with every element of h and (pq|rs) treated as independent;
* the full-space density matrices of |core> x |Psi_A> are
      gamma: 2 on the core diagonal, the active 1-RDM on A x A;
      Gamma: the active 2-RDM on A^4, and for core orbitals c != d and active
      p, q:  Gamma_ccdd = 4, Gamma_cccc = 2, Gamma_cddc = -2,
             Gamma_ccpq = Gamma_pqcc = 2 gamma_pq,
             Gamma_cqpc = Gamma_pccq = -gamma_pq;
* E_MBE = E_CAS(R) + sum of increments, and the increments are linear in the
  tuple energies, so the gradient is the same recursion (Eq. 2) applied to the
  per-tuple gradients d eps(S) = dE_CAS(R u S) - dE_CAS(R).

Pins (tests/test_oracle_adjoint.py): central finite differences of the oracle
energy, the energy recomputed from the density matrices, the homogeneity of the
Hubbard energy in (t, U), and trace(gamma) = number of electrons.
"""

from __future__ import annotations

import math
from typing import Dict, Sequence, Tuple

import numpy as np

from . import fci
from . import mbe as omb


def cas_gradient(h1, eri, occ, A: Sequence[int], two_body: bool = True, tol: float = 1e-13):
    """(E_CAS(A), dE/dh [norb, norb], dE/d(pq|rs) [norb]*4 or None)."""
    norb = len(occ)
    A = sorted(A)
    n = len(A)
    C = [c for c in range(norb) if occ[c] and c not in A]
    e_core, h_eff, eri_a = omb.frozen_core(h1, eri, occ, A)
    if n > 0:
        k = omb.n_active_electrons(occ, A)
        lam, v = fci.lowest_eigenpair(h_eff, eri_a, k, k, tol=tol, want_vector=True)
        gA, GA = fci.rdm12(n, k, k, v, two_body)
    else:
        lam, gA, GA = 0.0, np.zeros((0, 0)), np.zeros((0, 0, 0, 0))
    g = np.zeros((norb, norb))
    for c in C:
        g[c, c] = 2.0
    g[np.ix_(A, A)] = gA
    if not two_body:
        return e_core + lam, g, None
    G = np.zeros((norb,) * 4)
    G[np.ix_(A, A, A, A)] = GA
    for c in C:
        for d in C:
            if c == d:
                G[c, c, c, c] += 2.0
            else:
                G[c, c, d, d] += 4.0
                G[c, d, d, c] -= 2.0
        for a, p in enumerate(A):
            for b, q in enumerate(A):
                G[c, c, p, q] += 2.0 * gA[a, b]
                G[p, q, c, c] += 2.0 * gA[a, b]
                G[c, q, p, c] -= gA[a, b]
                G[p, c, c, q] -= gA[a, b]
    return e_core + lam, g, 0.5 * G


def mbe_gradient(h1, eri, occ, ref, exp, orders, skip: bool, two_body: bool = True):
    """E_MBE and its gradient: Eq. 2 applied to (eps, d eps/dh, d eps/d(pq|rs))."""
    e_R, g_R, G_R = cas_gradient(h1, eri, occ, ref, two_body)
    vals: Dict[int, Dict[Tuple[int, ...], tuple]] = {}
    for n in orders:
        vals[n] = {}
        for t in omb.tuples(exp, ref, occ, n, skip):
            e_S, g_S, G_S = cas_gradient(h1, eri, occ, sorted(set(ref) | set(t)), two_body)
            vals[n][t] = (e_S - e_R, g_S - g_R, (G_S - G_R) if two_body else None)
    inc: Dict[Tuple[int, ...], tuple] = {}
    for n in orders:
        for t, (e, g, G) in vals[n].items():
            subs = [inc[s] for s in omb.proper_subtuples(t) if s in inc]
            de = math.fsum([e] + [-x[0] for x in subs])
            dg = g - sum((x[1] for x in subs), np.zeros_like(g))
            dG = (G - sum((x[2] for x in subs), np.zeros_like(G))) if two_body else None
            inc[t] = (de, dg, dG)
    E = e_R + math.fsum(x[0] for x in inc.values())
    gh = g_R + sum((x[1] for x in inc.values()), np.zeros_like(g_R))
    ge = (G_R + sum((x[2] for x in inc.values()), np.zeros_like(G_R))) if two_body else None
    return E, gh, ge


def adjoint_weights(tuples_by_order: Dict[int, Sequence[Tuple[int, ...]]]):
    """Weights w(S) with E_MBE - E_CAS(R) = sum_S w(S) eps(S), from the transposed
    recursion w(S) = 1 - sum over computed proper supersets U of S of w(U)."""
    present = {n: set(ts) for n, ts in tuples_by_order.items()}
    orders = sorted(tuples_by_order)
    w: Dict[Tuple[int, ...], float] = {}
    for n in reversed(orders):
        for S in tuples_by_order[n]:
            acc = []
            for m in orders:
                if m <= n:
                    continue
                for U in present[m]:
                    if set(S) < set(U):
                        acc.append(w[U])
            w[S] = 1.0 - math.fsum(acc)
    return w
