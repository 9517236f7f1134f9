"""Oracle for the MBE-FCI hot path: tuples, tuple CASCI energies, Eq. 2 and Eq. 1.

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
leg of bench.py use this module; the CUDA product path never imports it.

Plain, literal restatement of the method:

* reference determinant energy (closed shell, doubly occupied set O)
      E_Phi = sum_{i in O} 2 h_ii + sum_{i,j in O} [ 2 (ii|jj) - (ij|ji) ];
* a tuple Omega of expansion orbitals defines the complete active space
  A = R u Omega (Eq. 1: "the composite space of orbital p and all of the
  reference space MOs"); occupied orbitals outside A are a frozen core
  C = O \\ A, virtual orbitals outside A are deleted.  With
      E_core = sum_{c in C} 2 h_cc + sum_{c,d in C} [ 2 (cc|dd) - (cd|dc) ]
      h_eff_pq = h_pq + sum_{c in C} [ 2 (pq|cc) - (pc|cq) ]        (p, q in A)
  the CASCI energy is E_CAS(A) = E_core + lowest eigenvalue of the A-space
  Hamiltonian built from h_eff and (pq|rs) restricted to A, in the sector with
  n_alpha = n_beta = |O n A| electrons;
* the tuple energy is measured from the reference: eps(Omega) = E_CAS(R u Omega)
  - E_Phi - E_ref,corr with E_ref,corr = E_CAS(R) - E_Phi (zero for R = {}),
  so that Eq. 1 sums correlation energies;
* the increment of Eq. 2: Delta eps(Omega) = eps(Omega) - sum of Delta eps(S)
  over every proper, non-empty sub-tuple S of Omega (a sub-tuple that was not
  computed, such as a skipped one, contributes zero);
* the order sums and the total of Eq. 1 (Eq. 3 for an empty reference space):
  E^(n) = sum over order-n tuples of Delta eps, E_corr = E_ref,corr + sum_n E^(n),
  E_tot = E_Phi + E_corr.

Tuples of order n are all n-subsets of the sorted expansion space in
lexicographic order.  With the skip rule (the vacuum-reference statement after
Eq. 3: only tuples holding both occupied and virtual orbitals contribute), a
tuple is dropped when A = R u Omega holds no occupied or no virtual orbital.

Screened expansion (Sec. 2, the child-spawning rule and Eq. 4):

* Eq. 4: a tuple's threshold is T_tup = 0 when M_tup < M_init and
  T_init * a^(M_tup - M_init) otherwise, with M_tup = max(number of occupied,
  number of virtual orbitals of the tuple Omega);
* the first order of the expansion (order 2 for an empty reference space with
  the skip rule, order 1 otherwise) holds every tuple; an order-(k+1) tuple is
  spawned when the absolute increment of at least one of its order-k sub-tuples
  exceeds the child's threshold, a sub-tuple that was not computed (skipped or
  not spawned) counting as zero; the skip rule still applies to the child.
  (The paper phrases this per parent tuple and candidate orbital; read as a
  condition on the child's order-k sub-tuples it does not depend on which
  parent generates the child.)

Pins (tests/test_oracle_pins.py): zero thresholds reproduce the complete tuple
sets and the unscreened energies, an unreachable threshold stops the expansion
after its first order, a hand-worked four-orbital example, Eq. 4 at hand-computed
points, monotonicity in a, and brute-force versus parent-driven enumeration.
"""

from __future__ import annotations

import itertools
import math
from typing import Dict, Iterable, List, Sequence, Tuple

import numpy as np

from . import fci


# The energies of the closed-shell determinants below are sums of hundreds of
# terms (529 pair terms for 23 occupied orbitals).  They are summed exactly
# (math.fsum, one rounding at the end): eps(Omega) is a small difference of two
# such sums, and left-to-right rounding of each (about 3e-13 E_h for the 46-site
# ring) would bias every tuple energy by about 1e-13 E_h.

def phi_energy(h1: np.ndarray, eri: np.ndarray, occ: np.ndarray) -> float:
    O = [i for i in range(len(occ)) if occ[i]]
    terms = [2.0 * h1[i, i] for i in O]
    for i in O:
        for j in O:
            terms += [2.0 * eri[i, i, j, j], -eri[i, j, j, i]]
    return math.fsum(terms)


def frozen_core(h1: np.ndarray, eri: np.ndarray, occ: np.ndarray, A: Sequence[int]):
    """(E_core, h_eff over A, eri over A) for the active space A."""
    A = list(A)
    C = [c for c in range(len(occ)) if occ[c] and c not in A]
    terms = [2.0 * h1[c, c] for c in C]
    for c in C:
        for d in C:
            terms += [2.0 * eri[c, c, d, d], -eri[c, d, d, c]]
    e_core = math.fsum(terms)
    n = len(A)
    h_eff = np.empty((n, n))
    for a, p in enumerate(A):
        for b, q in enumerate(A):
            terms = [h1[p, q]]
            for c in C:
                terms += [2.0 * eri[p, q, c, c], -eri[p, c, c, q]]
            h_eff[a, b] = math.fsum(terms)
    eri_a = np.ascontiguousarray(eri[np.ix_(A, A, A, A)])
    return float(e_core), h_eff, eri_a


def n_active_electrons(occ: np.ndarray, A: Sequence[int]) -> int:
    return int(sum(int(occ[p]) for p in A))


def casci_energy(h1, eri, occ, A, tol: float = 1e-13, even_only: bool = False) -> float:
    """E_CAS(A) = E_core + lowest eigenvalue of the A-space Hamiltonian; with
    even_only, the lowest one that is even under the alpha-beta string exchange
    (the closed-shell determinant's sector: states of even total spin)."""
    A = sorted(A)
    e_core, h_eff, eri_a = frozen_core(h1, eri, occ, A)
    if len(A) == 0:
        return e_core
    ne = n_active_electrons(occ, A)
    if even_only:
        return e_core + fci.lowest_eigenvalue_even(h_eff, eri_a, ne, tol=tol)
    lam = fci.lowest_eigenvalue(h_eff, eri_a, ne, ne, tol=tol)
    return e_core + lam


def ref_corr_energy(h1, eri, occ, ref: Sequence[int]) -> float:
    """E_ref,corr = E_CAS(R) - E_Phi; zero for an empty reference space."""
    if len(ref) == 0:
        return 0.0
    return casci_energy(h1, eri, occ, ref) - phi_energy(h1, eri, occ)


def tuple_energy(h1, eri, occ, ref, tup, e_phi: float, e_ref_corr: float, even_only: bool = False) -> float:
    """eps(Omega) = E_CAS(R u Omega) - E_Phi - E_ref,corr."""
    A = sorted(set(ref) | set(tup))
    return casci_energy(h1, eri, occ, A, even_only=even_only) - e_phi - e_ref_corr


def keep_tuple(tup: Sequence[int], ref: Sequence[int], occ: np.ndarray) -> bool:
    A = list(ref) + list(tup)
    n_occ = sum(1 for p in A if occ[p])
    return 0 < n_occ < len(A)


def tuples(exp: Sequence[int], ref: Sequence[int], occ: np.ndarray, order: int,
           skip: bool) -> List[Tuple[int, ...]]:
    """Order-n tuples of the sorted expansion space, lexicographic, skip rule optional."""
    out = []
    for t in itertools.combinations(sorted(exp), order):
        if skip and not keep_tuple(t, ref, occ):
            continue
        out.append(t)
    return out


def tuple_count_closed_form(m_occ: int, m_vir: int, ref_has_occ: bool, ref_has_vir: bool,
                            order: int, skip: bool) -> int:
    """Number of kept order-n tuples: C(M, n) minus the all-virtual and all-occupied ones."""
    total = math.comb(m_occ + m_vir, order)
    if not skip:
        return total
    if not ref_has_occ:
        total -= math.comb(m_vir, order)
    if not ref_has_vir:
        total -= math.comb(m_occ, order)
    return total


def proper_subtuples(t: Tuple[int, ...]) -> Iterable[Tuple[int, ...]]:
    for m in range(1, len(t)):
        for s in itertools.combinations(t, m):
            yield s


def increments(eps_by_order: Dict[int, Dict[Tuple[int, ...], float]]):
    """Eq. 2, literally: Delta eps(Omega) = eps(Omega) - sum over proper sub-tuples."""
    inc: Dict[Tuple[int, ...], float] = {}
    for order in sorted(eps_by_order):
        for t, e in eps_by_order[order].items():
            terms = [e] + [-inc.get(s, 0.0) for s in proper_subtuples(t)]
            inc[t] = math.fsum(terms)
    return inc


def order_sums(inc: Dict[Tuple[int, ...], float], orders: Sequence[int]) -> Dict[int, float]:
    out = {}
    for n in orders:
        out[n] = math.fsum(v for t, v in inc.items() if len(t) == n)
    return out


def run_mbe(h1, eri, occ, ref, exp, orders, skip: bool):
    """Full oracle MBE: per-tuple eps, increments, order sums and totals."""
    e_phi = phi_energy(h1, eri, occ)
    e_ref = ref_corr_energy(h1, eri, occ, ref)
    eps_by_order = {}
    for n in orders:
        eps_by_order[n] = {t: tuple_energy(h1, eri, occ, ref, t, e_phi, e_ref)
                           for t in tuples(exp, ref, occ, n, skip)}
    inc = increments(eps_by_order)
    e_order = order_sums(inc, orders)
    e_corr = math.fsum([e_ref] + [e_order[n] for n in orders])
    return dict(e_phi=e_phi, e_ref_corr=e_ref, eps=eps_by_order, inc=inc, e_order=e_order,
                e_corr=e_corr, e_tot=e_phi + e_corr)


def tuple_threshold(tup: Sequence[int], occ: np.ndarray, t_init: float, m_init: int, a: float) -> float:
    """Eq. 4: T_tup = 0 if M_tup < M_init, else T_init * a^(M_tup - M_init)."""
    n_occ = sum(1 for p in tup if occ[p])
    m_tup = max(n_occ, len(tup) - n_occ)
    if m_tup < m_init:
        return 0.0
    t = float(t_init)
    for _ in range(m_tup - m_init):  # repeated products, in this order
        t *= a
    return t


def first_order(ref: Sequence[int], skip: bool) -> int:
    """Lowest order with computed tuples: 2 for an empty reference space under the
    skip rule (no single orbital is both occupied and virtual), else 1."""
    return 2 if (skip and len(ref) == 0) else 1


def spawn(exp: Sequence[int], ref: Sequence[int], occ: np.ndarray, order: int,
          inc: Dict[Tuple[int, ...], float], skip: bool, t_init: float, m_init: int,
          a: float) -> List[Tuple[int, ...]]:
    """Order-(order+1) tuples spawned from the order-`order` increments `inc`
    (all (order+1)-subsets tested, lexicographic output)."""
    out = []
    for child in itertools.combinations(sorted(exp), order + 1):
        if skip and not keep_tuple(child, ref, occ):
            continue
        best = max(abs(inc.get(s, 0.0)) for s in itertools.combinations(child, order))
        if best > tuple_threshold(child, occ, t_init, m_init, a):
            out.append(child)
    return out


def run_mbe_screened(h1, eri, occ, ref, exp, max_order: int, skip: bool, t_init: float = 1e-10,
                     m_init: int = 3, a: float = 5.0):
    """Screened MBE: complete first order, then spawned orders until max_order or
    until no tuple is spawned."""
    e_phi = phi_energy(h1, eri, occ)
    e_ref = ref_corr_energy(h1, eri, occ, ref)
    k0 = first_order(ref, skip)
    eps_by_order: Dict[int, Dict[Tuple[int, ...], float]] = {}
    inc: Dict[Tuple[int, ...], float] = {}
    tups = tuples(exp, ref, occ, k0, skip)
    orders = []
    for k in range(k0, max_order + 1):
        if k > k0:
            tups = spawn(exp, ref, occ, k - 1, {t: inc[t] for t in eps_by_order[k - 1]}, skip,
                         t_init, m_init, a)
        if not tups:
            break
        eps_by_order[k] = {t: tuple_energy(h1, eri, occ, ref, t, e_phi, e_ref) for t in tups}
        inc = increments(eps_by_order)
        orders.append(k)
    e_order = order_sums(inc, orders)
    e_corr = math.fsum([e_ref] + [e_order[n] for n in orders])
    return dict(e_phi=e_phi, e_ref_corr=e_ref, eps=eps_by_order, inc=inc, e_order=e_order,
                e_corr=e_corr, e_tot=e_phi + e_corr, orders=orders,
                tuples={n: list(eps_by_order[n]) for n in orders})
