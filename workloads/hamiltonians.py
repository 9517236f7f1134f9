"""Model Hamiltonians for the MBE-FCI workloads.

Conventions used throughout the repository:

* ``h1`` is the real symmetric one-electron matrix h_pq, shape (N, N), float64.
* ``eri`` holds the real two-electron integrals in chemists' notation
  (pq|rs) = eri[p, q, r, s], shape (N, N, N, N), float64, with the 8-fold
  permutational symmetry of real orbitals.
* ``occ`` is a uint8 vector; occ[p] = 1 marks an orbital that is doubly
  occupied in the closed-shell reference determinant Phi.
* ``ref`` and ``exp`` are the reference space R and the expansion space X of
  the MBE-FCI partition (Eq. 1): sorted, disjoint lists of orbital indices.

The Hubbard ring is written in the real standing-wave ("momentum") basis that
diagonalises the hopping matrix: phi_0 = 1/sqrt(L); for k = 1 .. L/2-1 the pair
sqrt(2/L) cos(2 pi k i / L), sqrt(2/L) sin(2 pi k i / L); and, for even L,
phi_{L/2} = (-1)^i / sqrt(L).  Orbitals are ordered by their band energy
-2 t cos(2 pi k / L); inside a degenerate pair the cosine comes first.  The
site Hamiltonian is H = -t sum_<ij>,s a+_is a_js + U sum_i n_i,up n_i,down with
periodic boundary conditions, so in the site basis (ii|ii) = U.

The synthetic molecule has 40 orbitals and 16 electrons.  Its generator draws
from ``numpy.random.default_rng(seed)`` in a fixed order: first the N x N
off-diagonal noise of h1 (standard deviation 0.05, upper triangle mirrored),
then one N x N normal matrix G_L per auxiliary index L = 1 .. 120.  Each
B^L = (G_L + G_L^T)/2 * 0.3 exp(-L/30), and (pq|rs) = sum_L B^L_pq B^L_rs,
which is symmetric and positive semi-definite.  The diagonal of h1 is graded
linearly from -2 to +3 E_h.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class Workload:
    """One MBE-FCI problem: integrals, reference occupation and orbital partition."""

    name: str
    h1: np.ndarray
    eri: np.ndarray
    occ: np.ndarray
    ref: List[int]
    exp: List[int]
    orders: List[int]
    skip: bool
    description: str = ""
    params: dict = field(default_factory=dict)

    @property
    def norb(self) -> int:
        return int(self.h1.shape[0])

    @property
    def nocc(self) -> int:
        return int(self.occ.sum())


def _check(h1: np.ndarray, eri: np.ndarray) -> None:
    n = h1.shape[0]
    assert h1.shape == (n, n) and eri.shape == (n, n, n, n)
    assert h1.dtype == np.float64 and eri.dtype == np.float64


def hubbard_momentum_orbitals(L: int, t: float = 1.0):
    """Real standing-wave orbitals of the periodic ring and their band energies.

    Returns (C, eps) with C[i, p] the amplitude of orbital p on site i, columns
    ordered by ascending band energy (cosine before sine inside a pair).
    """
    sites = np.arange(L)
    cols, eps, keys = [], [], []
    cols.append(np.full(L, 1.0 / np.sqrt(L)))
    eps.append(-2.0 * t)
    keys.append((0, 0))
    for k in range(1, (L - 1) // 2 + 1):
        ang = 2.0 * np.pi * k * sites / L
        e = -2.0 * t * np.cos(2.0 * np.pi * k / L)
        cols.append(np.sqrt(2.0 / L) * np.cos(ang))
        eps.append(e)
        keys.append((k, 0))
        cols.append(np.sqrt(2.0 / L) * np.sin(ang))
        eps.append(e)
        keys.append((k, 1))
    if L % 2 == 0:
        cols.append(np.where(sites % 2 == 0, 1.0, -1.0) / np.sqrt(L))
        eps.append(2.0 * t)
        keys.append((L // 2, 0))
    C = np.stack(cols, axis=1)
    eps = np.array(eps)
    # Ascending energy; for t > 0 this is ascending k with cosine first, which
    # the (rounded energy, k, cos/sin) key makes explicit and tie-proof.
    order = sorted(range(L), key=lambda j: (round(float(eps[j]), 12), keys[j]))
    return C[:, order], eps[order]


def hubbard_site_integrals(L: int, t: float, U: float, periodic: bool = True):
    h = np.zeros((L, L))
    nbonds = L if periodic else L - 1
    for i in range(nbonds):
        j = (i + 1) % L
        h[i, j] -= t
        h[j, i] -= t
    eri = np.zeros((L, L, L, L))
    for i in range(L):
        eri[i, i, i, i] = U
    return h, eri


def hubbard_ring_momentum(L: int, t: float = 1.0, U: float = 4.0, nocc: Optional[int] = None):
    """Periodic Hubbard ring in the momentum basis: returns (h1, eri, occ, C)."""
    assert L >= 3
    C, _ = hubbard_momentum_orbitals(L, t)
    hs, _ = hubbard_site_integrals(L, t, U, periodic=True)
    h1 = C.T @ hs @ C
    h1 = 0.5 * (h1 + h1.T)
    eri = U * np.einsum("ip,iq,ir,is->pqrs", C, C, C, C, optimize=True)
    if nocc is None:
        nocc = L // 2
    occ = np.zeros(L, dtype=np.uint8)
    occ[:nocc] = 1
    _check(h1, eri)
    return np.ascontiguousarray(h1), np.ascontiguousarray(eri), occ, C


def pipek_mezey(C: np.ndarray, max_sweeps: int = 500, tol: float = 1e-12) -> np.ndarray:
    """Pipek-Mezey localisation (Pipek and Mezey, J. Chem. Phys. 90, 4916 (1989))
    of the orthonormal orbitals in the columns of C, given on an orthonormal
    site basis: Jacobi sweeps of 2x2 rotations, each at the angle that maximises
    the sum over orbitals and sites of the squared site populations (C[i, p]^2)^2.
    For the pair (p, q), with Q_pq = C[:, p] C[:, q] sitewise,
        A = sum (Q_pq^2 - (Q_pp - Q_qq)^2 / 4),  B = sum Q_pq (Q_pp - Q_qq),
    the rotation p' = cos g p + sin g q, q' = -sin g p + cos g q with
    4 g = atan2(B, -A) is optimal.  Deterministic for a given C."""
    C = np.array(C, dtype=np.float64, copy=True)
    n = C.shape[1]
    for _ in range(max_sweeps):
        biggest = 0.0
        for p in range(n):
            for q in range(p + 1, n):
                cp, cq = C[:, p].copy(), C[:, q].copy()
                qpq, qpp, qqq = cp * cq, cp * cp, cq * cq
                A = float(np.sum(qpq * qpq - 0.25 * (qpp - qqq) ** 2))
                B = float(np.sum(qpq * (qpp - qqq)))
                if A * A + B * B < 1e-28:
                    continue
                g = 0.25 * np.arctan2(B, -A)
                if abs(g) < 1e-15:
                    continue
                c, s = np.cos(g), np.sin(g)
                C[:, p] = c * cp + s * cq
                C[:, q] = -s * cp + c * cq
                biggest = max(biggest, abs(g))
        if biggest < tol:
            break
    return C


def pm_functional(C: np.ndarray) -> float:
    """Sum over orbitals and sites of the squared site populations."""
    return float(np.sum(C ** 4))


def hubbard_ring_pm(L: int, t: float = 1.0, U: float = 4.0, nocc: Optional[int] = None):
    """Periodic Hubbard ring in Pipek-Mezey orbitals: the momentum orbitals of the
    occupied and of the virtual space localised separately (the reference
    determinant is unchanged). Returns (h1, eri, occ, C)."""
    h1m, erim, occ, Cm = hubbard_ring_momentum(L, t, U, nocc)
    no = int(occ.sum())
    C = np.concatenate([pipek_mezey(Cm[:, :no]), pipek_mezey(Cm[:, no:])], axis=1)
    hs, _ = hubbard_site_integrals(L, t, U, periodic=True)
    h1 = C.T @ hs @ C
    h1 = 0.5 * (h1 + h1.T)
    eri = U * np.einsum("ip,iq,ir,is->pqrs", C, C, C, C, optimize=True)
    _check(h1, eri)
    return np.ascontiguousarray(h1), np.ascontiguousarray(eri), occ, C


def hubbard_open_dimer(t: float = 1.0, U: float = 4.0):
    """Two sites joined by one bond (no ring), in the site basis; site 0 occupied."""
    h1, eri = hubbard_site_integrals(2, t, U, periodic=False)
    occ = np.array([1, 0], dtype=np.uint8)
    return h1, eri, occ


def _low_rank_eri(rng: np.random.Generator, n: int, naux: int, scale: float, decay: float):
    B = np.empty((naux, n, n))
    for L in range(1, naux + 1):
        G = rng.normal(0.0, 1.0, size=(n, n))
        B[L - 1] = 0.5 * (G + G.T) * scale * np.exp(-L / decay)
    return np.einsum("Lpq,Lrs->pqrs", B, B, optimize=True)


def synthetic_molecule(seed: int = 1910, norb: int = 40, nocc: int = 8, naux: int = 120):
    """Seeded molecular-like Hamiltonian: returns (h1, eri, occ)."""
    rng = np.random.default_rng(seed)
    h1 = np.diag(np.linspace(-2.0, 3.0, norb))
    noise = np.triu(rng.normal(0.0, 0.05, size=(norb, norb)), 1)
    h1 = h1 + noise + noise.T
    eri = _low_rank_eri(rng, norb, naux, 0.3, 30.0)
    occ = np.zeros(norb, dtype=np.uint8)
    occ[:nocc] = 1
    _check(h1, eri)
    return np.ascontiguousarray(h1), np.ascontiguousarray(eri), occ


def random_system(n: int, nocc: int, seed: int, naux: int = 6, offdiag: float = 0.1,
                  eri_scale: float = 0.4):
    """Small random Hamiltonian with graded orbital energies, for tests."""
    rng = np.random.default_rng(seed)
    h1 = np.diag(np.linspace(-1.5, 1.5, n))
    noise = np.triu(rng.normal(0.0, offdiag, size=(n, n)), 1)
    h1 = h1 + noise + noise.T
    eri = _low_rank_eri(rng, n, naux, eri_scale, 4.0)
    occ = np.zeros(n, dtype=np.uint8)
    occ[:nocc] = 1
    _check(h1, eri)
    return np.ascontiguousarray(h1), np.ascontiguousarray(eri), occ


def block_decoupled_system(n1: int, nocc1: int, n2: int, nocc2: int, seed: int,
                           gap: float = 6.0):
    """Two random systems with no coupling at all, interleaved orbital order.

    Orbitals of block 1 and block 2 alternate in the index order (as far as the
    sizes allow), so that tuples mix both blocks.  h1 and (pq|rs) vanish unless
    all indices belong to one block.  Occupied orbital energies are lowered and
    virtual ones raised by gap/2, so that moving an electron from one block to
    the other (or flipping spins across blocks) costs far more than any
    correlation energy: the lowest state of every active space then keeps each
    block's electron count and is the sum of the two blocks' ground states.
    Returns (h1, eri, occ, block_of_orbital).
    """
    hA, eA, oA = random_system(n1, nocc1, seed)
    hB, eB, oB = random_system(n2, nocc2, seed + 1)
    for hh, oo in ((hA, oA), (hB, oB)):
        hh[np.diag_indices_from(hh)] += np.where(oo == 1, -0.5 * gap, 0.5 * gap)
    n = n1 + n2
    # Interleave: occupied orbitals first (so that occ is a prefix), then virtuals.
    slots = []
    ia_occ, ib_occ = list(range(nocc1)), list(range(nocc2))
    ia_vir, ib_vir = list(range(nocc1, n1)), list(range(nocc2, n2))
    while ia_occ or ib_occ:
        if ia_occ:
            slots.append((0, ia_occ.pop(0)))
        if ib_occ:
            slots.append((1, ib_occ.pop(0)))
    while ia_vir or ib_vir:
        if ia_vir:
            slots.append((0, ia_vir.pop(0)))
        if ib_vir:
            slots.append((1, ib_vir.pop(0)))
    h1 = np.zeros((n, n))
    eri = np.zeros((n, n, n, n))
    occ = np.zeros(n, dtype=np.uint8)
    block = np.zeros(n, dtype=np.int32)
    for blk, (hh, ee, oo) in enumerate(((hA, eA, oA), (hB, eB, oB))):
        idx = [g for g, (b, _) in enumerate(slots) if b == blk]
        loc = [l for (b, l) in slots if b == blk]
        ix = np.ix_(idx, idx)
        h1[ix] = hh[np.ix_(loc, loc)]
        eri[np.ix_(idx, idx, idx, idx)] = ee[np.ix_(loc, loc, loc, loc)]
        occ[idx] = oo[loc]
        block[idx] = blk
    _check(h1, eri)
    return h1, eri, occ, block


WORKLOAD_NAMES = ("hubbard8", "hubbard22", "molecule40", "hubbard46", "molecule20", "hubbard22pm", "hubbard46pm")


def workload(name: str) -> Workload:
    """The standard MBE-FCI workloads, by name.

    hubbard8   : L=8 ring, t=1, U=2, half filling, empty reference, expansion over
                 all 8 orbitals to full order 8, no tuple skipping (255 tuples).
    hubbard22  : L=22 ring, t=1, U=4, half filling, empty reference, orders 1-6,
                 tuples without an occupied or without a virtual orbital skipped.
    molecule40 : synthetic 40-orbital, 16-electron Hamiltonian (seed 1910); the
                 (6e,6o) reference space {5..10} around the Fermi level expanded
                 over the other 34 orbitals to order 4.
    hubbard46  : L=46 ring, t=1, U=4, half filling, empty reference, orders 1-4,
                 with the same skip rule as hubbard22.
    molecule20 : molecule40 truncated to orbitals 0..19 (same occupation and
                 reference space), orders 1-4; the adjoint workload.
    """
    if name == "hubbard8":
        h1, eri, occ, _ = hubbard_ring_momentum(8, 1.0, 2.0)
        return Workload(name, h1, eri, occ, [], list(range(8)), list(range(1, 9)), False,
                        "Hubbard ring L=8 t=1 U=2, full-order MBE", dict(L=8, t=1.0, U=2.0))
    if name == "hubbard22":
        h1, eri, occ, _ = hubbard_ring_momentum(22, 1.0, 4.0)
        return Workload(name, h1, eri, occ, [], list(range(22)), list(range(1, 7)), True,
                        "Hubbard ring L=22 t=1 U=4, orders 1-6", dict(L=22, t=1.0, U=4.0))
    if name in ("hubbard22pm", "hubbard46pm"):
        L = 22 if name == "hubbard22pm" else 46
        h1, eri, occ, _ = hubbard_ring_pm(L, 1.0, 4.0)
        return Workload(name, h1, eri, occ, [], list(range(L)), list(range(1, 7 if L == 22 else 5)), True,
                        f"Hubbard ring L={L} t=1 U=4, Pipek-Mezey orbitals", dict(L=L, t=1.0, U=4.0))
    if name == "hubbard46":
        h1, eri, occ, _ = hubbard_ring_momentum(46, 1.0, 4.0)
        return Workload(name, h1, eri, occ, [], list(range(46)), list(range(1, 5)), True,
                        "Hubbard ring L=46 t=1 U=4, orders 1-4", dict(L=46, t=1.0, U=4.0))
    if name == "molecule40":
        h1, eri, occ = synthetic_molecule(1910)
        ref = list(range(5, 11))
        exp = [p for p in range(40) if p not in ref]
        return Workload(name, h1, eri, occ, ref, exp, list(range(1, 5)), False,
                        "synthetic 40-orbital molecule, (6e,6o) reference, orders 1-4",
                        dict(seed=1910))
    if name == "molecule20":
        h1, eri, occ = synthetic_molecule(1910)
        keep = list(range(20))
        h1 = np.ascontiguousarray(h1[np.ix_(keep, keep)])
        eri = np.ascontiguousarray(eri[np.ix_(keep, keep, keep, keep)])
        ref = list(range(5, 11))
        exp = [p for p in range(20) if p not in ref]
        return Workload(name, h1, eri, occ[:20].copy(), ref, exp, list(range(1, 5)), False,
                        "synthetic molecule truncated to its first 20 orbitals, (6e,6o) reference, "
                        "orders 1-4", dict(seed=1910))
    raise KeyError(name)
