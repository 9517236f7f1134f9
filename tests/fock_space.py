"""Brute-force second-quantised Hamiltonian, used to pin the oracle.

Independent of oracle/: fermion annihilators are built as Kronecker products of
2x2 matrices (Jordan-Wigner), checked against the canonical anticommutation
relations, and the Hamiltonian
    H = sum_{pq,s} h_pq a+_ps a_qs + 1/2 sum_{pqrs,s,t} (pq|rs) a+_ps a+_rt a_st a_qs
is summed over every index with matrix products.  No excitation-level case
analysis and no phase bookkeeping is involved, so a wrong Slater-Condon rule,
sign or exchange term in the oracle shows up as a mismatch.

Basis: the state with occupation word w (bit k = spin orbital k; bits 0..n-1
alpha, n..2n-1 beta) is basis vector w, and a+_k acting on it picks up
(-1)^(occupied bits below k), i.e. determinants are products of creators in
ascending spin-orbital order.
"""

from __future__ import annotations

import functools

import numpy as np
import scipy.sparse as sp

_SM = np.array([[0.0, 1.0], [0.0, 0.0]])  # |0><1| : lowers occupation 1 -> 0
_Z = np.diag([1.0, -1.0])
_I = np.eye(2)


@functools.lru_cache(maxsize=8)
def annihilators(m: int):
    """Sparse annihilation matrices a_k (k = 0..m-1) on the 2^m Fock space."""
    ops = []
    for k in range(m):
        mat = sp.csr_matrix(np.ones((1, 1)))
        # kron puts its first factor on the most significant bit.
        for bit in range(m - 1, -1, -1):
            if bit > k:
                f = _I
            elif bit == k:
                f = _SM
            else:
                f = _Z
            mat = sp.kron(mat, sp.csr_matrix(f), format="csr")
        ops.append(mat)
    return ops


def hamiltonian(h: np.ndarray, eri: np.ndarray) -> np.ndarray:
    n = h.shape[0]
    a = annihilators(2 * n)
    ad = [x.T for x in a]
    dim = 2 ** (2 * n)
    H = sp.csr_matrix((dim, dim))
    for s in range(2):
        for p in range(n):
            for q in range(n):
                if h[p, q] != 0.0:
                    H += h[p, q] * (ad[p + s * n] @ a[q + s * n])
    for s in range(2):
        for t in range(2):
            for p in range(n):
                for q in range(n):
                    for r in range(n):
                        for u in range(n):
                            v = eri[p, q, r, u]
                            if v == 0.0:
                                continue
                            H += 0.5 * v * (ad[p + s * n] @ ad[r + t * n] @ a[u + t * n]
                                            @ a[q + s * n])
    return H


def sector_words(n: int, na: int, nb: int, must_occ=(), must_empty=()):
    """Occupation words with na alpha and nb beta electrons, in the oracle's order.

    Order: alpha string ascending (outer), beta string ascending (inner).
    must_occ / must_empty: spatial orbitals forced doubly occupied / empty.
    """
    def strings(k):
        out = []
        for x in range(2 ** n):
            if bin(x).count("1") != k:
                continue
            if any(not (x >> c) & 1 for c in must_occ):
                continue
            if any((x >> c) & 1 for c in must_empty):
                continue
            out.append(x)
        return out

    return [sa | (sb << n) for sa in strings(na) for sb in strings(nb)]


def sector_matrix(h, eri, na, nb, must_occ=(), must_empty=()):
    n = h.shape[0]
    H = hamiltonian(h, eri).tocsr()
    w = sector_words(n, na, nb, must_occ, must_empty)
    return H[w][:, w].toarray(), w
