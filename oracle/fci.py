"""Oracle CASCI: Slater-Condon Hamiltonian (C core) plus a library eigensolver.

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
leg of bench.py use this module; the CUDA product path never imports it.

The lowest eigenvalue of the determinant-basis Hamiltonian of a complete
active space is the CASCI energy that every MBE-FCI term is built from (the
"energy of a CASCI calculation" that defines epsilon in Eq. 1).  Determinant
order and signs follow the convention stated in fci.c: alpha strings and beta
strings in ascending bit-pattern order, index = I_a * N_b + I_b, creators in
ascending spin-orbital order with all alpha orbitals before all beta ones.

The eigensolver is a library routine: LAPACK (scipy.linalg.eigh) on the dense
matrix for small spaces, ARPACK (scipy.sparse.linalg.eigsh) on the sparse
matrix, or on an on-the-fly H*c operator, for larger ones.
"""

from __future__ import annotations

import ctypes
import functools
import math

import numpy as np

from . import build as _build

DENSE_MAX = 1500
SPARSE_MAX_ENTRIES = 64_000_000


@functools.lru_cache(maxsize=1)
def lib():
    path = _build.build()
    L = ctypes.CDLL(path)
    i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    P = ctypes.c_void_p
    L.oracle_binom.restype = i64
    L.oracle_binom.argtypes = [i32, i32]
    L.oracle_strings.restype = i64
    L.oracle_strings.argtypes = [i32, i32, P]
    L.oracle_hij.restype = dbl
    L.oracle_hij.argtypes = [i32, P, P, ctypes.c_uint64, ctypes.c_uint64]
    L.oracle_dets.restype = i32
    L.oracle_dets.argtypes = [i32, i32, i32, P]
    L.oracle_hdiag.restype = i32
    L.oracle_hdiag.argtypes = [i32, i32, i32, P, P, P]
    L.oracle_h_coo.restype = i64
    L.oracle_h_coo.argtypes = [i32, i32, i32, P, P, i64, P, P, P]
    L.oracle_sigma.restype = i32
    L.oracle_sigma.argtypes = [i32, i32, i32, P, P, P, P]
    L.oracle_rdm12.restype = i32
    L.oracle_rdm12.argtypes = [i32, i32, i32, P, P, P]
    L.oracle_sigma_rows.restype = i32
    L.oracle_sigma_rows.argtypes = [i32, i32, i32, P, P, P, i64, P, P]
    return L


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def binom(n: int, k: int) -> int:
    return int(lib().oracle_binom(n, k))


def strings(n: int, k: int) -> np.ndarray:
    """All k-electron strings over n orbitals as bit patterns, ascending."""
    cnt = binom(n, k)
    out = np.zeros(max(cnt, 1), dtype=np.uint64)
    got = lib().oracle_strings(n, k, _ptr(out))
    assert got == cnt
    return out[:cnt]


def dets(n: int, na: int, nb: int) -> np.ndarray:
    """2n-bit determinant words in index order (alpha low bits, beta high bits)."""
    N = binom(n, na) * binom(n, nb)
    out = np.zeros(max(N, 1), dtype=np.uint64)
    assert lib().oracle_dets(n, na, nb, _ptr(out)) == 0
    return out[:N]


def hij(h: np.ndarray, eri: np.ndarray, I: int, J: int) -> float:
    h, eri = _c(h), _c(eri)
    return float(lib().oracle_hij(h.shape[0], _ptr(h), _ptr(eri), int(I), int(J)))


def hdiag(h: np.ndarray, eri: np.ndarray, na: int, nb: int) -> np.ndarray:
    h, eri = _c(h), _c(eri)
    n = h.shape[0]
    N = binom(n, na) * binom(n, nb)
    out = np.zeros(max(N, 1))
    assert lib().oracle_hdiag(n, na, nb, _ptr(h), _ptr(eri), _ptr(out)) == 0
    return out[:N]


def h_coo(h: np.ndarray, eri: np.ndarray, na: int, nb: int):
    """(rows, cols, vals) of the sparse Hamiltonian of the (na, nb) sector."""
    h, eri = _c(h), _c(eri)
    n = h.shape[0]
    L = lib()
    need = L.oracle_h_coo(n, na, nb, _ptr(h), _ptr(eri), 0, None, None, None)
    cnt = -need if need < 0 else need
    rows = np.zeros(max(cnt, 1), dtype=np.int64)
    cols = np.zeros(max(cnt, 1), dtype=np.int64)
    vals = np.zeros(max(cnt, 1))
    got = L.oracle_h_coo(n, na, nb, _ptr(h), _ptr(eri), cnt, _ptr(rows), _ptr(cols), _ptr(vals))
    assert got == cnt
    return rows[:cnt], cols[:cnt], vals[:cnt]


def h_dense(h: np.ndarray, eri: np.ndarray, na: int, nb: int) -> np.ndarray:
    n = h.shape[0]
    N = binom(n, na) * binom(n, nb)
    rows, cols, vals = h_coo(h, eri, na, nb)
    H = np.zeros((N, N))
    np.add.at(H, (rows, cols), vals)
    return H


def sigma(h: np.ndarray, eri: np.ndarray, na: int, nb: int, c: np.ndarray) -> np.ndarray:
    """sigma = H c for the (na, nb) sector, computed one connection at a time."""
    h, eri, c = _c(h), _c(eri), _c(c)
    n = h.shape[0]
    N = binom(n, na) * binom(n, nb)
    assert c.shape == (N,)
    out = np.zeros(max(N, 1))
    assert lib().oracle_sigma(n, na, nb, _ptr(h), _ptr(eri), _ptr(c), _ptr(out)) == 0
    return out[:N]


def sigma_rows(h: np.ndarray, eri: np.ndarray, na: int, nb: int, c: np.ndarray,
               rows) -> np.ndarray:
    """Selected rows of H c, each from the connections of that determinant."""
    h, eri, c = _c(h), _c(eri), _c(c)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.zeros(max(len(rows), 1))
    assert lib().oracle_sigma_rows(h.shape[0], na, nb, _ptr(h), _ptr(eri), _ptr(c), len(rows),
                                   _ptr(rows), _ptr(out)) == 0
    return out[: len(rows)]


def rdm12(n: int, na: int, nb: int, c: np.ndarray, two_body: bool = True):
    """Spin-free 1-RDM gamma[p, q] and 2-RDM Gamma[p, q, r, s] (chemists' order) of c."""
    c = _c(c)
    g = np.zeros(n * n)
    G = np.zeros(n ** 4) if two_body else None
    assert lib().oracle_rdm12(n, na, nb, _ptr(c), _ptr(g), _ptr(G) if two_body else None) == 0
    return g.reshape(n, n), (G.reshape(n, n, n, n) if two_body else None)


def max_connections(n: int, na: int, nb: int) -> int:
    """Most non-zero elements in one row of the (na, nb) Hamiltonian: the determinant
    itself, its single replacements of either spin, and its same-spin and
    opposite-spin double replacements.  Only sizes the choice of eigensolver."""
    sa, sb = na * (n - na), nb * (n - nb)
    daa = math.comb(na, 2) * math.comb(n - na, 2)
    dbb = math.comb(nb, 2) * math.comb(n - nb, 2)
    return 1 + sa + sb + daa + dbb + sa * sb


def lowest_eigenpair(h: np.ndarray, eri: np.ndarray, na: int, nb: int, tol: float = 1e-13,
                     want_vector: bool = False):
    """Lowest eigenvalue (and optionally its eigenvector) of the CAS Hamiltonian."""
    import scipy.linalg
    import scipy.sparse
    import scipy.sparse.linalg

    n = h.shape[0]
    N = binom(n, na) * binom(n, nb)
    if N == 0:
        raise ValueError("empty determinant space")
    if N <= DENSE_MAX:
        H = h_dense(h, eri, na, nb)
        w, v = scipy.linalg.eigh(H, subset_by_index=[0, 0])
        return (float(w[0]), v[:, 0]) if want_vector else float(w[0])
    conn = max_connections(n, na, nb)
    v0 = np.cos(np.arange(N) * 0.7311) + 0.1  # deterministic start vector
    if N * conn <= SPARSE_MAX_ENTRIES:
        rows, cols, vals = h_coo(h, eri, na, nb)
        A = scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(N, N))
    else:
        A = scipy.sparse.linalg.LinearOperator((N, N), matvec=lambda x: sigma(h, eri, na, nb, x),
                                               dtype=np.float64)
    w, v = scipy.sparse.linalg.eigsh(A, k=1, which="SA", tol=tol, v0=v0, ncv=min(N, 40))
    return (float(w[0]), v[:, 0]) if want_vector else float(w[0])


def lowest_eigenvalue(h, eri, na, nb, tol: float = 1e-13) -> float:
    return lowest_eigenpair(h, eri, na, nb, tol=tol)


def even_sector_basis(n: int, ne: int):
    """Orthonormal basis (sparse, N x M) of the determinant vectors that are even
    under the exchange of the alpha and beta strings, c[Ia][Ib] = c[Ib][Ia]
    (n_alpha = n_beta = ne): e_d for Ia = Ib, (e_d + e_Pd)/sqrt(2) for Ia < Ib."""
    import scipy.sparse

    ns = binom(n, ne)
    rows, cols, vals = [], [], []
    m = 0
    for ia in range(ns):
        for ib in range(ia, ns):
            d, pd = ia * ns + ib, ib * ns + ia
            if d == pd:
                rows.append(d)
                cols.append(m)
                vals.append(1.0)
            else:
                rows += [d, pd]
                cols += [m, m]
                vals += [2.0 ** -0.5, 2.0 ** -0.5]
            m += 1
    return scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(ns * ns, m))


def lowest_eigenvalue_even(h: np.ndarray, eri: np.ndarray, ne: int, tol: float = 1e-13) -> float:
    """Lowest eigenvalue of the CAS Hamiltonian restricted to the even sector of
    the alpha-beta string exchange (the sector of the closed-shell
    determinants; for M_S = 0 these are the states of even total spin):
    Q^T H Q with Q from even_sector_basis, by LAPACK or ARPACK."""
    import scipy.linalg
    import scipy.sparse
    import scipy.sparse.linalg

    n = h.shape[0]
    N = binom(n, ne) ** 2
    Q = even_sector_basis(n, ne)
    if N <= DENSE_MAX:
        H = h_dense(h, eri, ne, ne)
        Hq = Q.T @ (Q.T @ H.T).T
        w = scipy.linalg.eigh(np.asarray(Hq), eigvals_only=True, subset_by_index=[0, 0])
        return float(w[0])
    rows, cols, vals = h_coo(h, eri, ne, ne)
    A = scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(N, N))
    Hq = (Q.T @ A @ Q).tocsr()
    v0 = np.cos(np.arange(Hq.shape[0]) * 0.7311) + 0.1
    w = scipy.sparse.linalg.eigsh(Hq, k=1, which="SA", tol=tol, v0=v0, ncv=min(Hq.shape[0], 40),
                                  return_eigenvectors=False)
    return float(w[0])


def s2_dense(n: int, na: int, nb: int) -> np.ndarray:
    """Total spin S^2 in the (na, nb) determinant basis (index I_a * N_b + I_b).

    State targeting (the paper converges its Cr2 expansion onto the 1Sigma_g+
    ground state) needs the spin of a CASCI state; S^2 is written out here from
    its second-quantised form, S^2 = S_- S_+ + S_z (S_z + 1), with
    S_+ = sum_p a+_{p,alpha} a_{p,beta}, S_- = sum_p a+_{p,beta} a_{p,alpha} and
    S_z = (na - nb) / 2.  Each creator or annihilator acts on the 2n-bit
    determinant word (alpha spin orbitals 0..n-1, beta n..2n-1) with the sign
    (-1)^(occupied spin orbitals below it), the convention of the Hamiltonian.
    Dense; small spaces only."""
    words = [int(w) for w in dets(n, na, nb)]
    index = {w: i for i, w in enumerate(words)}
    N = len(words)
    S2 = np.zeros((N, N))

    def hop(w: int, create: int, annihilate: int):
        """a+_create a_annihilate |w>: (sign, word), or None when it vanishes."""
        if not (w >> annihilate) & 1:
            return None
        s = bin(w & ((1 << annihilate) - 1)).count("1")
        w1 = w & ~(1 << annihilate)
        if (w1 >> create) & 1:
            return None
        s += bin(w1 & ((1 << create) - 1)).count("1")
        return (-1.0 if s & 1 else 1.0), w1 | (1 << create)

    sz = 0.5 * (na - nb)
    for j, w in enumerate(words):
        S2[j, j] += sz * (sz + 1.0)
        for p in range(n):  # S_+: the beta electron of orbital p becomes alpha
            r1 = hop(w, p, n + p)
            if r1 is None:
                continue
            for q in range(n):  # S_-: the alpha electron of orbital q becomes beta
                r2 = hop(r1[1], n + q, q)
                if r2 is None:
                    continue
                S2[index[r2[1]], j] += r1[0] * r2[0]
    return S2


def lowest_eigenvalue_spin(h: np.ndarray, eri: np.ndarray, ne: int, spin: float = 0.0) -> float:
    """Lowest eigenvalue of the CAS Hamiltonian (n_alpha = n_beta = ne) among the
    states of total spin S = `spin`: H restricted to the eigenspace of S^2 with
    eigenvalue S(S+1) (H and S^2 commute), by LAPACK.  Dense; small spaces only."""
    import scipy.linalg

    n = h.shape[0]
    H = h_dense(h, eri, ne, ne)
    w, U = scipy.linalg.eigh(s2_dense(n, ne, ne))
    Q = U[:, np.abs(w - spin * (spin + 1.0)) < 1e-6]
    if Q.shape[1] == 0:
        raise ValueError(f"no state of spin {spin} in this space")
    return float(scipy.linalg.eigh(Q.T @ H @ Q, eigvals_only=True, subset_by_index=[0, 0])[0])
