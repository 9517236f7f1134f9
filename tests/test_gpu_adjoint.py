"""Adjoint (density-matrix gradients of the MBE energy) on the GPU.

Checked against the oracle adjoint (weights and full gradients on small
systems), against central finite differences of GPU energies on the L=46
Hubbard ring (dE/dt, dE/dU) and on the 20-orbital molecule (dE/dh_pq and
dE/d(pq|rs) symmetry orbits at orders 1-2; directional derivatives over 50
random integral entries and over all of them at orders 1-3), and against the
exact Hubbard homogeneity
t dE/dt + U dE/dU = E and trace(gamma) = N.
"""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import adjoint, mbe as omb  # noqa: E402
from workloads import hubbard_ring_momentum, random_system, workload  # noqa: E402


@pytest.fixture(scope="module")
def eng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1910_03527_gb300 as e
    e.build()
    return e


@pytest.fixture(scope="module")
def ctx(eng):
    c = eng.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def _orbit(p, q, r, s):
    return {(p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r),
            (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)}


def test_weights_match_oracle(eng, ctx):
    h1, eri, occ, _ = hubbard_ring_momentum(8, 1.0, 2.0)
    orders = [1, 2, 3, 4, 5]
    out = eng.run_mbe(ctx, dev(h1), dev(eri), dev(occ), [], list(range(8)), orders, True)
    w, ref_w = ctx.mbe_weights(out["tuples"], list(range(8)))
    tup = {n: [tuple(r) for r in out["tuples"][i].cpu().tolist()] for i, n in enumerate(orders)}
    wo = adjoint.adjoint_weights(tup)
    for i, n in enumerate(orders):
        got = w[i].cpu().numpy()
        want = np.array([wo[t] for t in tup[n]])
        assert np.abs(got - want).max(initial=0.0) <= 1e-12
    # the reference-space weight is 1 - sum_S w(S) (the oracle's weights, summed exactly)
    want_r = 1.0 - math.fsum(wo[t] for n in orders for t in tup[n])
    assert abs(float(ref_w.item()) - want_r) <= 1e-9
    # sum_S w(S) eps(S) equals the sum of the increments
    lhs = sum(float((wi * e).sum()) for wi, e in zip(w, out["eps"]))
    rhs = float(out["e_order"].sum())
    assert abs(lhs - rhs) < 1e-10


@pytest.mark.parametrize("case", ["random_ref", "hubbard"])
def test_gradient_matches_oracle(eng, ctx, case):
    if case == "random_ref":
        h1, eri, occ = random_system(7, 3, seed=41)
        ref, exp, orders, skip = [2, 3], [0, 1, 4, 5, 6], [1, 2, 3], False
    else:
        # closed-shell ring: no tuple has a degenerate ground state, whose
        # 2-RDM (unlike its energy and 1-RDM) would not be unique
        h1, eri, occ, _ = hubbard_ring_momentum(10, 1.0, 3.0)
        ref, exp, orders, skip = [], list(range(10)), [1, 2, 3, 4], True
    E, gh_o, ge_o = adjoint.mbe_gradient(h1, eri, occ, ref, exp, orders, skip)
    gh, ge, out = eng.mbe_gradient(ctx, dev(h1), dev(eri), dev(occ), ref, exp, orders, skip,
                                   eng.Opts(tol=1e-10))
    assert abs(float(out["e_total"].item()) - E) < 1e-9
    assert np.abs(gh.cpu().numpy() - gh_o).max() < 1e-7
    assert np.abs(ge.cpu().numpy() - ge_o).max() < 1e-7
    # one-body only (warp solver path) gives the same dE/dh1
    gh1, ge1, _ = eng.mbe_gradient(ctx, dev(h1), dev(eri), dev(occ), ref, exp, orders, skip,
                                   eng.Opts(tol=1e-10), two_body=False, forward=out)
    assert ge1 is None and np.abs(gh1.cpu().numpy() - gh_o).max() < 1e-7


def test_autograd_function(eng, ctx):
    h1, eri, occ = random_system(6, 3, seed=5)
    ref, exp, orders = [2, 3], [0, 1, 4, 5], [1, 2]
    th1 = dev(h1).requires_grad_(True)
    teri = dev(eri).requires_grad_(True)
    E = eng.MBEEnergy.apply(th1, teri, ctx, dev(occ), ref, exp, orders, False, eng.Opts(tol=1e-10), True)
    (2.0 * E).sum().backward()
    _, gh_o, ge_o = adjoint.mbe_gradient(h1, eri, occ, ref, exp, orders, False)
    assert np.abs(th1.grad.cpu().numpy() - 2 * gh_o).max() < 2e-7
    assert np.abs(teri.grad.cpu().numpy() - 2 * ge_o).max() < 2e-7


def test_hubbard46_dE_dt_dU_finite_differences(eng, ctx):
    L, t, U, orders = 46, 1.0, 4.0, [1, 2, 3, 4]
    opts = eng.Opts(tol=1e-10)

    def energy(tt, uu):
        h1, eri, occ, _ = hubbard_ring_momentum(L, tt, uu)
        out = eng.run_mbe(ctx, dev(h1), dev(eri), dev(occ), [], list(range(L)), orders, True, opts,
                          occ_host=occ.tolist())
        return float(out["e_total"].item())

    h1, eri, occ, _ = hubbard_ring_momentum(L, t, U)
    gh, ge, out = eng.mbe_gradient(ctx, dev(h1), dev(eri), dev(occ), [], list(range(L)), orders, True, opts,
                                   occ_host=occ.tolist())
    E = float(out["e_total"].item())
    dEdt = float((gh * dev(h1)).sum()) / t
    dEdU = float((ge * dev(eri)).sum()) / U
    assert abs(t * dEdt + U * dEdU - E) < 1e-8
    assert abs(float(torch.trace(gh)) - L) < 1e-8
    d = 1e-4
    fd_t = (energy(t + d, U) - energy(t - d, U)) / (2 * d)
    fd_U = (energy(t, U + d) - energy(t, U - d)) / (2 * d)
    assert abs(fd_t - dEdt) < 1e-6 * max(1.0, abs(dEdt)), (fd_t, dEdt)
    assert abs(fd_U - dEdU) < 1e-6 * max(1.0, abs(dEdU)), (fd_U, dEdU)


def test_molecule20_gradient_finite_differences(eng, ctx):
    # The 20-orbital truncation of the synthetic molecule, orders 1-2 here: its
    # tuple ground states are strongly multi-configurational (the lowest diagonal
    # element lies ~10 E_h above the ground state), so higher orders need hundreds
    # of Davidson iterations per tuple for each of the 20 finite-difference energies.
    w = workload("molecule20")
    orders = [1, 2]
    opts = eng.Opts(tol=1e-9)
    occ_d = dev(w.occ)

    def energy(h, e):
        out = eng.run_mbe(ctx, dev(h), dev(e), occ_d, w.ref, w.exp, orders, w.skip, opts,
                          occ_host=w.occ.tolist())
        assert all(bool((s == 0).all()) for s in out["status"])
        return float(out["e_total"].item())

    gh, ge, fwd = eng.mbe_gradient(ctx, dev(w.h1), dev(w.eri), occ_d, w.ref, w.exp, orders, w.skip, opts,
                                   occ_host=w.occ.tolist())
    assert all(bool((s == 0).all()) for s in fwd["status"])
    gh, ge = gh.cpu().numpy(), ge.cpu().numpy()
    rng = np.random.default_rng(20)
    d = 1e-4
    for _ in range(5):
        p, q = (int(x) for x in rng.integers(0, 20, size=2))
        hp, hm = w.h1.copy(), w.h1.copy()
        for (a, b) in {(p, q), (q, p)}:
            hp[a, b] += d
            hm[a, b] -= d
        fd = (energy(hp, w.eri) - energy(hm, w.eri)) / (2 * d)
        want = gh[p, q] + (gh[q, p] if p != q else 0.0)
        assert abs(fd - want) < 1e-6 * max(1.0, abs(want)), ("h", p, q, fd, want)
    for _ in range(5):
        idx = tuple(int(x) for x in rng.integers(0, 20, size=4))
        orbit = _orbit(*idx)
        ep, em = w.eri.copy(), w.eri.copy()
        for o in orbit:
            ep[o] += d
            em[o] -= d
        fd = (energy(w.h1, ep) - energy(w.h1, em)) / (2 * d)
        want = sum(ge[o] for o in orbit)
        assert abs(fd - want) < 1e-6 * max(1.0, abs(want)), ("eri", idx, fd, want)


def _symmetric_h_direction(rng, n, entries):
    """Random symmetric one-body direction on `entries` random (p, q) pairs."""
    D = np.zeros((n, n))
    for _ in range(entries):
        p, q = (int(x) for x in rng.integers(0, n, size=2))
        D[p, q] = D[q, p] = rng.normal()
    return D


def _symmetric_eri_direction(rng, n, orbits):
    """Random direction with the 8-fold symmetry of (pq|rs) on `orbits` random orbits."""
    D = np.zeros((n,) * 4)
    for _ in range(orbits):
        v = rng.normal()
        for o in _orbit(*(int(x) for x in rng.integers(0, n, size=4))):
            D[o] = v
    return D


def test_molecule20_directional_derivatives_orders_1_3(eng, ctx):
    # Directional derivatives of the orders 1-3 MBE energy of the 20-orbital
    # molecule (364 order-3 tuples of 9 orbitals, 15,876 determinants, block
    # solver): dE along D = sum_pq dE/dh_pq D_pq + sum_pqrs dE/d(pq|rs) D_pqrs
    # from the adjoint, against the central difference of two GPU energies.
    # Three directions: 25 random one-body entries, 25 random two-electron
    # symmetry orbits (50 integral entries in all), and a dense direction over
    # every entry of both; each is scaled to unit norm.
    directional_check(eng, ctx, [1, 2, 3])


def directional_check(eng, ctx, orders):
    w = workload("molecule20")
    opts = eng.Opts(tol=1e-9)
    occ_d = dev(w.occ)

    def energy(h, e):
        out = eng.run_mbe(ctx, dev(h), dev(e), occ_d, w.ref, w.exp, orders, w.skip, opts,
                          occ_host=w.occ.tolist())
        assert all(bool((s == 0).all()) for s in out["status"])
        return float(out["e_total"].item())

    gh, ge, fwd = eng.mbe_gradient(ctx, dev(w.h1), dev(w.eri), occ_d, w.ref, w.exp, orders, w.skip, opts,
                                   occ_host=w.occ.tolist())
    assert all(bool((s == 0).all()) for s in fwd["status"])
    gh, ge = gh.cpu().numpy(), ge.cpu().numpy()
    n = w.h1.shape[0]
    rng = np.random.default_rng(2020)
    dense_h = rng.normal(size=(n, n))
    dense_e = rng.normal(size=(n,) * 4)
    dense_e = sum(np.transpose(dense_e, p) for p in
                  [(0, 1, 2, 3), (1, 0, 2, 3), (0, 1, 3, 2), (1, 0, 3, 2),
                   (2, 3, 0, 1), (3, 2, 0, 1), (2, 3, 1, 0), (3, 2, 1, 0)]) / 8.0
    directions = {
        "h entries": (_symmetric_h_direction(rng, n, 25), np.zeros((n,) * 4)),
        "eri orbits": (np.zeros((n, n)), _symmetric_eri_direction(rng, n, 25)),
        "dense": ((dense_h + dense_h.T) / 2.0, dense_e),
    }
    d = 1e-4
    for name, (Dh, De) in directions.items():
        norm = math.sqrt(float((Dh * Dh).sum() + (De * De).sum()))
        Dh, De = Dh / norm, De / norm
        want = float((gh * Dh).sum() + (ge * De).sum())
        fd = (energy(w.h1 + d * Dh, w.eri + d * De) - energy(w.h1 - d * Dh, w.eri - d * De)) / (2 * d)
        assert abs(fd - want) < 1e-6 * max(1.0, abs(want)), (name, fd, want)
