"""Parity of the CUDA path (through the C ABI) with the oracle.

Bit-exact: tuple lists, string tables and addressing.  Floating point: sigma
element by element (1e-11 relative to the largest |sigma|); tuple energies,
increments and totals within 1e-9 E_h in float64 mode and 1e-8 E_h in mixed
mode, except where a test states a wider bound and its reason.
"""

import itertools
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

# a tuple energy is valid with status OK (0) or DEGENERATE (4: the two spin-flip
# sectors' lowest eigenvalues coincide; the energy is unique, the state is not)
VALID = (0, 4)

from fock_space import annihilators  # noqa: E402
from oracle import fci, mbe as omb  # noqa: E402
from workloads import (hubbard_ring_momentum, random_system, workload)  # noqa: E402

TOL = {"fp64": 1e-9, "mixed": 1e-8}


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


def run_gpu(eng, ctx, w, orders, prec="fp64"):
    return eng.run_mbe(ctx, dev(w.h1), dev(w.eri), dev(w.occ), w.ref, w.exp, orders, w.skip,
                       eng.Opts(precision=prec), occ_host=w.occ.tolist())


# ----------------------------------------------------------------------------- a1, a3

@pytest.mark.parametrize("name", ["hubbard8", "hubbard22", "molecule40", "hubbard46"])
def test_tuples_bit_exact(eng, ctx, name):
    w = workload(name)
    for n in w.orders:
        got = ctx.mbe_tuples(w.norb, w.occ.tolist(), w.exp, w.ref, n, w.skip).cpu().numpy()
        want = omb.tuples(w.exp, w.ref, w.occ, n, w.skip)
        assert got.shape == (len(want), n)
        if len(want):
            assert np.array_equal(got, np.array(want, dtype=np.int32)), (name, n)


def test_tuples_unsorted_expansion_and_reference(eng, ctx):
    occ = [1, 1, 1, 0, 0, 0, 0, 0, 1, 0]
    exp = [9, 3, 0, 7, 5, 2]
    ref = [1, 4]
    for n in range(1, 5):
        for skip in (False, True):
            got = ctx.mbe_tuples(10, occ, exp, ref, n, skip).cpu().numpy()
            want = omb.tuples(exp, ref, np.array(occ), n, skip)
            assert got.tolist() == [list(t) for t in want]


@pytest.mark.parametrize("n,k", [(1, 1), (2, 1), (4, 2), (6, 3), (7, 2), (8, 4), (10, 5), (12, 6),
                                 (5, 0), (5, 5)])
def test_string_tables_bit_exact(eng, ctx, n, k):
    strings, table = ctx.mbe_string_table(n, k)
    strings = strings.cpu().numpy().astype(np.uint64)
    assert np.array_equal(strings, fci.strings(n, k))
    table = table.cpu().numpy()
    index = {int(s): i for i, s in enumerate(strings.tolist())}
    a = annihilators(n) if n <= 8 else None
    for i, s in enumerate(strings.tolist()):
        want = []
        for q in range(n):
            if not (s >> q) & 1:
                continue
            for p in range(n):
                if p != q and (s >> p) & 1:
                    continue
                J = (s & ~(1 << q)) | (1 << p)
                if a is not None:
                    sign = (a[p].T @ a[q])[J, s]
                else:
                    lo, hi = min(p, q), max(p, q)
                    sign = (-1) ** bin(s & (((1 << hi) - 1) & ~((1 << (lo + 1)) - 1))).count("1")
                hi, lo = max(p, q), min(p, q)
                want.append((index[J] << 9) | ((hi * (hi + 1) // 2 + lo) << 1) | int(sign < 0))
        assert table[i].tolist() == want


# ----------------------------------------------------------------------------- a2, a4, a5

@pytest.mark.parametrize("case", [
    ("random", 10, 5, [1, 2, 4, 5, 7, 8]),       # (3e,6o)-like: 3 occ in A
    ("random", 12, 6, [0, 2, 3, 5, 6, 7, 9, 11]),
    ("random", 12, 6, list(range(12))),          # (6e,12o): 853,776 determinants
    ("hubbard", 8, 4, [0, 1, 2, 3, 4, 5, 6, 7]),
    ("hubbard", 22, 11, [3, 7, 9, 11, 12, 15, 20]),
])
def test_sigma_and_diagonal_parity(eng, ctx, case):
    kind, N, nocc, A = case
    if kind == "random":
        h1, eri, occ = random_system(N, nocc, seed=N + len(A))
    else:
        h1, eri, occ, _ = hubbard_ring_momentum(N, 1.0, 3.0)
    e_core, h_eff, eri_a = omb.frozen_core(h1, eri, occ, A)
    k = omb.n_active_electrons(occ, A)
    ndet = fci.binom(len(A), k) ** 2
    c = np.random.default_rng(7).normal(size=ndet)
    sig, diag = ctx.casci_sigma(dev(h1), dev(eri), dev(occ), A, dev(c))
    sig, diag = sig.cpu().numpy(), diag.cpu().numpy()
    if ndet <= 50_000:
        want = fci.sigma(h_eff, eri_a, k, k, c)
        scale = np.abs(want).max()
        assert np.abs(sig - want).max() <= 1e-11 * scale
        want_d = fci.hdiag(h_eff, eri_a, k, k)
        assert np.abs(diag - want_d).max() <= 1e-11 * np.abs(want_d).max()
    else:
        # Sampled rows: (H c)_I one determinant at a time from the Slater-Condon rules.
        rows = np.random.default_rng(3).choice(ndet, size=200, replace=False)
        want = fci.sigma_rows(h_eff, eri_a, k, k, c, rows)
        assert np.abs(sig[rows] - want).max() <= 1e-11 * np.abs(want).max()


# ----------------------------------------------------------------------------- a6, a7, a8, a9

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_mbe_hubbard8(eng, ctx, prec):
    w = workload("hubbard8")
    ref = omb.run_mbe(w.h1, w.eri, w.occ, w.ref, w.exp, w.orders, w.skip)
    out = run_gpu(eng, ctx, w, w.orders, prec)
    tol = TOL[prec]
    for i, n in enumerate(w.orders):
        tup = [tuple(r) for r in out["tuples"][i].cpu().tolist()]
        assert tup == list(ref["eps"][n].keys())
        assert np.isin(out["status"][i].cpu().numpy(), VALID).all()
        eps = out["eps"][i].cpu().numpy()
        want = np.array([ref["eps"][n][t] for t in tup])
        assert np.abs(eps - want).max() <= tol, (n, np.abs(eps - want).max())
        inc = out["inc"][i].cpu().numpy()
        want_i = np.array([ref["inc"][t] for t in tup])
        assert np.abs(inc - want_i).max() <= tol
    e_order = out["e_order"].cpu().numpy()
    for i, n in enumerate(w.orders):
        assert abs(e_order[i] - ref["e_order"][n]) <= tol
    fci_e = fci.lowest_eigenvalue(w.h1, w.eri, 4, 4)
    assert abs(float(out["e_total"].item()) - fci_e) <= tol
    assert abs(float(out["e_phi"].item()) - ref["e_phi"]) <= 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_mbe_with_reference_space(eng, ctx, prec):
    h1, eri, occ = random_system(9, 4, seed=31)
    ref_space, exp = [2, 3, 4, 5], [0, 1, 6, 7, 8]
    orders = [1, 2, 3]
    ref = omb.run_mbe(h1, eri, occ, ref_space, exp, orders, skip=False)
    out = eng.run_mbe(ctx, dev(h1), dev(eri), dev(occ), ref_space, exp, orders, False,
                      eng.Opts(precision=prec), occ_host=occ.tolist())
    assert abs(out["e_ref_corr"] - ref["e_ref_corr"]) <= TOL[prec]
    for i, n in enumerate(orders):
        tup = [tuple(r) for r in out["tuples"][i].cpu().tolist()]
        eps = out["eps"][i].cpu().numpy()
        want = np.array([ref["eps"][n][t] for t in tup])
        assert np.abs(eps - want).max() <= TOL[prec]
    assert abs(float(out["e_total"].item()) - ref["e_tot"]) <= TOL[prec]


def _sampled_increments(w, tuples_by_order, eps_by_order, inc_by_order, order, rng, nsample, prec):
    """Oracle increments of sampled order-n tuples from the oracle energies of
    all their kept sub-tuples; compared with the GPU's eps and increments."""
    lists = {n: [tuple(r) for r in tuples_by_order[n].cpu().tolist()] for n in tuples_by_order}
    e_phi = omb.phi_energy(w.h1, w.eri, w.occ)
    e_ref = omb.ref_corr_energy(w.h1, w.eri, w.occ, w.ref)
    cache = {}

    def eps_o(t):
        if t not in cache:
            cache[t] = omb.tuple_energy(w.h1, w.eri, w.occ, w.ref, t, e_phi, e_ref)
        return cache[t]

    tl = lists[order]
    idx = rng.choice(len(tl), size=min(nsample, len(tl)), replace=False)
    gpu_eps = eps_by_order[order].cpu().numpy()
    gpu_inc = inc_by_order[order].cpu().numpy()
    worst_e = worst_i = 0.0
    for i in idx:
        t = tl[i]
        sub_eps = {}
        for m in range(1, order + 1):
            sub_eps[m] = {s: eps_o(s) for s in itertools.combinations(t, m)
                          if not w.skip or omb.keep_tuple(s, w.ref, w.occ)}
        inc = omb.increments(sub_eps)
        worst_e = max(worst_e, abs(gpu_eps[i] - sub_eps[order][t]))
        worst_i = max(worst_i, abs(gpu_inc[i] - inc[t]))
    assert worst_e <= TOL[prec], worst_e
    assert worst_i <= TOL[prec], worst_i


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_hubbard22_full_size_sampled(eng, ctx, prec):
    w = workload("hubbard22")
    out = run_gpu(eng, ctx, w, w.orders, prec)
    torch.cuda.synchronize()
    for i, n in enumerate(w.orders):
        st = out["status"][i].cpu().numpy()
        assert np.isin(st, VALID).all(), (n, np.bincount(st))
    tuples = {n: out["tuples"][i] for i, n in enumerate(w.orders)}
    eps = {n: out["eps"][i] for i, n in enumerate(w.orders)}
    inc = {n: out["inc"][i] for i, n in enumerate(w.orders)}
    rng = np.random.default_rng(22)
    for n, ns in ((2, 30), (3, 20), (4, 10), (5, 6), (6, 4)):
        _sampled_increments(w, tuples, eps, inc, n, rng, ns, prec)
    # order sums equal the sums of the returned increments
    e_order = out["e_order"].cpu().numpy()
    for i in range(len(w.orders)):
        assert abs(e_order[i] - math.fsum(out["inc"][i].cpu().numpy().tolist())) <= 1e-9


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_hubbard46_sampled(eng, ctx, prec):
    w = workload("hubbard46")
    out = run_gpu(eng, ctx, w, w.orders, prec)
    tuples = {n: out["tuples"][i] for i, n in enumerate(w.orders)}
    eps = {n: out["eps"][i] for i, n in enumerate(w.orders)}
    inc = {n: out["inc"][i] for i, n in enumerate(w.orders)}
    for i, n in enumerate(w.orders):
        assert np.isin(out["status"][i].cpu().numpy(), VALID).all()
    rng = np.random.default_rng(46)
    for n, ns in ((2, 20), (3, 15), (4, 10)):
        _sampled_increments(w, tuples, eps, inc, n, rng, ns, prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_molecule40_orders_1_2_sampled(eng, ctx, prec):
    w = workload("molecule40")
    out = run_gpu(eng, ctx, w, [1, 2], prec)
    e_ref = omb.ref_corr_energy(w.h1, w.eri, w.occ, w.ref)
    assert abs(out["e_ref_corr"] - e_ref) <= TOL[prec]
    tuples = {n: out["tuples"][i] for i, n in enumerate([1, 2])}
    eps = {n: out["eps"][i] for i, n in enumerate([1, 2])}
    inc = {n: out["inc"][i] for i, n in enumerate([1, 2])}
    for i in range(2):
        assert np.isin(out["status"][i].cpu().numpy(), VALID).all()
    rng = np.random.default_rng(40)
    _sampled_increments(w, tuples, eps, inc, 1, rng, 8, prec)
    _sampled_increments(w, tuples, eps, inc, 2, rng, 4, prec)


# ----------------------------------------------------------------------------- edge cases

def test_malformed_tuples_get_badinput_status(eng, ctx):
    h1, eri, occ, _ = hubbard_ring_momentum(6, 1.0, 2.0)
    tup = torch.tensor([[0, 3], [3, 0], [1, 1], [0, 9], [-1, 2], [2, 4]], dtype=torch.int32,
                       device="cuda")
    eps, st, _ = ctx.casci_batch(dev(h1), dev(eri), dev(occ), [], 0.0, 2, tup)
    st = st.cpu().numpy()
    assert st.tolist() == [0, 3, 3, 3, 3, 0]
    assert np.isnan(eps.cpu().numpy()[1:5]).all()
    e_phi = omb.phi_energy(h1, eri, occ)
    want = omb.tuple_energy(h1, eri, occ, [], (0, 3), e_phi, 0.0)
    assert abs(eps[0].item() - want) <= 1e-9
    # a tuple that overlaps the reference space is malformed too
    eps, st, _ = ctx.casci_batch(dev(h1), dev(eri), dev(occ), [3], 0.0, 1,
                                 torch.tensor([[3], [4]], dtype=torch.int32, device="cuda"))
    assert st.cpu().tolist() == [3, 0]


def test_single_determinant_tuples_are_exactly_zero(eng, ctx):
    h1, eri, occ, _ = hubbard_ring_momentum(8, 1.0, 2.0)
    tup = torch.tensor([[0, 1, 2], [4, 5, 6], [1, 2, 3], [5, 6, 7]], dtype=torch.int32, device="cuda")
    eps, st, it = ctx.casci_batch(dev(h1), dev(eri), dev(occ), [], 0.0, 3, tup)
    assert st.cpu().tolist() == [0, 0, 0, 0]
    assert eps.cpu().tolist() == [0.0, 0.0, 0.0, 0.0]


def test_empty_batch_and_order_zero(eng, ctx):
    h1, eri, occ = random_system(7, 3, seed=2)
    t = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
    eps, st, _ = ctx.casci_batch(dev(h1), dev(eri), dev(occ), [], 0.0, 2, t, n_tuples=0)
    assert eps.numel() == 0
    eps, st, _ = ctx.casci_batch(dev(h1), dev(eri), dev(occ), [1, 2, 3, 4], 0.0, 0, None)
    want = omb.ref_corr_energy(h1, eri, occ, [1, 2, 3, 4])
    assert st.item() == 0 and abs(eps.item() - want) <= 1e-9


def test_invalid_arguments_raise(eng, ctx):
    h1, eri, occ = random_system(5, 2, seed=1)
    with pytest.raises(eng.MbeError):
        ctx.casci_batch(dev(h1), dev(eri), dev(occ), [0, 0], 0.0, 1,
                        torch.tensor([[1]], dtype=torch.int32, device="cuda"))
    with pytest.raises(eng.MbeError):
        ctx.mbe_tuples(5, occ.tolist(), [0, 1, 1], [], 2, False)
    with pytest.raises(eng.MbeError):
        ctx.casci_batch(dev(h1), dev(eri), dev(occ), [], 0.0, 13,
                        torch.zeros((1, 13), dtype=torch.int32, device="cuda"))


def test_maxiter_status_is_reported(eng, ctx):
    h1, eri, occ, _ = hubbard_ring_momentum(8, 1.0, 4.0)
    tup = torch.tensor([[1, 2, 3, 4, 5, 6]], dtype=torch.int32, device="cuda")
    eps, st, it = ctx.casci_batch(dev(h1), dev(eri), dev(occ), [], 0.0, 6, tup,
                                  eng.Opts(max_iter=1, tol=1e-12))
    assert st.item() == 1 and np.isfinite(eps.item())


def test_deterministic_results(eng, ctx):
    w = workload("hubbard8")
    a = run_gpu(eng, ctx, w, [1, 2, 3, 4], "fp64")
    b = run_gpu(eng, ctx, w, [1, 2, 3, 4], "fp64")
    for x, y in zip(a["eps"], b["eps"]):
        assert torch.equal(x, y)
    assert torch.equal(a["e_total"], b["e_total"])
