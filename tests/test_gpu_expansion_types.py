"""Parity of Type-1 and Type-2 expansions (Sec. 1, Fig. 1) against the oracle.

Type-1 expands in the occupied orbitals with every virtual in the reference
space; Type-2 expands in the virtuals with every occupied orbital (and, in the
third case, one active virtual) in the reference space.  The spaces come from
expansion_spaces; the GPU path is run_mbe (tuples, tuple CASCI, increments and
totals, all through the C ABI) and the screened run_mbe_screened.  The tuple
active spaces run from 16 determinants (warp solver) to 3136 (block solver),
the last order being the full space, so the totals must also equal FCI.
"""

import itertools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

# a tuple energy is valid with status OK (0) or DEGENERATE (4: the two spin-flip
# sectors' lowest eigenvalues coincide; the energy is unique, the state is not)
VALID = (0, 4)

from oracle import fci, mbe as omb  # noqa: E402
from workloads import random_system  # noqa: E402

CASES = {"type1": ("type1", ()), "type2": ("type2", ()), "type2_active": ("type2", (3,))}
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


@pytest.fixture(scope="module")
def system():
    h1, eri, occ = random_system(8, 3, seed=51)
    return h1, eri, occ, fci.lowest_eigenvalue(h1, eri, 3, 3)


_oracle_cache = {}


def oracle_run(system, case):
    if case not in _oracle_cache:
        from paper_1910_03527_gb300.binding import expansion_spaces
        h1, eri, occ, _ = system
        ref, exp = expansion_spaces(occ, *CASES[case])
        _oracle_cache[case] = (ref, exp, omb.run_mbe(h1, eri, occ, ref, exp, list(range(1, len(exp) + 1)), True))
    return _oracle_cache[case]


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_expansion_type_matches_oracle(eng, ctx, system, case, prec):
    h1, eri, occ, fci_e = system
    ref, exp, want = oracle_run(system, case)
    orders = list(range(1, len(exp) + 1))
    got = eng.run_mbe(ctx, dev(h1), dev(eri), dev(occ), ref, exp, orders, True, eng.Opts(precision=prec),
                      occ_host=occ.tolist())
    tol = TOL[prec]
    assert abs(got["e_ref_corr"] - want["e_ref_corr"]) <= tol
    for i, n in enumerate(orders):
        tk = [tuple(int(x) for x in r) for r in got["tuples"][i].cpu().numpy()]
        assert tk == omb.tuples(exp, ref, occ, n, True)
        assert np.isin(got["status"][i].cpu().numpy(), VALID).all()
        eps = got["eps"][i].cpu().numpy()
        assert np.abs(eps - np.array([want["eps"][n][t] for t in tk])).max() <= tol, n
        inc = got["inc"][i].cpu().numpy()
        assert np.abs(inc - np.array([want["inc"][t] for t in tk])).max() <= tol, n
    e_order = got["e_order"].cpu().numpy()
    for i, n in enumerate(orders):
        assert abs(e_order[i] - want["e_order"][n]) <= 16 * tol
    assert abs(float(got["e_total"].item()) - want["e_tot"]) <= 32 * tol
    assert abs(float(got["e_total"].item()) - fci_e) <= 32 * tol


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_screened_type2_matches_oracle(eng, ctx, system, prec):
    from paper_1910_03527_gb300.binding import expansion_spaces
    h1, eri, occ, _ = system
    ref, exp = expansion_spaces(occ, "type2")
    # Type-2 tuples hold only virtuals, so M_tup of Eq. 4 is the tuple's order; these
    # thresholds drop one order-4 tuple and the order-5 one
    t_init, m_init, a, max_order = 1.5e-2, 3, 1.5, 5
    want = omb.run_mbe_screened(h1, eri, occ, ref, exp, max_order, True, t_init=t_init, m_init=m_init, a=a)
    assert want["orders"] == [1, 2, 3, 4] and len(want["tuples"][4]) == 4
    for k in want["orders"]:
        inc = {t: want["inc"][t] for t in want["tuples"][k]}
        for child in itertools.combinations(exp, k + 1):
            best = max(abs(inc.get(s, 0.0)) for s in itertools.combinations(child, k))
            thr = omb.tuple_threshold(child, occ, t_init, m_init, a)
            assert best == 0.0 or abs(best - thr) > 1e-5
    got = eng.run_mbe_screened(ctx, dev(h1), dev(eri), dev(occ), ref, exp, max_order, True, t_init=t_init,
                               m_init=m_init, a=a, opts=eng.Opts(precision=prec), occ_host=occ.tolist())
    assert got["orders"] == want["orders"]
    tol = TOL[prec]
    for k in want["orders"]:
        tk = [tuple(int(x) for x in r) for r in got["tuples"][k - 1].cpu().numpy()]
        assert tk == want["tuples"][k]
        gi = got["inc"][k - 1].cpu().numpy()
        assert np.abs(gi - np.array([want["inc"][t] for t in tk])).max() <= tol
    assert abs(float(got["e_total"].item()) - want["e_tot"]) <= 32 * tol


@pytest.mark.parametrize("case,large_ndet", [("type1", 100), ("type2", 200)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_routed_tuples_match_oracle(eng, ctx, system, case, large_ndet, prec):
    # tuples above large_ndet determinants (441 and 3136 for Type-1, 400 to 3136 for
    # Type-2) are solved one at a time by casci_solve; the rest by casci_batch
    h1, eri, occ, fci_e = system
    ref, exp, want = oracle_run(system, case)
    orders = list(range(1, len(exp) + 1))
    got = eng.run_mbe(ctx, dev(h1), dev(eri), dev(occ), ref, exp, orders, True, eng.Opts(precision=prec),
                      occ_host=occ.tolist(), large_ndet=large_ndet)
    tol = TOL[prec]
    n_routed = 0
    for i, n in enumerate(orders):
        tk = [tuple(int(x) for x in r) for r in got["tuples"][i].cpu().numpy()]
        assert np.isin(got["status"][i].cpu().numpy(), VALID).all()
        assert int((got["iters"][i] <= 0).sum()) == 0 or n == 1
        eps = got["eps"][i].cpu().numpy()
        assert np.abs(eps - np.array([want["eps"][n][t] for t in tk])).max() <= tol, n
        n_routed += sum(1 for t in tk if _ndet(occ, ref, t) > large_ndet)
    assert n_routed >= 2
    assert abs(float(got["e_total"].item()) - fci_e) <= 32 * tol


def _ndet(occ, ref, t):
    import math
    A = list(ref) + list(t)
    k = sum(int(occ[p]) for p in A)
    return math.comb(len(A), k) ** 2


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_active_spaces_beyond_the_batched_limit(eng, ctx, prec):
    # Two decoupled 7-orbital blocks (3 occupied each, interleaved): Type-2 with six
    # active virtuals puts 12 orbitals in R, so every tuple's active space (13 and 14
    # orbitals, up to 9,018,009 determinants) is beyond casci_batch's 12.  The exact
    # eps of an active space A is the sum over blocks of the oracle CASCI of A's part
    # in that block; the cross-block order-2 increment vanishes, and the full-order
    # total is the sum of the blocks' FCI energies.
    from workloads import block_decoupled_system

    h1, eri, occ, block = block_decoupled_system(7, 3, 7, 3, seed=8)
    ref, exp = eng.expansion_spaces(occ, "type2", active=list(range(6, 12)))
    assert len(ref) == 12 and exp == [12, 13] and block[12] != block[13]
    e_phi = omb.phi_energy(h1, eri, occ)

    def e_cas_minus_phi(A):
        return sum(omb.casci_energy(h1, eri, occ, [p for p in A if block[p] == b]) - e_phi for b in (0, 1))

    e_ref = e_cas_minus_phi(ref)
    want = {t: e_cas_minus_phi(sorted(ref + list(t))) - e_ref for t in [(12,), (13,), (12, 13)]}
    got = eng.run_mbe(ctx, dev(h1), dev(eri), dev(occ), ref, exp, [1, 2], True, eng.Opts(precision=prec),
                      occ_host=occ.tolist(), large_ndet=100000)
    tol = TOL[prec]
    assert abs(got["e_ref_corr"] - e_ref) <= tol
    for i, n in enumerate([1, 2]):
        assert np.isin(got["status"][i].cpu().numpy(), VALID).all()
        tk = [tuple(int(x) for x in r) for r in got["tuples"][i].cpu().numpy()]
        eps = got["eps"][i].cpu().numpy()
        assert np.abs(eps - np.array([want[t] for t in tk])).max() <= tol
    assert abs(float(got["inc"][1][0].item())) <= tol
    fci_blocks = e_phi + e_cas_minus_phi(list(range(14)))
    assert abs(float(got["e_total"].item()) - fci_blocks) <= 32 * tol
