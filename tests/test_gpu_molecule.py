"""The block solver at the synthetic 40-orbital molecule's full tuple sizes.

Order-3 and order-4 tuples of the (6e,6o) reference space {5..10} expanded over
the other 34 orbitals: active spaces of 9 and 10 orbitals, 7,056 to 63,504
determinants, Davidson vectors in the HBM workspace.  The expected energies are
the oracle's (tests/golden/molecule40_sample.json, written by
tests/golden/make_molecule_sample.py): the lowest eigenvalue of the whole
determinant space and of the even sector of the alpha-beta string exchange.  In
9 of the 35 sampled tuples the lowest state is odd under that exchange, 0.05 to
0.48 E_h below the lowest even state, so a wrong decision between the two
sectors cannot pass.
"""

import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

# a tuple energy is valid with status OK (0) or DEGENERATE (4: the two spin-flip
# sectors' lowest eigenvalues coincide; the energy is unique, the state is not)
VALID = (0, 4)

from workloads import workload  # noqa: E402

TOL = {"fp64": 1e-9, "mixed": 1e-8}
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "molecule40_sample.json")


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
def sample():
    return json.load(open(GOLDEN))


def test_sample_holds_both_sectors(sample):
    rows = sample["tuples"]
    odd = [r for r in rows if r["eps"] < r["eps_even"] - 1e-6]
    assert len(odd) >= 5 and len(rows) - len(odd) >= 5
    assert {r["order"] for r in rows} == {3, 4}
    assert max(r["ndet"] for r in rows) == 63504


@pytest.mark.parametrize("even_only", [False, True])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("order", [3, 4])
def test_block_solver_tuple_energies(eng, ctx, sample, order, prec, even_only):
    w = workload("molecule40")
    rows = [r for r in sample["tuples"] if r["order"] == order]
    dev = torch.device("cuda", 0)
    h1, eri, occ = (torch.tensor(np.ascontiguousarray(x), device=dev) for x in (w.h1, w.eri, w.occ))
    tup = torch.tensor([r["tuple"] for r in rows], dtype=torch.int32, device=dev)
    opts = eng.Opts(precision=prec, even_only=even_only)
    eps, st, it = ctx.casci_batch(h1, eri, occ, w.ref, sample["e_ref_corr"], order, tup, opts)
    eps, st = eps.cpu().numpy(), st.cpu().numpy()
    want = np.array([r["eps_even" if even_only else "eps"] for r in rows])
    assert np.isin(st, VALID).all(), st
    err = np.abs(eps - want)
    assert err.max() <= TOL[prec], [(r["tuple"], float(e)) for r, e in zip(rows, err) if e > TOL[prec]]
