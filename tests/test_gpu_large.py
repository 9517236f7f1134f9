"""One large active space on the whole GPU: casci_sigma_large and casci_solve.

Parity: sigma element by element against casci_sigma (<= 12 orbitals) and,
beyond the oracle's reach for a full sigma, on sampled rows computed by the
oracle one determinant at a time from the Slater-Condon rules; eigenvalues
against the oracle's ARPACK solution, and for (12e,12o) of the synthetic
molecule a row-sampled eigen-residual |(H c)_I - lambda c_I| of the GPU vector.
"""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

# a tuple energy is valid with status OK (0) or DEGENERATE (4: the two spin-flip
# sectors' lowest eigenvalues coincide; the energy is unique, the state is not)
VALID = (0, 4)

from oracle import fci, mbe as omb  # noqa: E402
from workloads import hubbard_ring_momentum, random_system, synthetic_molecule  # noqa: E402


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
def molecule():
    return synthetic_molecule(1910)


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("A", [[0, 2, 3, 5, 6, 7, 9, 11], list(range(12))])
def test_large_sigma_matches_casci_sigma(eng, ctx, A):
    h1, eri, occ = random_system(12, 6, seed=12)
    k = omb.n_active_electrons(occ, A)
    c = dev(np.random.default_rng(1).normal(size=math.comb(len(A), k) ** 2))
    want, wd = ctx.casci_sigma(dev(h1), dev(eri), dev(occ), A, c)
    got, gd = ctx.casci_sigma_large(dev(h1), dev(eri), dev(occ), A, c, "fp64", want_diag=True)
    w, g = want.cpu().numpy(), got.cpu().numpy()
    assert np.abs(g - w).max() <= 1e-11 * np.abs(w).max()
    assert np.abs(gd.cpu().numpy() - wd.cpu().numpy()).max() <= 1e-11 * np.abs(wd.cpu().numpy()).max()
    g32, _ = ctx.casci_sigma_large(dev(h1), dev(eri), dev(occ), A, c, "mixed")
    assert np.abs(g32.cpu().numpy() - w).max() <= 2e-5 * np.abs(w).max()


# float32 arithmetic: relative error of a sum of ~10^3 products of unit-scale terms
TOL_REL = {"fp64": 1e-11, "mixed": 2e-5}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_large_sigma_14_orbitals_sampled_rows(eng, ctx, molecule, prec):
    h1, eri, occ = molecule
    A = list(range(1, 15))  # (14e,14o): 11,778,624 determinants
    k = omb.n_active_electrons(occ, A)
    N = math.comb(14, k) ** 2
    assert N == 11_778_624
    rng = np.random.default_rng(14)
    c = rng.normal(size=N)
    got, _ = ctx.casci_sigma_large(dev(h1), dev(eri), dev(occ), A, dev(c), prec)
    got = got.cpu().numpy()
    _, h_eff, eri_a = omb.frozen_core(h1, eri, occ, A)
    rows = rng.choice(N, size=60, replace=False)
    want = fci.sigma_rows(h_eff, eri_a, k, k, c, rows)
    assert np.abs(got[rows] - want).max() <= TOL_REL[prec] * np.abs(want).max()


def test_large_sigma_16_orbitals_sampled_rows(eng, ctx, molecule):
    h1, eri, occ = molecule
    A = list(range(16))  # (16e,16o): 165,636,900 determinants
    k = omb.n_active_electrons(occ, A)
    N = math.comb(16, k) ** 2
    assert N == 165_636_900
    g = torch.Generator(device="cuda")
    g.manual_seed(16)
    c = torch.randn(N, dtype=torch.float64, device="cuda", generator=g)
    c_host = c.cpu().numpy()
    _, h_eff, eri_a = omb.frozen_core(h1, eri, occ, A)
    rows = np.random.default_rng(16).choice(N, size=40, replace=False)
    want = fci.sigma_rows(h_eff, eri_a, k, k, c_host, rows)
    for prec in ("fp64", "mixed"):
        got = ctx.casci_sigma_large(dev(h1), dev(eri), dev(occ), A, c, prec)[0]
        got = got[torch.as_tensor(rows, device="cuda")].cpu().numpy()
        assert np.abs(got - want).max() <= TOL_REL[prec] * np.abs(want).max(), prec


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_casci_solve_hubbard8_full_space(eng, ctx, prec):
    h1, eri, occ, _ = hubbard_ring_momentum(8, 1.0, 4.0)
    res = ctx.casci_solve(dev(h1), dev(eri), dev(occ), list(range(8)), eng.Opts(precision=prec, tol=1e-7))
    assert res["status"] in VALID
    exact = fci.lowest_eigenvalue(h1, eri, 4, 4)
    assert abs(res["lam"] - exact) < 1e-9
    assert abs(res["eps"] - (exact - omb.phi_energy(h1, eri, occ))) < 1e-9
    if prec == "mixed":
        assert res["n32"] > 0 and res["n64"] >= 1  # float64 sigmas: one per anchor


def test_casci_solve_molecule_12o_row_sampled_residual(eng, ctx, molecule):
    h1, eri, occ = molecule
    A = list(range(2, 14))  # (12e,12o): 853,776 determinants
    res = ctx.casci_solve(dev(h1), dev(eri), dev(occ), A, eng.Opts(precision="mixed", tol=1e-6, max_iter=3000),
                          want_vector=True)
    assert res["status"] in VALID and res["rnorm"] <= 1e-6, res
    c = res["c"].cpu().numpy()
    assert abs(np.linalg.norm(c) - 1.0) < 1e-10
    k = omb.n_active_electrons(occ, A)
    _, h_eff, eri_a = omb.frozen_core(h1, eri, occ, A)
    rows = np.random.default_rng(12).choice(len(c), size=200, replace=False)
    hc = fci.sigma_rows(h_eff, eri_a, k, k, c, rows)
    # the sampled components of H c - lambda c are bounded by the residual norm
    assert np.abs(hc - res["lam"] * c[rows]).max() <= 1e-6


def test_casci_solve_molecule_14o_row_sampled_residual(eng, ctx, molecule):
    """The largest CASCI of the paper's size class, (14e,14o) = 11,778,624
    determinants, solved in mixed precision (float32 sigma on the tensor cores,
    float64 anchors); 100 sampled rows of H c - lambda c from the oracle's
    Slater-Condon rows bound the GPU vector's eigen-residual."""
    h1, eri, occ = molecule
    A = list(range(1, 15))
    res = ctx.casci_solve(dev(h1), dev(eri), dev(occ), A, eng.Opts(precision="mixed", tol=1e-7, max_iter=3000),
                          want_vector=True)
    assert res["status"] in VALID and res["rnorm"] <= 1e-7, res
    assert res["n64"] >= 1 and res["n32"] > res["n64"]
    c = res["c"].cpu().numpy()
    assert len(c) == 11_778_624
    assert abs(np.linalg.norm(c) - 1.0) < 1e-10
    k = omb.n_active_electrons(occ, A)
    _, h_eff, eri_a = omb.frozen_core(h1, eri, occ, A)
    rows = np.random.default_rng(14).choice(len(c), size=100, replace=False)
    hc = fci.sigma_rows(h_eff, eri_a, k, k, c, rows)
    assert np.abs(hc - res["lam"] * c[rows]).max() <= 1e-7
