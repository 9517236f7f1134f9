"""The allocation-free sigma entry point, casci_sigma_noalloc.

Some callers cannot allocate device memory when they call into the library
(their device memory belongs to their own pool, or an allocation would stall or
be illegal in their execution model).  casci_sigma_noalloc serves them with a
fixed device scratch array instead of a context workspace.  This test calls it
through the C ABI twice in a row, on two different active spaces (the second
call reuses the scratch the first one left behind), and checks both results
against the regular casci_sigma entry point with the tolerance of the sigma
parity tests.  It also checks that a problem beyond the fixed limit is refused.

This file is named so that pytest collects it last.
"""

import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import mbe as omb  # noqa: E402
from workloads import hubbard_ring_momentum, random_system  # noqa: E402


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _noalloc(lib, h1, eri, occ, A, k, c, want_diag=True):
    sigma = torch.empty_like(c)
    diag = torch.empty_like(c) if want_diag else None
    A_h = (ctypes.c_int32 * len(A))(*A)
    stream = torch.cuda.current_stream()
    rc = lib.casci_sigma_noalloc(0, ctypes.c_void_p(stream.cuda_stream), h1.shape[0], _ptr(h1), _ptr(eri),
                                 _ptr(occ), len(A), A_h, k, _ptr(c), _ptr(sigma),
                                 _ptr(diag) if diag is not None else None)
    return rc, sigma, diag


def test_noalloc_sigma_matches_casci_sigma_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1910_03527_gb300 as eng
    eng.build()
    lib = eng.lib()
    ctx = eng.Context(0)
    h1a, eria, occa = random_system(12, 6, seed=17)
    h1b, erib, occb, _ = hubbard_ring_momentum(22, 1.0, 4.0)
    cases = [(h1a, eria, occa, [0, 2, 3, 5, 6, 7, 9, 10, 11]), (h1b, erib, occb, [3, 7, 9, 11, 12, 15])]
    for call, (h1, eri, occ, A) in enumerate(cases):
        k = omb.n_active_electrons(occ, A)
        ndet = math.comb(len(A), k) ** 2
        c = _dev(np.random.default_rng(call).normal(size=ndet))
        th1, teri, tocc = _dev(h1), _dev(eri), _dev(occ)
        want_s, want_d = ctx.casci_sigma(th1, teri, tocc, A, c)
        rc, got_s, got_d = _noalloc(lib, th1, teri, tocc, A, k, c)
        assert rc == 0, lib.mbe_last_error().decode()
        torch.cuda.synchronize()
        ws, gs = want_s.cpu().numpy(), got_s.cpu().numpy()
        wd, gd = want_d.cpu().numpy(), got_d.cpu().numpy()
        assert np.abs(gs - ws).max() <= 1e-11 * np.abs(ws).max(), call
        assert np.abs(gd - wd).max() <= 1e-11 * np.abs(wd).max(), call
    ctx.close()


def test_noalloc_rejects_problems_beyond_its_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1910_03527_gb300 as eng
    lib = eng.lib()
    h1, eri, occ = random_system(12, 6, seed=3)
    th1, teri, tocc = _dev(h1), _dev(eri), _dev(occ)
    c = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc, _, _ = _noalloc(lib, th1, teri, tocc, list(range(11)), 5, c)
    assert rc == -4
    assert "allocation-free limit" in lib.mbe_last_error().decode()


def test_noalloc_diagonal_in_scratch_and_explicit_sector():
    """Two paths the casci_sigma comparison cannot reach: the diagonal kept in the
    fixed array (diag NULL; the 10-orbital, 5-electron space, the largest within
    the limit of 10 orbitals, needs about 1.1 MB of the 2 MiB), and an electron
    count other than the reference occupation gives
    (n_el = 2 in a space whose occupied count is 3), checked against the oracle's
    sigma of that sector."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1910_03527_gb300 as eng
    from oracle import fci
    eng.build()
    lib = eng.lib()
    h1, eri, occ = random_system(12, 6, seed=23)
    th1, teri, tocc = _dev(h1), _dev(eri), _dev(occ)
    for A, k in ((list(range(1, 11)), 5), ([1, 3, 4, 6, 8, 9], 2)):
        ndet = math.comb(len(A), k) ** 2
        c = _dev(np.random.default_rng(k).normal(size=ndet))
        rc, got, _ = _noalloc(lib, th1, teri, tocc, A, k, c, want_diag=False)
        assert rc == 0, lib.mbe_last_error().decode()
        torch.cuda.synchronize()
        e_core, h_eff, eri_a = omb.frozen_core(h1, eri, occ, A)
        if ndet <= 50_000:
            want = fci.sigma(h_eff, eri_a, k, k, c.cpu().numpy())
            assert np.abs(got.cpu().numpy() - want).max() <= 1e-11 * np.abs(want).max()
        else:
            rows = np.random.default_rng(5).choice(ndet, size=300, replace=False)
            want = fci.sigma_rows(h_eff, eri_a, k, k, c.cpu().numpy(), rows)
            assert np.abs(got.cpu().numpy()[rows] - want).max() <= 1e-11 * np.abs(want).max()
