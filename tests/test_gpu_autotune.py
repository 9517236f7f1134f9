"""The autotuner of casci_batch's launch choices (mbe_autotune, mbe_tuning).

It times candidates of each launch choice on a sample of one order's tuples and
keeps the fastest; the energies must not depend on the choice (only the launch
shapes, the warp/block split and the block solver's basis size change), and the
choice must be one of the candidates.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from workloads import workload  # noqa: E402


@pytest.fixture(scope="module")
def eng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1910_03527_gb300 as e
    e.build()
    return e


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_autotune_choice_and_invariant_energies(eng, prec):
    ctx = eng.Context(0)
    w = workload("hubbard22")
    dev = torch.device("cuda", 0)
    h1, eri, occ = (torch.tensor(np.ascontiguousarray(x), device=dev) for x in (w.h1, w.eri, w.occ))
    tup = ctx.mbe_tuples(w.norb, w.occ.tolist(), w.exp, w.ref, 5, w.skip)
    sample = tup[::8].contiguous()
    opts = eng.Opts(precision=prec)
    default = ctx.get_tuning(prec, 5)
    assert default == dict(warp_max_ndet=416, warp_warps=4, block_basis=20)
    e_def, st_def, _ = ctx.casci_batch(h1, eri, occ, w.ref, 0.0, 5, sample, opts)
    best, recs = ctx.autotune(h1, eri, occ, w.ref, 0.0, 5, sample, opts)
    assert len(recs) == 8 and all(ms > 0 for _, ms in recs)
    assert best["warp_warps"] in (2, 4) and best["warp_max_ndet"] in (100, 225, 416)
    assert best["block_basis"] in (12, 16, 20)
    assert ctx.get_tuning(prec, 5) == best  # set on the context for |R| + order = 5
    assert ctx.get_tuning(prec, 6) == default  # other sizes untouched
    e_tun, st_tun, _ = ctx.casci_batch(h1, eri, occ, w.ref, 0.0, 5, sample, opts)
    tol = 1e-9 if prec == "fp64" else 1e-8
    assert np.isin(st_tun.cpu().numpy(), (0, 4)).all()
    assert np.abs(e_tun.cpu().numpy() - e_def.cpu().numpy()).max() <= tol
    # every candidate of the split between the solvers gives the same energies
    for nd in (100, 225):
        ctx.set_tuning(prec, 5, nd, 4, 20)
        e_nd, st_nd, _ = ctx.casci_batch(h1, eri, occ, w.ref, 0.0, 5, sample, opts)
        assert np.abs(e_nd.cpu().numpy() - e_def.cpu().numpy()).max() <= tol, nd
    with pytest.raises(eng.MbeError):
        ctx.set_tuning(prec, 5, 500, 4, 20)
    ctx.close()
