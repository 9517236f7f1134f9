"""The oracle MBE of a whole workload, with its tuple CASCIs spread over host
processes (test infrastructure: used by the full-size parity tests and by the
script that writes tests/golden/oracle_totals.json).

The arithmetic is oracle/mbe.py's, unchanged: tuples(), tuple_energy() for every
tuple, then the literal increments() (Eq. 2) and order_sums() (Eq. 1) in the
parent process.  Only the loop over tuple energies is split into chunks, which
"spawn" worker processes evaluate (a forked child of a process that already
used the GPU can hang; a spawned one starts clean).
"""

from __future__ import annotations

import math
import multiprocessing as mp
import os

from oracle import mbe as omb
from workloads import workload

_W = None
_E = None


def _init(name):
    global _W, _E
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    _W = workload(name)
    e_phi = omb.phi_energy(_W.h1, _W.eri, _W.occ)
    _E = (e_phi, omb.ref_corr_energy(_W.h1, _W.eri, _W.occ, _W.ref))


def _chunk(tuples):
    return [omb.tuple_energy(_W.h1, _W.eri, _W.occ, _W.ref, t, _E[0], _E[1]) for t in tuples]


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_mbe_parallel(name: str, orders=None, procs: int | None = None, chunk: int = 256):
    """omb.run_mbe on workload `name` (orders default to the workload's), with the
    tuple energies computed by `procs` spawned processes.  Same result dict."""
    w = workload(name)
    orders = list(w.orders if orders is None else orders)
    procs = procs or host_cores()
    e_phi = omb.phi_energy(w.h1, w.eri, w.occ)
    e_ref = omb.ref_corr_energy(w.h1, w.eri, w.occ, w.ref)
    lists = {n: omb.tuples(w.exp, w.ref, w.occ, n, w.skip) for n in orders}
    work = [(n, lists[n][i:i + chunk]) for n in orders for i in range(0, len(lists[n]), chunk)]
    eps_by_order = {n: {} for n in orders}
    with mp.get_context("spawn").Pool(procs, initializer=_init, initargs=(name,)) as pool:
        results = pool.map(_chunk, [c for _, c in work], chunksize=1)
    for (n, c), vals in zip(work, results):
        for t, e in zip(c, vals):
            eps_by_order[n][t] = e
    inc = omb.increments(eps_by_order)
    e_order = omb.order_sums(inc, orders)
    e_corr = math.fsum([e_ref] + [e_order[n] for n in orders])
    return dict(e_phi=e_phi, e_ref_corr=e_ref, eps=eps_by_order, inc=inc, e_order=e_order, e_corr=e_corr,
                e_tot=e_phi + e_corr)
