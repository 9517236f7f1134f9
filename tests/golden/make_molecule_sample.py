"""Writes tests/golden/molecule40_sample.json: oracle tuple energies of a seeded
sample of the synthetic 40-orbital molecule's order-3 and order-4 tuples
((6e,6o) reference space {5..10}, 34 expansion orbitals; tuple active spaces of 9
and 10 orbitals, up to 63,504 determinants), each with the lowest eigenvalue of
the whole determinant space and of the even sector of the alpha-beta string
exchange.  The sample is stratified by the number of occupied orbitals in the
tuple, so that every determinant-space size of both orders is present.  Calls
oracle/ only.

    python tests/golden/make_molecule_sample.py
"""

import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import fci, mbe as omb  # noqa: E402
from workloads import workload  # noqa: E402

PER_CLASS = {3: 5, 4: 3}  # tuples per (order, occupied count)


def one(args):
    order, t = args
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    w = workload("molecule40")
    e_phi = omb.phi_energy(w.h1, w.eri, w.occ)
    e_ref = omb.ref_corr_energy(w.h1, w.eri, w.occ, w.ref)
    A = sorted(set(w.ref) | set(t))
    k = omb.n_active_electrons(w.occ, A)
    t0 = time.time()
    e = omb.tuple_energy(w.h1, w.eri, w.occ, w.ref, t, e_phi, e_ref)
    ee = omb.tuple_energy(w.h1, w.eri, w.occ, w.ref, t, e_phi, e_ref, even_only=True)
    return dict(order=order, tuple=list(t), n=len(A), k=k, ndet=fci.binom(len(A), k) ** 2, eps=e, eps_even=ee,
                seconds=round(time.time() - t0, 1))


def main():
    w = workload("molecule40")
    rng = np.random.default_rng(1910)
    work = []
    for order, per in PER_CLASS.items():
        tl = omb.tuples(w.exp, w.ref, w.occ, order, w.skip)
        by_k = {}
        for t in tl:
            by_k.setdefault(sum(int(w.occ[p]) for p in t), []).append(t)
        for kk in sorted(by_k):
            lst = by_k[kk]
            for i in sorted(rng.choice(len(lst), size=min(per, len(lst)), replace=False)):
                work.append((order, lst[i]))
    procs = min(len(work), len(os.sched_getaffinity(0)))
    with mp.get_context("spawn").Pool(procs) as pool:
        rows = pool.map(one, work, chunksize=1)
    out = {"_note": "Oracle tuple energies (whole determinant space and its even alpha-beta exchange sector) of a "
                    "seeded sample of molecule40 order-3 and order-4 tuples; written by "
                    "tests/golden/make_molecule_sample.py.",
           "e_ref_corr": omb.ref_corr_energy(w.h1, w.eri, w.occ, w.ref), "tuples": rows}
    with open(os.path.join(HERE, "molecule40_sample.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
