"""Writes tests/golden/oracle_totals.json: the oracle's order sums and totals of
the full-size Hubbard workloads (L=22, U=4, orders 1-6; L=46, U=4, orders 1-4;
momentum basis, empty reference space, skip rule).  Calls oracle/ only (through
tests/oracle_full.py, which spreads the tuple CASCIs over host processes).

    python tests/golden/make_oracle_totals.py
"""

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
TESTS = os.path.dirname(HERE)
ROOT = os.path.dirname(TESTS)
for p in (ROOT, TESTS):
    if p not in sys.path:
        sys.path.insert(0, p)

from oracle_full import run_mbe_parallel  # noqa: E402
from workloads import workload  # noqa: E402


def main():
    out = {"_note": "Oracle (oracle/mbe.py run_mbe, tuple CASCIs by LAPACK/ARPACK at tol 1e-13) on the "
                    "full-size Hubbard workloads; written by tests/golden/make_oracle_totals.py.",
           "workloads": {}}
    for name in ("hubbard22", "hubbard46"):
        w = workload(name)
        t0 = time.time()
        r = run_mbe_parallel(name)
        out["workloads"][name] = {
            "description": w.description, "orders": list(w.orders),
            "tuples_per_order": {str(n): len(r["eps"][n]) for n in w.orders},
            "e_phi": r["e_phi"], "e_ref_corr": r["e_ref_corr"],
            "e_order": {str(n): r["e_order"][n] for n in w.orders},
            "e_corr": r["e_corr"], "e_tot": r["e_tot"],
            "seconds": round(time.time() - t0, 1)}
        print(name, out["workloads"][name]["e_tot"], out["workloads"][name]["seconds"], "s", flush=True)
    with open(os.path.join(HERE, "oracle_totals.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
