"""Write tests/golden/oracle_energies.json: FP64 oracle solutions of the
benchmark workloads, used as the reference energies of the GPU parity tests
and of bench.py's energy-error report.

Only the oracle and the seeded input generators are used.  Run from the
repository root:  python tests/golden/make_golden.py [name ...]
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import pb_inputs  # noqa: E402

OUT = os.path.join(HERE, "oracle_energies.json")
TOL = 1e-10


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        p = pb_inputs.by_name(name)
        t = time.time()
        r = oracle.solve(p.surface, p.charges, p.eps1, p.eps2, p.kappa, restart=10, tol=TOL, maxit=5000)
        entry = {"workload": p.name, "n": p.n, "nc": p.nc, "eps1": p.eps1, "eps2": p.eps2, "kappa": p.kappa,
                 "restart": 10, "tol": TOL, "iters": r["iters"], "converged": bool(r["converged"]),
                 "rel_resid": r["history"][-1], "energy_kcal": r["energy"],
                 "oracle_seconds": round(time.time() - t, 1), "oracle_threads": oracle.num_threads()}
        if p.sphere_radius is not None:
            entry["kirkwood_kcal"] = oracle.kirkwood_energy(p.charges, p.sphere_radius, p.eps1, p.eps2, p.kappa)
        data[name] = entry
        print(name, entry, flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["sphere1", "sphere2"])
