"""Write tests/golden/oracle_energies.json: FP64 oracle solutions of the
benchmark workloads, used as the reference energies of the GPU parity tests
and of bench.py's energy-error report.

Only the oracle and the seeded input generators are used.  Run from the
repository root:

    python tests/golden/make_golden.py [--tol T] [--checkpoint FILE] [name ...]

``--checkpoint FILE`` saves the GMRES iterate at every restart (an .npz) and,
when FILE already exists for the same workload, resumes from it: GMRES(m)
restarts from its current approximation anyway, so a resumed run with the
same settings takes exactly the steps the uninterrupted one would (and one
with another tolerance or restart length continues from the same iterate).  This lets the
300,000-triangle solve (hours of oracle time) survive an interruption.

Each entry records the surface's size, total area and centroid sum, so that a
reader on another host can check that its generator built the same mesh.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import pb_inputs  # noqa: E402

OUT = os.path.join(HERE, "oracle_energies.json")
TOL = 1e-10


def mesh_fingerprint(surface) -> dict:
    return {"area_sum": float(np.sum(surface.areas)),
            "centroid_sum": [float(v) for v in np.sum(surface.centroids, axis=0)]}


def run(name: str, tol: float, checkpoint: str | None, maxit: int, restart: int = 10) -> dict:
    p = pb_inputs.by_name(name)
    x0, it0, sec0 = None, 0, 0.0
    if checkpoint and os.path.exists(checkpoint):
        ck = np.load(checkpoint)
        keys = set(ck.files)
        # restarted GMRES continues from its current approximation, so a
        # saved iterate is a valid start whatever tolerance or restart length
        # the run that wrote it used
        if ({"name", "x", "iters", "seconds", "resid"} <= keys and str(ck["name"]) == name
                and ck["x"].shape == (2 * p.n,)):
            x0, it0, sec0 = ck["x"], int(ck["iters"]), float(ck["seconds"])
            print(f"{name}: resuming at iteration {it0}, rel. residual {float(ck['resid']):.3e}", flush=True)
    t = time.time()

    def save(x, iters, resid):
        print(f"{name}: iteration {it0 + iters}, rel. residual {resid:.3e}, "
              f"{sec0 + time.time() - t:.0f} s", flush=True)
        if checkpoint:
            tmp = checkpoint + ".tmp.npz"
            np.savez(tmp, x=x, iters=it0 + iters, resid=resid, tol=tol, name=name, restart=restart,
                     seconds=sec0 + time.time() - t)
            os.replace(tmp, checkpoint)

    r = oracle.solve(p.surface, p.charges, p.eps1, p.eps2, p.kappa, restart=restart, tol=tol, maxit=maxit,
                     x0=x0, callback=save)
    entry = {"workload": p.name, "n": p.n, "nc": p.nc, "eps1": p.eps1, "eps2": p.eps2, "kappa": p.kappa,
             "restart": restart, "tol": tol, "iters": it0 + r["iters"], "converged": bool(r["converged"]),
             "rel_resid": r["history"][-1], "energy_kcal": r["energy"],
             "oracle_seconds": round(sec0 + time.time() - t, 1), "oracle_threads": oracle.num_threads(),
             "mesh": mesh_fingerprint(p.surface)}
    if p.sphere_radius is not None:
        entry["kirkwood_kcal"] = oracle.kirkwood_energy(p.charges, p.sphere_radius, p.eps1, p.eps2, p.kappa)
    return entry


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="*", default=["sphere1", "sphere2"])
    ap.add_argument("--tol", type=float, default=TOL)
    ap.add_argument("--checkpoint", default=None)
    ap.add_argument("--maxit", type=int, default=5000)
    ap.add_argument("--restart", type=int, default=10,
                    help="GMRES restart length (any restart converges to the same discrete solution; a longer "
                         "one needs fewer oracle products on the 300,000-triangle solute)")
    a = ap.parse_args(argv)
    for name in a.names:
        entry = run(name, a.tol, a.checkpoint, a.maxit, a.restart)
        data = json.load(open(OUT)) if os.path.exists(OUT) else {}
        data[name] = entry
        print(name, entry, flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
