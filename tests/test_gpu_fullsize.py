"""Parity at the benchmark sizes, in the launch configuration bench.py times.

* The 81,920-triangle Kirkwood sphere: the GPU solves (FP64 and FP32-pair, the
  latter at the benchmark's tol 1e-4) against the FP64 oracle energy stored in
  tests/golden/oracle_energies.json (written by tests/golden/make_golden.py).
* Sampled rows of the product at 81,920 and ~300,000 triangles against the
  oracle's rows, computed one by one on the host; at ~300,000 the default
  products run in bands, and the FP32-pair product is also checked in one
  pass and under a 100 MiB scratch bound.
"""
import json
import os

import numpy as np
import pytest

import oracle
import pb_inputs as pi
from blockcheck import TOL_FP32PAIR, TOL_FP64, assert_rows_close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_energies.json")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import importlib
    importlib.import_module("paper_1301_5885_gb300.build").build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _pb():
    import paper_1301_5885_gb300 as pb
    return pb


def _ctx(p):
    s = p.surface
    return _pb().pb_create(s.centroids, s.normals, s.areas, p.charges, p.eps1, p.eps2, p.kappa,
                           stream=torch.cuda.current_stream())


@pytest.fixture(scope="module")
def sphere2():
    return pi.kirkwood_sphere_multi()


def _golden(name):
    return json.load(open(GOLDEN))[name]


def test_sphere2_fp32pair_solve_meets_the_energy_bound(sphere2):
    g = _golden("sphere2")
    assert g["n"] == sphere2.n and g["converged"]
    with _ctx(sphere2) as ctx:
        info = _pb().pb_solve(ctx, restart=10, tol=1e-4, maxit=500, prec="fp32pair")
    assert abs(info.energy_kcal - g["energy_kcal"]) <= 1e-5 * abs(g["energy_kcal"])


def test_sphere2_fp64_solve_matches_the_oracle(sphere2):
    g = _golden("sphere2")
    with _ctx(sphere2) as ctx:
        info = _pb().pb_solve(ctx, restart=10, tol=1e-10, maxit=500, prec="fp64")
    # both sides stop at true residual <= 1e-10; their energies agree to ~tol
    assert abs(info.energy_kcal - g["energy_kcal"]) <= 1e-9 * abs(g["energy_kcal"])


def test_sphere1_golden_energy(sphere2):
    p = pi.kirkwood_sphere_single()
    g = _golden("sphere1")
    with _ctx(p) as ctx:
        e64 = _pb().pb_solve(ctx, restart=10, tol=1e-10, maxit=500, prec="fp64").energy_kcal
        e32 = _pb().pb_solve(ctx, restart=10, tol=1e-4, maxit=500, prec="fp32pair").energy_kcal
    assert abs(e64 - g["energy_kcal"]) <= 1e-9 * abs(g["energy_kcal"])
    assert abs(e32 - g["energy_kcal"]) <= 1e-5 * abs(g["energy_kcal"])


def _sampled_rows(p, nrows, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.normal(size=2 * p.n)
    rows = np.sort(rng.choice(p.n, nrows, replace=False))
    rows[0], rows[-1] = 0, p.n - 1                  # first and last (ragged tile) rows
    r1, r2 = oracle.matvec_rows(p.surface, p.eps2 / p.eps1, p.kappa, u, rows)
    return u, rows, r1, r2


@pytest.mark.parametrize("which", ["sphere2", "sphere2_salt_free", "protein300k"])
def test_sampled_rows_at_full_size(which, sphere2):
    """Sampled rows (first and last included) of the products the benchmark
    times, at full size: the 81,920-triangle sphere with and without salt
    (the kappa = 0 symmetric kernel) and the 300,176-triangle solute."""
    pb = _pb()
    p = {"sphere2": lambda: sphere2, "sphere2_salt_free": lambda: pi.by_name("sphere2_salt_free"),
         "protein300k": lambda: pi.protein_like()}[which]()
    assert p.n > 80_000
    u, rows, r1, r2 = _sampled_rows(p, 96, seed=21)
    with _ctx(p) as ctx:
        ud = torch.tensor(u, device="cuda")
        y = torch.empty_like(ud)
        for prec, tol in (("fp64", TOL_FP64), ("float2", TOL_FP64), ("fp32pair", TOL_FP32PAIR)):
            pb.pb_matvec(ctx, ud, y, prec)
            torch.cuda.synchronize()
            yh = y.cpu().numpy()
            assert_rows_close(yh[rows], yh[p.n + rows], r1, r2, tol, prec)
        if which == "protein300k":
            # the defaults (the products above): automatic bands for each
            # symmetric product (79 for the FP32-pair one), within the 1 GiB bound
            for prec in ("fp32pair", "fp64", "float2"):
                bands, nbytes = pb.pb_scratch_plan(ctx, prec)
                assert bands >= 72 and nbytes <= 1 << 30
            assert pb.pb_scratch_plan(ctx, "fp32pair") == (79, 44_122_112)
            # one pass, and the FP32-pair product under a 100 MiB bound
            for bands_req, limit in ((1, 0), (0, 100 << 20)):
                pb.pb_set_bands(ctx, bands_req)
                pb.pb_set_scratch_limit(ctx, limit)
                bands, nbytes = pb.pb_scratch_plan(ctx, "fp32pair")
                assert (bands == 1) if bands_req == 1 else (bands > 1 and nbytes <= limit)
                pb.pb_matvec(ctx, ud, y, "fp32pair")
                torch.cuda.synchronize()
                yh = y.cpu().numpy()
                assert_rows_close(yh[rows], yh[p.n + rows], r1, r2, TOL_FP32PAIR, f"fp32pair {bands} bands")
