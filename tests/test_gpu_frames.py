"""Warm-started repeated solves (a trajectory of perturbed frames of one
solute, solved one after another): the solution of frame f - 1 as the
starting vector of frame f takes fewer GMRES iterations than a cold start,
and every frame's energy matches the oracle's solve of that frame."""
import numpy as np
import pytest

import oracle
import pb_inputs as pi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import importlib
    importlib.import_module("paper_1301_5885_gb300.build").build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("prec,tol,etol", [("fp32pair", 1e-7, 1e-5), ("fp64", 1e-11, 1e-9)])
def test_warm_started_frames_match_the_oracle_and_save_iterations(prec, tol, etol):
    import paper_1301_5885_gb300 as pb
    base = pi.protein_like(n_atoms=10, seed=6, target_triangles=None, spacing=1.6)
    frames = pi.md_frames(base, 5)
    x_prev = None
    cold_it, warm_it = [], []
    for f in frames:
        s = f.surface
        ref = oracle.solve(s, f.charges, f.eps1, f.eps2, f.kappa, tol=1e-12, maxit=2000)
        with pb.pb_create(s.centroids, s.normals, s.areas, f.charges, f.eps1, f.eps2, f.kappa,
                          stream=torch.cuda.current_stream()) as ctx:
            cold = pb.pb_solve(ctx, tol=tol, maxit=2000, prec=prec)
            x = torch.empty(2 * f.n, dtype=torch.float64, device="cuda")
            warm = pb.pb_solve(ctx, tol=tol, maxit=2000, prec=prec, x0=x_prev, x_out=x)
        assert cold.energy_kcal == pytest.approx(ref["energy"], rel=etol)
        assert warm.energy_kcal == pytest.approx(ref["energy"], rel=etol)
        if x_prev is not None:
            cold_it.append(cold.iters)
            warm_it.append(warm.iters)
        x_prev = x
    assert all(w < c for w, c in zip(warm_it, cold_it))
    assert sum(warm_it) <= 0.8 * sum(cold_it)
