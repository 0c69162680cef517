"""The spherical-cavity accuracy study of Section 3.2 on the GPU path.

The nine-charge helix in a radius-4 A sphere is solved on icospheres of
increasing level; the surface potential returned by pb_solve is compared with
the analytic Kirkwood surface potential (relative L-infinity error e_phi,
Eq. (15)) and the observed order per halving of the element area (Eq. (16))
is about 0.5, as in the paper's table.  Where the oracle is cheap enough the
GPU e_phi equals the oracle's e_phi.
"""
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


def _solve(p, prec, tol):
    import paper_1301_5885_gb300 as pb
    s = p.surface
    with pb.pb_create(s.centroids, s.normals, s.areas, p.charges, p.eps1, p.eps2, p.kappa) as ctx:
        x = torch.empty(2 * p.n, dtype=torch.float64, device="cuda")
        info = pb.pb_solve(ctx, tol=tol, maxit=2000, prec=prec, x_out=x)
    return x.cpu().numpy(), info.energy_kcal


@pytest.mark.parametrize("prec", ["fp32pair", "fp64"])
def test_surface_potential_error_and_order(prec):
    levels = (2, 3, 4, 5) if prec == "fp32pair" else (2, 3, 4)
    ephi, energies = [], []
    ek = oracle.kirkwood_energy(pi.helix_charges(), 4.0, 1.0, 80.0, 0.0)
    for lvl in levels:
        p = pi.helix_sphere(level=lvl)
        # FP32-pair products put a floor of about 1e-9 under the relative
        # residual (it depends on the kernel variant), far below the
        # discretisation error measured here
        x, e = _solve(p, prec, 1e-9 if prec == "fp64" else 1e-7)
        phi_ex, _ = oracle.kirkwood_surface(p.surface.centroids, p.charges, 4.0, p.eps1, p.eps2, p.kappa)
        ephi.append(oracle.error_linf(x[:p.n], phi_ex))
        energies.append(abs(e - ek) / abs(ek))
        if lvl <= 3:
            ref = oracle.solve(p.surface, p.charges, p.eps1, p.eps2, p.kappa, tol=1e-11)
            e_or = oracle.error_linf(ref["u"][:p.n], phi_ex)
            assert ephi[-1] == pytest.approx(e_or, rel=1e-4)
    assert all(b < a for a, b in zip(ephi, ephi[1:]))
    assert all(b < a for a, b in zip(energies, energies[1:]))
    orders = [oracle.order(a, b, 2.0) / 2.0 for a, b in zip(ephi, ephi[1:])]   # 4x area per level
    assert all(0.3 < o < 1.5 for o in orders), orders
