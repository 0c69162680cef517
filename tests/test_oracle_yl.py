"""The straightforward (Yoon-Lenhoff) system of Eqs. (6)-(7) in the oracle: a
CPU-only contrast to the paper's well-conditioned formulation (Section 2.1
sets it aside because its condition number grows with the number of
elements).  Pins for its operator come from identities of the layer
potentials, its energy from the Born closed form; then the contrast itself:
its condition number and GMRES iteration count grow under refinement while
those of Eqs. (12)-(13) stay flat."""
import numpy as np
import pytest

import oracle
import pb_inputs as pi


def test_double_layer_rows_follow_the_gauss_identity():
    """phi = 1, dphi = 0: the interior rows are 1/2 + sum W dG0/dny -> 0 and
    the exterior rows (kappa = 0) 1/2 - sum W dG0/dny -> 1, since the double
    layer of a unit density is -1/2 on the surface.  A sign error in either
    row's double-layer term moves these to 1 or 0."""
    s = pi.icosphere(3.0, 4)
    n = s.n
    y = oracle.yl_matvec(s, 80.0, 0.0, np.concatenate([np.ones(n), np.zeros(n)]))
    assert np.max(np.abs(y[:n])) < 0.02
    assert np.max(np.abs(y[n:] - 1.0)) < 0.02


@pytest.mark.parametrize("radius", [1.5, 3.0])
def test_single_layer_of_a_constant_density_is_the_radius(radius):
    """dphi = 1 on a sphere of radius a: the single-layer potential on the
    surface is a (the self element included through its equal-area disk), so
    the interior rows give -a and the exterior rows (kappa = 0) a / eps."""
    s = pi.icosphere(radius, 4)
    n = s.n
    y = oracle.yl_matvec(s, 80.0, 0.0, np.concatenate([np.zeros(n), np.ones(n)]))
    assert np.mean(y[:n]) == pytest.approx(-radius, rel=3e-3)
    assert np.mean(y[n:]) == pytest.approx(radius / 80.0, rel=3e-3)
    assert np.std(y[:n]) < 1e-3 * radius


def test_energy_converges_to_the_born_value():
    born = oracle.born_energy(1.0, 2.0, 1.0, 80.0, 0.1257)
    errs = []
    for lvl in (2, 3, 4):
        p = pi.kirkwood_sphere_single(level=lvl)
        r = oracle.yl_solve(p.surface, p.charges, p.eps1, p.eps2, p.kappa, tol=1e-9, maxit=3000)
        assert r["converged"]
        errs.append(abs(r["energy"] - born) / abs(born))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 5e-3


def test_conditioning_grows_with_n_unlike_the_well_posed_form():
    conds_yl, conds_j = [], []
    for lvl in (1, 2, 3):
        p = pi.kirkwood_sphere_single(level=lvl)
        conds_yl.append(np.linalg.cond(oracle.yl_assemble(p.surface, 80.0, p.kappa)))
        conds_j.append(np.linalg.cond(oracle.assemble(p.surface, 80.0, p.kappa)))
    assert all(b > 1.8 * a for a, b in zip(conds_yl, conds_yl[1:]))
    assert max(conds_j) < 1.05 * min(conds_j)
    its_yl, its_j = [], []
    for lvl in (1, 2, 3, 4):
        p = pi.kirkwood_sphere_single(level=lvl)
        its_yl.append(oracle.yl_solve(p.surface, p.charges, p.eps1, p.eps2, p.kappa, tol=1e-6, maxit=3000)["iters"])
        its_j.append(oracle.solve(p.surface, p.charges, p.eps1, p.eps2, p.kappa, tol=1e-6, maxit=3000)["iters"])
    assert all(b > a for a, b in zip(its_yl, its_yl[1:]))
    assert its_yl[-1] >= 2 * its_j[-1]
    assert max(its_j[1:]) - min(its_j[1:]) <= 3
