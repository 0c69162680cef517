"""Pins for the oracle as a whole: closed forms, invariants, brute force and the
paper's printed numbers.  None of these re-types the oracle's own formulas:
each compares it with something the physics or the paper fixes independently.
"""
import math
import os

import numpy as np
import pytest

import oracle
import pb_inputs as pi

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- Born / Kirkwood closed forms ----------------------------------------------
def test_born_closed_form_value():
    # one +1 charge at the centre of a 2 A cavity, eps 1/80, kappa 0.1257
    assert oracle.born_energy(1.0, 2.0, 1.0, 80.0, 0.1257) == pytest.approx(-82.18667, abs=1e-4)


def test_kirkwood_order_zero_is_born():
    for kappa in (0.0, 0.1257, 0.9):
        e = oracle.kirkwood_energy(np.array([[0.0, 0.0, 0.0, 1.3]]), 3.0, 2.0, 80.0, kappa, L=0)
        assert e == pytest.approx(oracle.born_energy(1.3, 3.0, 2.0, 80.0, kappa), rel=1e-13)


def test_kirkwood_exterior_radial_function_matches_library_bessel():
    """g_n from the khat polynomial equals x k_n'(x)/k_n(x) of scipy's modified
    spherical Bessel function of the second kind."""
    from scipy.special import spherical_kn
    for n in (0, 1, 2, 5, 10, 25):
        for x in (0.05, 0.5, 2.514, 7.0):
            ref = x * spherical_kn(n, x, derivative=True) / spherical_kn(n, x)
            assert oracle.kirkwood_g(n, x) == pytest.approx(ref, rel=1e-11)


def test_kirkwood_salt_free_coefficients():
    for n in range(6):
        assert oracle.kirkwood_R(n, 4.0, 1.0, 80.0, 0.0) == pytest.approx(
            (n + 1) * (1.0 - 80.0) / (n * 1.0 + (n + 1) * 80.0), rel=1e-14)


def test_kirkwood_series_truncation_converges():
    p = pi.kirkwood_sphere_multi(level=0)
    e60 = oracle.kirkwood_energy(p.charges, 20.0, 1.0, 80.0, 0.1257, L=60)
    e90 = oracle.kirkwood_energy(p.charges, 20.0, 1.0, 80.0, 0.1257, L=90)
    assert abs(e60 - e90) < 1e-9 * abs(e90)


def test_kirkwood_single_off_centre_charge_no_jump_is_zero():
    ch = np.array([[0.7, -0.2, 1.1, 0.8]])
    assert oracle.kirkwood_energy(ch, 2.0, 4.0, 4.0, 0.0) == pytest.approx(0.0, abs=1e-14)


# --- invariants -----------------------------------------------------------------
def test_identity_operator_without_dielectric_jump_or_salt():
    """eps1 = eps2 and kappa = 0: A = I exactly, so GMRES returns u = b (up to the
    rounding of one normalisation) and E_sol = 0 exactly."""
    p = pi.kirkwood_sphere_multi(level=2, radius=5.0, n_charges=4)
    rng = np.random.Generator(np.random.PCG64(0))
    u = rng.normal(size=2 * p.n)
    y = oracle.matvec(p.surface, 1.0, 0.0, u)
    assert np.array_equal(y, u)
    r = oracle.solve(p.surface, p.charges, 3.0, 3.0, 0.0, tol=1e-14)
    assert np.max(np.abs(r["u"] - r["b"])) <= 1e-15 * np.max(np.abs(r["b"]))
    assert r["energy"] == 0.0


def test_rigid_motion_and_scaling_invariance():
    """Rotation and translation leave E_sol unchanged; scaling lengths by s and
    kappa by 1/s scales E_sol by 1/s (the discrete system is exactly scale covariant)."""
    p = pi.kirkwood_sphere_multi(level=3, radius=6.0, n_charges=5, seed=7)
    base = oracle.solve(p.surface, p.charges, 1.0, 80.0, 0.3, tol=1e-13)["energy"]
    th = 0.7
    rot = np.array([[math.cos(th), -math.sin(th), 0.0], [math.sin(th), math.cos(th), 0.0], [0.0, 0.0, 1.0]])
    ax = np.array([[1.0, 0.0, 0.0], [0.0, math.cos(0.4), -math.sin(0.4)], [0.0, math.sin(0.4), math.cos(0.4)]])
    rot = ax @ rot
    shift = np.array([13.0, -4.0, 2.5])
    s2 = p.surface.transformed(rot, shift)
    ch2 = p.charges.copy()
    ch2[:, :3] = p.charges[:, :3] @ rot.T + shift
    moved = oracle.solve(s2, ch2, 1.0, 80.0, 0.3, tol=1e-13)["energy"]
    assert moved == pytest.approx(base, rel=1e-10)
    s = 2.5
    s3 = p.surface.transformed(scale=s)
    ch3 = p.charges.copy()
    ch3[:, :3] *= s
    scaled = oracle.solve(s3, ch3, 1.0, 80.0, 0.3 / s, tol=1e-13)["energy"]
    assert scaled == pytest.approx(base / s, rel=1e-10)


# --- Gauss identities -----------------------------------------------------------
def test_gauss_double_layer_identity():
    """sum_j W_j dG0(p, x_j)/dnu_j -> -1 inside, 0 outside, -1/2 at a centroid."""
    s = pi.icosphere(3.0, 4)
    inside = np.array([[0.0, 0.0, 0.0], [1.0, 0.5, -0.7], [0.0, 0.0, 2.0]])
    outside = np.array([[0.0, 0.0, 6.0], [4.0, 4.0, 0.0]])
    assert np.all(np.abs(oracle.gauss_sums(s, inside) + 1.0) < 5e-3)
    assert np.all(np.abs(oracle.gauss_sums(s, outside)) < 5e-3)
    on = oracle.gauss_sums(s, s.centroids[:50])
    assert np.all(np.abs(on + 0.5) < 2e-2)


def test_source_flux_is_minus_total_charge():
    """sum_i W_i S2(x_i) approximates the flux integral of dG0/dnu_x, which is -1
    for every enclosed unit charge: the total is -sum_k Q_k / eps1."""
    p = pi.kirkwood_sphere_multi(level=4, radius=5.0, n_charges=6, seed=4)
    b = oracle.source(p.surface, p.charges, 2.0)
    flux = float(np.sum(p.surface.areas * b[p.n:]))
    assert flux == pytest.approx(-p.charges[:, 3].sum() / 2.0, abs=2e-3 * np.abs(p.charges[:, 3]).sum())


# --- brute force ----------------------------------------------------------------
@pytest.mark.parametrize("which", ["sphere", "solute"])
def test_dense_assembly_and_lu_match_matrix_free_gmres(which):
    if which == "sphere":
        p = pi.kirkwood_sphere_multi(level=2, radius=4.0, n_charges=3, seed=1)
    else:
        p = pi.protein_like(n_atoms=6, seed=2, target_triangles=None, spacing=3.2)
    assert p.n <= 700
    eps = p.eps2 / p.eps1
    A = oracle.assemble(p.surface, eps, p.kappa)
    rng = np.random.Generator(np.random.PCG64(3))
    u = rng.normal(size=2 * p.n)
    y = oracle.matvec(p.surface, eps, p.kappa, u)
    assert np.max(np.abs(A @ u - y)) <= 1e-13 * np.max(np.abs(y))
    dense = oracle.solve_dense(p.surface, p.charges, p.eps1, p.eps2, p.kappa)
    it = oracle.solve(p.surface, p.charges, p.eps1, p.eps2, p.kappa, tol=1e-13)
    assert it["converged"]
    assert np.linalg.norm(it["u"] - dense["u"]) <= 1e-10 * np.linalg.norm(dense["u"])
    assert it["energy"] == pytest.approx(dense["energy"], rel=1e-10)


@pytest.mark.parametrize("which", ["sphere", "solute"])
def test_sampled_rows_equal_the_full_product_rows(which):
    """oracle.matvec_rows (the reference of the full-size sampled-row parity
    tests and of the CPU baseline) returns exactly rows i and N+i of the full
    product, bit for bit (same summation order), in the right output slots:
    the phi and psi halves of u are given scales 1 and 1000, so a swapped
    slot or a swapped u[j] / u[N+j] cannot pass.  Rows 0 and N-1 included,
    and a repeated row.  On the small case both also equal the dense A's
    rows (brute force)."""
    if which == "sphere":
        p = pi.kirkwood_sphere_multi(level=4, radius=7.0, n_charges=3, seed=5)
    else:
        p = pi.protein_like(n_atoms=10, seed=3, target_triangles=None, spacing=1.9)
    eps = p.eps2 / p.eps1
    rng = np.random.Generator(np.random.PCG64(17))
    u = np.concatenate([rng.normal(size=p.n), 1000.0 * rng.normal(size=p.n)])
    rows = np.concatenate([[0, p.n - 1], rng.choice(p.n, 40, replace=False), [7, 7]])
    full = oracle.matvec(p.surface, eps, p.kappa, u)
    y1, y2 = oracle.matvec_rows(p.surface, eps, p.kappa, u, rows)
    assert np.array_equal(y1, full[rows])
    assert np.array_equal(y2, full[p.n + rows])
    assert not np.allclose(y1, y2)
    small = p.surface.subset(np.arange(0, p.n, max(1, p.n // 400)))
    us = np.concatenate([rng.normal(size=small.n), 1000.0 * rng.normal(size=small.n)])
    A = oracle.assemble(small, eps, p.kappa)
    rs = np.array([0, small.n - 1, small.n // 2])
    z1, z2 = oracle.matvec_rows(small, eps, p.kappa, us, rs)
    dense = A @ us
    assert np.allclose(z1, dense[rs], rtol=1e-12, atol=1e-12 * np.abs(dense).max())
    assert np.allclose(z2, dense[small.n + rs], rtol=1e-12, atol=1e-12 * np.abs(dense).max())


def test_gmres_matches_lu_on_a_random_nonsymmetric_system():
    rng = np.random.Generator(np.random.PCG64(8))
    n = 60
    A = np.eye(n) * 3.0 + rng.normal(size=(n, n)) / math.sqrt(n)
    b = rng.normal(size=n)
    x, iters, hist, conv = oracle.gmres(lambda v: A @ v, b, restart=7, tol=1e-12, maxit=2000)
    assert conv and hist[-1] <= 1e-12
    assert np.allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-10)


# --- convergence to the analytic solution --------------------------------------
def test_born_energy_converges_under_refinement():
    exact = oracle.born_energy(1.0, 2.0, 1.0, 80.0, 0.1257)
    errs = []
    for lvl in (1, 2, 3, 4):
        p = pi.kirkwood_sphere_single(level=lvl)
        errs.append(abs(oracle.solve(p.surface, p.charges, p.eps1, p.eps2, p.kappa, tol=1e-10)["energy"] - exact))
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 0.01 * abs(exact)


def test_exact_surface_solution_nearly_satisfies_the_discrete_system():
    """Plugging the analytic (phi, dphi/dnu) into Au - b leaves only the
    discretisation error, which shrinks under refinement; the energy of the
    analytic data converges to the Kirkwood energy."""
    res, eerr = [], []
    for lvl in (2, 3, 4):
        p = pi.kirkwood_sphere_multi(level=lvl, radius=5.0, n_charges=6, seed=4)
        eps = p.eps2 / p.eps1
        phi, dphi = oracle.kirkwood_surface(p.surface.centroids, p.charges, 5.0, p.eps1, p.eps2, p.kappa)
        u = np.concatenate([phi, dphi])
        b = oracle.source(p.surface, p.charges, p.eps1)
        r = oracle.matvec(p.surface, eps, p.kappa, u) - b
        res.append(np.linalg.norm(r) / np.linalg.norm(b))
        ek = oracle.kirkwood_energy(p.charges, 5.0, p.eps1, p.eps2, p.kappa)
        eerr.append(abs(oracle.reaction_energy(p.surface, p.charges, eps, p.kappa, u) - ek) / abs(ek))
    assert res[0] > res[1] > res[2] and res[2] < 0.02
    assert eerr[0] > eerr[1] > eerr[2] and eerr[2] < 0.01


def test_multi_charge_kirkwood_energy_and_surface_potential_converge():
    """The nine-charge helix of Section 3.2 in a radius-4 sphere: E_sol and the
    surface-potential error e_phi (Eq. (15)) converge; the order per halving of
    the element area (Eq. (16)) is about 0.5 as in the paper's spherical test."""
    errs, ephi = [], []
    ek = oracle.kirkwood_energy(pi.helix_charges(), 4.0, 1.0, 80.0, 0.0)
    for lvl in (2, 3, 4):
        p = pi.helix_sphere(level=lvl)
        r = oracle.solve(p.surface, p.charges, p.eps1, p.eps2, p.kappa, tol=1e-10)
        errs.append(abs(r["energy"] - ek) / abs(ek))
        phi_ex, _ = oracle.kirkwood_surface(p.surface.centroids, p.charges, 4.0, p.eps1, p.eps2, p.kappa)
        ephi.append(oracle.error_linf(r["u"][:p.n], phi_ex))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.02
    orders = [oracle.order(a, b, 2.0) / 2.0 for a, b in zip(ephi, ephi[1:])]  # 4x area per level
    assert all(0.3 < o < 1.5 for o in orders), orders


# --- the paper's printed numbers ------------------------------------------------
def test_order_definition_reproduces_the_papers_table():
    """Eq. (16) applied to the printed e_phi column (density doubling each row)
    reproduces the printed order column of the spherical-cavity table."""
    rows = np.loadtxt(os.path.join(GOLDEN, "paper_sphere_table.txt"))
    for prev, cur in zip(rows, rows[1:]):
        assert cur[1] > prev[1]
        o = oracle.order(prev[3], cur[3], cur[0] / prev[0])
        assert o == pytest.approx(cur[4], abs=0.006)


def test_papers_sphere_energies_approach_their_exact_value_at_order_half():
    """The printed E_sol column approaches -952.52 with an error that halves
    roughly every fourfold increase in the element count (order about 0.5 in area)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "paper_sphere_table.txt"))
    err = np.abs(rows[:, 2] + 952.52)
    assert np.all(np.diff(err) < 0)
    slope = np.polyfit(np.log(rows[:, 1]), np.log(err), 1)[0]
    assert -0.6 < slope < -0.35
