"""GPU parity: the CUDA library, called through its C ABI, against the FP64 oracle.

Tolerances, each product compared per row block (phi rows, psi rows), with a
relative L2 bound and an element-wise bound against the block's largest entry:
  FP64 and float-float products   1e-10 / 1e-9;
  FP32-pair products              2e-5 / 1e-4.
  Source: FP64 rel-L2 <= 1e-12, FP32 pairs 2e-6.  Energy: FP64 rel <= 1e-10;
  the solvation energy of an FP32-pair solve rel <= 1e-5.
"""
import numpy as np
import pytest

import oracle
import pb_inputs as pi
from blockcheck import TOL_FP32PAIR, TOL_FP64, assert_blocks_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


def _ctx(surface, charges=None, eps1=1.0, eps2=80.0, kappa=0.1257):
    pb = _pb()
    return pb.pb_create(surface.centroids, surface.normals, surface.areas, charges, eps1, eps2, kappa,
                        stream=torch.cuda.current_stream())


def _u(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.normal(size=2 * n)


def _gpu_matvec(ctx, u, prec):
    pb = _pb()
    ud = torch.tensor(u, dtype=torch.float64, device="cuda")
    y = torch.full_like(ud, float("nan"))
    pb.pb_matvec(ctx, ud, y, prec)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def _surfaces():
    big = pi.icosphere(3.0, 4)
    out = [("ico0", pi.icosphere(2.0, 0)), ("ico2", pi.icosphere(2.0, 2)), ("ico3", pi.icosphere(5.0, 3)),
           ("ico4", big)]
    # ragged sizes: subsets that are not multiples of any tile size
    for n in (1, 2, 3, 33, 513, 777, 4099):
        out.append((f"sub{n}", big.subset(np.arange(n) * (big.n // n))))
    out.append(("solute", pi.protein_like(n_atoms=8, seed=1, target_triangles=None, spacing=1.6).surface))
    return out


SURFACES = _surfaces()


F64_VARIANTS = [1, 2, 3]   # plain, symmetric T1, symmetric T2


@pytest.mark.parametrize("name,surf", SURFACES, ids=[s[0] for s in SURFACES])
@pytest.mark.parametrize("kappa", [0.1257, 0.0])
@pytest.mark.parametrize("variant", F64_VARIANTS)
def test_matvec_fp64_matches_oracle(name, surf, kappa, variant):
    u = _u(surf.n, 1)
    with _ctx(surf, kappa=kappa) as ctx:
        assert _pb().pb_matvec_configure_fp64(ctx, variant) == variant
        y = _gpu_matvec(ctx, u, "fp64")
    ref = oracle.matvec(surf, 80.0, kappa, u)
    assert_blocks_close(y, ref, TOL_FP64)


@pytest.mark.parametrize("name,surf", SURFACES, ids=[s[0] for s in SURFACES])
@pytest.mark.parametrize("kappa", [0.1257, 0.0])
def test_matvec_float2_matches_oracle(name, surf, kappa):
    """Float-float pair arithmetic on the FP32 pipe: the FP64 bound."""
    u = _u(surf.n, 5)
    with _ctx(surf, kappa=kappa) as ctx:
        y = _gpu_matvec(ctx, u, "float2")
    ref = oracle.matvec(surf, 80.0, kappa, u)
    assert_blocks_close(y, ref, TOL_FP64)


def test_matvec_float2_symmetric_two_targets_matches_oracle():
    """From N = 16,384 the float-float product is the symmetric kernel with
    two targets per thread; ragged last tile, rows split over CTAs."""
    surf = pi.icosphere(8.0, 5)
    surf = surf.subset(np.arange(surf.n - 61))
    u = _u(surf.n, 15)
    with _ctx(surf) as ctx:
        y1 = _gpu_matvec(ctx, u, "float2")
        y2 = _gpu_matvec(ctx, u, "float2")
        y64 = _gpu_matvec(ctx, u, "fp64")
    ref = oracle.matvec(surf, 80.0, 0.1257, u)
    assert np.array_equal(y1, y2)
    assert_blocks_close(y1, ref, TOL_FP64)
    assert_blocks_close(y64, ref, TOL_FP64)


F32_VARIANTS = [1, 2, 3, 4, 5, 6]   # scalar T4, packed f32x2 T2, T4, T3, symmetric T2, T4


@pytest.mark.parametrize("name,surf", SURFACES, ids=[s[0] for s in SURFACES])
@pytest.mark.parametrize("kappa", [0.1257, 0.0])
@pytest.mark.parametrize("variant", F32_VARIANTS)
def test_matvec_fp32pair_matches_oracle(name, surf, kappa, variant):
    u = _u(surf.n, 2)
    with _ctx(surf, kappa=kappa) as ctx:
        _pb().pb_matvec_configure(ctx, variant, 0)
        y = _gpu_matvec(ctx, u, "fp32pair")
    ref = oracle.matvec(surf, 80.0, kappa, u)
    assert_blocks_close(y, ref, TOL_FP32PAIR)


@pytest.mark.parametrize("variant", F32_VARIANTS)
@pytest.mark.parametrize("ctas_per_sm", [1, 2])
def test_matvec_fp32pair_small_grids_match_oracle(variant, ctas_per_sm):
    """Fewer resident CTAs per SM changes the stream-K split (more tiles per CTA)."""
    surf = pi.icosphere(6.0, 4)
    u = _u(surf.n, 12)
    with _ctx(surf) as ctx:
        _pb().pb_matvec_configure(ctx, variant, ctas_per_sm)
        y = _gpu_matvec(ctx, u, "fp32pair")
    ref = oracle.matvec(surf, 80.0, 0.1257, u)
    assert_blocks_close(y, ref, TOL_FP32PAIR)


@pytest.mark.parametrize("variant", [5, 6])
@pytest.mark.parametrize("ctas_per_sm", [1, 3])
@pytest.mark.parametrize("kappa", [0.1257, 0.0])
def test_symmetric_matvec_rows_split_over_ctas(variant, ctas_per_sm, kappa):
    """More tile pairs than CTAs: CTA ranges cross row tiles, so rows are
    split over several CTAs (their partial row sides meet in the finishing
    kernel) and CTAs hold whole rows in between."""
    surf = pi.icosphere(8.0, 5)
    surf = surf.subset(np.arange(surf.n - 123))      # ragged last tile
    u = _u(surf.n, 13)
    pb = _pb()
    with _ctx(surf, kappa=kappa) as ctx:
        pb.pb_matvec_configure(ctx, variant, ctas_per_sm)
        assert pb.pb_matvec_get_config(ctx)["variant"] == variant
        y1 = _gpu_matvec(ctx, u, "fp32pair")
        y2 = _gpu_matvec(ctx, u, "fp32pair")
        pb.pb_matvec_configure(ctx, 3, 0)
        y3 = _gpu_matvec(ctx, u, "fp32pair")
    ref = oracle.matvec(surf, 80.0, kappa, u)
    assert np.array_equal(y1, y2)                     # fixed summation order
    assert_blocks_close(y1, ref, TOL_FP32PAIR)
    assert_blocks_close(y3, ref, TOL_FP32PAIR)


@pytest.mark.parametrize("variant", [2, 3])
def test_symmetric_fp64_matvec_rows_split_over_ctas(variant):
    """FP64 symmetric product with more tile pairs than CTAs (rows split over
    CTAs, ragged last tile): FP64 parity and a fixed summation order."""
    surf = pi.icosphere(8.0, 5)
    surf = surf.subset(np.arange(surf.n - 77))
    u = _u(surf.n, 14)
    pb = _pb()
    with _ctx(surf) as ctx:
        pb.pb_matvec_configure_fp64(ctx, variant)
        y1 = _gpu_matvec(ctx, u, "fp64")
        y2 = _gpu_matvec(ctx, u, "fp64")
        pb.pb_matvec_configure_fp64(ctx, 1)
        y3 = _gpu_matvec(ctx, u, "fp64")
    ref = oracle.matvec(surf, 80.0, 0.1257, u)
    assert np.array_equal(y1, y2)
    assert_blocks_close(y1, ref, TOL_FP64)
    assert_blocks_close(y3, ref, TOL_FP64)
    assert_blocks_close(y1, y3, TOL_FP64)             # the two FP64 kernels differ in summation order only


def test_fp64_configure_rejects_unknown_variants():
    surf = pi.icosphere(2.0, 1)
    pb = _pb()
    with _ctx(surf) as ctx:
        with pytest.raises(pb.PBError):
            pb.pb_matvec_configure_fp64(ctx, 4)


def test_autotune_picks_a_valid_variant_with_the_same_result():
    pb = _pb()
    surf = pi.icosphere(8.0, 5)
    u = _u(surf.n, 13)
    with _ctx(surf) as ctx:
        y0 = _gpu_matvec(ctx, u, "fp32pair")
        choice = pb.pb_matvec_autotune(ctx, reps=2)
        assert choice["variant"] in F32_VARIANTS and choice["ms"] > 0
        cfg = pb.pb_matvec_get_config(ctx)
        assert cfg["variant"] == choice["variant"] and cfg["ctas"] >= 1
        y1 = _gpu_matvec(ctx, u, "fp32pair")
    ref = oracle.matvec(surf, 80.0, 0.1257, u)
    assert_blocks_close(y0, ref, TOL_FP32PAIR)
    assert_blocks_close(y1, ref, TOL_FP32PAIR)
    with pytest.raises(pb.PBError):
        with _ctx(surf) as ctx:
            pb.pb_matvec_configure(ctx, 7, 0)


PREC_VARIANTS = ([("fp64", v) for v in F64_VARIANTS] + [("fp32pair", v) for v in F32_VARIANTS]
                 + [("float2", 0)])


def _configure(ctx, prec, variant):
    if prec == "fp64":
        _pb().pb_matvec_configure_fp64(ctx, variant)
    elif prec == "fp32pair":
        _pb().pb_matvec_configure(ctx, variant, 0)


@pytest.mark.parametrize("prec,variant", PREC_VARIANTS)
def test_matvec_is_identity_without_jump_or_salt(prec, variant):
    surf = pi.icosphere(2.0, 3)
    u = _u(surf.n, 3)
    with _ctx(surf, eps1=2.0, eps2=2.0, kappa=0.0) as ctx:
        _configure(ctx, prec, variant)
        y = _gpu_matvec(ctx, u, prec)
    assert np.array_equal(y, u)


@pytest.mark.parametrize("prec", ["fp64", "fp32pair"])
def test_single_element_has_only_the_diagonal(prec):
    surf = pi.icosphere(2.0, 1).subset([5])
    u = np.array([0.7, -1.3])
    with _ctx(surf) as ctx:
        y = _gpu_matvec(ctx, u, prec)
    assert y[0] == 0.5 * (1 + 80.0) * 0.7
    assert y[1] == 0.5 * (1 + 1 / 80.0) * -1.3


@pytest.mark.parametrize("prec,variant", PREC_VARIANTS)
def test_duplicate_centroids_are_dropped_like_the_self_term(prec, variant):
    base = pi.icosphere(2.0, 2)
    idx = np.concatenate([np.arange(base.n), [7, 7, 100]])
    surf = base.subset(idx)
    u = _u(surf.n, 4)
    with _ctx(surf) as ctx:
        _configure(ctx, prec, variant)
        y = _gpu_matvec(ctx, u, prec)
    ref = oracle.matvec(surf, 80.0, 0.1257, u)
    assert_blocks_close(y, ref, TOL_FP32PAIR if prec == "fp32pair" else TOL_FP64)


@pytest.mark.parametrize("prec", ["fp64", "fp32pair"])
def test_matvec_is_deterministic(prec):
    surf = pi.icosphere(4.0, 4)
    u = _u(surf.n, 5)
    with _ctx(surf) as ctx:
        y1 = _gpu_matvec(ctx, u, prec)
        y2 = _gpu_matvec(ctx, u, prec)
    assert np.array_equal(y1, y2)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("float2", 1e-12), ("fp32pair", 2e-6)])
def test_source_matches_oracle(prec, tol):
    pb = _pb()
    p = pi.kirkwood_sphere_multi(level=4, radius=10.0, n_charges=300, seed=3)
    with _ctx(p.surface, p.charges) as ctx:
        b = torch.empty(2 * p.n, dtype=torch.float64, device="cuda")
        pb.pb_source(ctx, b, prec)
        torch.cuda.synchronize()
        b = b.cpu().numpy()
    ref = oracle.source(p.surface, p.charges, 1.0)
    assert np.linalg.norm(b - ref) <= tol * np.linalg.norm(ref)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("float2", 1e-10), ("fp32pair", 1e-5)])
def test_energy_of_matches_oracle(prec, tol):
    pb = _pb()
    p = pi.kirkwood_sphere_multi(level=3, radius=8.0, n_charges=280, seed=6)
    u = _u(p.n, 7) * 1e-2
    with _ctx(p.surface, p.charges) as ctx:
        e = pb.pb_energy_of(ctx, torch.tensor(u, device="cuda"), prec)
    ref = oracle.reaction_energy(p.surface, p.charges, 80.0, 0.1257, u)
    assert e == pytest.approx(ref, rel=tol)


def _problems():
    return [pi.kirkwood_sphere_multi(level=3, radius=6.0, n_charges=7, seed=8),
            pi.kirkwood_sphere_single(level=3),
            pi.protein_like(n_atoms=10, seed=4, target_triangles=None, spacing=1.7)]


@pytest.mark.parametrize("k", range(3))
def test_solve_fp64_matches_oracle(k):
    pb = _pb()
    p = _problems()[k]
    ref = oracle.solve(p.surface, p.charges, p.eps1, p.eps2, p.kappa, tol=1e-12, maxit=2000)
    with _ctx(p.surface, p.charges, p.eps1, p.eps2, p.kappa) as ctx:
        x = torch.empty(2 * p.n, dtype=torch.float64, device="cuda")
        info = pb.pb_solve(ctx, restart=10, tol=1e-12, maxit=2000, prec="fp64", x_out=x)
        assert pb.pb_energy(ctx) == info.energy_kcal
    assert info.status == pb.PB_OK and info.rel_resid <= 1e-12
    u = x.cpu().numpy()
    assert np.linalg.norm(u - ref["u"]) <= 1e-9 * np.linalg.norm(ref["u"])
    assert info.energy_kcal == pytest.approx(ref["energy"], rel=1e-10)


@pytest.mark.parametrize("k", range(3))
def test_solve_fp32pair_energy_within_1e5(k):
    pb = _pb()
    p = _problems()[k]
    ref = oracle.solve(p.surface, p.charges, p.eps1, p.eps2, p.kappa, tol=1e-12, maxit=2000)
    with _ctx(p.surface, p.charges, p.eps1, p.eps2, p.kappa) as ctx:
        info = pb.pb_solve(ctx, restart=10, tol=1e-7, maxit=2000, prec="fp32pair")
    assert info.status == pb.PB_OK
    assert info.energy_kcal == pytest.approx(ref["energy"], rel=1e-5)


@pytest.mark.parametrize("k", range(3))
@pytest.mark.parametrize("refine_prec", ["fp64", "float2"])
def test_refinement_reaches_the_oracle_energy(k, refine_prec):
    """Row a6: FP32-pair GMRES, then FP64 (or float-float) residuals
    r = b - Ax and FP32-pair corrections.  Three refinement steps bring the
    FP64 residual to 1e-11 and the energy within 1e-10 of the oracle's tight
    FP64 solve; the unrefined FP32-pair solve stays at the 1e-5 level."""
    pb = _pb()
    p = _problems()[k]
    ref = oracle.solve(p.surface, p.charges, p.eps1, p.eps2, p.kappa, tol=1e-12, maxit=2000)
    with _ctx(p.surface, p.charges, p.eps1, p.eps2, p.kappa) as ctx:
        x = torch.empty(2 * p.n, dtype=torch.float64, device="cuda")
        plain = pb.pb_solve(ctx, restart=10, tol=1e-9, maxit=2000, prec="fp32pair", raise_on_noconv=False)
        refined = pb.pb_solve(ctx, restart=10, tol=1e-9, maxit=2000, prec="fp32pair", refine=3,
                              refine_prec=refine_prec, x_out=x)
    assert refined.refine_steps == 3
    assert refined.rel_resid_fp64 <= 1e-11
    assert refined.energy_kcal == pytest.approx(ref["energy"], rel=1e-10)
    assert abs(refined.energy_kcal - ref["energy"]) <= abs(plain.energy_kcal - ref["energy"]) + 1e-12 * abs(ref["energy"])
    u = x.cpu().numpy()
    assert np.linalg.norm(u - ref["u"]) <= 1e-9 * np.linalg.norm(ref["u"])


def test_float2_solve_matches_the_oracle():
    """A whole solve with float-float products reaches the FP64 bound."""
    pb = _pb()
    p = _problems()[0]
    ref = oracle.solve(p.surface, p.charges, p.eps1, p.eps2, p.kappa, tol=1e-12, maxit=2000)
    with _ctx(p.surface, p.charges, p.eps1, p.eps2, p.kappa) as ctx:
        ff = pb.pb_solve(ctx, restart=10, tol=1e-12, maxit=2000, prec="float2")
    assert ff.energy_kcal == pytest.approx(ref["energy"], rel=1e-10)


def test_float2_is_rejected_where_it_has_no_meaning():
    pb = _pb()
    surf = pi.icosphere(2.0, 1)
    with _ctx(surf, np.array([[0.0, 0.0, 0.0, 1.0]])) as ctx:
        with pytest.raises(pb.PBError):
            pb.pb_solve(ctx, prec="fp32pair", refine=1, refine_prec="fp32pair")


@pytest.mark.parametrize("kappa", [0.1257, 0.0])
def test_float2_source_and_energy_match_the_oracle_on_a_solute(kappa):
    """The float-float N x Nc pair sums (the source term and energy of the
    FP32-pair and float-float solves) on a protein-like surface with charges
    close to it, at the FP64 bound."""
    pb = _pb()
    p = pi.protein_like(n_atoms=30, seed=9, target_triangles=None, spacing=1.2)
    u = _u(p.n, 19) * 1e-2
    with _ctx(p.surface, p.charges, kappa=kappa) as ctx:
        b = torch.empty(2 * p.n, dtype=torch.float64, device="cuda")
        pb.pb_source(ctx, b, "float2")
        torch.cuda.synchronize()
        e = pb.pb_energy_of(ctx, torch.tensor(u, device="cuda"), "float2")
    ref_b = oracle.source(p.surface, p.charges, 1.0)
    assert_blocks_close(b.cpu().numpy(), ref_b, (1e-12, 1e-11))
    assert e == pytest.approx(oracle.reaction_energy(p.surface, p.charges, 80.0, kappa, u), rel=1e-10)


def test_cached_memory_release_keeps_live_contexts_working():
    pb = _pb()
    p = _problems()[0]
    with _ctx(p.surface, p.charges, p.eps1, p.eps2, p.kappa) as ctx:
        e1 = pb.pb_solve(ctx, tol=1e-8, prec="fp64").energy_kcal
        with _ctx(p.surface, p.charges, p.eps1, p.eps2, p.kappa) as other:
            pb.pb_solve(other, tol=1e-6)
        pb.pb_release_cached_memory()
        e2 = pb.pb_solve(ctx, tol=1e-8, prec="fp64").energy_kcal
    assert e2 == pytest.approx(e1, rel=1e-12)


def test_warm_start_takes_fewer_iterations_and_matches_the_oracle():
    """x0 from a solve with slightly different charges (the next frame): the
    warm solve takes fewer iterations and its solution and energy match the
    oracle's cold solve of the new charges."""
    pb = _pb()
    p = _problems()[0]
    q2 = p.charges.copy()
    q2[:, 3] *= 1.02
    q2[0, :3] += 0.05
    ref = oracle.solve(p.surface, q2, p.eps1, p.eps2, p.kappa, tol=1e-12, maxit=2000)
    with _ctx(p.surface, p.charges) as ctx:
        x = torch.empty(2 * p.n, dtype=torch.float64, device="cuda")
        pb.pb_solve(ctx, tol=1e-10, prec="fp64", x_out=x)
        pb.pb_set_charges(ctx, q2)
        cold = pb.pb_solve(ctx, tol=1e-10, prec="fp64")
        x2 = torch.empty_like(x)
        warm = pb.pb_solve(ctx, tol=1e-10, prec="fp64", x0=x, x_out=x2)
    assert warm.iters < cold.iters
    assert warm.energy_kcal == pytest.approx(ref["energy"], rel=1e-8)
    u = x2.cpu().numpy()
    assert np.linalg.norm(u - ref["u"]) <= 1e-8 * np.linalg.norm(ref["u"])


def test_no_charges_gives_zero_solution_and_energy():
    pb = _pb()
    s = pi.icosphere(2.0, 2)
    with _ctx(s) as ctx:
        x = torch.full((2 * s.n,), 5.0, dtype=torch.float64, device="cuda")
        info = pb.pb_solve(ctx, prec="fp32pair", x_out=x)
        assert info.energy_kcal == 0.0 and info.iters == 0
        assert torch.count_nonzero(x).item() == 0


def test_set_charges_changes_the_right_hand_side():
    pb = _pb()
    p = pi.kirkwood_sphere_multi(level=3, radius=6.0, n_charges=5, seed=9)
    q2 = p.charges.copy()
    q2[:, 3] *= -2.0
    with _ctx(p.surface, p.charges) as ctx:
        e1 = pb.pb_solve(ctx, tol=1e-10, prec="fp64").energy_kcal
        pb.pb_set_charges(ctx, q2)
        e2 = pb.pb_solve(ctx, tol=1e-10, prec="fp64").energy_kcal
    assert e2 == pytest.approx(4.0 * e1, rel=1e-8)     # E is quadratic in the charges


def test_bad_meshes_are_rejected():
    pb = _pb()
    s = pi.icosphere(2.0, 2)
    q = np.array([[0.0, 0.0, 0.0, 1.0]])
    bad = pi.Surface(s.centroids.copy(), s.normals.copy(), s.areas.copy())
    bad.areas[3] = 0.0
    with pytest.raises(pb.PBError) as ei:
        _ctx(bad, q)
    assert ei.value.status == pb.PB_ERR_BADMESH
    bad = pi.Surface(s.centroids.copy(), s.normals.copy() * 1.1, s.areas.copy())
    with pytest.raises(pb.PBError) as ei:
        _ctx(bad, q)
    assert ei.value.status == pb.PB_ERR_BADMESH
    inward = pi.Surface(s.centroids.copy(), -s.normals, s.areas.copy())
    with pytest.raises(pb.PBError) as ei:
        _ctx(inward, q)
    assert ei.value.status == pb.PB_ERR_BADMESH
    with pytest.raises(pb.PBError) as ei:
        _ctx(s, np.array([[5.0, 0.0, 0.0, 1.0]]))      # charge outside the surface
    assert ei.value.status == pb.PB_ERR_BADMESH


def test_geometry_info_and_translation_invariance():
    pb = _pb()
    p = pi.kirkwood_sphere_multi(level=3, radius=6.0, n_charges=5, seed=10)
    shift = np.array([1000.0, -250.0, 40.0])
    moved = p.surface.transformed(shift=shift)
    q = p.charges.copy()
    q[:, :3] += shift
    with _ctx(p.surface, p.charges) as a, _ctx(moved, q) as b:
        ia, ib = pb.pb_get_info(a), pb.pb_get_info(b)
        assert np.allclose(np.array(ib["center"]) - np.array(ia["center"]), shift)
        assert -1.05 < ia["gauss_min"] <= ia["gauss_max"] < -0.95
        ea = pb.pb_solve(a, tol=1e-7, prec="fp32pair").energy_kcal
        eb = pb.pb_solve(b, tol=1e-7, prec="fp32pair").energy_kcal
    assert eb == pytest.approx(ea, rel=1e-5)       # FP32 coordinates are centred first


@pytest.mark.parametrize("variant", F32_VARIANTS)
@pytest.mark.parametrize("kappa", [0.1257, 0.0])
def test_matvec_large_inputs_stay_finite(variant, kappa):
    """Inputs of size 1e6 (beyond anything GMRES feeds the product, whose
    vectors are unit-norm) give finite, correct rows: the self-pair clamp
    never forms an infinity."""
    surf = pi.icosphere(3.0, 3)
    u = _u(surf.n, 14) * 1e6
    with _ctx(surf, kappa=kappa) as ctx:
        _pb().pb_matvec_configure(ctx, variant, 0)
        y = _gpu_matvec(ctx, u, "fp32pair")
    ref = oracle.matvec(surf, 80.0, kappa, u)
    assert_blocks_close(y, ref, TOL_FP32PAIR)
