"""Batched lockstep solves (many surfaces of uneven N, several charge sets
each): every batched energy equals the one-at-a-time solve of the same
(surface, charge set) within the FP32-pair tolerance, and meets the 1e-5 bound
against the FP64 oracle where the oracle is cheap enough."""
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


def _pb():
    import paper_1301_5885_gb300 as pb
    return pb


def _mix():
    """Uneven surfaces, 1..8 charge sets each, kappa in {0, 0.1257}.  The
    20,480-triangle surfaces with one charge set take their own symmetric
    product (their contexts default to it), the rest share the batched one."""
    out = []
    for k, (lvl, rad, nq, nr, kap) in enumerate([(2, 3.0, 3, 1, 0.1257), (3, 5.0, 6, 4, 0.0),
                                                (4, 8.0, 10, 8, 0.1257), (3, 6.0, 5, 3, 0.1257),
                                                (5, 12.0, 8, 1, 0.0), (5, 14.0, 6, 1, 0.1257)]):
        p = pi.kirkwood_sphere_multi(level=lvl, radius=rad, n_charges=nq, seed=30 + k, kappa=kap)
        sets = pi.charge_variants(p.charges, nr, seed=40 + k, frac=0.3)
        out.append((p, sets))
    sol = pi.protein_like(n_atoms=12, seed=6, target_triangles=None, spacing=1.4)
    out.append((sol, pi.charge_variants(sol.charges, 2, seed=7, frac=0.2)))
    return out


@pytest.mark.parametrize("use_graph", [True, False])
def test_batched_energies_match_single_solves(use_graph):
    pb = _pb()
    mix = _mix()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctxs = [pb.pb_create(p.surface.centroids, p.surface.normals, p.surface.areas, sets[0], p.eps1, p.eps2,
                             p.kappa, stream=stream) for p, sets in mix]
        energies, info = pb.pb_batch_solve(ctxs, [sets for _, sets in mix], tol=1e-7, maxit=2000,
                                           use_graph=use_graph)
        assert info["instances"] == sum(len(s) for _, s in mix) == info["converged"]
        assert info["rhs_width"] == 8 and info["pair_products"] >= info["pair_evals"] > 0
        for (p, sets), ctx, es in zip(mix, ctxs, energies):
            assert len(es) == len(sets)
            for r, q in enumerate(sets):
                pb.pb_set_charges(ctx, q)
                single = pb.pb_solve(ctx, tol=1e-7, maxit=2000, prec="fp32pair").energy_kcal
                assert es[r] == pytest.approx(single, rel=2e-6, abs=1e-9)
        for c in ctxs:
            pb.pb_destroy(c)


def test_batched_energies_meet_the_bound_against_the_oracle():
    pb = _pb()
    p = pi.kirkwood_sphere_multi(level=3, radius=6.0, n_charges=8, seed=51)
    sets = pi.charge_variants(p.charges, 8, seed=52, frac=0.25)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = pb.pb_create(p.surface.centroids, p.surface.normals, p.surface.areas, sets[0], p.eps1, p.eps2,
                           p.kappa, stream=stream)
        energies, info = pb.pb_batch_solve([ctx], [sets], tol=1e-7)
        pb.pb_destroy(ctx)
    for r, q in enumerate(sets):
        ref = oracle.solve(p.surface, q, p.eps1, p.eps2, p.kappa, tol=1e-11)["energy"]
        assert energies[0][r] == pytest.approx(ref, rel=1e-5)


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_of_only_direct_surfaces(use_graph):
    """Every surface has one charge set on a symmetric-product context, so the
    batched work list is empty and each surface takes its own product."""
    pb = _pb()
    probs = [pi.kirkwood_sphere_multi(level=5, radius=12.0 + 2 * k, n_charges=6, seed=70 + k,
                                      kappa=(0.0 if k else 0.1257)) for k in range(2)]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctxs = [pb.pb_create(p.surface.centroids, p.surface.normals, p.surface.areas, p.charges, p.eps1, p.eps2,
                             p.kappa, stream=stream) for p in probs]
        energies, info = pb.pb_batch_solve(ctxs, [[p.charges] for p in probs], tol=1e-7, maxit=2000,
                                           use_graph=use_graph)
        assert info["converged"] == 2 and info["ctas"] == 0
        for p, ctx, es in zip(probs, ctxs, energies):
            single = pb.pb_solve(ctx, tol=1e-7, maxit=2000, prec="fp32pair").energy_kcal
            assert es[0] == pytest.approx(single, rel=2e-6)
        for c in ctxs:
            pb.pb_destroy(c)


def test_batch_rejects_bad_arguments():
    pb = _pb()
    p = pi.kirkwood_sphere_multi(level=2, radius=3.0, n_charges=2, seed=1)
    with pb.pb_create(p.surface.centroids, p.surface.normals, p.surface.areas, p.charges, 1.0, 80.0, 0.1) as ctx:
        with pytest.raises(pb.PBError):
            pb.pb_batch_solve([ctx], [np.repeat(p.charges[None], 9, axis=0)])   # more than 8 charge sets


def _small_mix():
    """A batch small enough to tune quickly: widths 8 (the widest set) with
    uneven surfaces, kappa in {0, 0.1257}, no direct surfaces."""
    out = []
    for k, (lvl, rad, nq, nr, kap) in enumerate([(3, 5.0, 6, 8, 0.1257), (4, 8.0, 10, 5, 0.0),
                                                (3, 6.0, 5, 3, 0.1257), (2, 3.0, 3, 1, 0.1257)]):
        p = pi.kirkwood_sphere_multi(level=lvl, radius=rad, n_charges=nq, seed=80 + k, kappa=kap)
        out.append((p, pi.charge_variants(p.charges, nr, seed=90 + k, frac=0.3)))
    return out


def _solve_mix(mix, **kw):
    pb = _pb()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctxs = [pb.pb_create(p.surface.centroids, p.surface.normals, p.surface.areas, sets[0], p.eps1, p.eps2,
                             p.kappa, stream=stream) for p, sets in mix]
        try:
            return pb.pb_batch_solve(ctxs, [sets for _, sets in mix], tol=1e-7, maxit=2000, **kw)
        finally:
            for c in ctxs:
                pb.pb_destroy(c)


@pytest.mark.parametrize("width", [1, 2, 4, 8])
def test_every_batched_product_shape_gives_the_same_energies(width):
    """Each instantiated shape (targets per thread, FP64 or float-float row
    sums in registers or shared memory) and CTA count computes the same
    products: energies within 2e-6 of the built-in default shape."""
    pb = _pb()
    mix = [(p, sets[:width]) for p, sets in _small_mix()]
    mix[0] = (mix[0][0], pi.charge_variants(mix[0][0].charges, width, seed=95, frac=0.3))
    pb.pb_batch_set_tuning(False)
    try:
        ref, info = _solve_mix(mix)
        assert info["rhs_width"] == width and info["tuned"] == 0
        for t, r in pb.pb_batch_shapes(width):
            for cps in (1, 0):
                pb.pb_batch_force_shape(width, t, r, cps)
                got, gi = _solve_mix(mix, use_graph=(cps == 0))
                assert (gi["targets_per_thread"], gi["row_sums"], gi["ctas_per_sm"]) == (t, r, cps)
                for a, b in zip(got, ref):
                    assert a == pytest.approx(b, rel=2e-6, abs=1e-9), (t, r, cps)
    finally:
        pb.pb_batch_force_shape(width)
        pb.pb_batch_set_tuning(True)


def test_autotuned_batch_matches_the_default_and_the_oracle():
    """The autotuner times every shape on the batch's own work list, caches
    the choice, and the tuned run gives the default run's energies to 2e-6
    and the oracle's to 1e-5; a second batch of the same size class reuses the
    cached choice without tuning."""
    pb = _pb()
    mix = _small_mix()
    pb.pb_batch_set_tuning(False)
    ref, _ = _solve_mix(mix)
    pb.pb_batch_set_tuning(True)
    pb.pb_batch_clear_tuning()
    got, info = _solve_mix(mix)
    assert info["tuned"] == 1 and info["tune_candidates"] >= len(pb.pb_batch_shapes(8))
    assert (info["targets_per_thread"], info["row_sums"]) in pb.pb_batch_shapes(8)
    for a, b in zip(got, ref):
        assert a == pytest.approx(b, rel=2e-6, abs=1e-9)
    again, info2 = _solve_mix(mix)
    assert info2["tuned"] == 0
    assert (info2["targets_per_thread"], info2["row_sums"], info2["ctas_per_sm"]) == \
        (info["targets_per_thread"], info["row_sums"], info["ctas_per_sm"])
    for (p, sets), es in zip(mix[:1], got[:1]):
        for r, q in enumerate(sets):
            e = oracle.solve(p.surface, q, p.eps1, p.eps2, p.kappa, tol=1e-11)["energy"]
            assert es[r] == pytest.approx(e, rel=1e-5)


def test_one_and_two_engines_give_the_same_energies():
    """The members split over two engines on two streams (the default) and
    all in one engine: the same energies within the FP32-pair tolerance (the
    products' work splits differ), and a single surface takes one engine."""
    pb = _pb()
    mix = _mix()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctxs = [pb.pb_create(p.surface.centroids, p.surface.normals, p.surface.areas, sets[0], p.eps1, p.eps2,
                             p.kappa, stream=stream) for p, sets in mix]
        try:
            sets = [s for _, s in mix]
            e2, i2 = pb.pb_batch_solve(ctxs, sets, tol=1e-7, maxit=2000, use_graph=True)
            pb.pb_batch_set_streams(1)
            e1, i1 = pb.pb_batch_solve(ctxs, sets, tol=1e-7, maxit=2000, use_graph=True)
            _, i_single = pb.pb_batch_solve(ctxs[:1], sets[:1], tol=1e-7, maxit=2000, use_graph=True)
        finally:
            pb.pb_batch_set_streams(2)
            for c in ctxs:
                pb.pb_destroy(c)
    assert i2["streams"] == 2 and i1["streams"] == 1 and i_single["streams"] == 1
    assert i2["converged"] == i2["instances"] == i1["converged"] == i1["instances"]
    for a, b in zip(e2, e1):
        assert a == pytest.approx(b, rel=2e-6, abs=1e-9)
    with pytest.raises(pb.PBError):
        pb.pb_batch_set_streams(3)


def test_two_engines_from_the_legacy_default_stream():
    """Contexts on the legacy default stream: the first engine launches its
    kernels one by one there (no graph), the second runs on the call's own
    stream; the energies equal the one-engine run's."""
    pb = _pb()
    mix = _mix()[:4]
    ctxs = [pb.pb_create(p.surface.centroids, p.surface.normals, p.surface.areas, sets[0], p.eps1, p.eps2, p.kappa,
                         stream=None) for p, sets in mix]
    try:
        sets = [s for _, s in mix]
        e2, i2 = pb.pb_batch_solve(ctxs, sets, tol=1e-7, maxit=2000, use_graph=True)
        pb.pb_batch_set_streams(1)
        e1, _ = pb.pb_batch_solve(ctxs, sets, tol=1e-7, maxit=2000, use_graph=True)
    finally:
        pb.pb_batch_set_streams(2)
        for c in ctxs:
            pb.pb_destroy(c)
    assert i2["streams"] == 2 and i2["converged"] == i2["instances"]
    for a, b in zip(e2, e1):
        assert a == pytest.approx(b, rel=2e-6, abs=1e-9)
