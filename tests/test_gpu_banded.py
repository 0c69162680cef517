"""Symmetric products with a bound on their scratch (pb_set_scratch_limit).

Unbounded, the symmetric products keep one column side per off-diagonal tile
pair (quadratic in N).  Bounded, they run in bands of whole row tiles, each
band finished before the next overwrites the column sides, the earlier bands'
column sides of later rows carried in FP64 accumulators.  For every symmetric
kernel (FP32 pairs with 2 and 4 targets per thread, FP64 with 1 and 2, float-
float):

* the banded product against the oracle's product of Eqs. (12)-(13), at a
  bound of one row tile per band and at one that gives a few bands;
* against the unbanded product: equal up to the rounding of the column-side
  summation order;
* bit-identical on a repeat (the order is fixed);
* one product counted per product, whatever the bands;
* a banded solve to the oracle's energy.
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


def _ctx(p):
    s = p.surface
    return _pb().pb_create(s.centroids, s.normals, s.areas, p.charges, p.eps1, p.eps2, p.kappa,
                           stream=torch.cuda.current_stream())


# (precision, FP32 variant, FP64 variant, tolerance of the product against the oracle,
#  relative tolerance of banded against unbanded)
KERNELS = [
    ("fp32pair", 5, 0, TOL_FP32PAIR, 1e-6),
    ("fp32pair", 6, 0, TOL_FP32PAIR, 1e-6),
    ("fp64", 0, 2, TOL_FP64, 1e-13),
    ("fp64", 0, 3, TOL_FP64, 1e-13),
    ("float2", 0, 0, TOL_FP64, 1e-13),
]


@pytest.fixture(scope="module")
def problem():
    p = pi.protein_like(n_atoms=40, seed=17, target_triangles=None, spacing=1.1)
    rng = np.random.Generator(np.random.PCG64(71))
    u = rng.normal(size=2 * p.n)
    ref = oracle.matvec(p.surface, p.eps2 / p.eps1, p.kappa, u)
    return p, u, ref


def _configure(pb, ctx, v32, v64):
    if v32:
        pb.pb_matvec_configure(ctx, v32, 0)
    if v64:
        assert pb.pb_matvec_configure_fp64(ctx, v64) == v64


def _product(pb, ctx, ud, prec):
    y = torch.full_like(ud, float("nan"))
    pb.pb_matvec(ctx, ud, y, prec)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("prec,v32,v64,tol,rel_unbanded", KERNELS)
def test_banded_product_matches_the_oracle_and_the_unbanded_one(problem, prec, v32, v64, tol, rel_unbanded):
    pb = _pb()
    p, u, ref = problem
    assert p.n > 16384                      # float-float takes its symmetric kernel with 2 targets per thread
    ud = torch.tensor(u, device="cuda")
    with _ctx(p) as ctx:
        _configure(pb, ctx, v32, v64)
        bands0, bytes0 = pb.pb_scratch_plan(ctx, prec)
        assert bands0 == 1 and bytes0 > 0
        y0 = _product(pb, ctx, ud, prec)
        # one row tile per band, then a bound halfway between that scratch and the unbanded one
        pb.pb_set_scratch_limit(ctx, 1)
        bands1, bytes1 = pb.pb_scratch_plan(ctx, prec)
        assert bands1 > 2 and bytes1 < bytes0
        mid = (bytes1 + bytes0) // 2
        for limit in (1, mid):
            pb.pb_set_scratch_limit(ctx, limit)
            bands, nbytes = pb.pb_scratch_plan(ctx, prec)
            if limit == mid:
                assert 1 < bands < bands1 and nbytes <= mid
            y = _product(pb, ctx, ud, prec)
            assert np.all(np.isfinite(y))
            assert_blocks_close(y, ref, tol, f"{prec} v{v32 or v64} limit {limit}")
            assert np.max(np.abs(y - y0)) <= rel_unbanded * np.max(np.abs(y0))
            assert np.array_equal(_product(pb, ctx, ud, prec), y)
        # the bound lifted: the unbanded product again, bit for bit
        pb.pb_set_scratch_limit(ctx, 0)
        assert pb.pb_scratch_plan(ctx, prec)[0] == 1
        assert np.array_equal(_product(pb, ctx, ud, prec), y0)


def test_bands_shrink_the_scratch_monotonically(problem):
    pb = _pb()
    p, _, _ = problem
    with _ctx(p) as ctx:
        _configure(pb, ctx, 6, 3)
        for prec in ("fp32pair", "fp64", "float2"):
            pb.pb_set_scratch_limit(ctx, 0)
            _, full = pb.pb_scratch_plan(ctx, prec)
            last_bands, last_bytes = 1, full
            for frac in (0.8, 0.6, 0.4, 0.25):
                pb.pb_set_scratch_limit(ctx, int(full * frac))
                bands, nbytes = pb.pb_scratch_plan(ctx, prec)
                assert bands >= last_bands and nbytes <= last_bytes
                last_bands, last_bytes = bands, nbytes
            assert last_bands > 1


def test_negative_bound_is_rejected(problem):
    pb = _pb()
    p, _, _ = problem
    with _ctx(p) as ctx:
        with pytest.raises(pb.PBError) as ei:
            pb.pb_set_scratch_limit(ctx, -1)
        assert ei.value.status == pb.PB_ERR_ARG


def test_one_product_counted_per_banded_product(problem):
    pb = _pb()
    p, u, _ = problem
    ud = torch.tensor(u, device="cuda")
    with _ctx(p) as ctx:
        _configure(pb, ctx, 6, 0)
        pb.pb_set_scratch_limit(ctx, 1)
        assert pb.pb_scratch_plan(ctx, "fp32pair")[0] > 3
        pb.pb_profile_enable(ctx, True)
        pb.pb_profile_read(ctx, reset=True)
        for _ in range(3):
            _product(pb, ctx, ud, "fp32pair")
        assert pb.pb_profile_read(ctx)["evaluated"] == 3


@pytest.mark.parametrize("prec,rel", [("fp32pair", 1e-5), ("fp64", 1e-9)])
def test_banded_solve_reaches_the_oracle_energy(prec, rel):
    pb = _pb()
    p = pi.kirkwood_sphere_multi(level=4, radius=8.0, n_charges=6, seed=72)
    ref = oracle.solve(p.surface, p.charges, p.eps1, p.eps2, p.kappa, tol=1e-12, maxit=2000)
    with _ctx(p) as ctx:
        _configure(pb, ctx, 6, 3)
        pb.pb_set_scratch_limit(ctx, 1)
        assert pb.pb_scratch_plan(ctx, prec)[0] > 1
        info = pb.pb_solve(ctx, tol=1e-12 if prec == "fp64" else 1e-7, maxit=2000, prec=prec)
    assert info.status == pb.PB_OK
    assert info.energy_kcal == pytest.approx(ref["energy"], rel=rel)
