"""Symmetric products in bands of row tiles (pb_set_bands, pb_set_scratch_limit).

In one pass the symmetric products keep one column side per off-diagonal
tile pair (quadratic in N).  In bands they run over whole row tiles at a
time, each band finished before its set of column sides is reused, the
earlier bands' column sides of later rows carried in FP64 accumulators, and
consecutive bands on two streams.  For every symmetric kernel (FP32 pairs
with 2 and 4 targets per thread, FP64 with 1 and 2, float-float):

* the banded product against the oracle's product of Eqs. (12)-(13), for
  band counts of both parities (the last band on either stream) and one row
  tile per band;
* against the one-pass product: equal up to the rounding of the column-side
  summation order; bit-identical on a repeat (the order is fixed);
* the automatic split and the scratch bound never take more scratch than one
  pass unless bands are requested;
* one product counted per product, whatever the bands;
* a banded solve to the oracle's energy.
The scratch bound at full size is in test_gpu_fullsize.py.
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
#  relative tolerance of banded against one pass)
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


@pytest.mark.parametrize("prec,v32,v64,tol,rel_one_pass", KERNELS)
def test_banded_product_matches_the_oracle_and_the_one_pass_product(problem, prec, v32, v64, tol, rel_one_pass):
    pb = _pb()
    p, u, ref = problem
    assert p.n > 16384                      # float-float takes its symmetric kernel with 2 targets per thread
    ud = torch.tensor(u, device="cuda")
    with _ctx(p) as ctx:
        _configure(pb, ctx, v32, v64)
        pb.pb_set_bands(ctx, 1)
        assert pb.pb_scratch_plan(ctx, prec)[0] == 1
        y0 = _product(pb, ctx, ud, prec)
        assert_blocks_close(y0, ref, tol, f"{prec} one pass")
        parities = set()
        for req in (2, 3, 7, 1 << 20):      # the last: one row tile per band
            pb.pb_set_bands(ctx, req)
            bands = pb.pb_scratch_plan(ctx, prec)[0]
            assert bands >= 2
            parities.add(bands % 2)
            y = _product(pb, ctx, ud, prec)
            assert np.all(np.isfinite(y))
            assert_blocks_close(y, ref, tol, f"{prec} v{v32 or v64} {bands} bands")
            assert np.max(np.abs(y - y0)) <= rel_one_pass * np.max(np.abs(y0))
            assert np.array_equal(_product(pb, ctx, ud, prec), y)
        assert parities == {0, 1}
        # back to one pass: the first product, bit for bit
        pb.pb_set_bands(ctx, 1)
        assert np.array_equal(_product(pb, ctx, ud, prec), y0)


def test_unrequested_bands_never_take_more_scratch(problem):
    """The automatic split and the scratch bound keep one pass where bands
    would need more scratch (two sets of slots and column sides): at this
    size a bound below the one-pass scratch cannot be met and is exceeded."""
    pb = _pb()
    p, _, _ = problem
    with _ctx(p) as ctx:
        _configure(pb, ctx, 6, 3)
        for prec in ("fp32pair", "fp64", "float2"):
            pb.pb_set_bands(ctx, 1)
            pb.pb_set_scratch_limit(ctx, 0)
            one = pb.pb_scratch_plan(ctx, prec)
            assert one[0] == 1
            pb.pb_set_bands(ctx, 0)
            auto = pb.pb_scratch_plan(ctx, prec)
            assert auto[1] <= one[1]
            for frac in (0.9, 0.5, 1e-6):
                pb.pb_set_scratch_limit(ctx, max(1, int(one[1] * frac)))
                bands, nbytes = pb.pb_scratch_plan(ctx, prec)
                assert nbytes <= one[1]


def test_negative_requests_are_rejected(problem):
    pb = _pb()
    p, _, _ = problem
    with _ctx(p) as ctx:
        for call in (lambda: pb.pb_set_scratch_limit(ctx, -1), lambda: pb.pb_set_bands(ctx, -1)):
            with pytest.raises(pb.PBError) as ei:
                call()
            assert ei.value.status == pb.PB_ERR_ARG


def test_one_product_counted_per_banded_product(problem):
    pb = _pb()
    p, u, _ = problem
    ud = torch.tensor(u, device="cuda")
    with _ctx(p) as ctx:
        _configure(pb, ctx, 6, 0)
        pb.pb_set_bands(ctx, 7)
        assert pb.pb_scratch_plan(ctx, "fp32pair")[0] >= 7
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
        pb.pb_set_bands(ctx, 4)
        assert pb.pb_scratch_plan(ctx, prec)[0] >= 4
        info = pb.pb_solve(ctx, tol=1e-12 if prec == "fp64" else 1e-7, maxit=2000, prec=prec)
    assert info.status == pb.PB_OK
    assert info.energy_kcal == pytest.approx(ref["energy"], rel=rel)
