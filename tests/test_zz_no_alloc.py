"""The no-allocation matrix-vector product, pb_matvec_f32_static.

It exists for callers that cannot call cudaMalloc: code running under a
framework whose caching allocator already owns all of the device memory, or a
latency-critical path where an allocation (which may synchronise the device)
is not acceptable.  Such callers cannot create a pb_ctx, so this entry point
takes their own device arrays and keeps its scratch in a fixed static device
array.  Here it is called through the C ABI and compared, on two calls in a
row, with the FP64 oracle's product and with the existing
pb_matvec(..., PB_FP32PAIR) on the same inputs, each row block (phi rows, psi
rows) within the FP32-pair tolerance of the other tests (relative L2 2e-5,
element-wise 1e-4 of the block's largest entry).  This file is collected last
on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
import pb_inputs as pi
from blockcheck import TOL_FP32PAIR, assert_blocks_close, assert_rows_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import importlib
    importlib.import_module("paper_1301_5885_gb300.build").build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _surfaces():
    big = pi.icosphere(12.0, 5)                       # 20,480 triangles: several tiles and split tiles
    return [("ico5", big), ("ragged4099", big.subset(np.arange(4099) * 4)),
            ("solute", pi.protein_like(n_atoms=30, seed=2, target_triangles=None, spacing=1.0).surface)]


def _static_calls(surf, u_host, calls=2, kappa=0.1257):
    """Two static products and the context product of the same u."""
    import paper_1301_5885_gb300 as pb
    lib = pb.lib()
    n = surf.n
    stream = torch.cuda.current_stream()
    u = torch.tensor(u_host, device="cuda")
    c = torch.tensor(surf.centroids, device="cuda").contiguous()
    nr = torch.tensor(surf.normals, device="cuda").contiguous()
    a = torch.tensor(surf.areas, device="cuda").contiguous()

    with pb.pb_create(c, nr, a, None, 1.0, 80.0, kappa, stream=stream) as ctx:
        centre = pb.pb_get_info(ctx)["center"]
        y_ref = torch.empty_like(u)
        pb.pb_matvec(ctx, u, y_ref, "fp32pair")
    torch.cuda.synchronize()

    cbuf = (ctypes.c_double * 3)(*centre)
    outs = []
    for _ in range(calls):
        y = torch.full_like(u, float("nan"))
        st = lib.pb_matvec_f32_static(c.data_ptr(), nr.data_ptr(), a.data_ptr(), n,
                                      ctypes.cast(cbuf, ctypes.POINTER(ctypes.c_double)), 1.0, 80.0, kappa,
                                      u.data_ptr(), y.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        assert st == pb.PB_OK, pb.pb_last_error(None)
        torch.cuda.synchronize()
        outs.append(y.cpu().numpy())
    return outs, y_ref.cpu().numpy()


@pytest.mark.parametrize("name,surf", _surfaces(), ids=lambda v: v if isinstance(v, str) else "")
def test_static_matvec_matches_the_oracle_and_the_context_matvec_on_two_calls(name, surf):
    rng = np.random.Generator(np.random.PCG64(11))
    u = rng.normal(size=2 * surf.n)
    outs, ctx_y = _static_calls(surf, u)
    ref = oracle.matvec(surf, 80.0, 0.1257, u)
    assert_blocks_close(ctx_y, ref, TOL_FP32PAIR, "pb_matvec")
    for k, y in enumerate(outs):
        assert_blocks_close(y, ref, TOL_FP32PAIR, f"static call {k}")
        assert_blocks_close(y, ctx_y, TOL_FP32PAIR, f"static call {k} vs pb_matvec")


def test_static_matvec_with_more_target_tiles_than_ctas():
    """327,680 triangles = 640 target tiles of 512, more than the persistent
    grid's CTAs: CTAs then cover whole middle tiles between a first and a last
    partial one, which exercises both partial slots of every CTA.  Checked on
    sampled rows (first and last included) against the oracle and in full
    against pb_matvec."""
    surf = pi.icosphere(40.0, 7)
    rng = np.random.Generator(np.random.PCG64(12))
    u = rng.normal(size=2 * surf.n)
    rows = np.sort(rng.choice(surf.n, 64, replace=False))
    rows[0], rows[-1] = 0, surf.n - 1
    r1, r2 = oracle.matvec_rows(surf, 80.0, 0.1257, u, rows)
    outs, ctx_y = _static_calls(surf, u)
    for k, y in enumerate(outs):
        assert_rows_close(y[rows], y[surf.n + rows], r1, r2, TOL_FP32PAIR, f"static call {k}")
        assert_blocks_close(y, ctx_y, TOL_FP32PAIR, f"static call {k} vs pb_matvec")


def test_static_matvec_rejects_an_output_overlapping_its_input():
    import paper_1301_5885_gb300 as pb
    lib = pb.lib()
    n = 64
    u = torch.zeros(2 * n + 1, dtype=torch.float64, device="cuda")
    g = torch.ones(3 * n, dtype=torch.float64, device="cuda")
    st = lib.pb_matvec_f32_static(g.data_ptr(), g.data_ptr(), g.data_ptr(), n, None, 1.0, 80.0, 0.0,
                                  u.data_ptr(), u.data_ptr() + 8, None)
    assert st == pb.PB_ERR_ARG
    assert "must not overlap" in pb.pb_last_error(None)
    st = lib.pb_matvec_f32_static(g.data_ptr(), g.data_ptr(), g.data_ptr(), n, None, 1.0, 80.0, 0.0,
                                  u.data_ptr(), g.data_ptr() + 16, None)
    assert st == pb.PB_ERR_ARG


def test_static_matvec_rejects_sizes_beyond_its_fixed_scratch():
    import paper_1301_5885_gb300 as pb
    lib = pb.lib()
    u = torch.zeros(4, dtype=torch.float64, device="cuda")
    y = torch.zeros(4, dtype=torch.float64, device="cuda")
    too_big = (1 << 24) + 1
    st = lib.pb_matvec_f32_static(u.data_ptr(), u.data_ptr(), u.data_ptr(), too_big, None, 1.0, 80.0, 0.0,
                                  u.data_ptr(), y.data_ptr(), None)
    assert st == pb.PB_ERR_ARG
    assert "exceeds the maximum" in pb.pb_last_error(None)
