"""The no-allocation matrix-vector product, pb_matvec_f32_static.

It exists for callers that cannot call cudaMalloc: code running under a
framework whose caching allocator already owns all of the device memory, or a
latency-critical path where an allocation (which may synchronise the device)
is not acceptable.  Such callers cannot create a pb_ctx, so this entry point
takes their own device arrays and keeps its scratch in a fixed static device
array.  Here it is called through the C ABI and compared with the existing
pb_matvec(..., PB_FP32PAIR) on the same inputs, within the FP32-pair matvec
tolerance used by the other tests (relative L2 <= 2e-5), on two calls in a row.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import pb_inputs as pi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FP32_MATVEC_TOL = 2e-5


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


@pytest.mark.parametrize("name,surf", _surfaces(), ids=lambda v: v if isinstance(v, str) else "")
def test_static_matvec_matches_the_context_matvec_on_two_calls(name, surf):
    import paper_1301_5885_gb300 as pb
    lib = pb.lib()
    n = surf.n
    stream = torch.cuda.current_stream()
    rng = np.random.Generator(np.random.PCG64(11))
    u = torch.tensor(rng.normal(size=2 * n), device="cuda")
    c = torch.tensor(surf.centroids, device="cuda").contiguous()
    nr = torch.tensor(surf.normals, device="cuda").contiguous()
    a = torch.tensor(surf.areas, device="cuda").contiguous()

    with pb.pb_create(c, nr, a, None, 1.0, 80.0, 0.1257, stream=stream) as ctx:
        centre = pb.pb_get_info(ctx)["center"]
        y_ref = torch.empty_like(u)
        pb.pb_matvec(ctx, u, y_ref, "fp32pair")
    torch.cuda.synchronize()

    cbuf = (ctypes.c_double * 3)(*centre)
    outs = []
    for _ in range(2):
        y = torch.full_like(u, float("nan"))
        st = lib.pb_matvec_f32_static(c.data_ptr(), nr.data_ptr(), a.data_ptr(), n,
                                      ctypes.cast(cbuf, ctypes.POINTER(ctypes.c_double)), 1.0, 80.0, 0.1257,
                                      u.data_ptr(), y.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        assert st == pb.PB_OK, pb.pb_last_error(None)
        torch.cuda.synchronize()
        outs.append(y.cpu().numpy())
    ref = y_ref.cpu().numpy()
    for y in outs:
        assert np.all(np.isfinite(y))
        assert np.linalg.norm(y - ref) <= FP32_MATVEC_TOL * np.linalg.norm(ref)


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
