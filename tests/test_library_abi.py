"""The C-ABI library builds, loads and exports every symbol include/pb.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1301_5885_gb300 as pb
import importlib
pkg_build = importlib.import_module("paper_1301_5885_gb300.build")

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "pb.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pb_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return pb.lib()


def test_every_declared_symbol_is_exported_and_bound(lib):
    names = _declared()
    assert "pb_create" in names and "pb_matvec" in names and "pb_solve" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(pb.SIGNATURES)


def test_status_strings(lib):
    for code, name in enumerate(["PB_OK", "PB_ERR_ARG", "PB_ERR_BADMESH", "PB_ERR_OOM", "PB_ERR_CUDA",
                                 "PB_ERR_NOCONV", "PB_ERR_NAN", "PB_ERR_TIMEOUT", "PB_ERR_ADMIT"]):
        assert pb.pb_status_string(code) == name
    assert pb.pb_status_string(99) == "PB_UNKNOWN_STATUS"


def test_create_rejects_bad_arguments_before_any_device_work(lib):
    out = ctypes.c_void_p(123)
    c = np.zeros(3)
    # NULL geometry
    assert lib.pb_create(None, None, None, 1, None, 0, 1.0, 80.0, 0.0, None, ctypes.byref(out)) == pb.PB_ERR_ARG
    assert out.value is None
    assert "NULL" in pb.pb_last_error(None)
    # N <= 0
    assert lib.pb_create(c.ctypes.data, c.ctypes.data, c.ctypes.data, 0, None, 0, 1.0, 80.0, 0.0, None,
                         ctypes.byref(out)) == pb.PB_ERR_ARG
    # non-positive dielectric, negative kappa
    for e1, e2, k in [(0.0, 80.0, 0.0), (1.0, -1.0, 0.0), (1.0, 80.0, -0.1), (float("nan"), 80.0, 0.0)]:
        assert lib.pb_create(c.ctypes.data, c.ctypes.data, c.ctypes.data, 1, None, 0, e1, e2, k, None,
                             ctypes.byref(out)) == pb.PB_ERR_ARG
    # charges announced but missing
    assert lib.pb_create(c.ctypes.data, c.ctypes.data, c.ctypes.data, 1, None, 3, 1.0, 80.0, 0.0, None,
                         ctypes.byref(out)) == pb.PB_ERR_ARG
    # NULL out pointer
    assert lib.pb_create(c.ctypes.data, c.ctypes.data, c.ctypes.data, 1, None, 0, 1.0, 80.0, 0.0, None,
                         None) == pb.PB_ERR_ARG


def test_null_context_calls_fail_cleanly(lib):
    assert lib.pb_matvec(None, None, None, 0) == pb.PB_ERR_ARG
    assert lib.pb_solve(None, None, None, None, None) == pb.PB_ERR_ARG
    e = ctypes.c_double()
    assert lib.pb_energy(None, ctypes.byref(e)) == pb.PB_ERR_ARG
    assert lib.pb_set_charges(None, None, 0) == pb.PB_ERR_ARG
    lib.pb_destroy(None)


def test_python_binding_raises_without_cpu_fallback(lib):
    with pytest.raises(pb.PBError) as ei:
        pb.pb_create(np.zeros((1, 3)), np.zeros((1, 3)), np.ones(1), None, 1.0, -80.0, 0.0)
    assert ei.value.status == pb.PB_ERR_ARG


def test_batched_product_shapes_and_overrides_are_checked_on_the_host(lib):
    for width in (1, 2, 4, 8):
        shapes = pb.pb_batch_shapes(width)
        assert len(shapes) >= 4 and len(set(shapes)) == len(shapes)
        assert all(t in (1, 2, 4) and r in pb._ffi.ROW_SUMS for t, r in shapes)
    assert pb.pb_batch_shapes(3) == []
    with pytest.raises(pb.PBError):
        pb.pb_batch_force_shape(3, 2, 0)
    with pytest.raises(pb.PBError):
        pb.pb_batch_force_shape(8, 4, 0)            # not instantiated
    t, r = pb.pb_batch_shapes(8)[1]
    pb.pb_batch_force_shape(8, t, r, 2)
    pb.pb_batch_force_shape(8)                      # cleared
    assert lib.pb_batch_set_tuning(2) == pb.PB_ERR_ARG
    pb.pb_batch_set_tuning(True)
    pb.pb_batch_clear_tuning()
