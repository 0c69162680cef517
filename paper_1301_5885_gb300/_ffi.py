"""ctypes binding of include/pb.h: the same entry points under the same names.

Argument marshalling only: every numerical step runs in libgabipb.so's CUDA
kernels.  Device vectors are torch CUDA tensors (float64, contiguous); geometry
and charges may be numpy arrays (host) or torch tensors (host or device).
The library must have been built (``build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np

from . import build as _build

PB_OK, PB_ERR_ARG, PB_ERR_BADMESH, PB_ERR_OOM, PB_ERR_CUDA, PB_ERR_NOCONV, PB_ERR_NAN, PB_ERR_TIMEOUT, PB_ERR_ADMIT = range(9)
PB_FP64, PB_FP32PAIR, PB_FLOAT2 = 0, 1, 2
PRECISIONS = {"fp64": PB_FP64, "fp32pair": PB_FP32PAIR, "float2": PB_FLOAT2,
              PB_FP64: PB_FP64, PB_FP32PAIR: PB_FP32PAIR, PB_FLOAT2: PB_FLOAT2}


class PBError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_string(status)}: {message}")
        self.status = status


class _Opts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("tol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("prec", ctypes.c_int), ("refine", ctypes.c_int), ("refine_prec", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("cycles", ctypes.c_int), ("rel_resid", ctypes.c_double),
                ("energy_kcal", ctypes.c_double), ("rel_resid_fp64", ctypes.c_double),
                ("refine_steps", ctypes.c_int), ("matvecs", ctypes.c_int64)]


class _BatchInfo(ctypes.Structure):
    _fields_ = [("instances", ctypes.c_int), ("converged", ctypes.c_int), ("cycles", ctypes.c_int),
                ("iters_max", ctypes.c_int), ("iters_sum", ctypes.c_int64), ("rel_resid_max", ctypes.c_double),
                ("rhs_width", ctypes.c_int), ("ctas", ctypes.c_int64), ("pair_evals", ctypes.c_int64),
                ("pair_products", ctypes.c_int64), ("matvec_launches", ctypes.c_int64),
                ("matvec_ms", ctypes.c_double), ("targets_per_thread", ctypes.c_int), ("row_sums", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_int), ("tuned", ctypes.c_int), ("tune_candidates", ctypes.c_int),
                ("tune_ms", ctypes.c_double), ("setup_ms", ctypes.c_double), ("cycles_ms", ctypes.c_double),
                ("energy_ms", ctypes.c_double), ("streams", ctypes.c_int)]


class _ServerOpts(ctypes.Structure):
    _fields_ = [("max_active", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_int64), ("restart", ctypes.c_int),
                ("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("split_n", ctypes.c_int64)]


class _ServerResult(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int), ("iters", ctypes.c_int),
                ("energy_kcal", ctypes.c_double), ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("n", ctypes.c_int64)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("failed", ctypes.c_int64), ("cycles", ctypes.c_int64),
                ("pair_evals", ctypes.c_int64), ("pair_products", ctypes.c_int64), ("active", ctypes.c_int),
                ("pending", ctypes.c_int), ("max_active_seen", ctypes.c_int), ("used_bytes", ctypes.c_int64)]


class _CtxInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nc", ctypes.c_int64), ("eps1", ctypes.c_double),
                ("eps2", ctypes.c_double), ("kappa", ctypes.c_double), ("center", ctypes.c_double * 3),
                ("gauss_min", ctypes.c_double), ("gauss_max", ctypes.c_double), ("device_bytes", ctypes.c_int64)]


# Every symbol include/pb.h declares, with (restype, argtypes).
_VP, _D, _I64, _I = ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, ctypes.c_int
SIGNATURES = {
    "pb_create": (_I, [_VP, _VP, _VP, _I64, _VP, _I64, _D, _D, _D, _VP, ctypes.POINTER(_VP)]),
    "pb_set_charges": (_I, [_VP, _VP, _I64]),
    "pb_source": (_I, [_VP, _VP, _I]),
    "pb_matvec": (_I, [_VP, _VP, _VP, _I]),
    "pb_solve": (_I, [_VP, ctypes.POINTER(_Opts), _VP, _VP, ctypes.POINTER(_Info)]),
    "pb_energy": (_I, [_VP, ctypes.POINTER(_D)]),
    "pb_energy_of": (_I, [_VP, _VP, _I, ctypes.POINTER(_D)]),
    "pb_get_info": (_I, [_VP, ctypes.POINTER(_CtxInfo)]),
    "pb_destroy": (None, [_VP]),
    "pb_status_string": (ctypes.c_char_p, [_I]),
    "pb_last_error": (ctypes.c_char_p, [_VP]),
    "pb_kernel_launches": (ctypes.c_uint64, []),
    "pb_release_cached_memory": (_I, []),
    "pb_profile_enable": (_I, [_VP, _I]),
    "pb_profile_read": (_I, [_VP, ctypes.POINTER(_D), ctypes.POINTER(_I64), ctypes.POINTER(_I64), _I]),
    "pb_matvec_f32_static": (_I, [_VP, _VP, _VP, _I64, ctypes.POINTER(_D), _D, _D, _D, _VP, _VP, _VP]),
    "pb_matvec_configure": (_I, [_VP, _I, _I]),
    "pb_server_create": (_I, [ctypes.POINTER(_ServerOpts), ctypes.POINTER(_VP)]),
    "pb_server_submit": (_I, [_VP, _VP, _VP, _VP, _I64, _VP, _I64, _D, _D, _D, ctypes.POINTER(ctypes.c_uint64)]),
    "pb_server_poll": (_I, [_VP, ctypes.POINTER(_ServerResult), _I]),
    "pb_server_wait": (_I, [_VP, _I64, _D]),
    "pb_server_get_stats": (_I, [_VP, ctypes.POINTER(_ServerStats)]),
    "pb_server_destroy": (None, [_VP]),
    "pb_batch_solve": (_I, [ctypes.POINTER(_VP), _I, ctypes.POINTER(_VP), ctypes.POINTER(_I64), ctypes.POINTER(_I),
                            ctypes.POINTER(_Opts), _I, ctypes.POINTER(_D), ctypes.POINTER(_BatchInfo)]),
    "pb_matvec_get_config": (_I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I64)]),
    "pb_matvec_autotune": (_I, [_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "pb_matvec_configure_fp64": (_I, [_VP, _I, ctypes.POINTER(_I)]),
    "pb_set_scratch_limit": (_I, [_VP, _I64]),
    "pb_set_bands": (_I, [_VP, _I]),
    "pb_sym_band_plan": (_I, [_I64, _I, _I64, _I, _I64, _I, ctypes.POINTER(_I64), _I, ctypes.POINTER(_I),
                              ctypes.POINTER(_I64)]),
    "pb_scratch_plan": (_I, [_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_I64)]),
    "pb_matvec_rows": (_I, [_VP, _VP, _VP, _I64, _I64, _I]),
    "pb_solve_sharded": (_I, [_VP, ctypes.POINTER(_Opts), _I, _I, _VP, _VP, _VP, _VP, ctypes.POINTER(_Info)]),
    "pb_shard_rows": (_I, [_I64, _I, _I, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "pb_shard_unpack_host": (_I, [_VP, _I64, _I, _VP]),
    "pb_batch_set_tuning": (_I, [_I]),
    "pb_batch_set_streams": (_I, [_I]),
    "pb_batch_force_shape": (_I, [_I, _I, _I, _I]),
    "pb_batch_clear_tuning": (_I, []),
    "pb_batch_shapes": (_I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_I), _I]),
}

ROW_SUMS = {0: "fp64-registers", 1: "fp64-shared", 2: "float-float-registers", 3: "float-float-shared"}

_LIB = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libgabipb.so (it must already be built: no silent rebuild, no fallback)."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: run paper_1301_5885_gb300.build.build() first "
                              "(there is no CPU fallback for this library)")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def status_string(s: int) -> str:
    try:
        return lib().pb_status_string(int(s)).decode()
    except Exception:  # pragma: no cover - only when the library itself is unavailable
        return f"status {s}"


def pb_status_string(s: int) -> str:
    return status_string(s)


def pb_last_error(ctx=None) -> str:
    h = ctx.handle if isinstance(ctx, Context) else ctx
    msg = lib().pb_last_error(h)
    return msg.decode() if msg else ""


def pb_kernel_launches() -> int:
    return int(lib().pb_kernel_launches())


def pb_release_cached_memory() -> None:
    """Return the library pool's unused device memory and cached pinned blocks."""
    _check(lib().pb_release_cached_memory())


def _check(status: int, ctx=None):
    if status != PB_OK:
        raise PBError(status, pb_last_error(ctx))


def _ptr_f64(a, length: int | None = None, name: str = "array", keep=None):
    """Pointer to float64 contiguous data from a numpy array or torch tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float64 or not a.is_contiguous():
                a = a.to(torch.float64).contiguous()
            if length is not None and a.numel() != length:
                raise ValueError(f"{name}: expected {length} elements, got {a.numel()}")
            if keep is not None:
                keep.append(a)
            return a.data_ptr()
    except ImportError:  # pragma: no cover
        pass
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if length is not None and arr.size != length:
        raise ValueError(f"{name}: expected {length} elements, got {arr.size}")
    if keep is not None:
        keep.append(arr)
    return arr.ctypes.data


def _device_vec(t, n2: int, name: str):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA torch tensor")
    if t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != n2:
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor of length {n2}")
    return t.data_ptr()


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class Context:
    """An owned pb_ctx handle."""

    def __init__(self, handle, n: int, nc: int, stream=None):
        self.handle = handle
        self.n = n
        self.nc = nc
        self.stream = stream

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        pb_destroy(self)

    def __del__(self):
        try:
            pb_destroy(self)
        except Exception:
            pass


@dataclasses.dataclass
class SolveInfo:
    status: int
    iters: int
    cycles: int
    rel_resid: float
    energy_kcal: float
    rel_resid_fp64: float
    refine_steps: int
    matvecs: int


def pb_create(centroids, normals, areas, charges, eps1: float, eps2: float, kappa: float, stream=None) -> Context:
    keep = []
    n = int(np.prod(np.shape(areas)))
    q = charges if charges is not None else np.zeros((0, 4))
    nc = int(np.prod(np.shape(q))) // 4
    out = ctypes.c_void_p()
    st = lib().pb_create(_ptr_f64(centroids, 3 * n, "centroids", keep), _ptr_f64(normals, 3 * n, "normals", keep),
                         _ptr_f64(areas, n, "areas", keep), n,
                         _ptr_f64(q, 4 * nc, "charges", keep) if nc > 0 else None, nc,
                         float(eps1), float(eps2), float(kappa), _stream_ptr(stream), ctypes.byref(out))
    _check(st)
    return Context(out.value, n, nc, stream)


def pb_set_charges(ctx: Context, charges) -> None:
    keep = []
    nc = int(np.prod(np.shape(charges))) // 4
    _check(lib().pb_set_charges(ctx.handle, _ptr_f64(charges, 4 * nc, "charges", keep) if nc > 0 else None, nc), ctx)
    ctx.nc = nc


def pb_source(ctx: Context, b, prec="fp64") -> None:
    _check(lib().pb_source(ctx.handle, _device_vec(b, 2 * ctx.n, "b"), PRECISIONS[prec]), ctx)


def pb_matvec(ctx: Context, u, y, prec="fp32pair") -> None:
    _check(lib().pb_matvec(ctx.handle, _device_vec(u, 2 * ctx.n, "u"), _device_vec(y, 2 * ctx.n, "y"),
                           PRECISIONS[prec]), ctx)


def pb_solve(ctx: Context, restart: int = 10, tol: float = 1e-4, maxit: int = 1000, prec="fp32pair",
             refine: int = 0, x0=None, x_out=None, raise_on_noconv: bool = True,
             refine_prec="fp64") -> SolveInfo:
    o = _Opts(int(restart), float(tol), int(maxit), PRECISIONS[prec], int(refine), PRECISIONS[refine_prec])
    info = _Info()
    x0p = _device_vec(x0, 2 * ctx.n, "x0") if x0 is not None else None
    xop = _device_vec(x_out, 2 * ctx.n, "x_out") if x_out is not None else None
    st = lib().pb_solve(ctx.handle, ctypes.byref(o), x0p, xop, ctypes.byref(info))
    if st != PB_OK and not (st == PB_ERR_NOCONV and not raise_on_noconv):
        _check(st, ctx)
    return SolveInfo(st, info.iters, info.cycles, info.rel_resid, info.energy_kcal, info.rel_resid_fp64,
                     info.refine_steps, info.matvecs)


def pb_matvec_rows(ctx: Context, u, y_rows, row0: int, nrows: int, prec="fp32pair") -> None:
    """Rows [row0, row0 + nrows) of both row blocks of A u into y_rows (2 nrows:
    phi rows, then psi rows); u is the full 2N device vector."""
    _check(lib().pb_matvec_rows(ctx.handle, _device_vec(u, 2 * ctx.n, "u"), _device_vec(y_rows, 2 * int(nrows), "y"),
                                int(row0), int(nrows), PRECISIONS[prec]), ctx)


def pb_shard_rows(n: int, world: int, rank: int):
    """(row0, nrows, rows_per_rank) of a rank in the row-sharded layout."""
    r0, nr, per = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().pb_shard_rows(int(n), int(world), int(rank), ctypes.byref(r0), ctypes.byref(nr), ctypes.byref(per)))
    return r0.value, nr.value, per.value


def pb_shard_unpack_host(gathered, n: int, world: int) -> np.ndarray:
    """The 2N vector [phi; psi] from a gathered host buffer of world blocks of
    2 P doubles (each rank's phi rows, then its psi rows, P slots each)."""
    g = np.ascontiguousarray(np.asarray(gathered, dtype=np.float64))
    per = (int(n) + int(world) - 1) // int(world)
    if g.size != 2 * per * int(world):
        raise ValueError(f"gathered buffer has {g.size} doubles, expected {2 * per * int(world)}")
    y = np.empty(2 * int(n))
    _check(lib().pb_shard_unpack_host(g.ctypes.data, int(n), int(world), y.ctypes.data))
    return y


class _DeviceArray:
    """A raw FP64 device array seen through __cuda_array_interface__, so that
    torch can wrap library-owned memory without a copy."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 2, "strides": None}


_GATHER_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                              ctypes.c_void_p)


def pb_solve_sharded(ctx: Context, group=None, restart: int = 10, tol: float = 1e-4, maxit: int = 1000,
                     prec="fp32pair", refine: int = 0, x0=None, x_out=None, raise_on_noconv: bool = True,
                     refine_prec="fp64", allgather=None) -> SolveInfo:
    """Row-sharded solve: this process is one rank of ``group`` (a
    torch.distributed process group, the default group if None), each rank on
    its own GPU with its own context of the whole surface.  Every product
    evaluates this rank's rows and gathers all ranks' rows with
    torch.distributed.all_gather_into_tensor on the context's stream.
    ``allgather(send, recv, count)``, if given, replaces the collective (it
    receives torch views of the library's buffers)."""
    import torch
    import torch.distributed as dist
    if allgather is None:
        world, rank = dist.get_world_size(group), dist.get_rank(group)
    else:
        world, rank = 1, 0
    stream = ctx.stream
    if stream is not None and not isinstance(stream, torch.cuda.Stream):
        stream = torch.cuda.ExternalStream(_stream_ptr(stream))
    errors = []

    def _gather(user, send, recv, count, cuda_stream):
        try:
            s = torch.as_tensor(_DeviceArray(send, count), device="cuda")
            r = torch.as_tensor(_DeviceArray(recv, count * world), device="cuda")
            st = stream if stream is not None else torch.cuda.default_stream()
            with torch.cuda.stream(st):
                if allgather is not None:
                    allgather(s, r, int(count))
                else:
                    dist.all_gather_into_tensor(r, s, group=group)
            return 0
        except Exception as e:          # reported through the status code
            errors.append(e)
            return 1

    cb = _GATHER_FN(_gather)
    o = _Opts(int(restart), float(tol), int(maxit), PRECISIONS[prec], int(refine), PRECISIONS[refine_prec])
    info = _Info()
    x0p = _device_vec(x0, 2 * ctx.n, "x0") if x0 is not None else None
    xop = _device_vec(x_out, 2 * ctx.n, "x_out") if x_out is not None else None
    st = lib().pb_solve_sharded(ctx.handle, ctypes.byref(o), int(rank), int(world), ctypes.cast(cb, ctypes.c_void_p),
                                None, x0p, xop, ctypes.byref(info))
    if errors:
        raise errors[0]
    if st != PB_OK and not (st == PB_ERR_NOCONV and not raise_on_noconv):
        _check(st, ctx)
    return SolveInfo(st, info.iters, info.cycles, info.rel_resid, info.energy_kcal, info.rel_resid_fp64,
                     info.refine_steps, info.matvecs)


def pb_energy(ctx: Context) -> float:
    e = ctypes.c_double()
    _check(lib().pb_energy(ctx.handle, ctypes.byref(e)), ctx)
    return e.value


def pb_energy_of(ctx: Context, u, prec="fp64") -> float:
    e = ctypes.c_double()
    _check(lib().pb_energy_of(ctx.handle, _device_vec(u, 2 * ctx.n, "u"), PRECISIONS[prec], ctypes.byref(e)), ctx)
    return e.value


def pb_get_info(ctx: Context) -> dict:
    i = _CtxInfo()
    _check(lib().pb_get_info(ctx.handle, ctypes.byref(i)), ctx)
    return {"n": i.n, "nc": i.nc, "eps1": i.eps1, "eps2": i.eps2, "kappa": i.kappa, "center": list(i.center),
            "gauss_min": i.gauss_min, "gauss_max": i.gauss_max, "device_bytes": i.device_bytes}


def pb_profile_enable(ctx: Context, enable: bool = True) -> None:
    _check(lib().pb_profile_enable(ctx.handle, 1 if enable else 0), ctx)


def pb_profile_read(ctx: Context, reset: bool = False) -> dict:
    ms, timed, ev = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().pb_profile_read(ctx.handle, ctypes.byref(ms), ctypes.byref(timed), ctypes.byref(ev),
                                 1 if reset else 0), ctx)
    return {"matvec_ms": ms.value, "timed_launches": timed.value, "evaluated": ev.value}


def pb_matvec_f32_static(centroids, normals, areas, u, y, eps1: float, eps2: float, kappa: float,
                         center=None, stream=None) -> None:
    """y = A u in FP32 pairs without any device allocation (see include/pb.h).
    centroids, normals, areas, u, y: contiguous float64 CUDA tensors."""
    import torch
    n = int(areas.numel())
    for name, t, ln in (("centroids", centroids, 3 * n), ("normals", normals, 3 * n), ("areas", areas, n)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
                and t.numel() == ln):
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor with {ln} elements")
    c = (ctypes.c_double * 3)(*[float(v) for v in center]) if center is not None else None
    st = lib().pb_matvec_f32_static(centroids.data_ptr(), normals.data_ptr(), areas.data_ptr(), n,
                                    ctypes.cast(c, ctypes.POINTER(ctypes.c_double)) if c is not None else None,
                                    float(eps1), float(eps2), float(kappa), _device_vec(u, 2 * n, "u"),
                                    _device_vec(y, 2 * n, "y"), _stream_ptr(stream))
    _check(st)


def pb_matvec_configure(ctx: Context, variant: int = 0, ctas_per_sm: int = 0) -> None:
    _check(lib().pb_matvec_configure(ctx.handle, int(variant), int(ctas_per_sm)), ctx)


def pb_matvec_get_config(ctx: Context) -> dict:
    v, c, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
    _check(lib().pb_matvec_get_config(ctx.handle, ctypes.byref(v), ctypes.byref(c), ctypes.byref(g)), ctx)
    return {"variant": v.value, "ctas_per_sm": c.value, "ctas": g.value}


def pb_matvec_configure_fp64(ctx: Context, variant: int = 0) -> int:
    """FP64 product variant: 1 plain, 2/3 symmetric (1/2 targets per thread), 0 default.
    Returns the variant in use."""
    v = ctypes.c_int()
    _check(lib().pb_matvec_configure_fp64(ctx.handle, int(variant), ctypes.byref(v)), ctx)
    return v.value


def pb_set_scratch_limit(ctx: Context, nbytes: int) -> None:
    """Bound each symmetric product's device scratch (0: no bound); the products
    then run in bands of row tiles."""
    _check(lib().pb_set_scratch_limit(ctx.handle, int(nbytes)), ctx)


def pb_set_bands(ctx: Context, bands: int) -> None:
    """Bands of the symmetric products: 0 automatic (the default), 1 none,
    n >= 2 at least n."""
    _check(lib().pb_set_bands(ctx.handle, int(bands)), ctx)


def pb_sym_band_plan(n: int, tile: int, ctas: int, elem: int, limit: int = 0, bands: int = 0):
    """(row-tile cuts, scratch bytes) of a symmetric product's band plan,
    computed on the host without a context (see include/pb.h)."""
    tiles = -(-int(n) // int(tile))
    buf = (_I64 * (tiles + 2))()
    nc, nb = ctypes.c_int(), ctypes.c_int64()
    _check(lib().pb_sym_band_plan(int(n), int(tile), int(ctas), int(elem), int(limit), int(bands), buf,
                                  tiles + 2, ctypes.byref(nc), ctypes.byref(nb)))
    return [buf[k] for k in range(nc.value)], nb.value


def pb_scratch_plan(ctx: Context, prec="fp32pair"):
    """(bands, scratch bytes) of the symmetric product of this precision at the
    current kernel choice and bound; (0, 0) when that product is not symmetric."""
    b, n = ctypes.c_int(), ctypes.c_int64()
    _check(lib().pb_scratch_plan(ctx.handle, PRECISIONS[prec], ctypes.byref(b), ctypes.byref(n)), ctx)
    return b.value, n.value


def pb_matvec_autotune(ctx: Context, reps: int = 3) -> dict:
    v, c, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().pb_matvec_autotune(ctx.handle, int(reps), ctypes.byref(v), ctypes.byref(c), ctypes.byref(ms)), ctx)
    return {"variant": v.value, "ctas_per_sm": c.value, "ms": ms.value}


def pb_batch_solve(ctxs, charge_sets, restart: int = 10, tol: float = 1e-4, maxit: int = 1000,
                   use_graph=True, raise_on_noconv: bool = True):
    """Solve every (surface, charge set) pair in lockstep.  ``ctxs``: list of
    contexts; ``charge_sets[s]``: array (R_s, Nc_s, 4) or (Nc_s, 4) of host
    charges.  Returns (energies as a list of R_s-length lists, info dict)."""
    n = len(ctxs)
    keep = []
    handles = (ctypes.c_void_p * n)(*[c.handle for c in ctxs])
    ptrs = (ctypes.c_void_p * n)()
    ncs = (ctypes.c_int64 * n)()
    nr = (ctypes.c_int * n)()
    for i, q in enumerate(charge_sets):
        a = np.ascontiguousarray(np.asarray(q, dtype=np.float64))
        if a.ndim == 2:
            a = a[None]
        keep.append(a)
        nr[i] = a.shape[0]
        ncs[i] = a.shape[1]
        ptrs[i] = a.ctypes.data if a.size else None
    total = sum(nr)
    en = (ctypes.c_double * total)()
    o = _Opts(int(restart), float(tol), int(maxit), PB_FP32PAIR, 0, PB_FP64)
    info = _BatchInfo()
    mode = 2 if use_graph == "timed" else (1 if use_graph else 0)
    st = lib().pb_batch_solve(handles, n, ptrs, ncs, nr, ctypes.byref(o), mode, en, ctypes.byref(info))
    if st != PB_OK and not (st == PB_ERR_NOCONV and not raise_on_noconv):
        _check(st, ctxs[0])
    out, k = [], 0
    for i in range(n):
        out.append([en[k + r] for r in range(nr[i])])
        k += nr[i]
    d = {f: getattr(info, f) for f, _ in _BatchInfo._fields_}
    d["status"] = st
    return out, d


def pb_batch_set_streams(n: int) -> None:
    """Engines (streams) of pb_batch_solve: 2 (default) or 1."""
    _check(lib().pb_batch_set_streams(int(n)))


def pb_batch_set_tuning(autotune: bool) -> None:
    """Autotune the batched product per (width, size class) (default), or use the built-in shapes."""
    _check(lib().pb_batch_set_tuning(1 if autotune else 0))


def pb_batch_force_shape(rhs_width: int, targets_per_thread: int = 0, row_sums: int = 0,
                         ctas_per_sm: int = 0) -> None:
    """Force the batched product's shape for one width (targets_per_thread = 0 clears it)."""
    _check(lib().pb_batch_force_shape(int(rhs_width), int(targets_per_thread), int(row_sums), int(ctas_per_sm)))


def pb_batch_clear_tuning() -> None:
    _check(lib().pb_batch_clear_tuning())


def pb_batch_shapes(rhs_width: int) -> list:
    """[(targets_per_thread, row_sums)] instantiated for a width, the default first."""
    t = (ctypes.c_int * 16)()
    r = (ctypes.c_int * 16)()
    n = lib().pb_batch_shapes(int(rhs_width), t, r, 16)
    return [(t[i], r[i]) for i in range(min(n, 16))]


class Server:
    """A solve server with continuous batching (pb_server_* of include/pb.h)."""

    def __init__(self, max_active: int = 8, hbm_budget_bytes: int = 8 << 30, restart: int = 10,
                 tol: float = 1e-4, maxit: int = 1000, split_n: int = 0):
        """split_n: requests with N >= split_n take the large lane (0: the
        library's default, 16,384; negative: one lane for all requests)."""
        o = _ServerOpts(int(max_active), int(hbm_budget_bytes), int(restart), float(tol), int(maxit), int(split_n))
        h = ctypes.c_void_p()
        _check(lib().pb_server_create(ctypes.byref(o), ctypes.byref(h)))
        self.handle = h.value

    def submit(self, centroids, normals, areas, charges, eps1: float, eps2: float, kappa: float) -> int:
        c = np.ascontiguousarray(centroids, dtype=np.float64)
        nr = np.ascontiguousarray(normals, dtype=np.float64)
        a = np.ascontiguousarray(areas, dtype=np.float64)
        q = np.ascontiguousarray(charges, dtype=np.float64).reshape(-1, 4)
        rid = ctypes.c_uint64()
        _check(lib().pb_server_submit(self.handle, c.ctypes.data, nr.ctypes.data, a.ctypes.data, a.size,
                                      q.ctypes.data if q.size else None, q.shape[0], float(eps1), float(eps2),
                                      float(kappa), ctypes.byref(rid)))
        return rid.value

    def poll(self, max_results: int = 256) -> list:
        buf = (_ServerResult * max_results)()
        n = lib().pb_server_poll(self.handle, buf, max_results)
        return [{f: getattr(buf[i], f) for f, _ in _ServerResult._fields_} for i in range(n)]

    def wait(self, n_results: int, timeout_s: float) -> None:
        _check(lib().pb_server_wait(self.handle, int(n_results), float(timeout_s)))

    def stats(self) -> dict:
        st = _ServerStats()
        _check(lib().pb_server_get_stats(self.handle, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in _ServerStats._fields_}

    def close(self) -> None:
        if self.handle:
            h, self.handle = self.handle, None
            lib().pb_server_destroy(h)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pb_destroy(ctx: Context) -> None:
    if ctx is not None and ctx.handle:
        h, ctx.handle = ctx.handle, None
        lib().pb_destroy(h)
