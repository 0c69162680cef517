"""Row-block products and the row-sharded solve on the GPU.

* pb_matvec_rows: row blocks (first, last, single rows, ragged) of the
  FP32-pair and FP64 products against the oracle's rows, per row block.
* The sharded product of W ranks, emulated on one GPU by evaluating every
  rank's rows in turn and unpacking the gathered blocks with the library's
  host unpack: equal to the oracle's full product.
* pb_solve_sharded with one rank, its allgather a device copy and, separately,
  a one-rank NCCL group: the oracle's energy (FP64: 1e-10; FP32 pairs: 1e-5).
Separate ranks on separate GPUs are not run here (one GPU); their host logic
is tested on CPU ranks in test_sharded_host.py.
"""
import os
import socket

import numpy as np
import pytest

import oracle
import pb_inputs as pi
from blockcheck import TOL_FP32PAIR, TOL_FP64, assert_blocks_close, assert_rows_close

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


def _ctx(p, kappa=None):
    s = p.surface
    return _pb().pb_create(s.centroids, s.normals, s.areas, p.charges, p.eps1, p.eps2,
                           p.kappa if kappa is None else kappa, stream=torch.cuda.current_stream())


TOLS = {"fp32pair": TOL_FP32PAIR, "fp64": TOL_FP64}


@pytest.mark.parametrize("prec", ["fp32pair", "fp64"])
@pytest.mark.parametrize("kappa", [0.1257, 0.0])
def test_row_blocks_match_the_oracle_rows(prec, kappa):
    pb = _pb()
    p = pi.kirkwood_sphere_multi(level=5, radius=12.0, n_charges=4, seed=31)
    n = p.n
    rng = np.random.Generator(np.random.PCG64(32))
    u = rng.normal(size=2 * n)
    ud = torch.tensor(u, device="cuda")
    blocks = [(0, 1), (0, n), (n - 1, 1), (37, 777), (4096, 5000), (n - 4099, 4099)]
    with _ctx(p, kappa) as ctx:
        for r0, nr in blocks:
            y = torch.full((2 * nr,), float("nan"), dtype=torch.float64, device="cuda")
            pb.pb_matvec_rows(ctx, ud, y, r0, nr, prec)
            torch.cuda.synchronize()
            yh = y.cpu().numpy()
            rows = np.arange(r0, r0 + nr)
            sample = rows if nr <= 800 else rows[np.linspace(0, nr - 1, 400).astype(int)]
            ref1, ref2 = oracle.matvec_rows(p.surface, p.eps2 / p.eps1, kappa, u, sample)
            assert_rows_close(yh[sample - r0], yh[nr + sample - r0], ref1, ref2, TOLS[prec], f"{prec} {r0}+{nr}")


def test_row_blocks_reject_bad_ranges():
    pb = _pb()
    p = pi.kirkwood_sphere_multi(level=2, radius=4.0, n_charges=2, seed=33)
    with _ctx(p) as ctx:
        u = torch.zeros(2 * p.n, dtype=torch.float64, device="cuda")
        y = torch.zeros(6, dtype=torch.float64, device="cuda")
        for r0, nr in ((-1, 3), (p.n - 2, 3)):
            with pytest.raises(pb.PBError) as ei:
                pb.pb_matvec_rows(ctx, u, y, r0, nr, "fp32pair")
            assert ei.value.status == pb.PB_ERR_ARG
        with pytest.raises(pb.PBError):
            pb.pb_matvec_rows(ctx, u, y, 0, 3, "float2")


@pytest.mark.parametrize("world", [2, 3, 5])
@pytest.mark.parametrize("prec", ["fp32pair", "fp64"])
def test_emulated_ranks_give_the_full_product(world, prec):
    """Every rank's rows evaluated in turn on one GPU, packed as the
    allgather delivers them and unpacked: the full product of Eqs. (12)-(13)."""
    pb = _pb()
    p = pi.protein_like(n_atoms=20, seed=5, target_triangles=None, spacing=1.2)
    n = p.n
    rng = np.random.Generator(np.random.PCG64(34))
    u = rng.normal(size=2 * n)
    ud = torch.tensor(u, device="cuda")
    gathered = []
    with _ctx(p) as ctx:
        for r in range(world):
            r0, nr, per = pb.pb_shard_rows(n, world, r)
            blk = np.zeros(2 * per)
            if nr:
                y = torch.empty(2 * nr, dtype=torch.float64, device="cuda")
                pb.pb_matvec_rows(ctx, ud, y, r0, nr, prec)
                torch.cuda.synchronize()
                yh = y.cpu().numpy()
                blk[:nr], blk[per:per + nr] = yh[:nr], yh[nr:]
            gathered.append(blk)
    y = pb.pb_shard_unpack_host(np.concatenate(gathered), n, world)
    ref = oracle.matvec(p.surface, p.eps2 / p.eps1, p.kappa, u)
    assert_blocks_close(y, ref, TOLS[prec])


def _copy_gather(send, recv, count):
    recv.copy_(send)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32pair", 1e-5)])
def test_one_rank_sharded_solve_matches_the_oracle(prec, tol):
    pb = _pb()
    p = pi.kirkwood_sphere_multi(level=4, radius=8.0, n_charges=6, seed=35)
    ref = oracle.solve(p.surface, p.charges, p.eps1, p.eps2, p.kappa, tol=1e-12, maxit=2000)
    stol = 1e-12 if prec == "fp64" else 1e-7
    with _ctx(p) as ctx:
        x = torch.empty(2 * p.n, dtype=torch.float64, device="cuda")
        info = pb.pb_solve_sharded(ctx, tol=stol, maxit=2000, prec=prec, x_out=x, allgather=_copy_gather)
        plain = pb.pb_solve(ctx, tol=stol, maxit=2000, prec=prec)
    assert info.status == pb.PB_OK and info.matvecs > 0
    assert info.energy_kcal == pytest.approx(ref["energy"], rel=tol)
    assert info.energy_kcal == pytest.approx(plain.energy_kcal, rel=max(tol, 2e-6))
    if prec == "fp64":
        assert np.linalg.norm(x.cpu().numpy() - ref["u"]) <= 1e-9 * np.linalg.norm(ref["u"])


def test_one_rank_sharded_solve_over_nccl():
    """The same solve with the default torch.distributed allgather on a
    one-rank NCCL group: the same energy as with the copy callback, bit for bit."""
    import torch.distributed as dist
    pb = _pb()
    p = pi.kirkwood_sphere_multi(level=4, radius=8.0, n_charges=6, seed=36)
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        with _ctx(p) as ctx:
            a = pb.pb_solve_sharded(ctx, tol=1e-8, prec="fp32pair")
            b = pb.pb_solve_sharded(ctx, tol=1e-8, prec="fp32pair", allgather=_copy_gather)
            c = pb.pb_solve_sharded(ctx, tol=1e-8, prec="fp32pair", refine=1, refine_prec="fp64")
    finally:
        dist.destroy_process_group()
    assert a.energy_kcal == b.energy_kcal and a.matvecs == b.matvecs
    assert c.refine_steps == 1 and c.rel_resid_fp64 <= 1e-8
    ref = oracle.solve(p.surface, p.charges, p.eps1, p.eps2, p.kappa, tol=1e-12, maxit=2000)
    assert a.energy_kcal == pytest.approx(ref["energy"], rel=1e-5)


def test_sharded_solve_rejects_float_float():
    pb = _pb()
    p = pi.kirkwood_sphere_multi(level=2, radius=4.0, n_charges=2, seed=37)
    with _ctx(p) as ctx:
        with pytest.raises(pb.PBError):
            pb.pb_solve_sharded(ctx, prec="float2", allgather=_copy_gather)
