"""Host logic of the row-sharded solve, on CPU ranks over gloo.

The GPU path (pb_solve_sharded) evaluates each rank's rows of A u on its own
GPU, allgathers the ranks' row blocks and unpacks them into the full 2N
vector, with GMRES replicated on every rank.  Here the same layout runs on CPU
ranks: the library's partition (pb_shard_rows) and unpacking
(pb_shard_unpack_host), the rows of each rank from the oracle, a gloo
allgather, and the oracle's GMRES on the gathered product.  The sharded
product must equal the oracle's full product bit for bit (each row is the
same sum in the same order), every rank must end with the same solution, and
the energy must equal the oracle's single-process solve."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pb():
    import importlib
    importlib.import_module("paper_1301_5885_gb300.build").build()
    import paper_1301_5885_gb300 as pb
    return pb


@pytest.mark.parametrize("n", [1, 2, 7, 1000, 1001, 300176])
@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_partition_covers_every_row_once_in_rank_order(pb, n, world):
    rows = [pb.pb_shard_rows(n, world, r) for r in range(world)]
    per = rows[0][2]
    assert per == -(-n // world)
    nxt = 0
    for r0, nr, p in rows:
        assert p == per and 0 <= nr <= per
        assert r0 == min(nxt, n)
        nxt = r0 + nr
    assert nxt == n
    assert sum(nr for _, nr, _ in rows) == n


def test_unpack_places_each_ranks_rows():
    import paper_1301_5885_gb300 as pb
    n, world = 11, 3
    per = -(-n // world)
    g = np.zeros(2 * per * world)
    for r in range(world):
        r0, nr, _ = pb.pb_shard_rows(n, world, r)
        g[2 * per * r: 2 * per * r + nr] = np.arange(r0, r0 + nr)              # phi rows
        g[2 * per * r + per: 2 * per * r + per + nr] = 100 + np.arange(r0, r0 + nr)   # psi rows
    y = pb.pb_shard_unpack_host(g, n, world)
    assert np.array_equal(y[:n], np.arange(n)) and np.array_equal(y[n:], 100 + np.arange(n))


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist

    import oracle
    import paper_1301_5885_gb300 as pb
    import pb_inputs as pi
    oracle.set_num_threads(2)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = pi.kirkwood_sphere_multi(level=3, radius=6.0, n_charges=5, seed=21)
        n, eps = p.n, p.eps2 / p.eps1
        r0, nr, per = pb.pb_shard_rows(n, world, rank)
        rows = np.arange(r0, r0 + nr)
        products = [0]

        def apply_A(u):
            send = np.zeros(2 * per)
            if nr:
                send[:nr], send[per:per + nr] = oracle.matvec_rows(p.surface, eps, p.kappa, u, rows)
            parts = [torch.zeros(2 * per, dtype=torch.float64) for _ in range(world)]
            dist.all_gather(parts, torch.from_numpy(send))
            products[0] += 1
            return pb.pb_shard_unpack_host(torch.cat(parts).numpy(), n, world)

        rng = np.random.Generator(np.random.PCG64(3))
        u = rng.normal(size=2 * n)
        y_sharded = apply_A(u)
        b = oracle.source(p.surface, p.charges, p.eps1)
        x, iters, hist, conv = oracle.gmres(apply_A, b, restart=10, tol=1e-12, maxit=500)
        energy = oracle.reaction_energy(p.surface, p.charges, eps, p.kappa, x)
        out.put((rank, y_sharded, x, energy, conv, products[0]))
    finally:
        dist.destroy_process_group()


def test_two_cpu_ranks_solve_to_the_oracle_energy(pb):
    import torch.multiprocessing as mp

    import oracle
    import pb_inputs as pi
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = dict((r, rest) for r, *rest in (q.get(timeout=300) for _ in procs))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = pi.kirkwood_sphere_multi(level=3, radius=6.0, n_charges=5, seed=21)
    eps = p.eps2 / p.eps1
    rng = np.random.Generator(np.random.PCG64(3))
    u = rng.normal(size=2 * p.n)
    full = oracle.matvec(p.surface, eps, p.kappa, u)
    ref = oracle.solve(p.surface, p.charges, p.eps1, p.eps2, p.kappa, tol=1e-12, maxit=500)
    (y0, x0, e0, c0, n0), (y1, x1, e1, c1, n1) = got[0], got[1]
    assert np.array_equal(y0, full) and np.array_equal(y1, full)      # the sharded product, bit for bit
    assert c0 and c1 and n0 == n1
    assert np.array_equal(x0, x1) and e0 == e1                         # replicated GMRES agrees on every rank
    assert e0 == pytest.approx(ref["energy"], rel=1e-10)
    assert np.linalg.norm(x0 - ref["u"]) <= 1e-9 * np.linalg.norm(ref["u"])
