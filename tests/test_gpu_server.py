"""The solve server with continuous batching: each result is the same alone
and in the mix (within the FP32-pair tolerance), admission respects the slot
limit and the memory budget, oversized requests are rejected, and waits are
bounded."""
import threading
import time

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


def _requests():
    out = []
    for k, (lvl, rad, nq, kap) in enumerate([(3, 5.0, 4, 0.1257), (4, 9.0, 12, 0.0), (2, 3.0, 2, 0.1257),
                                            (4, 12.0, 9, 0.1257), (3, 6.0, 5, 0.0), (5, 15.0, 20, 0.1257)]):
        out.append(pi.kirkwood_sphere_multi(level=lvl, radius=rad, n_charges=nq, seed=60 + k, kappa=kap))
    out.append(pi.protein_like(n_atoms=14, seed=8, target_triangles=None, spacing=1.3))
    return out


def _submit(sv, p):
    s = p.surface
    return sv.submit(s.centroids, s.normals, s.areas, p.charges, p.eps1, p.eps2, p.kappa)


def _collect(sv, n, timeout=120.0):
    sv.wait(n, timeout)
    res = sv.poll(4096)
    assert len(res) == n
    return {r["id"]: r for r in res}


def test_each_result_is_the_same_alone_and_in_the_mix():
    pb = _pb()
    reqs = _requests()
    alone = []
    with pb.Server(max_active=1, tol=1e-7) as sv:
        for p in reqs:
            rid = _submit(sv, p)
            r = _collect(sv, 1)[rid]
            assert r["status"] == pb.PB_OK
            alone.append(r["energy_kcal"])
    with pb.Server(max_active=8, tol=1e-7) as sv:
        ids = []
        # a first wave, then the rest staggered while the first wave runs
        for p in reqs[:3]:
            ids.append(_submit(sv, p))
        for p in reqs[3:]:
            time.sleep(0.01)
            ids.append(_submit(sv, p))
        got = _collect(sv, len(reqs))
        st = sv.stats()
    assert st["max_active_seen"] >= 2          # requests really overlapped
    for rid, e_alone, p in zip(ids, alone, reqs):
        r = got[rid]
        assert r["status"] == pb.PB_OK
        assert r["energy_kcal"] == pytest.approx(e_alone, rel=1e-6)
        assert 0.0 <= r["queue_ms"] <= r["latency_ms"]
    # the mixed results meet the 1e-5 bound against the FP64 oracle (the
    # requests small enough for a quick oracle solve: 320 to ~2,000 triangles)
    checked = 0
    for rid, p in zip(ids, reqs):
        if p.n > 2500:
            continue
        ref = oracle.solve(p.surface, p.charges, p.eps1, p.eps2, p.kappa, tol=1e-11, maxit=2000)["energy"]
        assert got[rid]["energy_kcal"] == pytest.approx(ref, rel=1e-5), p.name
        checked += 1
    assert checked >= 3
    # and the same as the one-at-a-time library solve
    for e_alone, p in zip(alone[:3], reqs[:3]):
        s = p.surface
        with pb.pb_create(s.centroids, s.normals, s.areas, p.charges, p.eps1, p.eps2, p.kappa) as ctx:
            e = pb.pb_solve(ctx, tol=1e-7, prec="fp32pair").energy_kcal
        assert e == pytest.approx(e_alone, rel=2e-6)


def test_submissions_from_several_threads():
    pb = _pb()
    reqs = _requests()[:4]
    with pb.Server(max_active=4, tol=1e-6) as sv:
        ids = []
        lock = threading.Lock()

        def worker(p):
            rid = _submit(sv, p)
            with lock:
                ids.append(rid)
        th = [threading.Thread(target=worker, args=(p,)) for p in reqs]
        for t in th:
            t.start()
        for t in th:
            t.join()
        got = _collect(sv, len(reqs))
    assert sorted(got) == sorted(ids)
    assert all(r["status"] == pb.PB_OK for r in got.values())


def test_admission_budget_and_rejection():
    pb = _pb()
    small = pi.kirkwood_sphere_multi(level=3, radius=5.0, n_charges=3, seed=70)
    big = pi.kirkwood_sphere_multi(level=6, radius=12.0, n_charges=3, seed=71)
    # each small request needs about 4.7 MB (4 MiB of it context scratch), the
    # big one about 34 MB: the budget holds two small ones and never the big one
    with pb.Server(max_active=8, hbm_budget_bytes=12 << 20, tol=1e-6) as sv:
        ids = [_submit(sv, small) for _ in range(4)]
        big_id = _submit(sv, big)
        got = _collect(sv, 5)
        st = sv.stats()
    assert got[big_id]["status"] == pb.PB_ERR_ADMIT
    assert all(got[i]["status"] == pb.PB_OK for i in ids)
    assert st["rejected"] == 1 and st["max_active_seen"] <= 2
    e = [got[i]["energy_kcal"] for i in ids]
    assert max(e) - min(e) <= 1e-9 * abs(e[0])


def test_wait_is_bounded():
    pb = _pb()
    with pb.Server(max_active=2) as sv:
        t = time.time()
        with pytest.raises(pb.PBError) as ei:
            sv.wait(1, 0.2)
        assert ei.value.status == pb.PB_ERR_TIMEOUT
        assert time.time() - t < 5.0


def test_two_lanes_and_one_lane_give_the_same_results():
    """The default server splits requests into a small and a large lane by N
    (two workers and streams; the large lane's products run with one CTA per
    SM fewer while small requests run).  The same requests through a
    one-lane server (split_n < 0) give the same energies (1e-6), and so does
    a split that puts every request in the large lane."""
    pb = _pb()
    reqs = _requests()
    out = {}
    for split in (0, -1, 1):
        with pb.Server(max_active=8, tol=1e-7, split_n=split) as sv:
            ids = [_submit(sv, p) for p in reqs]
            got = _collect(sv, len(reqs))
        assert all(got[i]["status"] == pb.PB_OK for i in ids)
        out[split] = [got[i]["energy_kcal"] for i in ids]
    for a, b, c in zip(out[0], out[-1], out[1]):
        assert a == pytest.approx(b, rel=1e-6)
        assert a == pytest.approx(c, rel=1e-6)
