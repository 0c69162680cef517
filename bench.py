#!/usr/bin/env python
"""Benchmark of the direct-sum boundary-integral PB solve on one or more GPUs.

One step = the whole hot path for one molecule: pb_create from device-resident
geometry (validation, centring, FP32/FP64 packing, orientation check), the
source term, restarted GMRES whose products with A are the FP32-pair
direct-sum matvec (FP64 accumulation, FP64 Krylov arithmetic), and the FP64
solvation-energy reduction; then the context is freed.

The default workload is the largest single-GPU configuration: the synthetic
protein-like solute of about 300,000 triangles (2,000 atoms and charges),
solved to a GMRES tolerance of 1e-6, the loosest that meets a relative
solvation-energy error of 1e-5 on that surface (at 1e-4 it is about 1e-4).

The headline value is the matvec pair rate of the whole step: (products with A
the device evaluated) x N(N-1) pairs / step time, in Gpairs/s.  The line also
reports solves/s, p50/p99 step latency, the relative energy error against the
stored FP64 oracle solution, the roofline fraction of the matvec kernel, an
end-to-end figure through the C ABI from pinned host buffers, the oracle
timed on the host cores, and a secondary line on the 81,920-triangle Kirkwood
sphere.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 launch with torchrun; every rank solves its own copy (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "matvec Gpairs/s; PB solves/s + p50/p99 latency at ≤1e-5 rel. energy error"
UNIT = "Gpairs/s"

# Roofline of the FP32-pair matvec (ALU bound, no tensor-core contraction).
# The FP32 pipe retires 128 lanes per clock per SM (an f32x2 instruction
# counts as two lanes' work), so for a kernel doing k FP32 add/mul/fma
# operations per ordered pair, peak pairs/s = SMs x 128 x f_max / k.  MUFU
# (16 per clock per SM, 2-3 per pair) and the ALU pipe are not binding.
# k per variant (kappa > 0, kappa = 0), from the operation counts in the
# kernels' comments; the symmetric kernels evaluate an unordered pair once for
# both rows, so k is half their per-pair count.
SMS = 152
SM_MAX_MHZ = 2070.0
# The work count of one ordered pair of the product evaluated on its own
# (kappa > 0): 45 FP32 operations evaluating K1..K4 for that pair alone.  The
# symmetric kernels do less per ordered pair, because one evaluation of an
# unordered pair serves both rows; their fraction on this basis can exceed 1.
ORDERED_PAIR_OPS = 45
MATVEC_KERNELS = {
    1: ("matvec_f32_kernel", 41, 41),
    2: ("matvec_f32x2_kernel<2>", 39, 18),
    3: ("matvec_f32x2_kernel<4>", 39, 18),
    4: ("matvec_f32x2_kernel<3>", 39, 18),
    5: ("matvec_sym_kernel<2> + finishing kernels", 23, 10),
    6: ("matvec_sym_kernel<4> + finishing kernels", 23, 10),
}


MATVEC64_KERNELS = {1: "matvec_f64_kernel", 2: "matvec_sym64_kernel<1> + matvec_sym_finalize<128, double>",
                    3: "matvec_sym64_kernel<2> + matvec_sym_finalize<256, double>"}


def matvec_peak_gpairs(ops_per_pair):
    return SMS * 128 * SM_MAX_MHZ * 1e6 / ops_per_pair / 1e9


# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the kernel on
# the 81,920-triangle sphere, from an ncu capture of the kernel as it is now
# (profiles/); a kernel that changed since its capture has no entry.
# DRAM bytes of one product by (kernel, workload, bands), from ncu captures
# without the cache flush (as in a solve); a configuration not captured
# reports no traffic
MATVEC_TRAFFIC_BYTES = {
    # profiles/matvec_sym_kernel_protein300k_traffic.md: one pass, 25 bands,
    # and the default 79 bands (MB to 0.1 and 0.01)
    ("matvec_sym_kernel<4> + finishing kernels", "protein300k", 1): (30.4 + 660.7 + 716.9 + 64.9) * 1e6,
    ("matvec_sym_kernel<4> + finishing kernels", "protein300k", 25): (13.54 + 453.29 + 1.74 + 78.41) * 1e6,
    ("matvec_sym_kernel<4> + finishing kernels", "protein300k", 79): (6.64 + 13.33 + 0.08 + 6.73) * 1e6,
}

WORKLOADS = {
    "sphere2": "Kirkwood sphere R=20 A, icosphere level 6 (81,920 triangles), 20 charges in 0.8R, "
               "eps 1/80, kappa 0.1257",
    "sphere2_salt_free": "the sphere2 surface and charges with kappa = 0 (salt-free; the kappa = 0 kernels)",
    "sphere1": "Born sphere R=2 A, icosphere level 4 (5,120 triangles), one central charge, eps 1/80, kappa 0.1257",
    "protein300k": "protein-like 2,000-atom chain, probe-inflated Gaussian isosurface (~300k triangles)",
}

DEFAULT_WORKLOAD = "protein300k"
SECONDARY_WORKLOAD = "sphere2"


def default_tol(mode: str, workload: str) -> float:
    """The loosest GMRES tolerance meeting a 1e-5 relative energy error: the
    protein-like surfaces need 1e-6 (measured at 300k triangles: 1.2e-4 error
    at 1e-4, 1.6e-5 at 1e-5, 8.6e-7 at 1e-6), the spheres meet it at 1e-4."""
    if mode in ("batch", "serve", "frames") or workload.startswith("protein"):
        return 1e-6
    return 1e-4


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--prec", choices=["fp32pair", "fp64", "float2"], default="fp32pair")
    ap.add_argument("--tol", type=float, default=None,
                    help="GMRES relative-residual tolerance (default: 1e-6 for the protein-like workloads, batch "
                         "and serve, where the solute surfaces need it for a 1e-5 energy error; 1e-4 for the "
                         "spheres)")
    ap.add_argument("--restart", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="oracle sample budget for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the 81,920-triangle sphere line")
    ap.add_argument("--mode", choices=["solve", "matvec", "batch", "serve", "frames", "sharded"], default="solve",
                    help="solve: one molecule per step (default); matvec: one FP32-pair product per step; "
                         "batch: 64 solutes x 8 charge sets per step; serve: Poisson request stream through "
                         "the solve server; frames: warm-started trajectory frames; sharded: one solve "
                         "row-sharded over the job's GPUs (strong scaling, launch with torchrun for N > 1)")
    ap.add_argument("--variant", type=int, default=0,
                    help="matvec mode: FP32-pair kernel variant (0: the library's default for N)")
    ap.add_argument("--scratch-mb", type=float, default=0.0,
                    help="solve/matvec modes: bound on the symmetric product's scratch in MiB "
                         "(0: the library's default bound, 1 GiB)")
    ap.add_argument("--bands", type=int, default=-1,
                    help="solve/matvec modes: bands of the symmetric product (-1: the library's default, "
                         "automatic; 1: one pass; n >= 2: at least n)")
    ap.add_argument("--n-solutes", type=int, default=64, help="batch mode: solutes per batch")
    ap.add_argument("--batch-streams", type=int, default=2, choices=[1, 2],
                    help="batch mode: engines (streams) the batch is split over")
    ap.add_argument("--frames", type=int, default=20, help="frames mode: trajectory length")
    ap.add_argument("--batch-shape", default=None,
                    help="batch mode: force the product shape T,row_sums,ctas_per_sm for 8 charge sets instead of "
                         "autotuning (for profiling one shape)")
    ap.add_argument("--requests", type=int, default=200, help="serve mode: requests in the stream")
    ap.add_argument("--pool", type=int, default=64, help="serve mode: distinct solutes the requests draw from")
    ap.add_argument("--gen-workers", type=int, default=0, help="processes generating solute meshes (0: auto)")
    return ap.parse_args()


def golden_n(name):
    path = os.path.join(ROOT, "tests", "golden", "oracle_energies.json")
    if not os.path.exists(path):
        return None
    return json.load(open(path)).get(name, {}).get("n")


def golden_energy(name, prob=None):
    """The stored FP64 oracle energy of a workload (tests/golden), or None when
    there is none or when ``prob``'s mesh is not the one it was computed on
    (triangle count, and total area to 1e-9 where the entry records it)."""
    path = os.path.join(ROOT, "tests", "golden", "oracle_energies.json")
    if not os.path.exists(path):
        return None
    g = json.load(open(path)).get(name)
    if not g:
        return None
    if prob is not None:
        if g.get("n") != prob.n:
            return None
        area = g.get("mesh", {}).get("area_sum")
        if area is not None:
            import numpy as np
            if abs(float(np.sum(prob.surface.areas)) - area) > 1e-9 * abs(area):
                return None
    return g.get("energy_kcal")


# --- clocks --------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampling every 200 ms while the timed region runs."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(", ") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        if self.uuid:
            mine = [r for r in rows if r and self.uuid in r[0]]
            rows = mine or rows
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --- the reference arm: the FP64 oracle on the host cores -----------------------
def oracle_rate(prob, seconds: float, seed: int = 0):
    """Time the oracle's direct-sum rows (Eqs. (12)-(13)) on a row sample sized to
    about ``seconds`` of host work.  Returns (Gpairs/s, rows, elapsed, threads)."""
    import numpy as np
    import oracle
    s = prob.surface
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.normal(size=2 * prob.n)
    eps = prob.eps2 / prob.eps1
    probe = min(prob.n, 512)   # enough rows to occupy every host thread
    t = time.perf_counter()
    oracle.matvec_rows(s, eps, prob.kappa, u, rng.choice(prob.n, probe, replace=False))
    dt = max(time.perf_counter() - t, 1e-6)
    rows = int(max(1, min(prob.n, probe * seconds / dt)))
    idx = rng.choice(prob.n, rows, replace=False)
    t = time.perf_counter()
    oracle.matvec_rows(s, eps, prob.kappa, u, idx)
    el = time.perf_counter() - t
    return rows * (prob.n - 1) / el / 1e9, rows, el, oracle.num_threads()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import pb_inputs
    prob = pb_inputs.by_name(args.workload)
    budget = max(1.0, min(8.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_rate(prob, budget * 0.25)
    rates, times, rows_total = [], [], 0
    for k in range(args.steps):
        r, rows, el, threads = oracle_rate(prob, budget, seed=k + 1)
        rates.append(r)
        times.append(el)
        rows_total += rows
    total_pairs = rows_total * (prob.n - 1)
    value = total_pairs / sum(times) / 1e9
    sample = (f"{rows_total // max(1, args.steps)} sampled rows (both row blocks) of the N={prob.n} direct-sum "
              f"matvec per step, FP64 oracle, {threads} OpenMP threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(config_dict(args, prob), precision="fp64 (the oracle)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def config_dict(args, prob):
    d = {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "n_triangles": prob.n,
         "n_charges": prob.nc, "precision": args.prec, "gmres_restart": args.restart, "gmres_tol": args.tol,
         "l2": "flushed between steps (256 MiB write)"}
    if getattr(args, "scratch_mb", 0):
        d["scratch_bound_mib"] = args.scratch_mb
    if getattr(args, "bands", -1) >= 0:
        d["bands_requested"] = args.bands
    return d


def reduce_over_ranks(total_ms: float, pairs: float, solves: float, device, dist=None):
    """Whole-job totals: the slowest rank's time (max) and the units of all ranks
    (sum).  ``dist`` is torch.distributed (or None for one process)."""
    import torch
    t = torch.tensor([float(total_ms), float(pairs), float(solves)], dtype=torch.float64, device=device)
    if dist is None:
        return t[0].item(), t[1].item(), t[2].item()
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return mx[0].item(), sm[1].item(), sm[2].item()


# --- our arm --------------------------------------------------------------------
class SolveLeg:
    """Timed whole solves of one workload: pb_create from the given (device or
    pinned host) inputs, source, GMRES with FP32-pair (or FP64) products, FP64
    energy, pb_destroy; the library's CUDA events around each product."""

    def __init__(self, pb, prob, args, tol, stream):
        self.pb, self.prob, self.args, self.tol, self.stream = pb, prob, args, tol, stream
        self.variant_seen, self.variant64_seen = [], []
        self.bands_seen = (0, 0)

    def step(self, c, nr, a, q, profile=False):
        pb, prob, args = self.pb, self.prob, self.args
        ctx = pb.pb_create(c, nr, a, q, prob.eps1, prob.eps2, prob.kappa, stream=self.stream)
        try:
            if args.scratch_mb:
                pb.pb_set_scratch_limit(ctx, int(args.scratch_mb * 2**20))
            if args.bands >= 0:
                pb.pb_set_bands(ctx, args.bands)
            self.variant_seen.append(pb.pb_matvec_get_config(ctx)["variant"])
            self.bands_seen = pb.pb_scratch_plan(ctx, args.prec)
            if args.prec == "fp64" and not self.variant64_seen:
                self.variant64_seen.append(pb.pb_matvec_configure_fp64(ctx, 0))   # the default, as created
            if profile:
                pb.pb_profile_enable(ctx, True)
            info = pb.pb_solve(ctx, restart=args.restart, tol=self.tol, maxit=3000, prec=args.prec)
            prof = pb.pb_profile_read(ctx) if profile else None
        finally:
            pb.pb_destroy(ctx)
        return info, prof

    def timed(self, inputs, steps, flush):
        """CUDA-event time of each step on the context's stream, L2 flushed before each."""
        import torch
        evs, infos, profs = [], [], []
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            info, prof = self.step(*inputs, profile=True)
            e1.record(self.stream)
            evs.append((e0, e1))
            infos.append(info)
            profs.append(prof)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs], infos, profs

    def kernel(self):
        """(kernel name, FP32 operations per ordered pair or None) of the product in use."""
        if self.args.prec == "fp32pair":
            kname, ops_k, ops_0 = MATVEC_KERNELS[self.variant_seen[-1]]
            return kname, (ops_0 if self.prob.kappa == 0.0 else ops_k)
        return MATVEC64_KERNELS.get(self.variant64_seen[-1] if self.variant64_seen else 1), None

    def roofline(self, profs, total_ms):
        n = self.prob.n
        mv_ms = sum(p["matvec_ms"] for p in profs)
        mv_n = sum(p["evaluated"] for p in profs)
        avg_ms = mv_ms / max(1, mv_n)
        achieved = n * (n - 1) / (avg_ms * 1e-3) / 1e9
        kname, ops = self.kernel()
        peak = matvec_peak_gpairs(ops) if ops else None
        out = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": peak, "unit": UNIT,
               "frac": achieved / peak if peak else None,
               "traffic": MATVEC_TRAFFIC_BYTES.get((kname, self.args.workload, self.bands_seen[0])),
               "bands": self.bands_seen[0], "scratch_bytes": self.bands_seen[1],
               "peak_basis": (f"FP32 pipe: {SMS} SMs x 128 lanes x {SM_MAX_MHZ:.0f} MHz / {ops} FP32 ops per "
                              "ordered pair, the kernel's own count (derived from unit counts and the maximum "
                              "SM clock; not a measured peak)") if ops else "FP64 pipe",
               "avg_launch_ms": avg_ms, "launches": mv_n, "share_of_step": mv_ms / total_ms}
        if self.args.prec == "fp32pair" and self.prob.kappa > 0.0:
            speak = matvec_peak_gpairs(ORDERED_PAIR_OPS)
            out["ordered_pair_basis"] = {
                "peak": speak, "frac": achieved / speak,
                "basis": f"{ORDERED_PAIR_OPS} FP32 ops per ordered pair (K1..K4 evaluated for every ordered "
                         "pair); the symmetric kernel evaluates each unordered pair once for both rows, so it "
                         "exceeds 1 on this basis"}
        return out


def run_ours(args):
    import numpy as np
    import torch

    import paper_1301_5885_gb300 as pb
    import pb_inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    prob = pb_inputs.by_name(args.workload)
    s = prob.surface
    n = prob.n
    pairs_per_mv = n * (n - 1)
    # inputs resident in HBM before the timed region
    dev_in = tuple(torch.tensor(x, device=dev) for x in (s.centroids, s.normals, s.areas, prob.charges))
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    leg = SolveLeg(pb, prob, args, args.tol, stream)

    for _ in range(args.warmup):
        leg.step(*dev_in)
    torch.cuda.synchronize()

    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = pb.pb_kernel_launches()
    step_ms, infos, profs = leg.timed(dev_in, args.steps, flush)
    if dist:
        dist.barrier()
    launches = pb.pb_kernel_launches() - launches0
    clocks = sampler.stop()
    total_ms = sum(step_ms)
    matvecs = sum(i.matvecs for i in infos)
    total_ms_max, all_pairs, all_solves = reduce_over_ranks(total_ms, matvecs * pairs_per_mv, args.steps, dev, dist)
    value = all_pairs / (total_ms_max * 1e-3) / 1e9

    result = None
    if rank == 0:
        ref_e = golden_energy(args.workload, prob)
        energies = [i.energy_kcal for i in infos]
        rel_err = max(abs(e - ref_e) / abs(ref_e) for e in energies) if ref_e else None
        result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                  "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
                  "scaling": "weak", "vs_baseline": None,
                  "dtype": "f32 pairs, f64 accumulation" if args.prec == "fp32pair" else "f64",
                  "data": "synthetic", "config": config_dict(args, prob),
                  "solves_per_s": all_solves / (total_ms_max * 1e-3),
                  "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                                 "p99": float(np.percentile(step_ms, 99))},
                  "energy_kcal": energies[-1], "oracle_energy_kcal": ref_e, "rel_energy_err": rel_err,
                  "gmres": {"iters": infos[-1].iters, "matvecs": infos[-1].matvecs,
                            "rel_resid": infos[-1].rel_resid},
                  "roofline": leg.roofline(profs, total_ms),
                  "gpu_launches": launches, "clocks": clocks}
    if dist:
        dist.barrier()

    if rank == 0 and not args.no_e2e:
        # end to end through the C ABI from pinned host buffers: H2D of the
        # inputs and D2H of the energy inside every timed step
        host_in = tuple(torch.tensor(x).pin_memory() for x in (s.centroids, s.normals, s.areas, prob.charges))
        leg.step(*host_in)
        torch.cuda.synchronize()
        e2e_steps = min(args.steps, 5)
        t = time.perf_counter()
        mvs = 0
        for _ in range(e2e_steps):
            info, _ = leg.step(*host_in)
            mvs += info.matvecs
        torch.cuda.synchronize()
        el = time.perf_counter() - t
        h2d = sum(x.numel() for x in host_in) * 8
        result["e2e"] = {"value": mvs * pairs_per_mv / el / 1e9, "unit": UNIT, "h2d_bytes_per_step": h2d,
                         "d2h_bytes_per_step": 8, "ms_per_step": 1e3 * el / e2e_steps,
                         "solves_per_s": e2e_steps / el, "steps": e2e_steps}
    if rank == 0 and args.prec == "fp32pair" and not args.no_e2e:
        # the precision pattern, once, outside the timed region: a loose
        # FP32-pair solve plus two refinement steps (r = b - A x with the
        # float-float product, FP64-level; A d = r in FP32 pairs; x += d)
        ref_e = golden_energy(args.workload, prob)
        ctx = pb.pb_create(*dev_in, prob.eps1, prob.eps2, prob.kappa, stream=stream)
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rinfo = pb.pb_solve(ctx, restart=args.restart, tol=1e-4, maxit=3000, prec="fp32pair", refine=2,
                                refine_prec="float2")
            t1 = time.perf_counter()
        finally:
            pb.pb_destroy(ctx)
        result["refinement"] = {
            "refine_steps": rinfo.refine_steps, "rel_resid": rinfo.rel_resid_fp64, "energy_kcal": rinfo.energy_kcal,
            "rel_energy_err": abs(rinfo.energy_kcal - ref_e) / abs(ref_e) if ref_e else None,
            "ms": 1e3 * (t1 - t0), "matvecs": rinfo.matvecs,
            "note": "pb_solve(tol 1e-4, refine=2, refine_prec=float2): FP32-pair GMRES, then 2 steps of "
                    "r = b - A x (float-float residual product), A d = r in FP32 pairs, x += d"}
    if rank == 0 and not args.no_secondary and args.workload != SECONDARY_WORKLOAD:
        # the 81,920-triangle Kirkwood sphere, the headline of earlier lines
        p2 = pb_inputs.by_name(SECONDARY_WORKLOAD)
        s2 = p2.surface
        in2 = tuple(torch.tensor(x, device=dev) for x in (s2.centroids, s2.normals, s2.areas, p2.charges))
        tol2 = default_tol("solve", SECONDARY_WORKLOAD)
        sargs = argparse.Namespace(**vars(args))
        sargs.workload = SECONDARY_WORKLOAD
        leg2 = SolveLeg(pb, p2, sargs, tol2, stream)
        for _ in range(3):
            leg2.step(*in2)
        torch.cuda.synchronize()
        ms2, inf2, prof2 = leg2.timed(in2, 10, flush)
        ref2 = golden_energy(SECONDARY_WORKLOAD, p2)
        t2 = sum(ms2)
        result["secondary"] = {
            "workload": f"{SECONDARY_WORKLOAD}: {WORKLOADS[SECONDARY_WORKLOAD]}", "n_triangles": p2.n,
            "gmres_tol": tol2, "steps": 10,
            "value": sum(i.matvecs for i in inf2) * p2.n * (p2.n - 1) / (t2 * 1e-3) / 1e9, "unit": UNIT,
            "solves_per_s": 10 / (t2 * 1e-3),
            "latency_ms": {"p50": float(np.percentile(ms2, 50)), "p99": float(np.percentile(ms2, 99))},
            "rel_energy_err": max(abs(i.energy_kcal - ref2) / abs(ref2) for i in inf2) if ref2 else None,
            "roofline": leg2.roofline(prof2, t2)}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        rate, rows, el, threads = oracle_rate(prob, args.cpu_seconds)
        # one core, as the paper's T1 column (a short sample of the same rows)
        oracle.set_num_threads(1)
        rate1, rows1, el1, _ = oracle_rate(prob, min(4.0, args.cpu_seconds / 3))
        oracle.set_num_threads(threads)
        result["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                  "sample": f"{rows} sampled rows (both row blocks) of the N={n} direct-sum matvec, "
                                            f"FP64 oracle, {threads} OpenMP threads, {el:.1f} s",
                                  "one_core": {"value": rate1, "unit": UNIT, "sample": f"{rows1} rows, {el1:.1f} s"}}
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# --- batch and serve modes --------------------------------------------------------
def _gen_solute(spec):
    """Build one protein-like solute (top-level so a spawn pool can pickle it)."""
    n_atoms, seed, target = spec
    import pb_inputs
    p = pb_inputs.protein_like(n_atoms=n_atoms, seed=seed, target_triangles=target)
    s = p.surface
    return s.centroids, s.normals, s.areas, p.charges


def make_solutes(specs, workers):
    """Generate meshes in a spawn process pool (started before any GPU call)."""
    if workers <= 1:
        return [_gen_solute(x) for x in specs]
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_gen_solute, specs, chunksize=1)


def batch_specs(n, seed=4):
    import pb_inputs
    return pb_inputs.batch_specs(n, seed)


def serve_specs(n, seed=5):
    import pb_inputs
    return pb_inputs.serve_specs(n, seed)


def _workers(args):
    return args.gen_workers if args.gen_workers > 0 else max(1, min(16, (os.cpu_count() or 2) - 1))


def _clock_and_uuid(torch, dev):
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    return ClockSampler(uuid)


ROW_SUMS = {0: "fp64 registers", 1: "fp64 shared memory", 2: "float-float registers",
            3: "float-float shared memory"}
BATCH_FP32_OPS_PER_EVAL = 36     # K1..K4 of one pair, packed FP32 (kappa > 0; 2 MUFU besides)
BATCH_FP32_OPS_PER_RHS = 4       # the two rows' accumulations per charge set


def run_matvec(args):
    """The product alone: y = A u for a fixed random u, one launch per step,
    timed with CUDA events on the context's stream (median over steps)."""
    import numpy as np
    import torch
    import paper_1301_5885_gb300 as pb
    import pb_inputs
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    prob = pb_inputs.by_name(args.workload)
    s = prob.surface
    stream = torch.cuda.current_stream()
    ctx = pb.pb_create(s.centroids, s.normals, s.areas, prob.charges, prob.eps1, prob.eps2, prob.kappa,
                       stream=stream)
    prec = args.prec
    if prec == "fp64":
        v64 = pb.pb_matvec_configure_fp64(ctx, args.variant)
    elif args.variant:
        pb.pb_matvec_configure(ctx, args.variant, 0)
    if args.scratch_mb:
        pb.pb_set_scratch_limit(ctx, int(args.scratch_mb * 2**20))
    if args.bands >= 0:
        pb.pb_set_bands(ctx, args.bands)
    cfg = pb.pb_matvec_get_config(ctx)
    if prec == "fp64":
        cfg["variant"] = v64
    bands, scratch = pb.pb_scratch_plan(ctx, prec)
    gen = torch.Generator(device=dev).manual_seed(7)
    u = torch.randn(2 * prob.n, dtype=torch.float64, device=dev, generator=gen)
    y = torch.empty_like(u)
    for _ in range(args.warmup):
        pb.pb_matvec(ctx, u, y, prec)
    torch.cuda.synchronize()
    sampler = _clock_and_uuid(torch, dev)
    sampler.start()
    l0 = pb.pb_kernel_launches()
    evs = []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pb.pb_matvec(ctx, u, y, prec)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    launches = pb.pb_kernel_launches() - l0
    clocks = sampler.stop()
    pb.pb_destroy(ctx)
    ms = np.array([a.elapsed_time(b) for a, b in evs])
    pairs = prob.n * (prob.n - 1)
    value = pairs / (np.median(ms) * 1e-3) / 1e9
    if prec == "fp64":
        kname = MATVEC64_KERNELS[cfg["variant"]]
        peak = None
    elif prec == "float2":
        kname, peak = "matvec_ff_kernel", None
    else:
        kname, ops_k, ops_0 = MATVEC_KERNELS[cfg["variant"]]
        ops = ops_0 if prob.kappa == 0.0 else ops_k
        peak = matvec_peak_gpairs(ops)
    line = {"metric": "matvec Gpairs/s", "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(np.median(ms)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "float2": "float-float pairs, f64 accumulation"}.get(
                prec, "f32 pairs, f64 accumulation"), "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload]}", "n_triangles": prob.n,
                       "variant": cfg["variant"], "ctas": cfg["ctas"], "bands": bands, "scratch_bytes": scratch,
                       "l2": "inputs L2-resident by design (the product is FP32-pipe bound)"},
            "roofline": {"kernel": kname, "bound": "alu", "achieved": value, "peak": peak, "unit": UNIT,
                         "frac": value / peak if peak else None,
                         "traffic": MATVEC_TRAFFIC_BYTES.get((kname, args.workload, max(bands, 1))),
                         "peak_basis": (f"FP32 pipe: {SMS} SMs x 128 lanes x {SM_MAX_MHZ:.0f} MHz / {ops} FP32 ops "
                                        "per ordered pair (derived)") if peak else
                                       "FP64 pipe (see the ncu FP64-pipe utilisation)"},
            "ms_min": float(ms.min()), "ms_max": float(ms.max()), "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    import numpy as np
    import pb_inputs
    specs = batch_specs(args.n_solutes)
    sols = make_solutes(specs, _workers(args))
    import torch
    import paper_1301_5885_gb300 as pb
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream()
    variants = [pb_inputs.charge_variants(q, 8, seed=3000 + i) for i, (_, _, _, q) in enumerate(sols)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        dev_in = [tuple(torch.tensor(a, device=dev) for a in (c, n, w, q)) for c, n, w, q in sols]
        ctxs = [pb.pb_create(c, n, w, q, 1.0, 80.0, 0.1257, stream=stream) for c, n, w, q in dev_in]
        ns = [c.n for c in ctxs]
        warm_info = None
        pb.pb_batch_set_streams(args.batch_streams)
        if args.batch_shape:
            t_, r_, c_ = (int(v) for v in args.batch_shape.split(","))
            pb.pb_batch_force_shape(8, t_, r_, c_)
        for _ in range(args.warmup):
            _, wi = pb.pb_batch_solve(ctxs, variants, restart=args.restart, tol=args.tol, use_graph=True,
                                      raise_on_noconv=False)
            warm_info = warm_info or wi       # the first call tunes the product (untimed)
        stream.synchronize()
        sampler = _clock_and_uuid(torch, dev)
        sampler.start()
        l0 = pb.pb_kernel_launches()
        times, infos, energies = [], [], None
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            energies, info = pb.pb_batch_solve(ctxs, variants, restart=args.restart, tol=args.tol, use_graph=True,
                                               raise_on_noconv=False)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            infos.append(info)
        launches = pb.pb_kernel_launches() - l0
        clocks = sampler.stop()
        # product kernel timing (one extra batch in one engine, kernels launched
        # one by one with events, so that the timed launches do not overlap)
        pb.pb_batch_set_streams(1)
        try:
            _, tinfo = pb.pb_batch_solve(ctxs, variants, restart=args.restart, tol=args.tol, use_graph="timed",
                                         raise_on_noconv=False)
        finally:
            pb.pb_batch_set_streams(args.batch_streams)
        # accuracy: every charge set of the surfaces with a stored FP64 oracle
        # solution (the four smallest; tests/golden), against that solution
        errs = []
        for i in range(len(ctxs)):
            for r in range(8):
                name = f"batch{i}_set{r}"
                ref = golden_energy(name)
                if ref is not None and golden_n(name) == ns[i]:
                    errs.append(abs(energies[i][r] - ref) / abs(ref))
        for c in ctxs:
            pb.pb_destroy(c)
    total_ms = sum(times)
    products = sum(i["pair_products"] for i in infos)
    nsolve = sum(i["instances"] for i in infos)
    width = tinfo["rhs_width"]
    peak = SMS * 128 * SM_MAX_MHZ * 1e6 / ((BATCH_FP32_OPS_PER_EVAL + BATCH_FP32_OPS_PER_RHS * width) / width) / 1e9
    achieved = tinfo["pair_products"] / (tinfo["matvec_ms"] * 1e-3) / 1e9
    line = {"metric": METRIC, "value": products / (total_ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 pairs, f64 accumulation",
            "data": "synthetic",
            "config": {"workload": f"batch: {len(ctxs)} protein-like solutes (atoms log-uniform 50-1500, "
                                   f"N {min(ns)}-{max(ns)}) x 8 charge variants, one lockstep batch per step",
                       "n_triangles_total": int(sum(ns)), "instances": int(infos[-1]["instances"]),
                       "gmres_restart": args.restart, "gmres_tol": args.tol, "cuda_graph": True,
                       "engines": infos[-1]["streams"],
                       "product_shape": {"targets_per_thread": infos[-1]["targets_per_thread"],
                                         "row_sums": ROW_SUMS.get(infos[-1]["row_sums"]),
                                         "ctas_per_sm": infos[-1]["ctas_per_sm"] or "occupancy",
                                         "autotuned": bool(warm_info and warm_info["tuned"]),
                                         "tune_candidates": warm_info["tune_candidates"] if warm_info else 0,
                                         "tune_ms": warm_info["tune_ms"] if warm_info else 0.0},
                       "l2": "flushed between steps (256 MiB write)"},
            "solves_per_s": nsolve / (total_ms * 1e-3),
            "latency_ms": {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99))},
            "rel_energy_err": {"max_vs_oracle": max(errs) if errs else None, "results_compared": len(errs),
                               "note": "against the stored FP64 oracle solutions (tests/golden) of the four "
                                       "smallest solutes, all 8 charge sets"},
            "gmres": {"iters_max": infos[-1]["iters_max"], "cycles": infos[-1]["cycles"],
                      "converged": f"{infos[-1]['converged']}/{infos[-1]['instances']}"},
            "phases_ms": {"setup": infos[-1]["setup_ms"], "cycles": infos[-1]["cycles_ms"],
                          "energies": infos[-1]["energy_ms"],
                          "note": "host time of the last timed batch: set-up (vectors, float-float source terms), "
                                  "restart cycles, float-float energies"},
            "roofline": {"kernel": f"bmatvec_kernel<{width}>", "bound": "alu", "achieved": achieved, "peak": peak,
                         "unit": UNIT, "frac": achieved / peak, "traffic": None,
                         "peak_basis": f"FP32 pipe: {SMS} SMs x 128 lanes x {SM_MAX_MHZ:.0f} MHz / "
                                       f"({BATCH_FP32_OPS_PER_EVAL} + {BATCH_FP32_OPS_PER_RHS} x {width}) / {width} "
                                       "FP32 ops per pair and charge set (derived)",
                         "products_ms": tinfo["matvec_ms"], "launches": tinfo["matvec_launches"],
                         "in_batch": {"achieved": infos[-1]["pair_products"] / (infos[-1]["cycles_ms"] * 1e-3) / 1e9,
                                      "frac": infos[-1]["pair_products"] / (infos[-1]["cycles_ms"] * 1e-3) / 1e9
                                              / peak,
                                      "note": "pair products over the host time of the restart cycles of the last "
                                              "timed batch (products, orthogonalisation and all, the engines "
                                              "overlapping): a lower bound on the product rate in the batch; "
                                              "`achieved` above times the product launches alone, in one engine"}},
            "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    import threading

    import numpy as np
    specs = serve_specs(args.pool)
    pool = make_solutes(specs, _workers(args))
    import torch
    import paper_1301_5885_gb300 as pb
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    kappas = (0.0, 0.1257)
    ns = [a.shape[0] for _, _, a, _ in pool]
    budget = 96 << 30

    def submit(sv, k, kap):
        c, n, a, q = pool[k]
        return sv.submit(c, n, a, q, 1.0, 80.0, kap)

    # capacity: every pool solute at both kappas submitted at once
    with pb.Server(max_active=16, hbm_budget_bytes=budget, tol=args.tol) as sv:
        t = time.perf_counter()
        for k in range(len(pool)):
            for kap in kappas:
                submit(sv, k, kap)
        sv.wait(2 * len(pool), 3600.0)
        cal = sv.poll(4096)
        t_cal = time.perf_counter() - t
    capacity = 2 * len(pool) / t_cal
    rate = 0.7 * capacity
    rng = np.random.Generator(np.random.PCG64(5))
    gaps = rng.exponential(1.0 / rate, size=args.requests)
    picks = rng.integers(0, len(pool), size=args.requests)
    kaps = rng.integers(0, 2, size=args.requests)
    def stream(split_n, sampler=None):
        """The Poisson stream through a server; returns (results, wall s,
        stats before, stats after, launches, request keys)."""
        with pb.Server(max_active=16, hbm_budget_bytes=budget, tol=args.tol, split_n=split_n) as sv:
            st0 = sv.stats()
            if sampler:
                sampler.start()
            l0 = pb.pb_kernel_launches()
            t_start = time.perf_counter()
            keys_by_id = {}

            def feeder():
                for g, k, kk in zip(gaps, picks, kaps):
                    time.sleep(float(g))
                    keys_by_id[submit(sv, int(k), kappas[int(kk)])] = (int(k), int(kk))
            th = threading.Thread(target=feeder)
            th.start()
            th.join()
            sv.wait(args.requests, 3600.0)
            t_end = time.perf_counter()
            out = sv.poll(4096)
            st = sv.stats()
            return out, t_end - t_start, st0, st, pb.pb_kernel_launches() - l0, keys_by_id

    sampler = _clock_and_uuid(torch, dev)
    res, wall, st0, st1, launches, req_key = stream(0, sampler)
    clocks = sampler.stop()
    res1, wall1, _, _, _, _ = stream(-1)

    def lat_split(rs):
        small = np.array([r["latency_ms"] for r in rs if r["n"] < 16384])
        large = np.array([r["latency_ms"] for r in rs if r["n"] >= 16384])
        f = lambda a, q: float(np.percentile(a, q)) if a.size else None
        return {"small_p50": f(small, 50), "small_p99": f(small, 99), "large_p50": f(large, 50),
                "large_p99": f(large, 99), "n_small": int(small.size), "n_large": int(large.size)}
    lat = np.array([r["latency_ms"] for r in res])
    lat1 = np.array([r["latency_ms"] for r in res1])
    ok = all(r["status"] == pb.PB_OK for r in res) and all(r["status"] == pb.PB_OK for r in res1)
    products = st1["pair_products"] - st0["pair_products"]
    # one-at-a-time baselines on the same request mix, from per-item solve
    # times: every distinct (solute, kappa) of the stream solved alone in FP32
    # pairs, and in plain FP64 (the paper's precision) where that takes at most
    # a few seconds (N <= 20,000); above that the FP64 time is extrapolated
    # from the FP32 solve's product count and the FP64 product rate measured
    # on the largest pool solute with N <= 60,000
    # every (solute, kappa) of the pool: the calibration set the server's
    # capacity was measured on, which contains every request of the stream
    keys = [(k, kk) for k in range(len(pool)) for kk in (0, 1)]
    seq32, mv32, seq64, est64 = {}, {}, {}, {}
    rate64 = None
    # (each timed solve includes pb_create from the host arrays and pb_destroy,
    # the work the server does for a request)
    with torch.cuda.stream(torch.cuda.Stream()):
        for k, kk in keys:
            c, n, a, q = pool[k]
            for prec in ("fp32pair", "fp64"):
                if prec == "fp64" and ns[k] > 20000:
                    continue
                torch.cuda.synchronize()
                t = time.perf_counter()
                with pb.pb_create(c, n, a, q, 1.0, 80.0, kappas[kk]) as ctx:
                    inf = pb.pb_solve(ctx, tol=args.tol, prec=prec, raise_on_noconv=False)
                if prec == "fp32pair":
                    seq32[(k, kk)] = time.perf_counter() - t
                    mv32[(k, kk)] = inf.matvecs
                else:
                    seq64[(k, kk)] = time.perf_counter() - t
        mid = max((i for i in range(len(pool)) if ns[i] <= 60000), key=lambda i: ns[i])
        c, n, a, q = pool[mid]
        with pb.pb_create(c, n, a, q, 1.0, 80.0, kappas[1]) as ctx:
            u = torch.randn(2 * ns[mid], dtype=torch.float64, device=dev)
            y = torch.empty_like(u)
            pb.pb_matvec(ctx, u, y, "fp64")
            torch.cuda.synchronize()
            t = time.perf_counter()
            pb.pb_matvec(ctx, u, y, "fp64")
            torch.cuda.synchronize()
            rate64 = ns[mid] * (ns[mid] - 1) / (time.perf_counter() - t)
    for key in keys:
        if key not in seq64:
            k = key[0]
            est64[key] = mv32[key] * ns[k] * (ns[k] - 1) / rate64
    check = [abs(mv32[x] * ns[x[0]] * (ns[x[0]] - 1) / rate64 - seq64[x]) / seq64[x] for x in seq64
             if ns[x[0]] >= 10000]
    # energies against the stored FP64 oracle solutions of the small pool solutes
    errs = []
    for r in res:
        key = req_key.get(r["id"])
        if key is None:
            continue
        ref = golden_energy(f"serve{key[0]}_kappa{key[1]}")
        if ref is not None and golden_n(f"serve{key[0]}_kappa{key[1]}") == ns[key[0]]:
            errs.append(abs(r["energy_kcal"] - ref) / abs(ref))
    stream_keys = [(int(k), int(kk)) for k, kk in zip(picks, kaps)]
    t32 = sum(seq32[x] for x in stream_keys)
    t64 = sum(seq64.get(x, est64.get(x, 0.0)) for x in stream_keys)
    n64m = sum(1 for x in stream_keys if x in seq64)
    t32_cal = sum(seq32[x] for x in keys)
    t64_cal = sum(seq64.get(x, est64.get(x, 0.0)) for x in keys)
    line = {"metric": METRIC, "value": products / wall / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.requests,
            "warmup": 2 * len(pool), "ms_per_step": 1e3 * wall / args.requests, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 pairs, f64 accumulation", "data": "synthetic",
            "config": {"workload": f"serve: {args.requests} Poisson arrivals at 0.7 x measured capacity "
                                   f"({rate:.2f}/s), drawn from {len(pool)} distinct protein-like solutes with N "
                                   f"log-uniform 5k-300k ({min(ns)}-{max(ns)}), kappa in {{0, 0.1257}}",
                       "distinct_requests": len(keys), "max_active": 16, "hbm_budget_bytes": budget,
                       "gmres_tol": args.tol, "l2": "inputs exceed L2 across the stream; no flush"},
            "solves_per_s": len(res) / wall,
            "latency_ms": dict({"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                "mean": float(lat.mean())}, **lat_split(res)),
            "one_lane": {"note": "the same stream through a server with one lane (split_n = -1): every request "
                                 "in one lockstep engine",
                         "solves_per_s": len(res1) / wall1,
                         "latency_ms": dict({"p50": float(np.percentile(lat1, 50)),
                                             "p99": float(np.percentile(lat1, 99))}, **lat_split(res1))},
            "all_converged": ok, "max_active_seen": st1["max_active_seen"],
            "rel_energy_err": {"max_vs_oracle": max(errs) if errs else None, "results_compared": len(errs),
                               "note": "against the stored FP64 oracle solutions (tests/golden) of the pool "
                                       "solutes small enough for the oracle"},
            "capacity_solves_per_s": capacity,
            "capacity_note": f"all {len(keys)} (solute, kappa) requests of the pool submitted at once; the "
                             "sequential rates on that same set are the capacity's baselines",
            "baselines": {
                "sequential_fp32_solves_per_s_calibration_set": len(keys) / t32_cal,
                "sequential_fp64_solves_per_s_calibration_set": len(keys) / t64_cal,
                "capacity_over_sequential_fp32": capacity / (len(keys) / t32_cal),
                "capacity_over_sequential_fp64": capacity / (len(keys) / t64_cal),
                "sequential_fp32_solves_per_s": args.requests / t32,
                "sequential_fp64_solves_per_s": args.requests / t64,
                "fp64_note": f"same {args.requests}-request mix solved one at a time in plain FP64 (symmetric FP64 "
                             f"product), each timed from pb_create to pb_destroy as the FP32 ones; "
                             f"{n64m} requests timed (N <= 20,000), the other "
                             f"{args.requests - n64m} extrapolated as FP32-solve products x N(N-1) / "
                             f"{rate64 / 1e9:.2f} Gpairs/s (the FP64 product rate measured at N = {ns[mid]})",
                "fp64_extrapolation_check": {"max_rel_dev_on_timed_N_ge_10k": max(check) if check else None,
                                             "timed": len(check)},
                "stream_note": "the last two are on the 200-request stream mix; the stream is offered at 0.7 x "
                               "capacity, so its served rate is not a capacity"},
            "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def run_frames(args):
    """Warm-started repeated solves: a trajectory of perturbed frames of one
    solute (pb_inputs.md_frames), each solved cold (x0 = 0) and warm (x0 =
    the previous frame's solution); per-frame CUDA-event times, iterations and
    the agreement of the two energies."""
    import numpy as np
    import pb_inputs
    import torch
    import paper_1301_5885_gb300 as pb
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    base = pb_inputs.protein_like(n_atoms=400, seed=11, target_triangles=60000)
    frames = pb_inputs.md_frames(base, args.frames)
    stream = torch.cuda.current_stream()
    n = base.n
    x_prev = None
    rows = []
    sampler = _clock_and_uuid(torch, dev)
    sampler.start()
    l0 = pb.pb_kernel_launches()
    for f in frames:
        s = f.surface
        dev_in = [torch.tensor(a, device=dev) for a in (s.centroids, s.normals, s.areas, f.charges)]
        ctx = pb.pb_create(*dev_in, f.eps1, f.eps2, f.kappa, stream=stream)
        try:
            out = {}
            x = torch.empty(2 * n, dtype=torch.float64, device=dev)
            for kind, x0, xo in (("cold", None, None), ("warm", x_prev, x)):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                info = pb.pb_solve(ctx, restart=args.restart, tol=args.tol, maxit=3000, prec="fp32pair", x0=x0,
                                   x_out=xo)
                e1.record(stream)
                e1.synchronize()
                out[kind] = (e0.elapsed_time(e1), info)
        finally:
            pb.pb_destroy(ctx)
        rows.append(out)
        x_prev = x
    launches = pb.pb_kernel_launches() - l0
    clocks = sampler.stop()
    later = rows[1:]
    cold_ms = sum(r["cold"][0] for r in later)
    warm_ms = sum(r["warm"][0] for r in later)
    cold_it = sum(r["cold"][1].iters for r in later)
    warm_it = sum(r["warm"][1].iters for r in later)
    warm_mv = sum(r["warm"][1].matvecs for r in later)
    dE = max(abs(r["warm"][1].energy_kcal - r["cold"][1].energy_kcal) / abs(r["cold"][1].energy_kcal) for r in rows)
    line = {"metric": METRIC, "value": warm_mv * n * (n - 1) / (warm_ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1,
            "steps": len(later), "warmup": 1, "ms_per_step": warm_ms / len(later), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 pairs, f64 accumulation", "data": "synthetic",
            "config": {"workload": f"frames: {args.frames} perturbed frames (smooth deformation, 0.06 A per frame; "
                                   f"charge jitter 0.02 e) of a 400-atom protein-like solute, N = {n}",
                       "gmres_restart": args.restart, "gmres_tol": args.tol},
            "solves_per_s": len(later) / (warm_ms * 1e-3),
            "frames": {"cold_ms": cold_ms, "warm_ms": warm_ms, "cold_iters": cold_it, "warm_iters": warm_it,
                       "time_saved": 1.0 - warm_ms / cold_ms, "iters_saved": 1.0 - warm_it / cold_it,
                       "per_frame_iters": [[r["cold"][1].iters, r["warm"][1].iters] for r in rows]},
            "rel_energy_err": {"max_warm_vs_cold": dE,
                               "note": "each frame's energy against the oracle: tests/test_gpu_frames.py"},
            "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def run_sharded(args):
    """One solve row-sharded over the N GPUs of the job (strong scaling): every
    rank holds the whole surface and evaluates its rows of each product,
    one NCCL allgather per product, GMRES replicated (pb_solve_sharded)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    import paper_1301_5885_gb300 as pb
    import pb_inputs
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl")
    else:
        import socket
        with socket.socket() as so:
            so.bind(("127.0.0.1", 0))
            port = so.getsockname()[1]
        dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    prob = pb_inputs.by_name(args.workload)
    s = prob.surface
    n = prob.n
    dev_in = [torch.tensor(a, device=dev) for a in (s.centroids, s.normals, s.areas, prob.charges)]
    stream = torch.cuda.current_stream()
    ctx = pb.pb_create(*dev_in, prob.eps1, prob.eps2, prob.kappa, stream=stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    try:
        for _ in range(args.warmup):
            pb.pb_solve_sharded(ctx, restart=args.restart, tol=args.tol, maxit=3000, prec="fp32pair")
        torch.cuda.synchronize()
        sampler = _clock_and_uuid(torch, dev)
        dist.barrier()
        torch.cuda.synchronize()
        sampler.start()
        l0 = pb.pb_kernel_launches()
        times, infos = [], []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos.append(pb.pb_solve_sharded(ctx, restart=args.restart, tol=args.tol, maxit=3000, prec="fp32pair"))
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        dist.barrier()
        launches = pb.pb_kernel_launches() - l0
        clocks = sampler.stop()
    finally:
        pb.pb_destroy(ctx)
    total = torch.tensor([sum(times)], dtype=torch.float64, device=dev)
    dist.all_reduce(total, op=dist.ReduceOp.MAX)
    total_ms = total.item()
    if rank == 0:
        ref = golden_energy(args.workload, prob)
        e = infos[-1].energy_kcal
        mv = sum(i.matvecs for i in infos)
        line = {"metric": METRIC, "value": mv * n * (n - 1) / (total_ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                "dtype": "f32 pairs, f64 accumulation", "data": "synthetic",
                "config": dict(config_dict(args, prob), parallelism=f"row-sharded over {world} GPU(s)"),
                "solves_per_s": args.steps / (total_ms * 1e-3),
                "latency_ms": {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99))},
                "energy_kcal": e, "oracle_energy_kcal": ref,
                "rel_energy_err": abs(e - ref) / abs(ref) if ref else None,
                "gmres": {"iters": infos[-1].iters, "matvecs": infos[-1].matvecs},
                "note": "value counts the N(N-1) pairs of every product of the solve once, over the slowest "
                        "rank's time; each rank evaluates its N/world rows of every product",
                "gpu_launches": launches, "clocks": clocks}
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.tol is None:
        args.tol = default_tol(args.mode, args.workload)
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "matvec":
        return run_matvec(args)
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "frames":
        return run_frames(args)
    if args.mode == "sharded":
        return run_sharded(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
