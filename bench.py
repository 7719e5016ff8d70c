#!/usr/bin/env python
"""Benchmark of the even-odd Wilson/clover solver path on one GB300.

Workload (default): even-odd clover operator on a 32^3 x 64 lattice,
c_sw = 1.0, kappa = 0.125, links exp(0.2 i A) (seed 2), one Gaussian source;
FP32 inner BiCGStab inside FP64 defect correction, solved to a true FP64
relative residual of 1e-10.

A step is one complete solve (setup excluded: gauge field and clover term are
resident).  value = algorithmic bytes moved by all kernels of the step (each
input read once, each output written once, as counted per launch by the
library) / step time -- the whole-job HBM throughput of the solve, to be read
against the HBM peak.  Beside it the line reports:

* roofline: the dominant kernel of the step, timed with CUDA events on the
  library stream in an event-profiled extra step;
* deo: the plain D_eo hopping kernel alone on resident FP32 fields;
* solve: the mixed solve against a plain FP64 BiCGStab solve of the same system;
* serving: p50/p99 latency of a short Poisson stream of requests through the
  continuous-batching engine;
* e2e: the same solve through bridge_solve with pinned host buffers
  (host->device copies of b and x0 and the device->host copy of x timed);
* cpu_baseline: the FP64 numpy oracle on a bounded sample of the workload.

``--impl reference`` times only the oracle (the reference for this path).

``--workload mobius_24x24x24x48x16`` runs the same measurements for the
Moebius domain-wall operator (Ls = 16, M5 = 1.8, b = 1.5, c = 0.5,
m_f = 0.01): a step is one mixed-precision CG solve on the normal equations
of the even-odd system (FP32 inner, FP64 defect correction, 1e-10), beside
D_eo alone and a plain FP64 CG solve.  ``--workload staggered_64x64x64x64``
does the same for the staggered operator (m = 0.05, CG on the even system);
``--workload mg_clover_32x32x32x64`` times the two-level multigrid solver
(setup reported separately) against the mixed BiCGStab on the same
near-critical clover system, for one and for twelve equations.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D_eo GB/s vs HBM peak; mixed vs FP64 solve time to 1e-10; p50/p99 solve latency"
UNIT = "GB/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="clover_32x32x32x64")
    ap.add_argument("--serving-requests", type=int, default=200)
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison solve")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg through host buffers")
    ap.add_argument("--inner", default=None, help="override the workload's inner storage precision (f32, f16, bf16)")
    ap.add_argument("--rate-factors", type=float, nargs="+", default=[0.5, 0.7, 0.9],
                    help="serving workload: arrival rates as fractions of the saturated rate")
    ap.add_argument("--oracle-sites", type=int, default=16384, help="sites per oracle sample")
    ap.add_argument("--multi-rhs", default="clover_48x48x48x96_12rhs",
                    help="clover workload: the multi-RHS workload measured beside it ('' to skip)")
    ap.add_argument("--multi-rhs-steps", type=int, default=2, help="timed solves of the multi-RHS workload")
    ap.add_argument("--oracle-solves", action="store_true",
                    help="reference arm: also time the oracle's even-odd BiCGStab on the 8^4 Wilson and a 16^4 clover system")
    ap.add_argument("--deo-only", action="store_true",
                    help="Moebius workload: only the operator legs (one Schur operator, then D_eo), for profiler captures")
    return ap.parse_args()


# --------------------------------------------------------------------- helpers


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples of the SM clock and throttle reasons while running."""

    FIELDS = (
        "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
        "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
        "clocks_event_reasons.sw_power_cap"
    )

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
            )
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) != 7:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), float(parts[2]), parts[3:]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower().startswith("active")})
        return {
            "sm_mhz": statistics.median(r[0] for r in rows),
            "sm_max_mhz": max(r[1] for r in rows),
            "power_w_max": max(r[2] for r in rows),
            "samples": len(rows),
            "reasons": reasons,
        }


def traffic_for(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it matches the current kernel source."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", text)
    if not m or not h or h.group(1) != kernel_source_hash(kernel):
        return None
    return float(m.group(1))


def kernel_source_hash(kernel: str = "") -> str:
    d = hashlib.sha256()
    files = ["common.cuh", "dslash.cuh", "dslash_tile.cuh", "reduce.cuh"] + (["dwf.cuh"] if kernel.startswith("dwf") else []) + (
        ["stag.cuh"] if kernel.startswith("stag") else []) + (["mg.cuh"] if kernel.startswith("mg") else [])
    for f in files:
        d.update(open(os.path.join(ROOT, "paper_2303_05883_gb300", "csrc", f), "rb").read())
    return d.hexdigest()[:16]


def cpu_cores_used(fn):
    t0, c0 = time.perf_counter(), os.times()
    r = fn()
    t1, c1 = time.perf_counter(), os.times()
    cpu = (c1.user - c0.user) + (c1.system - c0.system)
    return r, t1 - t0, max(1, round(cpu / max(t1 - t0, 1e-9)))


# oracle sample: the FP64 clover operator at randomly drawn sites of the workload
FP64_D_BYTES_PER_SITE = 192 + 8 * 144 + 576 + 192  # spinor in, 8 links, T, spinor out


def oracle_sample(w, U, b, nsites, seed):
    from oracle import dirac
    from oracle.lattice import Lattice

    lat = Lattice(w.dims)
    nsites = min(nsites, lat.V)
    sites = np.sort(np.random.default_rng(seed).choice(lat.V, nsites, replace=False))
    csw = w.csw if w.kind == "clover" else 0.0

    def run():
        return dirac.dirac(U, b, lat, w.kappa, csw, w.bc, sites=sites)

    _, secs, cores = cpu_cores_used(run)
    return nsites * FP64_D_BYTES_PER_SITE / secs / 1e9, secs, cores


_ORACLE_LAT = {}


def _oracle_chunk(args):
    """Worker of oracle_sample_pool: the clover D of the oracle at a chunk of
    sites, reading U and b from shared memory."""
    from multiprocessing import shared_memory

    from oracle import dirac
    from oracle.lattice import Lattice

    (un, ushape, bn, bshape, dims, kappa, csw, bc, sites) = args
    if len(sites) == 0:
        return 0
    lat = _ORACLE_LAT.get(tuple(dims))
    if lat is None:
        lat = _ORACLE_LAT[tuple(dims)] = Lattice(dims)
    su, sb = shared_memory.SharedMemory(name=un), shared_memory.SharedMemory(name=bn)
    try:
        U = np.ndarray(ushape, dtype=np.complex128, buffer=su.buf)
        b = np.ndarray(bshape, dtype=np.complex128, buffer=sb.buf)
        dirac.dirac(U, b, lat, kappa, csw, bc, sites=sites)
        del U, b
    finally:
        su.close()
        sb.close()
    return len(sites)


def oracle_sample_pool(w, U, b, nsites, seed, procs=None):
    """oracle_sample over every host core: the sampled sites split among
    spawned worker processes that read U and b from shared memory (worker
    start-up and the lattice tables are outside the timed map)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory

    procs = procs or os.cpu_count() or 1
    nsites = min(nsites, int(np.prod(w.dims)))
    sites = np.sort(np.random.default_rng(seed).choice(int(np.prod(w.dims)), nsites, replace=False))
    csw = w.csw if w.kind == "clover" else 0.0
    su = shared_memory.SharedMemory(create=True, size=U.nbytes)
    sb = shared_memory.SharedMemory(create=True, size=b.nbytes)
    try:
        np.ndarray(U.shape, dtype=U.dtype, buffer=su.buf)[...] = U
        np.ndarray(b.shape, dtype=b.dtype, buffer=sb.buf)[...] = b
        mk = lambda chunks: [(su.name, U.shape, sb.name, b.shape, tuple(w.dims), w.kappa, csw, tuple(w.bc), c)  # noqa: E731
                             for c in chunks]
        with mp.get_context("spawn").Pool(procs) as pool:
            pool.map(_oracle_chunk, mk(np.array_split(sites[: 4 * procs], procs)), chunksize=1)  # warm the workers
            t0 = time.perf_counter()
            done = sum(pool.map(_oracle_chunk, mk(np.array_split(sites, procs)), chunksize=1))
            secs = time.perf_counter() - t0
    finally:
        su.close()
        su.unlink()
        sb.close()
        sb.unlink()
    return done * FP64_D_BYTES_PER_SITE / secs / 1e9, secs, procs


# ------------------------------------------------------------------- serving


def serving_sample(api, n_requests, main_lattice, main_U, seed=5, rate_factor=0.7):
    """Poisson stream through the request engine; returns latency stats."""
    import synth

    rng = np.random.default_rng(seed)
    sizes = [(8, 8, 8, 8), (16, 16, 16, 16), (24, 24, 24, 48), (32, 32, 32, 64)]
    pool = {}
    for dims in sizes:
        for eps in (0.1, 0.3):
            if dims == main_lattice["dims"] and eps == 0.3:
                continue
            L = api.Lattice(dims)
            L.upload(synth.gauge_field(dims, eps, seed + len(pool)))
            pool[(dims, eps)] = L
    pool[(main_lattice["dims"], 0.2)] = main_lattice["L"]
    keys = list(pool)

    # one 12-source Gaussian pool per lattice size; a request takes the first
    # nrhs of them (a view: the library copies what it keeps)
    sources = {dims: synth.gaussian_spinor(dims, 1000 + k, nrhs=12) for k, dims in enumerate(sizes)}

    def make(i):
        dims, eps = keys[rng.integers(len(keys))]
        kappa = float(rng.uniform(0.11, 0.13))
        kind = "clover" if rng.integers(2) else "wilson"
        nrhs = int(rng.integers(1, 13))
        op = api.make_op(kind, kappa, 1.0 if kind == "clover" else 0.0)
        return pool[(dims, eps)], op, sources[dims][:nrhs]

    reqs = [make(i) for i in range(n_requests)]
    # past the critical kappa of the smooth (eps = 0.1) fields BiCGStab
    # stagnates; the automatic inner method then switches those requests to
    # CG on the normal equations.  A per-request cap bounds latency and is
    # reported.
    max_iter = 20000
    solver = api.make_solver(tol=1e-10, max_iter=max_iter)
    # saturated throughput from a burst of the first requests; every request
    # borrows its b from the shared source pools (no host copy while queued)
    burst = reqs[: max(4, min(100, n_requests // 4))]
    t0 = time.perf_counter()
    hs = [api.bridge_submit(L.handle, op, solver, b, borrow=True) for L, op, b in burst]
    for h in hs:
        api.bridge_wait(h, want_x=False)
        api.bridge_request_release(h)
    sat = len(burst) / (time.perf_counter() - t0)
    # Poisson arrivals at rate_factor x the saturated rate
    lam = rate_factor * sat
    arrivals = np.cumsum(rng.exponential(1.0 / lam, size=n_requests))
    import queue
    import threading

    pending = queue.Queue()
    results = []

    def collect():
        # release requests in the order they finish (a finished request holds
        # its result on the host until it is released), polling without a wait
        live, more = [], True
        while more or live:
            try:
                while True:
                    item = pending.get_nowait()
                    if item is None:
                        more = False
                        break
                    live.append(item)
            except queue.Empty:
                pass
            still = []
            for h, nr, size in live:
                r = api.bridge_wait(h, 0, want_x=False)
                if r is None:
                    still.append((h, nr, size))
                    continue
                st, _, info = r
                cg = any(i["cgnr_passes"] > 0 for i in info)
                results.append((st, nr, size, api.bridge_request_times(h), cg))
                api.bridge_request_release(h)
            live = still
            time.sleep(0.001)

    waiter = threading.Thread(target=collect)
    waiter.start()
    start = time.perf_counter()
    for (L, op, b), ta in zip(reqs, arrivals):
        delay = start + ta - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        pending.put((api.bridge_submit(L.handle, op, solver, b, borrow=True), b.shape[0], "x".join(map(str, L.dims))))
    pending.put(None)
    waiter.join()
    lat_ms, lat_ok, ok, nrhs_total, statuses, by_size = [], [], 0, 0, {}, {}
    waits, runs, n_cg, lat_cg = [], [], 0, []
    for st, nr, size, (ts, ta, td), cg in results:
        if cg:
            n_cg += 1
            lat_cg.append((td - ts) * 1e3)
        lat_ms.append((td - ts) * 1e3)
        waits.append((ta - ts) * 1e3)
        runs.append((td - ta) * 1e3)
        by_size.setdefault(size, []).append((td - ts) * 1e3)
        if st == 0:
            lat_ok.append((td - ts) * 1e3)
        ok += st == 0
        statuses[api.bridge_strerror(st)] = statuses.get(api.bridge_strerror(st), 0) + 1
        nrhs_total += nr
    wall = time.perf_counter() - start
    for k, L in pool.items():
        if L is not main_lattice["L"]:
            L.close()
    return {
        "requests": n_requests,
        "ok": ok,
        "arrival_rate_per_s": lam,
        "saturated_solves_per_s": sat,
        "solves_per_s": n_requests / wall,
        "statuses": statuses,
        "max_iter_per_request": max_iter,
        "requests_switched_to_cgnr": n_cg,
        "p50_ms_cgnr": float(np.percentile(lat_cg, 50)) if lat_cg else None,
        "p50_ms": float(np.percentile(lat_ms, 50)),
        "p99_ms": float(np.percentile(lat_ms, 99)),
        "p50_ms_converged": float(np.percentile(lat_ok, 50)) if lat_ok else None,
        "p99_ms_converged": float(np.percentile(lat_ok, 99)) if lat_ok else None,
        "rhs_solved": nrhs_total,
        "p50_ms_by_lattice": {k: float(np.percentile(v, 50)) for k, v in sorted(by_size.items())},
        "queue_wait_ms_p50_p99": [float(np.percentile(waits, 50)), float(np.percentile(waits, 99))],
        "run_ms_p50_p99": [float(np.percentile(runs, 50)), float(np.percentile(runs, 99))],
        "rate_factor": rate_factor,
        "lattices": ["x".join(map(str, d)) for d in sizes],
        "kappa": [0.11, 0.13],
        "nrhs": [1, 12],
    }


# ----------------------------------------------------------------------- main


def aggregate_ranks(ms: float, nbytes: float, device="cpu"):
    """Whole-job view over ranks: the slowest rank's time and the sum of work."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms, nbytes
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    b = torch.tensor([nbytes], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return float(t.item()), float(b.item())


def _parity_odd_index(dims):
    """For each lexicographic pair (2k, 2k+1), which member is the odd site."""
    Lx, Ly, Lz, Lt = dims
    k = np.arange(int(np.prod(dims)) // 2)
    rest = k // (Lx // 2)
    y, z, t = rest % Ly, (rest // Ly) % Lz, rest // (Ly * Lz)
    return ((1 + y + z + t) % 2).astype(np.int64)


def run_e2e(args, h, op, solver, b_dev, b_host, nrhs, total_bytes, world):
    """The same solve through bridge_solve with pinned host buffers."""
    import ctypes

    import torch

    from paper_2303_05883_gb300 import _abi

    if b_host is None:
        b_host = b_dev.cpu().numpy()
    b_pin = torch.from_numpy(b_host).pin_memory()
    x_pin = torch.zeros_like(b_pin).pin_memory()
    bn, xn = b_pin.numpy(), x_pin.numpy()
    lib = _abi.load()
    info = (_abi.bridge_info * nrhs)()
    dp = ctypes.POINTER(ctypes.c_double)
    bp, xp = ctypes.cast(b_pin.data_ptr(), dp), ctypes.cast(x_pin.data_ptr(), dp)
    e2e_t = []
    for k in range(args.steps):
        xn[...] = 0
        t0 = time.perf_counter()
        _abi.check(lib.bridge_solve(h, ctypes.byref(op), ctypes.byref(solver), bp, xp, nrhs, info), "bridge_solve")
        e2e_t.append(time.perf_counter() - t0)
    nbytes = b_host.nbytes
    e2e = {"value": (total_bytes / args.steps) / statistics.median(e2e_t) / 1e9 if world == 1 else None,
           "unit": UNIT, "h2d_bytes_per_step": 2 * nbytes, "d2h_bytes_per_step": nbytes,
           "ms_per_step": 1e3 * statistics.median(e2e_t)}

    return e2e


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    """The oracle as it stands on the host cores; rank 0 only."""
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    import synth

    w = synth.WORKLOADS[args.workload]
    U = w.gauge()
    b = w.sources()[0]
    # the oracle's operator of the workload's kind, at a bounded random sample of sites
    if args.workload.startswith("mobius"):
        n = max(16, args.oracle_sites // 64)
        fn = mobius_oracle_sample
        sample = (f"FP64 numpy oracle: Moebius D at {n} random four-dimensional sites x Ls = {w.Ls} of the "
                  f"{args.workload} lattice per step")
        config = {"workload": args.workload, "lattice": "x".join(map(str, w.dims)), "Ls": w.Ls, "M5": w.M5,
                  "b5": w.b5, "c5": w.c5, "mf": w.mf, "sample_sites": n}
    elif args.workload.startswith("staggered"):
        n = args.oracle_sites * 4
        fn = staggered_oracle_sample
        sample = f"FP64 numpy oracle: staggered D at {n} random sites of the {args.workload} lattice per step"
        config = {"workload": args.workload, "lattice": "x".join(map(str, w.dims)), "mass": w.mass, "sample_sites": n}
    else:
        n = args.oracle_sites
        fn = oracle_sample
        sample = f"FP64 numpy oracle: clover D at {n} random sites of the {args.workload} lattice per step"
        config = {"workload": args.workload, "lattice": "x".join(map(str, w.dims)), "kappa": w.kappa, "csw": w.csw,
                  "eps": w.eps, "sample_sites": n}
    vals, secs_all, cores_all = [], [], []
    for k in range(args.warmup + args.steps):
        v, secs, cores = fn(w, U, b, n, seed=k)
        if k >= args.warmup:
            vals.append(v)
            secs_all.append(secs)
            cores_all.append(cores)
    value = float(np.mean(vals))
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.mean(secs_all)),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": max(cores_all), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    if args.oracle_solves:
        line["oracle_solves"] = oracle_solves()
    print(json.dumps(line), flush=True)


def oracle_solves():
    """The oracle's even-odd BiCGStab, as it stands, on two whole systems: the
    8^4 Wilson workload (kappa 0.12, tol 1e-12) and a 16^4 clover system
    (kappa 0.125, c_sw 1, links exp(0.2 i A), tol 1e-10); one process."""
    import synth
    from oracle import evenodd, solvers
    from oracle.lattice import Lattice

    out = {}
    for name, dims, kappa, csw, eps, seed, tol in [("wilson_8x8x8x8", (8, 8, 8, 8), 0.12, 0.0, 0.3, 1, 1e-12),
                                                    ("clover_16x16x16x16", (16, 16, 16, 16), 0.125, 1.0, 0.2, 2, 1e-10)]:
        lat = Lattice(dims)
        U = synth.gauge_field(dims, eps, seed)
        b = synth.gaussian_spinor(dims, seed)
        t0 = time.perf_counter()
        eo = evenodd.EvenOdd(U, lat, kappa, csw)
        xe, info = solvers.bicgstab(eo.schur, eo.prepare(b), tol=tol)
        x = eo.reconstruct(xe, b)
        secs = time.perf_counter() - t0
        out[name] = {"seconds": secs, "iterations": info["iters"], "true_rel_residual": info["true_rel_residual"],
                     "cores": 1, "includes": "clover term setup, preparation, BiCGStab, reconstruction"}
        del x
    return out


def alu_peaks(api):
    """Measured scalar FMA throughput (TFLOP/s) of the FP32 and FP64 pipes."""
    return {"f32_tflops": api.bridge_alu_peak("f32") / 1e12, "f64_tflops": api.bridge_alu_peak("f64") / 1e12,
            "how": "bridge_alu_peak: every SM filled with independent scalar FMA chains, 2 flops per FMA, best of 5"}


def multi_rhs_leg(args, api, local, peak, alu):
    """The multi-RHS workload beside the plain FP64 solve.

    48^3 x 96 clover (c_sw = 1, kappa = 0.125, links exp(0.2 i A), seed 3),
    the 12 spin-colour point sources at the origin, FP16 storage with
    per-site scales, FP32 inner BiCGStab, FP64 defect correction to a true
    relative residual of 1e-10 for every right-hand side.  Timed: K solves of
    all 12 right-hand sides with resident inputs (CUDA events on the library
    stream), then one event-profiled solve for the per-kernel rooflines, then
    one plain FP64 BiCGStab solve of the first right-hand side (the
    comparison is 12 x that time).
    """
    import ctypes

    import torch

    import synth
    from paper_2303_05883_gb300 import _abi

    w = synth.WORKLOADS[args.multi_rhs]
    nrhs = w.nrhs
    t_setup = time.perf_counter()
    U = w.gauge()
    op = api.make_op(w.kind, w.kappa, w.csw, w.bc)
    L = api.Lattice(w.dims)
    L.upload(U, op)
    del U
    h = L.handle
    b = torch.zeros((nrhs, w.volume, 4, 3), dtype=torch.complex128, device=f"cuda:{local}")
    for k in range(nrhs):
        b[k, 0, k // 3, k % 3] = 1.0
    x = torch.zeros_like(b)
    lib = _abi.load()

    def solve(prm, n):
        x.zero_()
        torch.cuda.current_stream().synchronize()
        info = (_abi.bridge_info * n)()
        _abi.check(lib.bridge_solve_dev(h, ctypes.byref(op), ctypes.byref(prm), ctypes.c_void_p(b.data_ptr()),
                                        ctypes.c_void_p(x.data_ptr()), n, info), "bridge_solve_dev")
        return [info[k] for k in range(n)]

    api.bridge_tune(h, op, w.inner, nrhs)
    mixed = api.make_solver(tol=w.tol, inner_prec=w.inner, mixed=1)
    solve(mixed, nrhs)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    api.bridge_stats_reset(h)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    K = max(1, args.multi_rhs_steps)
    with Clocks(local) as clk:
        e0.record(L.stream)
        for _ in range(K):
            infos = solve(mixed, nrhs)
        e1.record(L.stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    st = api.bridge_stats(h)
    gbs = sum(v["bytes"] for v in st.values()) / K / (ms * 1e-3) / 1e9
    # one event-profiled solve: per-kernel times of exactly the iterations run
    api.bridge_stats_reset(h)
    api.bridge_profile(h, True)
    solve(mixed, nrhs)
    torch.cuda.synchronize()
    api.bridge_profile(h, False)
    pst = api.bridge_stats(h)
    step_ms = sum(v["ms"] for v in pst.values())
    site_rhs = nrhs * w.volume // 2
    flops_site = {"schur_pass1": 1848, "schur_pass2_alpha": 1944, "schur_pass2_omega": 1944}
    kernels = {}
    for k, fl in flops_site.items():
        d = pst.get(k)
        if not d or d["launches"] == 0:
            continue
        us = 1e3 * d["ms"] / d["launches"]
        ach = d["bytes"] / d["launches"] / (us * 1e-6) / 1e9
        tf = site_rhs * fl / (us * 1e-6) / 1e12
        kernels[k] = {"avg_launch_us": us, "algorithmic_bytes_per_launch": d["bytes"] / d["launches"],
                      "traffic": traffic_for(k, w.name),
                      "gbs": ach, "hbm_frac": ach / peak, "tflops": tf,
                      "fp32_frac": tf / alu["f32_tflops"] if alu else None,
                      "share_of_step": d["ms"] / step_ms if step_ms else None}
    shares = {k: round(v["ms"] / step_ms, 4) for k, v in pst.items() if v["ms"] > 0}
    res = max(i.true_rel_residual for i in infos)
    out = {"workload": w.name, "lattice": "x".join(map(str, w.dims)), "nrhs": nrhs, "inner_prec": w.inner,
           "mixed_ms": ms, "mixed_steps": K, "gbs": gbs, "inner_iters": max(i.inner_iters for i in infos),
           "outer_iters": max(i.outer_iters for i in infos), "true_rel_residual": res,
           "status": sorted({i.status for i in infos}), "kernels": kernels, "kernel_shares": shares,
           "launch_shapes": {k: {"block": v[0], "site_blocks": v[1], "variant": v[2]}
                             for k, v in api.bridge_tune_table(h).items() if k.startswith("hop/")},
           "clocks": clk.summary(), "setup_s": setup_s}
    if not args.no_fp64:
        api.bridge_tune(h, op, "f64", 1)
        s64 = api.make_solver(tol=w.tol, mixed=0)
        t0 = time.perf_counter()
        i64 = solve(s64, 1)[0]
        t64 = time.perf_counter() - t0
        out.update({"fp64_ms_one_rhs": 1e3 * t64, "fp64_ms": nrhs * 1e3 * t64, "fp64_inner_iters": i64.inner_iters,
                    "fp64_true_rel_residual": i64.true_rel_residual, "speedup": nrhs * 1e3 * t64 / ms})
    L.close()
    del b, x
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__ as g

    if rank == 0:
        g.build()
    if world > 1:
        dist.barrier()
    import synth
    from paper_2303_05883_gb300 import api

    w = synth.WORKLOADS[args.workload]
    U = w.gauge()
    nrhs = w.nrhs
    inner = args.inner or w.inner
    if w.source == "point":
        # the 12 spin-colour point sources at the origin, built on the device
        b_dev = torch.zeros((nrhs, w.volume, 4, 3), dtype=torch.complex128, device=f"cuda:{local}")
        for k in range(nrhs):
            b_dev[k, 0, k // 3, k % 3] = 1.0
        b_host = None
    else:
        b_host = w.sources()[0] if nrhs == 1 else w.sources()
        b_dev = torch.from_numpy(b_host).to(f"cuda:{local}")
    kind = w.kind
    op = api.make_op(kind, w.kappa, w.csw, w.bc)
    L = api.Lattice(w.dims)
    L.upload(U, op)
    h = L.handle
    solver = api.make_solver(tol=w.tol, inner_prec=inner, mixed=1)
    stream = L.stream
    x_dev = torch.zeros_like(b_dev)

    def solve_dev(prm, n=None):
        """One solve of the first n right-hand sides; returns the worst info record."""
        n = nrhs if n is None else n
        x_dev.zero_()
        torch.cuda.current_stream().synchronize()
        from ctypes import byref, c_void_p

        from paper_2303_05883_gb300 import _abi

        info = (_abi.bridge_info * n)()
        st = _abi.load().bridge_solve_dev(h, byref(op), byref(prm), c_void_p(b_dev.data_ptr()),
                                          c_void_p(x_dev.data_ptr()), n, info)
        _abi.check(st, "bridge_solve_dev")
        return max((info[k] for k in range(n)), key=lambda i: i.true_rel_residual)

    api.bridge_tune(h, op, inner, nrhs)
    if not args.no_fp64:
        api.bridge_tune(h, op, "f64", 1)
    for _ in range(args.warmup):
        solve_dev(solver)
    torch.cuda.synchronize()
    api.bridge_stats_reset(h)
    l0 = api.bridge_launch_count()
    infos = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        torch.cuda.nvtx.range_push("timed_steps")
        e0.record(stream)
        for _ in range(args.steps):
            infos.append(solve_dev(solver))
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    ms = e0.elapsed_time(e1)
    launches = api.bridge_launch_count() - l0
    st = api.bridge_stats(h)
    total_bytes = sum(v["bytes"] for v in st.values())
    ms, total_bytes = aggregate_ranks(ms, total_bytes, device=f"cuda:{local}")
    value = total_bytes / (ms * 1e-3) / 1e9
    res = max(i.true_rel_residual for i in infos)
    iters = statistics.median(i.inner_iters for i in infos)

    # ---- one event-profiled step: per-kernel times for the roofline
    api.bridge_stats_reset(h)
    api.bridge_profile(h, True)
    solve_dev(solver)
    torch.cuda.synchronize()
    api.bridge_profile(h, False)
    pst = api.bridge_stats(h)
    step_ms_prof = sum(v["ms"] for v in pst.values())
    dom = max(pst, key=lambda k: pst[k]["ms"])
    d = pst[dom]
    peak, peak_kind = peaks()
    achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9
    roofline = {
        "bound": "hbm",
        "kernel": dom,
        "achieved": achieved,
        "peak": peak,
        "peak_source": peak_kind,
        "unit": "GB/s",
        "frac": achieved / peak,
        "traffic": traffic_for(dom, args.workload),
        "algorithmic_bytes_per_launch": d["bytes"] / max(1, d["launches"]),
        "launches": d["launches"],
        "avg_launch_us": 1e3 * d["ms"] / max(1, d["launches"]),
        "share_of_step": d["ms"] / step_ms_prof if step_ms_prof else None,
    }
    shares = {k: round(v["ms"] / step_ms_prof, 4) for k, v in pst.items() if v["ms"] > 0}

    # ---- the plain D_eo hop kernel alone on resident FP32 fields
    fo = api.bridge_field_create(h, inner, 1, nrhs)
    fe = api.bridge_field_create(h, inner, 0, nrhs)
    # any odd half-lattice vectors do: use the odd sites of the source(s)
    half = b_dev.reshape(nrhs, w.volume // 2, 2, 4, 3)  # lexicographic pairs (2k, 2k+1)
    par = torch.from_numpy(_parity_odd_index(w.dims)).to(b_dev.device)
    src_odd = torch.gather(half, 2, par.view(1, -1, 1, 1, 1).expand(nrhs, -1, 1, 4, 3)).squeeze(2).contiguous()
    api.bridge_field_import(fo, src_odd)
    api.bridge_sync(h)
    for _ in range(3):
        api.bridge_apply(h, op, 1, fe, fo)
    reps = 50
    api.bridge_stats_reset(h)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(reps):
        api.bridge_apply(h, op, 1, fe, fo)
    a1.record(stream)
    torch.cuda.synchronize()
    deo_ms = a0.elapsed_time(a1) / reps
    deo_bytes = api.bridge_stats(h)["hop_deo"]["bytes"] / reps
    deo = {"kernel": "hop_deo", "prec": inner, "nrhs": nrhs, "gbs": deo_bytes / (deo_ms * 1e-3) / 1e9,
           "us_per_launch": deo_ms * 1e3, "bytes_per_launch": deo_bytes,
           "frac": deo_bytes / (deo_ms * 1e-3) / 1e9 / peak,
           "gflops": nrhs * w.volume / 2 * 1344 / (deo_ms * 1e-3) / 1e9}
    api.bridge_field_destroy(fo)
    api.bridge_field_destroy(fe)

    # ---- plain FP64 BiCGStab on the same system
    solve = {"mixed_ms": ms / args.steps, "mixed_inner_iters": iters, "mixed_true_rel_residual": res,
             "inner_prec": inner, "nrhs": nrhs}
    if not args.no_fp64:
        # plain FP64 BiCGStab on the first right-hand side; with several
        # right-hand sides the comparison is nrhs x that single solve
        s64 = api.make_solver(tol=w.tol, mixed=0)
        t0 = time.perf_counter()
        i64 = solve_dev(s64, n=1)
        t64 = time.perf_counter() - t0
        solve.update({"fp64_ms_one_rhs": t64 * 1e3, "fp64_ms": nrhs * t64 * 1e3, "fp64_inner_iters": i64.inner_iters,
                      "fp64_true_rel_residual": i64.true_rel_residual,
                      "speedup": nrhs * t64 * 1e3 / (ms / args.steps)})

    # ---- end to end through bridge_solve with pinned host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, h, op, solver, b_dev, b_host, nrhs, total_bytes, world)

    # ---- serving sample
    # ---- serving sample
    serving = None
    if args.serving_requests > 0 and rank == 0 and nrhs == 1:
        serving = serving_sample(api, args.serving_requests, {"dims": w.dims, "L": L}, U)

    # ---- CPU oracle baseline (rank 0, N = 1)
    cpu = None
    if rank == 0 and world == 1:
        # the oracle's cost does not depend on the values: time it on a Gaussian spinor
        b_cpu = synth.gaussian_spinor(w.dims, w.seed) if b_host is None else (b_host[0] if b_host.ndim == 4 else b_host)
        v1, secs1, cores1 = oracle_sample(w, U, b_cpu, 4 * args.oracle_sites, seed=0)
        n_all = min(4 * args.oracle_sites * (os.cpu_count() or 1), int(np.prod(w.dims)))
        v, secs, cores = oracle_sample_pool(w, U, b_cpu, n_all, seed=1)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"FP64 numpy oracle: clover D at {n_all} random sites of the {args.workload} lattice, "
                         f"split over {cores} spawned processes ({secs:.1f} s)",
               "single_core": {"value": v1, "cores": cores1,
                               "sample": f"{4 * args.oracle_sites} random sites in one process ({secs1:.1f} s)"}}

    # ---- measured FMA peaks and the multi-RHS workload (default workload only)
    alu = alu_peaks(api) if rank == 0 else None
    multi = None
    if args.multi_rhs and args.workload == "clover_32x32x32x64" and args.multi_rhs != args.workload:
        multi = multi_rhs_leg(args, api, local, peaks()[0], alu)

    if rank == 0:
        sb = {"f32": 96, "f16": 52, "bf16": 52, "f64": 192}[inner]
        working_set = (4 * w.volume * sb / 2 + w.volume * sb * 1.5 + nrhs * (12 * w.volume / 2 * sb + 3 * w.volume * 192)) / 1e9
        line = {
            "metric": METRIC,
            "value": value,
            "unit": UNIT,
            "value_is": ("algorithmic HBM GB/s of one whole mixed-precision solve (every kernel of the step: "
                         "Schur hops, BiCGStab vectors, FP64 residual), inputs resident; the D_eo kernel alone is "
                         "deo.gbs, the dominant kernel's is roofline.achieved"),
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": f"{'f32' if inner == 'f32' else inner + ' storage, f32 math'}+f64",
            "data": "synthetic",
            "config": {
                "workload": args.workload,
                "lattice": "x".join(map(str, w.dims)),
                "operator": f"{kind}, kappa={w.kappa}, c_sw={w.csw}, bc={list(w.bc)}",
                "links": f"exp({w.eps} i A), seed {w.seed}",
                "source": w.source if nrhs == 1 else f"{nrhs} {w.source} sources",
                "nrhs": nrhs,
                "solver": f"even-odd BiCGStab, {inner} inner, f64 defect correction",
                "tol": w.tol,
                "l2": f"inputs larger than L2 (solve working set ~{working_set:.1f} GB)",
                "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
            },
            "roofline": roofline,
            "kernel_shares": shares,
            "launch_shapes": {k: {"block": v[0], "site_blocks": v[1], "variant": v[2]}
                              for k, v in api.bridge_tune_table(h).items() if k.startswith("hop/")},
            "deo": deo,
            "solve": solve,
            "multi_rhs": multi,
            "alu_peaks": alu,
            "serving": serving,
            "e2e": e2e,
            "gpu_launches": launches,
            "inner_iters": iters,
            "true_rel_residual": res,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    L.close()
    if world > 1:
        dist.destroy_process_group()


def mobius_oracle_sample(w, U, b, nsites, seed):
    """The FP64 oracle's Moebius D at random four-dimensional sites (all Ls slices)."""
    from oracle import domainwall
    from oracle.lattice import Lattice

    lat = Lattice(w.dims)
    orc = domainwall.Mobius(U, lat, w.Ls, w.M5, w.b5, w.c5, w.mf, w.bc)
    sites = np.sort(np.random.default_rng(seed).choice(lat.V, nsites, replace=False))
    _, secs, cores = cpu_cores_used(lambda: orc.full(b, sites=sites))
    # per five-dimensional site: spinor in (plus P psi), 8 links, spinor out
    per_site = 192 + 8 * 144 / w.Ls + 192
    return nsites * w.Ls * per_site / secs / 1e9, secs, cores


def mobius_operator_leg(api, h, op, w, b_dev, stream):
    """One Schur operator application, then D_eo (B mix + hop) alone on
    resident FP32 fields, timed with CUDA events on the library stream."""
    import torch

    peak, _ = peaks()
    nrhs = w.nrhs
    nq = nrhs * w.Ls
    fo = api.bridge_field_create(h, "f32", 1, nq)
    fe = api.bridge_field_create(h, "f32", 0, nq)
    fe2 = api.bridge_field_create(h, "f32", 0, nq)
    half = b_dev.reshape(nq, w.volume // 2, 2, 4, 3)
    par = torch.from_numpy(_parity_odd_index(w.dims)).to(b_dev.device)
    src_odd = torch.gather(half, 2, par.view(1, -1, 1, 1, 1).expand(nq, -1, 1, 4, 3)).squeeze(2).contiguous()
    api.bridge_field_import(fo, src_odd)
    del src_odd, half
    api.bridge_sync(h)
    api.bridge_apply(h, op, 1, fe, fo)  # D_oe: an even input for the Schur operator
    api.bridge_apply(h, op, 3, fe2, fe)  # D^ once (its kernels come first in a profiler capture)
    for _ in range(3):
        api.bridge_apply(h, op, 1, fe, fo)
    reps = 30
    api.bridge_stats_reset(h)
    api.bridge_profile(h, True)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(reps):
        api.bridge_apply(h, op, 1, fe, fo)
    a1.record(stream)
    torch.cuda.synchronize()
    api.bridge_profile(h, False)
    dst = api.bridge_stats(h)
    deo_ms = a0.elapsed_time(a1) / reps
    deo_bytes = (dst["dwf_hop"]["bytes"] + dst["dwf_mix"]["bytes"]) / reps
    hop = dst["dwf_hop"]
    out = {"ops": "B mix + hop", "prec": "f32", "slices": nq, "gbs": deo_bytes / (deo_ms * 1e-3) / 1e9,
           "us_per_apply": deo_ms * 1e3, "bytes_per_apply": deo_bytes, "frac": deo_bytes / (deo_ms * 1e-3) / 1e9 / peak,
           "hop_gbs": hop["bytes"] / (hop["ms"] * 1e-3) / 1e9, "hop_frac": hop["bytes"] / (hop["ms"] * 1e-3) / 1e9 / peak,
           "hop_us": 1e3 * hop["ms"] / reps, "hop_bytes": hop["bytes"] / reps,
           "hop_gflops": hop["flops"] / (hop["ms"] * 1e-3) / 1e9}
    for f in (fo, fe, fe2):
        api.bridge_field_destroy(f)
    return out


def run_mobius(args):
    """Moebius domain wall: mixed CG solve steps, D_eo alone, FP64 CG, e2e, oracle."""
    import torch

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__ as g

    if rank == 0:
        g.build()
    if world > 1:
        dist.barrier()
    from ctypes import byref, c_void_p

    import synth
    from paper_2303_05883_gb300 import _abi, api

    w = synth.WORKLOADS[args.workload]
    U = w.gauge()
    b_host = w.sources()  # (nrhs, Ls, V, 4, 3)
    b_dev = torch.from_numpy(b_host).to(f"cuda:{local}")
    x_dev = None if args.deo_only else torch.zeros_like(b_dev)
    op = api.make_mobius(w.Ls, w.M5, w.b5, w.c5, w.mf, bc=w.bc)
    L = api.Lattice(w.dims)
    L.upload(U)
    h = L.handle
    stream = L.stream
    solver = api.make_solver(tol=w.tol, inner_prec="f32", mixed=1)
    nrhs = w.nrhs
    api.bridge_tune(h, op, "f32", nrhs)
    if args.deo_only:
        torch.cuda.nvtx.range_push("operator_legs")
        leg = mobius_operator_leg(api, h, op, w, b_dev, stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"workload": args.workload, "deo": leg,
                          "launch_shapes": {k: {"threads": v[0], "variant": v[2]}
                                            for k, v in api.bridge_tune_table(h).items() if k.startswith("dwf")}}),
              flush=True)
        L.close()
        return

    def solve_dev(prm):
        x_dev.zero_()
        torch.cuda.current_stream().synchronize()
        info = (_abi.bridge_info * nrhs)()
        st = _abi.load().bridge_solve_dev(h, byref(op), byref(prm), c_void_p(b_dev.data_ptr()),
                                          c_void_p(x_dev.data_ptr()), nrhs, info)
        _abi.check(st, "bridge_solve_dev")
        return max((info[k] for k in range(nrhs)), key=lambda i: i.true_rel_residual)

    for _ in range(args.warmup):
        solve_dev(solver)
    torch.cuda.synchronize()
    api.bridge_stats_reset(h)
    l0 = api.bridge_launch_count()
    infos = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        torch.cuda.nvtx.range_push("timed_steps")
        e0.record(stream)
        for _ in range(args.steps):
            infos.append(solve_dev(solver))
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    ms = e0.elapsed_time(e1)
    launches = api.bridge_launch_count() - l0
    st = api.bridge_stats(h)
    total_bytes = sum(v["bytes"] for v in st.values())
    ms, total_bytes = aggregate_ranks(ms, total_bytes, device=f"cuda:{local}")
    value = total_bytes / (ms * 1e-3) / 1e9
    res = max(i.true_rel_residual for i in infos)
    iters = statistics.median(i.inner_iters for i in infos)
    outer = statistics.median(i.outer_iters for i in infos)

    # ---- one event-profiled step
    api.bridge_stats_reset(h)
    api.bridge_profile(h, True)
    solve_dev(solver)
    torch.cuda.synchronize()
    api.bridge_profile(h, False)
    pst = api.bridge_stats(h)
    step_ms_prof = sum(v["ms"] for v in pst.values())
    dom = max(pst, key=lambda k: pst[k]["ms"])
    d = pst[dom]
    peak, peak_kind = peaks()
    achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9
    roofline = {
        "bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "peak_source": peak_kind, "unit": "GB/s",
        "frac": achieved / peak, "traffic": traffic_for(dom, args.workload),
        "algorithmic_bytes_per_launch": d["bytes"] / max(1, d["launches"]), "launches": d["launches"],
        "avg_launch_us": 1e3 * d["ms"] / max(1, d["launches"]),
        "share_of_step": d["ms"] / step_ms_prof if step_ms_prof else None,
    }
    shares = {k: round(v["ms"] / step_ms_prof, 4) for k, v in pst.items() if v["ms"] > 0}
    per_kernel = {k: {"launches": v["launches"], "gbs": v["bytes"] / (v["ms"] * 1e-3) / 1e9,
                      "tflops": v["flops"] / (v["ms"] * 1e-3) / 1e12}
                  for k, v in pst.items() if v["ms"] > 0}

    deo = mobius_operator_leg(api, h, op, w, b_dev, stream)
    peak, peak_kind = peaks()

    solve = {"mixed_ms": ms / args.steps, "mixed_cg_iters": iters, "mixed_outer": outer,
             "mixed_true_rel_residual": res, "inner_prec": "f32"}
    if not args.no_fp64:
        s64 = api.make_solver(tol=w.tol, mixed=0, max_iter=100000)
        t0 = time.perf_counter()
        i64 = solve_dev(s64)
        t64 = time.perf_counter() - t0
        solve.update({"fp64_ms": t64 * 1e3, "fp64_cg_iters": i64.inner_iters,
                      "fp64_true_rel_residual": i64.true_rel_residual, "speedup": t64 * 1e3 / (ms / args.steps)})

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, h, op, solver, b_dev, b_host, nrhs, total_bytes, world)

    cpu = None
    if rank == 0 and world == 1:
        n = max(16, args.oracle_sites // 64)
        v, secs, cores = mobius_oracle_sample(w, U, b_host[0], n, seed=0)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"FP64 numpy oracle: Moebius D at {n} random four-dimensional sites x Ls = {w.Ls} of the "
                         f"{args.workload} lattice ({secs:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {
                "workload": args.workload, "lattice": "x".join(map(str, w.dims)) + f"x{w.Ls}",
                "operator": f"Moebius domain wall, M5={w.M5}, b={w.b5}, c={w.c5}, m_f={w.mf}, bc={list(w.bc)}",
                "links": f"exp({w.eps} i A), seed {w.seed}", "source": "gaussian", "nrhs": nrhs,
                "solver": "even-odd CG on the normal equations, f32 inner, f64 defect correction", "tol": w.tol,
                "l2": "inputs larger than L2 (one five-dimensional FP32 field is 1 GB)",
                "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
            },
            "roofline": roofline, "kernel_shares": shares, "per_kernel": per_kernel, "deo": deo, "solve": solve,
            "launch_shapes": {k: {"threads": v[0], "variant": v[2]}
                              for k, v in api.bridge_tune_table(h).items() if k.startswith("dwf")},
            "e2e": e2e, "gpu_launches": launches, "inner_iters": iters, "true_rel_residual": res,
            "clocks": clk.summary(), "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    L.close()
    if world > 1:
        dist.destroy_process_group()


def staggered_oracle_sample(w, U, b, nsites, seed):
    """The FP64 oracle's staggered D at random sites."""
    from oracle import staggered
    from oracle.lattice import Lattice

    lat = Lattice(w.dims)
    orc = staggered.Staggered(U, lat, w.mass, w.bc)
    sites = np.sort(np.random.default_rng(seed).choice(lat.V, nsites, replace=False))
    _, secs, cores = cpu_cores_used(lambda: orc.full(b, sites=sites))
    per_site = 48 + 8 * 144 + 48  # vector in, 8 links, vector out (FP64)
    return nsites * per_site / secs / 1e9, secs, cores


def staggered_operator_leg(api, h, op, w, b_dev):
    """One Schur operator application (its two hop passes come first in a
    profiler capture), then D_eo alone: the hop kernel's event-timed
    launches inside bridge_mult_Deo_dev."""
    from ctypes import byref, c_void_p

    import torch

    from paper_2303_05883_gb300 import _abi

    peak, _ = peaks()
    nrhs = w.nrhs
    lib = _abi.load()
    half = torch.zeros((nrhs, w.volume // 2, 3), dtype=torch.complex128, device=b_dev.device)
    half.real.normal_()
    out = torch.empty_like(half)
    f32 = _abi.BRIDGE_F32
    _abi.check(lib.bridge_mult_Dhat_dev(h, byref(op), f32, c_void_p(half.data_ptr()), c_void_p(out.data_ptr()), nrhs),
               "bridge_mult_Dhat_dev")
    for _ in range(2):
        _abi.check(lib.bridge_mult_Deo_dev(h, byref(op), f32, 0, c_void_p(half.data_ptr()), c_void_p(out.data_ptr()),
                                           nrhs), "bridge_mult_Deo_dev")
    api.bridge_sync(h)
    api.bridge_stats_reset(h)
    api.bridge_profile(h, True)
    reps = 20
    for _ in range(reps):
        _abi.check(lib.bridge_mult_Deo_dev(h, byref(op), f32, 0, c_void_p(half.data_ptr()), c_void_p(out.data_ptr()),
                                           nrhs), "bridge_mult_Deo_dev")
    api.bridge_sync(h)
    api.bridge_profile(h, False)
    hop = api.bridge_stats(h)["stag_hop"]
    return {"kernel": "stag_hop", "prec": "f32", "gbs": hop["bytes"] / (hop["ms"] * 1e-3) / 1e9,
            "frac": hop["bytes"] / (hop["ms"] * 1e-3) / 1e9 / peak, "us_per_launch": 1e3 * hop["ms"] / reps,
            "bytes_per_launch": hop["bytes"] / reps, "gflops": hop["flops"] / (hop["ms"] * 1e-3) / 1e9}


def run_staggered(args):
    """Staggered: mixed CG solve steps, D_eo alone, FP64 CG, e2e, oracle."""
    import torch

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__ as g

    if rank == 0:
        g.build()
    if world > 1:
        dist.barrier()
    from ctypes import byref, c_void_p

    import synth
    from paper_2303_05883_gb300 import _abi, api

    w = synth.WORKLOADS[args.workload]
    U = w.gauge()
    b_host = w.sources()  # (nrhs, V, 3)
    b_dev = torch.from_numpy(b_host).to(f"cuda:{local}")
    x_dev = torch.zeros_like(b_dev)
    op = api.make_staggered(w.mass, bc=w.bc)
    L = api.Lattice(w.dims)
    L.upload(U)
    h = L.handle
    stream = L.stream
    nrhs = w.nrhs
    solver = api.make_solver(tol=w.tol, inner_prec=w.inner, mixed=1)
    peak, peak_kind = peaks()
    if args.deo_only:
        torch.cuda.nvtx.range_push("operator_legs")
        leg = staggered_operator_leg(api, h, op, w, b_dev)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"workload": args.workload, "deo": leg}), flush=True)
        L.close()
        return

    def solve_dev(prm):
        x_dev.zero_()
        torch.cuda.current_stream().synchronize()
        info = (_abi.bridge_info * nrhs)()
        st = _abi.load().bridge_solve_dev(h, byref(op), byref(prm), c_void_p(b_dev.data_ptr()),
                                          c_void_p(x_dev.data_ptr()), nrhs, info)
        _abi.check(st, "bridge_solve_dev")
        return max((info[k] for k in range(nrhs)), key=lambda i: i.true_rel_residual)

    for _ in range(args.warmup):
        solve_dev(solver)
    torch.cuda.synchronize()
    api.bridge_stats_reset(h)
    l0 = api.bridge_launch_count()
    infos = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        torch.cuda.nvtx.range_push("timed_steps")
        e0.record(stream)
        for _ in range(args.steps):
            infos.append(solve_dev(solver))
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    ms = e0.elapsed_time(e1)
    launches = api.bridge_launch_count() - l0
    st = api.bridge_stats(h)
    total_bytes = sum(v["bytes"] for v in st.values())
    ms, total_bytes = aggregate_ranks(ms, total_bytes, device=f"cuda:{local}")
    value = total_bytes / (ms * 1e-3) / 1e9
    res = max(i.true_rel_residual for i in infos)
    iters = statistics.median(i.inner_iters for i in infos)
    outer = statistics.median(i.outer_iters for i in infos)

    # ---- one event-profiled step
    api.bridge_stats_reset(h)
    api.bridge_profile(h, True)
    solve_dev(solver)
    torch.cuda.synchronize()
    api.bridge_profile(h, False)
    pst = api.bridge_stats(h)
    step_ms_prof = sum(v["ms"] for v in pst.values())
    dom = max(pst, key=lambda k: pst[k]["ms"])
    d = pst[dom]
    achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9
    roofline = {
        "bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "peak_source": peak_kind, "unit": "GB/s",
        "frac": achieved / peak, "traffic": traffic_for(dom, args.workload),
        "algorithmic_bytes_per_launch": d["bytes"] / max(1, d["launches"]), "launches": d["launches"],
        "avg_launch_us": 1e3 * d["ms"] / max(1, d["launches"]),
        "share_of_step": d["ms"] / step_ms_prof if step_ms_prof else None,
    }
    shares = {k: round(v["ms"] / step_ms_prof, 4) for k, v in pst.items() if v["ms"] > 0}
    per_kernel = {k: {"launches": v["launches"], "gbs": v["bytes"] / (v["ms"] * 1e-3) / 1e9,
                      "tflops": v["flops"] / (v["ms"] * 1e-3) / 1e12}
                  for k, v in pst.items() if v["ms"] > 0}

    deo = staggered_operator_leg(api, h, op, w, b_dev)

    solve = {"mixed_ms": ms / args.steps, "mixed_cg_iters": iters, "mixed_outer": outer,
             "mixed_true_rel_residual": res, "inner_prec": w.inner}
    if not args.no_fp64:
        s64 = api.make_solver(tol=w.tol, mixed=0, max_iter=100000)
        t0 = time.perf_counter()
        i64 = solve_dev(s64)
        t64 = time.perf_counter() - t0
        solve.update({"fp64_ms": t64 * 1e3, "fp64_cg_iters": i64.inner_iters,
                      "fp64_true_rel_residual": i64.true_rel_residual, "speedup": t64 * 1e3 / (ms / args.steps)})

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, h, op, solver, b_dev, b_host, nrhs, total_bytes, world)

    cpu = None
    if rank == 0 and world == 1:
        n = args.oracle_sites * 4
        v, secs, cores = staggered_oracle_sample(w, U, b_host[0], n, seed=0)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"FP64 numpy oracle: staggered D at {n} random sites of the {args.workload} lattice "
                         f"({secs:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {
                "workload": args.workload, "lattice": "x".join(map(str, w.dims)),
                "operator": f"staggered, m={w.mass}, bc={list(w.bc)}", "links": f"exp({w.eps} i A), seed {w.seed}",
                "source": "gaussian", "nrhs": nrhs,
                "solver": "even-odd CG (m^2 - D_eo D_oe), f32 inner, f64 defect correction", "tol": w.tol,
                "l2": "inputs larger than L2 (FP32 links 3.2 GB)",
                "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
            },
            "roofline": roofline, "kernel_shares": shares, "per_kernel": per_kernel, "deo": deo, "solve": solve,
            "e2e": e2e, "gpu_launches": launches, "inner_iters": iters, "true_rel_residual": res,
            "clocks": clk.summary(), "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    L.close()
    if world > 1:
        dist.destroy_process_group()


MG_PARAMS = dict(nvec=12, setup_steps=3, sap_cycles=2, mr_steps=6, coarse_tol=1e-1)


def run_mg(args):
    """Two-level multigrid (FBiCGStab + SAP + coarse BiCGStab) on the 32^3x64
    clover field near its critical kappa: setup, solve steps, the mixed
    BiCGStab on the same system, 1 and 12 equations including setup."""
    import torch

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__ as g

    if rank == 0:
        g.build()
    if world > 1:
        dist.barrier()
    from ctypes import byref, c_void_p

    import synth
    from paper_2303_05883_gb300 import _abi, api

    w = synth.WORKLOADS[args.workload]
    U = w.gauge()
    b_host = w.sources()[0]
    b_dev = torch.from_numpy(b_host).to(f"cuda:{local}")
    x_dev = torch.zeros_like(b_dev)
    op = api.make_op("clover", w.kappa, w.csw, w.bc)
    L = api.Lattice(w.dims)
    L.upload(U, op)
    h = L.handle
    stream = L.stream
    lib = _abi.load()
    peak, peak_kind = peaks()
    solver = api.make_solver(tol=w.tol, max_iter=1000)
    t0 = time.perf_counter()
    mg = api.Multigrid(L, op, api.make_mg_params(**MG_PARAMS))
    setup_s = time.perf_counter() - t0

    def mg_solve():
        x_dev.zero_()
        torch.cuda.current_stream().synchronize()
        info = (_abi.bridge_info * 1)()
        _abi.check(lib.bridge_mg_solve_dev(mg.handle, byref(solver), c_void_p(b_dev.data_ptr()),
                                           c_void_p(x_dev.data_ptr()), 1, info), "bridge_mg_solve_dev")
        return info[0]

    for _ in range(args.warmup):
        mg_solve()
    torch.cuda.synchronize()
    api.bridge_stats_reset(h)
    l0 = api.bridge_launch_count()
    c0 = mg.counters()
    infos, host_s = [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        torch.cuda.nvtx.range_push("timed_steps")
        e0.record(stream)
        for _ in range(args.steps):
            t1 = time.perf_counter()
            infos.append(mg_solve())
            host_s.append(time.perf_counter() - t1)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    ms = e0.elapsed_time(e1)
    launches = api.bridge_launch_count() - l0
    c1 = mg.counters()
    st = api.bridge_stats(h)
    total_bytes = sum(v["bytes"] for v in st.values())
    ms, total_bytes = aggregate_ranks(ms, total_bytes, device=f"cuda:{local}")
    value = total_bytes / (ms * 1e-3) / 1e9
    res = max(i.true_rel_residual for i in infos)

    # ---- one event-profiled solve
    api.bridge_stats_reset(h)
    api.bridge_profile(h, True)
    mg_solve()
    torch.cuda.synchronize()
    api.bridge_profile(h, False)
    pst = api.bridge_stats(h)
    step_ms_prof = sum(v["ms"] for v in pst.values())
    dom = max(pst, key=lambda k: pst[k]["ms"])
    d = pst[dom]
    achieved = d["bytes"] / (d["ms"] * 1e-3) / 1e9
    roofline = {
        "bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "peak_source": peak_kind, "unit": "GB/s",
        "frac": achieved / peak, "traffic": traffic_for(dom, args.workload),
        "algorithmic_bytes_per_launch": d["bytes"] / max(1, d["launches"]), "launches": d["launches"],
        "avg_launch_us": 1e3 * d["ms"] / max(1, d["launches"]),
        "share_of_step": d["ms"] / step_ms_prof if step_ms_prof else None,
    }
    shares = {k: round(v["ms"] / step_ms_prof, 4) for k, v in pst.items() if v["ms"] > 0}
    per_kernel = {k: {"launches": v["launches"], "gbs": v["bytes"] / (v["ms"] * 1e-3) / 1e9}
                  for k, v in pst.items() if v["ms"] > 0}

    # ---- the mixed BiCGStab on the same system (the paper's comparison)
    mixed = api.make_solver(tol=w.tol, inner_prec="f32", max_iter=20000)
    for _ in range(2):
        x_dev.zero_()
        torch.cuda.synchronize()
        info = (_abi.bridge_info * 1)()
        t1 = time.perf_counter()
        _abi.check(lib.bridge_solve_dev(h, byref(op), byref(mixed), c_void_p(b_dev.data_ptr()),
                                        c_void_p(x_dev.data_ptr()), 1, info), "bridge_solve_dev")
        bicg_s = time.perf_counter() - t1
    mg_s = statistics.median(host_s)
    solve = {
        "mg_setup_s": setup_s, "mg_solve_ms": ms / args.steps, "mg_outer_passes": statistics.median(i.outer_iters for i in infos),
        "mg_fbicgstab_iters": statistics.median(i.inner_iters for i in infos),
        "coarse_iters_per_solve": (c1[1] - c0[1]) / max(1, c1[0] - c0[0]),
        "mg_true_rel_residual": res, "bicgstab_ms": bicg_s * 1e3, "bicgstab_iters": info[0].inner_iters,
        "speedup_1_solve_excl_setup": bicg_s / mg_s,
        "one_equation_s": {"mg_incl_setup": setup_s + mg_s, "bicgstab": bicg_s},
        "twelve_equations_s": {"mg_incl_setup": setup_s + 12 * mg_s, "bicgstab": 12 * bicg_s},
        "params": MG_PARAMS,
    }

    # ---- end to end through bridge_mg_solve with pinned host buffers
    e2e = None
    if not args.no_e2e:
        b_pin = torch.from_numpy(b_host).pin_memory()
        x_pin = torch.zeros_like(b_pin).pin_memory()
        import ctypes

        dp = ctypes.POINTER(ctypes.c_double)
        bp, xp = ctypes.cast(b_pin.data_ptr(), dp), ctypes.cast(x_pin.data_ptr(), dp)
        ts = []
        for _ in range(args.steps):
            x_pin.zero_()
            info = (_abi.bridge_info * 1)()
            t1 = time.perf_counter()
            _abi.check(lib.bridge_mg_solve(mg.handle, byref(solver), bp, xp, 1, info), "bridge_mg_solve")
            ts.append(time.perf_counter() - t1)
        e2e = {"value": (total_bytes / args.steps) / statistics.median(ts) / 1e9 if world == 1 else None,
               "unit": UNIT, "h2d_bytes_per_step": 2 * b_host.nbytes, "d2h_bytes_per_step": b_host.nbytes,
               "ms_per_step": 1e3 * statistics.median(ts)}

    cpu = None
    if rank == 0 and world == 1:
        v, secs, cores = oracle_sample(w, U, b_host, 4 * args.oracle_sites, seed=0)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"FP64 numpy oracle: clover D at {4 * args.oracle_sites} random sites of the {args.workload} "
                         f"lattice ({secs:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f16 coarse+f64", "data": "synthetic",
            "config": {
                "workload": args.workload, "lattice": "x".join(map(str, w.dims)),
                "operator": f"clover, kappa={w.kappa}, c_sw={w.csw}, bc={list(w.bc)}",
                "links": f"exp({w.eps} i A), seed {w.seed}", "source": "gaussian", "nrhs": 1,
                "solver": "two-level multigrid: FBiCGStab (f32 passes, f64 defect correction), SAP smoother, "
                          "coarse BiCGStab; blocks 4^4",
                "tol": w.tol, "l2": "inputs larger than L2",
                "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
            },
            "roofline": roofline, "kernel_shares": shares, "per_kernel": per_kernel, "solve": solve, "e2e": e2e,
            "gpu_launches": launches, "true_rel_residual": res, "clocks": clk.summary(), "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    mg.close()
    L.close()
    if world > 1:
        dist.destroy_process_group()


def run_dd(args):
    """The decomposed Schur operator (slabs along t joined by a halo exchange)
    against the single-lattice one on the 32^3 x 64 clover workload, through
    the device-pointer entry points (canonical FP64 in and out, so the layout
    conversions are inside both timings), for 1, 2, 4 and 8 slabs; and the
    decomposed FP64 BiCGStab solve beside the plain FP64 one."""
    import torch

    torch.cuda.set_device(0)
    import __graft_entry__ as g

    g.build()
    import synth
    from paper_2303_05883_gb300 import _abi, api

    w = synth.WORKLOADS["clover_32x32x32x64"]
    op = api.make_op("clover", w.kappa, w.csw, w.bc)
    L = api.Lattice(w.dims)
    L.upload(w.gauge(), op)
    gen = torch.Generator(device="cuda").manual_seed(11)
    xe = torch.randn((w.volume // 2, 4, 3), dtype=torch.complex128, device="cuda", generator=gen)
    reps = max(3, args.steps)

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return 1e3 * (time.perf_counter() - t0) / reps

    out = {"plain": {}}
    for prec in ("f32", "f16"):
        out["plain"][prec] = timed(lambda: L.Dhat(op, xe, prec))
    ref = L.Dhat(op, xe, "f32")
    for n in (1, 2, 4, 8):
        dd = api.Decomposition(L, op, n)
        e = {prec: timed(lambda: dd.Dhat(xe, prec)) for prec in ("f32", "f16")}
        got = dd.Dhat(xe, "f32")
        e["rel_diff_f32"] = float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref))
        out[f"slabs_{n}"] = e
        dd.close()
    b = torch.from_numpy(w.sources()[0]).cuda()
    s64 = api.make_solver(tol=w.tol, mixed=0)
    t0 = time.perf_counter()
    _, info = L.solve(op, b, s64)
    t_plain = time.perf_counter() - t0
    dd = api.Decomposition(L, op, 4)
    t0 = time.perf_counter()
    _, dinfo = dd.solve(b, api.make_solver(tol=w.tol))
    t_dd = time.perf_counter() - t0
    dd.close()
    L.close()
    line = {
        "metric": "decomposed Schur operator and FP64 solve time (halo exchange between slabs on one GPU)",
        "value": out["slabs_4"]["f32"], "unit": "ms per D^ application (4 slabs, f32, canonical FP64 in/out)",
        "n_gpus": 1, "steps": reps, "warmup": 2, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 / f16 storage, f32 math; f64 solve", "data": "synthetic",
        "config": {"workload": "dd_clover_32x32x32x64", "lattice": "x".join(map(str, w.dims)),
                   "decomposition": "slabs along t", "transport": "device-to-device copies on one GPU"},
        "dhat_ms": out,
        "fp64_solve": {"plain_s": t_plain, "plain_iters": info[0]["inner_iters"],
                       "decomposed_4_slabs_s": t_dd, "decomposed_iters": dinfo[0]["inner_iters"],
                       "decomposed_true_rel_residual": dinfo[0]["true_rel_residual"]},
    }
    print(json.dumps(line), flush=True)


def run_serving(args):
    """The request stream alone: lattices {8^4, 16^4, 24^3x48, 32^3x64},
    kappa in [0.11, 0.13], 1-12 right-hand sides, Wilson or clover."""
    import torch

    torch.cuda.set_device(0)
    import __graft_entry__ as g

    g.build()
    import synth
    from paper_2303_05883_gb300 import api

    w = synth.WORKLOADS["clover_32x32x32x64"]
    L = api.Lattice(w.dims)
    U = w.gauge()
    L.upload(U)
    out = {}
    for f in args.rate_factors:
        out[str(f)] = serving_sample(api, args.serving_requests, {"dims": w.dims, "L": L}, U, rate_factor=f)
    L.close()
    first = out[str(args.rate_factors[0])]
    line = {
        "metric": METRIC,
        "value": first["p99_ms"],
        "unit": "ms (p99 latency)",
        "n_gpus": 1,
        "steps": args.serving_requests,
        "warmup": 0,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": "serving", "requests": args.serving_requests, "rate_factors": args.rate_factors},
        "serving": out,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload.startswith("mobius"):
        run_mobius(args)
    elif args.workload.startswith("staggered"):
        run_staggered(args)
    elif args.workload.startswith("mg_"):
        run_mg(args)
    elif args.workload.startswith("dd_"):
        run_dd(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
