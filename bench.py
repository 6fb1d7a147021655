#!/usr/bin/env python
"""Projection solves/s at 256^3, density ratio 1000, relative residual 1e-10:
mixed FP32/FP64 form vs plain FP64 form, with the HBM roofline fraction of the
dominant kernel.

One step = one whole projection (face coefficients from C, divergence of u*,
multigrid-preconditioned Poisson solve to 1e-10 in the L2 and L-infinity norms,
velocity correction) of the 256^3 drop field: 64 drops, periodic x/y, walls
in z, rho1/rho2 = 1000, dt = 1e-4, seeded synthetic input.  Every timed step
projects its own device-resident copy of u*, v*, w* from a zero initial
pressure; those copies are made before the timed region, which holds the
projection steps alone.  Each step reads more than the 129 MB L2 (C plus u*,
v*, w*, p: 671 MB), so no flush is needed.  Each step is bracketed by its own
CUDA event pair on the launching stream: value = steps / summed step time,
and the median, p10 and p90 of the step times are reported beside it.  Every
timed step must converge, or the run fails.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl paris|reference]
       python bench.py --jet | --adjoint | --viscous   (other workloads, one line each)
Multi-GPU (torchrun): every rank runs an independent replica ("replicas
only": one projection does not shard here), value = all ranks' solves / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# implicit viscous step of `--viscous`: mu of fluid 1 / fluid 2, and tau = this
# factor times h^2 / max nu_f
VISC_MU = (1.0e-3, 1.8e-5)
VISC_TAU_NU_OVER_H2 = 4.0

METRIC = "Projection solves/s at 256³, ρ ratio 1000, resid 1e-10: mixed vs FP64; % HBM"
UNIT = "solves/s"
STREAM_FLOATS = 1 << 27  # FP32 elements per vector of the streaming-rate probe (512 MB)

# DRAM bytes (read + write) per launch of the dominant kernel class, from one
# ncu capture of "python bench.py --single mixed", valid while the source file
# holding that kernel is unchanged (sha256 prefix); otherwise traffic is null.
NCU_TRAFFIC = {
    # finest-level colour pass: DRAM read + write bytes per launch from
    # "ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum
    #  -k regex:rbgs_rho_tile|... -c 60" of "bench.py --single mixed" (caches flushed
    # between launches): zero-initial passes 72.6 MB, the passes after them 113.5 MB,
    # the others 147.7 MB (rho/2 in FP16, two planes per block); 11, 11 and 66 per solve
    "smooth0": {"bytes_per_launch": 134.1e6, "source": "rho0.cu", "sha": "08c283ebe42f14f7"},
}


def kernel_source_sha(name: str) -> str:
    p = os.path.join(ROOT, "paper_2012_11744_gb300", "csrc", name)
    with open(p, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine() or "unknown"


def oracle_threads() -> int:
    """Threads the oracle's OpenMP loops run on (OMP_NUM_THREADS, else every core)."""
    try:
        return int(os.environ["OMP_NUM_THREADS"])
    except (KeyError, ValueError):
        return os.cpu_count() or 1


def step_stats(ms_list):
    """Median, p10 and p90 of per-step times (ms), nearest-rank percentiles."""
    a = sorted(ms_list)
    pick = lambda q: a[min(len(a) - 1, max(0, int(round(q * (len(a) - 1)))))]
    return {"median": statistics.median(a), "p10": pick(0.1), "p90": pick(0.9), "n": len(a)}


def require_converged(stats, what):
    bad = [i for i, s in enumerate(stats) if s.get("converged") != 1]
    if bad:
        raise RuntimeError(f"{what}: timed steps {bad} did not converge: {[stats[i] for i in bad]}")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.fh = None

    def __enter__(self):
        try:
            self.fh = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.fh is None:
            return None
        try:
            with open(self.fh.name) as fh:
                rows = [r.strip().split(",") for r in fh if r.strip()]
            os.unlink(self.fh.name)
        except Exception:
            return None
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
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if n_gpus > 0 else "gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------- CPU oracle ---

def oracle_sample(pr, budget_s: float, golden: dict | None):
    """Time the oracle (as it stands) on a bounded sample of the 256^3 solve:
    the full set-up (face coefficients, divergence, CSR assembly) plus CG
    iterations for about `budget_s` seconds; extrapolate to the CG iteration
    count of the full oracle solve (stored by tests/golden/make_drops256_golden.py)."""
    import oracle
    g = pr.grid
    if golden is None and g.ncells > SMALL_CELLS:
        raise FileNotFoundError(f"no stored oracle solve for {g.nx}x{g.ny}x{g.nz}")
    t0 = time.perf_counter()
    beta = oracle.face_coeffs(g, pr.C, pr.rho1, pr.rho2)
    b = oracle.divergence(g, pr.u, pr.v, pr.w, pr.dt)
    b0 = oracle.remove_mean(b)
    op = oracle.Operator(g, *beta)
    t1 = time.perf_counter()
    m = 10
    res = oracle.cg(op, -b0, tol=1e-300, max_iter=m, check=10 ** 9)
    t2 = time.perf_counter()
    per_it = (t2 - t1) / m
    m2 = max(10, int(budget_s / max(per_it, 1e-6)))
    t3 = time.perf_counter()
    res = oracle.cg(op, -b0, tol=1e-300, max_iter=m2, check=50)
    t4 = time.perf_counter()
    per_it = (t4 - t3) / max(res.iters, 1)
    if golden is not None:
        n_full = int(golden["oracle"]["cg_iters"])
    else:  # no stored full solve: small grids only, whose full solve is measured here
        if g.ncells > SMALL_CELLS:
            raise FileNotFoundError(f"no stored oracle solve for {g.nx}x{g.ny}x{g.nz}")
        n_full = oracle.cg(op, -b0, tol=1e-13).iters
    proj = oracle.project(g, *beta, res.x, pr.dt, pr.u, pr.v, pr.w)  # noqa: F841 (timed below)
    t5 = time.perf_counter()
    setup = (t1 - t0) + (t5 - t4)
    solve_s = setup + per_it * n_full
    return {"solve_s": solve_s, "setup_s": setup, "s_per_cg_iter": per_it, "cg_iters_sampled": res.iters,
            "cg_iters_full": n_full, "sample_s": t5 - t0}


def viscous_oracle_sample(pr, budget_s: float, golden: dict | None):
    """Time the viscous oracle (as it stands) on a bounded sample of the step
    `run_viscous` times: face viscosities of the three components, then
    oracle solves of the w component cut short after 1, 5 and m2 CG
    iterations (each assembles its operator; m2 sized from the first two so
    that the last one iterates for about `budget_s`).  The difference of the
    first and last gives the time of one iteration, the rest the set-up;
    extrapolated to the three components' iteration counts of the full oracle
    solves (stored by tests/golden/make_viscous256_golden.py)."""
    from oracle import viscous as V
    g = pr.grid
    if golden is None and g.ncells > SMALL_CELLS:
        raise FileNotFoundError(f"no stored viscous oracle solves for {g.nx}x{g.ny}x{g.nz}")
    t0 = time.perf_counter()
    nus = [V.face_nu(g, c, pr.C, VISC_MU[0], VISC_MU[1], pr.rho1, pr.rho2) for c in range(3)]
    tau = VISC_TAU_NU_OVER_H2 * g.h ** 2 / max(float(nu.max()) for nu in nus)
    t1 = time.perf_counter()
    un = V.interior(g, 2, pr.w)

    def cut(m):
        t = time.perf_counter()
        try:
            V.solve(g, 2, nus[2], tau, un, tol=1e-300, max_iter=m)
        except RuntimeError:  # stopped after m iterations, as intended
            pass
        return time.perf_counter() - t

    m1 = 1
    s1 = cut(m1)
    rough = max(cut(m1 + 4) - s1, 1e-6) / 4  # a first estimate of one iteration's time
    m2 = m1 + max(8, int(budget_s / rough))
    s2 = cut(m2)
    per_it = max(s2 - s1, 0.0) / (m2 - m1)
    setup = max(s1 - m1 * per_it, 0.0)
    if golden is not None:
        iters = [int(c["iters"]) for c in golden["components"]]
    else:  # no stored full solves: small grids only, whose full solves are counted here
        if g.ncells > SMALL_CELLS:
            raise FileNotFoundError(f"no stored viscous oracle solves for {g.nx}x{g.ny}x{g.nz}")
        iters = []
        for c in range(3):
            st = {}
            V.solve(g, c, nus[c], tau, V.interior(g, c, (pr.u, pr.v, pr.w)[c]), tol=1e-13, stats=st)
            iters.append(int(st["iters"]))
    step_s = (t1 - t0) + sum(setup + per_it * k for k in iters)
    return {"step_s": step_s, "setup_s": setup, "s_per_cg_iter": per_it, "cg_iters_sampled": [m1, m2],
            "cg_iters_full": iters, "sample_s": time.perf_counter() - t0}


def load_visc_golden(n):
    p = os.path.join(ROOT, "tests", "golden", f"viscous{n}_drops.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh)
    return None


SMALL_CELLS = 64 ** 3  # grids whose full oracle solve is cheap enough to run in a CPU-baseline sample


def load_golden(name, required=True):
    """A stored oracle solve (tests/golden/<name>.json), whose iteration count
    the CPU baseline extrapolates to.  Missing: an error when required, else
    None (the sample then solves small grids in full to count)."""
    p = os.path.join(ROOT, "tests", "golden", f"{name}.json")
    if not os.path.exists(p):
        if required:
            raise FileNotFoundError(f"{p} is missing: run tests/golden/make_*_golden.py first")
        return None
    with open(p) as fh:
        return json.load(fh)


def run_reference(args, rank, world):
    """--impl reference: the FP64 CPU oracle on the host cores, same metric."""
    if rank != 0:
        return
    import paris_inputs as pi
    pr = pi.config2(n=args.n)
    golden = load_golden(f"drops{args.n}_walls_z", required=args.n > 64)
    cores = oracle_threads()
    for _ in range(args.warmup):
        oracle_sample(pr, 0.5, golden)
    samples = [oracle_sample(pr, args.ref_budget, golden) for _ in range(args.steps)]
    total = sum(s["solve_s"] for s in samples)
    value = args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(args.n),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "cpu_model": cpu_model(), "kind": "oracle",
                         "sample": f"per step: oracle set-up + ~{args.ref_budget:.0f} s of CG iterations "
                                   f"on the {args.n}^3 system, extrapolated to the "
                                   f"{samples[0]['cg_iters_full']} iterations of the full oracle solve"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(n):
    return {"workload": f"drops{n}_walls_z: {n}^3 unit box, periodic x/y, walls z, 64 drops, "
                        f"rho 1000/1, dt 1e-4, tol 1e-10 (L2 and Linf)",
            "grid": [n, n, n], "precision": "mixed FP32 V-cycles in FP64 refinement (value) vs FP64",
            "l2": "no flush: each step projects its own copies of u*,v*,w* and p and reads C (5 x 134 MB > 129 MB L2)",
            "parallelism": "replicas"}


# ---------------------------------------------------------------- GPU arm ---

def run_paris(args, rank, world, local):
    import torch

    import paper_2012_11744_gb300 as paris
    from paper_2012_11744_gb300 import api
    import paris_inputs as pi

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    pr = pi.config2(n=args.n)
    g = pr.grid
    N = g.ncells
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    C = d(pr.C)
    u0, v0, w0 = d(pr.u), d(pr.v), d(pr.w)
    stream = torch.cuda.current_stream(dev)
    # every timed step projects its own copy of u*, v*, w* from a zero initial
    # pressure (the step corrects them in place): the copies are made before
    # the timed region, which then holds the projection steps alone
    nsets = max(args.steps, 1)
    sets = [(u0.clone(), v0.clone(), w0.clone(), torch.zeros(g.shape, dtype=torch.float64, device=dev))
            for _ in range(nsets)]

    def refill(K):
        for (u, v, w, p) in sets[:K]:
            u.copy_(u0)
            v.copy_(v0)
            w.copy_(w0)
            p.zero_()

    def timed(ctx, K, W, prof=False):
        """K projection steps, each between its own event pair on the
        launching stream; returns the summed ms, the per-step ms, the stats,
        the library's launches and (prof) the kernel-class profile."""
        for _ in range(W):
            refill(1)
            st = ctx.projection_step(C, pr.rho1, pr.rho2, pr.dt, *sets[0])
        refill(K)
        barrier(world)
        torch.cuda.synchronize(dev)
        if prof:
            ctx.profile(True)
        l0 = api.launch_count()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        sts = []
        for i in range(K):
            ev[i][0].record(stream)
            sts.append(ctx.projection_step(C, pr.rho1, pr.rho2, pr.dt, *sets[i]))
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        launches = api.launch_count() - l0
        per = [a.elapsed_time(b) for a, b in ev]
        prof_d = ctx.profile_read() if prof else None
        if prof:
            ctx.profile(False)
        return sum(per), per, sts, launches, prof_d

    hbm, peak_kind = measured_peaks()
    # mixed precision (headline)
    ctx = paris.Context(g, opts=paris.default_opts(precision=paris.MIXED), device=dev)
    with ClockSampler(local) as clk:
        ms_mixed, per_mixed, st_mixed, launches, _ = timed(ctx, args.steps, args.warmup)
    clocks = clk.summary()
    require_converged(st_mixed, "mixed")
    ms_mixed = allreduce_max(ms_mixed, world, dev)
    # the same steps again with an event pair around every launch of the
    # instrumented kernel classes (kernel times and the roofline)
    ms_prof, _, st_prof, _, prof = timed(ctx, args.steps, 1, prof=True)
    require_converged(st_prof, "mixed, profiled run")
    # this device's streaming rates over four FP32 vectors of 512 MB (a
    # read-only stream of 1.5 GB and a triad), the ceilings beside the copy peak
    sv = [torch.zeros(STREAM_FLOATS, dtype=torch.float32, device=dev) for _ in range(4)]
    stream_read, stream_triad = paris.stream_rates(*sv, reps=5)
    del sv
    # e2e through the host-buffer entry point (pinned host memory)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hC, hu0, hv0, hw0 = pin(pr.C), pin(pr.u), pin(pr.v), pin(pr.w)
    hu, hv, hw = hu0.clone().pin_memory(), hv0.clone().pin_memory(), hw0.clone().pin_memory()
    hp = torch.zeros(g.shape, dtype=torch.float64).pin_memory()
    ctx.projection_step_host(hC, pr.rho1, pr.rho2, pr.dt, hu, hv, hw, hp)  # allocates staging
    e2e_s = 0.0
    k_e2e = max(3, args.steps // 2)
    for i in range(args.warmup + k_e2e):
        hu.copy_(hu0)
        hv.copy_(hv0)
        hw.copy_(hw0)
        hp.zero_()
        t0 = time.perf_counter()
        ste = ctx.projection_step_host(hC, pr.rho1, pr.rho2, pr.dt, hu, hv, hw, hp)
        t1 = time.perf_counter()
        require_converged([ste], "e2e")
        if i >= args.warmup:
            e2e_s += t1 - t0
    e2e_s = allreduce_max(e2e_s, world, dev)
    h2d = 8 * (2 * N + sum(int(np.prod(g.face_shape(a))) for a in range(3)))
    d2h = h2d - 8 * N
    ctx.close()
    # plain FP64 form
    ctx = paris.Context(g, opts=paris.default_opts(precision=paris.FP64), device=dev)
    k64 = max(3, args.steps // 2)
    ms_fp64, per_fp64, st_fp64, _, _ = timed(ctx, k64, args.warmup)
    require_converged(st_fp64, "fp64")
    ms_fp64 = allreduce_max(ms_fp64, world, dev)
    _, _, st64p, _, prof64 = timed(ctx, k64, 1, prof=True)
    require_converged(st64p, "fp64, profiled run")
    ctx.close()

    # batched mode: 256 uneven periodic instances in one persistent launch
    batch = None
    if not args.no_batch:
        probs = pi.config4(count=256)
        with paris.Batch([q.grid for q in probs], device=dev) as b:
            bC = b.pack([q.C for q in probs], "C")
            bu0, bv0, bw0 = (b.pack([getattr(q, k) for q in probs], k) for k in ("u", "v", "w"))
            r1, r2, dts = [q.rho1 for q in probs], [q.rho2 for q in probs], [q.dt for q in probs]
            # the tuning is measured afresh on every run (a cache in the temporary
            # directory only spares repeated trials within one machine session)
            cache = os.path.join(tempfile.gettempdir(), f"paris_batch_autotune_{os.getuid()}.jsonl")
            b.autotune(bC, r1, r2, dts, bu0, bv0, bw0, cache_path=cache)
            bu, bv, bw = bu0.clone(), bv0.clone(), bw0.clone()
            bp = torch.zeros_like(bC)
            kb = 3
            tot = 0.0
            for i in range(1 + kb):
                bu.copy_(bu0)
                bv.copy_(bv0)
                bw.copy_(bw0)
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                bst = b.projection_step(bC, r1, r2, dts, bu, bv, bw, bp)
                t1 = time.perf_counter()
                if i > 0:
                    tot += t1 - t0
            cells = sum(q.grid.ncells for q in probs)
            batch = {"workload": "256 periodic boxes, axes from {32,48,64,96,128}, 1-8 drops, "
                                 "ratio log-U[1,1000], tol 1e-10", "cells": cells,
                     "solves_per_s": world * kb * len(probs) / tot, "ms_per_batch": 1e3 * tot / kb,
                     "converged": sum(s["converged"] for s in bst), "tuning": b.tuning(),
                     "launch_ctas": b.launch_ctas}
    if rank != 0:
        return
    value = world * args.steps / (ms_mixed / 1e3)
    fp64_value = world * k64 / (ms_fp64 / 1e3)
    # roofline of the dominant kernel class (largest summed time)
    from paper_2012_11744_gb300 import _abi as pabi
    dom = max(pabi.K_BYTES, key=lambda k: prof[k]["ms"])
    pk = prof[dom]
    achieved = pk["bytes"] / (pk["ms"] / 1e3) / 1e9 if pk["ms"] > 0 else None
    tr = NCU_TRAFFIC.get(dom)
    traffic = (tr["bytes_per_launch"] if tr and tr["bytes_per_launch"] and tr["sha"] == kernel_source_sha(tr["source"])
               else None)
    cpu = None
    if world == 1 and not args.no_cpu:
        import paris_inputs as pi2  # noqa: F401
        golden = load_golden(f"drops{args.n}_walls_z", required=args.n > 64)
        s = oracle_sample(pr, args.cpu_budget, golden)
        cpu = {"value": 1.0 / s["solve_s"], "unit": UNIT, "cores": oracle_threads(), "cpu_model": cpu_model(),
               "kind": "oracle",
               "sample": f"oracle set-up + {s['cg_iters_sampled']} CG iterations of the {args.n}^3 "
                         f"system ({s['sample_s']:.1f} s), extrapolated to the {s['cg_iters_full']} "
                         f"iterations of the full oracle solve"}
    its = [s["iters"] for s in st_mixed]

    def solve_roofline(k, v_cycle, outer, ms):
        # compulsory bytes of a solve: N (187 + k (V + outer)); 187 B/cell fixed
        # (face coefficients 44, coarse coefficients ~15, divergence 32, mean 16,
        # correction 80), V the bytes per cell of one V-cycle, outer those of one
        # Krylov iteration outside it, k the iterations
        b = N * (187.0 + k * (v_cycle + outer))
        t = b / (hbm * 1e9) * 1e3
        return {"model_bytes_per_solve": b, "iters": k, "roofline_ms": t, "measured_ms": ms,
                "pct_hbm": t / ms}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mixed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": workload_config(args.n),
        "step_ms": step_stats(per_mixed),
        "all_steps_converged": True,
        "iters_per_step": [x["iters"] for x in st_mixed],
        "fp64": {"value": fp64_value, "unit": UNIT, "ms_per_step": ms_fp64 / k64, "steps": k64,
                 "step_ms": step_stats(per_fp64), "all_steps_converged": True,
                 "iters": st_fp64[-1]["iters"], "rel_res_l2": st_fp64[-1]["rel_res_l2"],
                 "rel_res_linf": st_fp64[-1]["rel_res_linf"]},
        "mixed_over_fp64": value / fp64_value,
        "solve_roofline": {
            "model": "N (187 + k (V + outer)) bytes at the measured copy peak; V = 142.9 B/cell per FP32 "
                     "V-cycle (285.7 FP64), outer = 132 B/cell per mixed FCG iteration (140 FP64)",
            "mixed": solve_roofline(its[-1], 142.9, 132.0, ms_mixed / args.steps),
            "fp64": solve_roofline(st_fp64[-1]["iters"], 285.7, 140.0, ms_fp64 / k64)},
        "solve": {"iters": its[-1], "outer_iters": st_mixed[-1]["outer_iters"],
                  "rel_res_l2": st_mixed[-1]["rel_res_l2"], "rel_res_linf": st_mixed[-1]["rel_res_linf"],
                  "levels": st_mixed[-1]["levels"], "fell_back": st_mixed[-1]["fell_back"]},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": (achieved / hbm) if achieved else None, "traffic": traffic,
                     "peak_kind": peak_kind, "launches": pk["timed"],
                     "avg_launch_us": 1e3 * pk["ms"] / max(pk["timed"], 1),
                     "timing": f"CUDA events on the launching stream over {args.steps} further steps "
                               f"({ms_prof / args.steps:.2f} ms/step with the events): one pair around each "
                               f"smoothing phase's back-to-back finest-level passes (smooth0, 4 launches), "
                               f"one around each launch of the other classes",
                     "stream_read_only_gbs": stream_read, "stream_triad_gbs": stream_triad},
        "kernel_classes": {k: {"launches": v["timed"], "ms": v["ms"],
                               "gbs": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] > 0 else None}
                           for k, v in prof.items()},
        "kernel_classes_fp64": {k: {"launches": v["timed"], "ms": v["ms"],
                                    "gbs": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] > 0 else None}
                                for k, v in prof64.items()},
        "cpu_baseline": cpu,
        "e2e": {"value": world * k_e2e / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "batch": batch,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_single(args):
    """One projection of the workload (or, with --single viscous, the three
    multigrid component solves of --viscous), untimed: the target of ncu
    captures."""
    import torch

    import paper_2012_11744_gb300 as paris
    import paris_inputs as pi
    pr = pi.config2(n=args.n)
    g = pr.grid
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    if args.single == "viscous":
        ctx = paris.Context(g)
        C = d(pr.C)
        nus = [ctx.face_viscosity(c, C, VISC_MU[0], VISC_MU[1], pr.rho1, pr.rho2) for c in range(3)]
        tau = VISC_TAU_NU_OVER_H2 * g.h ** 2 / max(float(nu.max()) for nu in nus)
        sts = [ctx.viscous_solve(c, nus[c], tau, d((pr.u, pr.v, pr.w)[c]), tol=1e-10, multigrid=True)[1]
               for c in range(3)]
        torch.cuda.synchronize()
        print(json.dumps({"single": "viscous", "stats": sts}))
        return
    prec = paris.MIXED if args.single == "mixed" else paris.FP64
    kw = {} if args.smoother is None else {"smoother": args.smoother}
    ctx = paris.Context(g, opts=paris.default_opts(precision=prec, **kw))
    u, v, w = d(pr.u), d(pr.v), d(pr.w)
    p = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
    st = ctx.projection_step(d(pr.C), pr.rho1, pr.rho2, pr.dt, u, v, w, p)
    torch.cuda.synchronize()
    print(json.dumps({"single": args.single, "smoother": args.smoother, "stats": st}))


def run_viscous(args):
    """Implicit viscous step (Eq. muelliptic) of the three velocity components
    on the drop field, one JSON line.  nu_f from Eq. muH with water/air-like
    viscosities (mu 1e-3 / 1.8e-5) and the workload's densities; tau =
    4 h^2 / max nu_f (24 times the explicit stability limit of the viscous
    term); tol 1e-10.  One step = the three component solves from u*, v*, w*
    resident on the device, by the multigrid-preconditioned flexible CG
    (value) and by the Jacobi-preconditioned CG (beside it).  Algorithmic
    bytes per unknown and iteration: Jacobi-PCG 112 (q = A d: 24; x, r, z
    update: 64; d = z + beta d: 24); multigrid FCG 144 in FP64 (q = A d with
    the stored 1/(tau nu): 24; x, r update: 48; z.r, z.q: 24; d update: 24;
    the FP64/FP32 conversions at the V-cycle's ends: 24) plus the V-cycle,
    8/7 x 110 in FP32 (four colour sweeps of 20, the residual 16, the
    restriction 4.5, the prolongation 8.5 and the zeroing of x 4 on the
    finest level)."""
    import torch

    import paper_2012_11744_gb300 as paris
    import paris_inputs as pi
    pr = pi.config2(n=args.n)
    g = pr.grid
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx = paris.Context(g)
    C = d(pr.C)
    uvw = [d(pr.u), d(pr.v), d(pr.w)]
    nus = [ctx.face_viscosity(c, C, VISC_MU[0], VISC_MU[1], pr.rho1, pr.rho2) for c in range(3)]
    numax = max(float(nu.max()) for nu in nus)
    tau = VISC_TAU_NU_OVER_H2 * g.h ** 2 / numax
    outs = [torch.empty_like(x) for x in uvw]
    # unknowns of component c: its face grid without the wall faces of its own axis
    cells = (g.nx, g.ny, g.nz)
    unknowns = [int(np.prod([cells[a] - (1 if a == c and g.bc[a] == pi.WALL else 0) for a in range(3)]))
                for c in range(3)]
    hbm, kind = measured_peaks()
    res = {}
    for name, mg, per_it in (("multigrid", True, 144.0 + 110.0 * 8.0 / 7.0), ("jacobi", False, 112.0)):
        def step(i):
            return [ctx.viscous_solve(c, nus[c], tau, uvw[c], outs[c], tol=1e-10, multigrid=mg)[1] for c in range(3)]

        for _ in range(args.warmup):
            step(0)
        K = args.steps if mg else max(1, args.steps // 2)
        with ClockSampler(0) as clk:
            per, sts = event_steps(step, K, ctx.stream)
        last = sts[-1]
        require_converged([x for s3 in sts for x in s3], f"viscous {name}")
        iters = [x["iters"] for x in last]
        byt = sum(per_it * n * k for n, k in zip(unknowns, iters))
        ms = sum(per) / K
        gbs = byt / (ms * 1e-3) / 1e9
        res[name] = {"value": 3.0 / (ms * 1e-3), "ms_per_step": ms, "step_ms": step_stats(per), "steps": K,
                     "iters": iters, "levels": [x["levels"] for x in last],
                     "rel_res_l2": [x["rel_res_l2"] for x in last], "bytes_per_unknown_iteration": per_it,
                     "iteration_roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                                            "frac": gbs / hbm, "peak_kind": kind,
                                            "note": "whole iterations incl. the host read of the norms"},
                     "clocks": clk.summary()}
    cpu = None
    if not args.no_cpu:
        gold = load_visc_golden(args.n)
        smp = viscous_oracle_sample(pr, args.cpu_budget, gold)
        cpu = {"value": 3.0 / smp["step_s"], "unit": "solves/s", "cores": oracle_threads(),
               "cpu_model": cpu_model(), "kind": "oracle",
               "sample": f"scipy CG (sparse products on one thread), face viscosities, then the w solve cut after "
                         f"{smp['cg_iters_sampled'][0]}, 5 and {smp['cg_iters_sampled'][1]} iterations "
                         f"(set-up {smp['setup_s']:.2f} s, {smp['s_per_cg_iter']:.3f} s per iteration), "
                         f"extrapolated to the full oracle solves' {smp['cg_iters_full']} iterations"}
    m = res["multigrid"]
    print(json.dumps({
        "metric": "implicit viscous solves/s (u, v, w each a solve) at %d^3, tol 1e-10" % args.n,
        "value": m["value"], "unit": "solves/s", "ms_per_step": m["ms_per_step"], "step_ms": m["step_ms"],
        "steps": m["steps"], "warmup": args.warmup, "higher_is_better": True, "dtype": "f64+f32",
        "data": "synthetic", "method": "flexible CG (FP64) with an FP32 geometric-multigrid V-cycle",
        "iters": m["iters"], "levels": m["levels"], "rel_res_l2": m["rel_res_l2"], "all_steps_converged": True,
        "tau_nu_max_over_h2": VISC_TAU_NU_OVER_H2, "iteration_roofline": m["iteration_roofline"],
        "jacobi_pcg": res["jacobi"], "multigrid_over_jacobi": m["value"] / res["jacobi"]["value"],
        "clocks": m["clocks"], "cpu_baseline": cpu,
        "config": {"workload": workload_config(args.n)["workload"] + ", mu 1e-3/1.8e-5",
                   "l2": "no flush: each iteration streams several vectors of one component (> 129 MB L2)"}}),
        flush=True)


def event_steps(step, K, stream):
    """Run step() K times, each between its own event pair on `stream`;
    returns the per-step ms and the step results."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    out = []
    torch.cuda.synchronize()
    for i in range(K):
        ev[i][0].record(stream)
        out.append(step(i))
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev], out


def class_roofline(prof, hbm, kind):
    """Roofline of the dominant single-kernel class of a kernel-class profile."""
    from paper_2012_11744_gb300 import _abi as pabi
    dom = max(pabi.K_BYTES, key=lambda k: prof[k]["ms"])
    pk = prof[dom]
    ach = pk["bytes"] / (pk["ms"] / 1e3) / 1e9 if pk["ms"] > 0 else None
    return {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm, "unit": "GB/s",
            "frac": ach / hbm if ach else None, "traffic": None, "peak_kind": kind,
            "launches": pk["timed"], "avg_launch_us": 1e3 * pk["ms"] / max(pk["timed"], 1)}


def run_jet(args):
    """The 512x256x256 jet (periodic x, walls y/z, ratio 1000, dt 5e-5),
    mixed form to 1e-10: solves/s, and the pointwise error of the last
    step's p and u against the stored full FP64 oracle solve
    (tests/golden/jet512x256x256.json) at its sampled cells and faces."""
    import hashlib

    import torch

    import paper_2012_11744_gb300 as paris
    import paris_inputs as pi
    pr = pi.config3()
    g = pr.grid
    gold = load_golden("jet512x256x256")
    assert gold["C_sha256"] == hashlib.sha256(np.ascontiguousarray(pr.C).tobytes()).hexdigest()
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    C, u0, v0, w0 = d(pr.C), d(pr.u), d(pr.v), d(pr.w)
    K = args.steps
    sets = [(u0.clone(), v0.clone(), w0.clone(), torch.zeros(g.shape, dtype=torch.float64, device="cuda"))
            for _ in range(K)]
    ctx = paris.Context(g, opts=paris.default_opts(precision=paris.MIXED))
    for _ in range(args.warmup):
        uu, vv, ww, pp = u0.clone(), v0.clone(), w0.clone(), torch.zeros_like(sets[0][3])
        ctx.projection_step(C, pr.rho1, pr.rho2, pr.dt, uu, vv, ww, pp)
    with ClockSampler(0) as clk:
        per, sts = event_steps(lambda i: ctx.projection_step(C, pr.rho1, pr.rho2, pr.dt, *sets[i]), K, ctx.stream)
    require_converged(sts, "jet")
    uu, vv, ww, pp = u0.clone(), v0.clone(), w0.clone(), torch.zeros_like(sets[0][3])
    ctx.profile(True)
    ctx.projection_step(C, pr.rho1, pr.rho2, pr.dt, uu, vv, ww, pp)
    prof = ctx.profile_read()
    ctx.profile(False)
    ctx.close()
    p = sets[-1][3].cpu().numpy().ravel()
    uvw = [x.cpu().numpy().ravel() for x in sets[-1][:3]]
    cells = np.asarray(gold["cells"])
    p_err = float(np.abs(p[cells] - np.asarray(gold["p"])).max() / gold["p_max_abs"])
    umax = gold["ustar_max_abs"]
    u_err = max(float(np.abs(uvw[a][np.asarray(gold["faces"][a])] - np.asarray(gold["u"][a])).max())
                for a in range(3)) / umax
    hbm, kind = measured_peaks()
    total = sum(per)
    cpu = None
    if not args.no_cpu:
        smp = oracle_sample(pr, args.cpu_budget, gold)
        cpu = {"value": 1.0 / smp["solve_s"], "unit": UNIT, "cores": oracle_threads(), "cpu_model": cpu_model(),
               "kind": "oracle",
               "sample": f"oracle set-up + {smp['cg_iters_sampled']} CG iterations of the jet system "
                         f"({smp['sample_s']:.1f} s), extrapolated to the {smp['cg_iters_full']} iterations "
                         f"of the full oracle solve"}
    print(json.dumps({
        "metric": "jet projection solves/s at 512x256x256, rho ratio 1000, resid 1e-10 (mixed)",
        "value": K / (total / 1e3), "unit": UNIT, "steps": K, "warmup": args.warmup, "ms_per_step": total / K,
        "step_ms": step_stats(per), "higher_is_better": True, "dtype": "f32+f64", "data": "synthetic",
        "iters_per_step": [x["iters"] for x in sts], "rel_res_l2": sts[-1]["rel_res_l2"],
        "rel_res_linf": sts[-1]["rel_res_linf"], "all_steps_converged": True,
        "vs_oracle": {"p_rel_err_inf": p_err, "u_err_inf_over_max_ustar": u_err,
                      "samples": [len(cells), sum(len(f) for f in gold["faces"])],
                      "oracle_rel_res_l2": gold["oracle"]["rel_res_l2"],
                      "oracle_p_rel_err_bound": gold["bound"]["p_rel_err_bound"]},
        "roofline": class_roofline(prof, hbm, kind), "clocks": clk.summary(), "cpu_baseline": cpu,
        "config": {"workload": "jet512x256x256: L = (2,1,1), periodic x, walls y/z, cylinder R = 0.08 with 4 "
                               "sine modes, u_x = 1 in the liquid + U[-0.1,0.1] noise, rho 1000/1, dt 5e-5, "
                               "tol 1e-10 (L2 and Linf)",
                   "l2": "no flush: each step projects its own u*, v*, w*, p (4 x 268 MB > 129 MB L2)"}}),
        flush=True)


def run_adjoint(args):
    """The adjoint configuration: 128^3 periodic tanh drop (rho 100/1), loss
    L = 1/2 ||u - u_target||^2.  One step = the forward projection step plus
    the adjoint (paris_project_adjoint and paris_face_coeffs_adjoint) giving
    dL/du* and dL/dC, in FP64 and in the mixed form; value = gradients/s of
    the mixed form.  The two forms' gradients are compared with each other
    here; against the oracle adjoint and finite differences in the tests."""
    import torch

    import paper_2012_11744_gb300 as paris
    import paris_inputs as pi
    pr = pi.config5()
    g = pr.grid
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    C, u0, v0, w0 = d(pr.C), d(pr.u), d(pr.v), d(pr.w)
    tgt = [d(x) for x in pr.extra["target"]]
    res = {}
    for name, prec in (("mixed", paris.MIXED), ("fp64", paris.FP64)):
        ctx = paris.Context(g, opts=paris.default_opts(precision=prec))
        beta = ctx.empty_faces()
        p = torch.zeros(g.shape, dtype=torch.float64, device="cuda")

        def step(i):
            u, v, w = u0.clone(), v0.clone(), w0.clone()
            p.zero_()
            st = ctx.projection_step(C, pr.rho1, pr.rho2, pr.dt, u, v, w, p)
            ctx.face_coeffs(C, pr.rho1, pr.rho2, beta)
            gu = [(x - t).contiguous() for x, t in zip((u, v, w), tgt)]
            gus, gb, _, sta = ctx.project_adjoint(*beta, p, pr.dt, *gu)
            gC = ctx.face_coeffs_adjoint(pr.rho1, pr.rho2, *beta, *gb)
            return st, sta, gus, gC

        for _ in range(args.warmup):
            step(0)
        per, outs = event_steps(step, args.steps, ctx.stream)
        require_converged([o[0] for o in outs] + [o[1] for o in outs], f"adjoint {name}")
        res[name] = {"per": per, "gus": [x.cpu().numpy() for x in outs[-1][2]], "gC": outs[-1][3].cpu().numpy(),
                     "iters": [outs[-1][0]["iters"], outs[-1][1]["iters"]]}
        ctx.close()
    rel = lambda a, b: float(np.abs(a - b).max() / np.abs(b).max())
    tot = sum(res["mixed"]["per"])
    print(json.dumps({
        "metric": "adjoint gradients/s (forward projection + dL/du*, dL/dC) at 128^3, rho ratio 100",
        "value": args.steps / (tot / 1e3), "unit": "gradients/s", "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot / args.steps, "step_ms": step_stats(res["mixed"]["per"]), "higher_is_better": True,
        "dtype": "f32+f64", "data": "synthetic",
        "fp64": {"value": args.steps / (sum(res["fp64"]["per"]) / 1e3), "step_ms": step_stats(res["fp64"]["per"]),
                 "iters_forward_adjoint": res["fp64"]["iters"]},
        "iters_forward_adjoint": res["mixed"]["iters"],
        "mixed_vs_fp64": {"dL_du_star": max(rel(a, b) for a, b in zip(res["mixed"]["gus"], res["fp64"]["gus"])),
                          "dL_dC": rel(res["mixed"]["gC"], res["fp64"]["gC"])},
        "config": {"workload": "adjoint_drop128: 128^3 periodic, tanh drop r = 0.2 (w = 1.5h), rho 100/1, "
                               "u* ~ U[-1,1], divergence-free target, dt 1e-3, tol 1e-10",
                   "l2": "each step reads C, u*, target and writes the gradients (> 129 MB L2)"}}), flush=True)


def run_forcing(args):
    """The predictor forcing (capillary CSF term with the drops' curvature,
    sigma 0.07, and gravity -9.81 in z) fused into the projection step of the
    256^3 drop field, against the same step without forcing: solves/s of the
    forced step and the time of the face pass that carries the forcing."""
    import torch

    import paper_2012_11744_gb300 as paris
    import paris_inputs as pi
    pr = pi.config2(n=args.n)
    g = pr.grid
    kappa = pi.drop_curvature(g, pr.extra["spheres"])
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    C, K_, u0, v0, w0 = d(pr.C), d(kappa), d(pr.u), d(pr.v), d(pr.w)
    sigma, grav = 0.07, (0.0, 0.0, -9.81)
    K = args.steps
    sets = [(u0.clone(), v0.clone(), w0.clone(), torch.zeros(g.shape, dtype=torch.float64, device="cuda"))
            for _ in range(K)]

    def refill():
        for (u, v, w, p) in sets:
            u.copy_(u0)
            v.copy_(v0)
            w.copy_(w0)
            p.zero_()

    ctx = paris.Context(g, opts=paris.default_opts(precision=paris.MIXED))
    forced = lambda i: ctx.projection_step_forced(C, K_, pr.rho1, pr.rho2, sigma, grav, pr.dt, *sets[i])
    plain = lambda i: ctx.projection_step(C, pr.rho1, pr.rho2, pr.dt, *sets[i])
    for _ in range(args.warmup):
        refill()
        forced(0)
        refill()
        plain(0)
    refill()
    with ClockSampler(0) as clk:
        per_f, st_f = event_steps(forced, K, ctx.stream)
    require_converged(st_f, "forced")
    refill()
    per_p, st_p = event_steps(plain, K, ctx.stream)
    require_converged(st_p, "plain")
    # the face pass alone, with and without the forcing (events around each launch)
    N = g.ncells
    beta = ctx.empty_faces()
    uu, vv, ww = u0.clone(), v0.clone(), w0.clone()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    reps = 20
    t = {}
    for name, fn in (("forcing", lambda: ctx.predictor_forcing(C, K_, pr.rho1, pr.rho2, sigma, grav, pr.dt,
                                                               uu, vv, ww, beta)),
                     ("face_coeffs", lambda: ctx.face_coeffs(C, pr.rho1, pr.rho2, beta))):
        fn()
        e0, e1 = ev(), ev()
        e0.record(ctx.stream)
        for _ in range(reps):
            fn()
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        t[name] = e0.elapsed_time(e1) / reps
    ctx.close()
    nf = sum(int(np.prod(g.face_shape(a))) for a in range(3))
    byt_f = 8.0 * (2 * N + 3 * nf)  # C, kappa read; beta written, u^n read and u* written (8 B per face each)
    hbm, kind = measured_peaks()
    ach = byt_f / (t["forcing"] * 1e-3) / 1e9
    print(json.dumps({
        "metric": "forced projection solves/s at 256^3 (CSF + gravity in the face pass), rho 1000, resid 1e-10",
        "value": K / (sum(per_f) / 1e3), "unit": UNIT, "steps": K, "warmup": args.warmup,
        "ms_per_step": sum(per_f) / K, "step_ms": step_stats(per_f), "higher_is_better": True,
        "dtype": "f32+f64", "data": "synthetic", "all_steps_converged": True,
        "iters_per_step": [x["iters"] for x in st_f],
        "unforced": {"value": K / (sum(per_p) / 1e3), "step_ms": step_stats(per_p)},
        "face_pass_ms": {"with_forcing": t["forcing"], "face_coeffs_only": t["face_coeffs"]},
        "roofline": {"bound": "hbm", "kernel": "face_coeffs_kernel<FORCE>", "achieved": ach, "peak": hbm,
                     "unit": "GB/s", "frac": ach / hbm, "traffic": None, "peak_kind": kind,
                     "bytes_per_launch": byt_f,
                     "note": "C, kappa read (16 B/cell), beta written, u^n read, u* written (24 B/face each)"},
        "clocks": clk.summary(),
        "config": {"workload": workload_config(args.n)["workload"] + ", sigma 0.07, kappa = -2/r of the nearest "
                               "drop, g = -9.81 z", "l2": "no flush: fields > 129 MB L2"}}), flush=True)


def run_free_surface(args):
    """The free-surface projection of Sec. 3.7.5 on the 256^3 drop field read
    as 64 gas bubbles in liquid (C the gas fraction), liquid density 1000,
    theta ~ U[0.1, 1] per face, the bubbles' curvature, one gas pressure;
    then the phantom projection of the two gas layers on the result.  Both
    run the default mixed form (FP64 refinement around the FP32
    V-cycle-preconditioned CG, the Dirichlet diagonal excess on every level);
    the plain FP64 form is timed beside it."""
    import torch

    import paper_2012_11744_gb300 as paris
    import paris_inputs as pi
    pr = pi.config2(n=args.n)
    g = pr.grid
    rng = np.random.default_rng([400, args.n])
    theta = [rng.uniform(0.1, 1.0, g.face_shape(a)) for a in range(3)]
    kappa = pi.drop_curvature(g, pr.extra["spheres"])
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    C, K_, PG = d(pr.C), d(kappa), d(np.full(g.shape, 1.0e5))
    TH = [d(t) for t in theta]
    u0, v0, w0 = d(pr.u), d(pr.v), d(pr.w)
    K = args.steps
    sets = [(u0.clone(), v0.clone(), w0.clone(), torch.zeros(g.shape, dtype=torch.float64, device="cuda"))
            for _ in range(K)]

    def refill():
        for (u, v, w, p) in sets:
            u.copy_(u0)
            v.copy_(v0)
            w.copy_(w0)
            p.zero_()

    ctx = paris.Context(g)
    step = lambda i: ctx.free_surface_step(C, 1000.0, pr.dt, *sets[i][:3], sets[i][3], p_gas=PG, theta=TH,
                                           kappa=K_, sigma=0.07)
    phantom = lambda i: ctx.phantom_projection(C, *sets[i][:3], sets[i][3])[1]
    for _ in range(args.warmup):
        refill()
        step(0)
        phantom(0)
    refill()
    with ClockSampler(0) as clk:
        per, sts = event_steps(step, K, ctx.stream)
    require_converged(sts, "free surface")
    per_ph, sts_ph = event_steps(phantom, K, ctx.stream)
    require_converged(sts_ph, "phantom")
    u = [x.cpu().numpy() for x in sets[0][:3]]
    ctx.close()
    # the FP64 form on the same steps
    K64 = min(K, 10)
    ctx = paris.Context(g, opts=paris.default_opts(precision=paris.FP64))
    step = lambda i: ctx.free_surface_step(C, 1000.0, pr.dt, *sets[i][:3], sets[i][3], p_gas=PG, theta=TH,
                                           kappa=K_, sigma=0.07)
    refill()
    step(0)
    refill()
    per64, sts64 = event_steps(step, K64, ctx.stream)
    require_converged(sts64, "free surface (FP64 form)")
    ctx.close()
    import oracle
    div = oracle.divergence(g, *u, dt=1.0)
    liq = pr.C < 0.5
    print(json.dumps({
        "metric": "free-surface projection solves/s at 256^3 (ghost-fluid Dirichlet at 64 bubbles), resid 1e-10",
        "value": K / (sum(per) / 1e3), "unit": UNIT, "steps": K, "warmup": args.warmup,
        "ms_per_step": sum(per) / K, "step_ms": step_stats(per), "higher_is_better": True,
        "dtype": "f32+f64", "data": "synthetic", "all_steps_converged": True,
        "fell_back": sum(x["fell_back"] for x in sts),
        "iters_per_step": [x["iters"] for x in sts], "rel_res_l2": sts[-1]["rel_res_l2"],
        "rel_res_linf": sts[-1]["rel_res_linf"],
        "max_div_liquid_times_h": float(np.abs(div[liq]).max() * g.h),
        "phantom": {"value": K / (sum(per_ph) / 1e3), "step_ms": step_stats(per_ph),
                    "iters_per_step": [x["iters"] for x in sts_ph]},
        "fp64": {"value": K64 / (sum(per64) / 1e3), "step_ms": step_stats(per64),
                 "iters_per_step": [x["iters"] for x in sts64]},
        "clocks": clk.summary(),
        "config": {"workload": workload_config(args.n)["workload"].replace("64 drops, rho 1000/1", "64 gas bubbles")
                   + ", rho_l 1000, theta ~ U[0.1, 1], sigma 0.07, kappa of the nearest bubble, p_gas 1e5",
                   "l2": "no flush: fields > 129 MB L2"}}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="paris", choices=["paris", "reference"])
    ap.add_argument("--edge", dest="n", type=int, default=256, help="grid edge of the drop-field workload")
    ap.add_argument("--ref-budget", type=float, default=2.0,
                    help="seconds of oracle CG iterations per --impl reference step")
    ap.add_argument("--cpu-budget", type=float, default=6.0,
                    help="seconds of oracle CG iterations in the cpu_baseline sample")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-mode measurement")
    ap.add_argument("--single", choices=["mixed", "fp64", "viscous"], default=None,
                    help="run one untimed projection (the target of ncu captures) and exit")
    ap.add_argument("--viscous", action="store_true",
                    help="time the implicit viscous step of the three components instead and exit")
    ap.add_argument("--jet", action="store_true", help="time the 512x256x256 jet (mixed) instead and exit")
    ap.add_argument("--adjoint", action="store_true", help="time the 128^3 adjoint step instead and exit")
    ap.add_argument("--forcing", action="store_true",
                    help="time the projection step with the predictor forcing fused in instead and exit")
    ap.add_argument("--free-surface", dest="free_surface", action="store_true",
                    help="time the free-surface (ghost-fluid) and phantom projections instead and exit")
    ap.add_argument("--smoother", type=int, default=None,
                    help="with --single: 0 fused red-black, 1 Jacobi, 2 two-pass red-black")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.viscous:
        run_viscous(args)
        return
    if args.jet:
        run_jet(args)
        return
    if args.adjoint:
        run_adjoint(args)
        return
    if args.forcing:
        run_forcing(args)
        return
    if args.free_surface:
        run_free_surface(args)
        return
    if args.single:
        run_single(args)
        return
    if args.impl == "reference":
        # rank 0 alone runs the CPU oracle; other ranks exit without work
        run_reference(args, int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")))
        return
    rank, world, local = dist_setup(args.gpus)
    run_paris(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
