"""Benchmark: cell-stage updates/s of the HGKS stage sweep on the Taylor-Green
vortex at 128^3 (FP64 plain path, with the mixed FP32/FP64 path reported
beside it), plus the end-to-end rate through the C ABI with host buffers,
the roofline of the dominant kernel, clocks, and the oracle's CPU rate.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one two-stage fourth-order time step (CFL reduction, and per stage:
ghost fill, WENO-AO reconstruction, Gauss-point gas-kinetic flux, update);
one step is two cell-stage updates per cell.  Under torchrun (N > 1) every
rank advances its own 128^3 instance (the path is replicated, not sharded)
and the value is the aggregate over ranks.
"""
from __future__ import annotations

import argparse
import functools
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-stage updates/s at TGV 128^3 (FP64 vs mixed)"
UNIT = "cell-stage updates/s"

# Work per unit of the dominant kernel (the Gauss-point face flux): FP64
# flop per Gauss point on the FP64 pipe (2 per DFMA, 1 per DADD and DMUL)
# for the FP64 path, FP32 flop on the FMA pipe for the mixed path, fixed at
# the ncu instruction counters of one capture of the kernel on TGV 32^3.
# Later rewrites of the kernel (the Gauss-point polynomials as multiply-add
# chains, the scales 1/rho and 1/h moved from the slope data into the slope
# solves' constants) execute fewer flops for the same algorithm, so
# `achieved` is the rate of that fixed work per Gauss point (algorithm-
# equivalent flop), not of the flops the current kernel issues.  The DRAM
# traffic of that capture no longer describes the current kernel and is
# reported as null (FLUX_TRAFFIC_BYTES_PER_FACE keeps the last measured
# figure, bytes per face of a TGV 32^3 launch, for reference).
FLUX_FP64_FLOP_PER_GP = 3018.0
FLUX_FP32_FLOP_PER_GP = 2769.0
FLUX_TRAFFIC_BYTES_PER_FACE = {"fp64": 14.300e6 / 33792, "mixed": 7.209e6 / 33792}
FLUX_TRAFFIC_CURRENT = False
# GB300 ALU peaks derived from unit counts and clocks: 152 SMs x 2070 MHz x
# (FP64: 2 DFMA/clk/SM = 4 flop; FP32: 128 FMA/clk/SM = 256 flop).
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
PEAK_FP64_TFLOPS = SM_COUNT * SM_MAX_MHZ * 1e6 * 4 / 1e12
PEAK_FP32_TFLOPS = SM_COUNT * SM_MAX_MHZ * 1e6 * 256 / 1e12


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, dist=None, device="cuda"):
    """The largest x over the ranks (the timed region of the slowest rank);
    x itself on one process."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_rate(world, units_per_rank, seconds):
    """Whole-job throughput of `world` independent replicas (weak scaling):
    the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / seconds


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, val in zip(names, r[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


@functools.lru_cache(maxsize=2)
def workload(n):
    from paper_1909_01580_gb300 import workloads
    q, lo, hi = workloads.taylor_green((n, n, n), mach=0.1)
    return q, lo, hi


def run_gpu(args, rank, world, local, dist):
    import torch
    from paper_1909_01580_gb300 import hgks

    torch.cuda.set_device(local)
    hgks.load()
    n = args.n
    q0, lo, hi = workload(n)
    ncell = n ** 3
    mu, Pr = 1.0 / 1600.0, 0.72

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    slowest = functools.partial(max_over_ranks, dist=dist, device="cuda")

    results = {}
    for prec_name, prec in (("fp64", hgks.HGKS_FP64), ("mixed", hgks.HGKS_MIXED)):
        stream = torch.cuda.Stream()
        s = hgks.Solver((n, n, n), lo, hi, mu=mu, Pr=Pr, precision=prec, stream=stream.cuda_stream)
        qd = torch.from_numpy(q0).cuda()
        torch.cuda.synchronize()
        hgks.hgks_set_state(s.h, qd, 0.0)
        s.step(args.warmup, cfl=0.35)
        hgks.hgks_set_timing(s.h, 1)
        sampler = ClockSampler(local)
        sampler.start()
        barrier()
        l0 = s.launches
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        s.step(args.steps, cfl=0.35, sync=False)
        ev1.record(stream)
        ev1.synchronize()
        barrier()
        clocks = sampler.stop()
        launches = s.launches - l0
        ms = ev0.elapsed_time(ev1)
        ms_max = slowest(ms)
        timing = hgks.hgks_get_timing(s.h)
        hgks.hgks_set_timing(s.h, 0)
        t_now, steps_done = s.step(0)
        # the flux kernel: 3 launches per stage, 4 threads (Gauss points) per face
        flux_ms, flux_launches = timing["flux"]
        nface_stage = 3 * n * n * (n + 1)
        gp_per_launch = 4 * nface_stage / 3
        per_launch_s = flux_ms / 1e3 / max(flux_launches, 1)
        flop_gp = FLUX_FP64_FLOP_PER_GP if prec_name == "fp64" else FLUX_FP32_FLOP_PER_GP
        achieved = gp_per_launch * flop_gp / per_launch_s / 1e12
        peak = PEAK_FP64_TFLOPS if prec_name == "fp64" else PEAK_FP32_TFLOPS
        total_phase = sum(v[0] for v in timing.values())
        results[prec_name] = {
            "value": replicas_rate(world, ncell * 2 * args.steps, ms_max / 1e3),
            "ms_per_step": ms_max / args.steps,
            "launches": launches,
            "clocks": clocks,
            "phase_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in timing.items()},
            "flux_share": flux_ms / total_phase if total_phase > 0 else None,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "traffic": (FLUX_TRAFFIC_BYTES_PER_FACE[prec_name] * nface_stage / 3
                                     if FLUX_TRAFFIC_CURRENT else None),
                         "traffic_note": ("ncu dram read+write of a TGV 32^3 launch scaled to 128^3 faces"
                                          if FLUX_TRAFFIC_CURRENT else
                                          "null: the kernel changed after its last ncu capture (which read "
                                          f"{FLUX_TRAFFIC_BYTES_PER_FACE[prec_name]:.0f} B per face)"),
                         "work_note": (f"{flop_gp:.0f} flop per Gauss point, the executed count of an ncu "
                                       "capture of an earlier build of the kernel; the current build executes "
                                       "fewer for the same algorithm (algorithm-equivalent flop)"),
                         "kernel": "k_face_flux", "pipe": "fp64" if prec_name == "fp64" else "fp32",
                         "peak_source": "derived: 152 SMs x 2070 MHz x (4 FP64 | 256 FP32) flop/clk/SM"},
            "t_reached": t_now,
        }
        # end to end through the C ABI with host buffers: every step copies the
        # state in from pinned host memory and the result back out
        if not args.no_e2e:
            qh = torch.from_numpy(q0).pin_memory()
            qh_np = qh.numpy()
            out = torch.empty_like(qh).pin_memory()
            out_np = out.numpy()
            e2e_steps = max(1, min(args.steps, 5))
            barrier()
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                hgks.hgks_set_state(s.h, qh_np, 0.0)
                s.step(1, cfl=0.35)
                hgks.hgks_get_state(s.h, out_np)
            barrier()
            el = slowest(time.perf_counter() - t0)
            results[prec_name]["e2e"] = {"value": replicas_rate(world, ncell * 2 * e2e_steps, el), "unit": UNIT,
                                         "h2d_bytes_per_step": int(q0.nbytes), "d2h_bytes_per_step": int(q0.nbytes),
                                         "steps": e2e_steps}
        s.close()
        del stream
    return results


def moving_run(steps, warmup, n=96):
    """Density advection on the moving mesh x = xi + 0.05 sin(2 pi t)
    prod_d sin(pi xi_d) over [0,2]^3 (n^3 cells, CFL 0.35): cell-stage
    updates/s of the FP64 and mixed paths, CUDA events on the handle's
    stream, with the per-phase split (geometry included)."""
    import torch
    from paper_1909_01580_gb300 import hgks, workloads
    q0 = workloads.density_advection((n, n, n))
    out = {"workload": f"density advection {n}^3 on the moving mesh (amplitude 0.05, omega 2 pi), CFL 0.35"}
    for name, prec in (("fp64", hgks.HGKS_FP64), ("mixed", hgks.HGKS_MIXED)):
        stream = torch.cuda.Stream()
        s = hgks.Solver((n, n, n), (0, 0, 0), (2, 2, 2), precision=prec, stream=stream.cuda_stream,
                        mesh=2, mesh_amp=0.05, mesh_omega=2 * math.pi)
        s.set_state(q0, t=0.0)
        s.step(warmup, cfl=0.35)
        hgks.hgks_set_timing(s.h, 1)
        torch.cuda.synchronize()
        l0 = s.launches
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        s.step(steps, cfl=0.35, sync=False)
        ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1)
        timing = hgks.hgks_get_timing(s.h)
        out[name] = {"value": n ** 3 * 2 * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
                     "steps": steps, "launches": s.launches - l0,
                     "phase_ms_per_step": {k: round(v[0] / steps, 4) for k, v in timing.items()},
                     "note": "the halo phase includes the cell-geometry kernel of each stage"}
        s.close()
        del stream
    return out


def workload_run(name, q0, lo, hi, steps, warmup, solver_kw=None, options=None):
    """Cell-stage updates/s of one workload on one handle per precision
    (CFL 0.35, CUDA events on the handle's stream), with the per-phase split."""
    import torch
    from paper_1909_01580_gb300 import hgks
    n = q0.shape[1:][::-1]
    out = {"workload": name}
    for pname, prec in (("fp64", hgks.HGKS_FP64), ("mixed", hgks.HGKS_MIXED)):
        stream = torch.cuda.Stream()
        s = hgks.Solver(n, lo, hi, precision=prec, stream=stream.cuda_stream, **(solver_kw or {}))
        for k, v in (options or {}).items():
            hgks.hgks_set_option(s.h, k, v)
        s.set_state(q0, t=0.0)
        s.step(warmup, cfl=0.35)
        hgks.hgks_set_timing(s.h, 1)
        torch.cuda.synchronize()
        l0 = s.launches
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        s.step(steps, cfl=0.35, sync=False)
        ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1)
        timing = hgks.hgks_get_timing(s.h)
        cells = int(np.prod(n))
        out[pname] = {"value": cells * 2 * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
                      "steps": steps, "launches": s.launches - l0,
                      "phase_ms_per_step": {k: round(v[0] / steps, 4) for k, v in timing.items()}}
        s.close()
        del stream
    return out


def octant_run(steps, warmup, n=128):
    from paper_1909_01580_gb300 import workloads
    q0 = workloads.octant_riemann((n, n, n), seed=0)
    return workload_run(f"octant Riemann problem {n}^3 on [0,1]^3, reflective walls, seed 0, CFL 0.35", q0,
                        (0, 0, 0), (1, 1, 1), steps, warmup, solver_kw={"bc": (1,) * 6})


def turbulence_run(steps, warmup, n=128, mach=0.5):
    from paper_1909_01580_gb300 import workloads
    q0, lo, hi, P = workloads.isotropic_turbulence(n, mach, seed=0)
    return workload_run(f"compressible isotropic turbulence {n}^3, Ma_t {mach}, Re_lambda 72, mu ~ T^0.76, Pr 0.7",
                        q0, lo, hi, steps, warmup, solver_kw={"mu": P.mu0, "Pr": 0.7},
                        options={"mu_power": 0.76, "mu_T_ref": P.T0})


def serving_run(count=16, sizes=(24, 32, 48), steps=(20, 40), seed=0, load=1.25, precisions=("fp64", "mixed"),
                arena_gb=4.0):
    """Serving workload: seeded requests (density advection / TGV 50:50,
    uniform sizes, Mach U[0.05, 0.3], Re U[400, 3200]).  One-at-a-time FP64
    solves give the service times; arrivals are Poisson at `load` times that
    sequential capacity; the continuous-batching loop then serves the same
    arrivals in real time with an arena of arena_gb GB (admission by HBM
    footprint) for each precision."""
    from paper_1909_01580_gb300 import hgks, serving
    reqs = serving.request_stream(count=count, seed=seed, sizes=sizes, steps=steps)
    fifo = serving.serve_fifo(reqs, precision=hgks.HGKS_FP64)
    rate = load * count / fifo["busy"]
    serving.poisson_arrivals(reqs, rate, seed=seed)
    base = serving.fifo_latencies(reqs, fifo["service"])
    out = {"requests": count, "sizes": list(sizes), "steps": list(steps), "seed": seed,
           "arrival_rate_per_s": rate, "load_vs_sequential_fp64": load, "arena_gb": arena_gb,
           "fifo_fp64": serving.summary("fifo_fp64", base, reqs)}
    cells = sum(2 * r.cells * r.steps_target for r in reqs)
    # admission policies: every arrived request that fits (fifo), or the
    # least work first with a cap on the resident cells (sjf; FP64 fills the
    # GPU with one mid-size instance, the mixed path wants more per launch)
    caps = {"fp64": 120_000, "mixed": 1_000_000}
    for name in precisions:
        prec = hgks.HGKS_FP64 if name == "fp64" else hgks.HGKS_MIXED
        for policy in ("fifo", "sjf"):
            res = serving.serve_batched(reqs, precision=prec, arena_bytes=int(arena_gb * (1 << 30)),
                                        max_instances=64, steps_per_poll=4, keep_results=False, policy=policy,
                                        max_resident_cells=caps[name] if policy == "sjf" else None)
            key = f"batched_{name}" + ("_sjf" if policy == "sjf" else "")
            s = serving.summary(key, res, reqs)
            s["policy"] = policy if policy == "fifo" else f"sjf, resident cells <= {caps[name]}"
            s["max_resident"] = res["max_resident"]
            s["gpu_launches"] = res["launches"]
            s["cell_stage_updates_per_s"] = res["cell_stages"] / res["makespan"]
            out[key] = s
    out["approx_cell_stages"] = cells
    return out


def cpu_baseline(n, steps_budget_s=12.0, block=(32, 32, 16)):
    """The oracle as it stands on the host cores: one operator evaluation (one
    stage's reconstruction and face fluxes) over a contiguous block of cells of
    the same TGV 128^3 state, scaled to cell-stage updates/s."""
    import oracle
    q, lo, hi = workload(n)
    cfg = oracle.make_cfg((n, n, n), lo, hi, mu=1.0 / 1600.0, Pr=0.72)
    bx, by, bz = block
    cells = [i + n * (j + n * k) for k in range(bz) for j in range(by) for i in range(bx)]
    dt = 1e-3
    # a small calibration block, then a block sized to about steps_budget_s
    t0 = time.perf_counter()
    oracle.operator(cfg, q, dt, cells=cells[: bx * by * 2])
    t_cal = time.perf_counter() - t0
    ncal = bx * by * 2
    want = int(min(len(cells), max(ncal, steps_budget_s / max(t_cal, 1e-6) * ncal)))
    sample = cells[:want]
    t0 = time.perf_counter()
    oracle.operator(cfg, q, dt, cells=sample)
    el = time.perf_counter() - t0
    return {"value": len(sample) / el, "unit": UNIT, "cores": oracle.threads_used(cfg), "kind": "oracle",
            "sample": f"one stage (L and dL/dt) of {len(sample)} contiguous cells of TGV {n}^3, FP64, "
                      f"{el:.1f} s"}


def run_reference(args, rank):
    """The oracle timed as the reference arm: each step is one two-stage step
    (two operator evaluations) over a bounded block of TGV 128^3 cells."""
    import oracle
    n = args.n
    q, lo, hi = workload(n)
    cfg = oracle.make_cfg((n, n, n), lo, hi, mu=1.0 / 1600.0, Pr=0.72)
    bx, by, bz = 16, 16, 8
    cells = [i + n * (j + n * k) for k in range(bz) for j in range(by) for i in range(bx)]
    dt = 1e-3
    for _ in range(args.warmup):
        oracle.operator(cfg, q, dt, cells=cells)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.operator(cfg, q, dt, cells=cells)
        oracle.operator(cfg, q, dt, cells=cells)
    el = time.perf_counter() - t0
    value = len(cells) * 2 * args.steps / el
    cores = oracle.threads_used(cfg)
    sample = f"per step two operator evaluations over {len(cells)} contiguous cells of TGV {n}^3 (FP64)"
    return {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"Taylor-Green vortex {n}^3, Re 1600, Mach 0.1, Pr 0.72"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the small serving run of the default line")
    ap.add_argument("--no-moving", action="store_true", help="skip the 96^3 moving-mesh run of the default line")
    ap.add_argument("--moving-n", type=int, default=96, help="cells per axis of the moving-mesh run")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the octant-Riemann and isotropic-turbulence runs of the default line")
    ap.add_argument("--serving", action="store_true",
                    help="only the serving benchmark: 64 requests on 24^3..96^3, printed as its own line")
    ap.add_argument("--serving-steps-max", type=int, default=80)
    args = ap.parse_args()
    rank, world, local = _dist_env()

    if args.serving:
        if rank == 0:
            import torch
            torch.cuda.set_device(local)
            res = serving_run(count=64, sizes=(24, 32, 48, 64, 96), steps=(20, args.serving_steps_max), seed=0)
            print(json.dumps({"metric": "serving time-to-solution p50/p99 (continuous batching vs one at a time)",
                              "unit": "s", "higher_is_better": False, "data": "synthetic", **res}))
        return

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank)))
        return

    dist = None
    if world > 1:
        import torch.distributed as tdist
        import torch
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    res = run_gpu(args, rank, world, local, dist)
    if rank == 0:
        main_r = res["fp64"]
        line = {
            "metric": METRIC,
            "value": main_r["value"],
            "unit": UNIT,
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": main_r["ms_per_step"],
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"Taylor-Green vortex {args.n}^3 (periodic [-pi,pi]^3, Re 1600, Mach 0.1, "
                                   f"Pr 0.72, CFL 0.35), FP64 plain path",
                       "cells": args.n ** 3, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (about 2 GB touched per step)"},
            "roofline": main_r["roofline"],
            "clocks": main_r["clocks"],
            "gpu_launches": main_r["launches"],
            "phase_ms_per_step": main_r["phase_ms_per_step"],
            "mixed": {k: res["mixed"][k] for k in ("value", "ms_per_step", "roofline", "clocks", "launches",
                                                   "phase_ms_per_step") if k in res["mixed"]},
        }
        if "e2e" in main_r:
            line["e2e"] = main_r["e2e"]
            line["mixed"]["e2e"] = res["mixed"].get("e2e")
        if not args.no_moving and world == 1:
            line["moving_mesh"] = moving_run(steps=max(1, min(args.steps, 5)), warmup=2, n=args.moving_n)
        if not args.no_workloads and world == 1:
            line["octant_riemann"] = octant_run(steps=max(1, min(args.steps, 5)), warmup=2)
            line["isotropic_turbulence"] = turbulence_run(steps=max(1, min(args.steps, 5)), warmup=2)
        if not args.no_serving and world == 1:
            line["serving"] = serving_run()
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(args.n)
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
