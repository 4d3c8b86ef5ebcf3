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

# Work per unit of the dominant kernel (the Gauss-point face flux), the
# executed thread instructions of one ncu capture of the current build on a
# TGV 64^3 x-face launch (smsp__sass_thread_inst_executed_op_{dfma,dadd,dmul,
# ffma,fadd,fmul}_pred_on over its 1,064,960 Gauss points; 2 flop per FMA):
#   FP64 path:  1046.2 DFMA + 121.5 DADD + 411.0 DMUL = 2625 flop, 1579 FP64 instructions
#   mixed path: 965 FFMA + 111 FADD + 414 FMUL        = 2455 flop, 1490 FP32 instructions
# DRAM bytes per face (read + write) of one launch at 128^3 (inputs larger
# than L2), from `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum`.
FLUX_FLOP_PER_GP = {"fp64": 2625.0, "mixed": 2455.0}
FLUX_INST_PER_GP = {"fp64": 1579.0, "mixed": 1490.0}
# x-face launch of TGV 128^3 (2,113,536 faces): FP64 854.36 MB read + 157.89 MB
# written in 23.48 ms, mixed 511.24 MB + 151.72 MB in 0.492 ms (ncu, cold L2;
# the mixed records carry 2 unused floats per variable: 240 B read per face)
FLUX_TRAFFIC_BYTES_PER_FACE = {"fp64": (854355200 + 157892608) / 2113536,
                               "mixed": (511244288 + 151715072) / 2113536}
# the algorithmic bytes per face: the two cells' reconstruction records
# (Q_c and 9 coefficients of 5 variables) read once per face pair of a
# cell, i.e. one record per face, and the face's 10 FP64 sums written once
FLUX_ALGO_BYTES_PER_FACE = {"fp64": 50 * 8 + 10 * 8, "mixed": 50 * 4 + 10 * 8}
# GB300 ALU peaks derived from unit counts and clocks (the note beside the
# measured ones): 152 SMs x 2070 MHz x (FP64: 2 DFMA/clk/SM = 4 flop;
# FP32: 128 FMA/clk/SM = 256 flop).
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
PEAK_DERIVED_TFLOPS = {"fp64": SM_COUNT * SM_MAX_MHZ * 1e6 * 4 / 1e12,
                       "mixed": SM_COUNT * SM_MAX_MHZ * 1e6 * 256 / 1e12}


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


# the block of TGV cells whose operator the CPU-baseline leg evaluates with
# the oracle (x fastest, from the origin), and the dt of that evaluation
CPU_BLOCK = (32, 32, 16)
CPU_DT = 1e-3


def block_cells(n, block=CPU_BLOCK):
    bx, by, bz = block
    return [i + n * (j + n * k) for k in range(bz) for j in range(by) for i in range(bx)]


def measured_alu_peaks():
    """FMA rates of the FP64 and FP32 pipes of this GPU, measured by the
    library's probe (independent FMA chains on every SM, CUDA events)."""
    from paper_1909_01580_gb300 import hgks
    return {"fp64": hgks.hgks_alu_peak(hgks.HGKS_FP64), "mixed": hgks.hgks_alu_peak(hgks.HGKS_MIXED)}


def flux_roofline(prec_name, n, flux_ms, flux_launches, peaks):
    """Roofline of the Gauss-point flux kernel from its live CUDA-event time:
    Gauss points per launch x flop per Gauss point / time per launch."""
    nface_launch = n * n * (n + 1)
    gp_per_launch = 4 * nface_launch
    per_launch_s = flux_ms / 1e3 / max(flux_launches, 1)
    flop_gp = FLUX_FLOP_PER_GP[prec_name]
    achieved = gp_per_launch * flop_gp / per_launch_s / 1e12
    peak = peaks[prec_name]
    traffic_face = FLUX_TRAFFIC_BYTES_PER_FACE[prec_name]
    pipe = "fp64" if prec_name == "fp64" else "fp32"
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic_face * nface_launch if traffic_face is not None else None,
            "algorithmic_bytes": FLUX_ALGO_BYTES_PER_FACE[prec_name] * nface_launch,
            "kernel": "k_face_flux", "pipe": pipe, "launch_ms": per_launch_s * 1e3,
            "work": f"{gp_per_launch} Gauss points per launch x {flop_gp:.0f} {pipe.upper()} flop per Gauss point "
                    "(executed-instruction count of an ncu capture of this build)",
            # the kernel's share of the pipe's issue rate: instructions per Gauss
            # point against the measured FMA rate (one instruction per FMA)
            "issue_frac": gp_per_launch * FLUX_INST_PER_GP[prec_name] / per_launch_s / (peak * 1e12 / 2),
            "peak_source": f"measured: hgks_alu_peak ({pipe.upper()} FMA chains on every SM) = {peak:.3f} TFLOP/s; "
                           f"derived 152 SMs x 2070 MHz x {4 if pipe == 'fp64' else 256} flop/clk/SM = "
                           f"{PEAK_DERIVED_TFLOPS[prec_name]:.3f}"}


def mixed_accuracy(n, lo, hi, q0, nsteps, solver_kw=None, options=None, cfl=0.35):
    """Error of the mixed path against the FP64 path (which the parity tests
    hold to the oracle) after nsteps two-stage steps of one fixed dt (the
    FP64 CFL step of the initial state) from the same initial state: L1
    (volume-weighted with the reference cell volume) and L_inf of the density
    and the energy, and the largest per-variable max |diff| / max |Q|."""
    from paper_1909_01580_gb300 import hgks
    states, dt = {}, None
    for name, prec in (("fp64", hgks.HGKS_FP64), ("mixed", hgks.HGKS_MIXED)):
        s = hgks.Solver(n, lo, hi, precision=prec, **(solver_kw or {}))
        for k, v in (options or {}).items():
            hgks.hgks_set_option(s.h, k, v)
        if dt is None:
            s.set_state(q0, t=0.0)
            dt, _ = s.step(1, cfl=cfl)
        s.set_state(q0, t=0.0)
        t, done = s.step(nsteps, dt_fixed=dt)
        states[name], _ = s.get_state()
        s.close()
    ref, d = states["fp64"], states["mixed"] - states["fp64"]
    vol = float(np.prod([(hi[a] - lo[a]) / n[a] for a in range(3)]))
    rel = [float(np.abs(d[v]).max() / max(np.abs(ref[v]).max(), 1e-300)) for v in range(5)]
    return {"steps": nsteps, "dt": dt, "reference": "FP64 GPU path, same initial state and fixed dt",
            "l1_rho": float(np.abs(d[0]).sum() * vol), "linf_rho": float(np.abs(d[0]).max()),
            "l1_rhoE": float(np.abs(d[4]).sum() * vol), "linf_rhoE": float(np.abs(d[4]).max()),
            "max_rel": max(rel)}


def run_gpu(args, rank, world, local, dist):
    import torch
    from paper_1909_01580_gb300 import hgks

    torch.cuda.set_device(local)
    hgks.load()
    n = args.n
    q0, lo, hi = workload(n)
    ncell = n ** 3
    mu, Pr = 1.0 / 1600.0, 0.72
    peaks = measured_alu_peaks()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    slowest = functools.partial(max_over_ranks, dist=dist, device="cuda")

    results = {}
    for prec_name, prec in (("fp64", hgks.HGKS_FP64), ("mixed", hgks.HGKS_MIXED)):
        stream = torch.cuda.Stream()
        s = hgks.Solver((n, n, n), lo, hi, mu=mu, Pr=Pr, precision=prec, stream=stream.cuda_stream)
        # the operator at the initial state on the block of cells the
        # CPU-baseline leg evaluates with the oracle
        s.set_state(q0, t=0.0)
        L, dL = s.flux(CPU_DT)
        cells = block_cells(n)
        op_block = (L.reshape(5, -1)[:, cells].copy(), dL.reshape(5, -1)[:, cells].copy())
        del L, dL
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
        flux_ms, flux_launches = timing["flux"]
        total_phase = sum(v[0] for v in timing.values())
        results[prec_name] = {
            "value": replicas_rate(world, ncell * 2 * args.steps, ms_max / 1e3),
            "ms_per_step": ms_max / args.steps,
            "launches": launches,
            "clocks": clocks,
            "phase_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in timing.items()},
            "flux_share": flux_ms / total_phase if total_phase > 0 else None,
            "roofline": flux_roofline(prec_name, n, flux_ms, flux_launches, peaks),
            "t_reached": t_now,
            "op_block": op_block,
        }
        # end to end through the C ABI with host buffers: every step loads the
        # state from pinned host memory and reads the result back out (the
        # library's kernels read and write the pinned buffers directly)
        if not args.no_e2e:
            qh = torch.from_numpy(q0).pin_memory()
            qh_np = qh.numpy()
            out = torch.empty_like(qh).pin_memory()
            out_np = out.numpy()
            e2e_steps = max(1, min(args.steps, 5))
            # one untimed pass of the same calls first
            hgks.hgks_set_state(s.h, qh_np, 0.0)
            s.step(1, cfl=0.35)
            hgks.hgks_get_state(s.h, out_np)
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
    if world == 1 and not args.no_accuracy:
        results["mixed"]["err_vs_fp64"] = mixed_accuracy((n, n, n), lo, hi, q0, args.warmup + args.steps,
                                                         solver_kw={"mu": mu, "Pr": Pr})
    results["peaks"] = peaks
    return results


def moving_run(steps, warmup, n=96, accuracy=True):
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
    if accuracy:
        out["mixed"]["err_vs_fp64"] = mixed_accuracy((n, n, n), (0, 0, 0), (2, 2, 2), q0, warmup + steps,
                                                     solver_kw={"mesh": 2, "mesh_amp": 0.05,
                                                                "mesh_omega": 2 * math.pi})
    return out


def workload_run(name, q0, lo, hi, steps, warmup, solver_kw=None, options=None, accuracy=True):
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
    if accuracy:
        out["mixed"]["err_vs_fp64"] = mixed_accuracy(n, lo, hi, q0, warmup + steps, solver_kw=solver_kw,
                                                     options=options)
    return out


def octant_run(steps, warmup, n=128, accuracy=True):
    from paper_1909_01580_gb300 import workloads
    q0 = workloads.octant_riemann((n, n, n), seed=0)
    return workload_run(f"octant Riemann problem {n}^3 on [0,1]^3, reflective walls, seed 0, CFL 0.35", q0,
                        (0, 0, 0), (1, 1, 1), steps, warmup, solver_kw={"bc": (1,) * 6}, accuracy=accuracy)


def turbulence_run(steps, warmup, n=128, mach=0.5, accuracy=True):
    from paper_1909_01580_gb300 import workloads
    q0, lo, hi, P = workloads.isotropic_turbulence(n, mach, seed=0)
    return workload_run(f"compressible isotropic turbulence {n}^3, Ma_t {mach}, Re_lambda 72, mu ~ T^0.76, Pr 0.7",
                        q0, lo, hi, steps, warmup, solver_kw={"mu": P.mu0, "Pr": 0.7},
                        options={"mu_power": 0.76, "mu_T_ref": P.T0}, accuracy=accuracy)


def serving_run(count=64, sizes=(24, 32, 48, 64, 96), steps=(4, 16), seed=0, load=1.25, arena_gb=4.0,
                precisions=("fp64", "mixed")):
    """Serving workload: seeded requests (density advection / TGV 50:50,
    uniform over the sizes, Mach U[0.05, 0.3], Re U[400, 3200], log-uniform
    CFL steps in the range).  For each precision: one-at-a-time solves of
    every request (a handle each) give the service times; arrivals are
    Poisson at `load` times that precision's own sequential capacity; the
    continuous-batching loop then serves the same arrivals in real time from
    an arena of arena_gb GB (admission by HBM footprint), admitting every
    arrival that fits ("fifo") or the least work first with an age limit of
    twice the mean service time and a cap on the resident cells ("aged")."""
    from paper_1909_01580_gb300 import hgks, serving
    reqs = serving.request_stream(count=count, seed=seed, sizes=sizes, steps=steps)
    out = {"requests": count, "sizes": list(sizes), "steps": list(steps), "seed": seed,
           "load_vs_sequential": load, "arena_gb": arena_gb,
           "approx_cell_stages": sum(2 * r.cells * r.steps_target for r in reqs)}
    caps = {"fp64": 120_000, "mixed": 2_000_000}
    for name in precisions:
        prec = hgks.HGKS_FP64 if name == "fp64" else hgks.HGKS_MIXED
        fifo = serving.serve_fifo(reqs, precision=prec)
        rate = load * count / fifo["busy"]
        serving.poisson_arrivals(reqs, rate, seed=seed)
        base = serving.fifo_latencies(reqs, fifo["service"])
        arm = {"arrival_rate_per_s": rate, "mean_service_s": fifo["busy"] / count,
               "one_at_a_time": serving.summary(f"one_at_a_time_{name}", base, reqs)}
        age = 2.0 * fifo["busy"] / count
        for policy in ("fifo", "aged"):
            res = serving.serve_batched(reqs, precision=prec, arena_bytes=int(arena_gb * (1 << 30)),
                                        max_instances=64, steps_per_poll=4, keep_results=False, policy=policy,
                                        max_resident_cells=caps[name] if policy == "aged" else None,
                                        age_limit=age if policy == "aged" else None)
            sm = serving.summary(f"batched_{name}_{policy}", res, reqs)
            sm["policy"] = ("every arrival that fits" if policy == "fifo" else
                            f"least work first, age limit {age:.3f} s, resident cells <= {caps[name]}")
            sm["max_resident"] = res["max_resident"]
            sm["gpu_launches"] = res["launches"]
            sm["cell_stage_updates_per_s"] = res["cell_stages"] / res["makespan"]
            arm[f"batched_{policy}"] = sm
        out[name] = arm
    return out


def cpu_baseline(n, gpu_ops=None, budget_s=8.0):
    """The oracle as it stands on the host cores: one operator evaluation (one
    stage's reconstruction and face fluxes, L and dL/dt) over a prefix of a
    contiguous block of TGV 128^3 cells, scaled to cell-stage updates/s, on
    all cores and on one thread.  With gpu_ops (the GPU paths' L and dL/dt on
    the same block at the same state and dt) the oracle's values are also
    compared with them: per-variable max |diff| / max |oracle|."""
    import oracle
    q, lo, hi = workload(n)
    cells = block_cells(n)
    out = {"kind": "oracle", "unit": UNIT}
    lo_all = None
    for label, threads in (("all_cores", 0), ("one_thread", 1)):
        cfg = oracle.make_cfg((n, n, n), lo, hi, mu=1.0 / 1600.0, Pr=0.72, nthreads=threads)
        ncal = 256
        t0 = time.perf_counter()
        oracle.operator(cfg, q, CPU_DT, cells=cells[:ncal])
        t_cal = time.perf_counter() - t0
        want = int(min(len(cells), max(ncal, budget_s / max(t_cal, 1e-6) * ncal)))
        t0 = time.perf_counter()
        Lo, dLo = oracle.operator(cfg, q, CPU_DT, cells=cells[:want])
        el = time.perf_counter() - t0
        out[label] = {"value": want / el, "cores": oracle.threads_used(cfg),
                      "sample": f"one stage (L and dL/dt) of the first {want} cells of a {CPU_BLOCK[0]}x"
                                f"{CPU_BLOCK[1]}x{CPU_BLOCK[2]} block of TGV {n}^3, FP64, {el:.1f} s"}
        if label == "all_cores":
            lo_all = (want, Lo, dLo)
    out["value"] = out["all_cores"]["value"]
    out["cores"] = out["all_cores"]["cores"]
    out["sample"] = out["all_cores"]["sample"]
    if gpu_ops and lo_all is not None:
        want, Lo, dLo = lo_all
        par = {}
        for name, (L, dL) in gpu_ops.items():
            par[name] = {
                "L": max(float(np.abs(L[v, :want] - Lo[v]).max() / max(np.abs(Lo[v]).max(), 1e-300))
                         for v in range(5)),
                "dL_dt": max(float(np.abs(dL[v, :want] - dLo[v]).max() / max(np.abs(dLo[v]).max(), 1e-300))
                             for v in range(5)),
                "cells": want}
        out["gpu_vs_oracle"] = par
    return out


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
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the error statements of the mixed results against the FP64 path")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving run of the default line")
    ap.add_argument("--no-moving", action="store_true", help="skip the 96^3 moving-mesh run of the default line")
    ap.add_argument("--moving-n", type=int, default=96, help="cells per axis of the moving-mesh run")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the octant-Riemann and isotropic-turbulence runs of the default line")
    ap.add_argument("--serving", action="store_true",
                    help="only the serving benchmark (64 requests on 24^3..96^3), printed as its own line")
    ap.add_argument("--serving-steps", type=str, default="4,16",
                    help="range of CFL steps per serving request (log-uniform)")
    args = ap.parse_args()
    rank, world, local = _dist_env()
    serving_steps = tuple(int(x) for x in args.serving_steps.split(","))

    if args.serving:
        if rank == 0:
            import torch
            torch.cuda.set_device(local)
            res = serving_run(count=64, sizes=(24, 32, 48, 64, 96), steps=serving_steps, seed=0)
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
            "alu_peaks_measured_tflops": res["peaks"],
            "mixed": {k: res["mixed"][k] for k in ("value", "ms_per_step", "roofline", "clocks", "launches",
                                                   "phase_ms_per_step", "err_vs_fp64") if k in res["mixed"]},
        }
        if "e2e" in main_r:
            line["e2e"] = main_r["e2e"]
            line["mixed"]["e2e"] = res["mixed"].get("e2e")
        acc = not args.no_accuracy
        if not args.no_moving and world == 1:
            line["moving_mesh"] = moving_run(steps=max(1, min(args.steps, 5)), warmup=2, n=args.moving_n,
                                             accuracy=acc)
        if not args.no_workloads and world == 1:
            line["octant_riemann"] = octant_run(steps=max(1, min(args.steps, 5)), warmup=2, accuracy=acc)
            line["isotropic_turbulence"] = turbulence_run(steps=max(1, min(args.steps, 5)), warmup=2, accuracy=acc)
        if not args.no_serving and world == 1:
            line["serving"] = serving_run(steps=serving_steps)
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(args.n, gpu_ops={k: res[k]["op_block"] for k in ("fp64", "mixed")})
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
