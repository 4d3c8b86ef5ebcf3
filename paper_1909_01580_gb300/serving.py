"""Serving loop over the batched C ABI: simulation requests of different grid
sizes, Mach and Reynolds numbers arrive as a Poisson stream; each request's
state stays resident on the device from admission to completion; requests are
admitted in arrival order as slots and arena memory (HBM footprint) free up,
so new work joins the batch while earlier work is still running (continuous
batching); every batch step is one CUDA-graph launch that advances all
resident instances.  Reported: p50/p99 time from arrival to result on the
host, and throughput, beside a one-at-a-time baseline.

The loop itself only schedules and marshals; all arithmetic runs in the
library's kernels.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import hgks
from . import workloads


@dataclass
class Request:
    rid: int
    kind: str            # "advection" or "tgv"
    n: int               # cells per axis
    mach: float
    re: float
    steps_target: int
    arrival: float = 0.0
    t_end: float = 0.0
    lo: tuple = ()
    hi: tuple = ()
    mu: float = 0.0
    Pr: float = 1.0
    q0: np.ndarray = field(default=None, repr=False)

    @property
    def cells(self):
        return self.n ** 3


def make_request(rid, kind, n, mach, re, steps_target, gamma=1.4, cfl=0.35):
    """Initial state and end time of one request.  Density advection runs
    at the requested Mach number (pressure set from |U| and M, inviscid);
    Taylor-Green at Mach M0 with mu = 1/Re, Pr = 0.72.  The end time is
    steps_target initial CFL steps."""
    r = Request(rid, kind, n, mach, re, steps_target)
    if kind == "tgv":
        q, lo, hi = workloads.taylor_green((n, n, n), mach=mach, gamma=gamma)
        r.mu, r.Pr = 1.0 / re, 0.72
    else:
        q = workloads.density_advection((n, n, n), gamma=gamma)
        # p = rho |U|^2/(gamma M^2) with |U| = sqrt(3): rescale the energy
        p = 3.0 / (gamma * mach * mach)
        rho = q[0]
        q[4] = p / (gamma - 1.0) + 0.5 * rho * 3.0
        lo, hi = (0.0, 0.0, 0.0), (2.0, 2.0, 2.0)
        r.mu, r.Pr = 0.0, 1.0
    r.lo, r.hi, r.q0 = lo, hi, np.ascontiguousarray(q)
    rho, u, v, w, p = workloads.primitive(q, gamma)
    h = (hi[0] - lo[0]) / n
    smax = float(np.max(np.sqrt(u * u + v * v + w * w) + np.sqrt(gamma * p / rho)))
    r.t_end = steps_target * cfl * h / smax
    return r


def request_stream(count=64, seed=0, sizes=(24, 32, 48, 64, 96), steps=(20, 400), mach=(0.05, 0.3),
                   re=(400.0, 3200.0)):
    """Seeded mix: type advection/TGV 50/50, size uniform over sizes, Mach
    and Re uniform, steps log-uniform in the range."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        kind = "tgv" if rng.random() < 0.5 else "advection"
        n = int(rng.choice(sizes))
        m = float(rng.uniform(*mach))
        r = float(rng.uniform(*re))
        st = int(round(math.exp(rng.uniform(math.log(steps[0]), math.log(steps[1])))))
        out.append(make_request(i, kind, n, m, r, st))
    return out


def poisson_arrivals(reqs, rate, seed=0):
    rng = np.random.default_rng(seed + 1000)
    t = 0.0
    for r in reqs:
        t += rng.exponential(1.0 / rate)
        r.arrival = t
    return reqs


def percentile(xs, q):
    """nearest-rank percentile"""
    xs = sorted(xs)
    k = max(1, int(math.ceil(q / 100.0 * len(xs))))
    return xs[k - 1]


def solve_alone(r, precision=hgks.HGKS_FP64, cfl=0.35):
    """One request on its own handle: returns (final state, seconds)."""
    import torch
    t0 = time.perf_counter()
    s = hgks.Solver((r.n,) * 3, r.lo, r.hi, mu=r.mu, Pr=r.Pr, precision=precision)
    s.set_state(r.q0)
    s.step(100000, cfl=cfl, t_end=r.t_end)
    q, _ = s.get_state()
    s.close()
    torch.cuda.synchronize()
    return q, time.perf_counter() - t0


def fifo_latencies(reqs, service):
    """Latencies of a one-at-a-time server in arrival order, from measured
    service times {rid: seconds} on a virtual clock (a request starts when it
    has arrived and the previous one has finished)."""
    clock = 0.0
    lat = {}
    for r in sorted(reqs, key=lambda x: x.arrival):
        clock = max(clock, r.arrival) + service[r.rid]
        lat[r.rid] = clock - r.arrival
    return {"latency": lat, "makespan": clock, "busy": sum(service.values())}


def serve_fifo(reqs, precision=hgks.HGKS_FP64):
    """One-at-a-time baseline in arrival order: each request is solved alone
    on the GPU (its own handle) to measure its service time."""
    service, results = {}, {}
    for r in sorted(reqs, key=lambda x: x.arrival):
        results[r.rid], service[r.rid] = solve_alone(r, precision)
    out = fifo_latencies(reqs, service)
    out["results"] = results
    out["service"] = service
    return out


def next_admission(waiting, resident_cells, policy="fifo", max_resident_cells=None, now=None, age_limit=None):
    """Index into `waiting` (requests that have arrived, in arrival order) of
    the request to admit next, or None to wait.
      policy "fifo": the oldest request;
      policy "sjf":  the request with the least estimated work (cells x
                     target steps), ties by arrival;
      policy "aged": least work first, except that a request that has waited
                     longer than age_limit seconds at time `now` goes first
                     (the oldest such request), which bounds how long the
                     largest requests can be passed over.
    With max_resident_cells, a request is admitted only while the resident
    cells stay within the cap (always when nothing is resident), so that
    the batch holds enough work to fill the GPU without sharing it among
    more requests than that needs."""
    if not waiting:
        return None
    if policy == "fifo":
        k = 0
    elif policy in ("sjf", "aged"):
        k = min(range(len(waiting)), key=lambda i: (waiting[i].cells * waiting[i].steps_target, i))
        if policy == "aged":
            if now is None or age_limit is None:
                raise ValueError("policy 'aged' needs now and age_limit")
            if now - waiting[0].arrival > age_limit:
                k = 0
    else:
        raise ValueError(f"unknown policy {policy}")
    if max_resident_cells is not None and resident_cells > 0 and \
            resident_cells + waiting[k].cells > max_resident_cells:
        return None
    return k


def serve_batched(reqs, precision=hgks.HGKS_FP64, arena_bytes=4 << 30, max_instances=64, steps_per_poll=4,
                  tuning=None, cfl=0.35, keep_results=True, policy="fifo", max_resident_cells=None, age_limit=None):
    """Continuous batching in real time: arrivals are released at their
    arrival times (relative to the start of the call), admitted by
    next_admission() when the arena and a slot are free, advanced together by
    batch steps, and read back when they reach their end time."""
    b = hgks.Batch(precision, arena_bytes=arena_bytes, max_instances=max_instances)
    if tuning is not None:
        b.set_tuning(tuning)
    pending = sorted(reqs, key=lambda x: x.arrival)
    by_slot = {}
    lat, results, admitted_at = {}, {}, {}
    cell_stages = 0
    max_resident = 0
    t_start = time.perf_counter()
    last_steps = {}
    waiting = []
    rejected = {}
    while pending or waiting or by_slot:
        now = time.perf_counter() - t_start
        while pending and pending[0].arrival <= now:
            waiting.append(pending.pop(0))
        # admit by the policy while the choice fits the arena
        while waiting:
            k = next_admission(waiting, sum(r.cells for r in by_slot.values()), policy, max_resident_cells,
                               now=now, age_limit=age_limit)
            if k is None:
                break
            r = waiting[k]
            try:
                sl = b.add((r.n,) * 3, r.lo, r.hi, r.q0, t0=0.0, t_end=r.t_end, cfl=cfl, mu=r.mu, Pr=r.Pr)
            except hgks.HgksError as e:
                if e.code == hgks.HGKS_E_NOMEM:
                    if not by_slot:
                        raise RuntimeError(f"request {r.rid} ({r.n}^3) does not fit the arena alone") from e
                    break  # wait for memory or a slot
                if e.code == hgks.HGKS_E_NONPHYSICAL:
                    # refused at admission (non-finite or non-positive state):
                    # reported, and the resident requests go on untouched
                    rejected[r.rid] = str(e)
                    waiting.pop(k)
                    continue
                raise
            by_slot[sl] = r
            admitted_at[r.rid] = now
            last_steps[sl] = 0
            waiting.pop(k)
        max_resident = max(max_resident, len(by_slot))
        if not by_slot:
            if pending and not waiting:
                time.sleep(max(0.0, pending[0].arrival - (time.perf_counter() - t_start)))
            continue
        b.step(steps_per_poll)
        t, steps, state = b.poll()
        for sl in list(by_slot):
            cell_stages += 2 * by_slot[sl].cells * (int(steps[sl]) - last_steps[sl])
            last_steps[sl] = int(steps[sl])
            if state[sl] >= 2:
                r = by_slot.pop(sl)
                if state[sl] == 3:
                    raise RuntimeError(f"request {r.rid} became nonphysical")
                q = b.get_state(sl)
                b.remove(sl)
                lat[r.rid] = time.perf_counter() - t_start - r.arrival
                if keep_results:
                    results[r.rid] = q
    makespan = time.perf_counter() - t_start
    launches = b.launches
    b.close()
    return {"latency": lat, "makespan": makespan, "results": results, "cell_stages": cell_stages,
            "launches": launches, "max_resident": max_resident, "rejected": rejected}


def summary(name, out, reqs):
    lat = list(out["latency"].values())
    return {"name": name, "p50_s": percentile(lat, 50), "p99_s": percentile(lat, 99), "mean_s": float(np.mean(lat)),
            "makespan_s": out["makespan"], "requests_per_s": len(reqs) / out["makespan"]}
