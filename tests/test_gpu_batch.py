"""Batched persistent execution (tile table, CUDA graph, autotuner) and the
serving loop: through the C ABI, every instance of a batch computes exactly
what it computes alone, also when instances join, finish and leave at
different times; admission is bounded by the arena (HBM footprint)."""
import numpy as np
import pytest

from paper_1909_01580_gb300 import hgks, serving
from paper_1909_01580_gb300 import workloads as W
from tests._cases import max_rel, max_rel_momentum

pytestmark = pytest.mark.gpu


def _cases():
    adv = ((8, 8, 8), (0, 0, 0), (2, 2, 2), W.density_advection((8, 8, 8)), dict())
    q, lo, hi = W.taylor_green((12, 12, 12))
    tgv = ((12, 12, 12), lo, hi, q, dict(mu=1.0 / 800, Pr=0.72))
    n = (10, 9, 7)
    lo3, hi3 = (0, 0, 0), (1.0, 0.9, 0.7)
    smooth = (n, lo3, hi3, W.smooth_random(n, seed=3, lo=lo3, hi=hi3, amp=0.15), dict(bc=(1,) * 6))
    oct_ = ((16, 16, 16), (0, 0, 0), (1, 1, 1), W.octant_riemann((16, 16, 16), seed=2), dict(bc=(1,) * 6))
    return [adv, tgv, smooth, oct_]


def _alone(n, lo, hi, q, kw, t_end, precision, nsteps=100000):
    s = hgks.Solver(n, lo, hi, precision=precision, **kw)
    s.set_state(q)
    t, done = s.step(nsteps, cfl=0.35, t_end=t_end)
    out, _ = s.get_state()
    s.close()
    return out, t, done


@pytest.mark.parametrize("precision", [hgks.HGKS_FP64, hgks.HGKS_MIXED])
def test_batch_equals_alone_with_staggered_join_and_end(precision):
    hgks.load()
    cases = _cases()
    ends = [0.05, 0.02, 0.03, 0.04]
    b = hgks.Batch(precision, arena_bytes=256 << 20, max_instances=8)
    slots = []
    for (n, lo, hi, q, kw), te in zip(cases[:3], ends[:3]):
        slots.append(b.add(n, lo, hi, q, t_end=te, **kw))
    b.step(3)
    # the fourth joins after three batch steps
    n, lo, hi, q, kw = cases[3]
    slots.append(b.add(n, lo, hi, q, t_end=ends[3], **kw))
    for _ in range(200):
        b.step(2)
        t, steps, state = b.poll()
        if all(state[s] == 2 for s in slots):
            break
    t, steps, state = b.poll()
    assert all(state[s] == 2 for s in slots), state
    for (n, lo, hi, q, kw), te, sl in zip(cases, ends, slots):
        qa, ta, da = _alone(n, lo, hi, q, kw, te, precision)
        qb = b.get_state(sl)
        assert steps[sl] == da and abs(t[sl] - ta) == 0.0
        # FP64: the FP64 parity bar (the batched and solo kernels run the same
        # item code; the compiler may fuse multiply-adds differently in the
        # two); mixed: FP32 round-off, judged on the state's common scale (the
        # TGV's rho W starts at zero)
        if precision == hgks.HGKS_FP64:
            assert max_rel(qb, qa) <= 1e-11, max_rel(qb, qa)
        else:
            assert np.abs(qb - qa).max() <= 1e-6 * np.abs(qa).max()
    assert b.launches > 0
    b.close()


def test_admission_bounded_by_arena():
    hgks.load()
    n = (16, 16, 16)
    need = hgks.hgks_batch_footprint(n, (0, 0, 0), (2, 2, 2))
    assert need > 0
    b = hgks.Batch(hgks.HGKS_FP64, arena_bytes=int(2.5 * need), max_instances=8)
    q = W.density_advection(n)
    s0 = b.add(n, (0, 0, 0), (2, 2, 2), q, t_end=0.1)
    s1 = b.add(n, (0, 0, 0), (2, 2, 2), q, t_end=0.1)
    with pytest.raises(hgks.HgksError) as e:
        b.add(n, (0, 0, 0), (2, 2, 2), q, t_end=0.1)
    assert e.value.code == hgks.HGKS_E_NOMEM
    b.remove(s0)
    s2 = b.add(n, (0, 0, 0), (2, 2, 2), q, t_end=0.1)
    assert s2 == s0
    b.close()


def test_autotuner_keeps_results_exact():
    """Tuning changes tile sizes, persistent grids and the schedule, never the
    arithmetic of an item: a tuned batch is bit-identical to an untuned one,
    and both are within the FP64 parity bar of the solo runs (the batched and
    solo kernels inline the same item code, but the compiler may fuse
    multiply-adds differently in the two)."""
    hgks.load()
    cases = _cases()
    tuned = hgks.Batch(hgks.HGKS_FP64, arena_bytes=256 << 20, max_instances=8)
    plain = hgks.Batch(hgks.HGKS_FP64, arena_bytes=256 << 20, max_instances=8)
    slots = [tuned.add(n, lo, hi, q, t_end=10.0, **kw) for (n, lo, hi, q, kw) in cases]
    pslots = [plain.add(n, lo, hi, q, t_end=10.0, **kw) for (n, lo, hi, q, kw) in cases]
    params = tuned.tune(steps_per_trial=1)
    assert len(params) == hgks.HGKS_TUNE_NPARAM and params[0] in (0, 1, 2)
    assert tuned.get_tuning() == params
    tuned.step(2)
    t, steps, state = tuned.poll()
    # bring the untuned batch to the same step counts (tuning trials advanced
    # the tuned instances)
    assert len({int(steps[sl]) for sl in slots}) == 1  # every instance took every step
    plain.step(int(steps[slots[0]]))
    tp, sp, _ = plain.poll()
    for (n, lo, hi, q, kw), sl, ps in zip(cases, slots, pslots):
        assert sp[ps] == steps[sl]
        assert max_rel(tuned.get_state(sl), plain.get_state(ps)) == 0.0
        qa, ta, da = _alone(n, lo, hi, q, kw, 10.0, hgks.HGKS_FP64, nsteps=int(steps[sl]))
        assert max_rel(tuned.get_state(sl), qa) <= 1e-11
    tuned.close()
    plain.close()


def test_serving_results_same_alone_and_in_the_mix():
    """Continuous batching: six requests arrive while others run, share the
    GPU, and each result equals its solve alone (FP64, identical arithmetic)."""
    hgks.load()
    reqs = serving.request_stream(count=6, seed=4, sizes=(8, 12, 16), steps=(5, 20))
    serving.poisson_arrivals(reqs, rate=200.0, seed=4)
    out = serving.serve_batched(reqs, precision=hgks.HGKS_FP64, arena_bytes=256 << 20, max_instances=8,
                                steps_per_poll=2)
    assert out["max_resident"] >= 2
    assert set(out["latency"]) == {r.rid for r in reqs}
    for r in reqs:
        qa, _ = serving.solve_alone(r)
        assert max_rel(out["results"][r.rid], qa) <= 1e-11
    fifo = serving.serve_fifo(reqs)
    assert set(fifo["latency"]) == {r.rid for r in reqs}


@pytest.mark.parametrize("precision,tol", [(hgks.HGKS_FP64, 1e-11), (hgks.HGKS_MIXED, 1e-4)])
def test_batch_instances_against_the_oracle(precision, tol):
    """Every instance of a batch (staggered ends, reflective and periodic
    boxes) against the FP64 oracle run with the same CFL steps to the same
    end time: FP64 per variable <= 1e-11, mixed <= 1e-4 (the FP32
    reconstruction and flux; the momenta against the momentum scale, since
    rho W of the Taylor-Green vortex starts at zero)."""
    import oracle
    hgks.load()
    cases = _cases()[:3]
    ends = [0.05, 0.02, 0.03]
    b = hgks.Batch(precision, arena_bytes=256 << 20, max_instances=4)
    slots = [b.add(n, lo, hi, q, t0=0.0, t_end=te, **kw) for (n, lo, hi, q, kw), te in zip(cases, ends)]
    while True:
        b.step(2)
        t, steps, state = b.poll()
        if all(state[sl] == 2 for sl in slots):
            break
        assert not any(state[sl] == 3 for sl in slots)
    for sl, (n, lo, hi, q, kw), te in zip(slots, cases, ends):
        cfg = oracle.make_cfg(n, lo, hi, **kw)
        qo, to, done_o, _ = oracle.step(cfg, q, 0.0, 100000, cfl=0.35, t_end=te)
        assert abs(t[sl] - to) < 1e-13 and steps[sl] == done_o, (t[sl], to, steps[sl], done_o)
        qb = b.get_state(sl)
        err = max_rel(qb, qo) if precision == hgks.HGKS_FP64 else max_rel_momentum(qb, qo)
        assert err <= tol, (sl, err)
    b.close()


def test_served_requests_against_the_oracle():
    """Requests served by continuous batching (FP64) against the oracle's
    run of the same request to its end time, per variable <= 1e-11."""
    import oracle
    hgks.load()
    reqs = serving.request_stream(count=3, seed=9, sizes=(8, 12), steps=(4, 10))
    serving.poisson_arrivals(reqs, rate=500.0, seed=9)
    out = serving.serve_batched(reqs, precision=hgks.HGKS_FP64, arena_bytes=128 << 20, max_instances=4,
                                steps_per_poll=2)
    for r in reqs:
        cfg = oracle.make_cfg((r.n,) * 3, r.lo, r.hi, mu=r.mu, Pr=r.Pr)
        qo, to, _, _ = oracle.step(cfg, r.q0, 0.0, 100000, cfl=0.35, t_end=r.t_end)
        assert max_rel(out["results"][r.rid], qo) <= 1e-11, (r.rid, max_rel(out["results"][r.rid], qo))
