"""Failure handling of the serving path and checkpoint/resume, through the C
ABI: a request whose state is not physical is refused at admission while
the resident requests finish bit-identical to a run without it; a request
cancelled in mid-run frees its slot and arena memory without changing the
others; a state read back with hgks_get_state and loaded into a new handle
resumes bit-identically."""
import numpy as np
import pytest

from paper_1909_01580_gb300 import hgks, serving
from paper_1909_01580_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    hgks.load()


def _stream(count, seed):
    reqs = serving.request_stream(count=count, seed=seed, sizes=(8, 12, 16), steps=(5, 20))
    for r in reqs:
        r.arrival = 0.0
    return reqs


@pytest.mark.parametrize("bad", ["nan", "negative_pressure"])
def test_nonphysical_request_refused_others_bitwise_unchanged(bad):
    reqs = _stream(5, seed=7)
    x = serving.make_request(99, "tgv", 12, 0.1, 800.0, 10)
    x.arrival = 0.0
    if bad == "nan":
        x.q0[0, 2, 3, 4] = np.nan
    else:
        x.q0[4, 1, 1, 1] = 0.0  # energy below the kinetic energy: p < 0
    clean = serving.serve_batched(reqs, precision=hgks.HGKS_FP64, arena_bytes=256 << 20, max_instances=8)
    mixed = serving.serve_batched(reqs[:2] + [x] + reqs[2:], precision=hgks.HGKS_FP64, arena_bytes=256 << 20,
                                  max_instances=8)
    assert list(mixed["rejected"]) == [99]
    assert not clean["rejected"]
    assert sorted(mixed["results"]) == sorted(clean["results"]) == [r.rid for r in reqs]
    for rid, q in clean["results"].items():
        assert np.array_equal(mixed["results"][rid], q), rid


def _run_batch(entries, remove_after=None, add_later=None, precision=hgks.HGKS_FP64):
    """entries: requests admitted at once; remove_after: (rid, steps) to cancel
    one after that many batch steps; add_later: a request admitted right
    after the cancel.  Returns {rid: final state} of the requests that finish."""
    b = hgks.Batch(precision, arena_bytes=128 << 20, max_instances=4)
    slots = {}

    def admit(r):
        slots[b.add((r.n,) * 3, r.lo, r.hi, r.q0, t0=0.0, t_end=r.t_end, mu=r.mu, Pr=r.Pr)] = r.rid

    for r in entries:
        admit(r)
    done, steps = {}, 0
    while slots:
        b.step(1)
        steps += 1
        if remove_after is not None and steps == remove_after[1]:
            sl = [s for s, rid in slots.items() if rid == remove_after[0]][0]
            b.remove(sl)
            del slots[sl]
            if add_later is not None:
                admit(add_later)
        t, st, state = b.poll()
        for sl in list(slots):
            assert state[sl] != 3
            if state[sl] == 2:
                done[slots.pop(sl)] = b.get_state(sl)
                b.remove(sl)
    b.close()
    return done


@pytest.mark.parametrize("precision", [hgks.HGKS_FP64, hgks.HGKS_MIXED])
def test_cancel_mid_run_leaves_the_others_bitwise_unchanged(precision):
    a, c, d = _stream(3, seed=11)
    alone_c = _run_batch([c], precision=precision)
    alone_d = _run_batch([d], precision=precision)
    mix = _run_batch([a, c], remove_after=(a.rid, 3), add_later=d, precision=precision)
    assert a.rid not in mix
    assert np.array_equal(mix[c.rid], alone_c[c.rid])
    assert np.array_equal(mix[d.rid], alone_d[d.rid])


@pytest.mark.parametrize("precision", [hgks.HGKS_FP64, hgks.HGKS_MIXED])
def test_checkpoint_resume_is_bitwise(precision):
    n = (16, 16, 16)
    q0, lo, hi = W.taylor_green(n)
    kw = dict(mu=1.0 / 1600, Pr=0.72, precision=precision)
    s = hgks.Solver(n, lo, hi, **kw)
    s.set_state(q0)
    t10, done = s.step(10, cfl=0.35)
    q10, _ = s.get_state()
    s.close()
    s = hgks.Solver(n, lo, hi, **kw)
    s.set_state(q0)
    s.step(5, cfl=0.35)
    q5, t5 = s.get_state()
    s.close()
    r = hgks.Solver(n, lo, hi, **kw)
    r.set_state(q5, t=t5)
    t, done2 = r.step(5, cfl=0.35)
    q, tq = r.get_state()
    r.close()
    assert done == 10 and done2 == 5
    assert t == t10 and tq == t10
    assert np.array_equal(q, q10)
