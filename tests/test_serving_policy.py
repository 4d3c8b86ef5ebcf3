"""Admission policy of the serving loop (host logic, no GPU): first come
first served or shortest estimated work first, with a cap on the resident
cells that always lets one request in."""
from paper_1909_01580_gb300.serving import Request, next_admission


def _req(rid, n, steps, arrival):
    return Request(rid=rid, kind="advection", n=n, mach=0.1, re=1000.0, steps_target=steps, arrival=arrival)


def test_fifo_takes_the_oldest():
    w = [_req(0, 64, 100, 0.0), _req(1, 24, 20, 0.1)]
    assert next_admission(w, 0, "fifo") == 0


def test_sjf_takes_the_least_work_and_breaks_ties_by_arrival():
    w = [_req(0, 64, 100, 0.0), _req(1, 24, 20, 0.1), _req(2, 32, 20, 0.2), _req(3, 24, 20, 0.3)]
    assert next_admission(w, 0, "sjf") == 1
    # 24^3 x 20 steps = 276,480 cell-steps is less work than 32^3 x 10 = 327,680
    w2 = [_req(0, 32, 10, 0.0), _req(1, 24, 20, 0.1)]
    assert next_admission(w2, 0, "sjf") == 1


def test_cap_on_resident_cells():
    w = [_req(0, 48, 20, 0.0)]
    assert next_admission(w, 0, "sjf", max_resident_cells=1000) == 0  # nothing resident: always admit
    assert next_admission(w, 500, "sjf", max_resident_cells=1000) is None
    assert next_admission(w, 10_000, "sjf", max_resident_cells=200_000) == 0
    assert next_admission([], 0, "fifo") is None


def test_aged_least_work_first_lets_an_old_request_go_first():
    w = [_req(0, 96, 100, 0.0), _req(1, 24, 20, 0.5), _req(2, 32, 20, 0.6)]
    # young queue: least work first
    assert next_admission(w, 0, "aged", now=1.0, age_limit=2.0) == 1
    # the oldest request has waited past the limit: it goes first
    assert next_admission(w, 0, "aged", now=2.5, age_limit=2.0) == 0
    # the cap still applies to it
    assert next_admission(w, 50_000, "aged", max_resident_cells=100_000, now=2.5, age_limit=2.0) is None
