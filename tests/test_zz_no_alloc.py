"""The allocation-free entry point hgks_flux_noalloc, for callers that cannot
call cudaMalloc (a serving loop that must not block on an allocation's
implicit synchronisation, code inside another framework's memory pool):
through the C ABI its L and dL/dt equal those of hgks_flux on a handle, on
two calls in a row, and a grid too large for its fixed scratch is refused.
This file is collected last so that a run stopping at the first failure has
run every other test first."""
import numpy as np
import pytest

from paper_1909_01580_gb300 import hgks
from paper_1909_01580_gb300 import workloads as W
from tests._cases import max_rel

pytestmark = pytest.mark.gpu

TOL = 1e-11  # the parity tolerance of the FP64 path


def _reference(n, lo, hi, q, dt, **kw):
    """L, dL/dt from the handle-based entry point hgks_flux."""
    s = hgks.Solver(n, lo, hi, **kw)
    s.set_state(q)
    L, dL = s.flux(dt)
    s.close()
    return L, dL


def _noalloc(n, lo, hi, q, dt, **kw):
    import torch
    qd = torch.from_numpy(np.ascontiguousarray(q)).cuda()
    L = torch.full_like(qd, float("nan"))
    dL = torch.full_like(qd, float("nan"))
    torch.cuda.synchronize()
    hgks.hgks_flux_noalloc(n, lo, hi, qd, dt, L, dL, **kw)
    torch.cuda.synchronize()
    return L.cpu().numpy(), dL.cpu().numpy()


def test_noalloc_matches_handle_entry_point_on_consecutive_calls():
    import torch
    assert torch.cuda.is_available()
    hgks.load()
    # call 1: Taylor-Green 20^3, viscous with the Prandtl correction
    n1 = (20, 20, 20)
    q1, lo1, hi1 = W.taylor_green(n1)
    kw1 = dict(mu=1.0 / 1600, Pr=0.72)
    # call 2: a ragged smooth state with reflective walls (another layout of
    # the shared scratch, so nothing of call 1 may leak into it)
    n2 = (13, 11, 9)
    lo2, hi2 = (0.0, 0.0, 0.0), (1.0, 11.0 / 13, 9.0 / 13)
    q2 = W.smooth_random(n2, seed=5, lo=lo2, hi=hi2, amp=0.15)
    kw2 = dict(bc=(1, 1, 1, 1, 1, 1))
    for (n, lo, hi, q, kw, dt) in ((n1, lo1, hi1, q1, kw1, 1.5e-3), (n2, lo2, hi2, q2, kw2, 2e-3),
                                   (n1, lo1, hi1, q1, kw1, 1.5e-3)):
        L0, dL0 = _reference(n, lo, hi, q, dt, **kw)
        L1, dL1 = _noalloc(n, lo, hi, q, dt, **kw)
        assert np.isfinite(L1).all() and np.isfinite(dL1).all()
        assert max_rel(L1, L0) <= TOL, max_rel(L1, L0)
        assert max_rel(dL1, dL0) <= TOL, max_rel(dL1, dL0)


def test_noalloc_mixed_matches_handle():
    hgks.load()
    n = (16, 16, 16)
    q = W.density_advection(n)
    L0, dL0 = _reference(n, (0, 0, 0), (2, 2, 2), q, 0.02, precision=hgks.HGKS_MIXED)
    for _ in range(2):
        L1, dL1 = _noalloc(n, (0, 0, 0), (2, 2, 2), q, 0.02, precision=hgks.HGKS_MIXED)
        assert max_rel(L1, L0) <= TOL and max_rel(dL1, dL0) <= TOL


def test_noalloc_refuses_grid_beyond_its_scratch():
    import torch
    hgks.load()
    n = (40, 40, 40)
    q = torch.zeros((5, 40, 40, 40), dtype=torch.float64, device="cuda")
    L = torch.zeros_like(q)
    dL = torch.zeros_like(q)
    with pytest.raises(hgks.HgksError) as e:
        hgks.hgks_flux_noalloc(n, (0, 0, 0), (1, 1, 1), q, 1e-3, L, dL)
    assert e.value.code == hgks.HGKS_E_INVALID
    assert "bytes of scratch" in str(e.value)


def test_noalloc_refuses_a_time_step_that_is_not_finite():
    import torch
    hgks.load()
    n = (8, 8, 8)
    q = torch.from_numpy(W.density_advection(n)).cuda()
    L = torch.zeros_like(q)
    dL = torch.zeros_like(q)
    for dt in (float("inf"), float("nan"), 0.0, -1e-3):
        with pytest.raises(hgks.HgksError) as e:
            hgks.hgks_flux_noalloc(n, (0, 0, 0), (2, 2, 2), q, dt, L, dL)
        assert e.value.code == hgks.HGKS_E_INVALID
