"""Characteristic-variable reconstruction on the GPU (Sec. 4, uniform mesh)
against the oracle: the operator on smooth and discontinuous data with
mixed boundaries, multi-step runs, and the Sod problem (oscillations
reduced against the conservative reconstruction)."""
import numpy as np
import pytest

import oracle
from paper_1909_01580_gb300 import hgks
from paper_1909_01580_gb300 import workloads as W
from tests._cases import max_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    hgks.load()


def _solver(n, lo, hi, **kw):
    s = hgks.Solver(n, lo, hi, **kw)
    hgks.hgks_set_option(s.h, "characteristic", 1.0)
    return s


def _common(a, b):
    """max |a - b| on the common scale of all five variables"""
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("case", ["smooth", "octant"])
def test_operator_parity_characteristic(case):
    if case == "smooth":
        n, lo, hi = (10, 9, 8), (0.0, 0.0, 0.0), (1.0, 0.9, 0.8)
        q = W.smooth_random(n, seed=31, lo=lo, hi=hi, amp=0.2)
        bc = (2, 2, 1, 1, 0, 0)
        kw = dict(mu=1e-3, Pr=0.72)
    else:
        n, lo, hi = (12, 12, 12), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
        q = W.octant_riemann(n, seed=3)
        bc = (1, 2, 2, 1, 2, 2)
        kw = {}
    cfg = oracle.make_cfg(n, lo, hi, bc=bc, charvar=1, **kw)
    Lo, dLo = oracle.operator(cfg, q, 0.01)
    s = _solver(n, lo, hi, bc=bc, **kw)
    s.set_state(q)
    L, dL = s.flux(0.01)
    s.close()
    assert _common(L, Lo) <= 1e-11, _common(L, Lo)
    assert _common(dL, dLo) <= 1e-9, _common(dL, dLo)


def test_steps_parity_characteristic():
    n = (12, 12, 12)
    q0 = W.octant_riemann(n, seed=4)
    bc = (2, 2, 2, 2, 1, 1)
    cfg = oracle.make_cfg(n, (0, 0, 0), (1, 1, 1), bc=bc, charvar=1)
    qo, to, do, _ = oracle.step(cfg, q0, 0.0, 5, cfl=0.35)
    s = _solver(n, (0, 0, 0), (1, 1, 1), bc=bc)
    s.set_state(q0)
    t, done = s.step(5, cfl=0.35)
    q, _ = s.get_state()
    s.close()
    assert done == do == 5 and abs(t - to) < 1e-14
    assert max_rel(q, qo) <= 1e-11, max_rel(q, qo)


def test_reconstruct_refused_in_characteristic_mode():
    s = _solver((8, 8, 8), (0, 0, 0), (1, 1, 1))
    s.set_state(W.density_advection((8, 8, 8), hi=(1, 1, 1)))
    with pytest.raises(hgks.HgksError) as e:
        s.reconstruct()
    assert e.value.code == hgks.HGKS_E_STATE
    s.close()


def _tv_overshoot(line):
    rho = line[0]
    u = line[1] / rho
    return float(np.abs(np.diff(rho)).sum()), float(max(rho.max() - 1.0, 0.0) + max(0.125 - rho.min(), 0.0) +
                                                    max(u.max() - 0.9274526, 0.0))


@pytest.mark.parametrize("precision", [hgks.HGKS_FP64, hgks.HGKS_MIXED])
def test_sod_characteristic_reduces_oscillations(precision):
    n, lo, hi = (100, 4, 4), (0.0, 0.0, 0.0), (1.0, 0.04, 0.04)
    res = {}
    for cv in (0, 1):
        s = hgks.Solver(n, lo, hi, bc=(2,) * 6, precision=precision)
        hgks.hgks_set_option(s.h, "characteristic", float(cv))
        s.set_state(W.sod(n, lo, hi))
        s.step(100000, cfl=0.35, t_end=0.2)
        q, _ = s.get_state()
        s.close()
        res[cv] = _tv_overshoot(q[:, 0, 0, :])
    print("Sod TV / overshoot, conservative", res[0], "characteristic", res[1])
    assert res[1][0] <= res[0][0] and res[1][1] <= 0.5 * res[0][1]
