"""The alternative stencil S' (Remark of Sec. 2) on the GPU: reconstruction,
operator and multi-step parity with the oracle, and the accuracy test of
Table 1 ("these substitutions work as well": third order at errors close to
those of S)."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1909_01580_gb300 import hgks
from paper_1909_01580_gb300 import workloads as W
from tests._cases import max_rel

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    hgks.load()


def _solver(n, lo, hi, **kw):
    s = hgks.Solver(n, lo, hi, **kw)
    hgks.hgks_set_option(s.h, "stencil", 1.0)
    return s


def test_reconstruction_parity_sprime():
    n, lo, hi = (9, 8, 7), (0.0, 0.0, 0.0), (0.9, 0.8, 0.7)
    q = W.smooth_random(n, seed=41, lo=lo, hi=hi, amp=0.2)
    coef_o, flag_o, _ = oracle.reconstruct(oracle.make_cfg(n, lo, hi, stencil=1), q)
    s = _solver(n, lo, hi)
    s.set_state(q)
    coef, flag = s.reconstruct()
    s.close()
    assert (flag == flag_o).all()
    for v in range(5):
        ref = coef_o[:, v, 1:]
        assert np.abs(coef[:, v] - ref).max() <= 1e-12 * np.abs(ref).max(), v


@pytest.mark.parametrize("bc", [(0,) * 6, (1, 2, 1, 1, 2, 2)])
def test_operator_and_steps_parity_sprime(bc):
    n, lo, hi = (10, 10, 10), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    q0 = W.octant_riemann(n, seed=6) if bc[0] else W.smooth_random(n, seed=42, lo=lo, hi=hi, amp=0.2)
    cfg = oracle.make_cfg(n, lo, hi, bc=bc, stencil=1, mu=1e-3, Pr=0.72)
    Lo, dLo = oracle.operator(cfg, q0, 0.01)
    qo, to, do, _ = oracle.step(cfg, q0, 0.0, 4, cfl=0.35)
    s = _solver(n, lo, hi, bc=bc, mu=1e-3, Pr=0.72)
    s.set_state(q0)
    L, dL = s.flux(0.01)
    t, done = s.step(4, cfl=0.35)
    q, _ = s.get_state()
    s.close()
    assert np.abs(L - Lo).max() <= 1e-11 * np.abs(Lo).max()
    assert np.abs(dL - dLo).max() <= 1e-9 * np.abs(dLo).max()
    assert done == do == 4 and abs(t - to) < 1e-14
    assert max_rel(q, qo) <= 1e-11, max_rel(q, qo)


def test_table1_with_sprime():
    rows = np.loadtxt(os.path.join(GOLDEN, "table1_advection_uniform.txt"))
    ref = {int(r[0]): r[1] for r in rows}
    errs = {}
    for N in (16, 32, 64):
        s = _solver((N,) * 3, (0, 0, 0), (2, 2, 2), tau_eps=1e-4)
        s.set_state(W.density_advection((N,) * 3))
        s.step(100000, cfl=0.35, t_end=2.0)
        q, _ = s.get_state()
        s.close()
        exact = W.density_advection((N,) * 3, t=2.0)
        errs[N] = float(np.abs(q[0] - exact[0]).sum() * (2.0 / N) ** 3)
    print("Table 1 with S':", errs)
    # measured within 1.2% of the printed Table 1 at every size
    for N in errs:
        assert abs(errs[N] - ref[N]) < 0.03 * ref[N], (N, errs[N], ref[N])
    assert math.log2(errs[32] / errs[64]) > 2.8
