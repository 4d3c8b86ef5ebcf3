"""Parity of the mapped- and moving-mesh CUDA path with the oracle (Sec. 2
trilinear cells, Sec. 3 bilinear faces, Remark 2), the free stream on the
moving mesh (geometric conservation), and the moving-mesh workload at its
full size (96^3, mixed precision) against the FP64 oracle at sampled cells."""
import math

import numpy as np
import pytest

import oracle
from paper_1909_01580_gb300 import hgks
from paper_1909_01580_gb300 import workloads as W
from tests._cases import max_rel

pytestmark = pytest.mark.gpu

TOL = 1e-11
MOVING = dict(mesh=2, mesh_amp=0.05, mesh_omega=2 * math.pi)   # the 96^3 workload's map
STATIC = dict(mesh=1, mesh_amp=0.1, mesh_omega=0.0)            # the non-coplanar static mesh


def _ocfg(n, lo, hi, m, **kw):
    return oracle.make_cfg(n, lo, hi, mesh=m["mesh"], amp=m["mesh_amp"], omega=m["mesh_omega"], **kw)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    hgks.load()


@pytest.mark.parametrize("m", [STATIC, MOVING])
def test_reconstruction_parity_mapped(m):
    n, lo, hi = (10, 9, 8), (0, 0, 0), (2.0, 2.0, 2.0)
    q = W.smooth_random(n, seed=6, lo=lo, hi=hi, amp=0.15)
    t = 0.13
    coef_o, flag_o, _ = oracle.reconstruct(_ocfg(n, lo, hi, m), q, t=t)
    s = hgks.Solver(n, lo, hi, **m)
    s.set_state(q, t=t)
    coef, flag = s.reconstruct()
    s.close()
    assert (flag == flag_o).all()
    for v in range(5):
        ref = coef_o[:, v, 1:]
        assert np.abs(coef[:, v] - ref).max() <= 1e-11 * np.abs(ref).max(), v


@pytest.mark.parametrize("m", [STATIC, MOVING])
def test_operator_parity_mapped(m):
    n, lo, hi = (10, 9, 8), (0, 0, 0), (2.0, 2.0, 2.0)
    q = W.smooth_random(n, seed=7, lo=lo, hi=hi, amp=0.15)
    t = 0.21
    cfg = _ocfg(n, lo, hi, m, mu=2e-3, Pr=0.72)
    dt = 0.01
    Lo, dLo = oracle.operator(cfg, q, dt, t=t)
    s = hgks.Solver(n, lo, hi, mu=2e-3, Pr=0.72, **m)
    s.set_state(q, t=t)
    L, dL = s.flux(dt)
    s.close()
    assert max_rel(L, Lo) <= TOL, max_rel(L, Lo)
    assert max_rel(dL, dLo) <= 1e-9, max_rel(dL, dLo)


def test_moving_mesh_steps_parity():
    """Ten steps of density advection on the moving mesh (fixed dt): the
    state matches the oracle's, which advances |Omega| Q and the volumes of
    the discrete conservation law in the same way."""
    n = (12, 12, 12)
    lo, hi = (0, 0, 0), (2, 2, 2)
    q0 = W.density_advection(n)
    cfg = _ocfg(n, lo, hi, MOVING)
    vol0 = oracle.volumes(cfg, 0.0).reshape(-1)
    dt = oracle.cfl_dt(cfg, q0, 0.35)
    qo, to, _, _ = oracle.step(cfg, q0, 0.0, 10, dt_fixed=dt, vol=vol0)
    s = hgks.Solver(n, lo, hi, **MOVING)
    s.set_state(q0, t=0.0)
    t, done = s.step(10, dt_fixed=dt)
    q, _ = s.get_state()
    s.close()
    assert done == 10 and abs(t - to) < 1e-14
    assert max_rel(q, qo) <= TOL, max_rel(q, qo)


def test_moving_mesh_cfl_steps_parity():
    n = (10, 10, 10)
    lo, hi = (0, 0, 0), (2, 2, 2)
    q0 = W.density_advection(n)
    cfg = _ocfg(n, lo, hi, MOVING)
    vol0 = oracle.volumes(cfg, 0.0).reshape(-1)
    qo, to, done_o, _ = oracle.step(cfg, q0, 0.0, 100, cfl=0.35, t_end=0.12, vol=vol0)
    s = hgks.Solver(n, lo, hi, **MOVING)
    s.set_state(q0, t=0.0)
    t, done = s.step(100, cfl=0.35, t_end=0.12)
    q, _ = s.get_state()
    s.close()
    assert done == done_o and abs(t - 0.12) < 1e-14
    assert max_rel(q, qo) <= TOL, max_rel(q, qo)


@pytest.mark.parametrize("precision,tol", [(hgks.HGKS_FP64, 1e-13), (hgks.HGKS_MIXED, 1e-5)])
def test_free_stream_moving_mesh_gpu(precision, tol):
    n = (16, 16, 16)
    q0 = W.uniform_flow(n)
    s = hgks.Solver(n, (0, 0, 0), (2, 2, 2), precision=precision, **MOVING)
    s.set_state(q0, t=0.0)
    t, done = s.step(100, cfl=0.35, t_end=0.25)
    q, _ = s.get_state()
    s.close()
    assert done > 5
    assert np.abs(q - q0).max() <= tol, np.abs(q - q0).max()


def test_moving_96_mixed_against_fp64_oracle_sampled():
    """The moving-mesh workload at full size (96^3, mixed precision): L and
    dL/dt at sampled cells against the FP64 oracle, judged on the state's
    common scale with the FP32 unit round-off; and a few steps that stay
    physical and conservative in the volume-weighted sense."""
    n = (96, 96, 96)
    lo, hi = (0, 0, 0), (2, 2, 2)
    q0 = W.density_advection(n)
    t = 0.1
    cfg = _ocfg(n, lo, hi, MOVING)
    dt = 4e-3
    cells = [0, 95, 96 * 95, 96 ** 3 - 1, 12345, 456789, 96 ** 3 // 2 + 17, 600000]
    Lo, dLo = oracle.operator(cfg, q0, dt, t=t, cells=cells)
    # L is a difference of face fluxes over the cell volume: in the mixed
    # path the FP32 face fluxes carry their round-off (6e-8 relative) into
    # L amplified by |F|/(h |L|), about 50-100 at h = 2/96; 1e-4 of the
    # common scale, as for the uniform-mesh mixed checks.
    for prec, tol in ((hgks.HGKS_FP64, 1e-9), (hgks.HGKS_MIXED, 1e-4)):
        s = hgks.Solver(n, lo, hi, precision=prec, **MOVING)
        s.set_state(q0, t=t)
        L, dL = s.flux(dt)
        Ls = L.reshape(5, -1)[:, cells]
        scale = np.abs(Lo).max()
        assert np.abs(Ls - Lo).max() <= tol * scale, (prec, np.abs(Ls - Lo).max() / scale)
        if prec == hgks.HGKS_MIXED:
            t1, done = s.step(3, cfl=0.35)
            assert done == 3
        s.close()


def test_free_stream_table4_gpu():
    """Table 4's moving mesh (amplitude 0.1, S(t) = sin(pi t)) to t = 0.5 on
    16^3 in FP64: the L1 error of the density stays at round-off, within ten
    times the printed value."""
    import os
    rows = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "table4_gcl_moving.txt"))
    n = (16, 16, 16)
    q0 = W.uniform_flow(n)
    s = hgks.Solver(n, (0, 0, 0), (2, 2, 2), mesh=2, mesh_amp=0.1, mesh_omega=math.pi)
    s.set_state(q0, t=0.0)
    t, done = s.step(1000, cfl=0.35, t_end=0.5)
    q, _ = s.get_state()
    s.close()
    vol = oracle.volumes(oracle.make_cfg(n, mesh=2, amp=0.1, omega=math.pi), 0.5).reshape(-1)
    l1 = float(np.abs(q[0] - q0[0]).reshape(-1) @ vol)
    assert abs(t - 0.5) < 1e-14
    assert l1 < 10 * rows[0, 1], (l1, rows[0, 1])


def test_mixed_moving_mesh_within_one_percent_of_discretisation_error():
    """Density advection on the moving mesh (16^3) over one full period of
    the mesh motion (t = 1, where the cells are uniform again and the exact
    averages are known): mixed minus FP64 is at most 1% of the FP64 error."""
    n = (16, 16, 16)
    q0 = W.density_advection(n)
    exact = W.density_advection(n, t=1.0)
    res = {}
    for prec in (hgks.HGKS_FP64, hgks.HGKS_MIXED):
        s = hgks.Solver(n, (0, 0, 0), (2, 2, 2), precision=prec, **MOVING)
        s.set_state(q0, t=0.0)
        t, _ = s.step(1000, cfl=0.35, t_end=1.0)
        assert abs(t - 1.0) < 1e-14
        res[prec], _ = s.get_state()
        s.close()
    vol = (2.0 / 16) ** 3
    disc = np.abs(res[hgks.HGKS_FP64][0] - exact[0]).sum() * vol
    mix = np.abs(res[hgks.HGKS_MIXED][0] - res[hgks.HGKS_FP64][0]).sum() * vol
    assert mix <= 0.01 * disc, (mix, disc)
