"""Accuracy tables of Sec. 4 on the GPU (FP64): density advection to t = 2 at
CFL 0.35 on uniform meshes (Table 1), the static non-coplanar mesh (Table 2)
and the moving mesh (Table 3), 16^3 to 64^3.  The L1 errors (volume
weighted, Sec. 4) are compared with the printed ones and the observed
orders with the printed orders.

Reading (collision time of the accuracy tests): with the printed inviscid
collision time tau = 0.01 dt + |p_l - p_r|/(p_l + p_r) dt, the term
-tau (a.u + A) g0 of eq. (flux) is a heat conduction of order tau p ~ h,
a first-order error that the printed third-order convergence to 128^3 does
not show.  The printed formula reproduces Table 1 at 16^3 (checked below);
the convergence tables are checked in the limit of a small epsilon
(tau_eps = 1e-4), where the printed errors and orders are reproduced."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1909_01580_gb300 import hgks
from paper_1909_01580_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SIZES = (16, 32, 64)


def _table(name):
    rows = np.loadtxt(os.path.join(GOLDEN, name))
    return {int(r[0]): r[1] for r in rows}


def _run(n, mesh, amp, omega, q0, tau_eps=1e-4):
    s = hgks.Solver((n, n, n), (0, 0, 0), (2, 2, 2), mesh=mesh, mesh_amp=amp, mesh_omega=omega, tau_eps=tau_eps)
    s.set_state(q0, t=0.0)
    t, done = s.step(100000, cfl=0.35, t_end=2.0)
    q, _ = s.get_state()
    s.close()
    assert abs(t - 2.0) < 1e-13
    return q


def _check(errs, ref, rel):
    for n in SIZES:
        assert abs(errs[n] - ref[n]) <= rel * ref[n], (n, errs[n], ref[n])
    order = math.log2(errs[32] / errs[64])
    ref_order = math.log2(ref[32] / ref[64])
    assert order > ref_order - 0.05, (order, ref_order)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    hgks.load()


def test_table1_printed_collision_time_16():
    ref = _table("table1_advection_uniform.txt")
    n = 16
    q = _run(n, 0, 0.0, 0.0, W.density_advection((n, n, n)), tau_eps=0.01)
    exact = W.density_advection((n, n, n), t=2.0)
    l1 = float(np.abs(q[0] - exact[0]).sum() * (2.0 / n) ** 3)
    assert abs(l1 - ref[16]) <= 0.02 * ref[16], (l1, ref[16])


def test_table1_uniform():
    ref = _table("table1_advection_uniform.txt")
    errs = {}
    for n in SIZES:
        q = _run(n, 0, 0.0, 0.0, W.density_advection((n, n, n)))
        exact = W.density_advection((n, n, n), t=2.0)
        errs[n] = float(np.abs(q[0] - exact[0]).sum() * (2.0 / n) ** 3)
    print("Table 1 GPU L1:", errs)
    _check(errs, ref, 0.10)


def test_table2_noncoplanar():
    ref = _table("table2_advection_noncoplanar.txt")
    errs = {}
    for n in SIZES:
        q0 = W.density_advection_mapped((n, n, n), amp=0.1)
        q = _run(n, 1, 0.1, 0.0, q0)
        # at t = 2 the exact solution equals the initial one (period 2/3 in
        # x + y + z - 3t shifted by 6)
        exact = W.density_advection_mapped((n, n, n), amp=0.1, t=2.0)
        vol = oracle.volumes(oracle.make_cfg((n, n, n), mesh=1, amp=0.1, omega=0.0), 0.0)
        errs[n] = float((np.abs(q[0] - exact[0]) * vol).sum())
    print("Table 2 GPU L1:", errs)
    _check(errs, ref, 0.05)


def test_table3_moving():
    ref = _table("table3_advection_moving.txt")
    errs = {}
    for n in SIZES:
        # S(t) = sin(pi t) vanishes at t = 0 and t = 2: the mesh is the
        # uniform one at both ends
        q = _run(n, 2, 0.1, math.pi, W.density_advection((n, n, n)))
        exact = W.density_advection((n, n, n), t=2.0)
        errs[n] = float(np.abs(q[0] - exact[0]).sum() * (2.0 / n) ** 3)
    print("Table 3 GPU L1:", errs)
    _check(errs, ref, 0.05)
