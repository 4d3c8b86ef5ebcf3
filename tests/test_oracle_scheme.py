"""Pins of the oracle's full scheme (Sec. 3 finite-volume operator and
two-stage time stepping, Sec. 4 tests): free stream, conservation,
symmetry, the exact advection solution, third-order convergence, and the
accuracy table of the paper (slow)."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1909_01580_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _l1(err, cellvol):
    """volume-weighted L1 norm sum |e| |Omega| (reading of Tables 1-3)"""
    return float(np.sum(np.abs(err)) * cellvol)


def test_free_stream_uniform_mesh():
    n = (6, 5, 4)
    q = W.uniform_flow(n, rho=1.3, u=(0.4, -0.2, 0.7), p=0.9)
    cfg = oracle.make_cfg(n, (0, 0, 0), (1.2, 1.0, 0.8))
    q1, t, done, _ = oracle.step(cfg, q, 0.0, 2, cfl=0.35)
    assert done == 2
    np.testing.assert_allclose(q1, q, rtol=2e-15, atol=2e-15)


def test_conservation_periodic():
    n = (8, 7, 6)
    q = W.smooth_random(n, seed=3, lo=(0, 0, 0), hi=(1.0, 0.875, 0.75), amp=0.15)
    cfg = oracle.make_cfg(n, (0, 0, 0), (1.0, 0.875, 0.75), mu=1e-3, Pr=0.72)
    q1, t, done, _ = oracle.step(cfg, q, 0.0, 3, cfl=0.35)
    tot0 = q.reshape(5, -1).sum(axis=1)
    tot1 = q1.reshape(5, -1).sum(axis=1)
    np.testing.assert_allclose(tot1, tot0, rtol=0, atol=1e-12 * np.abs(q).sum(axis=(1, 2, 3)).max() / q[0].size)
    assert not np.allclose(q1, q)


def test_reflective_walls_conserve_mass_and_energy_and_mirror():
    n = (6, 6, 6)
    q = W.octant_riemann(n, seed=2)
    cfg = oracle.make_cfg(n, (0, 0, 0), (1, 1, 1), bc=(1,) * 6)
    q1, t, done, _ = oracle.step(cfg, q, 0.0, 2, cfl=0.35)
    for v in (0, 4):
        assert abs(q1[v].sum() - q[v].sum()) < 1e-12 * q[v].sum()
    # mirror the data in x: the solution mirrors
    qm = q[:, :, :, ::-1].copy()
    qm[1] *= -1
    q1m, _, _, _ = oracle.step(cfg, qm, 0.0, 2, cfl=0.35)
    back = q1m[:, :, :, ::-1].copy()
    back[1] *= -1
    np.testing.assert_allclose(back, q1, rtol=1e-12, atol=1e-12)


def test_axis_permutation_symmetry():
    """Cyclic relabelling x -> y -> z of a smooth state relabels the solution
    (the stencils, weights and Gauss rule are symmetric)."""
    n = (6, 6, 6)
    q = W.smooth_random(n, seed=9, amp=0.15)
    cfg = oracle.make_cfg(n, (0, 0, 0), (1, 1, 1))
    L, dL = oracle.operator(cfg, q, 0.01)
    # np.transpose(a, (1, 2, 0)) maps array axes (z, y, x) to (y, x, z):
    # new x' = old z, y' = old x, z' = old y, so U' = W, V' = U, W' = V
    def relabel(arr):
        out = np.stack([np.transpose(arr[v], (1, 2, 0)) for v in range(5)])
        out[1], out[2], out[3] = out[3].copy(), out[1].copy(), out[2].copy()
        return out

    qp2 = relabel(q)
    Lp, dLp = oracle.operator(cfg, qp2, 0.01)
    Lb2 = relabel(L)
    np.testing.assert_allclose(Lp, Lb2, rtol=1e-11, atol=1e-12 * np.abs(L).max())


def test_cfl_step_count_density_advection():
    """Reading of the CFL step h/(|U| + c): the 16^3 density advection at
    CFL 0.5 to t = 0.2 takes 10 steps."""
    n = (16, 16, 16)
    q = W.density_advection(n)
    cfg = oracle.make_cfg(n)
    dt = oracle.cfl_dt(cfg, q, 0.5)
    assert math.ceil(0.2 / dt - 1e-12) == 10


def test_density_advection_error_and_convergence():
    """Density advection depending on x + y only (z is periodic with 4
    cells): errors against the exact solution fall at third order."""
    errs = []
    for N in (6, 12, 24):
        n = (N, N, 4)
        lo, hi = (0, 0, 0), (2.0, 2.0, 8.0 / N)
        box = W.Box(n, lo, hi)
        x, y, z = box.centres()
        h = 2.0 / N
        a = 0.5 * math.pi * h
        fac = (math.sin(a) / a) ** 2

        def state(t):
            rho = 1.0 + 0.2 * np.sin(math.pi * (x + y - 2 * t)) * fac
            one = np.ones_like(rho)
            return np.stack([rho, rho, rho, np.zeros_like(rho), 1 / 0.4 + rho])

        cfg = oracle.make_cfg(n, lo, hi)
        q0 = state(0.0)
        t_end = 0.2
        q1, t, done, _ = oracle.step(cfg, q0, 0.0, 10000, cfl=0.35, t_end=t_end)
        assert abs(t - t_end) < 1e-12
        errs.append(_l1(q1[0] - state(t_end)[0], h * h * (8.0 / N / 4)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    print("advection errors", errs, "orders", orders)
    assert orders[1] > 2.6, (errs, orders)


@pytest.mark.slow
def test_table1_density_advection_16():
    """Table 1 (Sec. 4) at 16^3: L1 error at t = 2 within 2% of the printed
    1.4612e-1 (the oracle gives 1.4586e-1 with the readings of the CFL form,
    epsilon = 1e-8 and exponent 1)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "table1_advection_uniform.txt"))
    n = (16, 16, 16)
    cfg = oracle.make_cfg(n)
    q0 = W.density_advection(n)
    q1, t, done, _ = oracle.step(cfg, q0, 0.0, 100000, cfl=0.35, t_end=2.0)
    exact = W.density_advection(n, t=2.0)
    l1 = _l1(q1[0] - exact[0], (2.0 / 16) ** 3)
    ref = rows[0, 1]
    print(f"Table 1, 16^3: oracle L1 = {l1:.5e} (paper {ref:.5e}), {done} steps")
    assert abs(l1 - ref) < 0.02 * ref, (l1, ref)
