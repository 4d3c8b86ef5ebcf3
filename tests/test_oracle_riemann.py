"""Non-reflecting (outflow) boundaries and the Riemann problems of Sec. 4 in
the oracle: the exact Riemann solver used as the reference is pinned by the
Rankine-Hugoniot conditions and the Riemann invariants; the oracle's Sod
solution converges to it; outflow boundaries let the shock leave while a
reflective wall sends it back."""
import math

import numpy as np
import pytest

import oracle
from paper_1909_01580_gb300 import workloads as W
from tests._riemann import Riemann

SOD_L, SOD_R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)


def _flux(r, u, p, g=1.4):
    E = p / (g - 1.0) + 0.5 * r * u * u
    return np.array([r * u, r * u * u + p, u * (E + p)]), np.array([r, r * u, E])


def test_exact_solver_jump_conditions():
    """Across the right shock: F(star) - F(R) = S (U(star) - U(R)) for mass,
    momentum and energy; across the left rarefaction: the Riemann invariant
    u + 2c/(gamma-1) and the entropy p/rho^gamma are constant."""
    g = 1.4
    R = Riemann(SOD_L, SOD_R, g)
    rls, rrs = R.star_densities()
    S = R.shock_speed(+1)
    Fs, Us = _flux(rrs, R.u_star, R.p_star)
    Fr, Ur = _flux(*SOD_R)
    assert np.abs((Fs - Fr) - S * (Us - Ur)).max() < 1e-12
    cl = math.sqrt(g * SOD_L[2] / SOD_L[0])
    cls = math.sqrt(g * R.p_star / rls)
    assert abs((SOD_L[1] + 2 * cl / (g - 1)) - (R.u_star + 2 * cls / (g - 1))) < 1e-12
    assert abs(SOD_L[2] / SOD_L[0] ** g - R.p_star / rls ** g) < 1e-12
    # inside the fan the samples keep both invariants too
    for s in np.linspace(-cl + 1e-6, R.u_star - cls - 1e-6, 7):
        r, u, p = R.sample(s)
        c = math.sqrt(g * p / r)
        assert abs(u + 2 * c / (g - 1) - (SOD_L[1] + 2 * cl / (g - 1))) < 1e-12
        assert abs(p / r ** g - SOD_L[2] / SOD_L[0] ** g) < 1e-12
        assert abs(u - c - s) < 1e-12  # the fan is the family u - c = x/t


def _sod_oracle(nx, t_end, bc_x):
    n = (nx, 1, 1)
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0 / nx, 1.0 / nx)
    cfg = oracle.make_cfg(n, lo, hi, bc=(bc_x[0], bc_x[1], 2, 2, 2, 2))
    q0 = W.sod(n, lo, hi)
    q, t, done, _ = oracle.step(cfg, q0, 0.0, 100000, cfl=0.35, t_end=t_end)
    assert abs(t - t_end) < 1e-13
    return q


def _l1_rho(q, t, x_range=(0.0, 1.0)):
    nx = q.shape[3]
    edges = np.arange(nx + 1) / nx
    ref = Riemann(SOD_L, SOD_R).cell_averages(edges, t, 0.5, sub=100)
    cen = 0.5 * (edges[1:] + edges[:-1])
    sel = (cen > x_range[0]) & (cen < x_range[1])
    return float(np.abs(q[0, 0, 0, sel] - ref[0, sel]).sum() / nx)


def test_sod_oracle_converges_to_exact():
    e50 = _l1_rho(_sod_oracle(50, 0.2, (2, 2)), 0.2)
    e100 = _l1_rho(_sod_oracle(100, 0.2, (2, 2)), 0.2)
    print(f"Sod L1(rho) at t = 0.2: 50 cells {e50:.4e}, 100 cells {e100:.4e}")
    assert e50 < 0.012
    assert e100 < 0.65 * e50


def test_outflow_lets_the_shock_leave():
    """At t = 0.35 the shock (speed 1.752) has passed x = 1 (at t = 0.285).
    With outflow boundaries the region x > 0.85 is the post-shock state of
    the infinite-domain solution; a reflective wall sends a shock back into
    it."""
    e_out = _l1_rho(_sod_oracle(50, 0.35, (2, 2)), 0.35, (0.85, 1.0))
    e_ref = _l1_rho(_sod_oracle(50, 0.35, (2, 1)), 0.35, (0.85, 1.0))
    print(f"x > 0.85 at t = 0.35: outflow {e_out:.3e}, reflective {e_ref:.3e}")
    assert e_out < 0.1 * e_ref
    assert e_out < 2e-3
