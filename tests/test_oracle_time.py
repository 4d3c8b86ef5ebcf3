"""Pin of the oracle's two-stage fourth-order time step (Sec. 3):

    y*      = y^n + dt/2 L(y^n) + dt^2/8 dL/dt(y^n)
    y^{n+1} = y^n + dt L(y^n) + dt^2/6 (dL/dt(y^n) + 2 dL/dt(y*))

Every step of the oracle's scheme runs through the one routine
`orc_two_stage`, with the gas-kinetic rate pair (L, dL/dt) as its callback.
Here the same routine is driven by ODEs whose time derivative of the rate
is exact (dL/dt = L'(y) L(y)); the method is then fourth order, so the
global error must fall by 2^4 per halving of dt.  A wrong coefficient
anywhere in the two formulas drops the order to 3 or below.

(The gas-kinetic dL/dt of the full scheme is the time derivative of the
PDE evaluated on the reconstruction, not the exact derivative of the
semi-discrete system, so on a fixed mesh the full scheme's time error is
first order with a coefficient that belongs to the spatial error; the
order of the combination itself is pinned here.)
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm

import oracle

A = np.array([[-0.3, 1.0, 0.0], [-1.0, -0.3, 0.2], [0.0, -0.2, -0.5]])


def _linear(stage, y):
    L = A @ y
    return L, A @ L


def _riccati(stage, y):
    """y' = -y^2: L = -y^2, dL/dt = -2 y y' = 2 y^3."""
    return -y * y, 2.0 * y ** 3


def _orders(errs):
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


@pytest.mark.parametrize("case", ["linear", "riccati"])
def test_two_stage_step_is_fourth_order_with_exact_rates(case):
    T = 2.0
    if case == "linear":
        y0 = np.array([1.0, 0.5, -0.25])
        exact = expm(A * T) @ y0
        rate = _linear
    else:
        y0 = np.array([1.0, 0.5, 2.0])
        exact = y0 / (1.0 + y0 * T)
        rate = _riccati
    errs = []
    for nsteps in (20, 40, 80, 160):
        y = oracle.two_stage(y0, T / nsteps, nsteps, rate)
        errs.append(np.abs(y - exact).max())
    orders = _orders(errs)
    assert min(orders) > 3.8 and max(orders) < 4.3, (errs, orders)


def test_two_stage_step_single_step_taylor_terms():
    """One step on y' = a y reproduces exp(a dt) to the dt^4 term: the
    amplification factor is 1 + z + z^2/2 + z^3/6 + z^4/24 with z = a dt."""
    for z in (0.1, -0.37, 0.8):
        y = oracle.two_stage(np.array([1.0]), 1.0, 1, lambda s, y: (z * y, z * z * y))
        assert abs(y[0] - (1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24)) < 1e-15
