"""Characteristic-variable reconstruction in the oracle (Sec. 4): the basis
is the eigenbasis of the Euler flux Jacobian along the face normal, the
reconstruction in it reproduces linear data exactly (where the projection
cannot matter), and on the Sod problem it reduces the oscillations of the
conservative reconstruction."""
import numpy as np
import pytest

import oracle
from paper_1909_01580_gb300 import workloads as W


def _euler_flux(W, d, gamma=1.4):
    rho = W[0]
    u = W[1:4] / rho
    p = (gamma - 1.0) * (W[4] - 0.5 * rho * (u @ u))
    F = np.empty(5)
    F[0] = rho * u[d]
    F[1:4] = rho * u[d] * u
    F[1 + d] += p
    F[4] = u[d] * (W[4] + p)
    return F


@pytest.mark.parametrize("d", [0, 1, 2])
def test_basis_diagonalises_the_flux_jacobian(d):
    cfg = oracle.make_cfg((4, 4, 4))
    Wc = np.array([1.3, 0.4, -0.7, 0.25, 3.4])
    R, L = oracle.char_basis(cfg, Wc, d)
    # Jacobian by central differences of the Euler flux (independent of the oracle)
    h = 1e-6
    A = np.zeros((5, 5))
    for m in range(5):
        e = np.zeros(5)
        e[m] = h
        A[:, m] = (_euler_flux(Wc + e, d) - _euler_flux(Wc - e, d)) / (2 * h)
    rho = Wc[0]
    u = Wc[1:4] / rho
    p = 0.4 * (Wc[4] - 0.5 * rho * (u @ u))
    c = np.sqrt(1.4 * p / rho)
    lam = np.array([u[d] - c, u[d], u[d], u[d], u[d] + c])
    assert np.abs(A @ R - R * lam[None, :]).max() < 1e-7
    assert np.abs(L @ R - np.eye(5)).max() < 1e-13


def test_linear_data_same_as_conservative():
    """Linear conservative data: every indicator is equal, tau = 0 and the
    weights are the linear ones in any variables, so both reconstructions are
    the exact linear field and the operators agree to round-off (interior
    cells, away from the outflow ghosts)."""
    n = (8, 8, 8)
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    h = 1.0 / 8
    x = (np.arange(8) + 0.5) * h
    z, y, xx = np.meshgrid(x, x, x, indexing="ij")
    q = np.stack([1.0 + 0.1 * xx - 0.05 * y + 0.03 * z, 0.2 + 0.05 * y, -0.1 + 0.02 * xx + 0.04 * z,
                  0.3 - 0.03 * y, 2.6 + 0.2 * xx + 0.1 * z])
    cells = [i + 8 * (j + 8 * k) for k in range(2, 6) for j in range(2, 6) for i in range(2, 6)]
    out = {}
    for cv in (0, 1):
        cfg = oracle.make_cfg(n, lo, hi, bc=(2,) * 6, charvar=cv, mu=1e-3, Pr=0.72)
        out[cv] = oracle.operator(cfg, q, 0.01, cells=cells)
    # on the common scale of all five residuals (the mass residual of these
    # data is zero up to round-off)
    for a, b, tol in ((out[1][0], out[0][0], 1e-11), (out[1][1], out[0][1], 1e-9)):
        assert np.abs(a - b).max() <= tol * np.abs(b).max(), np.abs(a - b).max() / np.abs(b).max()


def _tv_and_overshoot(q):
    rho = q[0, 0, 0]
    u = q[1, 0, 0] / rho
    tv = float(np.abs(np.diff(rho)).sum())
    over = max(rho.max() - 1.0, 0.0) + max(0.125 - rho.min(), 0.0) + max(u.max() - 0.9274526, 0.0)
    return tv, over


def test_sod_characteristic_reduces_oscillations():
    n = (100, 1, 1)
    lo, hi = (0.0, 0.0, 0.0), (1.0, 0.01, 0.01)
    res = {}
    for cv in (0, 1):
        cfg = oracle.make_cfg(n, lo, hi, bc=(2,) * 6, charvar=cv)
        q, t, done, _ = oracle.step(cfg, W.sod(n, lo, hi), 0.0, 100000, cfl=0.35, t_end=0.2)
        res[cv] = _tv_and_overshoot(q)
    print("Sod total variation / overshoot: conservative", res[0], "characteristic", res[1])
    assert res[1][0] <= res[0][0]
    assert res[1][1] <= res[0][1]
