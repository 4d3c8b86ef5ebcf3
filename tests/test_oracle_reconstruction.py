"""Pins of the oracle's WENO-AO reconstruction (Sec. 2) against closed forms:
exact reproduction of quadratic data by the big-stencil polynomial P0,
exact reproduction of linear data by every P_m (then tau = 0 and the
nonlinear weights equal the linear ones), the smoothness indicator of a
quadratic on a cube, conservation of the cell mean, and third-order point
values under refinement."""
import math

import numpy as np
import pytest

import oracle
from paper_1909_01580_gb300 import workloads as W

GAMMA_LIN = 0.0025
# the 2-point Gauss nodes on [-1/2, 1/2]
S = math.sqrt(3.0) / 6.0


def _box_mean_monomial(lo, hi, e):
    """exact mean of x^e over [lo, hi]"""
    return (hi ** (e + 1) - lo ** (e + 1)) / ((e + 1) * (hi - lo))


def _quadratic_averages(n, lo, hi, coef):
    """Exact cell averages of Q(x) = c0 + c.x + sum_{d<=e} C_de x_d x_e.
    coef = (c0, c[3], C[3,3] upper triangle)."""
    c0, c1, C = coef
    h = [(hi[d] - lo[d]) / n[d] for d in range(3)]
    ax = [lo[d] + np.arange(n[d] + 1) * h[d] for d in range(3)]
    m1 = [np.array([_box_mean_monomial(ax[d][i], ax[d][i + 1], 1) for i in range(n[d])]) for d in range(3)]
    m2 = [np.array([_box_mean_monomial(ax[d][i], ax[d][i + 1], 2) for i in range(n[d])]) for d in range(3)]

    def grid(arrs):
        z, y, x = np.meshgrid(arrs[2], arrs[1], arrs[0], indexing="ij")
        return x, y, z

    X1 = grid(m1)
    X2 = grid(m2)
    val = np.full((n[2], n[1], n[0]), c0)
    for d in range(3):
        val = val + c1[d] * X1[d]
        for e in range(d, 3):
            if e == d:
                val = val + C[d, e] * X2[d]
            else:  # independent directions: mean of product = product of means
                val = val + C[d, e] * X1[d] * X1[e]
    return val


def _quad_eval(coef, x):
    c0, c1, C = coef
    v = c0 + sum(c1[d] * x[d] for d in range(3))
    for d in range(3):
        for e in range(d, 3):
            v = v + C[d, e] * x[d] * x[e]
    return v


def _quad_grad(coef, x):
    c0, c1, C = coef
    g = np.array(c1, dtype=float).copy()
    for d in range(3):
        for e in range(d, 3):
            g[d] += C[d, e] * x[e]
            g[e] += C[d, e] * x[d]
    return g


def _random_quadratic(rng, scale=0.05):
    c0 = rng.uniform(0.5, 1.0)
    c1 = rng.uniform(-scale, scale, 3)
    C = np.triu(rng.uniform(-scale, scale, (3, 3)))
    return c0, c1, C


def _state_from_scalars(fields):
    # five independent scalar fields used as the five "conservative" variables
    return np.stack(fields).astype(np.float64)


def test_P0_reproduces_quadratic_data_exactly():
    rng = np.random.default_rng(1)
    n, lo, hi = (6, 5, 7), (0.0, -0.3, 0.2), (1.2, 0.7, 1.6)
    quads = [_random_quadratic(rng) for _ in range(5)]
    # keep the state physical for the positivity check: rho, E large
    quads[0] = (2.0,) + quads[0][1:]
    quads[4] = (5.0,) + quads[4][1:]
    q = _state_from_scalars([_quadratic_averages(n, lo, hi, c) for c in quads])
    cfg = oracle.make_cfg(n, lo, hi)
    _, _, a0 = oracle.reconstruct(cfg, q)
    h = [(hi[d] - lo[d]) / n[d] for d in range(3)]
    assert abs(h[0] - h[1]) < 1e-12 and abs(h[1] - h[2]) < 1e-12
    hh = h[0]
    # cells whose stencil does not reach the (periodic) boundary
    interior = [(1, 1, 1), (2, 3, 4), (4, 3, 5), (3, 1, 2), (4, 3, 1)]
    for (i, j, k) in interior:
        lin = i + n[0] * (j + n[1] * k)
        xc = np.array([lo[0] + (i + 0.5) * hh, lo[1] + (j + 0.5) * hh, lo[2] + (k + 0.5) * hh])
        for v in range(5):
            c0, c1, C = quads[v]
            g = _quad_grad(quads[v], xc)
            expect = [hh * g[0], hh * g[1], hh * g[2],
                      hh * hh * C[0, 0], hh * hh * C[1, 1], hh * hh * C[2, 2],
                      hh * hh * C[0, 1], hh * hh * C[0, 2], hh * hh * C[1, 2]]
            np.testing.assert_allclose(a0[lin, v], expect, rtol=0, atol=1e-13)


def test_linear_data_gives_linear_weights_and_exact_values():
    rng = np.random.default_rng(2)
    n, lo, hi = (5, 5, 5), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    lins = []
    for v in range(5):
        c1 = rng.uniform(-0.2, 0.2, 3)
        lins.append((3.0 if v in (0, 4) else 0.5, c1, np.zeros((3, 3))))
    q = _state_from_scalars([_quadratic_averages(n, lo, hi, c) for c in lins])
    cfg = oracle.make_cfg(n, lo, hi)
    coef, flag, a0 = oracle.reconstruct(cfg, q)
    assert not flag.any()
    # interior cells (their stencils do not wrap around the periodic box)
    inner = [i + 5 * (j + 5 * k) for i in range(1, 4) for j in range(1, 4) for k in range(1, 4)]
    # P~ = P0 = the linear function
    np.testing.assert_allclose(coef[inner, :, 1:], a0[inner], rtol=0, atol=1e-14)
    np.testing.assert_allclose(a0[inner, :, 3:], 0.0, atol=1e-14)
    for lin in [inner[0], inner[13], inner[-1]]:
        beta, wbar = oracle.weno_weights(cfg, q, lin)
        # all indicators equal, so tau = 0 and wbar = gamma exactly
        np.testing.assert_allclose(beta, beta[:, :1] * np.ones((1, 25)), rtol=1e-12)
        g = np.full(25, GAMMA_LIN)
        g[0] = 1.0 - 24 * GAMMA_LIN
        np.testing.assert_allclose(wbar, np.tile(g, (5, 1)), rtol=1e-13)
        assert abs(g[0] - 0.94) < 1e-15 and abs(g.sum() - 1.0) < 1e-15 and (g > 0).all()
        # beta_m = |Omega|^{-1/3} int |grad P|^2 = h^2 |grad Q|^2
        h = 0.2
        for v in range(5):
            assert abs(beta[v, 0] - h * h * np.dot(lins[v][1], lins[v][1])) < 1e-14


def test_smoothness_indicator_of_quadratic_on_cube():
    """beta_0 of eq. (indicator) for P0 = Q + sum a_n p_n on a cube, worked by
    hand: first-derivative terms a_d^2 + (4 a_dd^2 + sum_{e!=d} a_de^2)/12,
    second-derivative terms 4 a_dd^2 and a_de^2 (each multi-index once)."""
    rng = np.random.default_rng(3)
    n = (5, 5, 5)
    q = W.smooth_random(n, seed=4, amp=0.2)
    cfg = oracle.make_cfg(n, (0, 0, 0), (1, 1, 1))
    _, _, a0 = oracle.reconstruct(cfg, q)
    for lin in [0, 62, 124]:
        beta, _ = oracle.weno_weights(cfg, q, lin)
        for v in range(5):
            a = a0[lin, v]
            ax, ay, az, axx, ayy, azz, axy, axz, ayz = a
            b1 = (ax ** 2 + (4 * axx ** 2 + axy ** 2 + axz ** 2) / 12
                  + ay ** 2 + (4 * ayy ** 2 + axy ** 2 + ayz ** 2) / 12
                  + az ** 2 + (4 * azz ** 2 + axz ** 2 + ayz ** 2) / 12)
            b2 = 4 * (axx ** 2 + ayy ** 2 + azz ** 2) + axy ** 2 + axz ** 2 + ayz ** 2
            assert abs(beta[v, 0] - (b1 + b2)) <= 1e-13 * (b1 + b2) + 1e-18


def test_nonlinear_weights_positive_normalised():
    q = W.octant_riemann((8, 8, 8), seed=1)
    cfg = oracle.make_cfg((8, 8, 8), (0, 0, 0), (1, 1, 1), bc=(1,) * 6)
    for lin in [0, 3 + 8 * 3 + 64 * 3, 4 + 8 * 4 + 64 * 4, 511]:
        beta, wbar = oracle.weno_weights(cfg, q, lin)
        assert (wbar > 0).all()
        np.testing.assert_allclose(wbar.sum(axis=1), 1.0, rtol=1e-14)
        assert (beta >= 0).all()


def test_reconstruction_keeps_cell_mean():
    """The combination coefficients sum to one and every p_n has zero mean,
    so the mean of P~ over the cell is the cell average (3-point Gauss)."""
    n = (6, 6, 6)
    q = W.smooth_random(n, seed=7, amp=0.2)
    cfg = oracle.make_cfg(n, (0, 0, 0), (1, 1, 1))
    g, w = np.polynomial.legendre.leggauss(3)
    g, w = 0.5 * g, 0.5 * w
    h = 1.0 / 6
    for lin in [0, 100, 215]:
        i, j, k = lin % 6, (lin // 6) % 6, lin // 36
        xc = np.array([(i + .5) * h, (j + .5) * h, (k + .5) * h])
        pts, wts = [], []
        for a in range(3):
            for b in range(3):
                for c in range(3):
                    pts.append(xc + h * np.array([g[a], g[b], g[c]]))
                    wts.append(w[a] * w[b] * w[c])
        out = oracle.eval_reconstruction(cfg, q, lin, np.array(pts))
        mean = np.einsum("p,pv->v", np.array(wts), out[:, :, 0])
        np.testing.assert_allclose(mean, q.reshape(5, -1)[:, lin], rtol=1e-14)


def test_point_values_third_order():
    """Point values at the face Gauss points from exact cell averages of a
    smooth profile converge at third order (P0 error O(h^3) and nonlinear
    weights gamma(1 + O(h)))."""
    errs = []
    for N in (8, 16, 32):
        n = (N, N, N)
        q = W.density_advection(n)
        cfg = oracle.make_cfg(n)
        h = 2.0 / N
        lin = (N // 4) + N * (N // 3) + N * N * (N // 2)
        i, j, k = lin % N, (lin // N) % N, lin // (N * N)
        xc = np.array([(i + .5) * h, (j + .5) * h, (k + .5) * h])
        pts = []
        for d in range(3):
            for side in (-0.5, 0.5):
                for ga in (-S, S):
                    for gb in (-S, S):
                        p = np.zeros(3)
                        p[d] = side
                        p[(d + 1) % 3] = ga
                        p[(d + 2) % 3] = gb
                        pts.append(xc + h * p)
        pts = np.array(pts)
        out = oracle.eval_reconstruction(cfg, q, lin, pts)
        exact = 1.0 + 0.2 * np.sin(math.pi * pts.sum(axis=1))
        errs.append(np.abs(out[:, 0, 0] - exact).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert orders[1] > 2.7, (errs, orders)
