"""Pins of the oracle's gas-kinetic parts (Sec. 3): Maxwellian moments by
brute-force velocity quadrature, the exact time integrals of eq. (flux) by
quadrature in t, the whole point flux against an independent brute-force
evaluation of the time-dependent distribution, the Euler flux of a uniform
state (also on a moving grid), and the Navier-Stokes limit (shear stress,
heat flux with the Prandtl-number correction)."""
import math

import numpy as np
import pytest

import oracle

GAMMA = 1.4
K = (5 - 3 * GAMMA) / (GAMMA - 1)  # = 2 internal degrees of freedom


def _quad(f, a, b, n=200):
    x, w = np.polynomial.legendre.leggauss(n)
    xm = 0.5 * (b - a) * x + 0.5 * (a + b)
    return 0.5 * (b - a) * np.sum(w * f(xm))


@pytest.mark.parametrize("U,lam", [(0.3, 2.0), (-1.7, 0.6), (2.5, 3.0), (0.0, 1.0)])
def test_1d_moments_by_quadrature(U, lam):
    g = lambda u: math.sqrt(lam / math.pi) * np.exp(-lam * (u - U) ** 2)
    R = 12.0 / math.sqrt(lam) + abs(U)
    for side in (0, 1, -1):
        m = oracle.moments_1d(U, lam, side)
        for nexp in range(9):
            f = lambda u: u ** nexp * g(u)
            if side == 0:
                ref = _quad(f, -R, 0, 300) + _quad(f, 0, R, 300)
            elif side == 1:
                ref = _quad(f, 0, R, 300)
            else:
                ref = _quad(f, -R, 0, 300)
            scale = max(1.0, abs(ref), (abs(U) + 1 / math.sqrt(lam)) ** nexp)
            assert abs(m[nexp] - ref) <= 1e-13 * scale, (side, nexp, m[nexp], ref)


def _velocity_grid(U, lam, n=80):
    """Brute-force nodes for one Maxwellian: Gauss-Legendre panels split at
    u = 0 (half spaces), Gauss-Legendre for v, w, and product Gauss-Hermite
    for the K = 2 internal degrees of freedom."""
    R = 8.5 / math.sqrt(lam)
    x, w = np.polynomial.legendre.leggauss(n)
    lo_u, hi_u = min(U[0] - R, -1e-3), max(U[0] + R, 1e-3)
    un = np.concatenate([0.5 * lo_u * (x + 1), 0.5 * hi_u * (x + 1)])
    uw = np.concatenate([-0.5 * lo_u * w, 0.5 * hi_u * w])
    vn = U[1] + R * x
    vw = R * w
    wn = U[2] + R * x
    ww = R * w
    return un, uw, vn, vw, wn, ww


def _xi_moments(lam):
    """<xi^(2k)>, k = 0..3, for K = 2 by product Gauss-Hermite quadrature"""
    t, w = np.polynomial.hermite.hermgauss(12)
    x1, x2 = np.meshgrid(t / math.sqrt(lam), t / math.sqrt(lam), indexing="ij")
    ww = np.outer(w, w) / math.pi
    r2 = x1 ** 2 + x2 ** 2
    return [float(np.sum(ww * r2 ** k)) for k in range(4)]


class Maxwell:
    """Brute-force Maxwellian of a conservative state (local frame)."""

    def __init__(self, Wc):
        self.rho = Wc[0]
        self.U = np.array(Wc[1:4]) / Wc[0]
        p = (GAMMA - 1) * (Wc[4] - 0.5 * self.rho * np.dot(self.U, self.U))
        self.lam = self.rho / (2 * p)
        un, uw, vn, vw, wn, ww = _velocity_grid(self.U, self.lam)
        self.u, self.v, self.w = np.meshgrid(un, vn, wn, indexing="ij")
        self.wt = np.einsum("i,j,k->ijk", uw, vw, ww)
        lam = self.lam
        self.g = (self.rho * (lam / math.pi) ** 1.5
                  * np.exp(-lam * ((self.u - self.U[0]) ** 2 + (self.v - self.U[1]) ** 2 + (self.w - self.U[2]) ** 2)))
        self.xi = _xi_moments(lam)

    def psi(self):
        """psi as a list of (array, xi-power) pairs per component"""
        u, v, w = self.u, self.v, self.w
        one = np.ones_like(u)
        return [[(one, 0)], [(u, 0)], [(v, 0)], [(w, 0)], [(0.5 * (u * u + v * v + w * w), 0), (0.5 * one, 1)]]

    def integrate(self, weight_terms, half=0):
        """int weight * psi * g over the domain; weight_terms: list of
        (array, xi-power); returns the 5-vector"""
        mask = 1.0
        if half > 0:
            mask = (self.u > 0).astype(float)
        elif half < 0:
            mask = (self.u < 0).astype(float)
        out = np.zeros(5)
        for i, ps in enumerate(self.psi()):
            s = 0.0
            for (pa, pk) in ps:
                for (wa, wk) in weight_terms:
                    s += self.xi[pk + wk] * np.sum(self.wt * mask * self.g * pa * wa)
            out[i] = s
        return out

    def apsi(self, a):
        """a . psi as weight terms"""
        u, v, w = self.u, self.v, self.w
        return [(a[0] + a[1] * u + a[2] * v + a[3] * w + 0.5 * a[4] * (u * u + v * v + w * w), 0),
                (0.5 * a[4] * np.ones_like(u), 1)]

    def moment_matrix(self):
        M = np.zeros((5, 5))
        for j, ps in enumerate(self.psi()):
            M[:, j] = self.integrate(ps)
        return M


def _times(terms, arr):
    return [(a * arr, k) for (a, k) in terms]


def _add(*lists):
    out = []
    for l in lists:
        out += l
    return out


def test_moment_matrix_by_quadrature_and_compatibility():
    cfg = oracle.make_cfg((4, 4, 4))
    rng = np.random.default_rng(0)
    for _ in range(3):
        rho, p = rng.uniform(0.3, 2.0), rng.uniform(0.3, 2.0)
        U = rng.uniform(-1, 1, 3)
        Wc = np.array([rho, *(rho * U), p / (GAMMA - 1) + 0.5 * rho * U @ U])
        M = oracle.moment_matrix(cfg, Wc)
        Mb = Maxwell(Wc).moment_matrix()
        np.testing.assert_allclose(M, Mb, rtol=1e-11, atol=1e-12)
        # compatibility: int psi g = W
        np.testing.assert_allclose(M[0], Wc, rtol=1e-13)


def test_time_integrals_by_quadrature():
    for delta, tau in [(1.0, 0.1), (0.3, 0.02), (2.0, 1.5), (1e-3, 1e-5)]:
        q = oracle.time_integrals(delta, tau)
        e = lambda t: np.exp(-t / tau)
        facs = [lambda t: 1 - e(t), lambda t: (t + tau) * e(t) - tau, lambda t: t - tau + tau * e(t),
                lambda t: e(t), lambda t: -(t + tau) * e(t), lambda t: -tau * e(t)]
        # graded panels resolve the e^{-t/tau} layer
        edges = np.unique(np.concatenate([[0.0], np.minimum(delta, tau * 2.0 ** np.arange(-4, 12)), [delta]]))
        for j, f in enumerate(facs):
            ref = sum(_quad(f, edges[i], edges[i + 1], 40) for i in range(len(edges) - 1))
            assert abs(q[j] - ref) <= 1e-13 * max(abs(ref), delta * max(delta, tau)), (j, q[j], ref)


def _brute_point_flux(inp, dt, mu=0.0, tau_eps=0.01, tau_C=1.0, Pr=1.0):
    """Independent evaluation of F^n, dF^n at one Gauss point straight from
    eq. (flux) of Sec. 3: slopes by solving with brute-force moment matrices,
    the equilibrium from the colliding half spaces (g_l for u > 0), the
    distribution evaluated on a velocity grid, time integrals by quadrature,
    then the 2x2 system for (F, dF)."""
    Wl, Wr = inp[0:5], inp[20:25]
    dWl = [inp[5 + 5 * d:10 + 5 * d] for d in range(3)]
    dWr = [inp[25 + 5 * d:30 + 5 * d] for d in range(3)]
    gl, gr = Maxwell(Wl), Maxwell(Wr)

    def slopes(g, dW):
        M = g.moment_matrix()
        a = [np.linalg.solve(M, dW[d]) for d in range(3)]
        vel = [g.u, g.v, g.w]
        au = _add(*[_times(g.apsi(a[d]), vel[d]) for d in range(3)])
        A = np.linalg.solve(M, -g.integrate(au))
        return a, A

    al, Al = slopes(gl, dWl)
    ar, Ar = slopes(gr, dWr)
    W0 = gl.integrate([(np.ones_like(gl.u), 0)], +1) + gr.integrate([(np.ones_like(gr.u), 0)], -1)
    dW0 = [gl.integrate(gl.apsi(al[d]), +1) + gr.integrate(gr.apsi(ar[d]), -1) for d in range(3)]
    g0 = Maxwell(W0)
    a0, A0 = slopes(g0, dW0)
    pl = (GAMMA - 1) * (Wl[4] - 0.5 * (Wl[1] ** 2 + Wl[2] ** 2 + Wl[3] ** 2) / Wl[0])
    pr = (GAMMA - 1) * (Wr[4] - 0.5 * (Wr[1] ** 2 + Wr[2] ** 2 + Wr[3] ** 2) / Wr[0])
    jump = abs((pl - pr) / (pl + pr))
    if mu > 0:
        tau = mu / (g0.rho / (2 * g0.lam)) + tau_C * jump * dt
    else:
        tau = tau_eps * dt + tau_C * jump * dt

    # velocity-moment pieces (time-independent), each a 5-vector of u*psi moments
    def pieces(g, a, A, half, weight):
        vel = [g.u, g.v, g.w]
        au = _add(*[_times(g.apsi(a[d]), vel[d]) for d in range(3)])
        base = weight(g)
        m1 = g.integrate(base, half)
        m2 = g.integrate([(wa * ta, wk + tk) for (wa, wk) in base for (ta, tk) in au], half)
        m3 = g.integrate([(wa * ta, wk + tk) for (wa, wk) in base for (ta, tk) in g.apsi(A)], half)
        return m1, m2, m3

    def uweight(g):
        return [(g.u, 0)]

    def heatweight(g):
        # (u-U0)((u-U0)^2+(v-V0)^2+(w-W0)^2+xi^2)/2 about the velocity of g0
        U0 = g0.U
        cx, cy, cz = g.u - U0[0], g.v - U0[1], g.w - U0[2]
        return [(0.5 * cx * (cx * cx + cy * cy + cz * cz), 0), (0.5 * cx, 1)]

    def Fhat(delta, weight, comp=None):
        P0 = pieces(g0, a0, A0, 0, weight)
        PL = pieces(gl, al, Al, +1, weight)
        PR = pieces(gr, ar, Ar, -1, weight)
        x, w = np.polynomial.legendre.leggauss(30)
        edges = np.unique(np.concatenate([[0.0], np.minimum(delta, tau * 2.0 ** np.arange(-3, 14)), [delta]]))
        out = np.zeros(5)
        for i in range(len(edges) - 1):
            a, b = edges[i], edges[i + 1]
            for t, wt in zip(0.5 * (b - a) * x + 0.5 * (a + b), 0.5 * (b - a) * w):
                e = math.exp(-t / tau)
                f = ((1 - e) * P0[0] + ((t + tau) * e - tau) * P0[1] + (t - tau + tau * e) * P0[2]
                     + e * (PL[0] - (tau + t) * PL[1] - tau * PL[2])
                     + e * (PR[0] - (tau + t) * PR[1] - tau * PR[2]))
                out += wt * f
        return out

    F1 = Fhat(dt, uweight)
    F2 = Fhat(0.5 * dt, uweight)
    if mu > 0 and Pr != 1.0:
        F1[4] += (1 / Pr - 1) * Fhat(dt, heatweight)[0]
        F2[4] += (1 / Pr - 1) * Fhat(0.5 * dt, heatweight)[0]
    M2 = np.array([[dt, 0.5 * dt * dt], [0.5 * dt, 0.125 * dt * dt]])
    sol = np.linalg.solve(M2, np.stack([F1, F2]))
    return sol[0], sol[1]


def _random_inputs(rng, grad=0.3, jump=0.2):
    def state(rho, U, p):
        return np.array([rho, *(rho * U), p / (GAMMA - 1) + 0.5 * rho * U @ U])

    rho, p = rng.uniform(0.6, 1.4), rng.uniform(0.6, 1.4)
    U = rng.uniform(-0.5, 0.5, 3)
    Wl = state(rho, U, p)
    Wr = state(rho * (1 + rng.uniform(-jump, jump)), U + rng.uniform(-jump, jump, 3), p * (1 + rng.uniform(-jump, jump)))
    inp = np.zeros(40)
    inp[0:5] = Wl
    inp[20:25] = Wr
    for s, Wc in ((0, Wl), (1, Wr)):
        for d in range(3):
            inp[20 * s + 5 + 5 * d: 20 * s + 10 + 5 * d] = grad * rng.uniform(-1, 1, 5) * np.abs(Wc)
    return inp


@pytest.mark.parametrize("seed,mu,Pr", [(0, 0.0, 1.0), (1, 0.0, 1.0), (2, 0.02, 1.0), (3, 0.02, 0.72)])
def test_point_flux_against_bruteforce_distribution(seed, mu, Pr):
    rng = np.random.default_rng(seed)
    inp = _random_inputs(rng)
    dt = 0.05
    cfg = oracle.make_cfg((4, 4, 4), mu=mu, Pr=Pr)
    F, dF = oracle.point_flux(cfg, inp, dt)
    Fb, dFb = _brute_point_flux(inp, dt, mu=mu, Pr=Pr)
    np.testing.assert_allclose(F, Fb, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(dF, dFb, rtol=1e-7, atol=1e-8 * np.abs(dFb).max())


def test_uniform_state_gives_euler_flux_also_on_moving_grid():
    rng = np.random.default_rng(5)
    cfg = oracle.make_cfg((4, 4, 4))
    for _ in range(4):
        rho, p = rng.uniform(0.2, 2), rng.uniform(0.2, 2)
        U = rng.uniform(-1, 1, 3)
        E = p / (GAMMA - 1) + 0.5 * rho * U @ U
        inp = np.zeros(40)
        inp[0:5] = inp[20:25] = [rho, *(rho * U), E]
        for ug in (np.zeros(3), rng.uniform(-0.5, 0.5, 3)):
            F, dF = oracle.point_flux(cfg, inp, 0.01, ug=ug)
            un = U[0] - ug[0]
            exact = np.array([rho * un, rho * U[0] * un + p, rho * U[1] * un, rho * U[2] * un, E * un + p * U[0]])
            np.testing.assert_allclose(F, exact, rtol=1e-12, atol=1e-13)
            assert np.abs(dF).max() < 1e-9


def test_mirror_symmetry_of_point_flux():
    """Reflecting u -> -u and swapping the sides reverses the normal mass and
    energy fluxes and keeps the normal momentum flux."""
    rng = np.random.default_rng(6)
    cfg = oracle.make_cfg((4, 4, 4))
    inp = _random_inputs(rng)
    mir = np.zeros(40)
    for s in range(2):
        src = inp[20 * (1 - s): 20 * (1 - s) + 20].copy()
        src[1] = -src[1]  # rho U
        for d in range(3):
            blk = src[5 + 5 * d: 10 + 5 * d]
            if d == 0:
                blk *= -1  # d/dn_x flips sign
            blk[1] = -blk[1]
            src[5 + 5 * d: 10 + 5 * d] = blk
        mir[20 * s: 20 * s + 20] = src
    F, dF = oracle.point_flux(cfg, inp, 0.02)
    Fm, dFm = oracle.point_flux(cfg, mir, 0.02)
    sgn = np.array([-1, 1, -1, -1, -1])
    np.testing.assert_allclose(Fm, sgn * F, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(dFm, sgn * dF, rtol=1e-9, atol=1e-10)


@pytest.mark.parametrize("Pr", [1.0, 0.72])
def test_navier_stokes_limit(Pr):
    """For smooth data and tau << dt the flux is the Navier-Stokes flux with
    mu = tau p: shear stress -mu dV/dx and heat flux -kappa dT/dx with
    kappa = mu gamma/((gamma - 1) Pr) (R = 1)."""
    rho, p = 1.0, 1.0
    mu = 1e-4
    dt = 0.05
    cfg = oracle.make_cfg((4, 4, 4), mu=mu, Pr=Pr, tau_C=0.0)
    inp = np.zeros(40)
    E = p / (GAMMA - 1)
    inp[0:5] = inp[20:25] = [rho, 0, 0, 0, E]
    # shear: d(rho V)/dn_x = s
    s = 0.5
    for side in (0, 20):
        inp[side + 5 + 2] = s
    F, _ = oracle.point_flux(cfg, inp, dt)
    assert abs(F[2] - (-mu * s / rho)) < 2e-3 * mu * s
    # heat: d(rho)/dn_x = r with uniform pressure, T = p/rho
    inp2 = np.zeros(40)
    inp2[0:5] = inp2[20:25] = [rho, 0, 0, 0, E]
    r = 0.4
    for side in (0, 20):
        inp2[side + 5 + 0] = r
    F2, _ = oracle.point_flux(cfg, inp2, dt)
    dTdx = -p / rho ** 2 * r
    kappa = mu * GAMMA / ((GAMMA - 1) * Pr)
    assert abs(F2[4] - (-kappa * dTdx)) < 2e-3 * abs(kappa * dTdx), (F2[4], -kappa * dTdx)


@pytest.mark.parametrize("rho,p", [(1.0, 1.0), (0.8, 2.5), (1.6, 0.4)])
def test_navier_stokes_limit_power_law_viscosity(rho, p):
    """Isotropic-turbulence viscosity law mu(T) = mu_ref (T/T_ref)^0.76 (Sec.
    4): in the Navier-Stokes limit the shear stress is -mu(T) dV/dx with T =
    p/rho of the interface state."""
    mu_ref, T_ref, dt = 1e-4, 0.7, 0.05
    cfg = oracle.make_cfg((4, 4, 4), mu=mu_ref, Pr=1.0, tau_C=0.0, mu_pow=0.76, T_ref=T_ref)
    inp = np.zeros(40)
    E = p / (GAMMA - 1)
    inp[0:5] = inp[20:25] = [rho, 0, 0, 0, E]
    s = 0.5
    for side in (0, 20):
        inp[side + 5 + 2] = s
    F, _ = oracle.point_flux(cfg, inp, dt)
    mu_T = mu_ref * (p / rho / T_ref) ** 0.76
    assert abs(F[2] - (-mu_T * s / rho)) < 2e-3 * mu_T * s, (F[2], -mu_T * s / rho)
    # the law is not the constant viscosity unless T = T_ref
    if abs(p / rho - T_ref) > 0.1:
        assert abs(F[2] - (-mu_ref * s / rho)) > 1e-2 * mu_ref * s
