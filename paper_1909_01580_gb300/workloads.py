"""Seeded, synthetic initial data for the test problems of Pan & Xu
(arXiv 1909.01580, Sec. 4) and the benchmark workloads.

This module only evaluates initial conditions; it holds none of the
scheme's arithmetic, so both the CUDA path and the oracle can take their
inputs from it.  Every state is returned as conservative cell averages
(rho, rho U, rho V, rho W, rho E) in SoA layout [5][nz][ny][nx], FP64.

Reading (cell averages versus point values): initial data are cell
averages.  The advection data are averaged exactly (the profile is a plane
sine wave); the Taylor-Green data are averaged with a 4-point Gauss-Legendre
rule per axis applied to the conservative variables; piecewise-constant
octant data are exact when the octant planes fall on cell faces.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Box:
    n: tuple
    lo: tuple
    hi: tuple

    @property
    def h(self):
        return tuple((self.hi[d] - self.lo[d]) / self.n[d] for d in range(3))

    def centres(self):
        """cell-centre coordinate arrays, each of shape [nz][ny][nx]"""
        ax = [self.lo[d] + (np.arange(self.n[d]) + 0.5) * self.h[d] for d in range(3)]
        z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        return x, y, z


def _conservative(rho, u, v, w, p, gamma):
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E]).astype(np.float64)


def density_advection(n, t=0.0, gamma=1.4, lo=(0.0, 0.0, 0.0), hi=(2.0, 2.0, 2.0), amp=0.2):
    """3D density advection (Sec. 4 accuracy test): rho = 1 + 0.2 sin(pi(x+y+z-t)),
    U = V = W = 1, p = 1 on [0,2]^3, periodic.  Exact cell averages at time t."""
    box = Box(tuple(n), tuple(lo), tuple(hi))
    x, y, z = box.centres()
    fac = 1.0
    for d in range(3):
        a = 0.5 * math.pi * box.h[d]
        fac *= math.sin(a) / a
    rho = 1.0 + amp * np.sin(math.pi * (x + y + z - 3.0 * t)) * fac
    one = np.ones_like(rho)
    # all conservative variables are affine in rho, so averaging is exact
    return _conservative(rho, one, one, one, one, gamma)


def _gauss4():
    g, w = np.polynomial.legendre.leggauss(4)
    return 0.5 * g, 0.5 * w  # on [-1/2, 1/2], weights sum to 1


def cell_average(box: Box, fn, gamma=1.4):
    """4-point Gauss-Legendre per axis average of the conservative variables
    returned by fn(x, y, z) -> (rho, u, v, w, p)."""
    g, w = _gauss4()
    x, y, z = box.centres()
    acc = np.zeros((5,) + x.shape)
    h = box.h
    for a in range(4):
        for b in range(4):
            for c in range(4):
                prims = fn(x + g[a] * h[0], y + g[b] * h[1], z + g[c] * h[2])
                acc += w[a] * w[b] * w[c] * _conservative(*prims, gamma)
    return acc


def density_advection_mapped(n, amp=0.1, t=0.0, gamma=1.4, lo=(0.0, 0.0, 0.0), hi=(2.0, 2.0, 2.0), amp_rho=0.2,
                             order=4):
    """Cell averages of the density-advection data of Sec. 4 at time t on
    the static non-coplanar mesh of Table 2: the vertices are the images of
    the uniform reference nodes under x = xi + amp prod_d sin(2 pi (xi_d -
    lo_d)/L_d) (the same shift in every coordinate), and each cell is the
    trilinear hexahedron through its 8 vertices.  The averages are taken
    with an order^3 Gauss-Legendre rule on the reference cube weighted by
    |det J| of the trilinear map (the data are smooth, so the rule's error
    is far below the scheme's)."""
    box = Box(tuple(n), tuple(lo), tuple(hi))
    L = [hi[d] - lo[d] for d in range(3)]
    nodes = [lo[d] + np.arange(n[d] + 1) * box.h[d] for d in range(3)]
    Z, Y, X = np.meshgrid(nodes[2], nodes[1], nodes[0], indexing="ij")
    s = (np.sin(2 * math.pi * (X - lo[0]) / L[0]) * np.sin(2 * math.pi * (Y - lo[1]) / L[1])
         * np.sin(2 * math.pi * (Z - lo[2]) / L[2]))
    V = np.stack([X + amp * s, Y + amp * s, Z + amp * s], axis=-1)  # [nz+1][ny+1][nx+1][3]
    nx, ny, nz = n
    # the 8 vertices of every cell, vertex (a, b, c) at index a + 2b + 4c
    corners = [V[c:c + nz, b:b + ny, a:a + nx] for c in (0, 1) for b in (0, 1) for a in (0, 1)]
    g, w = np.polynomial.legendre.leggauss(order)
    g = 0.5 * (g + 1.0)  # nodes on [0, 1]
    w = 0.5 * w
    num = np.zeros((nz, ny, nx))
    den = np.zeros((nz, ny, nx))
    for i, (pa, wa) in enumerate(zip(g, w)):
        for j, (pb, wb) in enumerate(zip(g, w)):
            for k, (pc, wc) in enumerate(zip(g, w)):
                p = (pa, pb, pc)
                x = np.zeros((nz, ny, nx, 3))
                J = np.zeros((nz, ny, nx, 3, 3))
                for q in range(8):
                    bits = (q & 1, (q >> 1) & 1, q >> 2)
                    f = [p[e] if bits[e] else 1.0 - p[e] for e in range(3)]
                    df = [1.0 if bits[e] else -1.0 for e in range(3)]
                    psi = f[0] * f[1] * f[2]
                    dpsi = (df[0] * f[1] * f[2], f[0] * df[1] * f[2], f[0] * f[1] * df[2])
                    x += corners[q] * psi
                    for e in range(3):
                        J[..., :, e] += corners[q] * dpsi[e]
                detJ = np.abs(np.linalg.det(J))
                rho = 1.0 + amp_rho * np.sin(math.pi * (x[..., 0] + x[..., 1] + x[..., 2] - 3.0 * t))
                wt = wa * wb * wc * detJ
                num += wt * rho
                den += wt
    rho = num / den
    one = np.ones_like(rho)
    # the conservative variables are affine in rho, so their averages follow
    return _conservative(rho, one, one, one, one, gamma)


def riemann_x(n, left, right, x0, lo=(0.0, 0.0, 0.0), hi=(1.0, 0.1, 0.1), gamma=1.4):
    """A 1D Riemann problem along x in a 3D box: (rho, U, p) = left for
    x < x0 and right for x > x0, V = W = 0.  Cell averages, exact when x0
    falls on a cell face; a cell cut by x0 gets the volume-weighted mix."""
    box = Box(tuple(n), tuple(lo), tuple(hi))
    hx = box.h[0]
    edges = lo[0] + np.arange(n[0] + 1) * hx
    frac_left = np.clip((x0 - edges[:-1]) / hx, 0.0, 1.0)  # fraction of each cell left of x0
    cons_l = np.array([left[0], left[0] * left[1], 0.0, 0.0, left[2] / (gamma - 1.0) + 0.5 * left[0] * left[1] ** 2])
    cons_r = np.array([right[0], right[0] * right[1], 0.0, 0.0,
                       right[2] / (gamma - 1.0) + 0.5 * right[0] * right[1] ** 2])
    line = cons_l[:, None] * frac_left[None, :] + cons_r[:, None] * (1.0 - frac_left[None, :])
    return np.ascontiguousarray(np.broadcast_to(line[:, None, None, :], (5, n[2], n[1], n[0])), dtype=np.float64)


def sod(n, lo=(0.0, 0.0, 0.0), hi=(1.0, 0.1, 0.1), gamma=1.4):
    """Sod problem of Sec. 4: (rho, U, p) = (1, 0, 1) for x < 0.5 and
    (0.125, 0, 0.1) for x > 0.5 on [0,1] x [0,0.1] x [0,0.1]."""
    return riemann_x(n, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.5, lo, hi, gamma)


def blast_wave(n, lo=(0.0, 0.0, 0.0), hi=(100.0, 10.0, 10.0), gamma=1.4, p_mid=0.01):
    """Woodward-Colella blast wave of Sec. 4 on [0,100] x [0,10] x [0,10]:
    rho = 1, U = 0 and p = 1000 for x < 10, p_mid (0.01 in the paper) for
    10 < x < 90, 100 for x > 90 (cell averages; the planes x = 10, 90 fall
    on faces when the cell size divides 10)."""
    box = Box(tuple(n), tuple(lo), tuple(hi))
    hx = box.h[0]
    edges = lo[0] + np.arange(n[0] + 1) * hx
    f1 = np.clip((10.0 - edges[:-1]) / hx, 0.0, 1.0)
    f3 = np.clip((edges[1:] - 90.0) / hx, 0.0, 1.0)
    p = 1000.0 * f1 + 100.0 * f3 + p_mid * (1.0 - f1 - f3)
    line = np.zeros((5, n[0]))
    line[0] = 1.0
    line[4] = p / (gamma - 1.0)
    return np.ascontiguousarray(np.broadcast_to(line[:, None, None, :], (5, n[2], n[1], n[0])), dtype=np.float64)


@dataclass
class TurbulenceParams:
    """Constants of the isotropic-turbulence workload (Sec. 4)."""
    A0: float
    k0: float
    u_rms: float
    K0: float          # initial turbulent kinetic energy (per unit mass)
    T0: float          # temperature p/rho (R = 1)
    p0: float
    mu0: float         # viscosity at T0; mu = mu0 (T/T0)^0.76
    tau_t0: float      # large-eddy-turnover time


def isotropic_turbulence(n, mach_t, seed=0, A0=1.3e-4, k0=8.0, re_lambda=72.0, gamma=1.4, rho0=1.0):
    """Compressible isotropic turbulence of Sec. 4 on [-pi, pi]^3: a seeded
    divergence-free random velocity with the spectrum E(k) = A0 k^4
    exp(-2 k^2/k0^2), uniform density rho0 and temperature T0 set by the
    turbulent Mach number Ma_t = sqrt(3) u_rms/sqrt(gamma T0), viscosity
    mu0 from the Taylor Reynolds number Re_lambda = (2 pi)^(1/4)/4 rho0/mu0
    sqrt(2 A0) k0^(3/2).  Every Fourier mode has the amplitude of the
    spectrum (|u_k|^2 = E(k)/(2 pi k^2)), a random direction normal to k
    and a random phase; the field is scaled to the u_rms of the continuous
    spectrum, u_rms^2 = 2 K0/3, K0 = 3 A0 sqrt(2 pi) k0^5/64.  Velocities are
    exact cell averages of that Fourier field (each mode times the cell's
    sinc factors); rho E uses the averaged velocity (reading).
    Returns (q, lo, hi, TurbulenceParams)."""
    rng = np.random.default_rng(seed)
    N = int(n)
    lo, hi = (-math.pi,) * 3, (math.pi,) * 3
    h = 2 * math.pi / N
    k1 = np.fft.fftfreq(N, d=1.0 / N)  # integer wavenumbers on a 2 pi box
    KZ, KY, KX = np.meshgrid(k1, k1, k1, indexing="ij")
    kk = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    # random real field per component -> divergence-free part -> amplitudes
    uh = [np.fft.fftn(rng.standard_normal((N, N, N))) for _ in range(3)]
    with np.errstate(invalid="ignore", divide="ignore"):
        kdotu = (KX * uh[0] + KY * uh[1] + KZ * uh[2]) / np.where(kk > 0, kk * kk, 1.0)
        uh = [uh[0] - KX * kdotu, uh[1] - KY * kdotu, uh[2] - KZ * kdotu]
        mag = np.sqrt(np.abs(uh[0]) ** 2 + np.abs(uh[1]) ** 2 + np.abs(uh[2]) ** 2)
        E = A0 * kk ** 4 * np.exp(-2.0 * kk ** 2 / k0 ** 2)
        amp = np.where((kk > 0) & (mag > 0), np.sqrt(E / (2 * math.pi * np.where(kk > 0, kk * kk, 1.0))) /
                       np.where(mag > 0, mag, 1.0), 0.0)
    # no Nyquist modes: their projection would break the symmetry of a real field
    nyq = (np.abs(KX) == N // 2) | (np.abs(KY) == N // 2) | (np.abs(KZ) == N // 2)
    amp = np.where(nyq, 0.0, amp)
    # FFT convention u(x) = sum_k u_k exp(i k x) with u_k = fftn(u) / N^3
    sinc = 1.0
    for K in (KX, KY, KZ):
        a = 0.5 * K * h
        sinc = sinc * np.where(a == 0, 1.0, np.sin(a) / np.where(a == 0, 1.0, a))
    u_pt = [np.real(np.fft.ifftn(uh[d] * amp)) * N ** 3 for d in range(3)]  # point values
    u_av = [np.real(np.fft.ifftn(uh[d] * amp * sinc)) * N ** 3 for d in range(3)]
    K0 = 3.0 * A0 * math.sqrt(2 * math.pi) * k0 ** 5 / 64.0
    u_rms = math.sqrt(2.0 * K0 / 3.0)
    scale = u_rms / math.sqrt(np.mean(u_pt[0] ** 2 + u_pt[1] ** 2 + u_pt[2] ** 2) / 3.0)
    u_av = [u * scale for u in u_av]
    T0 = 3.0 * u_rms ** 2 / (gamma * mach_t ** 2)
    p0 = rho0 * T0
    mu0 = (2 * math.pi) ** 0.25 / 4.0 * rho0 * math.sqrt(2 * A0) * k0 ** 1.5 / re_lambda
    tau_t0 = math.sqrt(32.0 / A0) * (2 * math.pi) ** 0.25 * k0 ** -3.5
    rho = np.full((N, N, N), rho0)
    q = np.stack([rho, rho * u_av[0], rho * u_av[1], rho * u_av[2],
                  p0 / (gamma - 1.0) + 0.5 * rho * (u_av[0] ** 2 + u_av[1] ** 2 + u_av[2] ** 2)]).astype(np.float64)
    return q, lo, hi, TurbulenceParams(A0, k0, u_rms, K0, T0, p0, mu0, tau_t0)


def turbulence_stats(q, gamma=1.4):
    """Volume statistics of a periodic cubic state: turbulent kinetic energy
    K = <rho |u|^2>/(2 <rho>), rho_rms, the velocity-derivative skewness
    S_u = <(du_i/dx_i)^3>/<(du_i/dx_i)^2>^(3/2) (mean over i, spectral
    derivatives on a 2 pi box) and the divergence rms."""
    rho = q[0]
    u = [q[1 + d] / rho for d in range(3)]
    K = float(np.mean(rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)) / (2.0 * np.mean(rho)))
    rho_rms = float(np.sqrt(np.mean((rho - rho.mean()) ** 2)))
    N = rho.shape[0]
    k1 = np.fft.fftfreq(N, d=1.0 / N)
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    ks = (kx, ky, kz)
    dii = [np.real(np.fft.ifftn(1j * ks[d] * np.fft.fftn(u[d]))) for d in range(3)]
    s3 = np.mean([np.mean(x ** 3) for x in dii])
    s2 = np.mean([np.mean(x ** 2) for x in dii])
    div = dii[0] + dii[1] + dii[2]
    return {"K": K, "rho_rms": rho_rms, "skewness": float(s3 / s2 ** 1.5), "div_rms": float(np.sqrt(np.mean(div ** 2)))}


def taylor_green(n, mach=0.1, gamma=1.4, L=1.0, V0=1.0, rho0=1.0):
    """Taylor-Green vortex on [-pi L, pi L]^3 (Sec. 4): u = V0 sin x cos y cos z,
    v = -V0 cos x sin y cos z, w = 0, p = p0 + rho0 V0^2/16 (cos 2x + cos 2y)(cos 2z + 2).
    Reading of "uniform temperature": rho = rho0 p/p0 with p0 = rho0 V0^2/(gamma M0^2)."""
    lo = (-math.pi * L,) * 3
    hi = (math.pi * L,) * 3
    p0 = rho0 * V0 * V0 / (gamma * mach * mach)
    box = Box(tuple(n), lo, hi)

    def fn(x, y, z):
        u = V0 * np.sin(x / L) * np.cos(y / L) * np.cos(z / L)
        v = -V0 * np.cos(x / L) * np.sin(y / L) * np.cos(z / L)
        w = np.zeros_like(u)
        p = p0 + rho0 * V0 * V0 / 16.0 * (np.cos(2 * x / L) + np.cos(2 * y / L)) * (np.cos(2 * z / L) + 2.0)
        rho = rho0 * p / p0
        return rho, u, v, w, p

    return cell_average(box, fn, gamma), lo, hi


def octant_riemann(n, seed=0, gamma=1.4):
    """3D octant Riemann problem on [0,1]^3: eight constant states, one per
    octant, rho, p ~ U[0.1, 1.5], velocity direction uniform on the sphere
    with magnitude U[0, 1] (seeded).  Exact averages for even n."""
    rng = np.random.default_rng(seed)
    rho_o = rng.uniform(0.1, 1.5, 8)
    p_o = rng.uniform(0.1, 1.5, 8)
    dirs = rng.normal(size=(8, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    vel = dirs * rng.uniform(0.0, 1.0, (8, 1))
    box = Box(tuple(n), (0.0,) * 3, (1.0,) * 3)
    x, y, z = box.centres()
    o = (x > 0.5).astype(int) + 2 * (y > 0.5).astype(int) + 4 * (z > 0.5).astype(int)
    return _conservative(rho_o[o], vel[o, 0], vel[o, 1], vel[o, 2], p_o[o], gamma)


def uniform_flow(n, rho=1.0, u=(1.0, 1.0, 1.0), p=1.0, gamma=1.4):
    """Uniform free stream (Sec. 4 geometric conservation test)."""
    shape = (n[2], n[1], n[0])
    one = np.ones(shape)
    return _conservative(rho * one, u[0] * one, u[1] * one, u[2] * one, p * one, gamma)


def smooth_random(n, seed=0, gamma=1.4, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), amp=0.1, modes=3):
    """Seeded smooth periodic state: a few random Fourier modes on each
    primitive variable around rho = 1, p = 1, |U| ~ 0.3 (point values at
    cell centres, taken as cell averages)."""
    rng = np.random.default_rng(seed)
    box = Box(tuple(n), tuple(lo), tuple(hi))
    x, y, z = box.centres()
    L = [hi[d] - lo[d] for d in range(3)]

    def field(base, a):
        f = np.full(x.shape, base, dtype=np.float64)
        for _ in range(modes):
            k = rng.integers(-2, 3, 3)
            ph = rng.uniform(0, 2 * math.pi)
            c = rng.uniform(-a, a)
            f += c * np.sin(2 * math.pi * (k[0] * (x - lo[0]) / L[0] + k[1] * (y - lo[1]) / L[1]
                                           + k[2] * (z - lo[2]) / L[2]) + ph)
        return f

    rho = field(1.0, amp)
    u = field(0.3, amp)
    v = field(-0.2, amp)
    w = field(0.1, amp)
    p = field(1.0, amp)
    return _conservative(rho, u, v, w, p, gamma)


def primitive(q, gamma=1.4):
    """(rho, u, v, w, p) of a conservative state array."""
    rho = q[0]
    u, v, w = q[1] / rho, q[2] / rho, q[3] / rho
    p = (gamma - 1.0) * (q[4] - 0.5 * rho * (u * u + v * v + w * w))
    return rho, u, v, w, p
