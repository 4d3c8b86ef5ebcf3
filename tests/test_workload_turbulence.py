"""Isotropic-turbulence initial data (Sec. 4), host only: divergence-free,
the specified u_rms and spectrum, Ma_t and Re_lambda as defined, uniform
density and temperature, reproducible from the seed."""
import math

import numpy as np

from paper_1909_01580_gb300 import workloads as W


def _spectrum(u, N):
    k1 = np.fft.fftfreq(N, d=1.0 / N)
    kz, ky, kx = np.meshgrid(k1, k1, k1, indexing="ij")
    kk = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    e = sum(np.abs(np.fft.fftn(c) / N ** 3) ** 2 for c in u) * 0.5
    shells = np.rint(kk).astype(int)
    return np.bincount(shells.ravel(), weights=e.ravel())


def test_turbulence_field():
    N, mach = 64, 0.5
    q, lo, hi, P = W.isotropic_turbulence(N, mach, seed=3)
    q2, _, _, _ = W.isotropic_turbulence(N, mach, seed=3)
    assert np.array_equal(q, q2)
    assert np.all(q[0] == 1.0)
    u = [q[1 + d] / q[0] for d in range(3)]
    p = 0.4 * (q[4] - 0.5 * q[0] * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2))
    assert np.abs(p - P.p0).max() < 1e-12 * P.p0
    st = W.turbulence_stats(q)
    # divergence-free to round-off against the velocity-gradient scale
    assert st["div_rms"] < 1e-12 * P.u_rms * P.k0
    # constants as defined
    assert abs(math.sqrt(3) * P.u_rms / math.sqrt(1.4 * P.T0) - mach) < 1e-12
    assert abs(P.u_rms ** 2 - 2 * P.K0 / 3) < 1e-12
    re_l = (2 * math.pi) ** 0.25 / 4 * 1.0 / P.mu0 * math.sqrt(2 * P.A0) * P.k0 ** 1.5
    assert abs(re_l - 72.0) < 1e-9
    # cell averages carry the sinc filter: about exp(-k0^2 h^2 / 12) of the energy
    h = 2 * math.pi / N
    assert 0.9 < st["K"] / P.K0 < 1.0
    # the shell spectrum of the averages is E(k) = A0 k^4 exp(-2 k^2/k0^2)
    # times the shell mean of the cells' sinc^2 factor, exp(-k^2 h^2/12) to
    # leading order (shells of integer radius hold about 4 pi k^2 modes, so
    # the shell sums scatter by a few per cent)
    E = _spectrum(u, N)
    for k in (4, 6, 8, 10, 12):
        Ek = P.A0 * k ** 4 * math.exp(-2 * k ** 2 / P.k0 ** 2)
        filt = math.exp(-(k * h) ** 2 / 12.0)
        assert abs(E[k] / filt - Ek) < 0.15 * Ek, (k, E[k] / filt, Ek)
