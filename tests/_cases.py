"""Shared helpers of the parity tests: seeded point-flux inputs and the
relative-difference metric.  No scheme arithmetic lives here."""
import numpy as np

GAMMA = 1.4


def conservative(rho, U, p, gamma=GAMMA):
    U = np.asarray(U, dtype=float)
    return np.array([rho, *(rho * U), p / (gamma - 1) + 0.5 * rho * U @ U])


def random_point_inputs(rng, npts, grad=0.3, jump=0.2):
    """npts Gauss-point inputs [npts, 40] in the local frame: a left state,
    a right state near it, and random directional derivatives."""
    out = np.zeros((npts, 40))
    for p in range(npts):
        rho, pr = rng.uniform(0.6, 1.4), rng.uniform(0.6, 1.4)
        U = rng.uniform(-0.5, 0.5, 3)
        Wl = conservative(rho, U, pr)
        Wr = conservative(rho * (1 + rng.uniform(-jump, jump)), U + rng.uniform(-jump, jump, 3),
                          pr * (1 + rng.uniform(-jump, jump)))
        out[p, 0:5] = Wl
        out[p, 20:25] = Wr
        for s, Wc in ((0, Wl), (1, Wr)):
            for d in range(3):
                out[p, 20 * s + 5 + 5 * d: 20 * s + 10 + 5 * d] = grad * rng.uniform(-1, 1, 5) * np.abs(Wc)
    return out


def max_rel(a, b, axis_vars=0):
    """Per conserved variable: max |a - b| / max |b| (the parity metric);
    returns the worst variable's value."""
    a = np.asarray(a)
    b = np.asarray(b)
    a2 = np.moveaxis(a, axis_vars, 0).reshape(a.shape[axis_vars], -1)
    b2 = np.moveaxis(b, axis_vars, 0).reshape(b.shape[axis_vars], -1)
    worst = 0.0
    for v in range(a2.shape[0]):
        den = np.abs(b2[v]).max()
        if den == 0.0:
            den = 1.0
        worst = max(worst, float(np.abs(a2[v] - b2[v]).max() / den))
    return worst


def max_rel_momentum(a, b):
    """The parity metric with the three momentum components measured against
    a common momentum scale (their largest |value| in b), the other variables
    against their own largest value: a momentum component that is zero at
    t = 0 (rho W of the Taylor-Green vortex) is no scale for the rounding of
    the momentum fluxes it shares with the other two."""
    a = np.asarray(a).reshape(5, -1)
    b = np.asarray(b).reshape(5, -1)
    mom = max(float(np.abs(b[1:4]).max()), 1e-300)
    worst = 0.0
    for v in range(5):
        den = mom if 1 <= v <= 3 else max(float(np.abs(b[v]).max()), 1e-300)
        worst = max(worst, float(np.abs(a[v] - b[v]).max() / den))
    return worst
