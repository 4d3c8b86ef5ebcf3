"""Pins of the oracle's positivity fallback (Sec. 4): a cell drops to first
order when the density or the pressure of any of its 25 candidate
polynomials (P0 and the 24 linear P_m) is negative at any of the 24 Gauss
points of its six faces, and only then.

The cells are built by hand on a uniform cube mesh, where the polynomials
have closed forms: P0 reproduces quadratic data, and each P_m is the
least-squares plane through its four neighbours.  The data below were
chosen so that

* case "one": exactly one P_m of one variable is negative, at exactly one
  of the 24 Gauss points (on a y-face), while P0 and the combined
  polynomial P~ stay positive at all of them -- an oracle that tests P0
  alone, P~ alone, or only the x-faces would not flag it;
* case "pressure": the same shape in the pressure with a uniform density
  -- an oracle that tests the density alone would not flag it;
* case "off_gauss": every candidate polynomial is positive at the 24 Gauss
  points, but one of them is negative at a face corner -- an oracle that
  samples the cell anywhere else would flag it.

The construction is checked in the test itself with numpy least squares on
the integer offsets (the closed form on cubes), independently of the
oracle's Householder solve over Gauss-quadrature moments.
"""
import itertools
import math

import numpy as np
import pytest

import oracle

GAMMA = 1.4
S3 = math.sqrt(3.0) / 6.0  # 2-point Gauss nodes on [-1/2, 1/2]
N = 5
C = (2, 2, 2)  # the hand-built cell (periodic 5^3 box)


def _gauss_points():
    pts = []
    for d in range(3):
        for s in (-0.5, 0.5):
            for a in (-S3, S3):
                for b in (-S3, S3):
                    p = [0.0, 0.0, 0.0]
                    p[d] = s
                    e = [x for x in range(3) if x != d]
                    p[e[0]], p[e[1]] = a, b
                    pts.append(p)
    return np.array(pts)


def _face_lattice():
    """Corners, edge midpoints and centres of the six faces."""
    pts = []
    for d in range(3):
        for s in (-0.5, 0.5):
            for a in (-0.5, 0.0, 0.5):
                for b in (-0.5, 0.0, 0.5):
                    p = [0.0, 0.0, 0.0]
                    p[d] = s
                    e = [x for x in range(3) if x != d]
                    p[e[0]], p[e[1]] = a, b
                    pts.append(p)
    return np.array(pts)


BIG = [o for o in itertools.product((-1, 0, 1), repeat=3) if o != (0, 0, 0) and sum(map(abs, o)) <= 2]


def _sub_stencils():
    """The 24 sub-stencils {c, s_a e_a, s_b e_b, s_a e_a + s_b e_b, s_c e_c}
    for the planes (a, b, c) = (x, y, z), (y, z, x), (z, x, y)."""
    subs = []
    for a, b, c in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
        for sa, sb, sc in itertools.product((1, -1), repeat=3):
            A = [0, 0, 0]
            A[a] = sa
            B = [0, 0, 0]
            B[b] = sb
            D = [0, 0, 0]
            D[a], D[b] = sa, sb
            Cc = [0, 0, 0]
            Cc[c] = sc
            subs.append([tuple(A), tuple(B), tuple(D), tuple(Cc)])
    return subs


def _candidates(qc, nb):
    """Closed-form candidate polynomials on a unit cube from the centre value
    qc and the neighbour values nb[offset]: P0's 9 coefficients (columns
    X, Y, Z, X^2, Y^2, Z^2, XY, XZ, YZ about zero-mean monomials) and the
    24 gradients of the P_m."""
    rows = np.array([[o[0], o[1], o[2], o[0] ** 2, o[1] ** 2, o[2] ** 2, o[0] * o[1], o[0] * o[2], o[1] * o[2]]
                     for o in BIG], float)
    a = np.linalg.lstsq(rows, np.array([nb[o] - qc for o in BIG]), rcond=None)[0]
    bs = [np.linalg.lstsq(np.array(S, float), np.array([nb[o] - qc for o in S]), rcond=None)[0]
          for S in _sub_stencils()]
    return a, bs


def _values(qc, a, bs, P):
    X, Y, Z = P.T
    m = 1.0 / 12.0
    p0 = (qc + a[0] * X + a[1] * Y + a[2] * Z + a[3] * (X * X - m) + a[4] * (Y * Y - m) + a[5] * (Z * Z - m)
          + a[6] * X * Y + a[7] * X * Z + a[8] * Y * Z)
    pm = np.array([qc + b[0] * X + b[1] * Y + b[2] * Z for b in bs])
    return p0, pm


def _case_one_values():
    """A linear field 1 + g.o with g = (-0.3, -0.2, 0.1), plus 1.7 on the
    neighbour (0, +1, 0) and 2.4 on (+1, 0, -1); every value >= 0.5."""
    g = np.array([-0.3, -0.2, 0.1])
    nb = {o: 1.0 + float(np.dot(g, o)) for o in BIG}
    nb[(0, 1, 0)] += 1.7
    nb[(1, 0, -1)] += 2.4
    return 1.0, nb


def _case_off_gauss_values():
    nb = {(-1, -1, 0): 1.0, (-1, 0, -1): 2.3, (-1, 0, 0): 1.8, (-1, 0, 1): 0.9, (-1, 1, 0): 2.1,
          (0, -1, -1): 0.9, (0, -1, 0): 0.1, (0, -1, 1): 0.1, (0, 0, -1): 1.4, (0, 0, 1): 0.2,
          (0, 1, -1): 2.1, (0, 1, 0): 1.4, (0, 1, 1): 0.8, (1, -1, 0): 0.1, (1, 0, -1): 1.1,
          (1, 0, 0): 0.7, (1, 0, 1): 0.1, (1, 1, 0): 1.2}
    return 1.0, nb


def _state(field, qc, nb):
    """Periodic 5^3 state at rest: the hand-built values in `field` ('rho':
    density, uniform pressure 1; 'p': pressure, uniform density 1) at the
    cell C and its 18 big-stencil neighbours, 1 elsewhere."""
    vals = np.ones((N, N, N))
    i, j, k = C
    vals[k, j, i] = qc
    for o, v in nb.items():
        vals[k + o[2], j + o[1], i + o[0]] = v
    q = np.zeros((5, N, N, N))
    if field == "rho":
        q[0] = vals
        q[4] = 1.0 / (GAMMA - 1.0)
    else:
        q[0] = 1.0
        q[4] = vals / (GAMMA - 1.0)
    return q


def _lin(c):
    return c[0] + N * (c[1] + N * c[2])


def _box():
    return (0.0, 0.0, 0.0), (float(N), float(N), float(N))


@pytest.mark.parametrize("field", ["rho", "p"])
def test_one_negative_substencil_value_flags(field):
    qc, nb = _case_one_values()
    a, bs = _candidates(qc, nb)
    p0, pm = _values(qc, a, bs, _gauss_points())
    neg = np.argwhere(pm < 0)
    # the construction: exactly one (P_m, Gauss point) pair negative, on a
    # y-face, with a clear margin; P0 positive everywhere on the 24 points
    assert neg.shape[0] == 1, neg
    m, g = neg[0]
    assert pm[m, g] < -0.09 and np.delete(pm.ravel(), m * 24 + g).min() > 0.07
    assert abs(_gauss_points()[g][1]) == 0.5
    assert p0.min() > 0.8
    lo, hi = _box()
    q = _state(field, qc, nb)
    coef, flag, _ = oracle.reconstruct(oracle.make_cfg((N, N, N), lo, hi), q)
    c = _lin(C)
    assert flag[c] == 1
    # the fallback: P~ := Q_c for all five variables
    assert np.all(coef[c, :, 1:] == 0.0)
    assert np.array_equal(coef[c, :, 0], q.reshape(5, -1)[:, c])
    # without the fallback, the combined polynomial P~ is positive at every
    # Gauss point, so a test of P~ alone would miss the negative P_m
    cfg0 = oracle.make_cfg((N, N, N), lo, hi, limiter=0)
    coef0, flag0, _ = oracle.reconstruct(cfg0, q)
    assert flag0[c] == 0 and np.any(coef0[c, :, 1:] != 0.0)
    xg = np.array(C, float) + 0.5 + _gauss_points()
    ev = oracle.eval_reconstruction(cfg0, q, c, xg)
    rho, mom, E = ev[:, 0, 0], ev[:, 1:4, 0], ev[:, 4, 0]
    p = (GAMMA - 1.0) * (E - 0.5 * (mom ** 2).sum(axis=1) / rho)
    assert rho.min() > 0.0 and p.min() > 0.0


@pytest.mark.parametrize("field", ["rho", "p"])
def test_negative_only_off_the_gauss_points_does_not_flag(field):
    qc, nb = _case_off_gauss_values()
    a, bs = _candidates(qc, nb)
    p0, pm = _values(qc, a, bs, _gauss_points())
    assert min(p0.min(), pm.min()) > 0.08
    f0, fm = _values(qc, a, bs, _face_lattice())
    assert min(f0.min(), fm.min()) < -0.2
    lo, hi = _box()
    q = _state(field, qc, nb)
    coef, flag, _ = oracle.reconstruct(oracle.make_cfg((N, N, N), lo, hi), q)
    assert flag[_lin(C)] == 0
    assert np.any(coef[_lin(C), 0 if field == "rho" else 4, 1:] != 0.0)


def test_smooth_positive_cell_does_not_flag_and_uniform_fallback_is_noop():
    """Linear data with all 25 polynomials positive: no flag; a uniform
    state: no flag and zero coefficients."""
    g = np.array([0.3, -0.2, 0.1])
    nb = {o: 1.0 + float(np.dot(g, o)) for o in BIG}
    lo, hi = _box()
    q = _state("rho", 1.0, nb)
    coef, flag, _ = oracle.reconstruct(oracle.make_cfg((N, N, N), lo, hi), q)
    assert flag[_lin(C)] == 0
    # linear data: P~ = P0 = the plane itself (scaled coefficients = g)
    assert np.allclose(coef[_lin(C), 0, 1:4], g, atol=1e-13)
