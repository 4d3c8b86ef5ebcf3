"""The alternative big stencil S' and its 8 sub-stencils (Remark of Sec. 2)
in the oracle: the tables against the printed ones, exact reproduction of
quadratic data by P0 over S', and linear weights for linear data."""
import os

import numpy as np

import oracle
from tests.test_oracle_reconstruction import (_quad_grad, _quadratic_averages, _random_quadratic,
                                              _state_from_scalars)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
GAMMA_LIN = 0.0025


def test_sprime_tables():
    big, sub = oracle.stencils_sprime()
    big_s, _ = oracle.stencils()
    assert {tuple(o) for o in big} == {tuple(o) for o in big_s} | {
        (s * (d == 0), s * (d == 1), s * (d == 2)) for d in range(3) for s in (-2, 2)}
    assert len({tuple(o) for o in big}) == 24
    rows = np.loadtxt(os.path.join(GOLDEN, "substencils_sprime_printed.txt"), dtype=int)
    for m in (1, 2, 3, 5, 6, 7):
        printed = {tuple(r[1:]) for r in rows if r[0] == m}
        assert {tuple(o) for o in sub[m - 1]} == printed, m
    # reading of the repeated S'_4 and S'_8: the family is the 8 octants
    octants = {tuple(int(np.sign(o).sum()) for o in np.array(sub[m]).T) for m in range(8)}
    assert len(octants) == 8
    for m in range(8):
        cells = np.array(sub[m])
        assert (np.abs(cells).sum(axis=1) == 1).all() and (np.abs(cells).sum(axis=0) == 1).all()


def test_sprime_P0_reproduces_quadratic_data_exactly():
    rng = np.random.default_rng(11)
    n, lo, hi = (7, 7, 7), (0.0, 0.0, 0.0), (1.4, 1.4, 1.4)
    quads = [_random_quadratic(rng) for _ in range(5)]
    quads[0] = (2.0,) + quads[0][1:]
    quads[4] = (5.0,) + quads[4][1:]
    q = _state_from_scalars([_quadratic_averages(n, lo, hi, c) for c in quads])
    cfg = oracle.make_cfg(n, lo, hi, stencil=1)
    _, _, a0 = oracle.reconstruct(cfg, q)
    hh = 0.2
    for (i, j, k) in [(2, 2, 2), (3, 4, 2), (4, 3, 4)]:
        lin = i + 7 * (j + 7 * k)
        xc = np.array([(i + 0.5) * hh, (j + 0.5) * hh, (k + 0.5) * hh])
        for v in range(5):
            g = _quad_grad(quads[v], xc)
            C = quads[v][2]
            expect = [hh * g[0], hh * g[1], hh * g[2], hh * hh * C[0, 0], hh * hh * C[1, 1], hh * hh * C[2, 2],
                      hh * hh * C[0, 1], hh * hh * C[0, 2], hh * hh * C[1, 2]]
            np.testing.assert_allclose(a0[lin, v], expect, rtol=0, atol=1e-13)


def test_sprime_linear_data_linear_weights():
    rng = np.random.default_rng(12)
    n, lo, hi = (7, 7, 7), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    lins = [(3.0 if v in (0, 4) else 0.5, rng.uniform(-0.2, 0.2, 3), np.zeros((3, 3))) for v in range(5)]
    q = _state_from_scalars([_quadratic_averages(n, lo, hi, c) for c in lins])
    cfg = oracle.make_cfg(n, lo, hi, stencil=1)
    coef, flag, a0 = oracle.reconstruct(cfg, q)
    assert not flag.any()
    lin = 3 + 7 * (3 + 7 * 3)
    np.testing.assert_allclose(coef[lin, :, 1:], a0[lin], rtol=0, atol=1e-14)
    beta, wbar = oracle.weno_weights(cfg, q, lin)
    g = np.zeros(25)
    g[0] = 1.0 - 8 * GAMMA_LIN
    g[1:9] = GAMMA_LIN
    np.testing.assert_allclose(wbar, np.tile(g, (5, 1)), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(beta[:, :9], beta[:, :1] * np.ones((1, 9)), rtol=1e-12)
