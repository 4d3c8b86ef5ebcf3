"""Writes tests/golden/tgv64_10steps_oracle.txt: the FP64 oracle's state after
10 fixed-dt two-stage steps (Sec. 3, the two-stage fourth-order update) of
the Navier-Stokes Taylor-Green vortex of Sec. 4 at 64^3 (periodic
[-pi, pi]^3, Mach 0.1, Re 1600, Pr 0.72, gamma 1.4), at sampled cells, with
the per-variable maxima of the whole state.

Only the oracle computes here (the initial cell averages come from the
seeded-input module, which holds none of the scheme's arithmetic).  The
run takes about half an hour on 8 cores:

    python tests/golden/make_tgv64_golden.py
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1909_01580_gb300 import workloads as W  # noqa: E402

N = 64
STEPS = 10
CFL = 0.35
MU, PR = 1.0 / 1600.0, 0.72
OUT = os.path.join(HERE, "tgv64_10steps_oracle.txt")


def sample_cells(n: int, seed: int = 64) -> np.ndarray:
    """Linear cell indices: the eight corners (periodic wrap on every side),
    one full x-line and one full z-line through the box, and 1500 seeded
    random cells."""
    corners = [i + n * (j + n * k) for k in (0, n - 1) for j in (0, n - 1) for i in (0, n - 1)]
    xline = [i + n * (17 + n * 40) for i in range(n)]
    zline = [5 + n * (n - 3 + n * k) for k in range(n)]
    rnd = np.random.default_rng(seed).choice(n ** 3, 1500, replace=False)
    return np.unique(np.concatenate([corners, xline, zline, rnd]).astype(np.int64))


def main() -> None:
    n = (N, N, N)
    q0, lo, hi = W.taylor_green(n)
    cfg = oracle.make_cfg(n, lo, hi, mu=MU, Pr=PR)
    dt = oracle.cfl_dt(cfg, q0, CFL)
    t0 = time.perf_counter()
    q, t, done, _ = oracle.step(cfg, q0, 0.0, STEPS, dt_fixed=dt)
    el = time.perf_counter() - t0
    assert done == STEPS
    flat = q.reshape(5, -1)
    cells = sample_cells(N)
    qmax = np.abs(flat).max(axis=1)
    with open(OUT, "w") as f:
        f.write("# FP64 oracle (oracle/hgks_oracle.c) state after 10 fixed-dt two-stage steps (Sec. 3) of the\n")
        f.write("# Navier-Stokes Taylor-Green vortex of Sec. 4: periodic [-pi,pi]^3, 64^3 cells, Mach 0.1,\n")
        f.write("# Re 1600 (mu = 1/1600), Pr 0.72, gamma 1.4; initial cell averages from\n")
        f.write("# paper_1909_01580_gb300.workloads.taylor_green; dt = 0.35 * min h/(|U| + c) of the initial state.\n")
        f.write(f"# written by tests/golden/make_tgv64_golden.py ({el:.0f} s on {oracle.threads_used(cfg)} threads)\n")
        f.write(f"n {N}\nsteps {STEPS}\ndt {dt!r}\nt {t!r}\n")
        f.write("qmax " + " ".join(repr(float(v)) for v in qmax) + "\n")
        f.write("qsum " + " ".join(repr(float(v)) for v in flat.sum(axis=1)) + "\n")
        f.write(f"cells {cells.size}\n")
        f.write("# cell rho rhoU rhoV rhoW rhoE\n")
        for c in cells:
            f.write(f"{int(c)} " + " ".join(repr(float(flat[v, c])) for v in range(5)) + "\n")
    print(f"wrote {OUT}: {cells.size} cells, dt {dt:.6e}, {el:.0f} s")


if __name__ == "__main__":
    main()
