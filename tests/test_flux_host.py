"""Host check of the Gauss-point gas-kinetic flux of the device header
(gks_flux compiled for the host) against the oracle's point flux (Sec. 3,
eq. (flux) and eq. (expansion-1)) on the same seeded inputs as the GPU point
flux tests: Euler, Navier-Stokes, and Navier-Stokes with the Prandtl
correction, FP64 to the GPU parity tolerances and FP32 to the mixed path's.
It checks the flux arithmetic of the CUDA path without a GPU; the GPU tests
check the same function in its kernels."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from tests._cases import max_rel, random_point_inputs

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1909_01580_gb300", "csrc")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    out = tmp_path_factory.mktemp("flux") / "flux_host_check"
    cmd = ["g++", "-std=c++17", "-O1", "-I/usr/local/cuda/include", "-I" + CSRC,
           os.path.join(HERE, "flux_host_check.cpp"), "-o", str(out)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "cuda_runtime.h" in r.stderr:
        pytest.skip("CUDA headers not found")
    assert r.returncode == 0, r.stderr
    return str(out)


def _host_flux(exe, tmp, inp, dt, gamma, mu, Pr, bits, gs=None):
    fin, fout = tmp / "in.bin", tmp / "out.bin"
    np.ascontiguousarray(inp, dtype=np.float64).tofile(fin)
    args = [exe, str(bits), repr(dt), repr(gamma), repr(mu), repr(Pr), "0.01", "1.0", str(len(inp)), str(fin),
            str(fout)] + ([repr(gs)] if gs is not None else [])
    r = subprocess.run(args, capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stderr)
    out = np.fromfile(fout, dtype=np.float64).reshape(len(inp), 10)
    return out[:, :5], out[:, 5:]


@pytest.mark.parametrize("mu,Pr", [(0.0, 1.0), (0.02, 1.0), (0.02, 0.72)])
@pytest.mark.parametrize("gs", [None, 16.0])
def test_host_flux_fp64_matches_oracle(exe, tmp_path, mu, Pr, gs):
    """gs: gradients passed in the scaled frame of a cube of edge 1/16 with
    the gradient scale, as the uniform mesh's face kernel passes them."""
    rng = np.random.default_rng(11)
    inp = random_point_inputs(rng, 48)
    dt = 0.05
    cfg = oracle.make_cfg((4, 4, 4), mu=mu, Pr=Pr)
    Fo, dFo = oracle.point_flux(cfg, inp, dt)
    F, dF = _host_flux(exe, tmp_path, inp, dt, 1.4, mu, Pr, 64, gs)
    assert max_rel(F, Fo, axis_vars=1) <= 1e-12
    assert max_rel(dF, dFo, axis_vars=1) <= 1e-9


@pytest.mark.parametrize("gs", [None, 16.0, 128.0 / (2.0 * np.pi)])
def test_host_flux_fp32_within_the_mixed_tolerance(exe, tmp_path, gs):
    """gs as above; 128/(2 pi) is the scale 1/h of the TGV 128^3 mesh, which
    the mixed face kernel folds into the FP32 constants of its slope solves."""
    rng = np.random.default_rng(13)
    inp = random_point_inputs(rng, 48)
    dt = 0.05
    cfg = oracle.make_cfg((4, 4, 4), mu=0.02, Pr=0.72)
    Fo, dFo = oracle.point_flux(cfg, inp, dt)
    F, dF = _host_flux(exe, tmp_path, inp, dt, 1.4, 0.02, 0.72, 32, gs)
    assert max_rel(F, Fo, axis_vars=1) <= 2e-5
