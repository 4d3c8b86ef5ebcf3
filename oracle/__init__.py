"""HGKS oracle: plain FP64 CPU implementation of the scheme of Pan & Xu
(arXiv 1909.01580), used to check the CUDA path.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package; the product
path (``paper_1909_01580_gb300``) never does and shares no code with it.

The arithmetic lives in ``hgks_oracle.c`` (compiled with gcc, no FP
contraction); this module only builds it and marshals NumPy arrays through
ctypes.  The C header comment says how the two parts that the paper's printed
values do not reach (the positivity fallback, the Prandtl-number correction)
are pinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hgks_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Cfg(ctypes.Structure):
    """Mirror of ``orc_cfg`` in hgks_oracle.c."""
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("mesh", ctypes.c_int),
        ("amp", ctypes.c_double),
        ("omega", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("Pr", ctypes.c_double),
        ("bc", ctypes.c_int * 6),
        ("Gamma_lin", ctypes.c_double),
        ("weno_eps", ctypes.c_double),
        ("weno_pow", ctypes.c_int),
        ("tau_eps", ctypes.c_double),
        ("tau_C", ctypes.c_double),
        ("limiter", ctypes.c_int),
        ("nthreads", ctypes.c_int),
        ("charvar", ctypes.c_int),
        ("mu_pow", ctypes.c_double),
        ("T_ref", ctypes.c_double),
        ("stencil", ctypes.c_int),
    ]


def make_cfg(n, lo=(0.0, 0.0, 0.0), hi=(2.0, 2.0, 2.0), *, gamma=1.4, mu=0.0, Pr=1.0,
             bc=(0, 0, 0, 0, 0, 0), mesh=0, amp=0.0, omega=0.0, Gamma_lin=0.0025,
             weno_eps=1e-8, weno_pow=1, tau_eps=0.01, tau_C=1.0, limiter=1, nthreads=0, charvar=0,
             mu_pow=0.0, T_ref=1.0, stencil=0) -> Cfg:
    """Configuration with the paper's defaults (Gamma = 0.0025, tau constants
    eps = 0.01 and C = 1 of Sec. 4, gamma = 1.4)."""
    c = Cfg()
    for d in range(3):
        c.n[d] = int(n[d])
        c.lo[d] = float(lo[d])
        c.hi[d] = float(hi[d])
    c.mesh, c.amp, c.omega = int(mesh), float(amp), float(omega)
    c.gamma, c.mu, c.Pr = float(gamma), float(mu), float(Pr)
    for i in range(6):
        c.bc[i] = int(bc[i])
    c.Gamma_lin, c.weno_eps, c.weno_pow = float(Gamma_lin), float(weno_eps), int(weno_pow)
    c.tau_eps, c.tau_C = float(tau_eps), float(tau_C)
    c.limiter, c.nthreads = int(limiter), int(nthreads)
    c.charvar = int(charvar)
    c.mu_pow, c.T_ref = float(mu_pow), float(T_ref)
    c.stencil = int(stencil)
    return c


# rate(ctx, stage, y, L, dL) of orc_two_stage
RATE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.POINTER
            D = ctypes.c_double
            dp = P(D)
            cp = P(Cfg)
            L.orc_point_flux.argtypes = [cp, dp, dp, D, dp, dp]
            L.orc_point_flux.restype = ctypes.c_int
            L.orc_operator.argtypes = [cp, dp, D, D, ctypes.c_long, P(ctypes.c_long), dp, dp]
            L.orc_operator.restype = ctypes.c_int
            L.orc_reconstruct.argtypes = [cp, dp, D, dp, P(ctypes.c_int), dp]
            L.orc_reconstruct.restype = ctypes.c_int
            L.orc_eval_reconstruction.argtypes = [cp, dp, D, ctypes.c_long, ctypes.c_int, dp, dp]
            L.orc_eval_reconstruction.restype = ctypes.c_int
            L.orc_weno_weights.argtypes = [cp, dp, D, ctypes.c_long, dp, dp]
            L.orc_weno_weights.restype = ctypes.c_int
            L.orc_cfl_dt.argtypes = [cp, dp, D, D]
            L.orc_cfl_dt.restype = D
            L.orc_volumes.argtypes = [cp, D, dp]
            L.orc_volumes.restype = ctypes.c_int
            L.orc_step.argtypes = [cp, dp, dp, ctypes.c_int, D, D, D, dp, P(ctypes.c_int)]
            L.orc_step.restype = ctypes.c_int
            L.orc_moments_1d.argtypes = [D, D, ctypes.c_int, dp]
            L.orc_moments_1d.restype = None
            L.orc_moment_matrix.argtypes = [cp, dp, dp]
            L.orc_moment_matrix.restype = None
            L.orc_time_integrals.argtypes = [D, D, dp]
            L.orc_time_integrals.restype = None
            L.orc_stencils.argtypes = [P(ctypes.c_int), P(ctypes.c_int)]
            L.orc_char_basis.argtypes = [cp, dp, ctypes.c_int, dp, dp]
            L.orc_stencils_sprime.argtypes = [P(ctypes.c_int), P(ctypes.c_int)]
            L.orc_char_basis.restype = ctypes.c_int
            L.orc_stencils.restype = None
            L.orc_two_stage.argtypes = [ctypes.c_long, dp, D, RATE_FN, ctypes.c_void_p]
            L.orc_two_stage.restype = ctypes.c_int
            L.orc_threads_used.argtypes = [cp]
            L.orc_threads_used.restype = ctypes.c_int
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def ncells(cfg: Cfg) -> int:
    return cfg.n[0] * cfg.n[1] * cfg.n[2]


def point_flux(cfg: Cfg, inp, dt: float, ug=None):
    """Gas-kinetic flux at Gauss points.  inp[..., 40] (local frame: W_l,
    dW_l/dn_x,y,z, W_r, dW_r/dn_x,y,z) -> (F[..., 5], dF[..., 5])."""
    inp = _f64(inp)
    shape = inp.shape[:-1]
    flat = inp.reshape(-1, 40)
    ugs = None if ug is None else _f64(np.broadcast_to(ug, shape + (3,))).reshape(-1, 3)
    F = np.zeros((flat.shape[0], 5))
    dF = np.zeros((flat.shape[0], 5))
    L = lib()
    for p in range(flat.shape[0]):
        row = np.ascontiguousarray(flat[p])
        u = None if ugs is None else np.ascontiguousarray(ugs[p])
        fo = np.zeros(5)
        dfo = np.zeros(5)
        rc = L.orc_point_flux(ctypes.byref(cfg), _dp(row), None if u is None else _dp(u), float(dt), _dp(fo), _dp(dfo))
        if rc != 0:
            raise RuntimeError("oracle point flux failed")
        F[p], dF[p] = fo, dfo
    return F.reshape(shape + (5,)), dF.reshape(shape + (5,))


def operator(cfg: Cfg, q, dt: float, t: float = 0.0, cells=None):
    """L(Q) and dL/dt(Q) (eq. finite and its time derivative).  q: [5][nz][ny][nx].
    With ``cells`` (linear indices), only those cells: outputs [5][len(cells)]."""
    q = _f64(q)
    if cells is None:
        n = ncells(cfg)
        ptr = None
        nc = -1
    else:
        cl = np.ascontiguousarray(np.asarray(cells, dtype=np.int64))
        n = cl.size
        ptr = cl.ctypes.data_as(ctypes.POINTER(ctypes.c_long))
        nc = n
    L = np.zeros((5, n))
    dL = np.zeros((5, n))
    rc = lib().orc_operator(ctypes.byref(cfg), _dp(q), float(t), float(dt), nc, ptr, _dp(L), _dp(dL))
    if rc != 0:
        raise RuntimeError("oracle operator failed")
    if cells is None:
        shp = (5, cfg.n[2], cfg.n[1], cfg.n[0])
        return L.reshape(shp), dL.reshape(shp)
    return L, dL


def reconstruct(cfg: Cfg, q, t: float = 0.0):
    """(coef[ncell,5,10], flag[ncell], a0[ncell,5,9]): P~ as (Q_c, 9 coefficients
    in the cell's scaled frame) and the big-stencil polynomial P0."""
    q = _f64(q)
    n = ncells(cfg)
    coef = np.zeros((n, 5, 10))
    a0 = np.zeros((n, 5, 9))
    flag = np.zeros(n, dtype=np.int32)
    lib().orc_reconstruct(ctypes.byref(cfg), _dp(q), float(t), _dp(coef),
                          flag.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(a0))
    return coef, flag, a0


def eval_reconstruction(cfg: Cfg, q, cell: int, x, t: float = 0.0):
    """Values and gradients of cell's P~ at physical points x[np,3] -> [np,5,4]."""
    q = _f64(q)
    x = _f64(x).reshape(-1, 3)
    out = np.zeros((x.shape[0], 5, 4))
    rc = lib().orc_eval_reconstruction(ctypes.byref(cfg), _dp(q), float(t), int(cell), x.shape[0], _dp(x), _dp(out))
    if rc != 0:
        raise RuntimeError("oracle eval failed")
    return out


def weno_weights(cfg: Cfg, q, cell: int, t: float = 0.0):
    """(beta[5,25], wbar[5,25]) of one cell; index 0 is the big stencil."""
    q = _f64(q)
    beta = np.zeros((5, 25))
    wbar = np.zeros((5, 25))
    rc = lib().orc_weno_weights(ctypes.byref(cfg), _dp(q), float(t), int(cell), _dp(beta), _dp(wbar))
    if rc != 0:
        raise RuntimeError("oracle weno weights failed")
    return beta, wbar


def cfl_dt(cfg: Cfg, q, cfl: float, t: float = 0.0) -> float:
    q = _f64(q)
    return float(lib().orc_cfl_dt(ctypes.byref(cfg), _dp(q), float(t), float(cfl)))


def volumes(cfg: Cfg, t: float = 0.0) -> np.ndarray:
    v = np.zeros(ncells(cfg))
    lib().orc_volumes(ctypes.byref(cfg), float(t), _dp(v))
    return v.reshape(cfg.n[2], cfg.n[1], cfg.n[0])


def step(cfg: Cfg, q, t: float, nsteps: int, cfl: float = 0.35, dt_fixed: float = 0.0,
         t_end: float = float("inf"), vol=None):
    """Advance nsteps two-stage steps.  Returns (q_new, t_new, steps_done, vol)."""
    q = _f64(q).copy()
    tt = ctypes.c_double(float(t))
    done = ctypes.c_int(0)
    v = None
    if vol is not None:
        v = _f64(vol).copy()
    rc = lib().orc_step(ctypes.byref(cfg), _dp(q), ctypes.byref(tt), int(nsteps), float(cfl), float(dt_fixed),
                        float(t_end), None if v is None else _dp(v), ctypes.byref(done))
    if rc != 0:
        raise RuntimeError("oracle step failed")
    return q, tt.value, done.value, v


def two_stage(y, dt: float, nsteps: int, rate):
    """Advance y by nsteps steps of the oracle's two-stage fourth-order
    routine (the one every scheme step runs through), with the rate pair
    supplied from Python: rate(stage, y) -> (L, dL/dt), arrays like y."""
    y = _f64(y).copy().ravel()
    n = y.size

    def cb(_ctx, stage, yp, Lp, dLp):
        yy = np.ctypeslib.as_array(yp, shape=(n,)).copy()
        L, dL = rate(int(stage), yy)
        np.ctypeslib.as_array(Lp, shape=(n,))[:] = L
        np.ctypeslib.as_array(dLp, shape=(n,))[:] = dL
        return 0

    fn = RATE_FN(cb)
    for _ in range(nsteps):
        if lib().orc_two_stage(n, _dp(y), float(dt), fn, None) != 0:
            raise RuntimeError("oracle two-stage step failed")
    return y


def moments_1d(U: float, lam: float, side: int) -> np.ndarray:
    out = np.zeros(11)
    lib().orc_moments_1d(float(U), float(lam), int(side), _dp(out))
    return out


def moment_matrix(cfg: Cfg, W) -> np.ndarray:
    W = _f64(W)
    M = np.zeros(25)
    lib().orc_moment_matrix(ctypes.byref(cfg), _dp(W), _dp(M))
    return M.reshape(5, 5)


def time_integrals(delta: float, tau: float) -> np.ndarray:
    q = np.zeros(6)
    lib().orc_time_integrals(float(delta), float(tau), _dp(q))
    return q


def stencils():
    big = np.zeros(18 * 3, dtype=np.int32)
    sub = np.zeros(24 * 4 * 3, dtype=np.int32)
    P = ctypes.POINTER(ctypes.c_int)
    lib().orc_stencils(big.ctypes.data_as(P), sub.ctypes.data_as(P))
    return big.reshape(18, 3), sub.reshape(24, 4, 3)


def stencils_sprime():
    """(big[24][3], sub[8][3][3]): the big stencil S' and its sub-stencils."""
    big = np.zeros(24 * 3, dtype=np.int32)
    sub = np.zeros(8 * 3 * 3, dtype=np.int32)
    P = ctypes.POINTER(ctypes.c_int)
    lib().orc_stencils_sprime(big.ctypes.data_as(P), sub.ctypes.data_as(P))
    return big.reshape(24, 3), sub.reshape(8, 3, 3)


def char_basis(cfg: Cfg, W, d: int):
    """(R, L): right eigenvectors (columns) of the Euler flux Jacobian along
    axis d at the conservative state W, and L = R^{-1}."""
    W = _f64(W)
    R = np.zeros(25)
    L = np.zeros(25)
    if lib().orc_char_basis(ctypes.byref(cfg), _dp(W), int(d), _dp(R), _dp(L)) != 0:
        raise RuntimeError("oracle char basis failed")
    return R.reshape(5, 5), L.reshape(5, 5)


def threads_used(cfg: Cfg) -> int:
    return int(lib().orc_threads_used(ctypes.byref(cfg)))
