"""Thin ctypes binding of libhgks.so (include/hgks.h), same names as the C ABI.

Argument marshalling only: every step of the scheme runs in the CUDA
kernels of the library.  Host buffers are NumPy arrays; device buffers are
CUDA torch tensors (passed as raw pointers).  There is no CPU fallback: if
the library is missing or no GPU is usable, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

HGKS_FP64 = 0
HGKS_MIXED = 1
HGKS_BC_PERIODIC = 0
HGKS_BC_REFLECTIVE = 1
HGKS_BC_OUTFLOW = 2
HGKS_OK = 0
HGKS_E_INVALID = -1
HGKS_E_NOMEM = -2
HGKS_E_CUDA = -3
HGKS_E_NONPHYSICAL = -4
HGKS_E_TIMEOUT = -5
HGKS_E_STATE = -6

# every symbol include/hgks.h declares
EXPORTS = ("hgks_create", "hgks_set_option", "hgks_set_state", "hgks_get_state", "hgks_step", "hgks_flux",
           "hgks_reconstruct", "hgks_point_flux", "hgks_set_timing", "hgks_get_timing", "hgks_launch_count",
           "hgks_device_bytes", "hgks_last_error", "hgks_destroy", "hgks_flux_noalloc", "hgks_alu_peak",
           "hgks_batch_create", "hgks_batch_footprint", "hgks_batch_add", "hgks_batch_remove", "hgks_batch_step",
           "hgks_batch_poll", "hgks_batch_get_state", "hgks_batch_tune", "hgks_batch_set_tuning",
           "hgks_batch_get_tuning", "hgks_batch_launch_count", "hgks_batch_last_error", "hgks_batch_destroy")
HGKS_TUNE_NPARAM = 11


class HgksError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"hgks error {code}: {msg}")
        self.code = code


class hgks_grid_t(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("mesh", ctypes.c_int),
        ("mesh_amp", ctypes.c_double),
        ("mesh_omega", ctypes.c_double),
        ("precision", ctypes.c_int),
    ]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libhgks.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise HgksError(HGKS_E_CUDA, f"CUDA library not built: {path}")
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    dp = P(ctypes.c_double)
    vp = ctypes.c_void_p
    L.hgks_create.argtypes = [P(hgks_grid_t), ctypes.c_double, ctypes.c_double, ctypes.c_double,
                              P(ctypes.c_int), vp, P(vp)]
    L.hgks_set_option.argtypes = [vp, ctypes.c_char_p, ctypes.c_double]
    L.hgks_set_state.argtypes = [vp, vp, ctypes.c_int, ctypes.c_double]
    L.hgks_get_state.argtypes = [vp, vp, ctypes.c_int, dp]
    L.hgks_step.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp,
                            P(ctypes.c_int)]
    L.hgks_flux.argtypes = [vp, ctypes.c_double, vp, vp, ctypes.c_int]
    L.hgks_reconstruct.argtypes = [vp, vp, vp]
    L.hgks_point_flux.argtypes = [ctypes.c_int, vp, vp, ctypes.c_double, dp, ctypes.c_int, vp, vp]
    L.hgks_flux_noalloc.argtypes = [P(hgks_grid_t), ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    P(ctypes.c_int), vp, ctypes.c_double, vp, vp, vp]
    L.hgks_flux_noalloc.restype = ctypes.c_int
    ip = P(ctypes.c_int)
    L.hgks_batch_create.argtypes = [ctypes.c_int, ctypes.c_ulonglong, ctypes.c_int, vp, P(vp)]
    L.hgks_batch_footprint.argtypes = [P(hgks_grid_t)]
    L.hgks_batch_footprint.restype = ctypes.c_ulonglong
    L.hgks_batch_add.argtypes = [vp, P(hgks_grid_t), ctypes.c_double, ctypes.c_double, ctypes.c_double, ip, vp,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_double, ip]
    L.hgks_batch_remove.argtypes = [vp, ctypes.c_int]
    L.hgks_batch_step.argtypes = [vp, ctypes.c_int]
    L.hgks_batch_poll.argtypes = [vp, vp, vp, vp]
    L.hgks_batch_get_state.argtypes = [vp, ctypes.c_int, vp]
    L.hgks_batch_tune.argtypes = [vp, ctypes.c_int, ip]
    L.hgks_batch_set_tuning.argtypes = [vp, ip]
    L.hgks_batch_get_tuning.argtypes = [vp, ip]
    for name in ("hgks_batch_create", "hgks_batch_add", "hgks_batch_remove", "hgks_batch_step", "hgks_batch_poll",
                 "hgks_batch_get_state", "hgks_batch_tune", "hgks_batch_set_tuning", "hgks_batch_get_tuning"):
        getattr(L, name).restype = ctypes.c_int
    L.hgks_batch_launch_count.argtypes = [vp]
    L.hgks_batch_launch_count.restype = ctypes.c_ulonglong
    L.hgks_batch_last_error.argtypes = [vp]
    L.hgks_batch_last_error.restype = ctypes.c_char_p
    L.hgks_batch_destroy.argtypes = [vp]
    L.hgks_batch_destroy.restype = None
    L.hgks_set_timing.argtypes = [vp, ctypes.c_int]
    L.hgks_set_timing.restype = ctypes.c_int
    L.hgks_get_timing.argtypes = [vp, dp, P(ctypes.c_ulonglong)]
    L.hgks_get_timing.restype = ctypes.c_int
    L.hgks_launch_count.argtypes = [vp]
    L.hgks_launch_count.restype = ctypes.c_ulonglong
    L.hgks_device_bytes.argtypes = [vp]
    L.hgks_device_bytes.restype = ctypes.c_ulonglong
    L.hgks_alu_peak.argtypes = [ctypes.c_int, vp, dp]
    L.hgks_alu_peak.restype = ctypes.c_int
    L.hgks_last_error.argtypes = [vp]
    L.hgks_last_error.restype = ctypes.c_char_p
    L.hgks_destroy.argtypes = [vp]
    L.hgks_destroy.restype = None
    for name in ("hgks_create", "hgks_set_option", "hgks_set_state", "hgks_get_state", "hgks_step", "hgks_flux",
                 "hgks_reconstruct", "hgks_point_flux"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc, handle=None):
    if rc != HGKS_OK:
        msg = load().hgks_last_error(handle)
        raise HgksError(rc, msg.decode() if msg else "")


def _ptr(a):
    """(pointer, on_device) of a NumPy array or a CUDA torch tensor (FP64, contiguous)."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host buffers must be C-contiguous float64")
        return a.ctypes.data, 0
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("device buffers must be contiguous float64")
        return a.data_ptr(), int(a.is_cuda)
    raise TypeError("expected a numpy array or a torch tensor")


# ---- functions with the C names -------------------------------------------------------------

def hgks_create(n, lo, hi, gamma=1.4, mu=0.0, Pr=1.0, bc=(0, 0, 0, 0, 0, 0), precision=HGKS_FP64, stream=None,
                mesh=0, mesh_amp=0.0, mesh_omega=0.0):
    g = hgks_grid_t()
    for d in range(3):
        g.n[d], g.lo[d], g.hi[d] = int(n[d]), float(lo[d]), float(hi[d])
    g.mesh, g.mesh_amp, g.mesh_omega, g.precision = int(mesh), float(mesh_amp), float(mesh_omega), int(precision)
    bcs = (ctypes.c_int * 6)(*[int(b) for b in bc])
    out = ctypes.c_void_p()
    st = None if stream is None else ctypes.c_void_p(int(stream))
    _check(load().hgks_create(ctypes.byref(g), float(gamma), float(mu), float(Pr), bcs, st, ctypes.byref(out)))
    return out.value


def hgks_set_option(h, key, value):
    _check(load().hgks_set_option(h, key.encode(), float(value)), h)


def hgks_set_state(h, q, t=0.0):
    p, dev = _ptr(q)
    _check(load().hgks_set_state(h, p, dev, float(t)), h)


def hgks_get_state(h, q):
    p, dev = _ptr(q)
    t = ctypes.c_double()
    _check(load().hgks_get_state(h, p, dev, ctypes.byref(t)), h)
    return t.value


def hgks_step(h, nsteps, cfl=0.35, dt_fixed=0.0, t_end=float("inf"), sync=True):
    t = ctypes.c_double()
    done = ctypes.c_int()
    if sync:
        _check(load().hgks_step(h, int(nsteps), float(cfl), float(dt_fixed), float(t_end), ctypes.byref(t),
                                ctypes.byref(done)), h)
        return t.value, done.value
    _check(load().hgks_step(h, int(nsteps), float(cfl), float(dt_fixed), float(t_end), None, None), h)
    return None


def hgks_flux(h, dt, L, dL):
    pl, dev = _ptr(L)
    pd, dev2 = _ptr(dL)
    if dev != dev2:
        raise ValueError("L and dL must both be host or both be device buffers")
    _check(load().hgks_flux(h, float(dt), pl, pd, dev), h)


def hgks_reconstruct(h, ncell):
    coef = np.zeros((ncell, 5, 9))
    flag = np.zeros(ncell, dtype=np.int32)
    _check(load().hgks_reconstruct(h, coef.ctypes.data, flag.ctypes.data), h)
    return coef, flag


def hgks_point_flux(inp, dt, params, precision=HGKS_FP64, ug=None):
    inp = np.ascontiguousarray(inp, dtype=np.float64).reshape(-1, 40)
    n = inp.shape[0]
    F = np.zeros((n, 5))
    dF = np.zeros((n, 5))
    ugp = None
    if ug is not None:
        ug = np.ascontiguousarray(np.broadcast_to(ug, (n, 3)), dtype=np.float64)
        ugp = ug.ctypes.data
    par = (ctypes.c_double * 5)(*[float(x) for x in params])
    _check(load().hgks_point_flux(n, inp.ctypes.data, ugp, float(dt), par, int(precision), F.ctypes.data,
                                  dF.ctypes.data))
    return F, dF


PHASES = ("halo", "recon", "flux", "update", "cfl")


def hgks_set_timing(h, enable):
    _check(load().hgks_set_timing(h, int(bool(enable))), h)


def hgks_get_timing(h):
    """{phase: (ms, launches)} accumulated since hgks_set_timing."""
    ms = (ctypes.c_double * 5)()
    nl = (ctypes.c_ulonglong * 5)()
    _check(load().hgks_get_timing(h, ms, nl), h)
    return {name: (ms[i], int(nl[i])) for i, name in enumerate(PHASES)}


def hgks_flux_noalloc(n, lo, hi, q, dt, L, dL, gamma=1.4, mu=0.0, Pr=1.0, bc=(0, 0, 0, 0, 0, 0),
                      precision=HGKS_FP64, stream=None):
    """L(Q), dL/dt(Q) without a handle and without allocating (device tensors
    only; ordered on ``stream``, not synchronised)."""
    g = hgks_grid_t()
    for d in range(3):
        g.n[d], g.lo[d], g.hi[d] = int(n[d]), float(lo[d]), float(hi[d])
    g.mesh, g.mesh_amp, g.mesh_omega, g.precision = 0, 0.0, 0.0, int(precision)
    bcs = (ctypes.c_int * 6)(*[int(b) for b in bc])
    pq, dq = _ptr(q)
    pl, dl = _ptr(L)
    pd, dd = _ptr(dL)
    if not (dq and dl and dd):
        raise ValueError("hgks_flux_noalloc takes device buffers only")
    st = None if stream is None else ctypes.c_void_p(int(stream))
    _check(load().hgks_flux_noalloc(ctypes.byref(g), float(gamma), float(mu), float(Pr), bcs, pq, float(dt), pl, pd,
                                    st))


def hgks_alu_peak(precision, stream=None) -> float:
    """Measured FMA rate (TFLOP/s) of the FP64 (HGKS_FP64) or FP32
    (HGKS_MIXED) pipe of the current device."""
    out = ctypes.c_double(0.0)
    _check(load().hgks_alu_peak(int(precision), ctypes.c_void_p(stream), ctypes.byref(out)))
    return out.value


def hgks_launch_count(h) -> int:
    return int(load().hgks_launch_count(h))


def hgks_device_bytes(h) -> int:
    return int(load().hgks_device_bytes(h))


def hgks_last_error(h=None) -> str:
    m = load().hgks_last_error(h)
    return m.decode() if m else ""


def hgks_destroy(h):
    if h:
        load().hgks_destroy(h)


class Solver:
    """Convenience owner of one handle (still only marshalling)."""

    def __init__(self, n, lo, hi, gamma=1.4, mu=0.0, Pr=1.0, bc=(0,) * 6, precision=HGKS_FP64, stream=None,
                 mesh=0, mesh_amp=0.0, mesh_omega=0.0,
                 **options):
        self.n = tuple(int(x) for x in n)
        self.h = hgks_create(self.n, lo, hi, gamma, mu, Pr, bc, precision, stream, mesh, mesh_amp, mesh_omega)
        for k, v in options.items():
            hgks_set_option(self.h, k, v)

    @property
    def ncell(self):
        return self.n[0] * self.n[1] * self.n[2]

    def set_state(self, q, t=0.0):
        if isinstance(q, np.ndarray):
            q = np.ascontiguousarray(q, dtype=np.float64)
        hgks_set_state(self.h, q, t)

    def get_state(self):
        q = np.zeros((5, self.n[2], self.n[1], self.n[0]))
        t = hgks_get_state(self.h, q)
        return q, t

    def step(self, nsteps, cfl=0.35, dt_fixed=0.0, t_end=float("inf"), sync=True):
        return hgks_step(self.h, nsteps, cfl, dt_fixed, t_end, sync)

    def flux(self, dt):
        L = np.zeros((5, self.n[2], self.n[1], self.n[0]))
        dL = np.zeros_like(L)
        hgks_flux(self.h, dt, L, dL)
        return L, dL

    def reconstruct(self):
        return hgks_reconstruct(self.h, self.ncell)

    @property
    def launches(self):
        return hgks_launch_count(self.h)

    def close(self):
        if self.h:
            hgks_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- batched execution ----------------------------------------------------------------------

def _grid(n, lo, hi, precision):
    g = hgks_grid_t()
    for d in range(3):
        g.n[d], g.lo[d], g.hi[d] = int(n[d]), float(lo[d]), float(hi[d])
    g.mesh, g.mesh_amp, g.mesh_omega, g.precision = 0, 0.0, 0.0, int(precision)
    return g


def _bcheck(rc, b=None):
    if rc != HGKS_OK:
        msg = load().hgks_batch_last_error(b)
        raise HgksError(rc, msg.decode() if msg else "")


def hgks_batch_footprint(n, lo, hi, precision=HGKS_FP64) -> int:
    return int(load().hgks_batch_footprint(ctypes.byref(_grid(n, lo, hi, precision))))


class Batch:
    """Owner of one hgks_batch_t (marshalling only)."""

    def __init__(self, precision=HGKS_FP64, arena_bytes=4 << 30, max_instances=64, stream=None):
        self.precision = int(precision)
        self.max_instances = int(max_instances)
        out = ctypes.c_void_p()
        st = None if stream is None else ctypes.c_void_p(int(stream))
        _bcheck(load().hgks_batch_create(self.precision, int(arena_bytes), self.max_instances, st, ctypes.byref(out)))
        self.b = out.value
        self.n = {}

    def add(self, n, lo, hi, q, t0=0.0, t_end=1.0, cfl=0.35, gamma=1.4, mu=0.0, Pr=1.0, bc=(0,) * 6):
        q = np.ascontiguousarray(q, dtype=np.float64)
        g = _grid(n, lo, hi, self.precision)
        bcs = (ctypes.c_int * 6)(*[int(x) for x in bc])
        slot = ctypes.c_int(-1)
        _bcheck(load().hgks_batch_add(self.b, ctypes.byref(g), float(gamma), float(mu), float(Pr), bcs, q.ctypes.data,
                                      float(t0), float(t_end), float(cfl), ctypes.byref(slot)), self.b)
        self.n[slot.value] = tuple(int(x) for x in n)
        return slot.value

    def remove(self, slot):
        _bcheck(load().hgks_batch_remove(self.b, int(slot)), self.b)
        self.n.pop(slot, None)

    def step(self, nsteps=1):
        _bcheck(load().hgks_batch_step(self.b, int(nsteps)), self.b)

    def poll(self):
        """(t, steps, state) arrays over all slots; state 0 free, 1 running,
        2 at its end time, 3 nonphysical."""
        t = np.zeros(self.max_instances)
        steps = np.zeros(self.max_instances, dtype=np.int32)
        state = np.zeros(self.max_instances, dtype=np.int32)
        _bcheck(load().hgks_batch_poll(self.b, t.ctypes.data, steps.ctypes.data, state.ctypes.data), self.b)
        return t, steps, state

    def get_state(self, slot):
        n = self.n[slot]
        q = np.zeros((5, n[2], n[1], n[0]))
        _bcheck(load().hgks_batch_get_state(self.b, int(slot), q.ctypes.data), self.b)
        return q

    def tune(self, steps_per_trial=2):
        p = (ctypes.c_int * HGKS_TUNE_NPARAM)()
        _bcheck(load().hgks_batch_tune(self.b, int(steps_per_trial), p), self.b)
        return list(p)

    def set_tuning(self, params):
        p = (ctypes.c_int * HGKS_TUNE_NPARAM)(*[int(x) for x in params])
        _bcheck(load().hgks_batch_set_tuning(self.b, p), self.b)

    def get_tuning(self):
        p = (ctypes.c_int * HGKS_TUNE_NPARAM)()
        _bcheck(load().hgks_batch_get_tuning(self.b, p), self.b)
        return list(p)

    @property
    def launches(self):
        return int(load().hgks_batch_launch_count(self.b))

    def close(self):
        if getattr(self, "b", None):
            load().hgks_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
