"""Thin ctypes binding of the C ABI in include/dpde.h (libdpde.so).

Argument marshalling only: every step of the method runs in the CUDA kernels
of the library. Functions keep the C names (dpde_create, dpde_set_state,
dpde_get_state, dpde_step, dpde_sync, dpde_observables, dpde_destroy, ...);
:class:`System` wraps a handle for convenience. Host arrays are numpy float64
arrays; device arrays may be passed as torch CUDA tensors (their data_ptr()
is handed to the library) with ``on_device=True``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

DPDE_OK = 0
DPDE_ERR_ARG = -1
DPDE_ERR_CUDA = -2
DPDE_ERR_OOM = -3
DPDE_ERR_NEG_EPS = -4
DPDE_ERR_NONFINITE = -5
DPDE_ERR_TIMEOUT = -6
DPDE_ERR_CAPACITY = -7

FP64, MIXED = 0, 1
DPDE_NOALLOC_MAX_N = 262144   # particle limit of dpde_observables_noalloc (dpde.h)
SER, HYBRID, SEM, SSA = 0, 1, 2, 3
SCHEMES = {"SER": SER, "HYBRID": HYBRID, "SEM": SEM, "SSA": SSA}
PRECISIONS = {"fp64": FP64, "mixed": MIXED}


class DPDEError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"dpde error {code}: {msg}")
        self.code = code


class dpde_params(C.Structure):
    _fields_ = [("mass", C.c_double), ("r_cut", C.c_double), ("a", C.c_double),
                ("sigma", C.c_double), ("seed", C.c_uint64), ("precision", C.c_int32),
                ("potential", C.c_int32), ("lj_eps", C.c_double), ("lj_r", C.c_double)]


class dpde_replica(C.Structure):
    _fields_ = [("n", C.c_int64), ("box", C.c_double * 3), ("cv", C.c_double),
                ("bricks", C.c_int32 * 3), ("walls", C.c_int32), ("wall_u", C.c_double)]


class dpde_obs(C.Structure):
    _fields_ = [("E", C.c_double), ("K", C.c_double), ("U", C.c_double), ("Eint", C.c_double),
                ("P", C.c_double * 3), ("Tkin", C.c_double), ("Tint", C.c_double),
                ("Tpot_num", C.c_double), ("Tpot_den", C.c_double), ("step", C.c_int64),
                ("n", C.c_int64), ("neg_eps", C.c_int64), ("nonfinite", C.c_int64)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "P"}
        d["Px"], d["Py"], d["Pz"] = self.P[0], self.P[1], self.P[2]
        return d


class dpde_tuning(C.Structure):
    _fields_ = [("tile_edge", C.c_int32), ("block", C.c_int32), ("ssa_block", C.c_int32),
                ("ssa_mode", C.c_int32), ("ssa_group", C.c_int32), ("reserved", C.c_int32),
                ("ms_per_step", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


_lib = None
EXPORTS = ["dpde_create", "dpde_set_state", "dpde_get_state", "dpde_step", "dpde_sync",
           "dpde_observables", "dpde_get_step", "dpde_destroy", "dpde_last_error",
           "dpde_debug_philox", "dpde_debug_gaussian", "dpde_step_profiled", "dpde_get_cells",
           "dpde_checkpoint", "dpde_restore", "dpde_observables_noalloc", "dpde_noalloc_last_error",
           "dpde_step_launches", "dpde_get_tuning", "dpde_set_tuning", "dpde_autotune",
           "dpde_set_projection", "dpde_set_wait_budget"]
PHASES = ["kick_drift", "scan", "gather", "force", "ssa", "sweep1", "sweep2", "other", "ssa_gauss"]


def lib():
    """Loads the in-tree libdpde.so (building it when it is missing or stale).
    Raises when the library cannot be built or loaded: there is no fallback."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp = C.c_void_p
        dp = C.POINTER(C.c_double)
        u32p = C.POINTER(C.c_uint32)
        L.dpde_create.argtypes = [C.POINTER(dpde_params), C.c_int32, C.POINTER(dpde_replica), vp,
                                  C.POINTER(vp)]
        L.dpde_set_state.argtypes = [vp, vp, vp, vp, C.c_int64, C.c_int32]
        L.dpde_get_state.argtypes = [vp, vp, vp, vp, C.c_int32]
        L.dpde_step.argtypes = [vp, C.c_int64, C.c_double, C.c_int32, C.c_int32]
        L.dpde_sync.argtypes = [vp]
        L.dpde_observables.argtypes = [vp, C.POINTER(dpde_obs)]
        L.dpde_get_step.argtypes = [vp, C.POINTER(C.c_int64)]
        L.dpde_destroy.argtypes = [vp]
        L.dpde_last_error.argtypes = [vp]
        L.dpde_last_error.restype = C.c_char_p
        L.dpde_observables_noalloc.argtypes = [C.POINTER(dpde_params), C.POINTER(dpde_replica), vp, vp, vp,
                                               vp, C.POINTER(dpde_obs)]
        L.dpde_noalloc_last_error.argtypes = []
        L.dpde_noalloc_last_error.restype = C.c_char_p
        L.dpde_checkpoint.argtypes = [vp, vp, C.POINTER(C.c_uint64)]
        L.dpde_restore.argtypes = [vp, vp, C.c_uint64]
        L.dpde_get_cells.argtypes = [vp, C.POINTER(C.c_int32)]
        L.dpde_step_launches.argtypes = [vp, C.c_int32, C.POINTER(C.c_int64)]
        L.dpde_get_tuning.argtypes = [vp, C.POINTER(dpde_tuning)]
        L.dpde_set_projection.argtypes = [vp, C.c_int32, C.POINTER(C.c_double)]
        L.dpde_set_wait_budget.argtypes = [vp, C.c_int64]
        L.dpde_set_tuning.argtypes = [vp, C.POINTER(dpde_tuning)]
        L.dpde_autotune.argtypes = [vp, C.c_int32, C.c_double, C.c_int32, C.POINTER(dpde_tuning)]
        L.dpde_step_profiled.argtypes = [vp, C.c_int64, C.c_double, C.c_int32, dp]
        L.dpde_debug_philox.argtypes = [C.c_int64, u32p, u32p, u32p]
        L.dpde_debug_gaussian.argtypes = [C.c_int64, C.c_uint64, u32p, u32p, u32p, u32p,
                                          C.c_int32, dp]
        _lib = L
    return _lib


def _addr(x):
    """Pointer of a numpy array (host) or a torch tensor (device or host)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    return C.c_void_p(x.ctypes.data)


def _check(h, rc):
    if rc != DPDE_OK:
        raise DPDEError(rc, lib().dpde_last_error(h).decode())
    return rc


def dpde_create(params: dpde_params, replicas, stream=None):
    reps = (dpde_replica * len(replicas))(*replicas)
    h = C.c_void_p()
    rc = lib().dpde_create(C.byref(params), len(replicas), reps,
                           C.c_void_p(stream) if stream else None, C.byref(h))
    if rc != DPDE_OK:
        raise DPDEError(rc, lib().dpde_last_error(None).decode())
    return h


def dpde_set_state(h, q, p, eps, step=0, on_device=False):
    return _check(h, lib().dpde_set_state(h, _addr(q), _addr(p), _addr(eps), int(step),
                                          int(on_device)))


def dpde_get_state(h, q, p, eps, on_device=False):
    return lib().dpde_get_state(h, _addr(q), _addr(p), _addr(eps), int(on_device))


def dpde_step(h, n, dt, scheme, use_graph=True):
    return _check(h, lib().dpde_step(h, int(n), float(dt), SCHEMES.get(scheme, scheme),
                                     int(use_graph)))


def dpde_step_profiled(h, n, dt, scheme) -> dict:
    ms = np.zeros(len(PHASES))
    _check(h, lib().dpde_step_profiled(h, int(n), float(dt), SCHEMES.get(scheme, scheme),
                                       ms.ctypes.data_as(C.POINTER(C.c_double))))
    return dict(zip(PHASES, ms.tolist()))


def dpde_step_launches(h, scheme) -> int:
    """Kernel launches in one step of `scheme`."""
    out = C.c_int64(0)
    _check(h, lib().dpde_step_launches(h, SCHEMES.get(scheme, scheme), C.byref(out)))
    return int(out.value)


def dpde_get_step(h) -> int:
    out = C.c_int64(0)
    _check(h, lib().dpde_get_step(h, C.byref(out)))
    return int(out.value)


def dpde_set_projection(h, enable=True, E0=None):
    """Projection on the internal energies (Sec. IV.C); E0 per replica, or
    None for the current energies."""
    arr = None
    if E0 is not None:
        arr = np.ascontiguousarray(np.asarray(E0, dtype=np.float64).ravel())
    _check(h, lib().dpde_set_projection(h, 1 if enable else 0,
                                        arr.ctypes.data_as(C.POINTER(C.c_double)) if arr is not None else None))


def dpde_get_tuning(h) -> dict:
    t = dpde_tuning()
    _check(h, lib().dpde_get_tuning(h, C.byref(t)))
    return t.as_dict()


def dpde_set_tuning(h, tile_edge=None, block=None, ssa_block=None, ssa_mode=None, ssa_group=None):
    t = dpde_tuning()
    _check(h, lib().dpde_get_tuning(h, C.byref(t)))
    if tile_edge is not None:
        t.tile_edge = int(tile_edge)
    if block is not None:
        t.block = int(block)
    if ssa_block is not None:
        t.ssa_block = int(ssa_block)
    if ssa_mode is not None:
        t.ssa_mode = int(ssa_mode)
    if ssa_group is not None:
        t.ssa_group = int(ssa_group)
    _check(h, lib().dpde_set_tuning(h, C.byref(t)))


def dpde_autotune(h, scheme, dt, steps=3) -> dict:
    t = dpde_tuning()
    _check(h, lib().dpde_autotune(h, SCHEMES.get(scheme, scheme), float(dt), int(steps), C.byref(t)))
    return t.as_dict()


def dpde_sync(h):
    return lib().dpde_sync(h)


def dpde_observables(h, n_replicas):
    out = (dpde_obs * n_replicas)()
    rc = lib().dpde_observables(h, out)
    return rc, [o.as_dict() for o in out]


def _noalloc_arg(x, numel: int, name: str):
    """A state argument of dpde_observables_noalloc: a contiguous float64 CUDA
    tensor with at least `numel` elements (the C side also refuses host
    pointers)."""
    if x is None or not hasattr(x, "is_cuda"):
        raise DPDEError(DPDE_ERR_ARG, f"{name} must be a CUDA tensor (got {type(x).__name__})")
    import torch
    if not x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous() or x.numel() < numel:
        raise DPDEError(DPDE_ERR_ARG, f"{name} must be a contiguous float64 CUDA tensor of at least "
                                      f"{numel} elements (got {x.dtype}, {tuple(x.shape)}, device {x.device})")
    return x


def dpde_observables_noalloc(params: dpde_params, replica: dpde_replica, q, p, eps, stream=None):
    """Observables of one system from device arrays (contiguous float64 torch
    CUDA tensors: q and p of 3n elements, eps of n), computed without any
    device allocation."""
    n = int(replica.n)
    if 0 < n <= DPDE_NOALLOC_MAX_N:
        q = _noalloc_arg(q, 3 * n, "q")
        p = _noalloc_arg(p, 3 * n, "p")
        eps = _noalloc_arg(eps, n, "eps")
    out = dpde_obs()
    rc = lib().dpde_observables_noalloc(C.byref(params), C.byref(replica), _addr(q), _addr(p), _addr(eps),
                                        C.c_void_p(stream) if stream else None, C.byref(out))
    if rc not in (DPDE_OK, DPDE_ERR_NEG_EPS, DPDE_ERR_NONFINITE):
        raise DPDEError(rc, lib().dpde_noalloc_last_error().decode())
    return rc, out.as_dict()


def dpde_set_wait_budget(h, cycles: int):
    return _check(h, lib().dpde_set_wait_budget(h, int(cycles)))


def dpde_destroy(h):
    return lib().dpde_destroy(h)


def dpde_debug_philox(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, np.uint32).reshape(-1, 2)
    out = np.empty_like(ctr)
    u = C.POINTER(C.c_uint32)
    _check(None, lib().dpde_debug_philox(len(ctr), ctr.ctypes.data_as(u), key.ctypes.data_as(u),
                                         out.ctypes.data_as(u)))
    return out


def dpde_debug_gaussian(seed, step, replica, id_a, id_b, precision="fp64") -> np.ndarray:
    shape = np.broadcast(step, replica, id_a, id_b).shape
    arrs = [np.ascontiguousarray(np.broadcast_to(x, shape), np.uint32).ravel()
            for x in (step, replica, id_a, id_b)]
    out = np.empty((arrs[0].size, 3))
    u = C.POINTER(C.c_uint32)
    _check(None, lib().dpde_debug_gaussian(arrs[0].size, seed, *(a.ctypes.data_as(u) for a in arrs),
                                           PRECISIONS.get(precision, precision),
                                           out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


POT_SOFT, POT_LJ = 0, 1


def make_params(mass=1.0, r_cut=1.0, a=25.0, sigma=3.0, seed=0, precision="mixed", potential=POT_SOFT,
                lj_eps=1.0, lj_r=1.0) -> dpde_params:
    return dpde_params(mass, r_cut, a, sigma, seed, PRECISIONS.get(precision, precision), potential,
                       lj_eps, lj_r)


def make_replica(n, box, cv, bricks=(1, 1, 1), walls=0, wall_u=0.0) -> dpde_replica:
    """walls = 1: specular walls along z at 0 and L_z + wall_u n dt (dpde.h)."""
    if np.isscalar(box):
        box = (box, box, box)
    r = dpde_replica()
    r.n = int(n)
    r.box[:] = [float(x) for x in box]
    r.cv = float(cv)
    r.bricks[:] = [int(b) for b in bricks]
    r.walls = int(walls)
    r.wall_u = float(wall_u)
    return r


class System:
    """A handle over one or more replicas (arrays concatenated by replica;
    ids are indices within a replica)."""

    def __init__(self, params: dpde_params, replicas, stream=None):
        self.params = params
        self.replicas = list(replicas)
        self.R = len(self.replicas)
        self.N = int(sum(r.n for r in self.replicas))
        self.h = dpde_create(params, self.replicas, stream)

    def set_state(self, q, p, eps, step=0, on_device=False):
        if not on_device:
            q = np.ascontiguousarray(q, np.float64)
            p = np.ascontiguousarray(p, np.float64)
            eps = np.ascontiguousarray(eps, np.float64)
        dpde_set_state(self.h, q, p, eps, step, on_device)

    def get_state(self, check=True):
        q = np.empty((self.N, 3))
        p = np.empty((self.N, 3))
        e = np.empty(self.N)
        rc = dpde_get_state(self.h, q, p, e)
        if check:
            _check(self.h, rc)
        return q, p, e

    def checkpoint(self) -> bytes:
        """Raw internal state for a bit-exact restart."""
        size = C.c_uint64(0)
        _check(self.h, lib().dpde_checkpoint(self.h, None, C.byref(size)))
        buf = C.create_string_buffer(size.value)
        _check(self.h, lib().dpde_checkpoint(self.h, buf, C.byref(size)))
        return buf.raw[:size.value]

    def restore(self, blob: bytes):
        _check(self.h, lib().dpde_restore(self.h, blob, len(blob)))

    def get_cells(self):
        """Cell coordinates (N, 3) of every particle, id order."""
        out = np.empty((self.N, 3), np.int32)
        _check(self.h, lib().dpde_get_cells(self.h, out.ctypes.data_as(C.POINTER(C.c_int32))))
        return out

    def step_launches(self, scheme) -> int:
        return dpde_step_launches(self.h, scheme)

    def set_projection(self, enable=True, E0=None):
        dpde_set_projection(self.h, enable, E0)

    def tuning(self) -> dict:
        return dpde_get_tuning(self.h)

    def set_tuning(self, **kw):
        dpde_set_tuning(self.h, **kw)

    def autotune(self, scheme, dt, steps=3) -> dict:
        return dpde_autotune(self.h, scheme, dt, steps)

    def step(self, n, dt, scheme, use_graph=True):
        dpde_step(self.h, n, dt, scheme, use_graph)

    def step_profiled(self, n, dt, scheme) -> dict:
        return dpde_step_profiled(self.h, n, dt, scheme)

    def sync(self):
        return dpde_sync(self.h)

    def observables(self, check=False):
        rc, obs = dpde_observables(self.h, self.R)
        if check:
            _check(self.h, rc)
        return obs

    def close(self):
        if self.h:
            dpde_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
