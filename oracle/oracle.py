"""ctypes wrapper of the FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. The product library
never imports this module. The oracle follows the paper (Homman, Maillet,
Roussel, Stoltz, arXiv:1507.06643) step by step; see ``oracle.h`` for the
equations each function implements.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")

SER, HYBRID, SEM, SSA = 0, 1, 2, 3
SCHEMES = {"SER": SER, "HYBRID": HYBRID, "SEM": SEM, "SSA": SSA}


def build(force: bool = False) -> str:
    """Compiles ``oracle.c`` with gcc (plain C11, no fast-math, no FMA
    contraction so that x86 and Arm give identical bits)."""
    src = os.path.join(HERE, "oracle.c")
    hdr = os.path.join(HERE, "oracle.h")
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wextra", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class Params(C.Structure):
    _fields_ = [("mass", C.c_double), ("r_cut", C.c_double), ("a", C.c_double),
                ("sigma", C.c_double), ("seed", C.c_uint64), ("noise", C.c_int32),
                ("potential", C.c_int32), ("lj_eps", C.c_double), ("lj_r", C.c_double)]


POT_SOFT, POT_LJ = 0, 1


class Replica(C.Structure):
    _fields_ = [("n", C.c_int64), ("box", C.c_double * 3), ("cv", C.c_double),
                ("bricks", C.c_int32 * 3), ("walls", C.c_int32), ("wall_u", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB_PATH)
        dp = C.POINTER(C.c_double)
        u32p = C.POINTER(C.c_uint32)
        i64p = C.POINTER(C.c_int64)
        i32p = C.POINTER(C.c_int32)
        L.ora_philox_batch.argtypes = [C.c_int64, u32p, u32p, u32p]
        L.ora_gaussian_batch.argtypes = [C.c_int64, C.c_uint64, u32p, u32p, u32p, u32p, dp]
        L.ora_pairs_brute.argtypes = [C.POINTER(Replica), C.c_double, dp, C.c_int64, i64p, i64p]
        L.ora_pairs_brute.restype = C.c_int64
        L.ora_pairs_cells.argtypes = [C.POINTER(Replica), C.c_double, dp, C.c_int64, i64p, i64p]
        L.ora_pairs_cells.restype = C.c_int64
        L.ora_forces.argtypes = [C.POINTER(Replica), C.POINTER(Params), dp, dp]
        L.ora_fd.argtypes = [C.POINTER(Replica), C.c_int32, C.POINTER(Params), dp, dp, dp,
                             C.c_uint32, C.c_double, C.c_int32]
        L.ora_run.argtypes = [C.c_int32, C.POINTER(Replica), C.POINTER(Params), dp, dp, dp, dp,
                              C.c_int64, C.c_int64, C.c_double, C.c_int32]
        L.ora_observables.argtypes = [C.POINTER(Replica), C.POINTER(Params), dp, dp, dp, dp]
        L.ora_cell_grid.argtypes = [C.POINTER(Replica), C.c_double, i32p, i32p]
        L.ora_project.argtypes = [C.POINTER(Replica), C.POINTER(Params), dp, dp, dp, C.c_double]
        L.ora_pair_potential.argtypes = [C.POINTER(Params), C.c_double, dp, dp, dp]
        L.ora_ssa_order.argtypes = [C.POINTER(Replica), C.c_double, dp, C.c_int32, C.c_int64,
                                    i64p, i64p]
        L.ora_ssa_order.restype = C.c_int64
        _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_params(mass=1.0, r_cut=1.0, a=25.0, sigma=3.0, seed=0, noise=True, potential=POT_SOFT,
                lj_eps=1.0, lj_r=1.0) -> Params:
    return Params(mass, r_cut, a, sigma, seed, 1 if noise else 0, potential, lj_eps, lj_r)


def pair_potential(prm: Params, r: float):
    """(v, v', v'') of the pair potential at r."""
    v, dv, d2v = C.c_double(), C.c_double(), C.c_double()
    lib().ora_pair_potential(C.byref(prm), float(r), C.byref(v), C.byref(dv), C.byref(d2v))
    return v.value, dv.value, d2v.value


def make_replica(n, box, cv, bricks=(1, 1, 1), walls=0, wall_u=0.0) -> Replica:
    """walls = 1: specular walls at z = 0 and z = L_z + wall_u n dt (oracle.h)."""
    if np.isscalar(box):
        box = (box, box, box)
    r = Replica()
    r.n = int(n)
    r.box[:] = [float(x) for x in box]
    r.cv = float(cv)
    r.bricks[:] = [int(b) for b in bricks]
    r.walls = int(walls)
    r.wall_u = float(wall_u)
    return r


def philox(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    out = np.empty_like(ctr)
    lib().ora_philox_batch(len(ctr), _ptr(ctr, C.c_uint32), _ptr(key, C.c_uint32),
                           _ptr(out, C.c_uint32))
    return out


def gaussian(seed, step, replica, id_a, id_b) -> np.ndarray:
    step, replica, id_a, id_b = (np.ascontiguousarray(np.broadcast_to(x, np.broadcast(
        step, replica, id_a, id_b).shape), dtype=np.uint32).ravel()
        for x in (step, replica, id_a, id_b))
    out = np.empty((len(id_a), 3))
    lib().ora_gaussian_batch(len(id_a), seed, _ptr(step, C.c_uint32), _ptr(replica, C.c_uint32),
                             _ptr(id_a, C.c_uint32), _ptr(id_b, C.c_uint32), _ptr(out, C.c_double))
    return out


def pairs(rep: Replica, r_cut: float, q, method="cells") -> np.ndarray:
    """Interacting pairs (i<j) as an (np, 2) array sorted lexicographically."""
    q = _f64(q)
    fn = lib().ora_pairs_cells if method == "cells" else lib().ora_pairs_brute
    npairs = fn(C.byref(rep), r_cut, _ptr(q, C.c_double), 0, None, None)
    if npairs < 0:
        raise ValueError("invalid cell grid")
    pi = np.empty(max(npairs, 1), np.int64)
    pj = np.empty(max(npairs, 1), np.int64)
    fn(C.byref(rep), r_cut, _ptr(q, C.c_double), npairs, _ptr(pi, C.c_int64), _ptr(pj, C.c_int64))
    P = np.stack([pi[:npairs], pj[:npairs]], axis=1)
    order = np.lexsort((P[:, 1], P[:, 0]))
    return P[order]


def ssa_order(rep: Replica, r_cut: float, q, whole_box=False) -> np.ndarray:
    q = _f64(q)
    n = lib().ora_ssa_order(C.byref(rep), r_cut, _ptr(q, C.c_double), int(whole_box), 0, None, None)
    if n < 0:
        raise ValueError("invalid cell grid")
    pi = np.empty(max(n, 1), np.int64)
    pj = np.empty(max(n, 1), np.int64)
    lib().ora_ssa_order(C.byref(rep), r_cut, _ptr(q, C.c_double), int(whole_box), n,
                        _ptr(pi, C.c_int64), _ptr(pj, C.c_int64))
    return np.stack([pi[:n], pj[:n]], axis=1)


def cell_grid(rep: Replica, r_cut: float):
    nc = (C.c_int32 * 3)()
    k = (C.c_int32 * 3)()
    if lib().ora_cell_grid(C.byref(rep), r_cut, nc, k) != 0:
        raise ValueError("invalid cell grid")
    return tuple(nc), tuple(k)


def forces(rep: Replica, prm: Params, q) -> np.ndarray:
    q = _f64(q)
    F = np.empty_like(q)
    if lib().ora_forces(C.byref(rep), C.byref(prm), _ptr(q, C.c_double), _ptr(F, C.c_double)):
        raise ValueError("invalid cell grid")
    return F


def fd(rep: Replica, ridx: int, prm: Params, q, p, eps, step: int, dt: float, scheme) -> tuple:
    """One fluctuation/dissipation sub-step (no Verlet), returns new (p, eps)."""
    scheme = SCHEMES.get(scheme, scheme)
    q = _f64(q)
    p = _f64(p).copy()
    eps = _f64(eps).copy()
    rc = lib().ora_fd(C.byref(rep), ridx, C.byref(prm), _ptr(q, C.c_double), _ptr(p, C.c_double),
                      _ptr(eps, C.c_double), step, dt, scheme)
    if rc:
        raise ValueError("ora_fd failed")
    return p, eps


class System:
    """A batch of replicas advanced by the oracle (arrays concatenated by
    replica, ids = index within the replica)."""

    def __init__(self, reps, prm: Params, q, p, eps, step: int = 0):
        self.reps = list(reps)
        self.R = len(self.reps)
        self.rep_arr = (Replica * self.R)(*self.reps)
        self.prm = prm
        self.q = _f64(q).reshape(-1, 3).copy()
        self.p = _f64(p).reshape(-1, 3).copy()
        self.eps = _f64(eps).ravel().copy()
        self.step = int(step)
        self.offsets = np.concatenate([[0], np.cumsum([r.n for r in self.reps])]).astype(np.int64)
        for r in range(self.R):
            self._wrap(r)
        self.F = np.zeros_like(self.q)
        for r in range(self.R):
            s = slice(self.offsets[r], self.offsets[r + 1])
            self.F[s] = forces(self.reps[r], prm, self.q[s])

    def _wrap(self, r):
        """Periodic axes into [0, L); the z axis of a replica closed by walls
        (Sec. V: no periodicity along the shock axis) is left as given, so a
        particle on the upper wall face z = L_z stays there."""
        s = slice(self.offsets[r], self.offsets[r + 1])
        box = np.array(self.reps[r].box[:])
        axes = [0, 1] if self.reps[r].walls else [0, 1, 2]
        q = self.q[s]
        q[:, axes] = np.mod(q[:, axes], box[axes])
        q[:, axes] = np.where(q[:, axes] >= box[axes], q[:, axes] - box[axes], q[:, axes])
        self.q[s] = q

    projection = None   # per-replica E0 when the projection of Sec. IV.C is on

    def set_projection(self, E0=None, on=True):
        """Turns the projection on (E0 per replica; default: the current
        energies) or off."""
        if not on:
            self.projection = None
        else:
            self.projection = [self.observables(r)["E"] for r in range(self.R)] if E0 is None else list(E0)

    def run(self, nsteps: int, dt: float, scheme) -> None:
        scheme = SCHEMES.get(scheme, scheme)
        per_call = 1 if self.projection is not None else nsteps
        done = 0
        while done < nsteps:
            k = min(per_call, nsteps - done)
            rc = lib().ora_run(self.R, self.rep_arr, C.byref(self.prm), _ptr(self.q, C.c_double),
                               _ptr(self.p, C.c_double), _ptr(self.eps, C.c_double),
                               _ptr(self.F, C.c_double), self.step, k, dt, scheme)
            if rc:
                raise ValueError("ora_run failed")
            self.step += k
            done += k
            if self.projection is not None:
                for r in range(self.R):
                    s = slice(self.offsets[r], self.offsets[r + 1])
                    q, p = np.ascontiguousarray(self.q[s]), np.ascontiguousarray(self.p[s])
                    e = np.ascontiguousarray(self.eps[s])
                    if lib().ora_project(C.byref(self.reps[r]), C.byref(self.prm), _ptr(q, C.c_double),
                                         _ptr(p, C.c_double), _ptr(e, C.c_double), self.projection[r]):
                        raise ValueError("ora_project failed")
                    self.eps[s] = e

    def observables(self, r: int = 0) -> dict:
        s = slice(self.offsets[r], self.offsets[r + 1])
        out = np.empty(13)
        q, p, e = (np.ascontiguousarray(x[s]) for x in (self.q, self.p, self.eps))
        lib().ora_observables(C.byref(self.reps[r]), C.byref(self.prm), _ptr(q, C.c_double),
                              _ptr(p, C.c_double), _ptr(e, C.c_double), _ptr(out, C.c_double))
        keys = ["E", "K", "U", "Eint", "Px", "Py", "Pz", "Tkin", "Tint", "Tpot_num", "Tpot_den",
                "neg_eps", "nonfinite"]
        return dict(zip(keys, out.tolist()))
