"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method: it only draws initial states
(positions, momenta, internal energies) and names the workloads. Both the GPU
library and the CPU oracle are fed from here.

Recipe (per replica): positions uniform in the periodic box; momenta
Maxwellian at temperature kT (each component ~ N(0, m kT)) with the mean
removed so that the total momentum is zero (the setting of Eq. Tkin, P_0 = 0);
internal energies eps_i = C_v kT (1 + 0.05 u_i), u_i ~ U(-1, 1), i.e. the
equation of state eps = C_v T of Sec. IV.A with 5% spread. The paper's own
initial states come from melted crystals that are not available; these stand
in for them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class ReplicaSpec:
    n: int
    box: tuple
    cv: float
    kT: float = 1.0
    bricks: tuple = (1, 1, 1)
    vz_split: float = 0.0     # +v for z < Lz/2, -v above (shock set-up)
    vz_shift: float = 0.0     # v added to every particle along z (piston set-up)
    walls: int = 0            # 1: specular walls along z (see the library header)
    wall_u: float = 0.0       # velocity of the upper wall (walls = 1)


@dataclasses.dataclass
class Workload:
    name: str
    replicas: list
    mass: float = 1.0
    r_cut: float = 1.0
    a: float = 25.0
    sigma: float = 3.0
    dt: float = 0.01
    steps: int = 100
    seed: int = 1000
    precision: str = "mixed"

    @property
    def n_total(self) -> int:
        return int(sum(r.n for r in self.replicas))


def cubic_box(n: int, density: float = 3.0) -> tuple:
    L = (n / density) ** (1.0 / 3.0)
    return (L, L, L)


def replica_state(spec: ReplicaSpec, mass: float, rng: np.random.Generator,
                  eps_spread: float = 0.05, float32: bool = False):
    """Returns q (n,3), p (n,3), eps (n,) as float64 arrays. With float32=True
    q and p are rounded to float (so a mixed-precision run and the oracle start
    from the same values)."""
    n = spec.n
    box = np.asarray(spec.box, dtype=np.float64)
    q = rng.random((n, 3)) * box
    p = rng.standard_normal((n, 3)) * math.sqrt(mass * spec.kT)
    if n > 0:
        p -= p.mean(axis=0, keepdims=True)
    if spec.vz_split and n > 0:
        p[:, 2] += np.where(q[:, 2] < 0.5 * box[2], spec.vz_split, -spec.vz_split) * mass
    if spec.vz_shift and n > 0:
        p[:, 2] += spec.vz_shift * mass
    eps = spec.cv * spec.kT * (1.0 + eps_spread * rng.uniform(-1.0, 1.0, n))
    if float32:
        q = q.astype(np.float32).astype(np.float64)
        q = np.where(q >= box, 0.0, q)
        p = p.astype(np.float32).astype(np.float64)
    return q, p, eps


def workload_state(w: Workload, seed: int | None = None, float32: bool | None = None):
    """Concatenated (q, p, eps) of every replica of a workload."""
    rng = np.random.default_rng(w.seed if seed is None else seed)
    f32 = (w.precision == "mixed") if float32 is None else float32
    qs, ps, es = [], [], []
    for spec in w.replicas:
        q, p, e = replica_state(spec, w.mass, rng, float32=f32)
        qs.append(q)
        ps.append(p)
        es.append(e)
    return np.concatenate(qs), np.concatenate(ps), np.concatenate(es)


def plain_n1000(precision: str = "fp64") -> Workload:
    """N=1000 at density 3 (L ~ 6.93), C_v=100, kT=1, a=25, sigma=3,
    dt=0.01, 100 steps; Hybrid domains 2x2x2."""
    return Workload("plain_n1000", [ReplicaSpec(1000, cubic_box(1000), 100.0, 1.0, (2, 2, 2))],
                    steps=100, seed=1001, precision=precision)


def equilibrium_n108000(precision: str = "mixed") -> Workload:
    """N=108,000 at density 3 (L ~ 33.0), C_v=100; Hybrid domains 5x5x5
    (864 particles each)."""
    return Workload("equilibrium_n108000",
                    [ReplicaSpec(108000, cubic_box(108000), 100.0, 1.0, (5, 5, 5))],
                    steps=100000, seed=1002, precision=precision)


def large_n4m(precision: str = "mixed") -> Workload:
    """N=4,000,000 at density 3 (L ~ 110.1), C_v=50, 1000 timed steps;
    Hybrid domains 18x18x18 (~686 particles each)."""
    return Workload("large_n4m", [ReplicaSpec(4_000_000, cubic_box(4_000_000), 50.0, 1.0,
                                              (18, 18, 18))],
                    steps=1000, seed=1003, precision=precision)


def medium_n1m(precision: str = "mixed") -> Workload:
    """The large fluid at a quarter of its size: N=1,000,000 at density 3
    (L ~ 69.3), C_v=50; Hybrid domains 11x11x11 (6^3 cells each). Small
    enough for detailed kernel captures, larger than L2."""
    return Workload("medium_n1m", [ReplicaSpec(1_000_000, cubic_box(1_000_000), 50.0, 1.0, (11, 11, 11))],
                    steps=1000, seed=1006, precision=precision)


def shock_40x40x800(precision: str = "mixed") -> Workload:
    """Box 40 x 40 x 800 at density 3 (3.84M particles), periodic in all
    directions, halves moving at +-2 along z on a kT=1 Maxwellian, C_v=100,
    dt=0.005; Hybrid domains 8x8x160."""
    n = 3 * 40 * 40 * 800
    return Workload("shock_40x40x800",
                    [ReplicaSpec(n, (40.0, 40.0, 800.0), 100.0, 1.0, (8, 8, 160), vz_split=2.0)],
                    dt=0.005, steps=20000, seed=1004, precision=precision)


def shock_walls_40x40x800(precision: str = "mixed") -> Workload:
    """The shock set-up of Sec. V in its hard-wall reading: box 40 x 40 x 800
    at density 3 (3.84M particles), periodic along x and y, walls along z --
    fixed at z = 0, the upper one moving at u_p = -2 -- and every particle
    given v_z = u_p on a kT=1 Maxwellian, so that a shock runs up from the
    fixed wall; C_v=100, dt=0.005; Hybrid domains 8x8x160."""
    n = 3 * 40 * 40 * 800
    return Workload("shock_walls_40x40x800",
                    [ReplicaSpec(n, (40.0, 40.0, 800.0), 100.0, 1.0, (8, 8, 160), vz_shift=-2.0, walls=1,
                                 wall_u=-2.0)],
                    dt=0.005, steps=20000, seed=1007, precision=precision)


def batched_256(precision: str = "mixed", n_replicas: int = 256, seed: int = 1005,
                n_min: int = 2000, n_max: int = 64000) -> Workload:
    """256 independent systems, n_r log-uniform in [2000, 64000] at density 3,
    kT_r ~ U[0.5, 2], C_v in {10, 50, 100}; one Hybrid domain per ~1000."""
    rng = np.random.default_rng(seed)
    reps = []
    for _ in range(n_replicas):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        box = cubic_box(n)
        b = max(1, int(round((n / 1000.0) ** (1.0 / 3.0))))
        while b > 1 and math.floor(box[0] / b) * b < 3:
            b -= 1
        reps.append(ReplicaSpec(n, box, float(rng.choice([10.0, 50.0, 100.0])),
                                float(rng.uniform(0.5, 2.0)), (b, b, b)))
    return Workload("batched_256", reps, steps=1000, seed=seed, precision=precision)


def fcc_state(cells: int, density: float, kT: float, cv: float, mass: float, seed: int,
              jitter: float = 0.02):
    """Face-centred cubic crystal of cells^3 unit cells (4 sites each) at the
    given number density, sites displaced by N(0, jitter^2) per component,
    Maxwellian momenta at kT with the mean removed, eps = cv kT (1 +- 5%).
    Returns (q, p, eps, L)."""
    rng = np.random.default_rng(seed)
    a = (4.0 / density) ** (1.0 / 3.0)
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    grid = np.stack(np.meshgrid(np.arange(cells), np.arange(cells), np.arange(cells), indexing="ij"), -1)
    q = ((grid.reshape(-1, 1, 3) + base.reshape(1, 4, 3)).reshape(-1, 3) + 0.25) * a
    L = cells * a
    q = np.mod(q + rng.normal(0.0, jitter, q.shape), L)
    n = len(q)
    p = rng.standard_normal((n, 3)) * math.sqrt(mass * kT)
    p -= p.mean(axis=0)
    e = cv * kT * (1 + 0.05 * rng.uniform(-1, 1, n))
    return q, p, e, L


WORKLOADS = {
    "plain_n1000": plain_n1000,
    "equilibrium_n108000": equilibrium_n108000,
    "large_n4m": large_n4m,
    "medium_n1m": medium_n1m,
    "shock_40x40x800": shock_40x40x800,
    "shock_walls_40x40x800": shock_walls_40x40x800,
    "batched_256": batched_256,
}
