"""Pins of the oracle's walled replicas: specular walls along z at z = 0 and at
z_w(n) = L_z + u n dt (the hard-wall reading of the confining walls of the
shock set-up, Sec. V).

- A free particle moves on the triangle wave of uniform motion folded at the
  walls (exact for a hard wall), p_z flipping sign at each bounce.
- A particle at rest hit by the moving wall leaves with p_z = 2 m u (elastic
  collision with an infinitely heavy wall) from the mirrored position.
- No pair interacts across the z boundary: brute force == cell list ==
  scipy's k-d tree periodic in x, y only.
- With sigma = 0 the walled step stays exactly time reversible (a reflection
  that lost the momentum flip or mirrored the wrong way would not be), and
  its energy error vanishes with dt.
- The SSA sequence of a walled replica covers every pair once and its colour
  classes stay independent (no periodic ring colours along z).
"""
import math

import numpy as np
import pytest


def state(n, box, seed, cv=100.0, kT=1.0):
    rng = np.random.default_rng(seed)
    box = np.asarray(box, float)
    q = rng.random((n, 3)) * box
    p = rng.standard_normal((n, 3)) * math.sqrt(kT)
    p -= p.mean(axis=0)
    eps = cv * kT * (1 + 0.05 * rng.uniform(-1, 1, n))
    return q, p, eps


def triangle(u, L):
    """Position and direction sign of uniform motion u folded into [0, L]."""
    w = np.mod(u, 2 * L)
    return (w, 1.0) if w <= L else (2 * L - w, -1.0)


def test_free_particle_bounces_between_walls(ora):
    box = (3.0, 3.5, 4.0)
    rep = ora.make_replica(1, box, 100.0, walls=1)
    prm = ora.make_params(sigma=0.0)
    q0 = np.array([[1.0, 2.0, 0.7]])
    p0 = np.array([[0.3, -0.2, 2.3]])
    S = ora.System([rep], prm, q0, p0, np.array([100.0]))
    dt = 0.05
    for n in range(1, 200):
        S.run(1, dt, "SER")
        z, sgn = triangle(0.7 + 2.3 * n * dt, box[2])
        assert abs(S.q[0, 2] - z) < 1e-11, n
        assert S.p[0, 2] == sgn * 2.3, n
        # x and y stay periodic and untouched by the walls
        assert abs(S.q[0, 0] - np.mod(1.0 + 0.3 * n * dt, box[0])) < 1e-11
        assert abs(S.q[0, 1] - np.mod(2.0 - 0.2 * n * dt, box[1])) < 1e-11
        assert S.p[0, 0] == 0.3 and S.p[0, 1] == -0.2


def test_moving_wall_reflects_with_twice_its_velocity(ora):
    box, u, dt, m = (3.0, 3.0, 5.0), -1.0, 0.1, 1.7
    rep = ora.make_replica(1, box, 100.0, walls=1, wall_u=u)
    prm = ora.make_params(mass=m, sigma=0.0)
    S = ora.System([rep], prm, np.array([[1.0, 1.0, 4.95]]), np.zeros((1, 3)), np.array([100.0]))
    S.run(1, dt, "SER")
    zw = 5.0 + u * dt
    assert abs(S.q[0, 2] - (2 * zw - 4.95)) < 1e-12
    assert abs(S.p[0, 2] - 2 * m * u) < 1e-15
    # then it moves away at velocity p / m = 2u, twice the wall's
    S.run(1, dt, "SER")
    assert abs(S.q[0, 2] - (2 * zw - 4.95 + 2 * u * dt)) < 1e-12
    # the step index sets the wall position: a run started at step 10 meets a
    # wall already 1.0 lower
    T = ora.System([rep], prm, np.array([[1.0, 1.0, 4.2]]), np.zeros((1, 3)), np.array([100.0]), step=10)
    T.run(1, dt, "SER")
    zw = 5.0 + u * 11 * dt
    assert abs(T.q[0, 2] - (2 * zw - 4.2)) < 1e-12 and abs(T.p[0, 2] - 2 * m * u) < 1e-15


def test_no_pair_across_the_walls(ora):
    box = (3.0, 3.0, 4.0)
    q = np.array([[1.0, 1.0, 0.2], [1.0, 1.0, 3.8], [1.5, 1.0, 0.3]])
    prm = ora.make_params()
    for walls, expect in ((0, {(0, 1), (0, 2), (1, 2)}), (1, {(0, 2)})):
        rep = ora.make_replica(3, box, 100.0, walls=walls)
        for method in ("brute", "cells"):
            assert {tuple(x) for x in ora.pairs(rep, 1.0, q, method)} == expect
    rep = ora.make_replica(3, box, 100.0, walls=1)
    F = ora.forces(rep, prm, q)
    assert np.all(F[1] == 0.0)                     # particle 1 only neighbours across the wall
    assert np.allclose(F[0], -F[2]) and F[0, 0] < 0


def test_particles_on_the_wall_faces_stay_there(ora):
    """A particle on the upper wall face z = L_z is not wrapped to z = 0 (the
    walled z axis has no periodic image): it keeps its position in the
    System, and the potential energy equals a brute-force sum with the
    minimum image along x and y only."""
    n, box = 400, (5.0, 5.0, 6.2)
    q, p, e = state(n, box, 51)
    q[:20, 2] = 0.0
    q[20:40, 2] = box[2]
    q[40:60, 2] = box[2] - 1e-12      # within 1e-12 of the face-bound ones' plane
    S = ora.System([ora.make_replica(n, box, 100.0, walls=1)], ora.make_params(), q, p, e)
    assert np.array_equal(S.q, q)
    L = np.asarray(box)
    U = 0.0
    for i in range(n):
        d = q[i] - q[i + 1:]
        d[:, :2] -= L[:2] * np.round(d[:, :2] / L[:2])
        r = np.sqrt((d * d).sum(axis=1))
        U += (12.5 * (1 - r[r < 1.0]) ** 2).sum()
    assert S.observables()["U"] == pytest.approx(U, rel=1e-12)
    # the periodic reading would wrap the face particles onto z = 0
    P = ora.System([ora.make_replica(n, box, 100.0)], ora.make_params(), q, p, e)
    assert np.all(P.q[20:40, 2] == 0.0)
    assert abs(P.observables()["U"] - U) > 1.0


@pytest.mark.parametrize("n,box,bricks", [(64, (3.3, 6.9, 9.9), (1, 2, 3)), (1000, (6.934,) * 3, (2, 2, 2)),
                                          (600, (5.0, 5.0, 8.1), (1, 1, 1))])
def test_pairs_with_walls_brute_cells_kdtree(ora, n, box, bricks):
    from scipy.spatial import cKDTree
    q, _, _ = state(n, box, seed=n + 5)
    rep = ora.make_replica(n, box, 100.0, bricks, walls=1)
    brute = ora.pairs(rep, 1.0, q, "brute")
    cells = ora.pairs(rep, 1.0, q, "cells")
    assert np.array_equal(brute, cells)
    # periodic along x and y only: a z period far longer than the box never wraps
    tree = cKDTree(q, boxsize=np.array([box[0], box[1], 10 * box[2]]))
    ref = np.array(sorted(tree.query_pairs(1.0 - 1e-12)), dtype=np.int64).reshape(-1, 2)
    assert np.array_equal(brute, ref)


@pytest.mark.parametrize("scheme,bricks", [("SER", (1, 1, 1)), ("SSA", (1, 1, 1)), ("HYBRID", (1, 1, 2))])
def test_walled_verlet_is_time_reversible(ora, scheme, bricks):
    n, box = 200, (4.05, 4.05, 6.2)
    q, p, eps = state(n, box, seed=41)
    p[:, 2] += 1.5                                 # a flux into the upper wall
    rep = ora.make_replica(n, box, 100.0, bricks, walls=1)
    prm = ora.make_params(sigma=0.0)
    S = ora.System([rep], prm, q, p, eps)
    S.run(80, 0.005, scheme)
    assert np.all(S.q[:, 2] >= 0) and np.all(S.q[:, 2] <= box[2])
    S.p = -S.p
    S.run(80, 0.005, scheme)
    dxy = S.q[:, :2] - q[:, :2]
    dxy -= np.asarray(box[:2]) * np.round(dxy / np.asarray(box[:2]))
    assert np.max(np.abs(dxy)) < 1e-9 and np.max(np.abs(S.q[:, 2] - q[:, 2])) < 1e-9
    assert np.max(np.abs(S.p + p)) < 1e-9


def test_walled_verlet_energy_error_vanishes_with_dt(ora):
    """The reflection flips the wall-normal part of the first half-kick but
    not of the second, an O(F v dt) energy error per wall collision; with a
    dt-independent collision rate the error is first order in dt (second
    order away from the walls)."""
    n, box = 150, (4.05, 4.05, 3.4)
    q, p, eps = state(n, box, seed=42)
    rep = ora.make_replica(n, box, 100.0, walls=1)
    prm = ora.make_params(sigma=0.0)
    S = ora.System([rep], prm, q, p, eps)
    S.run(200, 0.002, "SER")
    q0, p0, e0 = S.q.copy(), S.p.copy(), S.eps.copy()
    errs = []
    for dt in (0.004, 0.002):
        T = ora.System([rep], prm, q0, p0, e0)
        E0 = T.observables()["E"]
        worst = 0.0
        for _ in range(int(round(0.4 / dt))):
            T.run(1, dt, "SER")
            worst = max(worst, abs(T.observables()["E"] - E0))
        errs.append(worst)
    assert errs[0] < 1e-3 * abs(E0)
    assert 1.5 < errs[0] / errs[1] < 5.0, errs


@pytest.mark.parametrize("bricks,box", [((1, 1, 1), (6.934, 7.5, 9.7)), ((1, 2, 3), (6.934, 7.5, 9.7)),
                                        ((1, 1, 1), (3.2, 4.4, 3.3))])
@pytest.mark.parametrize("whole_box", [False, True])
def test_walled_ssa_order(ora, bricks, box, whole_box):
    n = int(3 * np.prod(box))
    q, _, _ = state(n, box, seed=18)
    rep = ora.make_replica(n, box, 100.0, bricks, walls=1)
    nc, k = ora.cell_grid(rep, 1.0)
    cell = np.stack([np.minimum(nc[d] - 1, (q[:, d] * (nc[d] / box[d])).astype(int)) for d in range(3)], axis=1)
    allp = {tuple(x) for x in ora.pairs(rep, 1.0, q)}
    seq = ora.ssa_order(rep, 1.0, q, whole_box=whole_box)
    got = [tuple(sorted(x)) for x in seq]
    if whole_box:
        assert len(got) == len(set(got)) and set(got) == allp
    dom_k = np.array(nc if whole_box else k)
    # rings (extra colours) only along periodic axes that one domain spans
    ring = [(whole_box or bricks[d] == 1) and d != 2 for d in range(3)]

    def colour(c):
        out = []
        for d, P in enumerate((3, 3, 2)):
            l = c[d] % dom_k[d]
            full = P * (dom_k[d] // P)
            out.append(P + l - full if ring[d] and l >= full else l % P)
        return (out[2], out[1], out[0])

    cols = [colour(cell[i]) for i, _ in seq]
    assert cols == sorted(cols)
    for col in set(cols):
        touched = {}
        for u in (u for u, c in enumerate(cols) if c == col):
            i, j = seq[u]
            for x in (i, j):
                assert touched.setdefault(int(x), tuple(cell[i])) == tuple(cell[i])
