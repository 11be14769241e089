"""Pins of the oracle's pair search, forces and observables.

- Pair set: brute force over all pairs == cell list == scipy's periodic
  k-d tree (an independent library routine).
- Forces: F = -grad U by central finite differences of U; Newton's third law.
- Laplacian of U (denominator of Eq. Tcon) by finite differences of F.
- Two-particle hand case of the soft force and potential.
- Eq. (Tint) harmonic mean and Eq. (Tkin) on hand-made states.
"""
import math

import numpy as np
import pytest


def random_state(n, box, seed, spread=0.05, cv=100.0):
    rng = np.random.default_rng(seed)
    box = np.asarray(box, float)
    q = rng.random((n, 3)) * box
    p = rng.standard_normal((n, 3))
    p -= p.mean(axis=0)
    eps = cv * (1 + spread * rng.uniform(-1, 1, n))
    return q, p, eps


@pytest.mark.parametrize("n,box,bricks", [
    (2, (3.0, 3.0, 3.0), (1, 1, 1)),
    (17, (3.1, 3.5, 4.2), (1, 1, 1)),
    (64, (4.0, 4.0, 4.0), (2, 2, 2)),
    (64, (3.3, 6.9, 9.9), (1, 2, 3)),
    (1000, (6.934, 6.934, 6.934), (2, 2, 2)),
    (3000, (7.0, 10.0, 14.3), (1, 2, 2)),
])
def test_pairs_brute_cells_kdtree(ora, n, box, bricks):
    from scipy.spatial import cKDTree
    q, _, _ = random_state(n, box, seed=n)
    rep = ora.make_replica(n, box, 100.0, bricks)
    brute = ora.pairs(rep, 1.0, q, "brute")
    cells = ora.pairs(rep, 1.0, q, "cells")
    assert np.array_equal(brute, cells)
    tree = cKDTree(q, boxsize=np.asarray(box))
    ref = np.array(sorted(tree.query_pairs(1.0 - 1e-12)), dtype=np.int64).reshape(-1, 2)
    assert np.array_equal(brute, ref)


def test_pairs_edge_positions(ora):
    # particles on the box faces, at the same point, and exactly r_cut apart
    box = (5.0, 5.0, 5.0)
    q = np.array([[0.0, 0.0, 0.0], [4.999999999, 0.0, 0.0], [0.0, 0.0, 0.0],
                  [2.0, 2.0, 2.0], [3.0, 2.0, 2.0], [2.5, 2.5, 4.9999]])
    rep = ora.make_replica(len(q), box, 100.0)
    P = ora.pairs(rep, 1.0, q, "cells")
    assert np.array_equal(P, ora.pairs(rep, 1.0, q, "brute"))
    s = {tuple(x) for x in P}
    assert (0, 1) in s and (0, 2) in s and (1, 2) in s
    assert (3, 4) not in s      # r == r_cut does not interact


def energy(ora, rep, prm, q):
    return ora.System([rep], prm, q, np.zeros_like(q), np.full(len(q), 100.0)).observables()["U"]


def test_forces_are_minus_gradient(ora):
    n, box = 40, (3.4, 3.4, 3.4)
    q, _, _ = random_state(n, box, seed=3)
    rep = ora.make_replica(n, box, 100.0)
    prm = ora.make_params(a=25.0)
    F = ora.forces(rep, prm, q)
    h = 1e-6
    Ffd = np.zeros_like(F)
    for i in range(n):
        for d in range(3):
            qp = q.copy(); qp[i, d] += h
            qm = q.copy(); qm[i, d] -= h
            Ffd[i, d] = -(energy(ora, rep, prm, qp) - energy(ora, rep, prm, qm)) / (2 * h)
    assert np.max(np.abs(F - Ffd)) < 1e-5 * max(1.0, np.max(np.abs(F)))
    assert np.max(np.abs(F.sum(axis=0))) < 1e-11


def test_laplacian_by_finite_differences(ora):
    n, box = 30, (3.2, 3.2, 3.2)
    q, p, eps = random_state(n, box, seed=4)
    rep = ora.make_replica(n, box, 100.0)
    prm = ora.make_params(a=25.0)
    obs = ora.System([rep], prm, q, p, eps).observables()
    h = 1e-5
    lap = 0.0
    for i in range(n):
        for d in range(3):
            qp = q.copy(); qp[i, d] += h
            qm = q.copy(); qm[i, d] -= h
            lap += -(ora.forces(rep, prm, qp)[i, d] - ora.forces(rep, prm, qm)[i, d]) / (2 * h)
    assert abs(lap - obs["Tpot_den"]) < 1e-4 * abs(lap)
    F = ora.forces(rep, prm, q)
    assert abs(obs["Tpot_num"] - (F**2).sum()) < 1e-9 * (F**2).sum()


def test_two_particle_force_hand_case(ora):
    # r = 0.5 along x, a = 25, r_cut = 1: |F| = a (1 - r) = 12.5, repulsive;
    # v = (a/2)(1 - r)^2 = 3.125
    box = (4.0, 4.0, 4.0)
    q = np.array([[1.5, 1.0, 1.0], [1.0, 1.0, 1.0]])
    rep = ora.make_replica(2, box, 100.0)
    prm = ora.make_params(a=25.0)
    F = ora.forces(rep, prm, q)
    assert np.allclose(F, [[12.5, 0, 0], [-12.5, 0, 0]], atol=1e-14)
    assert abs(energy(ora, rep, prm, q) - 3.125) < 1e-14
    # across the periodic boundary: q_x = 0.2 and 3.9 are 0.3 apart
    q2 = np.array([[0.2, 1.0, 1.0], [3.9, 1.0, 1.0]])
    F2 = ora.forces(rep, prm, q2)
    assert np.allclose(F2, [[25 * 0.7, 0, 0], [-25 * 0.7, 0, 0]], atol=1e-12)


def test_temperatures_hand_case(ora):
    box = (4.0, 4.0, 4.0)
    q = np.array([[0.5, 0.5, 0.5], [2.5, 2.5, 2.5], [0.5, 2.5, 0.5]])
    p = np.array([[1.0, 0.0, 0.0], [0.0, -2.0, 0.0], [-1.0, 2.0, 0.0]])
    eps = np.array([100.0, 200.0, 50.0])
    rep = ora.make_replica(3, box, 100.0)
    o = ora.System([rep], ora.make_params(), q, p, eps).observables()
    K = (1 + 4 + 5) / 2.0
    assert o["K"] == pytest.approx(K, abs=1e-14)
    assert o["Tkin"] == pytest.approx(2 * K / (3 * 2), abs=1e-14)        # d (N-1) = 6
    assert o["Tint"] == pytest.approx(3 / (1 / 1.0 + 1 / 2.0 + 1 / 0.5), abs=1e-14)
    assert o["Eint"] == 350.0 and o["U"] == 0.0 and o["E"] == pytest.approx(350.0 + K)
    assert (o["Px"], o["Py"], o["Pz"]) == (0.0, 0.0, 0.0)
