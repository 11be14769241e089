"""Pins of the oracle's fluctuation/dissipation schemes (Sec. III).

Hand cases (two particles, noise switched off) for SER and SSA; the exact
invariants the paper states (momentum for every scheme; total energy for SER,
SSA and Hybrid; SEM as the negative control); the reductions Hybrid(one
domain) = SSA, Hybrid(no intra-domain pair) = SER, p-update(SER) =
p-update(SEM); the SSA pair map checked against an Euler-Maruyama simulation
of the pair SDE Eq. (DPDE_ij); and the mean internal-energy increment of SER
against SEM (Appendix B.2: E[B_ij] = d sigma^2 chi / m).
"""
import math

import numpy as np
import pytest


def state(n, box, seed, cv=100.0, spread=0.05):
    rng = np.random.default_rng(seed)
    q = rng.random((n, 3)) * np.asarray(box)
    p = rng.standard_normal((n, 3))
    p -= p.mean(axis=0)
    eps = cv * (1 + spread * rng.uniform(-1, 1, n))
    return q, p, eps


def kinetic(p, m=1.0):
    return (p * p).sum() / (2 * m)


# ---- hand cases -------------------------------------------------------------

def two_particles():
    # r = 0.5 (chi = 1/4), T_i = T_j = 1, sigma = 3 -> gamma = 9/4 * 2 = 4.5
    q = np.array([[1.5, 1.0, 1.0], [1.0, 1.0, 1.0]])
    p = np.array([[0.5, 0.0, 0.0], [-0.5, 0.0, 0.0]])
    eps = np.array([100.0, 100.0])
    return q, p, eps


def test_ser_hand_case(ora):
    # Eq. (SER_p): dp_ij = -gamma chi v_ij dt = -4.5 * 0.25 * 1 * 0.01 = -0.01125
    # Eq. (SER_eint_discretization): Delta eps_i = -1/2 dp_ij (v_ij + (dp_i - dp_j)/2)
    #   = 0.005625 * (1 - 0.01125) = 0.00556171875 for both particles
    q, p, eps = two_particles()
    rep = ora.make_replica(2, (4.0, 4.0, 4.0), 100.0)
    prm = ora.make_params(sigma=3.0, noise=False)
    p1, e1 = ora.fd(rep, 0, prm, q, p, eps, 0, 0.01, "SER")
    assert np.allclose(p1, [[0.48875, 0, 0], [-0.48875, 0, 0]], atol=1e-15, rtol=0)
    assert np.allclose(e1 - eps, [0.00556171875, 0.00556171875], atol=3e-14, rtol=0)
    assert kinetic(p1) - kinetic(p) == pytest.approx(-0.0111234375, abs=1e-15)


def test_ssa_hand_case(ora):
    # a = 2 gamma chi dt / m = 0.0225; p_ij = (1, 0, 0);
    # Delta = 1/2 (e^{-a} - 1) p_ij ; eps_i, eps_j -= Delta K / 2
    q, p, eps = two_particles()
    rep = ora.make_replica(2, (4.0, 4.0, 4.0), 100.0)
    prm = ora.make_params(sigma=3.0, noise=False)
    p1, e1 = ora.fd(rep, 0, prm, q, p, eps, 0, 0.01, "SSA")
    delta = 0.5 * (math.exp(-0.0225) - 1.0)
    assert p1[0, 0] == pytest.approx(0.5 + delta, abs=1e-15)
    assert p1[1, 0] == pytest.approx(-0.5 - delta, abs=1e-15)
    dK = (0.5 + delta) ** 2 - 0.25
    assert np.allclose(e1 - eps, [-dK / 2, -dK / 2], atol=3e-14, rtol=0)


# Unequal internal temperatures pin gamma_ij = sigma^2/4 (1/T_i + 1/T_j) of
# Eq. (DPDE_fd) with T_i = eps_i / C_v (Eq. DPDE_internalEOS at constant C_v).
# The cases are chosen so that 1/T_i + 1/T_j differs from T_i + T_j, from
# 2 / mean(T) and from the equal-temperature value: a formula using T in place
# of beta, or dropping one particle's term, fails them.
#   cv = 100, eps = (200, 100): beta = (1/2, 1),  gamma = 9/4 * 3/2 = 27/8
#   cv =  50, eps = (25, 200):  beta = (2, 1/4),  gamma = 9/4 * 9/4 = 81/16
UNEQUAL_T = [
    # cv, eps_i, eps_j, gamma
    (100.0, 200.0, 100.0, 27.0 / 8.0),
    (50.0, 25.0, 200.0, 81.0 / 16.0),
]


@pytest.mark.parametrize("cv,ei,ej,gam", UNEQUAL_T)
def test_ser_hand_case_unequal_temperatures(ora, cv, ei, ej, gam):
    # chi = 1/4, v_ij = 1, dt = 0.01: dp_ij = -gamma / 400; every term of
    # Eq. (SER_eint_discretization) is exact in binary for these gammas:
    # Delta eps_i = Delta eps_j = -1/2 dp_ij (1 + dp_ij)
    q, p, _ = two_particles()
    eps = np.array([ei, ej])
    rep = ora.make_replica(2, (4.0, 4.0, 4.0), cv)
    prm = ora.make_params(sigma=3.0, noise=False)
    p1, e1 = ora.fd(rep, 0, prm, q, p, eps, 0, 0.01, "SER")
    dp = -gam / 400.0
    expect_p = {27.0 / 8.0: 0.4915625, 81.0 / 16.0: 0.48734375}[gam]
    expect_de = {27.0 / 8.0: 0.004183154296875, 81.0 / 16.0: 0.00624803466796875}[gam]
    assert 0.5 + dp == expect_p
    assert np.allclose(p1, [[expect_p, 0, 0], [-expect_p, 0, 0]], atol=1e-15, rtol=0)
    assert np.allclose(e1 - eps, [expect_de, expect_de], atol=3e-14, rtol=0)


@pytest.mark.parametrize("cv,ei,ej,gam", UNEQUAL_T)
def test_ssa_hand_case_unequal_temperatures(ora, cv, ei, ej, gam):
    # a = 2 gamma chi dt / m = gamma / 200 (0.016875 and 0.0253125)
    q, p, _ = two_particles()
    eps = np.array([ei, ej])
    rep = ora.make_replica(2, (4.0, 4.0, 4.0), cv)
    prm = ora.make_params(sigma=3.0, noise=False)
    p1, e1 = ora.fd(rep, 0, prm, q, p, eps, 0, 0.01, "SSA")
    a = {27.0 / 8.0: 0.016875, 81.0 / 16.0: 0.0253125}[gam]
    delta = 0.5 * math.expm1(-a)
    assert p1[0, 0] == pytest.approx(0.5 + delta, abs=1e-15)
    assert p1[1, 0] == pytest.approx(-0.5 - delta, abs=1e-15)
    dK = (0.5 + delta) ** 2 - 0.25
    assert np.allclose(e1 - eps, [-dK / 2, -dK / 2], atol=3e-14, rtol=0)


@pytest.mark.parametrize("cv,ei,ej,gam", UNEQUAL_T)
def test_sem_hand_case_unequal_temperatures(ora, cv, ei, ej, gam):
    # Eq. (SEM_fd), G = 0: Delta eps = 1/2 (gamma - 27) / 400 for both
    # (-0.02953125 and -0.027421875)
    q, p, _ = two_particles()
    eps = np.array([ei, ej])
    rep = ora.make_replica(2, (4.0, 4.0, 4.0), cv)
    prm = ora.make_params(sigma=3.0, noise=False)
    p1, e1 = ora.fd(rep, 0, prm, q, p, eps, 0, 0.01, "SEM")
    expect = {27.0 / 8.0: -0.02953125, 81.0 / 16.0: -0.027421875}[gam]
    assert np.allclose(e1 - eps, [expect, expect], atol=3e-14, rtol=0)


def test_sem_hand_case(ora):
    # Eq. (SEM_fd) with G = 0: Delta eps_i = 1/2 (gamma v_ij^2 - d sigma^2/m) chi dt
    #   = 0.5 * (4.5 - 27) * 0.25 * 0.01 = -0.028125
    q, p, eps = two_particles()
    rep = ora.make_replica(2, (4.0, 4.0, 4.0), 100.0)
    prm = ora.make_params(sigma=3.0, noise=False)
    p1, e1 = ora.fd(rep, 0, prm, q, p, eps, 0, 0.01, "SEM")
    assert np.allclose(p1, [[0.48875, 0, 0], [-0.48875, 0, 0]], atol=1e-15, rtol=0)
    assert np.allclose(e1 - eps, [-0.028125, -0.028125], atol=3e-14, rtol=0)


# ---- invariants ---------------------------------------------------------------

@pytest.mark.parametrize("scheme", ["SER", "HYBRID", "SSA", "SEM"])
def test_fd_conserves_momentum(ora, scheme):
    n, box = 1000, (6.934,) * 3
    q, p, eps = state(n, box, seed=11)
    rep = ora.make_replica(n, box, 100.0, (2, 2, 2))
    prm = ora.make_params(sigma=3.0, seed=5)
    p1, _ = ora.fd(rep, 0, prm, q, p, eps, 3, 0.01, scheme)
    assert np.max(np.abs(p1.sum(axis=0) - p.sum(axis=0))) < 1e-12
    assert np.max(np.abs(p1 - p)) > 1e-3   # the map did act


@pytest.mark.parametrize("scheme", ["SER", "HYBRID", "SSA"])
def test_fd_conserves_energy(ora, scheme):
    n, box = 1000, (6.934,) * 3
    q, p, eps = state(n, box, seed=12)
    rep = ora.make_replica(n, box, 100.0, (2, 2, 2))
    prm = ora.make_params(sigma=3.0, seed=6)
    p1, e1 = ora.fd(rep, 0, prm, q, p, eps, 4, 0.01, scheme)
    E0 = kinetic(p) + eps.sum()
    E1 = kinetic(p1) + e1.sum()
    assert abs(E1 - E0) < 1e-12 * E0
    assert np.max(np.abs(e1 - eps)) > 1e-4


def test_sem_does_not_conserve_energy(ora):
    n, box = 1000, (6.934,) * 3
    q, p, eps = state(n, box, seed=12)
    rep = ora.make_replica(n, box, 100.0)
    prm = ora.make_params(sigma=3.0, seed=6)
    p1, e1 = ora.fd(rep, 0, prm, q, p, eps, 4, 0.01, "SEM")
    E0 = kinetic(p) + eps.sum()
    assert abs(kinetic(p1) + e1.sum() - E0) > 1e-6 * E0


# ---- reductions ---------------------------------------------------------------

def test_hybrid_one_domain_is_ssa(ora):
    n, box = 500, (5.5, 5.5, 5.5)
    q, p, eps = state(n, box, seed=13)
    rep = ora.make_replica(n, box, 100.0, (1, 1, 1))
    prm = ora.make_params(seed=7)
    ph, eh = ora.fd(rep, 0, prm, q, p, eps, 9, 0.01, "HYBRID")
    ps, es = ora.fd(rep, 0, prm, q, p, eps, 9, 0.01, "SSA")
    assert np.array_equal(ph, ps) and np.array_equal(eh, es)


def test_hybrid_without_intra_pairs_is_ser(ora):
    # one particle per domain: every interacting pair crosses domains
    rng = np.random.default_rng(14)
    B = (4, 4, 4)
    box = (4.4, 4.4, 4.4)
    cells = np.array([(x, y, z) for z in range(4) for y in range(4) for x in range(4)], float)
    q = (cells + rng.random(cells.shape)) * 1.1
    n = len(q)
    p = rng.standard_normal((n, 3))
    eps = 100 * (1 + 0.05 * rng.uniform(-1, 1, n))
    rep = ora.make_replica(n, box, 100.0, B)
    prm = ora.make_params(seed=8)
    assert len(ora.ssa_order(rep, 1.0, q)) == 0
    assert len(ora.pairs(rep, 1.0, q)) > 20
    ph, eh = ora.fd(rep, 0, prm, q, p, eps, 2, 0.01, "HYBRID")
    ps, es = ora.fd(rep, 0, prm, q, p, eps, 2, 0.01, "SER")
    assert np.array_equal(ph, ps) and np.array_equal(eh, es)


def test_ser_and_sem_share_the_momentum_update(ora):
    n, box = 800, (6.5, 6.5, 6.5)
    q, p, eps = state(n, box, seed=15)
    rep = ora.make_replica(n, box, 100.0)
    prm = ora.make_params(seed=9)
    p_ser, _ = ora.fd(rep, 0, prm, q, p, eps, 1, 0.01, "SER")
    p_sem, _ = ora.fd(rep, 0, prm, q, p, eps, 1, 0.01, "SEM")
    assert np.array_equal(p_ser, p_sem)


@pytest.mark.parametrize("bricks", [(1, 1, 1), (2, 2, 2), (1, 2, 3), (3, 1, 1)])
def test_ssa_order_covers_each_pair_once(ora, bricks):
    n, box = 1500, (6.934, 7.5, 9.7)
    q, _, _ = state(n, box, seed=16)
    rep = ora.make_replica(n, box, 100.0, bricks)
    allp = {tuple(x) for x in ora.pairs(rep, 1.0, q)}
    whole = [tuple(sorted(x)) for x in ora.ssa_order(rep, 1.0, q, whole_box=True)]
    assert len(whole) == len(set(whole)) and set(whole) == allp
    nc, k = ora.cell_grid(rep, 1.0)
    brick = np.stack([np.minimum(nc[d] - 1, (q[:, d] * (nc[d] / box[d])).astype(int)) // k[d]
                      for d in range(3)], axis=1)
    intra = {pr for pr in allp if np.array_equal(brick[pr[0]], brick[pr[1]])}
    got = [tuple(sorted(x)) for x in ora.ssa_order(rep, 1.0, q)]
    assert len(got) == len(set(got)) and set(got) == intra


@pytest.mark.parametrize("bricks,box", [((1, 1, 1), (6.934, 7.5, 9.7)), ((2, 2, 2), (6.934, 7.5, 9.7)),
                                        ((1, 2, 3), (6.934, 7.5, 9.7)), ((3, 1, 1), (7.5, 4.2, 5.3)),
                                        ((2, 1, 1), (4.1, 3.4, 5.3)), ((1, 1, 1), (3.2, 4.4, 3.3))])
@pytest.mark.parametrize("whole_box", [False, True])
def test_ssa_order_colour_classes_are_independent(ora, bricks, box, whole_box):
    """The sequence is a run of colour classes; inside one class the pairs of
    different cells touch disjoint particles, so any interleaving of those
    cells (the parallel execution) applies the same maps to the same values.
    Inside a cell, the first particles come in ascending id."""
    n = int(3 * np.prod(box))
    q, _, _ = state(n, box, seed=17)
    rep = ora.make_replica(n, box, 100.0, bricks)
    nc, k = ora.cell_grid(rep, 1.0)
    cell = np.stack([np.minimum(nc[d] - 1, (q[:, d] * (nc[d] / box[d])).astype(int)) for d in range(3)], axis=1)
    dom_k = np.array(nc if whole_box else k)
    periodic = [whole_box or bricks[d] == 1 for d in range(3)]

    def colour(c):
        out = []
        for d, P in enumerate((3, 3, 2)):
            l = c[d] % dom_k[d]
            full = P * (dom_k[d] // P)
            out.append(P + l - full if periodic[d] and l >= full else l % P)
        return (out[2], out[1], out[0])

    seq = ora.ssa_order(rep, 1.0, q, whole_box=whole_box)
    assert len(seq) > 0
    cols = [colour(cell[i]) for i, _ in seq]
    assert cols == sorted(cols)                      # classes in lexicographic order
    for col in set(cols):
        idx = [u for u, c in enumerate(cols) if c == col]
        touched = {}
        for u in idx:
            i, j = seq[u]
            owner = tuple(cell[i])
            for x in (i, j):
                assert touched.setdefault(int(x), owner) == owner
        # per cell, a contiguous block with i non-decreasing
        owners = [tuple(cell[seq[u][0]]) for u in idx]
        for o in set(owners):
            pos = [v for v, w in enumerate(owners) if w == o]
            assert pos == list(range(pos[0], pos[0] + len(pos)))
            firsts = [seq[idx[v]][0] for v in pos]
            assert firsts == sorted(firsts)


# ---- statistics -----------------------------------------------------------------

def test_ssa_map_matches_pair_sde(ora):
    """Isolated pairs, fixed gamma: the SSA map is the exact transition of the
    pair dynamics Eq. (DPDE_ij). Compare its one-step law with a fine
    Euler-Maruyama integration of that SDE (independent of the closed form)."""
    M, dt, sigma, m = 12000, 0.2, 3.0, 1.0
    side = int(math.ceil(M ** (1 / 3)))
    sites = np.array([(x, y, z) for z in range(side) for y in range(side) for x in range(side)][:M],
                     float) * 3.0
    L = side * 3.0
    q = np.empty((2 * M, 3))
    q[0::2] = sites + 0.5
    q[1::2] = sites + 0.5 + np.array([0.5, 0.0, 0.0])
    p = np.empty((2 * M, 3))
    p0 = np.array([0.8, -0.3, 0.1])
    p[0::2] = p0 / 2
    p[1::2] = -p0 / 2
    cv = 1e9                      # gamma stays fixed to ~1e-9 during the step
    eps = np.full(2 * M, cv)      # T = 1
    rep = ora.make_replica(2 * M, (L, L, L), cv)
    prm = ora.make_params(sigma=sigma, seed=21)
    p1, _ = ora.fd(rep, 0, prm, q, p, eps, 0, dt, "SSA")
    pij = p1[0::2] - p1[1::2]
    # Euler-Maruyama of d p_ij = -(2 gamma chi / m) p_ij dt + 2 sigma sqrt(chi) dW
    chi, gamma = 0.25, sigma**2 / 4 * 2.0
    rng = np.random.default_rng(3)
    x = np.tile(p0, (M, 1))
    nsub = 400
    h = dt / nsub
    for _ in range(nsub):
        x = x - 2 * gamma * chi / m * x * h + 2 * sigma * math.sqrt(chi * h) * rng.standard_normal(x.shape)
    for k in range(3):
        se = math.sqrt(x[:, k].var() / M)
        assert abs(pij[:, k].mean() - x[:, k].mean()) < 5 * math.sqrt(2) * se
        assert abs(pij[:, k].var() / x[:, k].var() - 1) < 0.06
    # the mean decays as e^{-a}, a = 2 gamma chi dt / m = 0.45
    assert abs(pij[:, 0].mean() / p0[0] - math.exp(-0.45)) < 0.03


def test_ser_energy_increment_mean_matches_sem(ora):
    """Appendix B.2: the SER energy update differs from SEM's by terms with
    zero mean (C_ij) and by B_ij - d sigma^2 chi / m, whose mean vanishes.
    Averaged over noise draws, Delta eps(SER) - Delta eps(SEM) = O(dt^2)."""
    n, box, dt = 60, (3.3, 3.3, 3.3), 0.002
    q, p, eps = state(n, box, seed=17)
    rep = ora.make_replica(n, box, 100.0)
    diffs, sem_noise_term = [], None
    for s in range(1500):
        prm = ora.make_params(sigma=3.0, seed=1000 + s)
        _, e_ser = ora.fd(rep, 0, prm, q, p, eps, 0, dt, "SER")
        _, e_sem = ora.fd(rep, 0, prm, q, p, eps, 0, dt, "SEM")
        diffs.append(e_ser - e_sem)
    diffs = np.array(diffs)
    mean = diffs.mean(axis=0)
    se = diffs.std(axis=0) / math.sqrt(len(diffs))
    # the term that a wrong sign of (dp_i - dp_j) would leave: d sigma^2 chi dt / (2m) per pair
    P = ora.pairs(rep, 1.0, q)
    scale = np.zeros(n)
    for i, j in P:
        r = np.linalg.norm((q[i] - q[j] + 1.65) % 3.3 - 1.65)
        scale[i] += 3 * 9 * (1 - r) ** 2 * dt / 2
        scale[j] += 3 * 9 * (1 - r) ** 2 * dt / 2
    assert np.all(np.abs(mean) < 5 * se + 0.05 * scale)
    assert np.mean(np.abs(mean)) < 0.2 * np.mean(scale)
