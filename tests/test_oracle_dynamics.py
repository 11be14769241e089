"""Pins of the oracle's full timestep: velocity Verlet (Sec. III.A) and the
equilibrium the fluctuation/dissipation relation fixes (Sec. II.B).

- With sigma = 0 the FD part is the identity and the step is plain velocity
  Verlet: energy error O(dt^2), exact time reversibility, exact momentum.
- Equilibrium: T_kin = T_int at equilibrium (Eq. Tkin, Eq. Tint and the
  remark that all temperature estimators agree).
- A run split in two pieces equals the same run done at once (the noise is a
  pure function of (seed, step, ids)).
"""
import math

import numpy as np
import pytest


def state(n, box, seed, cv=100.0, kT=1.0):
    rng = np.random.default_rng(seed)
    q = rng.random((n, 3)) * np.asarray(box)
    p = rng.standard_normal((n, 3)) * math.sqrt(kT)
    p -= p.mean(axis=0)
    eps = cv * kT * (1 + 0.05 * rng.uniform(-1, 1, n))
    return q, p, eps


def min_image(d, box):
    box = np.asarray(box)
    return d - box * np.round(d / box)


def test_verlet_energy_error_is_second_order(ora):
    n, box = 200, (4.05,) * 3
    q, p, eps = state(n, box, seed=31)
    rep = ora.make_replica(n, box, 100.0)
    prm = ora.make_params(sigma=0.0)
    # relax overlaps first so that the energy error is in the asymptotic regime
    S = ora.System([rep], prm, q, p, eps)
    S.run(200, 0.002, "SER")
    q0, p0, e0 = S.q.copy(), S.p.copy(), S.eps.copy()
    errs = []
    for dt in (0.01, 0.005):
        S = ora.System([rep], prm, q0, p0, e0)
        E0 = S.observables()["E"]
        worst = 0.0
        for _ in range(int(round(0.5 / dt))):
            S.run(1, dt, "SER")
            worst = max(worst, abs(S.observables()["E"] - E0))
        errs.append(worst)
        assert np.array_equal(S.eps, e0)          # sigma = 0: FD is the identity
    ratio = errs[0] / errs[1]
    assert 3.0 < ratio < 5.0, ratio


def test_verlet_time_reversible_and_momentum(ora):
    n, box = 200, (4.05,) * 3
    q, p, eps = state(n, box, seed=32)
    rep = ora.make_replica(n, box, 100.0)
    prm = ora.make_params(sigma=0.0)
    S = ora.System([rep], prm, q, p, eps)
    P0 = S.p.sum(axis=0)
    S.run(100, 0.005, "SER")
    assert np.max(np.abs(S.p.sum(axis=0) - P0)) < 1e-11
    S.p = -S.p
    S.run(100, 0.005, "SER")
    assert np.max(np.abs(min_image(S.q - q, box))) < 1e-9
    assert np.max(np.abs(S.p + p)) < 1e-9


@pytest.mark.parametrize("scheme", ["SER", "HYBRID", "SSA", "SEM"])
def test_split_run_equals_single_run(ora, scheme):
    n, box = 300, (4.64,) * 3
    q, p, eps = state(n, box, seed=33)
    rep = ora.make_replica(n, box, 100.0, (1, 1, 1) if scheme != "HYBRID" else (1, 2, 1))
    prm = ora.make_params(seed=77)
    A = ora.System([rep], prm, q, p, eps)
    A.run(10, 0.01, scheme)
    B = ora.System([rep], prm, q, p, eps)
    B.run(4, 0.01, scheme)
    C = ora.System([rep], prm, B.q, B.p, B.eps, step=B.step)
    C.run(6, 0.01, scheme)
    assert np.array_equal(A.q, C.q) and np.array_equal(A.p, C.p) and np.array_equal(A.eps, C.eps)


def test_replicas_are_independent(ora):
    box = (4.64,) * 3
    q1, p1, e1 = state(300, box, seed=34)
    q2, p2, e2 = state(200, (4.2,) * 3, seed=35, cv=10.0)
    r1 = ora.make_replica(300, box, 100.0)
    r2 = ora.make_replica(200, (4.2,) * 3, 10.0)
    prm = ora.make_params(seed=5)
    both = ora.System([r1, r2], prm, np.vstack([q1, q2]), np.vstack([p1, p2]), np.concatenate([e1, e2]))
    both.run(5, 0.01, "SER")
    alone = ora.System([r1], prm, q1, p1, e1)
    alone.run(5, 0.01, "SER")
    assert np.array_equal(both.p[:300], alone.p) and np.array_equal(both.eps[:300], alone.eps)
    # replica index enters the noise: replica 1 alone (index 0) differs
    alone2 = ora.System([r2], prm, q2, p2, e2)
    alone2.run(5, 0.01, "SER")
    assert not np.array_equal(both.p[300:], alone2.p)


@pytest.mark.parametrize("scheme,dt,tol,kT", [("SSA", 0.01, 0.04, 1.0), ("HYBRID", 0.01, 0.04, 1.0),
                                              ("SSA", 0.01, 0.04, 2.0), ("HYBRID", 0.01, 0.04, 2.0),
                                              ("SER", 0.005, 0.05, 2.0)])
def test_equilibrium_kinetic_equals_internal_temperature(ora, scheme, dt, tol, kT):
    """At kT = 1 every beta_i = C_v / eps_i is close to T_i = eps_i / C_v, so
    only the run at kT = 2 (beta ~ 1/2, T ~ 2) tells the fluctuation/
    dissipation relation Eq. (DPDE_fd), gamma ~ 1/T_i + 1/T_j, from a wrong
    one: with gamma ~ T_i + T_j the kinetic temperature would settle near
    1/T_int instead of T_int."""
    n, box = 300, (4.64,) * 3
    q, p, eps = state(n, box, seed=36, cv=10.0, kT=kT)
    rep = ora.make_replica(n, box, 10.0, (2, 1, 1))
    S = ora.System([rep], ora.make_params(sigma=3.0, seed=3), q, p, eps)
    S.run(int(5.0 / dt), dt, scheme)              # relax
    tk, ti = [], []
    for _ in range(200):
        S.run(int(0.1 / dt), dt, scheme)
        o = S.observables()
        tk.append(o["Tkin"])
        ti.append(o["Tint"])
    tk, ti = np.mean(tk), np.mean(ti)
    assert abs(tk / ti - 1) < tol, (tk, ti)
    assert kT < tk < 1.5 * kT, tk                  # heated a little by the relaxing overlaps


def test_equilibrium_internal_energies_are_gamma_distributed(ora):
    """Canonical measure of the internal energies (Sec. IV.B; the invariant
    measure Eq. (DPDE_invariant_measure_general) with s'(eps) = 1/T(eps) =
    C_v / eps): eps_i has density ~ eps^C_v exp(-eps / k_B T), the Gamma law of
    shape C_v + 1 and scale k_B T. Its scale must equal the kinetic
    temperature, and its shape is checked by the relative variance 1/(C_v + 1)
    and a Kolmogorov-Smirnov distance. Run at kT = 2, where beta_i and T_i
    differ."""
    stats = pytest.importorskip("scipy.stats")
    n, box, cv, dt = 300, (4.64,) * 3, 10.0, 0.01
    q, p, eps = state(n, box, seed=37, cv=cv, kT=2.0)
    rep = ora.make_replica(n, box, cv, (1, 1, 1))
    S = ora.System([rep], ora.make_params(sigma=3.0, seed=4), q, p, eps)
    S.run(500, dt, "SSA")
    samples, tk = [], []
    for _ in range(150):
        S.run(40, dt, "SSA")
        samples.append(S.eps.copy())
        tk.append(S.observables()["Tkin"])
    e = np.concatenate(samples)
    theta = e.mean() / (cv + 1.0)
    assert abs(theta / np.mean(tk) - 1) < 0.03, (theta, np.mean(tk))
    rel_var = e.var() / e.mean() ** 2
    assert abs(rel_var * (cv + 1.0) - 1) < 0.06, rel_var      # shape C_v would give 1.1
    D = stats.kstest(e, stats.gamma(cv + 1.0, scale=theta).cdf).statistic
    D_wrong = stats.kstest(e, stats.gamma(cv, scale=e.mean() / cv).cdf).statistic
    assert D < 0.03, D
    assert D_wrong > 2 * D, (D, D_wrong)


# ---- projection on the internal energies (Sec. IV.C) ---------------------------

def test_projection_holds_the_energy(ora):
    """With the projection, E after every step equals E0 to rounding; without
    it the same run drifts; and the projection lowers every eps_i by the same
    amount (E - E0)/N."""
    from paper_1507_06643_gb300 import inputs
    w = inputs.plain_n1000("fp64")
    spec = w.replicas[0]
    q, p, e = inputs.workload_state(w)
    rep = ora.make_replica(spec.n, spec.box, spec.cv, spec.bricks)
    prm = ora.make_params(w.mass, w.r_cut, w.a, w.sigma, w.seed)
    free = ora.System([rep], prm, q, p, e)
    proj = ora.System([rep], prm, q, p, e)
    proj.set_projection()
    E0 = proj.projection[0]
    drift_free = 0.0
    for _ in range(15):
        free.run(1, 0.02, "HYBRID")
        before = proj.eps.copy()
        pre = ora.System([rep], prm, proj.q, proj.p, proj.eps, step=proj.step)
        pre.F[:] = proj.F
        pre.run(1, 0.02, "HYBRID")
        proj.run(1, 0.02, "HYBRID")
        shift = pre.eps - proj.eps
        assert np.allclose(shift, shift[0], rtol=0, atol=1e-12)
        E_pre = pre.observables()["E"]
        assert shift[0] == pytest.approx((E_pre - E0) / spec.n, rel=1e-9, abs=1e-15)
        assert abs(proj.observables()["E"] - E0) < 1e-11 * abs(E0)
        drift_free = max(drift_free, abs(free.observables()["E"] - E0) / abs(E0))
    assert drift_free > 1e-9
