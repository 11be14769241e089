"""Pins of the oracle's splined Lennard-Jones potential, Eq. (Ep).

v(r) = 4 eps_LJ((r_LJ/r)^12 - (r_LJ/r)^6) - eps_sh - f_sp (r - r_cut) below
r_cut, eps_sh and f_sp fixed by v(r_cut) = v'(r_cut) = 0. The reference values
come from sympy, which differentiates the textbook 12-6 form and solves the
two conditions for eps_sh and f_sp itself; forces are checked as -grad U by
finite differences, the Laplacian as the divergence of -F, and a noiseless,
frictionless run (sigma = 0) conserves the Hamiltonian energy.
"""
import numpy as np
import pytest

sympy = pytest.importorskip("sympy")

LJ = dict(lj_eps=1.3, lj_r=0.9, r_cut=2.5 * 0.9)


def sympy_potential(eps, rlj, rc):
    r, esh, fsp = sympy.symbols("r esh fsp", real=True)
    vlj = 4 * eps * ((rlj / r) ** 12 - (rlj / r) ** 6)
    v = vlj - esh - fsp * (r - rc)
    sol = sympy.solve([v.subs(r, rc), sympy.diff(v, r).subs(r, rc)], [esh, fsp], dict=True)[0]
    v = v.subs(sol)
    return [sympy.lambdify(r, e, "math") for e in (v, sympy.diff(v, r), sympy.diff(v, r, 2))]


def test_lj_matches_the_textbook_form_and_spline_conditions(ora):
    prm = ora.make_params(potential=ora.POT_LJ, **LJ)
    fv, fdv, fd2v = sympy_potential(LJ["lj_eps"], LJ["lj_r"], LJ["r_cut"])
    for r in np.linspace(0.8, LJ["r_cut"], 23):
        v, dv, d2v = ora.pair_potential(prm, r)
        assert v == pytest.approx(fv(r), rel=1e-12, abs=1e-12)
        assert dv == pytest.approx(fdv(r), rel=1e-12, abs=1e-12)
        assert d2v == pytest.approx(fd2v(r), rel=1e-12, abs=1e-12)
    v, dv, _ = ora.pair_potential(prm, LJ["r_cut"])
    assert abs(v) < 1e-14 and abs(dv) < 1e-13
    # the 12-6 well: v + f_sp r is stationary at r = 2^(1/6) r_LJ
    rm = 2 ** (1 / 6) * LJ["lj_r"]
    _, dv_m, _ = ora.pair_potential(prm, rm)
    assert dv_m == pytest.approx(fdv(rm), rel=1e-12)


def lj_state(cells=3, seed=3):
    from paper_1507_06643_gb300 import inputs
    q, p, e, L = inputs.fcc_state(cells, 0.8095, 1.0, 50.0, 1.0, seed, jitter=0.05)
    return q, p, e, L


def test_lj_forces_are_minus_grad_u(ora):
    prm = ora.make_params(potential=ora.POT_LJ, **LJ)
    q, p, e, L = lj_state()
    rep = ora.make_replica(len(q), (L, L, L), 50.0)
    F = ora.forces(rep, prm, q)

    def U(x):
        return ora.System([rep], prm, x, p, e).observables()["U"]

    h = 1e-6
    for i in (0, 17, 63):
        for d in range(3):
            qp, qm = q.copy(), q.copy()
            qp[i, d] += h
            qm[i, d] -= h
            assert -(U(qp) - U(qm)) / (2 * h) == pytest.approx(F[i, d], rel=1e-6, abs=1e-6)


def test_lj_laplacian_is_the_divergence_of_minus_f(ora):
    prm = ora.make_params(potential=ora.POT_LJ, **LJ)
    q, p, e, L = lj_state()
    rep = ora.make_replica(len(q), (L, L, L), 50.0)
    lap = ora.System([rep], prm, q, p, e).observables()["Tpot_den"]
    h = 1e-5
    div = 0.0
    for i in range(len(q)):
        for d in range(3):
            qp, qm = q.copy(), q.copy()
            qp[i, d] += h
            qm[i, d] -= h
            div -= (ora.forces(rep, prm, qp)[i, d] - ora.forces(rep, prm, qm)[i, d]) / (2 * h)
    assert lap == pytest.approx(div, rel=1e-6)


def test_lj_hamiltonian_run_conserves_energy(ora):
    prm = ora.make_params(sigma=0.0, noise=False, potential=ora.POT_LJ, **LJ)
    q, p, e, L = lj_state(cells=4)
    rep = ora.make_replica(len(q), (L, L, L), 50.0, (1, 1, 1))
    S = ora.System([rep], prm, q, p, e)
    E0 = S.observables()["E"] - S.observables()["Eint"]
    dev = 0.0
    for _ in range(40):
        S.run(10, 0.002, "SER")
        o = S.observables()
        dev = max(dev, abs(o["E"] - o["Eint"] - E0) / abs(E0))
    assert dev < 2e-4
    assert np.array_equal(S.eps, e)          # sigma = 0: the FD part leaves eps untouched
