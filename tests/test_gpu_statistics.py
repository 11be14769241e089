"""Long-run statistical agreement of the library with the oracle.

Over 10^4 steps the two trajectories decorrelate (chaos), so they are
compared as samples of the same equilibrium: the time averages of the
kinetic temperature (Eq. Tkin), the internal temperature (Eq. Tint) and the
configurational temperature (Eq. Tcon, <|grad U|^2> / <Laplacian U>) must
agree within their combined standard errors (block averages). The workload
is the plain N = 1000 fluid (C_v = 100, kT = 1, density 3, Hybrid with 2^3
domains, dt = 0.01).
"""
import math

import numpy as np
import pytest

from gpu_util import make_state

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

STEPS, EVERY, RELAX, BLOCKS = 10000, 10, 500, 20


def _series(step, obs):
    out = {"Tkin": [], "Tint": [], "num": [], "den": []}
    for _ in range(STEPS // EVERY):
        step(EVERY)
        o = obs()
        out["Tkin"].append(o["Tkin"])
        out["Tint"].append(o["Tint"])
        out["num"].append(o["Tpot_num"])
        out["den"].append(o["Tpot_den"])
    return {k: np.asarray(v) for k, v in out.items()}


def _blocks(s):
    """Per block: T_kin, T_int, T_pot = <num>/<den>."""
    nb = len(s["Tkin"]) // BLOCKS
    res = {"Tkin": [], "Tint": [], "Tpot": []}
    for b in range(BLOCKS):
        sl = slice(b * nb, (b + 1) * nb)
        res["Tkin"].append(s["Tkin"][sl].mean())
        res["Tint"].append(s["Tint"][sl].mean())
        res["Tpot"].append(s["num"][sl].mean() / s["den"][sl].mean())
    return {k: (float(np.mean(v)), float(np.std(v, ddof=1) / math.sqrt(BLOCKS))) for k, v in res.items()}


def _state():
    n = 1000
    L = (n / 3.0) ** (1.0 / 3.0)
    specs = [(n, (L, L, L), 100.0, 1.0, (2, 2, 2))]
    return specs, L


@pytest.fixture(scope="module")
def oracle_stats():
    from oracle import oracle as O
    specs, L = _state()
    q, p, e = make_state(specs, 71, False)
    S = O.System([O.make_replica(1000, (L, L, L), 100.0, (2, 2, 2))], O.make_params(seed=17), q, p, e)
    S.run(RELAX, 0.01, "HYBRID")
    return _blocks(_series(lambda k: S.run(k, 0.01, "HYBRID"), lambda: S.observables()))


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_long_run_temperatures_match_oracle(oracle_stats, precision):
    from paper_1507_06643_gb300 import dpde
    specs, L = _state()
    q, p, e = make_state(specs, 71, precision == "mixed")
    S = dpde.System(dpde.make_params(seed=17, precision=precision), [dpde.make_replica(1000, (L, L, L), 100.0,
                                                                                        (2, 2, 2))])
    S.set_state(q, p, e)
    S.step(RELAX, 0.01, "HYBRID")
    got = _blocks(_series(lambda k: S.step(k, 0.01, "HYBRID"), lambda: S.observables(check=True)[0]))
    S.close()
    for key in ("Tkin", "Tint", "Tpot"):
        (mg, sg), (mo, so) = got[key], oracle_stats[key]
        assert abs(mg - mo) < 4.0 * math.hypot(sg, so), (key, got[key], oracle_stats[key])
        assert sg < 0.02 and so < 0.02, (key, sg, so)          # the averages are resolved
    # and each side is in equilibrium: T_kin = T_int within their errors
    for side in (got, oracle_stats):
        assert abs(side["Tkin"][0] - side["Tint"][0]) < 4.0 * math.hypot(side["Tkin"][1], side["Tint"][1]) + 0.01
