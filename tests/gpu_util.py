"""Helpers shared by the GPU tests: run the library and the oracle on the same
seeded inputs and measure their differences."""
import numpy as np

from oracle import oracle as O
from paper_1507_06643_gb300 import dpde


def rel_err(a, b):
    den = np.max(np.abs(b)) if b.size else 1.0
    return float(np.max(np.abs(a - b)) / max(den, 1e-300)) if a.size else 0.0


def q_err(qg, qo, boxes, offsets):
    d = qg - qo
    for r in range(len(boxes)):
        s = slice(offsets[r], offsets[r + 1])
        box = np.asarray(boxes[r], float)
        d[s] -= box * np.round(d[s] / box)
    den = np.max(np.abs(qo)) if qo.size else 1.0
    return float(np.max(np.abs(d)) / den) if d.size else 0.0


def make_state(specs, seed, float32):
    """specs: list of (n, box, cv, kT, bricks)."""
    rng = np.random.default_rng(seed)
    qs, ps, es = [], [], []
    for n, box, cv, kT, _ in specs:
        box = np.broadcast_to(np.asarray(box, float), (3,))
        q = rng.random((n, 3)) * box
        p = rng.standard_normal((n, 3)) * np.sqrt(kT)
        if n:
            p -= p.mean(axis=0)
        e = cv * kT * (1 + 0.05 * rng.uniform(-1, 1, n))
        if float32:
            q = q.astype(np.float32).astype(np.float64)
            q = np.where(q >= box, 0.0, q)
            p = p.astype(np.float32).astype(np.float64)
        qs.append(q); ps.append(p); es.append(e)
    return np.concatenate(qs), np.concatenate(ps), np.concatenate(es)


def run_both(specs, precision, scheme, nsteps, dt=0.01, seed=1, a=25.0, sigma=3.0, prm_seed=42,
             use_graph=True, state=None):
    q, p, e = state if state is not None else make_state(specs, seed, precision == "mixed")
    reps = [dpde.make_replica(n, box, cv, br) for n, box, cv, _, br in specs]
    S = dpde.System(dpde.make_params(1.0, 1.0, a, sigma, prm_seed, precision), reps)
    S.set_state(q, p, e)
    S.step(nsteps, dt, scheme, use_graph)
    qg, pg, eg = S.get_state()
    obs_g = S.observables()
    S.close()
    oreps = [O.make_replica(n, box, cv, br) for n, box, cv, _, br in specs]
    ref = O.System(oreps, O.make_params(1.0, 1.0, a, sigma, prm_seed), q, p, e)
    ref.run(nsteps, dt, scheme)
    boxes = [np.broadcast_to(np.asarray(b, float), (3,)) for _, b, _, _, _ in specs]
    errs = {"q": q_err(qg, ref.q, boxes, ref.offsets), "p": rel_err(pg, ref.p),
            "eps": rel_err(eg, ref.eps)}
    return errs, (qg, pg, eg, obs_g), ref
