"""Helpers shared by the GPU tests: run the library and the oracle on the same
seeded inputs and measure their differences.

Decision flips. SSA and Hybrid take discrete decisions from positions: the
cell of a particle fixes the round in which its pairs enter the SSA sequence
and its domain fixes whether a pair goes to SSA or to SER. In the mixed mode
the library takes them from float positions, the oracle from double ones, so
a particle lying within rounding of a cell face can be binned differently.
Such a run is not comparable element by element (the SSA maps do not
commute). ``run_both`` therefore records, at every step, the cell of every
particle on both sides (the library's through dpde_get_cells); tests compare runs without flips strictly
and, where flips are unavoidable (full size), exclude only the particles
within reach of a flipped one.
"""
import numpy as np

from oracle import oracle as O
from paper_1507_06643_gb300 import dpde


def rel_err(a, b):
    den = np.max(np.abs(b)) if b.size else 1.0
    return float(np.max(np.abs(a - b)) / max(den, 1e-300)) if a.size else 0.0


def q_diff(qg, qo, boxes, offsets):
    d = qg - qo
    for r in range(len(boxes)):
        s = slice(offsets[r], offsets[r + 1])
        box = np.asarray(boxes[r], float)
        d[s] -= box * np.round(d[s] / box)
    return d


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


def oracle_cells(q, specs, offsets, r_cut=1.0):
    """The oracle's cell coordinates c_d = min(nc_d - 1, (int)(x * (nc_d / L_d)))."""
    out = np.empty(q.shape, np.int64)
    for r, (n, box, cv, kT, br) in enumerate(specs):
        s = slice(offsets[r], offsets[r + 1])
        rep = O.make_replica(n, box, cv, br)
        nc, _ = O.cell_grid(rep, r_cut)
        for d in range(3):
            x = q[s, d] * (nc[d] / rep.box[d])
            out[s, d] = np.minimum(nc[d] - 1, np.maximum(0, np.trunc(x).astype(np.int64)))
    return out


def run_both(specs, precision, scheme, nsteps, dt=0.01, seed=1, a=25.0, sigma=3.0, prm_seed=42,
             use_graph=True, state=None, r_cut=1.0, pot=None, walls=(0, 0.0)):
    """Runs both sides step by step. Returns (errs, flips, gpu_state, ref) where
    flips is the set of particles whose cell differed between the two sides at
    some step (the per-step decision positions are the end-of-step positions).
    walls = (walls, wall_u) of every replica."""
    q, p, e = state if state is not None else make_state(specs, seed, precision == "mixed")
    reps = [dpde.make_replica(n, box, cv, br, *walls) for n, box, cv, _, br in specs]
    pot = pot or {}
    S = dpde.System(dpde.make_params(1.0, r_cut, a, sigma, prm_seed, precision, **pot), reps)
    S.set_state(q, p, e)
    oreps = [O.make_replica(n, box, cv, br, *walls) for n, box, cv, _, br in specs]
    ref = O.System(oreps, O.make_params(1.0, r_cut, a, sigma, prm_seed, **pot), q, p, e)
    flips = set()
    for _ in range(nsteps):
        S.step(1, dt, scheme, use_graph)
        ref.run(1, dt, scheme)
        bad = np.any(S.get_cells() != oracle_cells(ref.q, specs, ref.offsets, r_cut), axis=1)
        flips.update(np.nonzero(bad)[0].tolist())
    qg, pg, eg = S.get_state()
    obs_g = S.observables()
    S.close()
    boxes = [np.broadcast_to(np.asarray(b, float), (3,)) for _, b, _, _, _ in specs]
    dq = q_diff(qg, ref.q, boxes, ref.offsets)
    # positions relative to the oracle's displacement from the start (minimum
    # image), not to the box: the box scale would hide errors at large L
    moved = q_diff(ref.q, q, boxes, ref.offsets)
    errs = {"q": float(np.max(np.abs(dq)) / max(np.max(np.abs(moved)), 1e-300)) if len(dq) else 0.0,
            "p": rel_err(pg, ref.p), "eps": rel_err(eg, ref.eps)}
    return errs, flips, (qg, pg, eg, obs_g), ref


ORDER_DEPENDENT = ("SSA", "HYBRID")


def assert_parity(specs, precision, scheme, nsteps, tol, seeds, **kw):
    """Strict parity on every run whose discrete decisions agree; runs of an
    order-dependent scheme with a decision flip are skipped (at least one
    run must be comparable)."""
    compared = 0
    for seed in seeds:
        errs, flips, gpu, ref = run_both(specs, precision, scheme, nsteps, seed=seed, **kw)
        if flips and scheme in ORDER_DEPENDENT:
            continue
        assert max(errs.values()) < tol, (seed, errs, len(flips))
        compared += 1
        yield errs, gpu, ref
    assert compared >= 1, "every run had a decision flip"
