"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances: 1e-11 relative in FP64 mode and 2e-5 relative in the mixed mode
(per array: max |x_gpu - x_oracle| / max |x_oracle|, positions compared by
minimum image), trajectory-wise over up to 10 steps. Integer work (noise bits)
is compared bit for bit.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

from gpu_util import assert_parity, make_state, q_diff, rel_err, run_both

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "mixed": 2e-5}
DENSE = 3.0


@pytest.fixture(scope="module", autouse=True)
def cuda():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1507_06643_gb300 import dpde
    dpde.lib()


def cube(n):
    return (n / DENSE) ** (1 / 3)


# ---- noise --------------------------------------------------------------------

def test_device_philox_bit_exact(ora):
    from paper_1507_06643_gb300 import dpde
    rng = np.random.default_rng(0)
    n = 50000
    ctr = rng.integers(0, 2**32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, (n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:3] = 0
    ctr[3:6] = 0xFFFFFFFF
    key[:2] = 0
    assert np.array_equal(dpde.dpde_debug_philox(ctr, key), ora.philox(ctr, key))


def test_oracle_philox_matches_curand(ora):
    rng = np.random.default_rng(1)
    n = 4096
    ctr = rng.integers(0, 2**32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, (n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    key[0] = 0
    here = os.path.dirname(os.path.abspath(__file__))
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "curand_philox")
        subprocess.run(["/usr/local/cuda/bin/nvcc", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-o", exe, os.path.join(here, "curand_philox.cu")], check=True)
        fin, fout = os.path.join(d, "in.bin"), os.path.join(d, "out.bin")
        np.concatenate([ctr.ravel(), key.ravel()]).astype(np.uint32).tofile(fin)
        subprocess.run([exe, fin, fout, str(n)], check=True)
        ref = np.fromfile(fout, dtype=np.uint32).reshape(n, 4)
    assert np.array_equal(ora.philox(ctr, key), ref)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("mixed", 3e-6)])
def test_device_gaussian_matches_oracle(ora, precision, tol):
    from paper_1507_06643_gb300 import dpde
    rng = np.random.default_rng(2)
    n = 100000
    a = rng.integers(0, 2**31, n)
    b = rng.integers(0, 2**31, n)
    step = rng.integers(0, 2**32, n, dtype=np.uint64)
    rep = rng.integers(0, 300, n)
    g = dpde.dpde_debug_gaussian(77, step, rep, a, b, precision)
    o = ora.gaussian(77, step, rep, a, b)
    assert np.max(np.abs(g - o)) < tol


# ---- trajectories ----------------------------------------------------------------

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("scheme", ["SER", "HYBRID", "SEM", "SSA"])
def test_parity_plain_n1000(precision, scheme):
    specs = [(1000, (cube(1000),) * 3, 100.0, 1.0, (2, 2, 2))]
    for _ in assert_parity(specs, precision, scheme, 10, TOL[precision], seeds=range(1001, 1009)):
        break


@pytest.mark.parametrize("n,box,bricks", [
    (1, (4.0, 4.0, 4.0), (1, 1, 1)),
    (2, (3.0, 3.0, 3.0), (1, 1, 1)),
    (64, (3.2, 3.2, 3.2), (1, 1, 1)),
    (777, (5.0, 7.3, 7.1), (1, 2, 3)),
    (3000, (7.0, 10.5, 13.6), (2, 3, 1)),
    (2500, (9.3, 9.3, 9.7), (3, 3, 3)),
    (6000, (12.6, 12.6, 12.6), (1, 1, 1)),   # one domain too large for shared memory
])
@pytest.mark.parametrize("scheme", ["SER", "HYBRID", "SSA"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_parity_sizes(n, box, bricks, scheme, precision):
    specs = [(n, box, 50.0, 1.0, bricks)]
    for _ in assert_parity(specs, precision, scheme, 6, TOL[precision], seeds=range(n, n + 8)):
        break


@pytest.mark.parametrize("scheme", ["SER", "HYBRID", "SEM", "SSA"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_parity_with_an_empty_replica(precision, scheme):
    """A batch with an empty replica between two others: the empty one stays
    empty and the others match the oracle, in every SSA form."""
    from paper_1507_06643_gb300 import dpde
    specs = [(500, (cube(500),) * 3, 50.0, 1.0, (2, 2, 2)), (0, (4.0, 4.0, 4.0), 50.0, 1.0, (1, 1, 1)),
             (700, (cube(700),) * 3, 100.0, 1.5, (1, 1, 1))]
    for _, (qg, pg, eg, obs), _ in assert_parity(specs, precision, scheme, 4, TOL[precision],
                                                 seeds=range(71, 79)):
        assert len(qg) == 1200 and obs[1]["K"] == 0.0 and obs[1]["U"] == 0.0
        break
    if scheme in ("HYBRID", "SSA"):
        q, p, e = make_state(specs, 71, precision == "mixed")
        outs = []
        for mode in (0, 1, 2, 3):
            S = dpde.System(dpde.make_params(precision=precision),
                            [dpde.make_replica(n, box, cv, br) for n, box, cv, _, br in specs])
            S.set_tuning(ssa_mode=mode)
            S.set_state(q, p, e)
            S.step(3, 0.01, scheme)
            assert S.sync() == dpde.DPDE_OK
            outs.append(S.get_state())
            S.close()
        for out in outs[1:]:
            for a, b in zip(outs[0], out):
                assert np.array_equal(a, b)


def test_empty_system_steps_cleanly():
    """A handle with no particles at all: every call succeeds and does nothing."""
    from paper_1507_06643_gb300 import dpde
    S = dpde.System(dpde.make_params(precision="mixed"), [dpde.make_replica(0, 4.0, 50.0, (1, 1, 1))])
    z3, z1 = np.zeros((0, 3)), np.zeros(0)
    S.set_state(z3, z3, z1)
    S.step(3, 0.01, "HYBRID")
    S.step(2, 0.01, "SER", use_graph=False)
    assert S.sync() == dpde.DPDE_OK
    q, p, e = S.get_state()
    assert q.shape == (0, 3) and p.shape == (0, 3) and e.shape == (0,)
    o = S.observables()[0]
    assert o["K"] == 0.0 and o["U"] == 0.0 and o["Eint"] == 0.0
    assert dpde.dpde_get_step(S.h) == 5
    S.close()


# ---- walls along z (the shock set-up's confining walls, Sec. V) ---------------------------

@pytest.mark.parametrize("wall_u", [0.0, -1.5])
@pytest.mark.parametrize("scheme,bricks", [("SER", (1, 1, 1)), ("HYBRID", (2, 2, 3)), ("SSA", (1, 1, 1)),
                                           ("SEM", (1, 1, 1)), ("HYBRID", (1, 1, 1))])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_parity_walls(precision, scheme, bricks, wall_u):
    # a flux into both walls, a piston moving in, 12 steps
    specs = [(1600, (7.0, 7.0, 10.5), 50.0, 1.0, bricks)]
    for errs, gpu, ref in assert_parity(specs, precision, scheme, 12, TOL[precision],
                                        seeds=range(700, 708), walls=(1, wall_u)):
        qg = gpu[0]
        zw = 10.5 + wall_u * 12 * 0.01
        assert np.all(qg[:, 2] >= 0.0) and np.all(qg[:, 2] <= zw + 1e-6)
        break


def test_walled_replicas_beside_periodic_ones():
    # one launch over a walled and a periodic replica: each matches its own oracle run
    from paper_1507_06643_gb300 import dpde
    from oracle import oracle as O
    specs = [(900, (6.5, 6.5, 7.2), 50.0, 1.0, (1, 1, 2)), (700, (6.0, 6.0, 6.4), 50.0, 1.0, (1, 1, 1))]
    q, p, e = make_state(specs, 55, True)
    reps = [dpde.make_replica(900, (6.5, 6.5, 7.2), 50.0, (1, 1, 2), 1, -0.5),
            dpde.make_replica(700, (6.0, 6.0, 6.4), 50.0, (1, 1, 1))]
    S = dpde.System(dpde.make_params(precision="fp64", seed=9), reps)
    S.set_state(q, p, e)
    S.step(8, 0.01, "HYBRID")
    qg, pg, eg = S.get_state()
    S.close()
    oreps = [O.make_replica(900, (6.5, 6.5, 7.2), 50.0, (1, 1, 2), 1, -0.5),
             O.make_replica(700, (6.0, 6.0, 6.4), 50.0, (1, 1, 1))]
    ref = O.System(oreps, O.make_params(seed=9), q, p, e)
    ref.run(8, 0.01, "HYBRID")
    assert rel_err(pg, ref.p) < 1e-11 and rel_err(eg, ref.eps) < 1e-11


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_walled_ssa_forms_agree_bit_for_bit(precision):
    # non-periodic z colours in both SSA forms; bricks one and several along z
    from paper_1507_06643_gb300 import dpde
    specs = [(1500, (7.0, 7.0, 10.3), 50.0, 1.0, (1, 1, 3)), (800, (5.5, 5.5, 9.1), 50.0, 1.0, (1, 1, 1))]
    q, p, e = make_state(specs, 64, precision == "mixed")
    outs = []
    for mode in (0, 1, 2, 3):
        S = dpde.System(dpde.make_params(precision=precision),
                        [dpde.make_replica(n, box, cv, br, 1, -0.7) for n, box, cv, _, br in specs])
        S.set_tuning(ssa_mode=mode)
        S.set_state(q, p, e)
        S.step(6, 0.01, "HYBRID")
        outs.append(S.get_state())
        S.close()
    for out in outs[1:]:
        for a, b in zip(outs[0], out):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_state_through_device_pointers_equals_host_path(precision):
    # set_state / get_state with torch CUDA tensors (on_device = 1) and with
    # host arrays give the same state bit for bit, after steps too
    torch = pytest.importorskip("torch")
    from paper_1507_06643_gb300 import dpde
    specs = [(3000, (cube(3000),) * 3, 50.0, 1.0, (2, 2, 2)), (1200, (cube(1200),) * 3, 80.0, 1.0, (1, 1, 1))]
    q, p, e = make_state(specs, 71, precision == "mixed")
    reps = [dpde.make_replica(n, box, cv, br) for n, box, cv, _, br in specs]
    A = dpde.System(dpde.make_params(precision=precision), reps)
    A.set_state(q, p, e)
    B = dpde.System(dpde.make_params(precision=precision), reps)
    qd, pd, ed = (torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (q, p, e))
    torch.cuda.synchronize()
    B.set_state(qd, pd, ed, on_device=True)
    for S in (A, B):
        S.step(3, 0.01, "HYBRID")
    qa, pa, ea = A.get_state()
    qo, po, eo = (torch.empty_like(x) for x in (qd, pd, ed))
    torch.cuda.synchronize()
    assert dpde.dpde_get_state(B.h, qo, po, eo, True) == dpde.DPDE_OK
    torch.cuda.synchronize()
    for a, b in ((qa, qo), (pa, po), (ea, eo)):
        assert np.array_equal(a, b.cpu().numpy())
    A.close()
    B.close()


def test_piston_overrun_and_bad_walls_reported():
    from paper_1507_06643_gb300 import dpde
    # a sparse fluid (no neighbour-list overflow while it is squeezed)
    rep = dpde.make_replica(60, (4.0, 4.0, 4.0), 50.0, walls=1, wall_u=-20.0)
    q, p, e = make_state([(60, (4.0, 4.0, 4.0), 50.0, 1.0, (1, 1, 1))], 3, False)
    S = dpde.System(dpde.make_params(precision="fp64"), [rep])
    S.set_state(q, p, e)
    S.step(10, 0.01, "SER")              # z_w = 4 - 0.2 (n + 1) > 1: still fine
    assert S.sync() == dpde.DPDE_OK
    S.step(10, 0.01, "SER")              # the wall passes z = ell_z = 1 at n = 15
    assert S.sync() == dpde.DPDE_ERR_ARG
    S.close()
    for w, u in ((2, 0.0), (1, 0.5)):
        with pytest.raises(dpde.DPDEError):
            dpde.System(dpde.make_params(), [dpde.make_replica(300, (4.0, 4.0, 4.0), 50.0, walls=w, wall_u=u)])


def slab_state(seed, L=12.0, rho=3.0, rho_slab=9.0, slab=4.0, float32=False):
    """Uniform fluid at rho with a slab z < `slab` at rho_slab: cells there
    hold ~3x the mean, so SSA chains overflow the per-cell row table and the
    per-block Gaussian staging."""
    rng = np.random.default_rng(seed)
    n0 = int(rho * L ** 3)
    n1 = int((rho_slab - rho) * L * L * slab)
    q = np.concatenate([rng.random((n0, 3)) * L, rng.random((n1, 3)) * np.array([L, L, slab])])
    n = len(q)
    p = rng.standard_normal((n, 3))
    p -= p.mean(axis=0)
    e = 50.0 * (1 + 0.05 * rng.uniform(-1, 1, n))
    if float32:
        q = q.astype(np.float32).astype(np.float64)
        q = np.where(q >= L, 0.0, q)
        p = p.astype(np.float32).astype(np.float64)
    return q, p, e


@pytest.mark.parametrize("bricks", [(1, 1, 1), (2, 2, 2)])
@pytest.mark.parametrize("scheme", ["HYBRID", "SSA"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_parity_dense_slab(precision, scheme, bricks):
    compared = 0
    for seed in range(31, 39):
        state = slab_state(seed, float32=precision == "mixed")
        specs = [(len(state[0]), (12.0, 12.0, 12.0), 50.0, 1.0, bricks)]
        errs, flips, _, _ = run_both(specs, precision, scheme, 4, state=state)
        if flips:
            continue
        assert max(errs.values()) < TOL[precision], (seed, errs)
        compared += 1
        if compared == 2:
            break
    assert compared >= 1


def test_parity_tiles_beyond_the_dense_capacity():
    """Tile edge 2 and a slab at 2.9x the mean density: slab tiles overflow
    both the regular and the dense halo capacity and take the global path."""
    from oracle import oracle as O
    from paper_1507_06643_gb300 import dpde
    q, p, e = slab_state(5, L=24.0, rho=3.0, rho_slab=14.0, slab=4.0)
    n, box = len(q), (24.0, 24.0, 24.0)
    S = dpde.System(dpde.make_params(precision="fp64", seed=42), [dpde.make_replica(n, box, 50.0, (2, 2, 2))])
    S.set_tuning(tile_edge=2)
    S.set_state(q, p, e)
    S.step(2, 0.01, "HYBRID")
    qg, pg, eg = S.get_state()
    S.close()
    ref = O.System([O.make_replica(n, box, 50.0, (2, 2, 2))], O.make_params(seed=42), q, p, e)
    ref.run(2, 0.01, "HYBRID")
    assert rel_err(pg, ref.p) < TOL["fp64"] and rel_err(eg, ref.eps) < TOL["fp64"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("scheme", ["SER", "HYBRID", "SSA"])
def test_parity_batched_replicas(precision, scheme):
    rng = np.random.default_rng(5)
    specs = []
    for r in range(7):
        n = int(np.exp(rng.uniform(np.log(200), np.log(4000))))
        L = cube(n)
        b = 2 if L >= 6 else 1
        specs.append((n, (L, L, L), float(rng.choice([10.0, 50.0, 100.0])),
                      float(rng.uniform(0.5, 2.0)), (b, b, b)))
    for errs, (qg, pg, eg, obs), ref in assert_parity(specs, precision, scheme, 5, TOL[precision],
                                                      seeds=range(55, 63)):
        break
    tol = TOL[precision] * 10
    for r in range(len(specs)):
        o = ref.observables(r)
        for k in ("K", "U", "Eint", "Tkin", "Tint", "Tpot_num", "Tpot_den"):
            assert abs(obs[r][k] - o[k]) <= tol * max(1.0, abs(o[k])), (r, k, obs[r][k], o[k])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_observables_match_oracle(precision):
    specs = [(1000, (cube(1000),) * 3, 100.0, 1.0, (2, 2, 2))]
    for errs, (_, _, _, obs), ref in assert_parity(specs, precision, "HYBRID", 3, TOL[precision],
                                                   seeds=range(9, 17)):
        break
    o = ref.observables(0)
    tol = 1e-10 if precision == "fp64" else 1e-5
    for k in ("E", "K", "U", "Eint", "Tkin", "Tint", "Tpot_num", "Tpot_den"):
        assert abs(obs[0][k] - o[k]) <= tol * abs(o[k]), (k, obs[0][k], o[k])
    # total momentum: exact in FP64; float rounding of each p_i in the mixed mode
    ptol = 1e-9 if precision == "fp64" else 1e-4
    for k in ("Px", "Py", "Pz"):
        assert abs(obs[0][k] - o[k]) < ptol


# ---- determinism, resume, graphs ----------------------------------------------

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("scheme", ["SER", "HYBRID", "SEM", "SSA"])
def test_checkpoint_restart_and_graph_are_bit_exact(precision, scheme):
    """10 steps as one graph-replayed run == 4 eager steps, a raw checkpoint
    restored into a fresh handle, and 6 more graph steps (bit for bit); a
    restart through absolute coordinates (get_state/set_state) agrees to
    rounding."""
    from paper_1507_06643_gb300 import dpde
    specs = [(3000, (cube(3000),) * 3, 100.0, 1.0, (2, 2, 2))]
    q, p, e = make_state(specs, 3, precision == "mixed")
    rep = [dpde.make_replica(3000, (cube(3000),) * 3, 100.0, (2, 2, 2))]
    prm = dpde.make_params(seed=9, precision=precision)
    A = dpde.System(prm, rep)
    A.set_state(q, p, e)
    A.step(10, 0.01, scheme, use_graph=True)
    a = A.get_state()
    B = dpde.System(prm, rep)
    B.set_state(q, p, e)
    B.step(4, 0.01, scheme, use_graph=False)
    blob = B.checkpoint()
    mid = B.get_state()
    obs_mid = B.observables()[0]
    C = dpde.System(prm, rep)
    C.restore(blob)
    assert C.observables()[0] == obs_mid          # a fresh handle: cell starts rebuilt
    C.step(6, 0.01, scheme, use_graph=True)
    for x, y in zip(a, C.get_state()):
        assert np.array_equal(x, y)
    C.restore(blob)                                 # a stepped handle: stale cell starts replaced
    assert C.observables()[0] == obs_mid
    D = dpde.System(prm, rep)
    D.set_state(*mid, step=4)
    D.step(6, 0.01, scheme, use_graph=True)
    tol = 1e-9 if precision == "fp64" else 1e-3
    for x, y in zip(a, D.get_state()):
        assert np.max(np.abs(x - y)) / np.max(np.abs(x)) < tol
    for S in (A, B, C, D):
        S.close()


def test_restore_rejects_a_foreign_checkpoint():
    from paper_1507_06643_gb300 import dpde
    rep = [dpde.make_replica(500, (cube(500),) * 3, 100.0)]
    A = dpde.System(dpde.make_params(seed=1, precision="mixed"), rep)
    q, p, e = make_state([(500, (cube(500),) * 3, 100.0, 1.0, (1, 1, 1))], 1, True)
    A.set_state(q, p, e)
    blob = A.checkpoint()
    B = dpde.System(dpde.make_params(seed=2, precision="mixed"), rep)
    with pytest.raises(dpde.DPDEError) as ei:
        B.restore(blob)
    assert ei.value.code == dpde.DPDE_ERR_ARG
    A.close()
    B.close()


def test_momentum_is_conserved():
    from paper_1507_06643_gb300 import dpde
    specs = [(20000, (cube(20000),) * 3, 100.0, 1.0, (3, 3, 3))]
    q, p, e = make_state(specs, 4, False)
    S = dpde.System(dpde.make_params(precision="fp64"), [dpde.make_replica(*specs[0][:3], (3, 3, 3))])
    S.set_state(q, p, e)
    P0 = S.observables()[0]
    S.step(50, 0.01, "HYBRID")
    P1 = S.observables()[0]
    for k in ("Px", "Py", "Pz"):
        assert abs(P1[k] - P0[k]) < 1e-9


@pytest.mark.parametrize("box,bricks", [((6.93, 6.93, 6.93), (2, 2, 2)), ((5.0, 7.3, 7.1), (1, 2, 3)),
                                        ((7.0, 10.5, 13.6), (2, 3, 1))])
def test_ssa_launches_follow_colour_classes(box, bricks):
    """One SSA launch per non-empty colour class: P = 3, 3, 2 colours along
    x, y, z, plus one per leftover cell (k mod P) along a periodic domain
    axis."""
    from paper_1507_06643_gb300 import dpde
    n = int(DENSE * np.prod(box))
    S = dpde.System(dpde.make_params(precision="mixed"), [dpde.make_replica(n, box, 50.0, bricks)])

    def classes(whole):
        out = 1
        for d, P in enumerate((3, 3, 2)):
            nc = bricks[d] * int(np.floor(box[d] / bricks[d]))
            k = nc if whole else nc // bricks[d]
            periodic = whole or bricks[d] == 1
            out *= min(P, k) + (k % P if periodic and k >= P else 0)
        return out

    S.set_tuning(ssa_mode=0)
    ser, hyb, ssa = (S.step_launches(x) for x in ("SER", "HYBRID", "SSA"))
    assert hyb - ser == classes(False) + 1     # + the Gaussian pass
    assert ssa - (ser - 1) == classes(True) + 1   # SSA: one copy-back in place of the two sweeps
    # per-domain form: one launch for every class of every domain; DPDE_SSA unchanged
    S.set_tuning(ssa_mode=1)
    assert S.step_launches("HYBRID") - ser == 2
    assert S.step_launches("SSA") == ssa
    # level form: three schedule launches (the regular one and two for deferred
    # domains) and five execution launches (the regular one, two for the
    # domains it defers, two for those the schedule deferred), for bricks and
    # whole replicas
    S.set_tuning(ssa_mode=2)
    assert S.step_launches("HYBRID") - ser == 8
    assert S.step_launches("SSA") - (ser - 1) == 8
    # persistent form: the Gaussian pass and one cooperative launch over all classes
    S.set_tuning(ssa_mode=3)
    assert S.step_launches("HYBRID") - ser == 2
    assert S.step_launches("SSA") - (ser - 1) == 2
    S.close()


# ---- splined Lennard-Jones potential, Eq. (Ep) -----------------------------------------

LJ_POT = {"potential": 1, "lj_eps": 1.0, "lj_r": 1.0}


def lj_case(cells, seed, precision):
    from paper_1507_06643_gb300 import inputs
    q, p, e, L = inputs.fcc_state(cells, 0.8095, 1.0, 50.0, 1.0, seed)
    if precision == "mixed":
        q = q.astype(np.float32).astype(np.float64)
        q = np.where(q >= L, 0.0, q)
        p = p.astype(np.float32).astype(np.float64)
    return (q, p, e), L


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("scheme,bricks", [("SER", (1, 1, 1)), ("HYBRID", (2, 2, 2)), ("SSA", (1, 1, 1)),
                                           ("SEM", (1, 1, 1))])
def test_parity_lennard_jones(precision, scheme, bricks):
    """An FCC crystal at the paper's density 0.8095 (8^3 cells, 2048
    particles, r_cut = 2.5 r_LJ, sigma = 4), 10 steps of dt = 0.002."""
    compared = 0
    for seed in range(61, 69):
        state, L = lj_case(8, seed, precision)
        specs = [(len(state[0]), (L, L, L), 50.0, 1.0, bricks)]
        errs, flips, (_, _, _, obs), ref = run_both(specs, precision, scheme, 10, dt=0.002, sigma=4.0,
                                                   state=state, r_cut=2.5, pot=LJ_POT)
        if flips and scheme in ("SSA", "HYBRID"):
            continue
        assert max(errs.values()) < TOL[precision], (seed, errs)
        o = ref.observables(0)
        for k in ("U", "Tpot_num", "Tpot_den"):
            assert abs(obs[0][k] - o[k]) <= 10 * TOL[precision] * max(1.0, abs(o[k])), (k, obs[0][k], o[k])
        compared += 1
        if compared == 2:
            break
    assert compared >= 1


def test_lj_rejects_bad_parameters():
    from paper_1507_06643_gb300 import dpde
    rep = [dpde.make_replica(500, (12.0, 12.0, 12.0), 50.0)]
    for kw in ({"potential": 2}, {"potential": 1, "lj_r": 0.0}, {"potential": 1, "lj_eps": -1.0}):
        with pytest.raises(dpde.DPDEError):
            dpde.System(dpde.make_params(r_cut=2.5, **kw), rep)


# ---- projection on the internal energies (Sec. IV.C) ----------------------------------

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("scheme", ["HYBRID", "SER"])
def test_parity_with_projection(precision, scheme):
    """Projected steps against the projected oracle, both from the oracle's E0."""
    from oracle import oracle as O
    from paper_1507_06643_gb300 import dpde
    from gpu_util import oracle_cells
    specs = [(1000, (cube(1000),) * 3, 100.0, 1.0, (2, 2, 2))]
    compared = 0
    for seed in range(41, 49):
        q, p, e = make_state(specs, seed, precision == "mixed")
        S = dpde.System(dpde.make_params(1.0, 1.0, 25.0, 3.0, 42, precision),
                        [dpde.make_replica(1000, specs[0][1], 100.0, (2, 2, 2))])
        S.set_state(q, p, e)
        ref = O.System([O.make_replica(1000, specs[0][1], 100.0, (2, 2, 2))], O.make_params(1.0, 1.0, 25.0, 3.0, 42),
                       q, p, e)
        ref.set_projection()
        S.set_projection(True, ref.projection)
        flips = False
        for _ in range(8):
            S.step(1, 0.01, scheme)
            ref.run(1, 0.01, scheme)
            flips |= bool(np.any(S.get_cells() != oracle_cells(ref.q, specs, ref.offsets)))
        qg, pg, eg = S.get_state()
        S.close()
        if flips and scheme == "HYBRID":
            continue
        tol = TOL[precision]
        assert rel_err(pg, ref.p) < tol and rel_err(eg, ref.eps) < tol, seed
        compared += 1
        if compared == 2:
            break
    assert compared >= 1


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 2e-7)])
def test_projection_holds_the_energy(precision, tol):
    from paper_1507_06643_gb300 import dpde
    specs = [(20000, (cube(20000),) * 3, 50.0, 1.0, (3, 3, 3))]
    q, p, e = make_state(specs, 12, precision == "mixed")
    S = dpde.System(dpde.make_params(precision=precision), [dpde.make_replica(*specs[0][:3], (3, 3, 3))])
    S.set_state(q, p, e)
    S.step(20, 0.01, "HYBRID")
    E0 = S.observables()[0]["E"]
    S.set_projection()
    S.step(50, 0.01, "HYBRID")
    assert abs(S.observables()[0]["E"] - E0) < tol * abs(E0)
    S.set_projection(False)
    S.step(50, 0.01, "HYBRID")
    assert abs(S.observables()[0]["E"] - E0) > tol * abs(E0)
    S.close()


def test_step_profiled_reports_each_phase():
    from paper_1507_06643_gb300 import dpde
    specs = [(20000, (cube(20000),) * 3, 50.0, 1.0, (3, 3, 3))]
    q, p, e = make_state(specs, 3, True)
    S = dpde.System(dpde.make_params(precision="mixed"), [dpde.make_replica(*specs[0][:3], (3, 3, 3))])
    S.set_state(q, p, e)
    ph = S.step_profiled(2, 0.01, "HYBRID")
    assert set(ph) == set(dpde.PHASES)
    for k in ("kick_drift", "scan", "gather", "force", "ssa", "ssa_gauss", "sweep1", "sweep2"):
        assert ph[k] > 0, k
    assert ph["other"] == 0          # no projection
    assert dpde.dpde_get_step(S.h) == 2
    S.close()


# ---- tuning -------------------------------------------------------------------------

def _run_tuned(precision, tuning, steps=5, scheme="HYBRID"):
    from paper_1507_06643_gb300 import dpde
    specs = [(3000, (cube(3000),) * 3, 50.0, 1.0, (2, 2, 2))]
    q, p, e = make_state(specs, 77, precision == "mixed")
    S = dpde.System(dpde.make_params(precision=precision), [dpde.make_replica(*specs[0][:3], (2, 2, 2))])
    if tuning:
        S.set_tuning(**tuning)
    S.set_state(q, p, e)
    S.step(steps, 0.01, scheme)
    out = S.get_state()
    S.close()
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_block_sizes_do_not_change_results(precision):
    ref = _run_tuned(precision, None)
    for t in ({"block": 128, "ssa_block": 32}, {"block": 512, "ssa_block": 128}, {"block": 64, "ssa_block": 96}):
        got = _run_tuned(precision, t)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b), t


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("scheme", ["HYBRID", "SSA"])
def test_ssa_modes_agree_bit_for_bit(precision, scheme):
    # the per-domain launch (mode 1) and the per-class launches (mode 0) apply the same sequence
    ref = _run_tuned(precision, {"ssa_mode": 0}, scheme=scheme)
    for t in ({"ssa_mode": 1}, {"ssa_mode": 1, "ssa_block": 32}, {"ssa_mode": 1, "ssa_block": 128},
              {"ssa_mode": 1, "ssa_group": 1}, {"ssa_mode": 1, "ssa_group": 3},
              {"ssa_mode": 1, "ssa_group": 8, "ssa_block": 96},
              {"ssa_mode": 2}, {"ssa_mode": 2, "ssa_block": 32}, {"ssa_mode": 2, "ssa_block": 128},
              {"ssa_mode": 3}, {"ssa_mode": 3, "ssa_block": 32}, {"ssa_mode": 3, "ssa_block": 128}):
        got = _run_tuned(precision, t, scheme=scheme)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b), t


@pytest.mark.parametrize("scheme", ["HYBRID", "SSA"])
def test_ssa_modes_agree_on_thin_and_batched_boxes(scheme):
    # three cells along an axis (the +2 and -1 offsets name the same cell), bricks two cells
    # thick, and replicas of different sizes in one launch
    from paper_1507_06643_gb300 import dpde
    specs = [(1200, (3.2, 3.2, 38.0), 60.0, 1.0, (1, 1, 4)),
             (900, (cube(900),) * 3, 40.0, 1.0, (2, 1, 3)),
             (2000, (4.1, 9.0, 16.5), 80.0, 1.0, (1, 3, 1))]
    q, p, e = make_state(specs, 91, True)
    outs = []
    for mode, group in ((0, 0), (1, 0), (1, 2), (1, 5), (2, 0), (3, 0)):
        S = dpde.System(dpde.make_params(precision="mixed"),
                        [dpde.make_replica(n, box, cv, br) for n, box, cv, _, br in specs])
        S.set_tuning(ssa_mode=mode, ssa_group=group)
        S.set_state(q, p, e)
        S.step(4, 0.01, scheme)
        outs.append(S.get_state())
        assert S.tuning()["ssa_mode"] == mode
        S.close()
    for out in outs[1:]:
        for a, b in zip(outs[0], out):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["dense_brick", "denser_brick", "densest_brick", "global_state", "no_schedule",
                                  "beyond_level_form"])
def test_ssa_level_form_fallbacks_agree_bit_for_bit(precision, case):
    """The level form's paths beyond its regular shared-memory capacities give
    the colour order's bits: a brick holding more particles than the regular
    execution stages (deferred to the launch with ~2.5x the capacity), one
    denser still (both kernels deferred once), one beyond 2.5x the mean
    (both deferred to the largest tier); one domain too large for any
    staging (levels run on the state in global memory); one domain with more
    forward entries than a schedule holds (run class by class along the
    colour order); one domain above the 16,384 particles the level form
    takes at all (ssa_mode 2 then runs the colour classes, launch for
    launch)."""
    from paper_1507_06643_gb300 import dpde
    rng = np.random.default_rng(41)
    if case in ("dense_brick", "denser_brick", "densest_brick"):
        n0, L, bricks = 4000, cube(4000), (2, 2, 2)
        q, p, e = make_state([(n0, (L,) * 3, 50.0, 1.0, bricks)], 42, precision == "mixed")
        extra_n, half = {"dense_brick": (300, 2.0), "denser_brick": (1000, 0.49 * L / 2),
                         "densest_brick": (1600, 0.49 * L / 2)}[case]
        extra = 0.25 * L + rng.uniform(-half, half, (extra_n, 3))   # inside brick (0, 0, 0)
        q = np.vstack([q, extra])
        p = np.vstack([p, rng.standard_normal((extra_n, 3))])
        e = np.concatenate([e, 50.0 * (1 + 0.05 * rng.uniform(-1, 1, extra_n))])
        if precision == "mixed":
            q = q.astype(np.float32).astype(np.float64)
            p = p.astype(np.float32).astype(np.float64)
        n = n0 + extra_n
    else:
        n = {"global_state": 8000, "no_schedule": 15000, "beyond_level_form": 20000}[case]
        L, bricks = cube(n), (1, 1, 1)
        q, p, e = make_state([(n, (L,) * 3, 50.0, 1.0, bricks)], 43, precision == "mixed")
    outs, launches = [], []
    for mode in (0, 2):
        S = dpde.System(dpde.make_params(precision=precision), [dpde.make_replica(n, (L,) * 3, 50.0, bricks)])
        S.set_tuning(ssa_mode=mode)
        S.set_state(q, p, e)
        S.step(3, 0.01, "HYBRID")
        assert S.sync() == dpde.DPDE_OK
        outs.append(S.get_state())
        launches.append(S.step_launches("HYBRID"))
        S.close()
    if case == "beyond_level_form":
        assert launches[0] == launches[1]
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ssa_two_streams_agree_with_one(precision):
    """An uneven batch whose large domains the level form defers: a brick
    grid of 500-particle domains, single-domain replicas of 3000 and 1500
    particles (deferred by the regular schedule, so scheduled and executed on
    the second stream beside the regular execution) and one of 1100 (kept by
    the regular schedule, deferred by the regular execution). The graph
    (two streams), eager launches (two streams) and the profiled step (one
    stream, phase by phase) give the colour order's bits."""
    from paper_1507_06643_gb300 import dpde
    specs = [(4000, (cube(4000),) * 3, 50.0, 1.0, (2, 2, 2)), (3000, (cube(3000),) * 3, 50.0, 1.5, (1, 1, 1)),
             (1500, (cube(1500),) * 3, 100.0, 0.7, (1, 1, 1)), (1100, (cube(1100),) * 3, 10.0, 1.2, (1, 1, 1))]
    q, p, e = make_state(specs, 51, precision == "mixed")

    def run(mode, how):
        S = dpde.System(dpde.make_params(precision=precision),
                        [dpde.make_replica(n, box, cv, br) for n, box, cv, _, br in specs])
        S.set_tuning(ssa_mode=mode)
        S.set_state(q, p, e)
        if how == "graph":
            S.step(3, 0.01, "HYBRID")
        elif how == "eager":
            S.step(3, 0.01, "HYBRID", use_graph=False)
        else:
            S.step_profiled(3, 0.01, "HYBRID")
        assert S.sync() == dpde.DPDE_OK
        out = S.get_state()
        S.close()
        return out

    ref = run(0, "graph")
    for how in ("graph", "eager", "profiled"):
        for a, b in zip(ref, run(2, how)):
            assert np.array_equal(a, b), how


@pytest.mark.parametrize("edge", [2, 4, 5, 8])
def test_tile_edge_changes_rounding_only(edge):
    ref = _run_tuned("fp64", None)
    got = _run_tuned("fp64", {"tile_edge": edge})
    assert rel_err(got[1], ref[1]) < 1e-12 and rel_err(got[2], ref[2]) < 1e-12


def test_autotune_keeps_the_state():
    from paper_1507_06643_gb300 import dpde
    specs = [(20000, (cube(20000),) * 3, 50.0, 1.0, (3, 3, 3))]
    q, p, e = make_state(specs, 8, True)
    S = dpde.System(dpde.make_params(precision="mixed"), [dpde.make_replica(*specs[0][:3], (3, 3, 3))])
    S.set_state(q, p, e)
    S.step(2, 0.01, "HYBRID")
    before = S.get_state()
    obs_before = S.observables()[0]
    step0 = dpde.dpde_get_step(S.h)
    t = S.autotune("HYBRID", 0.01, 2)
    assert t["tile_edge"] in (4, 5, 6, 7, 8) and t["block"] in (128, 256, 512)
    assert t["ssa_block"] in (32, 64, 128) and t["ssa_mode"] in (0, 1, 2, 3) and t["ms_per_step"] > 0
    assert 1 <= t["ssa_group"] <= 8
    assert S.tuning()["tile_edge"] == t["tile_edge"]
    after = S.get_state()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    assert dpde.dpde_get_step(S.h) == step0
    assert S.observables()[0] == obs_before
    # stepping on continues like an untuned handle switched to the same tile edge
    S.step(2, 0.01, "HYBRID")
    got = S.get_state()
    R = dpde.System(dpde.make_params(precision="mixed"), [dpde.make_replica(*specs[0][:3], (3, 3, 3))])
    R.set_state(q, p, e)
    R.step(2, 0.01, "HYBRID")
    R.set_tuning(tile_edge=t["tile_edge"])
    R.step(2, 0.01, "HYBRID")
    for a, b in zip(got, R.get_state()):
        assert np.array_equal(a, b)
    S.close()
    R.close()


def test_bad_tuning_rejected():
    from paper_1507_06643_gb300 import dpde
    S = dpde.System(dpde.make_params(precision="mixed"), [dpde.make_replica(300, (cube(300),) * 3, 50.0)])
    for kw in ({"tile_edge": 1}, {"tile_edge": 9}, {"block": 48}, {"block": 2048}, {"ssa_block": 256},
               {"ssa_block": 48}, {"ssa_mode": 4}, {"ssa_mode": -1}, {"ssa_group": 9}, {"ssa_group": -1}):
        with pytest.raises(dpde.DPDEError):
            S.set_tuning(**kw)
    S.close()


# ---- errors -------------------------------------------------------------------------

def test_negative_and_nonfinite_state_reported():
    from paper_1507_06643_gb300 import dpde
    specs = [(500, (cube(500),) * 3, 100.0, 1.0, (1, 1, 1))]
    q, p, e = make_state(specs, 6, False)
    S = dpde.System(dpde.make_params(precision="fp64"), [dpde.make_replica(500, (cube(500),) * 3, 100.0)])
    e2 = e.copy()
    e2[17] = -1.0
    with pytest.raises(dpde.DPDEError) as ei:
        S.set_state(q, p, e2)
    assert ei.value.code == dpde.DPDE_ERR_NEG_EPS
    p2 = p.copy()
    p2[3, 1] = np.nan
    with pytest.raises(dpde.DPDEError) as ei:
        S.set_state(q, p2, e)
    assert ei.value.code == dpde.DPDE_ERR_NONFINITE
    S.set_state(q, p, e)     # a clean state clears the condition
    S.step(2, 0.01, "SER")
    assert S.sync() == dpde.DPDE_OK
    S.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("scheme", ["SER", "HYBRID", "SSA"])
def test_neighbour_list_overflow_reported(precision, scheme):
    """A host-built dense cluster -- 150 particles within 0.25 of one point in
    a fluid at density 3 -- gives each of them ~150 neighbours, beyond the list
    capacity (3 x the mean count + 32, ~70 at density 3). The step completes
    with the lists truncated (no write past them) and dpde_sync reports
    DPDE_ERR_CAPACITY; after a clean state the condition is gone."""
    from paper_1507_06643_gb300 import dpde
    n = 1500
    L = cube(n)
    specs = [(n, (L,) * 3, 100.0, 1.0, (2, 2, 2))]
    q, p, e = make_state(specs, 31, precision == "mixed")
    rng = np.random.default_rng(32)
    q2 = q.copy()
    q2[:150] = 0.5 * L + rng.uniform(-0.25, 0.25, (150, 3))
    S = dpde.System(dpde.make_params(precision=precision), [dpde.make_replica(n, (L,) * 3, 100.0, (2, 2, 2))])
    S.set_state(q2, p, e)
    S.step(1, 0.01, scheme)
    assert S.sync() == dpde.DPDE_ERR_CAPACITY
    assert "capacity" in dpde.lib().dpde_last_error(S.h).decode()
    S.set_state(q, p, e)
    S.step(2, 0.01, scheme)
    assert S.sync() == dpde.DPDE_OK
    S.close()


@pytest.mark.parametrize("scheme", ["SSA", "HYBRID"])
def test_persistent_ssa_barrier_timeout_reported(scheme):
    """The persistent SSA launch (ssa_mode 3) bounds the wait of its grid
    barriers: with a wait budget of 0 cycles every block that reaches a
    barrier before the last one gives up at once, the launch ends, and
    dpde_sync reports DPDE_ERR_TIMEOUT; the context stays usable, and with
    the default budget restored the same steps run clean."""
    from paper_1507_06643_gb300 import dpde
    n = 20000
    L = cube(n)
    specs = [(n, (L,) * 3, 50.0, 1.0, (2, 2, 2))]
    q, p, e = make_state(specs, 33, True)
    S = dpde.System(dpde.make_params(precision="mixed"), [dpde.make_replica(n, (L,) * 3, 50.0, (2, 2, 2))])
    S.set_tuning(ssa_mode=3)
    S.set_state(q, p, e)
    dpde.dpde_set_wait_budget(S.h, 0)
    S.step(1, 0.01, scheme)
    assert S.sync() == dpde.DPDE_ERR_TIMEOUT
    assert "budget" in dpde.lib().dpde_last_error(S.h).decode()
    with pytest.raises(dpde.DPDEError):
        dpde.dpde_set_wait_budget(S.h, -1)
    dpde.dpde_set_wait_budget(S.h, 2_000_000_000)
    S.set_state(q, p, e)
    S.step(3, 0.01, scheme)
    assert S.sync() == dpde.DPDE_OK
    got = S.get_state()
    S.close()
    R = dpde.System(dpde.make_params(precision="mixed"), [dpde.make_replica(n, (L,) * 3, 50.0, (2, 2, 2))])
    R.set_tuning(ssa_mode=0)
    R.set_state(q, p, e)
    R.step(3, 0.01, scheme)
    for a, b in zip(got, R.get_state()):
        assert np.array_equal(a, b)
    R.close()


# ---- the benchmark's workload at full size ------------------------------------------

@pytest.mark.parametrize("precision,scheme", [("mixed", "HYBRID"), ("mixed", "SER"), ("fp64", "HYBRID")])
def test_full_size_large_n4m_one_step(precision, scheme):
    """The benchmark's workload (4M particles) in the benchmark's launch
    configuration, one step, element by element against the oracle. In the
    mixed Hybrid run some particles sit within float rounding of a cell face;
    particles within 2 r_cut of such a flip are excluded (they must be < 1%)."""
    from scipy.spatial import cKDTree
    from paper_1507_06643_gb300 import inputs
    w = inputs.large_n4m(precision)
    spec = w.replicas[0]
    state = inputs.workload_state(w)
    specs = [(spec.n, spec.box, spec.cv, spec.kT, spec.bricks)]
    errs, flips, (qg, pg, eg, _), ref = run_both(specs, precision, scheme, 1, dt=w.dt, a=w.a,
                                                  sigma=w.sigma, prm_seed=w.seed, state=state)
    keep = np.ones(spec.n, bool)
    if flips and scheme == "HYBRID":
        box = np.asarray(spec.box)
        tree = cKDTree(np.mod(ref.q, box), boxsize=box)
        near = tree.query_ball_point(np.mod(ref.q[sorted(flips)], box), 2.0)
        for lst in near:
            keep[lst] = False
        assert keep.mean() > 0.99, keep.mean()
    dq = q_diff(qg, ref.q, [spec.box], ref.offsets)
    moved = q_diff(ref.q, state[0], [spec.box], ref.offsets)   # the oracle's displacement from the start
    e = {"q": float(np.max(np.abs(dq[keep])) / np.max(np.abs(moved))),
         "p": rel_err(pg[keep], ref.p[keep]), "eps": rel_err(eg[keep], ref.eps[keep])}
    assert max(e.values()) < TOL[precision], (e, len(flips))
