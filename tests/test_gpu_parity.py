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

from gpu_util import make_state, rel_err, run_both

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
    errs, _, _ = run_both(specs, precision, scheme, 10, seed=1001)
    assert max(errs.values()) < TOL[precision], errs


@pytest.mark.parametrize("n,box,bricks", [
    (1, (4.0, 4.0, 4.0), (1, 1, 1)),
    (2, (3.0, 3.0, 3.0), (1, 1, 1)),
    (64, (cube(64),) * 3, (1, 1, 1)),
    (777, (5.0, 7.3, 7.1), (1, 2, 3)),
    (3000, (7.0, 10.5, 13.6), (2, 3, 1)),
    (2500, (9.3, 9.3, 9.7), (3, 3, 3)),
])
@pytest.mark.parametrize("scheme", ["SER", "HYBRID"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_parity_sizes(n, box, bricks, scheme, precision):
    specs = [(n, box, 50.0, 1.0, bricks)]
    errs, _, _ = run_both(specs, precision, scheme, 6, seed=n)
    assert max(errs.values()) < TOL[precision], errs


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
    errs, (qg, pg, eg, obs), ref = run_both(specs, precision, scheme, 5, seed=55)
    assert max(errs.values()) < TOL[precision], errs
    tol = TOL[precision] * 10
    for r in range(len(specs)):
        o = ref.observables(r)
        for k in ("K", "U", "Eint", "Tkin", "Tint", "Tpot_num", "Tpot_den"):
            assert abs(obs[r][k] - o[k]) <= tol * max(1.0, abs(o[k])), (r, k, obs[r][k], o[k])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_observables_match_oracle(precision):
    specs = [(1000, (cube(1000),) * 3, 100.0, 1.0, (2, 2, 2))]
    errs, (_, _, _, obs), ref = run_both(specs, precision, "HYBRID", 3, seed=9)
    o = ref.observables(0)
    tol = 1e-10 if precision == "fp64" else 1e-5
    for k in ("E", "K", "U", "Eint", "Tkin", "Tint", "Tpot_num", "Tpot_den"):
        assert abs(obs[0][k] - o[k]) <= tol * abs(o[k]), (k, obs[0][k], o[k])
    for k in ("Px", "Py", "Pz"):
        assert abs(obs[0][k] - o[k]) < 1e-9


# ---- determinism, resume, graphs ----------------------------------------------

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("scheme", ["SER", "HYBRID"])
def test_resume_and_graph_are_bit_exact(precision, scheme):
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
    mid = B.get_state()
    C = dpde.System(prm, rep)
    C.set_state(*mid, step=4)
    C.step(6, 0.01, scheme, use_graph=True)
    c = C.get_state()
    for x, y in zip(a, c):
        assert np.array_equal(x, y)


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


# ---- the benchmark's workload at full size ------------------------------------------

@pytest.mark.parametrize("precision,scheme", [("mixed", "HYBRID"), ("mixed", "SER"), ("fp64", "HYBRID")])
def test_full_size_large_n4m_one_step(precision, scheme):
    from paper_1507_06643_gb300 import inputs
    w = inputs.large_n4m(precision)
    spec = w.replicas[0]
    state = inputs.workload_state(w)
    specs = [(spec.n, spec.box, spec.cv, spec.kT, spec.bricks)]
    errs, _, _ = run_both(specs, precision, scheme, 1, dt=w.dt, a=w.a, sigma=w.sigma,
                          prm_seed=w.seed, state=state)
    assert max(errs.values()) < TOL[precision], errs
