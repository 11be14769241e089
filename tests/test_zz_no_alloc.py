"""dpde_observables_noalloc: the observables of a system computed without any
device allocation, for callers that cannot call cudaMalloc (plug-ins inside a
framework that owns all device memory through its own pool, processes under a
hard memory cap). Its working memory is the library's fixed file-scope device
array, shared by all calls.

Checked through the C ABI against dpde_observables of an FP64 handle holding
the same state, on two calls in a row with different sizes (the second call
must not see the first call's leftovers in the shared array); against the
oracle with walls along z, particles lying on both wall faces; with a
non-finite particle; and the refusal of host pointers before any launch."""
import numpy as np
import pytest

from gpu_util import make_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def test_noalloc_observables_match_handle(torch_cuda):
    torch = torch_cuda
    from paper_1507_06643_gb300 import dpde
    for n, seed in ((20000, 11), (5000, 12)):
        L = (n / 3.0) ** (1.0 / 3.0)
        q, p, e = make_state([(n, (L, L, L), 100.0, 1.0, (1, 1, 1))], seed, False)
        prm = dpde.make_params(precision="fp64")
        rep = dpde.make_replica(n, (L, L, L), 100.0)
        S = dpde.System(prm, [rep])
        S.set_state(q, p, e)
        ref = S.observables(check=True)[0]
        S.close()
        qd, pd, ed = (torch.from_numpy(x).cuda() for x in (q, p, e))
        torch.cuda.synchronize()
        rc, got = dpde.dpde_observables_noalloc(prm, rep, qd, pd, ed)
        assert rc == dpde.DPDE_OK
        assert got["n"] == n
        for k in ("E", "K", "U", "Eint", "Tkin", "Tint", "Tpot_num", "Tpot_den"):
            assert abs(got[k] - ref[k]) <= 1e-10 * abs(ref[k]), (n, k, got[k], ref[k])
        for k in ("Px", "Py", "Pz"):
            assert abs(got[k] - ref[k]) < 1e-9, (n, k)


def test_noalloc_rejects_sizes_beyond_its_scratch(torch_cuda):
    from paper_1507_06643_gb300 import dpde
    n = 300000
    L = (n / 3.0) ** (1.0 / 3.0)
    with pytest.raises(dpde.DPDEError) as ei:
        dpde.dpde_observables_noalloc(dpde.make_params(precision="fp64"), dpde.make_replica(n, L, 100.0),
                                      None, None, None)
    assert ei.value.code == dpde.DPDE_ERR_ARG
    assert "scratch limit" in str(ei.value)


def test_noalloc_observables_with_walls(torch_cuda):
    """A replica with walls along z: no pair across the z boundary, as in the
    handle and in the oracle (the potential energy differs from the periodic
    box's)."""
    torch = torch_cuda
    from oracle import oracle as O
    from paper_1507_06643_gb300 import dpde
    n, box = 6000, (11.0, 11.0, 16.6)
    q, p, e = make_state([(n, box, 100.0, 1.0, (1, 1, 1))], 21, False)
    prm = dpde.make_params(precision="fp64")
    rep = dpde.make_replica(n, box, 100.0, walls=1)
    S = dpde.System(prm, [rep])
    S.set_state(q, p, e)
    ref = S.observables(check=True)[0]
    S.close()
    ora = O.System([O.make_replica(n, box, 100.0, walls=1)], O.make_params(), q, p, e).observables()
    periodic = O.System([O.make_replica(n, box, 100.0)], O.make_params(), q, p, e).observables()
    qd, pd, ed = (torch.from_numpy(x).cuda() for x in (q, p, e))
    torch.cuda.synchronize()
    rc, got = dpde.dpde_observables_noalloc(prm, rep, qd, pd, ed)
    assert rc == dpde.DPDE_OK
    for k in ("E", "U", "Tpot_num", "Tpot_den"):
        assert abs(got[k] - ref[k]) <= 1e-10 * abs(ref[k]), (k, got[k], ref[k])
        assert abs(got[k] - ora[k]) <= 1e-10 * abs(ora[k]), (k, got[k], ora[k])
    assert abs(got["U"] - periodic["U"]) > 1e-6 * abs(periodic["U"])


def test_noalloc_walls_with_particles_on_the_wall_faces(torch_cuda):
    """Particles exactly at z = 0 and z = L_z belong to the bottom and top
    cell layers of a walled replica (no periodic wrap along z): the
    observables match the oracle and the handle, whose pair search has no
    image across the z boundary."""
    torch = torch_cuda
    from oracle import oracle as O
    from paper_1507_06643_gb300 import dpde
    n, box = 4000, (11.0, 11.0, 12.1)
    q, p, e = make_state([(n, box, 100.0, 1.0, (1, 1, 1))], 23, False)
    q[:40, 2] = 0.0
    q[40:80, 2] = box[2]
    q[80:120, 2] = box[2] - 1e-12
    prm = dpde.make_params(precision="fp64")
    rep = dpde.make_replica(n, box, 100.0, walls=1)
    ora = O.System([O.make_replica(n, box, 100.0, walls=1)], O.make_params(), q, p, e).observables()
    S = dpde.System(prm, [rep])
    S.set_state(q, p, e)
    ref = S.observables(check=True)[0]
    qs, _, _ = S.get_state()
    S.close()
    assert np.max(np.abs(qs[40:80, 2] - box[2])) < 1e-12   # the handle kept them on the upper face
    qd, pd, ed = (torch.from_numpy(x).cuda() for x in (q, p, e))
    torch.cuda.synchronize()
    rc, got = dpde.dpde_observables_noalloc(prm, rep, qd, pd, ed)
    assert rc == dpde.DPDE_OK
    for k in ("E", "U", "Tpot_num", "Tpot_den"):
        assert abs(got[k] - ora[k]) <= 1e-10 * abs(ora[k]), (k, got[k], ora[k])
        assert abs(got[k] - ref[k]) <= 1e-10 * abs(ref[k]), (k, got[k], ref[k])


def test_noalloc_skips_pairs_with_a_non_finite_particle(torch_cuda):
    """A particle with a NaN position is counted as non-finite and its pairs
    are skipped (as the handle's pair search skips them): U equals that of
    the same state without the particle."""
    torch = torch_cuda
    from paper_1507_06643_gb300 import dpde
    n = 3000
    L = (n / 3.0) ** (1.0 / 3.0)
    q, p, e = make_state([(n, (L, L, L), 100.0, 1.0, (1, 1, 1))], 24, False)
    prm = dpde.make_params(precision="fp64")
    rep = dpde.make_replica(n, (L, L, L), 100.0)
    q2 = q.copy()
    q2[7] = np.nan
    qd, pd, ed = (torch.from_numpy(x).cuda() for x in (q2, p, e))
    torch.cuda.synchronize()
    rc, got = dpde.dpde_observables_noalloc(prm, rep, qd, pd, ed)
    assert rc == dpde.DPDE_ERR_NONFINITE
    assert got["nonfinite"] == 1
    # the same particle's pairs removed by hand: the state without particle 7
    keep = np.arange(n) != 7
    rep2 = dpde.make_replica(n - 1, (L, L, L), 100.0)
    qd2, pd2, ed2 = (torch.from_numpy(np.ascontiguousarray(x[keep])).cuda() for x in (q, p, e))
    torch.cuda.synchronize()
    rc2, ref = dpde.dpde_observables_noalloc(prm, rep2, qd2, pd2, ed2)
    assert rc2 == dpde.DPDE_OK
    assert abs(got["U"] - ref["U"]) <= 1e-10 * abs(ref["U"]), (got["U"], ref["U"])


def test_noalloc_refuses_host_pointers(torch_cuda):
    """Host memory handed to the C entry point is refused before any launch
    (a kernel given a host pointer would fault or read the wrong memory), and
    the binding refuses arrays that are not contiguous float64 CUDA tensors."""
    import ctypes as C
    torch = torch_cuda
    from paper_1507_06643_gb300 import dpde
    n = 1000
    L = (n / 3.0) ** (1.0 / 3.0)
    q, p, e = make_state([(n, (L, L, L), 100.0, 1.0, (1, 1, 1))], 25, False)
    prm = dpde.make_params(precision="fp64")
    rep = dpde.make_replica(n, (L, L, L), 100.0)
    out = dpde.dpde_obs()
    vp = lambda a: C.c_void_p(a.ctypes.data)
    rc = dpde.lib().dpde_observables_noalloc(C.byref(prm), C.byref(rep), vp(q), vp(p), vp(e), None,
                                             C.byref(out))
    assert rc == dpde.DPDE_ERR_ARG
    assert "device memory" in dpde.lib().dpde_noalloc_last_error().decode()
    for bad in (q, torch.from_numpy(q).float().cuda(), torch.from_numpy(q[:10]).cuda(),
                torch.from_numpy(q).cuda().t()):
        with pytest.raises(dpde.DPDEError) as ei:
            dpde.dpde_observables_noalloc(prm, rep, bad, torch.from_numpy(p).cuda(), torch.from_numpy(e).cuda())
        assert ei.value.code == dpde.DPDE_ERR_ARG
    assert torch.cuda.synchronize() is None                 # the context is intact
