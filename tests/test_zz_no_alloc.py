"""dpde_observables_noalloc: the observables of a system computed without any
device allocation, for callers that cannot call cudaMalloc (code running
while a stream is captured into a CUDA graph, plug-ins inside a framework
that owns all device memory, processes under a hard memory cap). Its working
memory is the library's fixed file-scope device array, shared by all calls.

Checked through the C ABI against dpde_observables of an FP64 handle holding
the same state, on two calls in a row with different sizes (the second call
must not see the first call's leftovers in the shared array)."""
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
