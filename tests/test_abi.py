"""The C-ABI library loads, exports every symbol include/dpde.h declares, and
rejects invalid arguments before touching a GPU (no compute call here)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "dpde.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dpde_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_1507_06643_gb300 import dpde
    L = dpde.lib()
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(dpde.EXPORTS)


def test_invalid_arguments_are_rejected():
    from paper_1507_06643_gb300 import dpde
    good = dpde.make_replica(100, 5.0, 100.0)
    for prm, reps in [
        (dpde.make_params(mass=-1.0), [good]),
        (dpde.make_params(r_cut=0.0), [good]),
        (dpde.make_params(precision=7), [good]),
        (dpde.make_params(), [dpde.make_replica(100, 2.5, 100.0)]),          # 2 cells per axis
        (dpde.make_params(), [dpde.make_replica(100, 5.0, 100.0, (6, 1, 1))]),  # brick < r_cut
        (dpde.make_params(), [dpde.make_replica(100, 5.0, -1.0)]),
        (dpde.make_params(), [dpde.make_replica(-5, 5.0, 100.0)]),
    ]:
        with pytest.raises(dpde.DPDEError) as ei:
            dpde.dpde_create(prm, reps)
        assert ei.value.code == dpde.DPDE_ERR_ARG
    h = C.c_void_p()
    assert dpde.lib().dpde_create(None, 1, None, None, C.byref(h)) == dpde.DPDE_ERR_ARG
    assert dpde.lib().dpde_step(None, 1, 0.01, 0, 1) == dpde.DPDE_ERR_ARG
    assert dpde.lib().dpde_destroy(None) == dpde.DPDE_OK
