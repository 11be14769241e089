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
        (dpde.make_params(), [dpde.make_replica((1 << 27) + 1, 356.0, 100.0)]),   # particle limit
        (dpde.make_params(), [dpde.make_replica(100, 1100.0, 100.0)]),            # cell limit 2^30
    ]:
        with pytest.raises(dpde.DPDEError) as ei:
            dpde.dpde_create(prm, reps)
        assert ei.value.code == dpde.DPDE_ERR_ARG
    h = C.c_void_p()
    assert dpde.lib().dpde_create(None, 1, None, None, C.byref(h)) == dpde.DPDE_ERR_ARG
    assert dpde.lib().dpde_step(None, 1, 0.01, 0, 1) == dpde.DPDE_ERR_ARG
    assert dpde.lib().dpde_destroy(None) == dpde.DPDE_OK


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes structures of the binding have the C header's sizes and
    field offsets (a drifted layout would pass garbage silently)."""
    import shutil
    import subprocess
    from paper_1507_06643_gb300 import dpde
    if shutil.which("gcc") is None:
        pytest.skip("gcc is needed to compile the layout probe")
    structs = {"dpde_params": dpde.dpde_params, "dpde_replica": dpde.dpde_replica, "dpde_obs": dpde.dpde_obs,
               "dpde_tuning": dpde.dpde_tuning}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dpde.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "size")] == C.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def test_invalid_walls_are_rejected():
    from paper_1507_06643_gb300 import dpde
    for walls, u in ((2, 0.0), (-1, 0.0), (1, 0.25)):
        with pytest.raises(dpde.DPDEError) as ei:
            dpde.dpde_create(dpde.make_params(), [dpde.make_replica(100, 5.0, 100.0, walls=walls, wall_u=u)])
        assert ei.value.code == dpde.DPDE_ERR_ARG


def test_oracle_struct_layouts_match_its_header(tmp_path):
    import shutil
    import subprocess
    from oracle import oracle as O
    if shutil.which("gcc") is None:
        pytest.skip("gcc is needed to compile the layout probe")
    structs = {"ora_params": O.Params, "ora_replica": O.Replica}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "oracle.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "oracle"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "size")] == C.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def test_noalloc_limit_matches_the_header():
    from paper_1507_06643_gb300 import dpde
    text = open(os.path.join(ROOT, "include", "dpde.h")).read()
    m = re.search(r"#define DPDE_NOALLOC_MAX_N\s+(\d+)", text)
    assert m and int(m.group(1)) == dpde.DPDE_NOALLOC_MAX_N
