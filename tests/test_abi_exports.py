"""The C-ABI library builds, loads and exports every function include/emg.h declares
(no GPU needed: nothing here calls into the device)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "emg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s+(emg_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1807_01151_gb300 import build
    build.build()
    from paper_1807_01151_gb300 import _lib
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("emg_create_mesh", "emg_set_state", "emg_vcycle", "emg_solve_steady", "emg_residual_norm"):
        assert n in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    from paper_1807_01151_gb300 import _lib
    assert set(declared_functions()) == set(_lib.EXPORTS)


def test_host_only_calls(lib):
    from paper_1807_01151_gb300 import _lib
    p = _lib.ParamsC()
    lib.emg_default_params(p)
    assert p.gamma == 1.4 and p.krylov_m == 30 and p.rk_stages == 4 and p.cfl_max == 100.0 and p.pre_smooth == 2
    assert b"sm_103a" in lib.emg_build_info()
    assert lib.emg_profile_class_name(0) == b"residual_face_flux"
    assert lib.emg_last_error(None) == b"null context"


def test_ctypes_structs_match_the_header_layout(tmp_path):
    """Every struct the binding mirrors has the header's size and field offsets, as a C
    compiler lays them out (gcc on the header itself, as strict C99)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_1807_01151_gb300 import _lib
    pairs = {"emg_mesh_desc": _lib.MeshDescC, "emg_params": _lib.ParamsC, "emg_cycle_info": _lib.CycleInfoC,
             "emg_solve_report": _lib.SolveReportC, "emg_server_params": _lib.ServerParamsC,
             "emg_request_result": _lib.RequestResultC}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "emg.h"', 'int main(void) {']
    for cname, py in pairs.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c99", "-pedantic-errors", "-Wall", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    import ctypes
    got = {}
    for line in out:
        if line.strip():
            cname, field, val = line.split()
            got[cname, field] = int(val)
    for cname, py in pairs.items():
        assert got[cname, "sizeof"] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[cname, f] == getattr(py, f).offset, (cname, f)
