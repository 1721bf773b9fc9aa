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
