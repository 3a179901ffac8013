"""The C-ABI library loads on a CPU-only host and exports every symbol that
include/bal.h declares (no compute calls)."""
import os
import re

import pytest

from paper_2407_00046_b300 import bal, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "bal.h")).read()
    return sorted(set(re.findall(r"BAL_API\s+[\w\s\*]+?\b(bal_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return bal.load()


def test_header_declares_entry_points():
    names = declared()
    for n in ("bal_create_scene", "bal_assemble_hessian", "bal_pcg_solve", "bal_newton_step",
              "bal_time_step"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared():
        assert hasattr(lib, name), name


def test_binding_structs_match_the_library_layout(lib):
    import ctypes as C
    mirrors = [bal.Params, bal.SceneDesc, bal.BsrView, bal.ALState, bal.SolveInfo, bal.NewtonInfo,
               bal.StepInfo]
    for which, cls in enumerate(mirrors):
        assert lib.bal_struct_size(which) == C.sizeof(cls), cls.__name__
    assert lib.bal_struct_size(99) == 0


def test_default_params_follow_the_paper(lib):
    p = bal.default_params()
    assert p.newton_tol == 1e-4 and p.pcg_tol == 1e-4 and p.pcg_stall_window == 100
    assert p.ap_ratio == 1e-2 and p.sigma_growth == 1.2 and p.sigma_cap == 100.0
    assert p.ls_min_alpha == 1e-9 and p.ls_extra_pcg == 100
    assert p.friction == 0.0 and p.friction_eps_v == 0.0      # frictionless unless asked


@pytest.mark.parametrize("field,value", [("friction", -0.1), ("friction_eps_v", -1.0),
                                         ("step_bound", 1.0), ("al_mode", 7)])
def test_create_scene_rejects_invalid_params(lib, field, value):
    """Parameters are validated on the host before any device allocation."""
    from paper_2407_00046_b300 import scenes
    with pytest.raises(bal.BalError) as e:
        bal.Scene(scenes.two_cubes(n=1), bal.default_params(**{field: value}))
    assert e.value.status == 1


def test_last_error_is_a_string(lib):
    assert isinstance(lib.bal_last_error(), bytes)


def test_create_scene_rejects_bad_args(lib):
    import ctypes as C
    h = C.c_void_p()
    assert lib.bal_create_scene(None, None, C.byref(h)) == 1
    assert b"null" in lib.bal_last_error()
