"""The C-ABI library loads on a machine without a GPU and exports every
function that include/hp.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "hp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:hp_status|void|int|const char\s*\*)\s*(hp_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_04644_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("hp_mesh_create", "hp_geom_factors", "hp_op_apply", "hp_op_create", "hp_mesh_layout"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_status_strings(lib):
    lib.hp_status_str.restype = ctypes.c_char_p
    assert lib.hp_status_str(0) == b"HP_OK"
    assert lib.hp_status_str(4) == b"HP_ERR_GEOM"


def test_binding_names_match_header(lib):
    from paper_2604_04644_gb300 import hp
    assert sorted(hp.EXPORTED) == sorted(f for f in declared_functions() if f in hp.EXPORTED)
    for f in hp.EXPORTED:
        assert hasattr(hp, f)


def test_null_arguments_are_rejected_without_gpu(lib):
    # argument validation happens before any CUDA call
    lib.hp_mesh_create.restype = ctypes.c_int
    assert lib.hp_mesh_create(None, 0, None) == 1          # HP_ERR_ARG
    lib.hp_op_apply.restype = ctypes.c_int
    lib.hp_op_apply.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.hp_op_apply(None, 1.0, None, None, None) == 1
    lib.hp_op_set_collocated.restype = ctypes.c_int
    lib.hp_op_set_collocated.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert lib.hp_op_set_collocated(None, 0) == 1
    lib.hp_op_strategies.restype = ctypes.c_int
    lib.hp_op_strategies.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int]
    assert lib.hp_op_strategies(None, None, 0, 0) == 1


def test_binding_constants_match_header():
    """Every enumerator the header gives an explicit value has the same value in
    the binding (strategies, shapes, dtypes, statuses, operator kinds)."""
    from paper_2604_04644_gb300 import hp
    txt = open(os.path.join(ROOT, "include", "hp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    values = dict((k, int(v)) for k, v in re.findall(r"\b(HP_[A-Z0-9_]+)\s*=\s*(\d+)", txt))
    assert values["HP_STRAT_MATRIX"] == 4 and values["HP_STRAT_AUTO"] == 3
    for name, v in values.items():
        assert getattr(hp, name) == v, name


def test_mesh2d_arguments_are_checked_without_gpu(lib):
    from paper_2604_04644_gb300 import hp, inputs
    lib.hp_mesh2d_create.restype = ctypes.c_int
    assert lib.hp_mesh2d_create(None, 0, None) == 1
    mesh = inputs.square_mesh_2d(2, 1, 3)
    for key, val in (("shape", 3), ("P", 11)):
        bad = dict(mesh)
        bad[key] = mesh[key].copy()
        bad[key][0] = val
        with pytest.raises(hp.HpError) as ei:
            hp.hp_mesh2d_create(bad, 0)
        assert ei.value.status == hp.HP_ERR_ARG
    bad = dict(mesh)
    bad["vert"] = mesh["vert"].copy()
    bad["vert"][0, 0] = mesh["n_vert"]
    with pytest.raises(hp.HpError) as ei:
        hp.hp_mesh2d_create(bad, 0)
    assert ei.value.status == hp.HP_ERR_ARG
