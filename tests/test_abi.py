"""CPU checks of the boundary: the library builds, loads and exports every symbol the
public header declares; argument checks that need no GPU return their error codes."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "commet.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(commet_[A-Za-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_2510_00884_gb300 as p
    p.build()
    from paper_2510_00884_gb300 import _lib
    return _lib.load()


def test_header_declares_the_boundary():
    fns = declared_functions()
    for f in ("commet_const_update", "commet_elem_assemble", "commet_const_backward"):
        assert f in fns


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_the_header(lib):
    from paper_2510_00884_gb300 import _lib
    assert sorted(_lib.EXPORTED) == declared_functions()


def test_status_strings(lib):
    from paper_2510_00884_gb300 import _lib
    for code in range(5):
        assert len(_lib.status_string(code)) > 0
    assert _lib.status_string(99) == "unknown status code"


def test_host_side_argument_checks(lib):
    """Checks that return before any CUDA call."""
    from paper_2510_00884_gb300 import _lib
    out = C.c_void_p()
    assert lib.commet_model_create(None, 0, C.byref(out)) == _lib.ERR_INVALID_ARG
    desc = _lib.ModelDesc(kinematics=7, d=3, W=16, L=2)
    assert lib.commet_model_create(C.byref(desc), 0, C.byref(out)) == _lib.ERR_INVALID_ARG
    desc = _lib.ModelDesc(kinematics=0, d=3, W=16, L=2)
    assert lib.commet_model_create(C.byref(desc), 9, C.byref(out)) == _lib.ERR_INVALID_ARG
    desc = _lib.ModelDesc(kinematics=2, n_fibres=1, d=5, W=16, L=2)  # polyconvex takes no fibres
    assert lib.commet_model_create(C.byref(desc), 0, C.byref(out)) == _lib.ERR_INVALID_ARG
    desc = _lib.ModelDesc(kinematics=2, d=5, W=16, L=2)                # and d = 3
    assert lib.commet_model_create(C.byref(desc), 0, C.byref(out)) == _lib.ERR_INVALID_ARG
    assert lib.commet_const_update(None, 1, None, None, None, None, None, None) == _lib.ERR_INVALID_ARG
    assert lib.commet_mesh_create(-1, None, 0, None, 0, C.byref(out)) == _lib.ERR_INVALID_ARG
    X = (C.c_double * 24)(*([0.0] * 24))
    conn = (C.c_int32 * 8)(0, 1, 2, 3, 4, 5, 6, 99)
    assert lib.commet_mesh_create(8, X, 1, conn, 0, C.byref(out)) == _lib.ERR_INVALID_ARG
    assert lib.commet_elem_assemble(None, 0, None, None, None, None, None, None, None) == _lib.ERR_INVALID_ARG
    assert lib.commet_target_stress(0, 1, None, 0, None, 1.0, 2.0, 0.5, 10.0, None, None) == \
        _lib.ERR_INVALID_ARG
    assert lib.commet_const_backward(None, 1, None, None, None, None, None, 0, None) == _lib.ERR_INVALID_ARG
    assert lib.commet_model_n_params(None) == -1
    # host-buffer pipeline: no model, no chunk
    assert lib.commet_const_update_host(None, None, 8, None, None, None, None, None, None, None, 0, 4,
                                        None) == _lib.ERR_INVALID_ARG
    assert lib.commet_const_update_host_workspace(None, None, 4, 1) == 0


def test_product_path_does_not_touch_the_oracle():
    """The package imports nothing from oracle/ and names no oracle file."""
    pkg_dir = os.path.join(ROOT, "paper_2510_00884_gb300")
    for dirpath, _, files in os.walk(pkg_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "commet_oracle" not in src and "liboracle" not in src, f
