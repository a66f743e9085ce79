"""ctypes declarations of libcommet.so (the C ABI in include/commet.h).

Argument marshalling only. Loading fails loudly when the library has not been built:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcommet.so")

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_CUDA, ERR_NO_CSR = 0, 1, 2, 3, 4
F64, F32, BF16_MLP = 0, 1, 2
KIN_ISO_SHIFTED, KIN_RAW = 0, 1
ACT_SOFTPLUS = 0

EXPORTED = [
    "commet_model_create", "commet_model_destroy", "commet_model_n_params", "commet_const_update",
    "commet_const_update_spatial", "commet_elem_assemble_spatial",
    "commet_mesh_create", "commet_mesh_destroy", "commet_mesh_info", "commet_mesh_csr", "commet_compute_F",
    "commet_elem_assemble", "commet_elem_assemble_symmetric", "commet_newton_assemble",
    "commet_const_backward_workspace",
    "commet_const_backward", "commet_target_stress", "commet_status_string", "commet_const_backward_noalloc",
    "commet_mesh_set_dirichlet", "commet_set_dirichlet_values", "commet_apply_dirichlet", "commet_cg_workspace",
    "commet_cg_solve", "commet_add_increment", "commet_norm2", "commet_residual_adjoint", "commet_compute_F_adjoint",
    "commet_const_update_host_workspace", "commet_const_update_host",
]


class ModelDesc(C.Structure):
    _fields_ = [("kinematics", C.c_int32), ("n_fibres", C.c_int32), ("fibres", C.POINTER(C.c_double)),
                ("d", C.c_int32), ("W", C.c_int32), ("L", C.c_int32),
                ("W1", C.POINTER(C.c_double)), ("A", C.POINTER(C.c_double)), ("B", C.POINTER(C.c_double)),
                ("c", C.POINTER(C.c_double)), ("a_out", C.POINTER(C.c_double)),
                ("b_out", C.POINTER(C.c_double)), ("activation", C.c_int32), ("kappa", C.c_double),
                ("stress_free", C.c_int32), ("inner", C.c_int32), ("cann_terms", C.c_int32),
                ("cann_kind", C.POINTER(C.c_int32)), ("cann_w", C.POINTER(C.c_double)),
                ("kan_layers", C.c_int32), ("kan_widths", C.POINTER(C.c_int32)), ("kan_degree", C.c_int32),
                ("kan_grid", C.c_int32), ("kan_lo", C.POINTER(C.c_double)), ("kan_hi", C.POINTER(C.c_double)),
                ("kan_params", C.POINTER(C.c_double))]

INNER_MICNN, INNER_CANN, INNER_GENT_THOMAS, INNER_ICKAN = 0, 1, 2, 3


class CommetError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} failed: {status_string(code)} (code {code})")
        self.code = code


_lib = None


def load() -> C.CDLL:
    """Load libcommet.so (built by paper_2510_00884_gb300.build). Raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'` "
                           "(the CUDA library is required: there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    pm = C.POINTER(C.c_void_p)
    sig = {
        "commet_model_create": ([C.POINTER(ModelDesc), i32, pm], C.c_int),
        "commet_model_destroy": ([vp], C.c_int),
        "commet_model_n_params": ([vp], i64),
        "commet_const_update": ([vp, i64, vp, vp, vp, vp, vp, vp], C.c_int),
        "commet_mesh_create": ([i64, C.POINTER(C.c_double), i64, C.POINTER(C.c_int32), i32, pm], C.c_int),
        "commet_mesh_destroy": ([vp], C.c_int),
        "commet_mesh_info": ([vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i32)], C.c_int),
        "commet_mesh_csr": ([vp, C.POINTER(i64), C.POINTER(i32)], C.c_int),
        "commet_compute_F": ([vp, i32, vp, vp, vp], C.c_int),
        "commet_elem_assemble": ([vp, i32, vp, vp, vp, vp, vp, vp, vp], C.c_int),
        "commet_elem_assemble_symmetric": ([vp, i32, vp, vp, vp, vp, vp, vp, vp], C.c_int),
        "commet_const_update_spatial": ([vp, i64, vp, vp, vp, vp, vp, vp], C.c_int),
        "commet_elem_assemble_spatial": ([vp, i32, vp, vp, vp, vp, vp, vp, vp, vp], C.c_int),
        "commet_newton_assemble": ([vp, vp, vp, vp, vp, vp, vp], C.c_int),
        "commet_const_backward_workspace": ([vp, i64], C.c_size_t),
        "commet_const_backward": ([vp, i64, vp, vp, vp, vp, vp, C.c_size_t, vp], C.c_int),
        "commet_target_stress": ([i32, i64, vp, i32, C.POINTER(C.c_double), C.c_double, C.c_double,
                                  C.c_double, C.c_double, vp, vp], C.c_int),
        "commet_status_string": ([C.c_int], C.c_char_p),
        "commet_const_backward_noalloc": ([vp, i64, vp, vp, vp, vp, vp], C.c_int),
        "commet_mesh_set_dirichlet": ([vp, i64, C.POINTER(i64)], C.c_int),
        "commet_set_dirichlet_values": ([vp, i32, C.POINTER(C.c_double), vp, vp], C.c_int),
        "commet_apply_dirichlet": ([vp, i32, vp, vp, C.POINTER(C.c_double), vp], C.c_int),
        "commet_cg_workspace": ([vp, i32], C.c_size_t),
        "commet_cg_solve": ([vp, i32, vp, vp, vp, C.c_double, i32, vp, C.c_size_t, C.POINTER(i32),
                             C.POINTER(C.c_double), vp], C.c_int),
        "commet_add_increment": ([vp, i32, vp, C.c_double, vp, vp], C.c_int),
        "commet_norm2": ([vp, i32, i64, vp, C.POINTER(C.c_double), vp], C.c_int),
        "commet_residual_adjoint": ([vp, i32, vp, vp, vp], C.c_int),
        "commet_compute_F_adjoint": ([vp, i32, vp, vp, vp], C.c_int),
        "commet_const_update_host_workspace": ([vp, vp, i64, i32], C.c_size_t),
        "commet_const_update_host": ([vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, C.c_size_t, i64, vp], C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def status_string(code: int) -> str:
    return load().commet_status_string(code).decode()


def check(fn: str, code: int) -> None:
    if code != OK:
        raise CommetError(fn, code)
