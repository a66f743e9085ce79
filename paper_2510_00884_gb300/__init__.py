"""GB300 (sm_103a) neural-constitutive hot path of COMMET: fused MICNN constitutive
update (P and the 81-entry tangent by the CGO chain rule), hex8 element assembly and
CSR scatter, behind the C ABI of include/commet.h.

``build()`` compiles libcommet.so in-tree; the API classes load it and raise if it is
missing (no CPU fallback).
"""
from .build import build  # noqa: F401
from . import _lib  # noqa: F401


def __getattr__(name):
    # torch-facing API is imported lazily so that ``build`` works without a GPU
    if name in ("Model", "Mesh", "Assembler", "newton_assemble", "newton_solve", "target_stress", "ConstUpdateP",
                "ComputeF", "AssembleResidual"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
