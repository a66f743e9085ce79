"""PyTorch-facing wrappers of the C ABI: device tensors in, device tensors out.

Layouts (see include/commet.h): per-qp tables are component-major, F[9, n_qp],
P[9, n_qp], A[81, n_qp]; element tables f_e[24, n_el], K_e[576, n_el]; nodal
vectors u[3, n_nodes]; the global residual r[3 * n_nodes] is node-major. All work
runs in libcommet's CUDA kernels on torch's current stream.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib

_PREC = {"f64": _lib.F64, "f32": _lib.F32, "bf16": _lib.BF16_MLP}
_DTYPE = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.float32}


def _stream() -> C.c_void_p:
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _dbl(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _check_dev(t, dtype, shape=None, name="tensor"):
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


class Model:
    """A MICNN strain energy on the GPU (one precision per handle).

    ``spec`` is any object with the attributes d, W, L, kin, fibres, W1, Ak, Bk, c, a, b,
    kappa and stress_free (row-major float64 arrays, see workload.ModelSpec).
    """

    def __init__(self, spec, precision: str = "f64"):
        lib = _lib.load()
        self.precision = precision
        self.dtype = _DTYPE[precision]
        self.d, self.W, self.L = int(spec.d), int(spec.W), int(spec.L)
        self._keep = []
        fib, pfib = _dbl(np.asarray(spec.fibres).reshape(-1, 3) if len(spec.fibres) else np.zeros((1, 3)))
        W1, pW1 = _dbl(spec.W1)
        Ak, pA = _dbl(spec.Ak if self.L > 1 else np.zeros(1))
        Bk, pB = _dbl(spec.Bk if self.L > 1 else np.zeros(1))
        c, pc = _dbl(spec.c)
        a, pa = _dbl(spec.a)
        b, pb = _dbl(spec.b)
        self._keep += [fib, W1, Ak, Bk, c, a, b]
        desc = _lib.ModelDesc(kinematics=int(spec.kin), n_fibres=int(len(spec.fibres)), fibres=pfib,
                              d=self.d, W=self.W, L=self.L, W1=pW1, A=pA, B=pB, c=pc, a_out=pa, b_out=pb,
                              activation=_lib.ACT_SOFTPLUS, kappa=float(spec.kappa),
                              stress_free=int(bool(spec.stress_free)))
        h = C.c_void_p()
        _lib.check("commet_model_create", lib.commet_model_create(C.byref(desc), _PREC[precision], C.byref(h)))
        self.handle = h
        self.n_params = int(lib.commet_model_n_params(h))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib._lib is not None:
            _lib._lib.commet_model_destroy(h)
            self.handle = None

    def const_update(self, F: torch.Tensor, want_A: bool = True, want_psi: bool = True, status: bool = False,
                     out=None):
        """psi[n], P[9, n], A[81, n] (or None) for F[9, n]; with status=True also the
        device int32[2] status (bad-point count, first bad index)."""
        _check_dev(F, self.dtype, name="F")
        n = F.shape[1]
        if out is None:
            psi = torch.empty(n, dtype=self.dtype, device=F.device) if want_psi else None
            P = torch.empty(9, n, dtype=self.dtype, device=F.device)
            A = torch.empty(81, n, dtype=self.dtype, device=F.device) if want_A else None
        else:
            psi, P, A = out
        st = torch.empty(2, dtype=torch.int32, device=F.device) if status else None
        _lib.check("commet_const_update", _lib.load().commet_const_update(
            self.handle, n, _ptr(F), _ptr(psi), _ptr(P), _ptr(A), _ptr(st), _stream()))
        return (psi, P, A, st) if status else (psi, P, A)

    def const_update_spatial(self, F: torch.Tensor, want_c: bool = True, want_psi: bool = True,
                             status: bool = False, out=None):
        """psi[n], tau[6, n], c[21, n] (or None) for F[9, n]: Kirchhoff stress and spatial
        stiffness in Voigt form (11, 22, 33, 23, 13, 12; c as the row-major upper triangle
        of the 6 x 6 matrix)."""
        _check_dev(F, self.dtype, name="F")
        n = F.shape[1]
        if out is None:
            psi = torch.empty(n, dtype=self.dtype, device=F.device) if want_psi else None
            tau = torch.empty(6, n, dtype=self.dtype, device=F.device)
            c = torch.empty(21, n, dtype=self.dtype, device=F.device) if want_c else None
        else:
            psi, tau, c = out
        st = torch.empty(2, dtype=torch.int32, device=F.device) if status else None
        _lib.check("commet_const_update_spatial", _lib.load().commet_const_update_spatial(
            self.handle, n, _ptr(F), _ptr(psi), _ptr(tau), _ptr(c), _ptr(st), _stream()))
        return (psi, tau, c, st) if status else (psi, tau, c)

    def backward(self, F: torch.Tensor, G: torch.Tensor, want_dF: bool = True, workspace=None, out=None):
        """dL/dF[9, n] (or None) and dL/dtheta[n_params] for upstream G = dL/dP [9, n]."""
        _check_dev(F, self.dtype, name="F")
        _check_dev(G, self.dtype, shape=F.shape, name="G")
        lib = _lib.load()
        n = F.shape[1]
        if out is None:
            dF = torch.empty_like(F) if want_dF else None
            dth = torch.empty(self.n_params, dtype=self.dtype, device=F.device)
        else:
            dF, dth = out
        ws_bytes = int(lib.commet_const_backward_workspace(self.handle, n))
        if workspace is None or workspace.numel() < ws_bytes:
            workspace = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=F.device)
        _lib.check("commet_const_backward", lib.commet_const_backward(
            self.handle, n, _ptr(F), _ptr(G), _ptr(dF), _ptr(dth), _ptr(workspace), ws_bytes, _stream()))
        return dF, dth


class Mesh:
    """Hex8 mesh on the GPU: X[n_nodes, 3] (float64) and conn[n_el, 8] (int32), host arrays."""

    def __init__(self, X, conn, want_csr: bool = False):
        lib = _lib.load()
        X = np.ascontiguousarray(X, dtype=np.float64)
        conn = np.ascontiguousarray(conn, dtype=np.int32)
        self.n_nodes, self.n_el = X.shape[0], conn.shape[0]
        h = C.c_void_p()
        _lib.check("commet_mesh_create", lib.commet_mesh_create(
            self.n_nodes, X.ctypes.data_as(C.POINTER(C.c_double)), self.n_el,
            conn.ctypes.data_as(C.POINTER(C.c_int32)), int(want_csr), C.byref(h)))
        self.handle = h
        n_rows, nnz, ncol = C.c_int64(), C.c_int64(), C.c_int32()
        _lib.check("commet_mesh_info", lib.commet_mesh_info(h, C.byref(n_rows), C.byref(nnz), C.byref(ncol)))
        self.n_rows, self.nnz, self.n_colours = n_rows.value, nnz.value, ncol.value
        self.has_csr = bool(want_csr)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib._lib is not None:
            _lib._lib.commet_mesh_destroy(h)
            self.handle = None

    def csr(self):
        """Host (rowptr int64[n_rows+1], col int32[nnz]) of the global stiffness pattern."""
        rowptr = np.empty(self.n_rows + 1, dtype=np.int64)
        col = np.empty(max(self.nnz, 1), dtype=np.int32)
        _lib.check("commet_mesh_csr", _lib.load().commet_mesh_csr(
            self.handle, rowptr.ctypes.data_as(C.POINTER(C.c_int64)), col.ctypes.data_as(C.POINTER(C.c_int32))))
        return rowptr, col[:self.nnz]

    def compute_F(self, u: torch.Tensor, precision: str = "f64", out=None) -> torch.Tensor:
        """F[9, 8 n_el] from u[3, n_nodes]."""
        dt = _DTYPE[precision]
        _check_dev(u, dt, shape=(3, self.n_nodes), name="u")
        F = out if out is not None else torch.empty(9, 8 * self.n_el, dtype=dt, device=u.device)
        _lib.check("commet_compute_F", _lib.load().commet_compute_F(
            self.handle, _PREC[precision], _ptr(u), _ptr(F), _stream()))
        return F

    def elem_assemble(self, P: torch.Tensor, A: torch.Tensor | None, precision: str = "f64",
                      want_f: bool = True, want_K: bool = True, want_r: bool = False, want_Kcsr: bool = False,
                      out=None):
        """(f_e[24, n_el], K_e[576, n_el], r[3 n_nodes], K_vals[nnz]); entries not wanted are None."""
        dt = _DTYPE[precision]
        n_qp = 8 * self.n_el
        _check_dev(P, dt, shape=(9, n_qp), name="P")
        if A is not None:
            _check_dev(A, dt, shape=(81, n_qp), name="A")
        dev = P.device
        if out is None:
            f_e = torch.empty(24, self.n_el, dtype=dt, device=dev) if want_f else None
            K_e = torch.empty(576, self.n_el, dtype=dt, device=dev) if (want_K and A is not None) else None
            r = torch.empty(3 * self.n_nodes, dtype=dt, device=dev) if want_r else None
            Kv = torch.empty(self.nnz, dtype=dt, device=dev) if want_Kcsr else None
        else:
            f_e, K_e, r, Kv = out
        _lib.check("commet_elem_assemble", _lib.load().commet_elem_assemble(
            self.handle, _PREC[precision], _ptr(P), _ptr(A), _ptr(f_e), _ptr(K_e), _ptr(r), _ptr(Kv), _stream()))
        return f_e, K_e, r, Kv


    def elem_assemble_spatial(self, F: torch.Tensor, tau: torch.Tensor, c: torch.Tensor | None,
                              precision: str = "f64", want_f: bool = True, want_K: bool = True,
                              want_r: bool = False, want_Kcsr: bool = False, out=None):
        """Spatial-form element integrals from F[9, n_qp], tau[6, n_qp], c[21, n_qp]:
        (f_e[24, n_el], K_e[576, n_el], r[3 n_nodes], K_vals[nnz]); entries not wanted are None."""
        dt = _DTYPE[precision]
        n_qp = 8 * self.n_el
        _check_dev(F, dt, shape=(9, n_qp), name="F")
        _check_dev(tau, dt, shape=(6, n_qp), name="tau")
        if c is not None:
            _check_dev(c, dt, shape=(21, n_qp), name="c")
        dev = F.device
        if out is None:
            f_e = torch.empty(24, self.n_el, dtype=dt, device=dev) if want_f else None
            K_e = torch.empty(576, self.n_el, dtype=dt, device=dev) if (want_K and c is not None) else None
            r = torch.empty(3 * self.n_nodes, dtype=dt, device=dev) if want_r else None
            Kv = torch.empty(self.nnz, dtype=dt, device=dev) if want_Kcsr else None
        else:
            f_e, K_e, r, Kv = out
        _lib.check("commet_elem_assemble_spatial", _lib.load().commet_elem_assemble_spatial(
            self.handle, _PREC[precision], _ptr(F), _ptr(tau), _ptr(c), _ptr(f_e), _ptr(K_e), _ptr(r), _ptr(Kv),
            _stream()))
        return f_e, K_e, r, Kv


def newton_assemble(model: Model, mesh: Mesh, u: torch.Tensor, status: bool = False, out=None):
    """Fused u -> r[3 n_nodes], K_vals[nnz] (CSR of mesh.csr())."""
    _check_dev(u, model.dtype, shape=(3, mesh.n_nodes), name="u")
    if out is None:
        r = torch.empty(3 * mesh.n_nodes, dtype=model.dtype, device=u.device)
        Kv = torch.empty(mesh.nnz, dtype=model.dtype, device=u.device)
    else:
        r, Kv = out
    st = torch.empty(2, dtype=torch.int32, device=u.device) if status else None
    _lib.check("commet_newton_assemble", _lib.load().commet_newton_assemble(
        model.handle, mesh.handle, _ptr(u), _ptr(r), _ptr(Kv), _ptr(st), _stream()))
    return (r, Kv, st) if status else (r, Kv)


def target_stress(F: torch.Tensor, fibres, mu: float, k1: float, k2: float, kappa: float) -> torch.Tensor:
    """P[9, n] of the closed-form Neo-Hookean-plus-fibre target model."""
    prec = "f64" if F.dtype == torch.float64 else "f32"
    _check_dev(F, F.dtype, name="F")
    fib, pf = _dbl(np.asarray(fibres).reshape(-1, 3) if len(fibres) else np.zeros((1, 3)))
    P = torch.empty_like(F)
    _lib.check("commet_target_stress", _lib.load().commet_target_stress(
        _PREC[prec], F.shape[1], _ptr(F), int(len(fibres)), pf, mu, k1, k2, kappa, _ptr(P), _stream()))
    return P


class ConstUpdateP(torch.autograd.Function):
    """P(F) as an autograd node: forward runs the constitutive kernel (stress only),
    backward runs the adjoint kernel and returns dL/dF and dL/dtheta (the latter is
    attached to ``theta_grad_sink`` because the weights live in the model handle)."""

    @staticmethod
    def forward(ctx, F, theta_grad_sink, model):
        ctx.model = model
        ctx.save_for_backward(F)
        _, P, _ = model.const_update(F.contiguous(), want_A=False, want_psi=False)
        return P

    @staticmethod
    def backward(ctx, G):
        (F,) = ctx.saved_tensors
        dF, dth = ctx.model.backward(F.contiguous(), G.contiguous())
        return dF, dth, None
