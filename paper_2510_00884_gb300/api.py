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
    """A strain energy on the GPU (one precision per handle).

    ``spec`` is any object with the attributes d, kin, fibres, kappa and stress_free and,
    by its ``inner_name`` (default "micnn"):
      micnn        W, L, W1, Ak, Bk, c, a, b (row-major float64 arrays, see workload.ModelSpec)
      cann         n, kinds[n][3], w[d][n][2] (see workload.CannSpec)
      gent_thomas  nothing more (eq. gt on raw kinematics)
      ickan        widths, degree, G, lo, hi, params (see workload.IckanSpec)
    """

    def __init__(self, spec, precision: str = "f64"):
        lib = _lib.load()
        self.precision = precision
        self.dtype = _DTYPE[precision]
        self._keep = []
        fib, pfib = _dbl(np.asarray(spec.fibres).reshape(-1, 3) if len(spec.fibres) else np.zeros((1, 3)))
        inner = getattr(spec, "inner_name", "micnn")
        if inner != "micnn":
            self.d, self.W, self.L = int(spec.d), 0, 0
            desc = _lib.ModelDesc(kinematics=int(spec.kin), n_fibres=int(len(spec.fibres)), fibres=pfib,
                                  d=self.d, kappa=float(spec.kappa), stress_free=int(bool(spec.stress_free)))
            if inner == "cann":
                kinds = np.ascontiguousarray(spec.kinds, dtype=np.int32)
                w, pw = _dbl(spec.w)
                self._keep += [kinds, w]
                desc.inner = _lib.INNER_CANN
                desc.cann_terms = int(spec.n)
                desc.cann_kind = kinds.ctypes.data_as(C.POINTER(C.c_int32))
                desc.cann_w = pw
            elif inner == "gent_thomas":
                desc.inner = _lib.INNER_GENT_THOMAS
            elif inner == "ickan":
                widths = np.ascontiguousarray(spec.widths, dtype=np.int32)
                lo, plo = _dbl(spec.lo)
                hi, phi = _dbl(spec.hi)
                par, ppar = _dbl(spec.params)
                self._keep += [widths, lo, hi, par]
                desc.inner = _lib.INNER_ICKAN
                desc.kan_layers = int(widths.size - 1)
                desc.kan_widths = widths.ctypes.data_as(C.POINTER(C.c_int32))
                desc.kan_degree = int(spec.degree)
                desc.kan_grid = int(spec.G)
                desc.kan_lo, desc.kan_hi, desc.kan_params = plo, phi, ppar
            else:
                raise ValueError(f"unknown inner function {inner!r}")
            self._keep.append(fib)
            h = C.c_void_p()
            _lib.check("commet_model_create", lib.commet_model_create(C.byref(desc), _PREC[precision], C.byref(h)))
            self.handle = h
            self.n_params = int(lib.commet_model_n_params(h))
            return
        self.d, self.W, self.L = int(spec.d), int(spec.W), int(spec.L)
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

    def const_update_host(self, F: torch.Tensor, mesh: "Mesh | None" = None, out=None, chunk: int | None = None,
                          want_A: bool = True, want_psi: bool = True, want_f: bool = True, want_K: bool = True,
                          workspace: torch.Tensor | None = None):
        """The update (and, with a mesh, the element integrals) on HOST tensors, pipelined in
        chunks (points, or elements with a mesh) so that the copies overlap the kernels.
        F[9, n] is a CPU tensor, ideally pinned; returns CPU tensors
        (psi[n], P[9, n], A[81, n], f_e[24, n_el], K_e[576, n_el]), entries not wanted (or
        without a mesh: f_e, K_e) None. ``out`` supplies them (pinned for overlap). Complete
        when the current stream reaches the end of the call (synchronise before reading)."""
        if F.device.type != "cpu" or F.dtype != self.dtype or F.dim() != 2 or F.shape[0] != 9 \
                or not F.is_contiguous():
            raise ValueError(f"F must be a contiguous CPU tensor [9, n] of {self.dtype}")
        n = F.shape[1]
        n_el = mesh.n_el if mesh is not None else 0
        if mesh is not None and n != 8 * n_el:
            raise ValueError("F must hold the 8 points of every element of the mesh")
        if out is None:
            pin = F.is_pinned()

            def mk(*shape):
                return torch.empty(*shape, dtype=self.dtype, pin_memory=pin)
            psi = mk(n) if want_psi else None
            P, A = mk(9, n), (mk(81, n) if want_A else None)
            f_e = mk(24, n_el) if (mesh is not None and want_f) else None
            K_e = mk(576, n_el) if (mesh is not None and want_K and want_A) else None
        else:
            psi, P, A, f_e, K_e = out
        if chunk is None:
            # every strided host copy then moves rows of at least 128 KB
            es = 8 if self.dtype == torch.float64 else 4
            chunk = (131072 // es) if mesh is not None else 131072
        lib = _lib.load()
        mh = mesh.handle if mesh is not None else None
        need = int(lib.commet_const_update_host_workspace(self.handle, mh, chunk, 1 if A is not None else 0))
        if workspace is None or workspace.numel() < need:
            workspace = torch.empty(max(need, 1), dtype=torch.uint8, device="cuda")
        _lib.check("commet_const_update_host", lib.commet_const_update_host(
            self.handle, mh, n, _ptr(F), _ptr(psi), _ptr(P), _ptr(A), _ptr(f_e), _ptr(K_e), _ptr(workspace),
            workspace.numel(), chunk, _stream()))
        self._host_ws = workspace  # keeps the device buffers alive until the next call
        return psi, P, A, f_e, K_e

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
                      out=None, symmetric: bool = False):
        """(f_e[24, n_el], K_e[576, n_el], r[3 n_nodes], K_vals[nnz]); entries not wanted are None.
        ``symmetric``: A is major symmetric (the update's own tangent), K_e from its upper blocks."""
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
        name = "commet_elem_assemble_symmetric" if symmetric else "commet_elem_assemble"
        _lib.check(name, getattr(_lib.load(), name)(
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


    # ---- adjoints of the assembly chain (residual-based losses)
    def residual_adjoint(self, lam: torch.Tensor, precision: str = "f64", out=None):
        """dL/dP [9, 8 n_el] for dL/dr = lam [3 n_nodes] (dof 3 node + i)."""
        dt = _DTYPE[precision]
        _check_dev(lam, dt, shape=(3 * self.n_nodes,), name="lam")
        G = torch.empty(9, 8 * self.n_el, dtype=dt, device=lam.device) if out is None else out
        _lib.check("commet_residual_adjoint", _lib.load().commet_residual_adjoint(
            self.handle, _PREC[precision], _ptr(lam), _ptr(G), _stream()))
        return G

    def compute_F_adjoint(self, dF: torch.Tensor, precision: str = "f64", out=None):
        """dL/du [3, n_nodes] for dL/dF = dF [9, 8 n_el]."""
        dt = _DTYPE[precision]
        _check_dev(dF, dt, shape=(9, 8 * self.n_el), name="dF")
        du = torch.empty(3, self.n_nodes, dtype=dt, device=dF.device) if out is None else out
        _lib.check("commet_compute_F_adjoint", _lib.load().commet_compute_F_adjoint(
            self.handle, _PREC[precision], _ptr(dF), _ptr(du), _stream()))
        return du

    # ---- the Newton step after assembly (Sec. 4.3)
    def set_dirichlet(self, dofs):
        """Fixed dofs (3 node + i), a strictly increasing integer list; empty clears them."""
        d = np.ascontiguousarray(np.asarray(dofs, dtype=np.int64))
        self.n_fixed = int(d.size)
        _lib.check("commet_mesh_set_dirichlet", _lib.load().commet_mesh_set_dirichlet(
            self.handle, d.size, d.ctypes.data_as(C.POINTER(C.c_int64)) if d.size else None))

    def set_dirichlet_values(self, values, u: torch.Tensor, precision: str = "f64"):
        """u[:, node] <- the prescribed values of the fixed dofs (host array in dof order)."""
        _check_dev(u, _DTYPE[precision], shape=(3, self.n_nodes), name="u")
        v = np.ascontiguousarray(np.asarray(values, dtype=np.float64))
        if v.size != getattr(self, "n_fixed", 0):
            raise ValueError("one value per fixed dof is required")
        _lib.check("commet_set_dirichlet_values", _lib.load().commet_set_dirichlet_values(
            self.handle, _PREC[precision], v.ctypes.data_as(C.POINTER(C.c_double)), _ptr(u), _stream()))

    def apply_dirichlet(self, r: torch.Tensor | None, K_vals: torch.Tensor | None, precision: str = "f64",
                        delta=None):
        """Dirichlet rows and columns; ``delta`` (host, one value per fixed dof) makes the next
        update u <- u - du move the fixed dofs by delta."""
        d = None if delta is None else np.ascontiguousarray(np.asarray(delta, dtype=np.float64))
        if d is not None and d.size != getattr(self, "n_fixed", 0):
            raise ValueError("one increment per fixed dof is required")
        _lib.check("commet_apply_dirichlet", _lib.load().commet_apply_dirichlet(
            self.handle, _PREC[precision], _ptr(r), _ptr(K_vals),
            d.ctypes.data_as(C.POINTER(C.c_double)) if d is not None else None, _stream()))

    def cg_solve(self, K_vals: torch.Tensor, b: torch.Tensor, precision: str = "f64", rtol: float = 1e-10,
                 max_iter: int = 10000, x=None, workspace=None):
        """Jacobi-preconditioned CG: (x, iterations, |b - K x| / |b|)."""
        lib = _lib.load()
        dt = _DTYPE[precision]
        _check_dev(K_vals, dt, shape=(self.nnz,), name="K_vals")
        _check_dev(b, dt, shape=(3 * self.n_nodes,), name="b")
        x = torch.empty_like(b) if x is None else x
        nb = int(lib.commet_cg_workspace(self.handle, _PREC[precision]))
        if workspace is None or workspace.numel() < nb:
            workspace = torch.empty(max(nb, 1), dtype=torch.uint8, device=b.device)
        it, res = C.c_int32(0), C.c_double(0.0)
        _lib.check("commet_cg_solve", lib.commet_cg_solve(
            self.handle, _PREC[precision], _ptr(K_vals), _ptr(b), _ptr(x), float(rtol), int(max_iter),
            _ptr(workspace), nb, C.byref(it), C.byref(res), _stream()))
        return x, int(it.value), float(res.value)

    def add_increment(self, du: torch.Tensor, alpha: float, u: torch.Tensor, precision: str = "f64"):
        _lib.check("commet_add_increment", _lib.load().commet_add_increment(
            self.handle, _PREC[precision], _ptr(du), float(alpha), _ptr(u), _stream()))

    def norm2(self, x: torch.Tensor, precision: str = "f64") -> float:
        out = C.c_double(0.0)
        _lib.check("commet_norm2", _lib.load().commet_norm2(
            self.handle, _PREC[precision], x.numel(), _ptr(x), C.byref(out), _stream()))
        return float(out.value)


class Assembler:
    """u -> (r, K_vals) of a mesh: the fused Newton kernel, or compute_F + const_update +
    element integrals with the colour scatter, whichever is faster for the precision (in FP64
    the separate kernels are: the element integrals of one element per warp in the fused
    kernel cost more FP64 instructions than the element kernel's four per warp)."""

    def __init__(self, model: Model, mesh: "Mesh", fused: bool | None = None):
        self.model, self.mesh = model, mesh
        self.fused = (model.precision != "f64") if fused is None else fused
        self.r = self.Kv = None
        if not self.fused:
            n_qp, dt, dev = 8 * mesh.n_el, model.dtype, torch.device("cuda", torch.cuda.current_device())
            self.F = torch.empty(9, n_qp, dtype=dt, device=dev)
            self.P = torch.empty(9, n_qp, dtype=dt, device=dev)
            self.A = torch.empty(81, n_qp, dtype=dt, device=dev)
            self.psi = torch.empty(n_qp, dtype=dt, device=dev)

    def __call__(self, u: torch.Tensor):
        m, g = self.model, self.mesh
        if self.r is None:
            self.r = torch.empty(3 * g.n_nodes, dtype=m.dtype, device=u.device)
            self.Kv = torch.empty(g.nnz, dtype=m.dtype, device=u.device)
        if self.fused:
            newton_assemble(m, g, u, out=(self.r, self.Kv))
        else:
            g.compute_F(u, m.precision, out=self.F)
            m.const_update(self.F, out=(self.psi, self.P, self.A))
            g.elem_assemble(self.P, self.A, m.precision, want_f=False, want_K=False, want_r=True, want_Kcsr=True,
                            out=(None, None, self.r, self.Kv), symmetric=True)  # the update's own tangent
        return self.r, self.Kv


def newton_solve(model: Model, mesh: Mesh, u: torch.Tensor, steps, tol: float = 1e-10, max_newton: int = 25,
                 cg_rtol: float = 1e-10, cg_max_iter: int = 20000, fused: bool | None = None):
    """Load-stepped Newton-Raphson on the GPU (the solve of Sec. 4.3). ``steps`` is a list of
    (fixed dofs, prescribed values) per load step, the same dofs in every step. Each iteration
    assembles r and K (fused kernel), applies the Dirichlet rows and columns, solves K du = r
    by Jacobi-CG and updates u <- u - du. The first iteration of a step is the predictor: it
    moves the fixed dofs by their prescribed increment through the system (apply_dirichlet
    with delta), after which they are set to their values exactly; the step ends when
    |r_free| <= tol max(1, |r_free| after the predictor). u [3][n_nodes], updated in place,
    must hold the first step's starting state (fixed dofs included). Returns per step the
    list of (|r_free|, CG iterations of the solve that followed)."""
    prec = model.precision
    hist = []
    assemble = Assembler(model, mesh, fused)
    du = ws = None
    prev = None
    for dofs, vals in steps:
        vals = np.asarray(vals, dtype=np.float64)
        if prev is None:
            mesh.set_dirichlet(dofs)
            prev = np.zeros_like(vals)
        h = []
        for it in range(max_newton):
            r, Kv = assemble(u)
            if it == 0:
                mesh.apply_dirichlet(r, Kv, prec, delta=vals - prev)
            else:
                mesh.apply_dirichlet(r, Kv, prec)
                rn = mesh.norm2(r, prec)
                if rn <= tol * max(1.0, h[0][0] if h else rn):
                    h.append((rn, 0))
                    break
            du, n_cg, _ = mesh.cg_solve(Kv, r, prec, cg_rtol, cg_max_iter, x=du, workspace=ws)
            mesh.add_increment(du, -1.0, u, prec)
            if it == 0:
                mesh.set_dirichlet_values(vals, u, prec)
            else:
                h.append((rn, n_cg))
        prev = vals
        hist.append(h)
    return hist


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


class ComputeF(torch.autograd.Function):
    """F(u) at every Gauss point as an autograd node (Algorithm 1's trial F); backward is the
    transposed kernel. Call as ComputeF.apply(u [3, n_nodes], mesh, precision)."""

    @staticmethod
    def forward(ctx, u, mesh, precision):
        ctx.mesh, ctx.precision = mesh, precision
        return mesh.compute_F(u.contiguous(), precision)

    @staticmethod
    def backward(ctx, dF):
        return ctx.mesh.compute_F_adjoint(dF.contiguous(), ctx.precision), None, None


class AssembleResidual(torch.autograd.Function):
    """The global residual r [3 n_nodes] of eq. r-quad from P [9, 8 n_el] as an autograd node
    (element integrals and the colour scatter); backward is the transposed kernel. The mesh
    needs the CSR pattern. Call as AssembleResidual.apply(P, mesh, precision)."""

    @staticmethod
    def forward(ctx, P, mesh, precision):
        ctx.mesh, ctx.precision = mesh, precision
        _, _, r, _ = mesh.elem_assemble(P.contiguous(), None, precision, want_f=False, want_K=False, want_r=True)
        return r

    @staticmethod
    def backward(ctx, lam):
        return ctx.mesh.residual_adjoint(lam.contiguous(), ctx.precision), None, None
