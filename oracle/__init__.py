"""ctypes front end of the FP64 CPU oracle (``commet_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` are the only callers. The product path never imports this package.

Layouts here are qp-major (F[n][9], P[n][9], A[n][81]) and element-major
(f_e[n_el][24], K_e[n_el][24][24]), all float64.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "commet_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

INNER_MICNN, INNER_GENT_THOMAS, INNER_HGO, INNER_CANN, INNER_ICKAN = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", _SRC,
                               "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Model(C.Structure):
    _fields_ = [("d", C.c_int), ("W", C.c_int), ("L", C.c_int), ("kin", C.c_int),
                ("n_fib", C.c_int), ("fib", C.POINTER(C.c_double)), ("inner", C.c_int),
                ("W1", C.POINTER(C.c_double)), ("Ak", C.POINTER(C.c_double)),
                ("Bk", C.POINTER(C.c_double)), ("c", C.POINTER(C.c_double)),
                ("a", C.POINTER(C.c_double)), ("b", C.POINTER(C.c_double)),
                ("kappa", C.c_double), ("stress_free", C.c_int),
                ("mu", C.c_double), ("k1", C.c_double), ("k2", C.c_double),
                ("cann_n", C.c_int), ("cann_kind", C.POINTER(C.c_int)), ("cann_w", C.POINTER(C.c_double)),
                ("kan_R", C.c_int), ("kan_deg", C.c_int), ("kan_G", C.c_int), ("kan_w", C.POINTER(C.c_int)),
                ("kan_lo", C.POINTER(C.c_double)), ("kan_hi", C.POINTER(C.c_double)),
                ("kan_par", C.POINTER(C.c_double))]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.POINTER
        d, i64, i32 = P(C.c_double), C.c_int64, P(C.c_int32)
        _lib.oracle_const_update.argtypes = [P(_Model), i64, d, d, d, d]
        _lib.oracle_const_update.restype = C.c_int
        _lib.oracle_kinematics_at.argtypes = [P(_Model), d, d, d, d]
        _lib.oracle_kinematics_at.restype = C.c_int
        _lib.oracle_inner.argtypes = [P(_Model), d, d, d, d]
        _lib.oracle_hex8_gradients.argtypes = [d, d, d]
        _lib.oracle_compute_F.argtypes = [i64, i32, d, d, d]
        _lib.oracle_elem_assemble.argtypes = [i64, i32, d, d, d, d, d]
        _lib.oracle_scatter_residual.argtypes = [i64, i32, d, i64, d]
        _lib.oracle_residual_adjoint.argtypes = [i64, i32, d, d, d]
        _lib.oracle_compute_F_adjoint.argtypes = [i64, i32, d, d, i64, d]
        _lib.oracle_kan_basis.argtypes = [P(_Model), C.c_int, C.c_double, d, d, d]
        _lib.oracle_kan_basis.restype = C.c_int
        _lib.oracle_push_forward.argtypes = [d, d, d, d, d]
        _lib.oracle_elem_assemble_spatial.argtypes = [i64, i32, d, d, d, d, d, d]
        _lib.oracle_scatter_csr.argtypes = [i64, i32, d, i64, P(C.c_int64), i32, d]
        _lib.oracle_scatter_csr.restype = C.c_int64
        _lib.oracle_n_params.argtypes = [C.c_int, C.c_int, C.c_int]
        _lib.oracle_n_params.restype = C.c_int64
        _lib.oracle_const_backward.argtypes = [P(_Model), i64, d, d, d, d, d]
        _lib.oracle_const_backward.restype = C.c_int
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleModel:
    """Holds contiguous float64 copies of a model's arrays and the C struct pointing at them."""

    def __init__(self, spec=None, inner: int = INNER_MICNN, kin: int | None = None,
                 fibres=None, kappa: float | None = None, mu=1.0, k1=2.0, k2=0.5,
                 stress_free: bool | None = None):
        self.kind = self.cw = None
        self.kan = None
        cann_n = 0
        if spec is not None and getattr(spec, "inner_name", "micnn") != "micnn":
            # closed-form and CANN inner functions: no network arrays
            inner = {"cann": INNER_CANN, "gent_thomas": INNER_GENT_THOMAS, "ickan": INNER_ICKAN}[spec.inner_name]
            kin = spec.kin if kin is None else kin
            fibres = spec.fibres if fibres is None else fibres
            kappa = spec.kappa if kappa is None else kappa
            stress_free = spec.stress_free if stress_free is None else stress_free
            d, W, L = spec.d, 1, 1
            self.arrs = {"W1": np.zeros((1, d)), "Ak": np.zeros(1), "Bk": np.zeros(1),
                         "c": np.zeros((1, 1)), "a": np.zeros(1), "b": np.zeros(d)}
            if spec.inner_name == "cann":
                cann_n = int(spec.n)
                self.kind = np.ascontiguousarray(spec.kinds, dtype=np.int32).reshape(cann_n, 3)
                self.cw = _c64(spec.w).reshape(d, cann_n, 2)
            if spec.inner_name == "ickan":
                self.kan = {"w": np.ascontiguousarray(spec.widths, dtype=np.int32), "lo": _c64(spec.lo),
                            "hi": _c64(spec.hi), "par": _c64(spec.params)}
                self.kan_meta = (len(spec.widths) - 1, int(spec.degree), int(spec.G))
        elif spec is not None:
            d, W, L = spec.d, spec.W, spec.L
            kin = spec.kin if kin is None else kin
            fibres = spec.fibres if fibres is None else fibres
            kappa = spec.kappa if kappa is None else kappa
            stress_free = spec.stress_free if stress_free is None else stress_free
            self.arrs = {k: _c64(getattr(spec, k)) for k in ("W1", "Ak", "Bk", "c", "a", "b")}
        else:
            fibres = np.zeros((0, 3)) if fibres is None else fibres
            d = 3 + 2 * len(fibres) if kin == 1 else 3
            W, L = 1, 1
            self.arrs = {"W1": np.zeros((1, d)), "Ak": np.zeros(1), "Bk": np.zeros(1),
                         "c": np.zeros((1, 1)), "a": np.zeros(1), "b": np.zeros(d)}
            kappa = 0.0 if kappa is None else kappa
            stress_free = bool(stress_free)
        self.fib = _c64(np.asarray(fibres).reshape(-1, 3)) if len(fibres) else np.zeros((1, 3))
        self.d, self.W, self.L = d, W, L
        self.s = _Model(d=d, W=W, L=L, kin=int(kin), n_fib=int(len(fibres)), fib=_dp(self.fib),
                        inner=int(inner), W1=_dp(self.arrs["W1"]), Ak=_dp(self.arrs["Ak"]),
                        Bk=_dp(self.arrs["Bk"]), c=_dp(self.arrs["c"]), a=_dp(self.arrs["a"]),
                        b=_dp(self.arrs["b"]), kappa=float(kappa), stress_free=int(bool(stress_free)),
                        mu=float(mu), k1=float(k1), k2=float(k2), cann_n=cann_n,
                        cann_kind=self.kind.ctypes.data_as(C.POINTER(C.c_int)) if self.kind is not None else None,
                        cann_w=_dp(self.cw))
        if self.kan is not None:
            R, k, G = self.kan_meta
            self.s.kan_R, self.s.kan_deg, self.s.kan_G = R, k, G
            self.s.kan_w = self.kan["w"].ctypes.data_as(C.POINTER(C.c_int))
            self.s.kan_lo, self.s.kan_hi, self.s.kan_par = _dp(self.kan["lo"]), _dp(self.kan["hi"]), _dp(self.kan["par"])


def const_update(model: OracleModel, F: np.ndarray, want_A: bool = True):
    """Psi[n], P[n][9], A[n][81] (A None if not wanted) for F[n][9]."""
    lib = _load()
    F = _c64(F).reshape(-1, 9)
    n = F.shape[0]
    psi = np.empty(n)
    P = np.empty((n, 9))
    A = np.empty((n, 81)) if want_A else None
    rc = lib.oracle_const_update(C.byref(model.s), n, _dp(F), _dp(psi), _dp(P), _dp(A))
    if rc != 0:
        raise RuntimeError(f"oracle_const_update rc={rc}")
    return psi, P, A


def kinematics(model: OracleModel, F: np.ndarray):
    """K[d], dK[d][9], d2K[d][81] at one F."""
    lib = _load()
    F = _c64(F).reshape(9)
    K = np.zeros(16)
    dK = np.zeros((16, 9))
    d2K = np.zeros((16, 81))
    d = lib.oracle_kinematics_at(C.byref(model.s), _dp(F), _dp(K), _dp(dK), _dp(d2K))
    return K[:d], dK[:d], d2K[:d]


def inner(model: OracleModel, K: np.ndarray):
    """Inner function value N, gradient dN[d], Hessian d2N[d][d] at K (Algorithm 4 for MICNN)."""
    lib = _load()
    K = _c64(K)
    d = K.size
    N = np.zeros(1)
    dN = np.zeros(d)
    d2N = np.zeros((d, d))
    lib.oracle_inner(C.byref(model.s), _dp(K), _dp(N), _dp(dN), _dp(d2N))
    return N[0], dN, d2N


def kan_basis(model: OracleModel, r: int, x: float):
    """B-spline basis functions of ICKAN layer r at x and their first and second derivatives."""
    lib = _load()
    nb = model.kan_meta[2] + model.kan_meta[1]
    B, dB, d2B = np.zeros(nb + 8), np.zeros(nb + 8), np.zeros(nb + 8)
    n = lib.oracle_kan_basis(C.byref(model.s), r, float(x), _dp(B), _dp(dB), _dp(d2B))
    return B[:n], dB[:n], d2B[:n]


def hex8_gradients(Xe: np.ndarray):
    """dphi[8 qp][8 nodes][3] and w[8] for one element with node coordinates Xe[8][3]."""
    lib = _load()
    Xe = _c64(Xe).reshape(8, 3)
    dphi = np.zeros((8, 8, 3))
    w = np.zeros(8)
    lib.oracle_hex8_gradients(_dp(Xe), _dp(dphi), _dp(w))
    return dphi, w


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def compute_F(mesh, u: np.ndarray) -> np.ndarray:
    """F[n_el*8][9] from nodal displacements u[n_nodes][3]."""
    lib = _load()
    conn = np.ascontiguousarray(mesh.conn, dtype=np.int32)
    X = _c64(mesh.X)
    u = _c64(u)
    F = np.empty((8 * conn.shape[0], 9))
    lib.oracle_compute_F(conn.shape[0], _ip(conn), _dp(X), _dp(u), _dp(F))
    return F


def elem_assemble(mesh, P: np.ndarray, A: np.ndarray | None, want_K: bool = True, el=None):
    """f_e[n][24], K_e[n][24][24] for the elements ``el`` (all if None); P, A are the
    qp tables of those elements (element e's qp at rows 8e..8e+7 of the subset)."""
    lib = _load()
    conn = np.ascontiguousarray(mesh.conn if el is None else mesh.conn[el], dtype=np.int32)
    X = _c64(mesh.X)
    n = conn.shape[0]
    P = _c64(P)
    A = _c64(A) if A is not None else None
    f = np.empty((n, 24))
    K = np.empty((n, 24, 24)) if (want_K and A is not None) else None
    lib.oracle_elem_assemble(n, _ip(conn), _dp(X), _dp(P), _dp(A), _dp(f), _dp(K))
    return f, K


VOIGT = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))


def push_forward(F: np.ndarray, P: np.ndarray, A: np.ndarray | None):
    """Kirchhoff stress tau[n][6] (Voigt 11 22 33 23 13 12) and spatial stiffness c[n][21]
    (upper triangle of the 6 x 6 Voigt matrix, row-major) per point (App. A.1)."""
    lib = _load()
    F, P = _c64(F).reshape(-1, 9), _c64(P).reshape(-1, 9)
    n = F.shape[0]
    A = _c64(A).reshape(n, 81) if A is not None else None
    tau = np.empty((n, 6))
    c = np.empty((n, 21)) if A is not None else None
    for q in range(n):
        lib.oracle_push_forward(_dp(F[q]), _dp(P[q]), _dp(A[q]) if A is not None else None, _dp(tau[q]),
                                _dp(c[q]) if c is not None else None)
    return tau, c


def elem_assemble_spatial(mesh, F: np.ndarray, tau: np.ndarray, c: np.ndarray | None, el=None):
    """f_e[n][24], K_e[n][24][24] from F, tau, c by the spatial eq. r-quad / k-quad."""
    lib = _load()
    conn = np.ascontiguousarray(mesh.conn if el is None else mesh.conn[el], dtype=np.int32)
    X = _c64(mesh.X)
    n = conn.shape[0]
    F, tau = _c64(F), _c64(tau)
    c = _c64(c) if c is not None else None
    f = np.empty((n, 24))
    K = np.empty((n, 24, 24)) if c is not None else None
    lib.oracle_elem_assemble_spatial(n, _ip(conn), _dp(X), _dp(F), _dp(tau), _dp(c), _dp(f), _dp(K))
    return f, K


def residual_adjoint(mesh, lam: np.ndarray) -> np.ndarray:
    """dL/dP [n_qp][9] for dL/dr = lam [n_nodes][3] (transpose of eq. r-quad and the scatter)."""
    lib = _load()
    conn = np.ascontiguousarray(mesh.conn, dtype=np.int32)
    G = np.empty((8 * conn.shape[0], 9))
    lib.oracle_residual_adjoint(conn.shape[0], _ip(conn), _dp(_c64(mesh.X)), _dp(_c64(lam)), _dp(G))
    return G


def compute_F_adjoint(mesh, dF: np.ndarray) -> np.ndarray:
    """dL/du [n_nodes][3] for dL/dF = dF [n_qp][9] (transpose of the trial F)."""
    lib = _load()
    conn = np.ascontiguousarray(mesh.conn, dtype=np.int32)
    du = np.empty((mesh.n_nodes, 3))
    lib.oracle_compute_F_adjoint(conn.shape[0], _ip(conn), _dp(_c64(mesh.X)), _dp(_c64(dF)), mesh.n_nodes, _dp(du))
    return du


def scatter_residual(mesh, f_e: np.ndarray) -> np.ndarray:
    lib = _load()
    conn = np.ascontiguousarray(mesh.conn, dtype=np.int32)
    r = np.empty(3 * mesh.n_nodes)
    lib.oracle_scatter_residual(conn.shape[0], _ip(conn), _dp(_c64(f_e)), mesh.n_nodes, _dp(r))
    return r


def scatter_csr(mesh, K_e: np.ndarray, rowptr: np.ndarray, col: np.ndarray):
    """CSR values of the global K for the caller's pattern; returns (vals, missing)."""
    lib = _load()
    conn = np.ascontiguousarray(mesh.conn, dtype=np.int32)
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    vals = np.empty(int(rowptr[-1]))
    missing = lib.oracle_scatter_csr(conn.shape[0], _ip(conn), _dp(_c64(K_e)), rowptr.size - 1,
                                     rowptr.ctypes.data_as(C.POINTER(C.c_int64)), _ip(col), _dp(vals))
    return vals, int(missing)


def n_params(d: int, W: int, L: int) -> int:
    return int(_load().oracle_n_params(d, W, L))


def const_backward(model: OracleModel, F: np.ndarray, G: np.ndarray, want_abs: bool = False):
    """dL/dF[n][9] and dL/dtheta[n_params] for upstream G = dL/dP [n][9]. With ``want_abs``
    also sum_q |dL/dtheta of point q| per entry: the magnitude the floating-point sum over
    points is rounded against. Points run on all OpenMP threads in contiguous blocks whose
    sums are added in thread order."""
    lib = _load()
    F = _c64(F).reshape(-1, 9)
    G = _c64(G).reshape(-1, 9)
    n = F.shape[0]
    dF = np.empty((n, 9))
    npar = model.cw.size if model.cw is not None else n_params(model.d, model.W, model.L)
    dth = np.empty(npar)
    dabs = np.empty(npar) if want_abs else None
    rc = lib.oracle_const_backward(C.byref(model.s), n, _dp(F), _dp(G), _dp(dF), _dp(dth), _dp(dabs))
    if rc != 0:
        raise RuntimeError(f"oracle_const_backward rc={rc}")
    return (dF, dth, dabs) if want_abs else (dF, dth)
