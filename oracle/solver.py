"""FP64 oracle of the solve around the assembly: Dirichlet conditions on the assembled
system, the Jacobi-preconditioned conjugate gradient method of the paper's linear solves
(Sec. 4.3: conjugate gradients with Jacobi relaxation as the preconditioner), and the
Newton-Raphson load stepping of its twisting-cube benchmark (Sec. 4.3).

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's CPU legs use it;
the product path never does. Plain numpy and scipy; the element work is the C oracle's.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import compute_F, const_update, elem_assemble, OracleModel


def apply_dirichlet(rowptr, col, vals, r, fixed, delta=None):
    """Dirichlet conditions on K du = r (followed by u <- u - du): rows and columns of the
    fixed dofs zeroed with 1 on their diagonal, so the matrix stays symmetric. Without
    delta the fixed right-hand side is 0 (fixed dofs keep their value). With delta (dense
    over the dofs, read at the fixed ones) the fixed dofs move by delta: r_c = -delta_c and
    the free rows take the coupling they lose, r_f += K_fc delta_c. Returns new (vals, r)."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    n = rowptr.size - 1
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    vals = np.array(vals, dtype=np.float64, copy=True)
    r = np.array(r, dtype=np.float64, copy=True)
    if delta is not None:
        d = np.where(fixed, delta, 0.0)
        coupling = np.zeros(n)
        np.add.at(coupling, rows, vals * d[col])
        r = np.where(fixed, -d, r + coupling)
    else:
        r[fixed] = 0.0
    vals[fixed[rows] | fixed[col]] = 0.0
    vals[fixed[rows] & (rows == col)] = 1.0
    return vals, r


def pcg_jacobi(rowptr, col, vals, b, rtol: float, max_iter: int):
    """Conjugate gradients (Hestenes and Stiefel) preconditioned by the inverse diagonal,
    from x0 = 0, stopped when |b - K x| <= rtol |b| (the recursively updated residual).
    Returns (x, iterations, |r| / |b|)."""
    K = sp.csr_matrix((np.asarray(vals, dtype=np.float64), np.asarray(col), np.asarray(rowptr)))
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x, 0, 0.0
    dinv = 1.0 / K.diagonal()
    r = b.copy()
    z = dinv * r
    p = z.copy()
    rz = r @ z
    for it in range(1, max_iter + 1):
        Ap = K @ p
        alpha = rz / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        rn = np.linalg.norm(r)
        if rn <= rtol * bn:
            return x, it, rn / bn
        z = dinv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, max_iter, np.linalg.norm(r) / bn


def global_system(mesh, P, A, f_e=None, K_e=None):
    """Global residual (dof 3 node + i) and stiffness as a scipy CSR matrix, summed from the
    element integrals of the C oracle."""
    if f_e is None:
        f_e, K_e = elem_assemble(mesh, P, A)
    conn = np.asarray(mesh.conn, dtype=np.int64)
    dof = (3 * conn[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 24)
    n = 3 * mesh.n_nodes
    r = np.zeros(n)
    np.add.at(r, dof.ravel(), f_e.ravel())
    rows = np.repeat(dof, 24, axis=1).ravel()
    cols = np.tile(dof, (1, 24)).ravel()
    K = sp.csr_matrix((K_e.reshape(-1), (rows, cols)), shape=(n, n))
    K.sum_duplicates()
    K.sort_indices()
    return r, K


def newton_twist(mesh, spec, n_steps: int, tol: float = 1e-10, max_newton: int = 20, stretch: float = 1.0,
                 turns: float = 0.5):
    """Load-stepped Newton-Raphson for the twisting cube (Sec. 4.3). Per load step the first
    iteration is a predictor that moves the fixed dofs by their prescribed increment through
    the linear system (apply_dirichlet with delta), after which they hold their values
    exactly; the following iterations solve with homogeneous conditions until
    |r_free| <= tol max(1, |r_free| after the predictor). Linear solves are direct (exact).
    Returns (u[n_nodes][3], per-step residual histories after the predictor)."""
    import workload as wl
    m = OracleModel(spec)
    n = 3 * mesh.n_nodes
    u = np.zeros(n)
    prev = np.zeros(n)
    hist = []
    for s in range(1, n_steps + 1):
        dofs, vals = wl.twist_dirichlet(mesh, s / n_steps, stretch, turns)
        fixed = np.zeros(n, dtype=bool)
        fixed[dofs] = True
        target = np.zeros(n)
        target[dofs] = vals
        h = []
        for it in range(max_newton):
            F = compute_F(mesh, u.reshape(-1, 3))
            _, P, A = const_update(m, F)
            r, K = global_system(mesh, P, A)
            vals_bc, r_bc = apply_dirichlet(K.indptr, K.indices, K.data, r, fixed,
                                            delta=(target - prev) if it == 0 else None)
            if it > 0:
                rn = np.linalg.norm(r_bc)
                h.append(rn)
                if rn <= tol * max(1.0, h[0]):
                    break
            Kb = sp.csr_matrix((vals_bc, K.indices, K.indptr), shape=K.shape)
            u -= spla.spsolve(Kb.tocsc(), r_bc)
            if it == 0:
                u[dofs] = vals
        prev = target
        hist.append(h)
    return u.reshape(-1, 3), hist
