"""Pins of the solver oracle (oracle/solver.py): Dirichlet rows and columns, Jacobi-PCG
(Sec. 4.3) and the Newton-Raphson twisting cube, against direct solves, a discrete closed
form and the convergence the methods guarantee (CPU only)."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
import workload as wl
from oracle import solver


def test_pcg_on_the_discrete_poisson_problem():
    """-u'' = 1 on (0, 1), u(0) = u(1) = 0, n interior nodes: the discrete solution is
    u_i = x_i (1 - x_i) / 2 exactly, and CG ends in at most n iterations (here n / 2, as the
    Jacobi-scaled matrix has n / 2 distinct eigenvalues pairs)."""
    n = 63
    h = 1.0 / (n + 1)
    K = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr") / h ** 2
    b = np.ones(n)
    x, it, res = solver.pcg_jacobi(K.indptr, K.indices, K.data, b, 1e-12, 1000)
    xs = np.arange(1, n + 1) * h
    assert np.abs(x - xs * (1 - xs) / 2).max() < 1e-12
    assert it <= n and res <= 1e-12


def small_system(seed=1):
    mesh = wl.structured_mesh(3)
    rng = np.random.Generator(np.random.PCG64(seed))
    spec = wl.make_model(rng, wl.KIN_POLYCONVEX, 0, W=8, L=2, kappa=0.0)
    u = 0.02 * rng.normal(size=mesh.X.shape)
    F = oracle.compute_F(mesh, u)
    _, P, A = oracle.const_update(oracle.OracleModel(spec), F)
    r, K = solver.global_system(mesh, P, A)
    return mesh, r, K


def test_dirichlet_system_equals_the_reduced_system():
    mesh, r, K = small_system()
    dofs, _ = wl.twist_dirichlet(mesh, 0.1)
    fixed = np.zeros(r.size, dtype=bool)
    fixed[dofs] = True
    vals, rb = solver.apply_dirichlet(K.indptr, K.indices, K.data, r, fixed)
    Kb = sp.csr_matrix((vals, K.indices, K.indptr), shape=K.shape)
    assert abs(Kb - Kb.T).max() <= 1e-14 * abs(Kb).max()
    x = spla.spsolve(Kb.tocsc(), rb)
    free = ~fixed
    xr = spla.spsolve(K[free][:, free].tocsc(), r[free])
    assert np.all(x[fixed] == 0.0)
    assert np.abs(x[free] - xr).max() <= 1e-12 * np.abs(xr).max()


def test_prescribed_increment_moves_the_fixed_dofs():
    """With delta, the solution of the modified system is the solution of K du = r over the
    free dofs with du_c = -delta_c substituted (the affine constraint)."""
    mesh, r, K = small_system(3)
    dofs, vals = wl.twist_dirichlet(mesh, 0.05)
    fixed = np.zeros(r.size, dtype=bool)
    fixed[dofs] = True
    delta = np.zeros(r.size)
    delta[dofs] = vals
    Kv, rb = solver.apply_dirichlet(K.indptr, K.indices, K.data, r, fixed, delta=delta)
    du = spla.spsolve(sp.csr_matrix((Kv, K.indices, K.indptr), shape=K.shape).tocsc(), rb)
    assert np.abs(du[fixed] + delta[fixed]).max() <= 1e-15 * np.abs(delta).max()
    free = ~fixed
    ref = spla.spsolve(K[free][:, free].tocsc(), r[free] - K[free][:, fixed] @ (-delta[fixed]))
    assert np.abs(du[free] - ref).max() <= 1e-11 * np.abs(ref).max()


def test_pcg_matches_the_direct_solve():
    mesh, r, K = small_system(2)
    dofs, _ = wl.twist_dirichlet(mesh, 0.1)
    fixed = np.zeros(r.size, dtype=bool)
    fixed[dofs] = True
    vals, rb = solver.apply_dirichlet(K.indptr, K.indices, K.data, r, fixed)
    x, it, res = solver.pcg_jacobi(K.indptr, K.indices, vals, rb, 1e-13, 5000)
    Kb = sp.csr_matrix((vals, K.indices, K.indptr), shape=K.shape)
    xd = spla.spsolve(Kb.tocsc(), rb)
    assert res <= 1e-13 and it < rb.size
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_newton_twist_converges_quadratically():
    """A 3^3 cube, a tenth of the benchmark's motion in two load steps, with the
    paper's NCM architecture: every step ends at |r| <= 1e-10 and the last iterations show
    the quadratic rate of Newton's method with the exact tangent."""
    mesh = wl.structured_mesh(3)
    spec = wl.workload_paper_ncm(n=1)["model"]
    u, hist = solver.newton_twist(mesh, spec, 2, tol=1e-10, stretch=0.1, turns=0.05)
    for h in hist:
        assert h[-1] <= 1e-10 * max(1.0, h[0])
        assert len(h) <= 8
        # quadratic: e_{k+1} <= C e_k^2 over the last steps before convergence
        if len(h) >= 4:
            assert h[-2] <= 10.0 * h[-3] ** 2 / max(h[0], 1.0) + 1e-12
    dofs, vals = wl.twist_dirichlet(mesh, 1.0, 0.1, 0.05)
    assert np.abs(u.ravel()[dofs] - vals).max() == 0.0


def test_twist_dirichlet_geometry():
    mesh = wl.structured_mesh(2)
    dofs, vals = wl.twist_dirichlet(mesh, 1.0)
    X = mesh.X
    nodes = dofs[::3] // 3
    u = vals.reshape(-1, 3)
    x_new = X[nodes] + u
    right = np.isclose(X[nodes, 0], 1.0)
    # half a turn about (y, z) = (1/2, 1/2) and a unit stretch: (y, z) -> (1 - y, 1 - z), x -> 2
    assert np.allclose(x_new[right, 0], 2.0)
    assert np.allclose(x_new[right, 1:], 1.0 - X[nodes[right], 1:], atol=1e-15)
    assert np.all(u[~right] == 0.0)
