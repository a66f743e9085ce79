"""GPU parity of the Newton step after assembly (Sec. 4.3): Dirichlet rows and columns,
Jacobi-preconditioned CG and the load-stepped twisting cube, against oracle/solver.py."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
import workload as wl
from oracle import solver

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2510_00884_gb300 as p
    p.build()
    return p


def assembled(pkg, n=4, seed=1, frac=0.05):
    mesh = wl.structured_mesh(n)
    spec = wl.workload_paper_ncm(n=1)["model"]
    gm = pkg.Mesh(mesh.X, mesh.conn, want_csr=True)
    m = pkg.Model(spec, "f64")
    rng = np.random.Generator(np.random.PCG64(seed))
    u_np = 0.02 * rng.normal(size=mesh.X.shape)
    dofs, vals = wl.twist_dirichlet(mesh, frac)
    u_np.ravel()[dofs] = vals
    u = torch.from_numpy(np.ascontiguousarray(u_np.T)).cuda()
    r, Kv = pkg.newton_assemble(m, gm, u)
    return mesh, gm, m, u, r, Kv, dofs, vals


def test_dirichlet_rows_and_columns(pkg):
    mesh, gm, m, u, r, Kv, dofs, vals = assembled(pkg)
    rowptr, col = gm.csr()
    r0, K0 = r.cpu().numpy(), Kv.cpu().numpy()
    gm.set_dirichlet(dofs)
    gm.apply_dirichlet(r, Kv)
    fixed = np.zeros(r0.size, dtype=bool)
    fixed[dofs] = True
    K_r, r_r = solver.apply_dirichlet(rowptr, col, K0, r0, fixed)
    assert np.array_equal(Kv.cpu().numpy(), K_r)
    assert np.array_equal(r.cpu().numpy(), r_r)
    # prescribed increments: r_c = -delta_c, r_f += K_fc delta_c
    r2, Kv2 = pkg.newton_assemble(m, gm, u)
    gm.apply_dirichlet(r2, Kv2, delta=vals)
    dense = np.zeros(r0.size)
    dense[dofs] = vals
    K_d, r_d = solver.apply_dirichlet(rowptr, col, K0, r0, fixed, delta=dense)
    assert np.array_equal(Kv2.cpu().numpy(), K_d)
    assert np.abs(r2.cpu().numpy() - r_d).max() <= 1e-14 * np.abs(r_d).max()
    # values, increment and norm
    u2 = torch.zeros_like(u)
    gm.set_dirichlet_values(vals, u2)
    assert np.array_equal(u2.cpu().numpy().T.ravel()[dofs], vals)
    du = torch.arange(3 * mesh.n_nodes, dtype=torch.float64, device="cuda")
    gm.add_increment(du, -0.5, u2)
    ref = np.zeros(3 * mesh.n_nodes)
    ref[dofs] = vals
    ref -= 0.5 * np.arange(3 * mesh.n_nodes)
    assert np.array_equal(u2.cpu().numpy().T.ravel(), ref)
    assert abs(gm.norm2(r) - np.linalg.norm(r_r)) <= 1e-14 * np.linalg.norm(r_r)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_cg_vs_oracle(pkg, prec):
    mesh, gm, m, u, r, Kv, dofs, _ = assembled(pkg, n=5, seed=2)
    gm.set_dirichlet(dofs)
    gm.apply_dirichlet(r, Kv)
    rowptr, col = gm.csr()
    K_h, b_h = Kv.cpu().numpy(), r.cpu().numpy()
    dt = torch.float64 if prec == "f64" else torch.float32
    rtol = 1e-12 if prec == "f64" else 1e-5
    Kd, bd = Kv.to(dt), r.to(dt)
    x, it, res = gm.cg_solve(Kd, bd, prec, rtol=rtol, max_iter=5000)
    assert res <= rtol
    K_in, b_in = Kd.double().cpu().numpy(), bd.double().cpu().numpy()
    x_r, it_r, _ = solver.pcg_jacobi(rowptr, col, K_in, b_in, rtol, 5000)
    K = sp.csr_matrix((K_in, col, rowptr))
    xd = spla.spsolve(K.tocsc(), b_in)
    xg = x.double().cpu().numpy()
    if prec == "f64":
        # same recurrence in FP64: the iteration counts agree to rounding, the answers to
        # the stopping tolerance times the conditioning
        assert abs(it - it_r) <= 2
        assert np.linalg.norm(xg - xd) <= 1e-8 * np.linalg.norm(xd)
        assert np.linalg.norm(b_in - K @ xg) <= 1.5 * rtol * np.linalg.norm(b_in)
    else:
        assert np.linalg.norm(xg - xd) <= 1e-2 * np.linalg.norm(xd)
        assert np.linalg.norm(b_in - K @ xg) <= 1e-4 * np.linalg.norm(b_in)
    # deterministic: the same solve twice gives the same bits
    x2, it2, res2 = gm.cg_solve(Kd, bd, prec, rtol=rtol, max_iter=5000)
    assert torch.equal(x, x2) and it2 == it and res2 == res
    # b = 0: x = 0 in no iteration
    x0, it0, _ = gm.cg_solve(Kd, torch.zeros_like(bd), prec)
    assert it0 == 0 and torch.count_nonzero(x0) == 0


def test_newton_twist_vs_oracle(pkg):
    """The twisting cube on a 3^3 mesh with the paper's NCM (two load steps of a tenth of
    the motion): the GPU Newton with Jacobi-CG ends where the oracle's Newton with direct
    solves does."""
    mesh = wl.structured_mesh(3)
    spec = wl.workload_paper_ncm(n=1)["model"]
    u_r, hist_r = solver.newton_twist(mesh, spec, 2, tol=1e-10, stretch=0.1, turns=0.05)
    gm = pkg.Mesh(mesh.X, mesh.conn, want_csr=True)
    m = pkg.Model(spec, "f64")
    u = torch.zeros(3, mesh.n_nodes, dtype=torch.float64, device="cuda")
    steps = [wl.twist_dirichlet(mesh, s / 2, 0.1, 0.05) for s in (1, 2)]
    hist = pkg.newton_solve(m, gm, u, steps, tol=1e-10, cg_rtol=1e-12)
    for h, hr in zip(hist, hist_r):
        assert h[-1][0] <= 1e-10 * max(1.0, h[0][0])
        assert abs(len(h) - len(hr)) <= 1
        # the first residual after the predictor is the same state on both sides
        assert abs(h[0][0] - hr[0]) <= 1e-6 * hr[0]
    ug = u.cpu().numpy().T
    assert np.abs(ug - u_r).max() <= 1e-8 * np.abs(u_r).max()


def test_newton_twist_full_motion(pkg):
    """The paper's full motion (unit stretch, half turn) on a 4^3 mesh in 16 load steps:
    every step converges, and the x = 1 face ends at x = 2 turned by half a turn."""
    mesh = wl.structured_mesh(4)
    spec = wl.workload_paper_ncm(n=1)["model"]
    gm = pkg.Mesh(mesh.X, mesh.conn, want_csr=True)
    m = pkg.Model(spec, "f64")
    u = torch.zeros(3, mesh.n_nodes, dtype=torch.float64, device="cuda")
    steps = [wl.twist_dirichlet(mesh, s / 16) for s in range(1, 17)]
    hist = pkg.newton_solve(m, gm, u, steps, tol=1e-9, cg_rtol=1e-10)
    for h in hist:
        assert h[-1][0] <= 1e-9 * max(1.0, h[0][0]) and len(h) <= 25
    ug = u.cpu().numpy().T
    right = np.isclose(mesh.X[:, 0], 1.0)
    assert np.allclose((mesh.X + ug)[right, 0], 2.0)
    # the global residual at the end, from the oracle at the GPU's u
    F = oracle.compute_F(mesh, ug)
    _, P, A = oracle.const_update(oracle.OracleModel(spec), F)
    r, K = solver.global_system(mesh, P, A)
    fixed = np.zeros(r.size, dtype=bool)
    fixed[steps[-1][0]] = True
    assert np.linalg.norm(r[~fixed]) <= 1e-8 * max(1.0, hist[-1][0][0])


def test_solver_argument_checks(pkg):
    from paper_2510_00884_gb300 import _lib
    mesh = wl.structured_mesh(2)
    gm = pkg.Mesh(mesh.X, mesh.conn, want_csr=True)
    with pytest.raises(_lib.CommetError):
        gm.set_dirichlet([3, 2])          # not increasing
    with pytest.raises(_lib.CommetError):
        gm.set_dirichlet([3 * mesh.n_nodes])  # out of range
    g2 = pkg.Mesh(mesh.X, mesh.conn, want_csr=False)
    b = torch.zeros(3 * mesh.n_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.CommetError) as ei:
        g2.apply_dirichlet(b, None)
    assert ei.value.code == _lib.ERR_NO_CSR
    Kv = torch.zeros(gm.nnz, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.CommetError):
        gm.cg_solve(Kv, b, max_iter=0)


@pytest.mark.parametrize("max_iter", [16, 21, 40])
def test_cg_graph_chunks_and_tail(pkg, max_iter):
    """The solve replays chunks of 16 iterations as a CUDA graph and launches the rest
    directly: stopped by max_iter (16 = one replayed chunk, 21 = one chunk and 5 direct
    iterations, 40 = two chunks and 8), it runs exactly max_iter iterations and lands where
    the oracle's PCG does after the same number."""
    mesh, gm, m, u, r, Kv, dofs, _ = assembled(pkg, n=5, seed=3)
    gm.set_dirichlet(dofs)
    gm.apply_dirichlet(r, Kv)
    rowptr, col = gm.csr()
    x, it, res = gm.cg_solve(Kv, r, "f64", rtol=1e-30, max_iter=max_iter)
    assert it == max_iter
    x_r, it_r, res_r = solver.pcg_jacobi(rowptr, col, Kv.cpu().numpy(), r.cpu().numpy(), 1e-30, max_iter)
    assert it_r == max_iter
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - x_r) <= 1e-9 * np.linalg.norm(x_r)
    assert abs(res - res_r) <= 1e-6 * res_r
