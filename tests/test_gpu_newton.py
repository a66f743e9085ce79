"""GPU parity of the fused Newton-iteration assembly (u -> r, CSR K in one pass per colour)
against the FP64 oracle chain (F, update, element integrals, scatter in element order)."""
import numpy as np
import pytest

import oracle
import workload as wl
from tests.parity import TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {"f64": torch.float64, "f32": torch.float32}


@pytest.fixture(scope="module")
def pkg():
    import paper_2510_00884_gb300 as p
    p.build()
    return p


def oracle_chain(mesh, spec, u):
    F = oracle.compute_F(mesh, u)
    _, P, A = oracle.const_update(oracle.OracleModel(spec), F)
    f_e, K_e = oracle.elem_assemble(mesh, P, A)
    return f_e, K_e


def distorted(nx, ny, nz, seed):
    mesh = wl.structured_mesh(nx, ny, nz, lengths=(1.0, 0.7, 0.5))
    rng = np.random.Generator(np.random.PCG64(seed))
    X = mesh.X + 0.2 / nx * rng.uniform(-1, 1, size=mesh.X.shape)
    return wl.Mesh(X=X, conn=mesh.conn, n=mesh.n)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("net", ["aniso_w32", "iso_w16", "poly_w16"])
def test_newton_small_mesh(pkg, prec, net):
    mesh = distorted(6, 5, 4, 3)
    rng = np.random.Generator(np.random.PCG64(41))
    if net == "aniso_w32":
        spec = wl.make_model(rng, wl.KIN_RAW, 2, W=32, L=3, kappa=1.0)
    elif net == "iso_w16":
        spec = wl.make_model(rng, wl.KIN_ISO_SHIFTED, 0, W=16, L=2, kappa=10.0)
    else:
        spec = wl.make_model(rng, wl.KIN_POLYCONVEX, 0, W=16, L=3, kappa=0.0)
    u_np = 0.02 * rng.normal(size=mesh.X.shape)
    gm = pkg.Mesh(mesh.X, mesh.conn, want_csr=True)
    m = pkg.Model(spec, prec)
    u = torch.from_numpy(np.ascontiguousarray(u_np.T)).to(DT[prec]).cuda()
    r, Kv, st = pkg.newton_assemble(m, gm, u, status=True)
    torch.cuda.synchronize()
    assert int(st[0]) == 0
    u_in = u.double().cpu().numpy().T
    f_e, K_e = oracle_chain(mesh, spec, u_in)
    r_ref = oracle.scatter_residual(mesh, f_e)
    rowptr, col = gm.csr()
    Kv_ref, missing = oracle.scatter_csr(mesh, K_e, rowptr, col)
    assert missing == 0
    tol = (1e-12 if prec == "f64" else 1e-4)
    rr, kk = r.double().cpu().numpy(), Kv.double().cpu().numpy()
    assert np.abs(rr - r_ref).max() <= tol * np.abs(r_ref).max()
    assert np.abs(kk - Kv_ref).max() <= tol * np.abs(Kv_ref).max()
    # the unfused GPU path gives the same sums
    F = gm.compute_F(u, prec)
    _, P, A = m.const_update(F)
    _, _, r2, Kv2 = gm.elem_assemble(P, A, prec, want_f=False, want_K=False, want_r=True, want_Kcsr=True)
    tol2 = 1e-13 if prec == "f64" else 1e-5
    assert (r2 - r).abs().max().item() <= tol2 * r.abs().max().item()
    assert (Kv2 - Kv).abs().max().item() <= tol2 * Kv.abs().max().item()


def test_newton_reports_inverted_elements(pkg):
    mesh = wl.structured_mesh(3)
    rng = np.random.Generator(np.random.PCG64(42))
    spec = wl.make_model(rng, wl.KIN_RAW, 2, W=32, L=3, kappa=0.0)
    u_np = np.zeros_like(mesh.X)
    u_np[13] = [-2.0, -2.0, -2.0]  # folds the elements around node 13
    gm = pkg.Mesh(mesh.X, mesh.conn, want_csr=True)
    m = pkg.Model(spec, "f64")
    u = torch.from_numpy(np.ascontiguousarray(u_np.T)).cuda()
    r, Kv, st = pkg.newton_assemble(m, gm, u, status=True)
    torch.cuda.synchronize()
    F = oracle.compute_F(mesh, u_np)
    bad = np.nonzero(np.linalg.det(F.reshape(-1, 3, 3)) <= 0)[0]
    assert bad.size > 0
    assert int(st[0]) == bad.size and int(st[1]) == bad.min()
    assert torch.isnan(Kv).any()


def test_newton_c4_full_size_sampled(pkg):
    """96^3 cantilever (884,736 elements, 7,077,888 points, FP32, the benchmark's launch):
    r and whole CSR rows at sampled nodes against the oracle on the surrounding elements."""
    w = wl.workload_c4()
    mesh, spec, u_np = w["mesh"], w["model"], w["u"]
    gm = pkg.Mesh(mesh.X, mesh.conn, want_csr=True)
    assert gm.n_colours == 8
    m = pkg.Model(spec, "f32")
    u = torch.from_numpy(np.ascontiguousarray(u_np.T)).float().cuda()
    r, Kv, st = pkg.newton_assemble(m, gm, u, status=True)
    torch.cuda.synchronize()
    assert int(st[0]) == 0
    rowptr, col = gm.csr()
    rng = np.random.Generator(np.random.PCG64(43))
    nodes = np.unique(np.concatenate([rng.choice(mesh.n_nodes, 40, replace=False), [0, mesh.n_nodes - 1]]))
    el = np.nonzero(np.isin(mesh.conn, nodes).any(axis=1))[0]
    sub = wl.Mesh(X=mesh.X, conn=mesh.conn[el], n=mesh.n)
    u_in = u.double().cpu().numpy().T
    f_e, K_e = oracle_chain(sub, spec, u_in)
    r_ref = oracle.scatter_residual(sub, f_e).reshape(-1, 3)
    rr = r.double().cpu().numpy().reshape(-1, 3)
    kk = Kv.double().cpu().numpy()
    scale_r = np.abs(r_ref[nodes]).max()
    assert np.abs(rr[nodes] - r_ref[nodes]).max() <= 1e-4 * scale_r
    # CSR rows of the sampled nodes
    dofs = (3 * sub.conn[:, :, None] + np.arange(3)).reshape(-1, 24)
    worst = 0.0
    for n in nodes:
        for i in range(3):
            row = 3 * n + i
            cols = col[rowptr[row]:rowptr[row + 1]]
            ref = np.zeros(cols.size)
            for e_loc in np.nonzero((sub.conn == n).any(axis=1))[0]:
                a = int(np.nonzero(dofs[e_loc] == row)[0][0])
                for b in range(24):
                    ref[np.searchsorted(cols, dofs[e_loc, b])] += K_e[e_loc, a, b]
            got = kk[rowptr[row]:rowptr[row + 1]]
            worst = max(worst, np.abs(got - ref).max() / np.abs(ref).max())
    assert worst < 1e-4, worst
