"""GPU parity of the fused Newton-iteration assembly (u -> r, CSR K in one pass per colour)
against the FP64 oracle chain (F, update, element integrals, scatter in element order)."""
import numpy as np
import pytest

import oracle
import workload as wl
from tests.parity import TOL, assembly_scales, csr_rows_rel_err, rel_err

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
    return f_e, K_e, P, A


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
    f_e, K_e, P_r, A_r = oracle_chain(mesh, spec, u_in)
    r_ref = oracle.scatter_residual(mesh, f_e)
    rowptr, col = gm.csr()
    Kv_ref, missing = oracle.scatter_csr(mesh, K_e, rowptr, col)
    assert missing == 0
    # per node (r) and per CSR row (K) against the magnitudes of their element terms,
    # at the per-point tolerance of the path (the bound derived in tests/parity.py)
    s_r, s_K = assembly_scales(mesh, P_r, A_r, rowptr, col)
    tol = TOL[prec]
    rr, kk = r.double().cpu().numpy(), Kv.double().cpu().numpy()
    e_r = rel_err(rr.reshape(-1, 3), r_ref.reshape(-1, 3), s_r.reshape(-1, 3))
    e_K = csr_rows_rel_err(kk, Kv_ref, s_K, rowptr)
    assert e_r.max() < tol, (e_r.max(), int(e_r.argmax()))
    assert e_K.max() < tol, (e_K.max(), int(e_K.argmax()))
    # the unfused GPU path gives the same sums, row by row
    F = gm.compute_F(u, prec)
    _, P, A = m.const_update(F)
    _, _, r2, Kv2 = gm.elem_assemble(P, A, prec, want_f=False, want_K=False, want_r=True, want_Kcsr=True)
    e2_r = rel_err(r2.double().cpu().numpy().reshape(-1, 3), rr.reshape(-1, 3), s_r.reshape(-1, 3))
    e2_K = csr_rows_rel_err(Kv2.double().cpu().numpy(), kk, s_K, rowptr)
    assert e2_r.max() < tol and e2_K.max() < tol, (e2_r.max(), e2_K.max())


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
    f_e, K_e, P_r, A_r = oracle_chain(sub, spec, u_in)
    r_ref = oracle.scatter_residual(sub, f_e).reshape(-1, 3)
    Kv_ref, missing = oracle.scatter_csr(sub, K_e, rowptr, col)
    assert missing == 0
    s_r, s_K = assembly_scales(sub, P_r, A_r, rowptr, col)
    rr = r.double().cpu().numpy().reshape(-1, 3)
    kk = Kv.double().cpu().numpy()
    # r at the sampled nodes and their whole CSR rows, each against its own magnitude
    e_r = rel_err(rr[nodes], r_ref[nodes], s_r.reshape(-1, 3)[nodes])
    assert e_r.max() < TOL["f32"], (e_r.max(), int(nodes[e_r.argmax()]))
    rows = (3 * nodes[:, None] + np.arange(3)).ravel()
    e_K = csr_rows_rel_err(kk, Kv_ref, s_K, rowptr, rows)
    assert e_K.max() < TOL["f32"], (e_K.max(), int(rows[e_K.argmax()]))
