"""GPU parity of the adjoints of the assembly chain and of the autograd graph of a
residual-based loss (eq. loss of App. C) against the oracle."""
import numpy as np
import pytest

import oracle
import workload as wl
from tests.parity import TOL, adjoint_u_scale, assert_close, cm_to_pm, elem_geometry, pm_to_cm, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {"f64": torch.float64, "f32": torch.float32}


@pytest.fixture(scope="module")
def pkg():
    import paper_2510_00884_gb300 as p
    p.build()
    return p


def distorted(nx, ny, nz, seed):
    mesh = wl.structured_mesh(nx, ny, nz, lengths=(1.0, 0.8, 0.6))
    rng = np.random.Generator(np.random.PCG64(seed))
    X = mesh.X + 0.02 * rng.uniform(-1, 1, size=mesh.X.shape)
    return wl.Mesh(X=X, conn=mesh.conn, n=mesh.n)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_adjoint_kernels(pkg, prec):
    mesh = distorted(5, 4, 3, 800)
    rng = np.random.Generator(np.random.PCG64(801))
    gm = pkg.Mesh(mesh.X, mesh.conn, want_csr=True)
    dt = DT[prec]
    lam = torch.from_numpy(rng.normal(size=3 * mesh.n_nodes)).to(dt).cuda()
    G = gm.residual_adjoint(lam, prec)
    G_r = oracle.residual_adjoint(mesh, lam.double().cpu().numpy().reshape(-1, 3))
    assert_close(cm_to_pm(G), G_r, TOL[prec], "dL/dP")
    dF = pm_to_cm(rng.normal(size=(8 * mesh.n_el, 9)), dt)
    du = gm.compute_F_adjoint(dF, prec)
    du_r = oracle.compute_F_adjoint(mesh, cm_to_pm(dF).astype(np.float64))
    # du at a node sums the element terms dF_iJ dphi_I,J: measured against their magnitudes
    s_u = adjoint_u_scale(mesh, cm_to_pm(dF).astype(np.float64))
    e_u = rel_err(du.double().cpu().numpy().T, du_r, s_u)
    assert e_u.max() < TOL[prec], (e_u.max(), int(e_u.argmax()))
    # deterministic (colour scatter)
    du2 = gm.compute_F_adjoint(dF, prec)
    assert torch.equal(du, du2)


def residual_chain_bounds(mesh, spec, F_r, P_r, A_r, lam, G_r, dF_r, dth_abs, fixed, t):
    """First-order bounds on the errors of the residual-loss chain
    u -> F -> P -> r (masked) = lam -> G -> (dL/dF, dL/dtheta) -> dL/du when every kernel
    is within the relative per-point tolerance t of its exact result on its own inputs
    (the per-point, per-element and per-row measures the other parity tests check).
    Each step is linear in the previous step's error, so magnitudes propagate with
    absolute values (a running error bound):
      P:      t (|P|_F + |A|_F |F|_F)                      (the update; F's rounding through A)
      r:      sum_e sum_q w (dP + t |P|_F) |dphi_I|_1        (eq. r-quad, masked)
      G:      w sum_I (dr_I + t |lam_I|) |dphi_I|            per component iJ
      dL/dF:  |A|_F (|dG|_F + t |G|_F)
      dL/du:  sum_e sum_q (d(dF) + t |dF|_F) |dphi_I|_1
      dtheta: sum_q sum_c |d dtheta_q / dG_c| dG_c + t sum_q |dtheta_q|
    The last needs the Jacobian of each point's dtheta in G, which the oracle gives
    column by column (dtheta is linear in G). Returns the bounds on r [n, 3], dL/du
    [n, 3] and dtheta [n_params], and the per-point G bound [n_qp, 9]."""
    dphi, w = elem_geometry(mesh)
    n_el = dphi.shape[0]
    conn = np.asarray(mesh.conn)
    g1 = np.abs(dphi).sum(axis=3)
    nrm = lambda a, k: np.linalg.norm(np.asarray(a).reshape(n_el, 8, k), axis=2)
    nF, nP, nA, nG, ndF = nrm(F_r, 9), nrm(P_r, 9), nrm(A_r, 81), nrm(G_r, 9), nrm(dF_r, 9)
    dP = t * (nP + nA * nF)
    n_nodes = mesh.X.shape[0]
    R = np.zeros(n_nodes)
    np.add.at(R, conn.ravel(), np.einsum("eq,eqI->eI", w * (dP + t * nP), g1).ravel())
    Rb = np.repeat(R[:, None], 3, axis=1)
    Rb[fixed] = 0.0
    lam3 = np.abs(np.asarray(lam).reshape(-1, 3))
    # per point: dG_iJ <= w sum_I (Rb_I,i + t |lam_I,i|) |dphi_I,J|
    src = (Rb + t * lam3)[conn]  # [e][I][i]
    dG = w[:, :, None, None] * np.einsum("eIi,eqIJ->eqiJ", src, np.abs(dphi))
    ddF = nA * (np.linalg.norm(dG.reshape(n_el, 8, 9), axis=2) + t * nG)
    U = np.zeros(n_nodes)
    np.add.at(U, conn.ravel(), np.einsum("eq,eqI->eI", ddF + t * ndF, g1).ravel())
    m = oracle.OracleModel(spec)
    Fq = np.asarray(F_r).reshape(-1, 9)
    dGq = dG.reshape(-1, 9)
    bth = t * np.asarray(dth_abs)
    for q in range(Fq.shape[0]):
        for c in range(9):
            e_c = np.zeros((1, 9))
            e_c[0, c] = 1.0
            _, col = oracle.const_backward(m, Fq[q:q + 1], e_c)
            bth += np.abs(col) * dGq[q, c]
    return Rb, np.repeat(U[:, None], 3, axis=1), bth, dGq


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_residual_loss_autograd(pkg, prec):
    """L = 1/2 |r_free(u; theta)|^2 through ComputeF -> ConstUpdateP -> AssembleResidual:
    torch autograd over the library's kernels gives L, dL/du and dL/dtheta equal to the
    oracle's adjoint chain (pinned by central differences) within the bounds that the
    per-point tolerance of each step propagates to (residual_chain_bounds)."""
    mesh = distorted(4, 3, 3, 802)
    rng = np.random.Generator(np.random.PCG64(803))
    spec = wl.make_model(rng, wl.KIN_RAW, 2, W=16, L=3, kappa=1.0, bias_std=0.1)
    gm = pkg.Mesh(mesh.X, mesh.conn, want_csr=True)
    m = pkg.Model(spec, prec)
    dt = DT[prec]
    u_np = 0.02 * rng.normal(size=mesh.X.shape)
    fixed = np.zeros((mesh.n_nodes, 3), dtype=bool)
    fixed[np.isclose(mesh.X[:, 0], mesh.X[:, 0].min())] = True
    mask = torch.from_numpy((~fixed).ravel().astype(np.float64)).to(dt).cuda()
    u = torch.from_numpy(np.ascontiguousarray(u_np.T)).to(dt).cuda().requires_grad_(True)
    sink = torch.zeros(m.n_params, dtype=dt, device="cuda", requires_grad=True)
    F = pkg.ComputeF.apply(u, gm, prec)
    P = pkg.ConstUpdateP.apply(F, sink, m)
    r = pkg.AssembleResidual.apply(P, gm, prec) * mask
    loss = 0.5 * (r * r).sum()
    loss.backward()
    # oracle chain at the same (rounded) inputs
    u_in = u.detach().double().cpu().numpy().T
    F_r = oracle.compute_F(mesh, u_in)
    _, P_r, A_r = oracle.const_update(oracle.OracleModel(spec), F_r)
    f_e, _ = oracle.elem_assemble(mesh, P_r, None, want_K=False)
    r_r = oracle.scatter_residual(mesh, f_e).reshape(-1, 3)
    r_r[fixed] = 0.0
    G_r = oracle.residual_adjoint(mesh, r_r)
    dF_r, dth_r, dth_abs = oracle.const_backward(oracle.OracleModel(spec), F_r, G_r, want_abs=True)
    du_r = oracle.compute_F_adjoint(mesh, dF_r)
    t = TOL[prec]
    b_r, b_u, b_th, _ = residual_chain_bounds(mesh, spec, F_r, P_r, A_r, r_r, G_r, dF_r, dth_abs, fixed, t)
    rg = r.detach().double().cpu().numpy().reshape(-1, 3)
    assert np.all(np.abs(rg - r_r) <= b_r), np.max(np.abs(rg - r_r) / np.maximum(b_r, 1e-300))
    L_r = 0.5 * (r_r * r_r).sum()
    assert abs(loss.item() - L_r) <= (np.abs(r_r) * b_r).sum() + 0.5 * (b_r ** 2).sum() + t * L_r
    gu = u.grad.double().cpu().numpy().T
    assert np.all(np.abs(gu - du_r) <= b_u), np.max(np.abs(gu - du_r) / np.maximum(b_u, 1e-300))
    gth = sink.grad.double().cpu().numpy()
    assert np.all(np.abs(gth - dth_r) <= b_th), np.max(np.abs(gth - dth_r) / np.maximum(b_th, 1e-300))


def test_residual_loss_full_size_sampled(pkg):
    """The residual-loss gradient step on the 64^3 cantilever in FP64, launched as the
    benchmark launches it; dL/du at sampled nodes (corners, faces, the clamped face,
    interior) against the oracle chain on the elements within two rings of each node (the
    only ones dL/du there depends on: r at the nodes of the node's elements is complete
    over those)."""
    import bench
    w = wl.workload_residual()
    run = bench.Run("resid", w, "f64", torch.device("cuda", 0), pkg, torch)
    run.step()
    torch.cuda.synchronize()
    du = run.du.cpu().numpy().T
    assert np.isfinite(du).all() and np.isfinite(run.dth.cpu().numpy()).all()
    n = w["mesh"].n[0]
    m = oracle.OracleModel(w["model"])
    rng = np.random.Generator(np.random.PCG64(804))
    picks = [(0, 0, 0), (n, n, n), (0, 17, 30), (n, 5, 0), (1, 1, 1), (33, 0, 12)]
    picks += [tuple(int(v) for v in rng.integers(0, n + 1, size=3)) for _ in range(6)]
    got, ref = [], []
    for (i, j, k) in picks:
        rg = [np.arange(max(0, c - 2), min(n - 1, c + 1) + 1) for c in (i, j, k)]
        ez, ey, ex = np.meshgrid(rg[2], rg[1], rg[0], indexing="ij")
        el = (ex + n * (ey + n * ez)).ravel()
        sub = wl.Mesh(X=w["mesh"].X, conn=w["mesh"].conn[el], n=w["mesh"].n)
        F = oracle.compute_F(sub, w["u"])
        _, P, _ = oracle.const_update(m, F, want_A=False)
        f_e, _ = oracle.elem_assemble(sub, P, None, want_K=False)
        lam = w["free"] * oracle.scatter_residual(sub, f_e)
        G = oracle.residual_adjoint(sub, lam.reshape(-1, 3))
        dF, _ = oracle.const_backward(m, F, G)
        node = i + (n + 1) * (j + (n + 1) * k)
        ref.append(oracle.compute_F_adjoint(sub, dF)[node])
        got.append(du[node])
    got, ref = np.array(got), np.array(ref)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
