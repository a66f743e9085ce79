"""GPU parity of the spatial (Voigt) outputs and of the spatial-form element integrals
(App. A.1; eq. r-quad, k-quad) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
import workload as wl
from tests.parity import TOL, assert_close, cm_to_pm, csr_rows_rel_err, pm_to_cm, rel_err, spatial_assembly_scales

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.float32}


@pytest.fixture(scope="module")
def pkg():
    import paper_2510_00884_gb300 as p
    p.build()
    return p


NETS = {
    "aniso_w32": lambda rng: wl.make_model(rng, wl.KIN_RAW, 2, W=32, L=3, kappa=1.0),
    "iso_w64": lambda rng: wl.make_model(rng, wl.KIN_ISO_SHIFTED, 0, W=64, L=3, kappa=10.0),
    "poly_w16": lambda rng: wl.make_model(rng, wl.KIN_POLYCONVEX, 0, W=16, L=3, kappa=0.0),
    "iso_w16_shift": lambda rng: wl.make_model(rng, wl.KIN_ISO_SHIFTED, 0, W=16, L=2, kappa=3.0, bias_std=0.1,
                                               stress_free=True),
}
# (network, precision): the BF16 path is built for d3 W32/W64 and d7 W32
CASES = [(n, p) for n in ("aniso_w32", "iso_w64", "poly_w16", "iso_w16_shift") for p in ("f64", "f32")] + \
        [("aniso_w32", "bf16"), ("iso_w64", "bf16")]


@pytest.mark.parametrize("net,prec", CASES, ids=[f"{n}-{p}" for n, p in CASES])
def test_spatial_update_vs_oracle(pkg, net, prec):
    rng = np.random.Generator(np.random.PCG64(500 + len(net)))
    spec = NETS[net](rng)
    n = 3001
    F = wl.random_F(rng, n, 0.15)
    Fd = pm_to_cm(F, DT[prec])
    Fin = cm_to_pm(Fd).astype(np.float64)
    m = pkg.Model(spec, prec)
    psi, tau, c, st = m.const_update_spatial(Fd, status=True)
    torch.cuda.synchronize()
    assert int(st[0]) == 0
    psi_r, P_r, A_r = oracle.const_update(oracle.OracleModel(spec), Fin)
    tau_r, c_r = oracle.push_forward(Fin, P_r, A_r)
    scale_t = scale_c = None
    if spec.stress_free and prec != "f64":
        # the stress-free shift makes tau a difference of O(1) terms: scale by the unshifted one
        unshifted = wl.ModelSpec(**{**spec.__dict__, "stress_free": False})
        _, P_u, A_u = oracle.const_update(oracle.OracleModel(unshifted), Fin)
        scale_t, scale_c = oracle.push_forward(Fin, P_u, A_u)
    assert_close(cm_to_pm(tau), tau_r, TOL[prec], f"{net} {prec} tau", scale_t)
    assert_close(cm_to_pm(c), c_r, TOL[prec], f"{net} {prec} c", scale_c)
    assert_close(psi.cpu().numpy()[:, None], psi_r[:, None], TOL[prec], f"{net} {prec} psi")
    if prec != "bf16":
        # the material outputs of the same kernels, pushed forward on the host, agree closely
        _, P, A = m.const_update(Fd)
        tau_m, c_m = oracle.push_forward(Fin, cm_to_pm(P).astype(np.float64), cm_to_pm(A).astype(np.float64))
        assert_close(cm_to_pm(tau), tau_m, 1e-13 if prec == "f64" else 1e-6, "tau vs pushed material")
        assert_close(cm_to_pm(c), c_m, 1e-13 if prec == "f64" else 1e-6, "c vs pushed material")


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_spatial_stress_only_and_edges(pkg, prec):
    rng = np.random.Generator(np.random.PCG64(510))
    spec = NETS["iso_w64" if prec == "bf16" else "aniso_w32"](rng)
    m = pkg.Model(spec, prec)
    F0 = torch.empty(9, 0, dtype=DT[prec], device="cuda")
    _, t0, c0 = m.const_update_spatial(F0)
    assert t0.shape == (6, 0) and c0.shape == (21, 0)
    F = wl.random_F(rng, 37, 0.15)
    F[5] = np.array([1, 0, 0, 0, 1, 0, 0, 0, -1.0])  # J < 0: reported, NaN outputs
    Fd = pm_to_cm(F, DT[prec])
    psi, tau, c, st = m.const_update_spatial(Fd, status=True)
    _, tau_s, c_s, _ = m.const_update_spatial(Fd, want_c=False, status=True)
    torch.cuda.synchronize()
    assert c_s is None
    assert int(st[0]) == 1 and int(st[1]) == 5
    tt, cc = cm_to_pm(tau), cm_to_pm(c)
    assert np.all(np.isnan(tt[5])) and np.all(np.isnan(cc[5])) and np.isnan(psi[5].item())
    good = np.arange(37) != 5
    # the stress-only form stages only what tau needs (a separately compiled staging):
    # equal to rounding
    ts = cm_to_pm(tau_s)[good]
    same_tol = 1e-14 if prec == "f64" else 1e-6
    assert np.abs(ts - tt[good]).max() <= same_tol * np.abs(tt[good]).max()
    assert np.isnan(cm_to_pm(tau_s)[5]).all()
    Fin = cm_to_pm(Fd).astype(np.float64)[good]
    _, P_r, A_r = oracle.const_update(oracle.OracleModel(spec), Fin)
    tau_r, c_r = oracle.push_forward(Fin, P_r, A_r)
    assert_close(tt[good], tau_r, TOL[prec], "tau")
    assert_close(cc[good], c_r, TOL[prec], "c")


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_spatial_elem_assemble_and_scatter(pkg, prec):
    """Distorted 5x4x3 mesh: spatial f_e, K_e, r, CSR values against the oracle's spatial
    eq. r-quad / k-quad on the same tau, c; and against the material-form GPU kernel."""
    mesh = wl.structured_mesh(5, 4, 3, lengths=(1.0, 0.8, 0.6))
    rng = np.random.Generator(np.random.PCG64(520))
    X = mesh.X + 0.02 * rng.uniform(-1, 1, size=mesh.X.shape)
    mesh = wl.Mesh(X=X, conn=mesh.conn, n=mesh.n)
    spec = NETS["aniso_w32"](rng)
    u_np = 0.01 * rng.normal(size=mesh.X.shape)
    gm = pkg.Mesh(mesh.X, mesh.conn, want_csr=True)
    dt = DT[prec]
    u = torch.from_numpy(np.ascontiguousarray(u_np.T)).to(dt).cuda()
    F = gm.compute_F(u, prec)
    m = pkg.Model(spec, prec)
    _, tau, c = m.const_update_spatial(F)
    f_e, K_e, r, Kv = gm.elem_assemble_spatial(F, tau, c, prec, want_r=True, want_Kcsr=True)
    F_in, t_in, c_in = (cm_to_pm(x).astype(np.float64) for x in (F, tau, c))
    f_r, K_r = oracle.elem_assemble_spatial(mesh, F_in, t_in, c_in)
    assert_close(cm_to_pm(f_e), f_r, TOL[prec], "spatial f_e")
    assert_close(cm_to_pm(K_e), K_r.reshape(-1, 576), TOL[prec], "spatial K_e")
    r_r = oracle.scatter_residual(mesh, f_r)
    rowptr, col = gm.csr()
    Kv_r, missing = oracle.scatter_csr(mesh, K_r, rowptr, col)
    assert missing == 0
    # per node and per CSR row against the magnitudes of their element terms
    s_r, s_K = spatial_assembly_scales(mesh, F_in, t_in, c_in, rowptr, col)
    e_r = rel_err(r.double().cpu().numpy().reshape(-1, 3), r_r.reshape(-1, 3), s_r.reshape(-1, 3))
    assert e_r.max() < TOL[prec], (e_r.max(), int(e_r.argmax()))
    e_K = csr_rows_rel_err(Kv.double().cpu().numpy(), Kv_r, s_K, rowptr)
    assert e_K.max() < TOL[prec], (e_K.max(), int(e_K.argmax()))
    # same element integrals as the material form (App. A.1)
    _, P, A = m.const_update(F)
    f_m, K_m, _, _ = gm.elem_assemble(P, A, prec)
    tol_m = 1e-12 if prec == "f64" else 2e-5
    assert_close(cm_to_pm(f_e), cm_to_pm(f_m).astype(np.float64), tol_m, "f_e spatial vs material")
    assert_close(cm_to_pm(K_e), cm_to_pm(K_m).astype(np.float64), tol_m, "K_e spatial vs material")
    # stress only
    f2, K2, _, _ = gm.elem_assemble_spatial(F, tau, None, prec)
    assert K2 is None and torch.equal(f2, f_e)


def test_spatial_c1_full_size_sampled(pkg):
    """The 64^3 anisotropic workload in FP64 through the spatial entry points, in the bench's
    launch configuration; sampled points and elements against the oracle."""
    w = wl.workload_c1()
    spec, mesh = w["model"], w["mesh"]
    m = pkg.Model(spec, "f64")
    F = pm_to_cm(w["F"], torch.float64)
    _, tau, c, st = m.const_update_spatial(F, status=True)
    gm = pkg.Mesh(mesh.X, mesh.conn)
    f_e, K_e, _, _ = gm.elem_assemble_spatial(F, tau, c, "f64")
    torch.cuda.synchronize()
    assert int(st[0]) == 0
    rng = np.random.Generator(np.random.PCG64(530))
    el = np.sort(rng.choice(mesh.n_el, 64, replace=False))
    el[-1] = mesh.n_el - 1
    qp = (8 * el[:, None] + np.arange(8)[None, :]).ravel()
    Fs = w["F"][qp]
    _, P_r, A_r = oracle.const_update(oracle.OracleModel(spec), Fs)
    tau_r, c_r = oracle.push_forward(Fs, P_r, A_r)
    idx = torch.from_numpy(qp).cuda()
    assert_close(cm_to_pm(tau[:, idx]), tau_r, 1e-12, "C1 tau")
    assert_close(cm_to_pm(c[:, idx]), c_r, 1e-12, "C1 c")
    f_r, K_r = oracle.elem_assemble_spatial(mesh, Fs, tau_r, c_r, el=el)
    eidx = torch.from_numpy(el).cuda()
    assert_close(cm_to_pm(f_e[:, eidx]), f_r, 1e-12, "C1 f_e")
    assert_close(cm_to_pm(K_e[:, eidx]), K_r.reshape(-1, 576), 1e-12, "C1 K_e")
