"""GPU parity: every CUDA output against the FP64 oracle on the same seeded inputs.

All calls go through the C ABI (libcommet.so) via the package's thin binding.
"""
import numpy as np
import pytest

import oracle
import workload as wl
from tests.parity import TOL, assembly_scales, assert_close, blocks_rel, cm_to_pm, csr_rows_rel_err, pm_to_cm, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {"f64": torch.float64, "f32": torch.float32}


@pytest.fixture(scope="module")
def pkg():
    import paper_2510_00884_gb300 as p
    p.build()
    return p


def run_update(pkg, spec, F_pm, prec, want_A=True):
    m = pkg.Model(spec, prec)
    F = pm_to_cm(F_pm, DT[prec])
    psi, P, A, st = m.const_update(F, want_A=want_A, status=True)
    torch.cuda.synchronize()
    return (psi.cpu().numpy(), cm_to_pm(P), cm_to_pm(A) if A is not None else None, st.cpu().numpy())


def oracle_update(spec, F_pm, prec):
    Fin = np.asarray(F_pm, dtype=np.float32 if prec == "f32" else np.float64).astype(np.float64)
    return oracle.const_update(oracle.OracleModel(spec), Fin)


def check_update(pkg, spec, F_pm, prec, what):
    psi, P, A, st = run_update(pkg, spec, F_pm, prec)
    psi_r, P_r, A_r = oracle_update(spec, F_pm, prec)
    tol = TOL[prec]
    assert st[0] == 0 and st[1] == np.iinfo(np.int32).max, f"{what}: status {st}"
    scale = None
    if spec.stress_free and prec != "f64":
        # The stress-free shift subtracts n0 = dN/dK(K(I)) from dN/dK (Z8 reading of the
        # stress-free reference state): P is the difference of two O(1) gradients, so the
        # FP32 rounding scales with the unshifted stress, which is the scale used here.
        unshifted = wl.ModelSpec(**{**spec.__dict__, "stress_free": False})
        _, P_scale, _ = oracle_update(unshifted, F_pm, prec)
        scale = P_scale
    eP = assert_close(P, P_r, tol, what + " P", scale)
    eA = assert_close(A, A_r, tol, what + " A")
    epsi = assert_close(psi[:, None], psi_r[:, None], tol, what + " psi")
    return eP, eA, epsi


# ------------------------------------------------------------------ C0 (plain FP64)

def test_c0_full_chain_fp64(pkg):
    """8^3 cube: F from u, P/A/psi, f_e and K_e, all against the oracle at 1e-12."""
    w = wl.workload_c0()
    mesh, spec = w["mesh"], w["model"]
    gm = pkg.Mesh(mesh.X, mesh.conn)
    u = torch.from_numpy(np.ascontiguousarray(w["u"].T)).cuda()
    F = gm.compute_F(u, "f64")
    F_ref = oracle.compute_F(mesh, w["u"])
    assert_close(cm_to_pm(F), F_ref, TOL["f64"], "C0 F")
    m = pkg.Model(spec, "f64")
    psi, P, A, st = m.const_update(F, status=True)
    psi_r, P_r, A_r = oracle.const_update(oracle.OracleModel(spec), F_ref)
    assert st.cpu().numpy()[0] == 0
    assert_close(cm_to_pm(P), P_r, TOL["f64"], "C0 P")
    assert_close(cm_to_pm(A), A_r, TOL["f64"], "C0 A")
    assert_close(psi.cpu().numpy()[:, None], psi_r[:, None], TOL["f64"], "C0 psi")
    f_e, K_e, _, _ = gm.elem_assemble(P, A, "f64")
    f_r, K_r = oracle.elem_assemble(mesh, P_r, A_r)
    assert_close(cm_to_pm(f_e), f_r, TOL["f64"], "C0 f_e")
    assert_close(cm_to_pm(K_e), K_r.reshape(-1, 576), TOL["f64"], "C0 K_e")


# --------------------------------------------------------- shapes, both precisions

CASES = [
    # (kin, n_fib, W, L, kappa, bias, stress_free, n_qp)
    (wl.KIN_ISO_SHIFTED, 0, 16, 2, 10.0, False, False, 4099),
    (wl.KIN_RAW, 2, 32, 3, 0.0, False, False, 5003),
    (wl.KIN_ISO_SHIFTED, 0, 64, 3, 10.0, False, False, 2053),
    (wl.KIN_RAW, 1, 16, 1, 2.0, True, False, 1031),
    (wl.KIN_RAW, 2, 16, 4, 1.0, True, True, 1500),
    (wl.KIN_ISO_SHIFTED, 0, 32, 5, 3.0, True, True, 777),
    (wl.KIN_RAW, 1, 32, 2, 0.5, False, False, 7),
    # the polyconvex layer of the paper's NCMs (App. C): the 3x16 network itself, and
    # a biased, shifted variant with a volumetric penalty
    (wl.KIN_POLYCONVEX, 0, 16, 3, 0.0, False, False, 3001),
    (wl.KIN_POLYCONVEX, 0, 32, 2, 5.0, True, True, 1025),
    # the narrow networks of the paper's model-size study (App. D)
    (wl.KIN_POLYCONVEX, 0, 4, 2, 0.0, False, False, 1001),
    (wl.KIN_ISO_SHIFTED, 0, 8, 4, 5.0, True, False, 2049),
    # the widest, deepest networks of the study (W64 L4, the paper's largest): the hidden
    # weights crowd the point slabs out of shared memory and are read from global memory
    (wl.KIN_ISO_SHIFTED, 0, 64, 4, 3.0, True, False, 1537),
    (wl.KIN_RAW, 2, 64, 4, 1.0, False, False, 1029),
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("case", CASES, ids=[f"k{c[0]}f{c[1]}w{c[2]}l{c[3]}n{c[7]}" for c in CASES])
def test_const_update_shapes(pkg, case, prec):
    kin, nf, W, L, kappa, bias, sf, n = case
    rng = np.random.Generator(np.random.PCG64(100 + W + L + nf))
    spec = wl.make_model(rng, kin, nf, W=W, L=L, kappa=kappa, bias_std=0.1 if bias else None, stress_free=sf)
    F = wl.random_F(rng, n, 0.15)
    check_update(pkg, spec, F, prec, f"{case} {prec}")


def test_stress_free_reference_state(pkg):
    rng = np.random.Generator(np.random.PCG64(5))
    spec = wl.make_model(rng, wl.KIN_RAW, 2, W=32, L=3, kappa=1.0, stress_free=True)
    F = np.tile(np.eye(3).ravel(), (16, 1))
    _, P, _, _ = run_update(pkg, spec, F, "f64")
    assert np.abs(P).max() < 1e-14


# ------------------------------------------------------------------- edge cases

@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_empty_and_tiny(pkg, prec):
    """No points, and 1, 2, 8, 9 points (a part of one warp's 8-point tile and one more),
    for the update and for the backward: the backward of no points returns a zero
    dL/dtheta, and of one point the oracle's."""
    rng = np.random.Generator(np.random.PCG64(6))
    spec = wl.make_model(rng, wl.KIN_RAW, 2, W=32, L=3, kappa=0.0)
    m = pkg.Model(spec, prec)
    F0 = torch.empty(9, 0, dtype=DT[prec], device="cuda")
    psi, P, A = m.const_update(F0)
    assert P.shape == (9, 0)
    for n in (1, 2, 8, 9):
        check_update(pkg, spec, wl.random_F(rng, n, 0.15), prec, f"n={n}")
    dF0 = torch.empty(9, 0, dtype=DT[prec], device="cuda")
    dth0 = torch.full((m.n_params,), 7.0, dtype=DT[prec], device="cuda")
    m.backward(F0, torch.empty_like(F0), out=(dF0, dth0))
    torch.cuda.synchronize()
    assert bool((dth0 == 0).all())
    for n in (1, 9):
        F = wl.random_F(rng, n, 0.15)
        G = rng.normal(size=F.shape)
        Fd, Gd = pm_to_cm(F, DT[prec]), pm_to_cm(G, DT[prec])
        dF, dth = m.backward(Fd, Gd)
        Fin, Gin = cm_to_pm(Fd).astype(np.float64), cm_to_pm(Gd).astype(np.float64)
        dF_r, dth_r, dth_abs = oracle.const_backward(oracle.OracleModel(spec), Fin, Gin, want_abs=True)
        assert_close(cm_to_pm(dF), dF_r, TOL[prec], f"backward n={n} dF")
        e = blocks_rel(dth.cpu().numpy().astype(np.float64), dth_r, spec, dth_abs)
        assert e.max() < (1e-12 if prec == "f64" else 1e-4), (n, e)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_single_element_mesh(pkg, prec):
    """The smallest mesh, one distorted hex8 element: F from u, the element integrals, the
    global r and the CSR K (one 24 x 24 block) and the fused Newton kernel, against the
    oracle; every CSR row against the magnitudes of its terms (R14)."""
    mesh = wl.structured_mesh(1, 1, 1, lengths=(0.9, 1.1, 0.7))
    rng = np.random.Generator(np.random.PCG64(61))
    X = mesh.X + 0.05 * rng.uniform(-1, 1, size=mesh.X.shape)
    mesh = wl.Mesh(X=X, conn=mesh.conn, n=mesh.n)
    spec = wl.make_model(rng, wl.KIN_RAW, 2, W=32, L=3, kappa=1.0)
    gm = pkg.Mesh(mesh.X, mesh.conn, want_csr=True)
    rowptr, col = gm.csr()
    assert rowptr[-1] == 24 * 24
    dt = DT[prec]
    u = torch.from_numpy(np.ascontiguousarray((0.03 * rng.normal(size=mesh.X.shape)).T)).to(dt).cuda()
    u_in = u.double().cpu().numpy().T
    F = gm.compute_F(u, prec)
    assert_close(cm_to_pm(F), oracle.compute_F(mesh, u_in), TOL[prec], "1-element F")
    m = pkg.Model(spec, prec)
    _, P, A = m.const_update(F)
    P_in, A_in = cm_to_pm(P).astype(np.float64), cm_to_pm(A).astype(np.float64)
    f_e, K_e, r, Kv = gm.elem_assemble(P, A, prec, want_r=True, want_Kcsr=True)
    f_r, K_r = oracle.elem_assemble(mesh, P_in, A_in)
    assert_close(cm_to_pm(f_e), f_r, TOL[prec], "1-element f_e")
    assert_close(cm_to_pm(K_e), K_r.reshape(-1, 576), TOL[prec], "1-element K_e")
    r_r = oracle.scatter_residual(mesh, f_r)
    Kv_r, missing = oracle.scatter_csr(mesh, K_r, rowptr, col)
    assert missing == 0
    s_r, s_K = assembly_scales(mesh, P_in, A_in, rowptr, col)
    assert rel_err(r.double().cpu().numpy().reshape(-1, 3), r_r.reshape(-1, 3), s_r.reshape(-1, 3)).max() < TOL[prec]
    assert csr_rows_rel_err(Kv.double().cpu().numpy(), Kv_r, s_K, rowptr).max() < TOL[prec]
    # fused: u -> r, CSR K in one pass, against the oracle chain from the same u
    r2, Kv2, st = pkg.newton_assemble(m, gm, u, status=True)
    torch.cuda.synchronize()
    assert int(st[0]) == 0
    F_o = oracle.compute_F(mesh, u_in)
    _, P_o, A_o = oracle.const_update(oracle.OracleModel(spec), F_o)
    f_o, K_o = oracle.elem_assemble(mesh, P_o, A_o)
    Kv_o, _ = oracle.scatter_csr(mesh, K_o, rowptr, col)
    s_r2, s_K2 = assembly_scales(mesh, P_o, A_o, rowptr, col)
    r_o = oracle.scatter_residual(mesh, f_o)
    assert rel_err(r2.double().cpu().numpy().reshape(-1, 3), r_o.reshape(-1, 3), s_r2.reshape(-1, 3)).max() < TOL[prec]
    assert csr_rows_rel_err(Kv2.double().cpu().numpy(), Kv_o, s_K2, rowptr).max() < TOL[prec]


def test_bad_points_are_reported(pkg):
    """J <= 0 and non-finite F give NaN outputs at those points and a status count."""
    rng = np.random.Generator(np.random.PCG64(7))
    spec = wl.make_model(rng, wl.KIN_RAW, 2, W=32, L=3, kappa=0.0)
    F = wl.random_F(rng, 100, 0.15)
    F[17] = np.diag([1.0, 1.0, -1.0]).ravel()
    F[42, 3] = np.nan
    F[63] = 0.0
    psi, P, A, st = run_update(pkg, spec, F, "f64")
    assert st[0] == 3 and st[1] == 17
    for q in (17, 42, 63):
        assert np.all(np.isnan(P[q])) and np.all(np.isnan(A[q])) and np.isnan(psi[q])
    good = np.setdiff1d(np.arange(100), [17, 42, 63])
    _, P_r, A_r = oracle_update(spec, F[good], "f64")
    assert_close(P[good], P_r, 1e-12, "good points P")
    assert_close(A[good], A_r, 1e-12, "good points A")


def test_invalid_arguments(pkg):
    from paper_2510_00884_gb300 import _lib
    lib = _lib.load()
    rng = np.random.Generator(np.random.PCG64(8))
    spec = wl.make_model(rng, wl.KIN_RAW, 2, W=32, L=3, kappa=0.0)
    m = pkg.Model(spec, "f64")
    F = torch.zeros(9, 10, dtype=torch.float64, device="cuda")
    P = torch.zeros(9, 10, dtype=torch.float64, device="cuda")
    import ctypes as C
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.commet_const_update(m.handle, 10, None, None, C.c_void_p(P.data_ptr()), None, None, s) == \
        _lib.ERR_INVALID_ARG
    assert lib.commet_const_update(m.handle, -1, C.c_void_p(F.data_ptr()), None, C.c_void_p(P.data_ptr()),
                                   None, None, s) == _lib.ERR_INVALID_ARG
    assert lib.commet_const_update(m.handle, 10, C.c_void_p(F.data_ptr() + 8), None, C.c_void_p(P.data_ptr()),
                                   None, None, s) == _lib.ERR_INVALID_ARG
    spec65 = wl.make_model(rng, wl.KIN_RAW, 2, W=65, L=2, kappa=0.0)
    with pytest.raises(_lib.CommetError) as ei:
        pkg.Model(spec65, "f64")
    assert ei.value.code == _lib.ERR_UNSUPPORTED
    bad = wl.make_model(rng, wl.KIN_RAW, 2, W=32, L=3, kappa=0.0)
    bad.d = 5
    with pytest.raises(_lib.CommetError) as ei:
        pkg.Model(bad, "f64")
    assert ei.value.code == _lib.ERR_INVALID_ARG


# ------------------------------------------------------------- element assembly

@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_elem_assemble_and_csr_scatter(pkg, prec):
    """Distorted 5x4x3 mesh: F, f_e, K_e, r and the CSR values against the oracle."""
    mesh = wl.structured_mesh(5, 4, 3, lengths=(1.0, 0.8, 0.6))
    rng = np.random.Generator(np.random.PCG64(9))
    X = mesh.X + 0.02 * rng.uniform(-1, 1, size=mesh.X.shape)
    mesh = wl.Mesh(X=X, conn=mesh.conn, n=mesh.n)
    spec = wl.make_model(rng, wl.KIN_RAW, 2, W=32, L=3, kappa=1.0)
    u_np = 0.01 * rng.normal(size=mesh.X.shape)
    gm = pkg.Mesh(mesh.X, mesh.conn, want_csr=True)
    assert gm.n_colours == 8
    dt = DT[prec]
    u = torch.from_numpy(np.ascontiguousarray(u_np.T)).to(dt).cuda()
    F = gm.compute_F(u, prec)
    u_in = u.double().cpu().numpy().T
    F_r = oracle.compute_F(mesh, u_in)
    assert_close(cm_to_pm(F), F_r, TOL[prec], "F")
    m = pkg.Model(spec, prec)
    _, P, A = m.const_update(F)
    P_in, A_in = cm_to_pm(P).astype(np.float64), cm_to_pm(A).astype(np.float64)
    f_e, K_e, r, Kv = gm.elem_assemble(P, A, prec, want_r=True, want_Kcsr=True)
    f_r, K_r = oracle.elem_assemble(mesh, P_in, A_in)
    assert_close(cm_to_pm(f_e), f_r, TOL[prec], "f_e")
    assert_close(cm_to_pm(K_e), K_r.reshape(-1, 576), TOL[prec], "K_e")
    r_r = oracle.scatter_residual(mesh, f_r)
    rowptr, col = gm.csr()
    Kv_r, missing = oracle.scatter_csr(mesh, K_r, rowptr, col)
    assert missing == 0
    # per node and per CSR row against the magnitudes of their element terms (the bound
    # derived in tests/parity.py), at the path's per-point tolerance
    s_r, s_K = assembly_scales(mesh, P_in, A_in, rowptr, col)
    rr = r.cpu().numpy().astype(np.float64)
    e_r = rel_err(rr.reshape(-1, 3), r_r.reshape(-1, 3), s_r.reshape(-1, 3))
    assert e_r.max() < TOL[prec], (e_r.max(), int(e_r.argmax()))
    kk = Kv.cpu().numpy().astype(np.float64)
    e_K = csr_rows_rel_err(kk, Kv_r, s_K, rowptr)
    assert e_K.max() < TOL[prec], (e_K.max(), int(e_K.argmax()))


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n", [(5, 4, 3), (1, 1, 1), (3, 1, 2)])
def test_elem_assemble_symmetric(pkg, prec, n):
    """commet_elem_assemble_symmetric (upper node blocks of K_e for a major-symmetric A):
    on distorted meshes (ragged last CTA of 16 elements, a single element), f_e, K_e, r and
    the CSR values against the oracle's full eq. r-quad / k-quad on the same P and A (the
    update's own tangent), and K_e exactly symmetric."""
    mesh = wl.structured_mesh(*n, lengths=(1.0, 0.8, 0.6))
    rng = np.random.Generator(np.random.PCG64(19 + sum(n)))
    X = mesh.X + 0.02 * rng.uniform(-1, 1, size=mesh.X.shape)
    mesh = wl.Mesh(X=X, conn=mesh.conn, n=mesh.n)
    spec = wl.make_model(rng, wl.KIN_RAW, 2, W=32, L=3, kappa=1.0)
    gm = pkg.Mesh(mesh.X, mesh.conn, want_csr=True)
    dt = DT[prec]
    u = torch.from_numpy(np.ascontiguousarray((0.01 * rng.normal(size=mesh.X.shape)).T)).to(dt).cuda()
    F = gm.compute_F(u, prec)
    _, P, A = pkg.Model(spec, prec).const_update(F)
    P_in, A_in = cm_to_pm(P).astype(np.float64), cm_to_pm(A).astype(np.float64)
    f_e, K_e, r, Kv = gm.elem_assemble(P, A, prec, want_r=True, want_Kcsr=True, symmetric=True)
    f_e2, K_e2, _, _ = gm.elem_assemble(P, A, prec, symmetric=True)
    f_r, K_r = oracle.elem_assemble(mesh, P_in, A_in)
    for fe, Ke, what in ((f_e, K_e, "scatter launch"), (f_e2, K_e2, "plain launch")):
        assert_close(cm_to_pm(fe), f_r, TOL[prec], f"f_e {what}")
        assert_close(cm_to_pm(Ke), K_r.reshape(-1, 576), TOL[prec], f"K_e {what}")
    # the off-diagonal node blocks are written as exact transposes (the diagonal ones are
    # formed whole, symmetric to rounding)
    Kh = cm_to_pm(K_e).reshape(-1, 8, 3, 8, 3)
    for I in range(8):
        for K in range(8):
            if I != K:
                assert np.array_equal(Kh[:, I, :, K, :], np.transpose(Kh[:, K, :, I, :], (0, 2, 1))), (I, K)
    r_r = oracle.scatter_residual(mesh, f_r)
    rowptr, col = gm.csr()
    Kv_r, missing = oracle.scatter_csr(mesh, K_r, rowptr, col)
    assert missing == 0
    s_r, s_K = assembly_scales(mesh, P_in, A_in, rowptr, col)
    e_r = rel_err(r.cpu().numpy().astype(np.float64).reshape(-1, 3), r_r.reshape(-1, 3), s_r.reshape(-1, 3))
    assert e_r.max() < TOL[prec], (e_r.max(), int(e_r.argmax()))
    e_K = csr_rows_rel_err(Kv.cpu().numpy().astype(np.float64), Kv_r, s_K, rowptr)
    assert e_K.max() < TOL[prec], (e_K.max(), int(e_K.argmax()))


def test_target_stress(pkg):
    rng = np.random.Generator(np.random.PCG64(10))
    F = wl.random_F(rng, 3001, 0.15)
    tgt = oracle.OracleModel(None, inner=oracle.INNER_HGO, kin=wl.KIN_RAW, fibres=wl.FIBRES_PM30,
                             kappa=10.0, mu=1.0, k1=2.0, k2=0.5)
    _, P_r, _ = oracle.const_update(tgt, F, want_A=False)
    for prec in ("f64", "f32"):
        Fd = pm_to_cm(F, DT[prec])
        P = pkg.target_stress(Fd, wl.FIBRES_PM30, 1.0, 2.0, 0.5, 10.0)
        Fin = cm_to_pm(Fd).astype(np.float64)
        _, P_r2, _ = oracle.const_update(tgt, Fin, want_A=False)
        assert_close(cm_to_pm(P), P_r2, TOL[prec], f"target {prec}")


# ---------------------------------------------------- full-size sampled parity

def sample_idx(n, F_pm, k=1500, seed=0):
    """Strided sample plus every point with |J - 1| < 1e-3 or J < 0.8."""
    idx = np.unique(np.linspace(0, n - 1, k).astype(np.int64))
    J = np.linalg.det(F_pm.reshape(-1, 3, 3))
    special = np.nonzero((np.abs(J - 1.0) < 1e-3) | (J < 0.8))[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    if special.size > 500:
        special = rng.choice(special, 500, replace=False)
    return np.unique(np.concatenate([idx, special, [n - 1]]))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_c1_full_size_sampled(pkg, prec):
    """64^3 mesh, 2,097,152 points (the benchmark's launch): sampled points and elements."""
    w = wl.workload_c1()
    spec, mesh, F_pm = w["model"], w["mesh"], w["F"]
    n = F_pm.shape[0]
    m = pkg.Model(spec, prec)
    F = pm_to_cm(F_pm, DT[prec])
    psi, P, A, st = m.const_update(F, status=True)
    gm = pkg.Mesh(mesh.X, mesh.conn)
    f_e, K_e, _, _ = gm.elem_assemble(P, A, prec)
    torch.cuda.synchronize()
    assert st.cpu().numpy()[0] == 0
    idx = sample_idx(n, F_pm)
    Fin = F_pm[idx].astype(np.float32 if prec == "f32" else np.float64).astype(np.float64)
    psi_r, P_r, A_r = oracle.const_update(oracle.OracleModel(spec), Fin)
    it = torch.from_numpy(idx).cuda()
    assert_close(P.index_select(1, it).cpu().numpy().T, P_r, TOL[prec], "C1 P")
    assert_close(A.index_select(1, it).cpu().numpy().T, A_r, TOL[prec], "C1 A")
    el = np.unique(np.linspace(0, mesh.n_el - 1, 300).astype(np.int64))
    qp = (8 * el[:, None] + np.arange(8)[None, :]).ravel()
    qt = torch.from_numpy(qp).cuda()
    P_in = P.index_select(1, qt).cpu().numpy().T.astype(np.float64)
    A_in = A.index_select(1, qt).cpu().numpy().T.astype(np.float64)
    f_r, K_r = oracle.elem_assemble(mesh, P_in, A_in, el=el)
    et = torch.from_numpy(el).cuda()
    assert_close(f_e.index_select(1, et).cpu().numpy().T, f_r, TOL[prec], "C1 f_e")
    assert_close(K_e.index_select(1, et).cpu().numpy().T, K_r.reshape(-1, 576), TOL[prec], "C1 K_e")


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_stress_only_path(pkg, prec):
    """Without A the kernels skip the tangent pass and stage only what P needs; P agrees
    with the full path to rounding and with the oracle at the tolerance, psi exactly."""
    rng = np.random.Generator(np.random.PCG64(51))
    spec = wl.make_model(rng, wl.KIN_RAW, 2, W=32, L=3, kappa=1.0)
    F = wl.random_F(rng, 3001, 0.15)
    m = pkg.Model(spec, prec)
    Fd = pm_to_cm(F, torch.float64 if prec == "f64" else torch.float32)
    psi1, P1, A1 = m.const_update(Fd)
    psi2, P2, A2 = m.const_update(Fd, want_A=False)
    assert A2 is None
    torch.cuda.synchronize()
    # the stress-only path stages only what P needs, in a separately compiled copy of the
    # staging: the two agree to rounding (FP64 1e-14, FP32 a few ulp)
    same_tol = 1e-14 if prec == "f64" else 1e-6
    assert torch.equal(P1, P2) or (P1 - P2).abs().max().item() <= same_tol * P1.abs().max().item()
    assert torch.equal(psi1, psi2)
    _, P_r, _ = oracle.const_update(oracle.OracleModel(spec), cm_to_pm(Fd).astype(np.float64))
    assert_close(cm_to_pm(P2), P_r, TOL[prec], f"stress only {prec}")


@pytest.mark.parametrize("bias_std", [0.0, 3.0, 40.0])
def test_fp64_activation_range(pkg, bias_std):
    """Pre-activations from about -120 to 120 (biases ~ N(0, bias_std)) exercise every
    branch of the FP64 softplus evaluation; FP64 parity at 1e-12 against libm in the oracle."""
    rng = np.random.Generator(np.random.PCG64(61 + int(bias_std)))
    spec = wl.make_model(rng, wl.KIN_RAW, 2, W=32, L=3, kappa=1.0, bias_std=bias_std if bias_std else None)
    if bias_std == 0.0:
        spec.c[:] = 0.0
        spec.W1[:] *= 1e-8  # pre-activations near 0: e = exp(-|y|) near 1
    check_update(pkg, spec, wl.random_F(rng, 2000, 0.15), "f64", f"activation range {bias_std}")


# ---------------------------------------------------- the paper's polyconvex NCM

@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_polyconvex_ncm(pkg, prec):
    """MICNN 3x16 without biases on K = (Ibar1 - 3, Ibar2^{3/2} - 3^{3/2}, (J - 1)^2):
    parity on a 16^3 mesh of random F, and P(I) = 0 with A(I) != 0 (App. C)."""
    w = wl.workload_paper_ncm(n=16)
    spec = w["model"]
    check_update(pkg, spec, w["F"], prec, f"paper NCM {prec}")
    _, P, A, st = run_update(pkg, spec, np.tile(np.eye(3).ravel(), (37, 1)), prec)
    assert st[0] == 0
    assert np.abs(P).max() < (1e-14 if prec == "f64" else 1e-6)
    assert np.abs(A).max() > 1e-3


def test_polyconvex_rejects_fibres(pkg):
    from paper_2510_00884_gb300 import _lib
    rng = np.random.Generator(np.random.PCG64(9))
    spec = wl.make_model(rng, wl.KIN_RAW, 2, W=16, L=3, kappa=0.0)
    spec.kin = wl.KIN_POLYCONVEX
    with pytest.raises(_lib.CommetError) as ei:
        pkg.Model(spec, "f64")
    assert ei.value.code == _lib.ERR_INVALID_ARG


@pytest.mark.parametrize("n", [(5, 4, 3), (7, 3, 1)])
def test_elem_assemble_tiles_fp32(pkg, n):
    """Element integrals without scatter in FP32 (the kernel fed by 2D tensor copies of
    16-element tiles): ragged last tiles (60 and 21 elements), with and without K_e, against
    the oracle on the same P, A."""
    mesh = wl.structured_mesh(*n, lengths=(1.0, 0.8, 0.6))
    rng = np.random.Generator(np.random.PCG64(90 + n[2]))
    X = mesh.X + 0.02 * rng.uniform(-1, 1, size=mesh.X.shape)
    mesh = wl.Mesh(X=X, conn=mesh.conn, n=mesh.n)
    spec = wl.make_model(rng, wl.KIN_RAW, 2, W=32, L=3, kappa=1.0)
    F = wl.random_F(rng, 8 * mesh.n_el, 0.15)
    m = pkg.Model(spec, "f32")
    gm = pkg.Mesh(mesh.X, mesh.conn)
    _, P, A = m.const_update(pm_to_cm(F, torch.float32))
    f_e, K_e, _, _ = gm.elem_assemble(P, A, "f32")
    P_in, A_in = cm_to_pm(P).astype(np.float64), cm_to_pm(A).astype(np.float64)
    f_r, K_r = oracle.elem_assemble(mesh, P_in, A_in)
    assert_close(cm_to_pm(f_e), f_r, TOL["f32"], "f_e")
    assert_close(cm_to_pm(K_e), K_r.reshape(-1, 576), TOL["f32"], "K_e")
    f2, K2, _, _ = gm.elem_assemble(P, None, "f32")
    assert K2 is None
    assert_close(cm_to_pm(f2), f_r, TOL["f32"], "f_e without K")


# ------------------------------------------------ widths run zero-padded (exact)

PAD_CASES = [(wl.KIN_POLYCONVEX, 0, 2, 3), (wl.KIN_ISO_SHIFTED, 0, 5, 2), (wl.KIN_RAW, 2, 8, 2),
             (wl.KIN_RAW, 1, 24, 3), (wl.KIN_ISO_SHIFTED, 0, 40, 2)]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("case", PAD_CASES, ids=[f"k{c[0]}f{c[1]}w{c[2]}l{c[3]}" for c in PAD_CASES])
def test_padded_widths(pkg, case, prec):
    """Widths the kernels are not built for (2, 5, 24, 40, and 8 with fibres) run as the next
    built width with zero rows and columns: the update and the backward match the oracle on
    the caller's network, and dL/dtheta comes back in the caller's theta layout."""
    kin, nf, W, L = case
    rng = np.random.Generator(np.random.PCG64(700 + W))
    spec = wl.make_model(rng, kin, nf, W=W, L=L, kappa=2.0, bias_std=0.1)
    F = wl.random_F(rng, 1003, 0.15)
    check_update(pkg, spec, F, prec, f"padded {case} {prec}")
    m = pkg.Model(spec, prec)
    assert m.n_params == spec.theta().size
    G = rng.normal(size=F.shape)
    Fd, Gd = pm_to_cm(F, DT[prec]), pm_to_cm(G, DT[prec])
    from paper_2510_00884_gb300 import _lib
    try:
        dF, dth = m.backward(Fd, Gd)
    except _lib.CommetError as e:
        # a 64-wide network whose backward does not fit in shared memory
        assert W > 32 and e.code == _lib.ERR_UNSUPPORTED
        return
    Fin, Gin = cm_to_pm(Fd).astype(np.float64), cm_to_pm(Gd).astype(np.float64)
    dF_r, dth_r, dth_abs = oracle.const_backward(oracle.OracleModel(spec), Fin, Gin, want_abs=True)
    assert_close(cm_to_pm(dF), dF_r, TOL[prec], "padded dF")
    # each entry of dtheta is a sum over points: against sum_q |dtheta_q| of that entry
    e = np.abs(dth.cpu().numpy().astype(np.float64) - dth_r) / np.maximum(dth_abs, 1e-300)
    assert e.max() < (1e-12 if prec == "f64" else 1e-4), (e.max(), int(e.argmax()))
