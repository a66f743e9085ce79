"""GPU parity of the inner functions other than the MICNN: the CANN of eq. cann-def and
the closed-form Gent-Thomas energy of eq. gt, in both output forms, against the oracle."""
import dataclasses

import numpy as np
import pytest

import oracle
import workload as wl
from tests.parity import TOL, assert_close, cm_to_pm, pm_to_cm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {"f64": torch.float64, "f32": torch.float32}

ALL_KINDS = np.array([[wl.CANN_F0_ID, 1, wl.CANN_F2_LINEAR], [wl.CANN_F0_ID, 2, wl.CANN_F2_EXP],
                      [wl.CANN_F0_MACAULAY, 3, wl.CANN_F2_LINEAR], [wl.CANN_F0_ABS, 2, wl.CANN_F2_LOG],
                      [wl.CANN_F0_ABS, 1, wl.CANN_F2_EXP], [wl.CANN_F0_MACAULAY, 2, wl.CANN_F2_LOG]],
                     dtype=np.int32)


@pytest.fixture(scope="module")
def pkg():
    import paper_2510_00884_gb300 as p
    p.build()
    return p


def specs():
    rng = np.random.Generator(np.random.PCG64(600))
    return {
        "cann_paper_poly": wl.make_cann(rng),
        "cann_all_raw2": wl.make_cann(rng, wl.KIN_RAW, 2, kinds=ALL_KINDS, kappa=1.0, std=0.005),
        "cann_all_iso_shift": wl.make_cann(rng, wl.KIN_ISO_SHIFTED, 0, kinds=ALL_KINDS, kappa=5.0, std=0.2,
                                           stress_free=True),
        "cann_all_raw1": wl.make_cann(rng, wl.KIN_RAW, 1, kinds=ALL_KINDS[:5], kappa=0.0, std=0.005),
        "gent_thomas": wl.GentThomasSpec(),
        "ickan_k4_poly": wl.make_ickan(rng),
        "ickan_k2_iso": wl.make_ickan(rng, kin=wl.KIN_ISO_SHIFTED, widths=(3, 5, 1), degree=2, G=16, lo0=-0.8,
                                      kappa=3.0),
        "ickan_k3_iso_shift": dataclasses.replace(
            wl.make_ickan(rng, kin=wl.KIN_ISO_SHIFTED, widths=(3, 8, 3, 2, 1), degree=3, G=20, lo0=-0.8, kappa=1.0),
            stress_free=True),
    }


SPECS = specs()


def check(pkg, spec, F, prec, what):
    Fd = pm_to_cm(F, DT[prec])
    Fin = cm_to_pm(Fd).astype(np.float64)
    m = pkg.Model(spec, prec)
    psi, P, A, st = m.const_update(Fd, status=True)
    psi_s, tau, c, st_s = m.const_update_spatial(Fd, status=True)
    torch.cuda.synchronize()
    assert int(st[0]) == 0 and int(st_s[0]) == 0
    psi_r, P_r, A_r = oracle.const_update(oracle.OracleModel(spec), Fin)
    scale = None
    if spec.stress_free and prec != "f64":
        _, scale, _ = oracle.const_update(oracle.OracleModel(dataclasses.replace(spec, stress_free=False)), Fin)
    assert_close(cm_to_pm(P), P_r, TOL[prec], f"{what} P", scale)
    assert_close(cm_to_pm(A), A_r, TOL[prec], f"{what} A")
    assert_close(psi.cpu().numpy()[:, None], psi_r[:, None], TOL[prec], f"{what} psi")
    tau_r, c_r = oracle.push_forward(Fin, P_r, A_r)
    tscale = None if scale is None else oracle.push_forward(Fin, scale, None)[0]
    assert_close(cm_to_pm(tau), tau_r, TOL[prec], f"{what} tau", tscale)
    assert_close(cm_to_pm(c), c_r, TOL[prec], f"{what} c")
    assert torch.equal(psi, psi_s)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("name", list(SPECS))
def test_inner_vs_oracle(pkg, name, prec):
    rng = np.random.Generator(np.random.PCG64(610))
    F = wl.random_F(rng, 2053, 0.15)
    check(pkg, SPECS[name], F, prec, f"{name} {prec}")


def test_cann_parameter_count_and_stress_free(pkg):
    spec = SPECS["cann_paper_poly"]
    m = pkg.Model(spec, "f64")
    assert m.n_params == 24
    F = torch.eye(3, dtype=torch.float64).reshape(9, 1).repeat(1, 17).cuda().contiguous()
    _, P, _ = m.const_update(F)
    assert P.abs().max().item() < 1e-15


def test_cann_log_domain_is_reported(pkg):
    """-ln(1 - w1 y) with w1 y >= 1 has no value: such points are reported and NaN."""
    w = np.zeros((3, 1, 2))
    w[0, 0] = (2.0, 1.0)
    spec = wl.CannSpec(d=3, kin=wl.KIN_ISO_SHIFTED, fibres=np.zeros((0, 3)), n=1,
                       kinds=np.array([[wl.CANN_F0_ID, 1, wl.CANN_F2_LOG]], dtype=np.int32), w=w)
    F = np.tile(np.eye(3).ravel(), (8, 1))
    F[3] = np.diag([2.0, 1.0, 1.0]).ravel()  # Ibar1 - 3 ~ 0.78: w1 y > 1
    m = pkg.Model(spec, "f64")
    psi, P, A, st = m.const_update(pm_to_cm(F, torch.float64), status=True)
    torch.cuda.synchronize()
    assert int(st[0]) == 1 and int(st[1]) == 3
    assert torch.isnan(P[:, 3]).all() and torch.isnan(psi[3])
    good = [q for q in range(8) if q != 3]
    assert torch.isfinite(P[:, good]).all()


def test_unsupported_paths(pkg):
    from paper_2510_00884_gb300 import _lib
    spec = SPECS["cann_paper_poly"]
    with pytest.raises(_lib.CommetError) as ei:
        pkg.Model(spec, "bf16")
    assert ei.value.code == _lib.ERR_UNSUPPORTED
    m = pkg.Model(spec, "f64")
    F = torch.eye(3, dtype=torch.float64).reshape(9, 1).repeat(1, 8).cuda().contiguous()
    # the closed-form Gent-Thomas energy has no parameters to differentiate: no backward
    with pytest.raises(_lib.CommetError) as ei:
        pkg.Model(SPECS["gent_thomas"], "f64").backward(F, torch.zeros_like(F))
    assert ei.value.code == _lib.ERR_UNSUPPORTED
    # nor a stress-free CANN (its shift n0 depends on the weights)
    with pytest.raises(_lib.CommetError) as ei:
        pkg.Model(SPECS["cann_all_iso_shift"], "f64").backward(F, torch.zeros_like(F))
    assert ei.value.code == _lib.ERR_UNSUPPORTED
    mesh = wl.structured_mesh(1)
    gm = pkg.Mesh(mesh.X, mesh.conn, want_csr=True)
    u = torch.zeros(3, mesh.n_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.CommetError) as ei:
        pkg.newton_assemble(m, gm, u)
    assert ei.value.code == _lib.ERR_UNSUPPORTED
    bad = wl.GentThomasSpec(kin=wl.KIN_ISO_SHIFTED)
    with pytest.raises(_lib.CommetError) as ei:
        pkg.Model(bad, "f64")
    assert ei.value.code == _lib.ERR_INVALID_ARG
    kinds = np.array([[0, 4, 0]], dtype=np.int32)  # exponent 4 is not in the menu
    with pytest.raises(_lib.CommetError) as ei:
        pkg.Model(wl.CannSpec(d=3, kin=wl.KIN_POLYCONVEX, fibres=np.zeros((0, 3)), n=1, kinds=kinds,
                              w=np.ones((3, 1, 2))), "f64")
    assert ei.value.code == _lib.ERR_INVALID_ARG


def test_ickan_parameter_count(pkg):
    spec = SPECS["ickan_k4_poly"]
    m = pkg.Model(spec, "f64")
    assert m.n_params == spec.params.size == (12 + 16 + 4) * (1 + 30 + 4)


@pytest.mark.parametrize("name", ["cann_polyconvex", "gent_thomas", "ickan"])
def test_full_size_sampled(pkg, name):
    """The 64^3 CANN and Gent-Thomas workloads in FP64 as the bench launches them; sampled
    points (including the last) against the oracle."""
    w = {"cann_polyconvex": wl.workload_cann, "gent_thomas": wl.workload_gent_thomas,
         "ickan": wl.workload_ickan}[name]()
    spec = w["model"]
    m = pkg.Model(spec, "f64")
    F = pm_to_cm(w["F"], torch.float64)
    _, P, A, st = m.const_update(F, status=True)
    torch.cuda.synchronize()
    assert int(st[0]) == 0
    n = w["F"].shape[0]
    rng = np.random.Generator(np.random.PCG64(620))
    qp = np.sort(rng.choice(n, 512, replace=False))
    qp[-1] = n - 1
    _, P_r, A_r = oracle.const_update(oracle.OracleModel(spec), w["F"][qp])
    idx = torch.from_numpy(qp).cuda()
    assert_close(cm_to_pm(P[:, idx]), P_r, 1e-12, f"{name} P")
    assert_close(cm_to_pm(A[:, idx]), A_r, 1e-12, f"{name} A")


# ------------------------------------------------------------ backward of the CANN

BW_SPECS = {
    "cann_paper_poly": SPECS["cann_paper_poly"],
    "cann_all_raw2": SPECS["cann_all_raw2"],
    "cann_all_raw1": SPECS["cann_all_raw1"],
    "cann_all_iso": dataclasses.replace(SPECS["cann_all_iso_shift"], stress_free=False),
}


def cann_backward_check(pkg, spec, F, G, prec, what):
    """dL/dF per point at the path's tolerance; dL/dw per weight against the sum of the
    per-point terms' magnitudes (a floating-point sum's bound), 1e-12 in FP64 and 1e-4 in
    FP32, against the oracle on the same (rounded) inputs."""
    m = pkg.Model(spec, prec)
    Fd, Gd = pm_to_cm(F, DT[prec]), pm_to_cm(G, DT[prec])
    dF, dth = m.backward(Fd, Gd)
    dF2, dth2 = m.backward(Fd, Gd)
    torch.cuda.synchronize()
    assert torch.equal(dth, dth2) and torch.equal(dF, dF2), "backward not deterministic"
    Fin, Gin = cm_to_pm(Fd).astype(np.float64), cm_to_pm(Gd).astype(np.float64)
    dF_r, dth_r, dth_abs = oracle.const_backward(oracle.OracleModel(spec), Fin, Gin, want_abs=True)
    assert dth.numel() == dth_r.size == 2 * spec.d * spec.n
    assert_close(cm_to_pm(dF), dF_r, TOL[prec], f"{what} dL/dF")
    e = np.abs(dth.cpu().numpy().astype(np.float64) - dth_r) / np.maximum(dth_abs, 1e-300)
    assert e.max() < (1e-12 if prec == "f64" else 1e-4), f"{what} dL/dw {e.max():.3e}"
    return dF, dth


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("name", list(BW_SPECS))
@pytest.mark.parametrize("n", [3001, 9])
def test_cann_backward_vs_oracle(pkg, name, prec, n):
    """Backward of the CANN (eq. cann-def): dL/dF = G : A and dL/dw for every menu entry of
    eq. cann-fs on the polyconvex, raw-with-fibres and shifted isochoric layers; 3001 points
    span many CTA tiles with a ragged last one, 9 points one partial tile."""
    rng = np.random.Generator(np.random.PCG64(620 + n))
    F = wl.random_F(rng, n, 0.15)
    G = rng.normal(size=F.shape)
    cann_backward_check(pkg, BW_SPECS[name], F, G, prec, f"{name} {prec} n={n}")


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_cann_backward_edge_cases(pkg, prec):
    """No points (dL/dw zeroed), one point, and a batch with one inadmissible point (J < 0):
    NaN in its dL/dF, nothing from it in dL/dw (compared with the oracle on the others)."""
    spec = BW_SPECS["cann_all_raw2"]
    m = pkg.Model(spec, prec)
    empty = torch.empty(9, 0, dtype=DT[prec], device="cuda")
    dF0, dth0 = m.backward(empty, empty)
    torch.cuda.synchronize()
    assert dth0.numel() == 2 * spec.d * spec.n and bool((dth0 == 0).all())
    rng = np.random.Generator(np.random.PCG64(631))
    F1 = wl.random_F(rng, 1, 0.15)
    cann_backward_check(pkg, spec, F1, rng.normal(size=F1.shape), prec, f"one point {prec}")
    F = wl.random_F(rng, 77, 0.15)
    G = rng.normal(size=F.shape)
    F[5] = np.diag([-1.0, 1.0, 1.0]).ravel()  # J = -1
    dF, dth = m.backward(pm_to_cm(F, DT[prec]), pm_to_cm(G, DT[prec]))
    torch.cuda.synchronize()
    dFh = cm_to_pm(dF)
    assert np.isnan(dFh[5]).all() and np.isfinite(np.delete(dFh, 5, axis=0)).all()
    keep = np.delete(np.arange(77), 5)
    Fin = cm_to_pm(pm_to_cm(F, DT[prec])).astype(np.float64)[keep]
    Gin = cm_to_pm(pm_to_cm(G, DT[prec])).astype(np.float64)[keep]
    _, dth_r, dth_abs = oracle.const_backward(oracle.OracleModel(spec), Fin, Gin, want_abs=True)
    e = np.abs(dth.cpu().numpy().astype(np.float64) - dth_r) / np.maximum(dth_abs, 1e-300)
    assert e.max() < (1e-12 if prec == "f64" else 1e-4), e.max()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_cann_backward_out_of_range_point(pkg, prec):
    """On the paper's CANN (no logarithmic terms, so every F with J > 0 is in the energy's
    domain) F = diag(5, 1/2, 1/2) takes the exponential terms to psi ~ 1e63, A ~ 2e68 and
    dL/dw ~ 5e68: finite in FP64, where the point is kept and matches the oracle, but past
    the FP32 range, where it gets NaN in dL/dF and adds nothing to dL/dw (the other points'
    sum then matches the oracle over them alone)."""
    spec = BW_SPECS["cann_paper_poly"]
    m = pkg.Model(spec, prec)
    rng = np.random.Generator(np.random.PCG64(632))
    F = wl.random_F(rng, 100, 0.15)
    G = rng.normal(size=F.shape)
    F[37] = np.diag([5.0, 0.5, 0.5]).ravel()
    dF, dth = m.backward(pm_to_cm(F, DT[prec]), pm_to_cm(G, DT[prec]))
    torch.cuda.synchronize()
    dFh = cm_to_pm(dF)
    keep = np.arange(100) if prec == "f64" else np.delete(np.arange(100), 37)
    if prec == "f32":
        assert np.isnan(dFh[37]).all()
    assert np.isfinite(dFh[keep]).all()
    Fin = cm_to_pm(pm_to_cm(F, DT[prec])).astype(np.float64)[keep]
    Gin = cm_to_pm(pm_to_cm(G, DT[prec])).astype(np.float64)[keep]
    dF_r, dth_r, dth_abs = oracle.const_backward(oracle.OracleModel(spec), Fin, Gin, want_abs=True)
    tol = 1e-12 if prec == "f64" else 1e-4
    e = np.abs(dth.cpu().numpy().astype(np.float64) - dth_r) / np.maximum(dth_abs, 1e-300)
    assert e.max() < tol, e.max()
    ef = np.linalg.norm(dFh[keep] - dF_r, axis=1) / np.maximum(np.linalg.norm(dF_r, axis=1), 1e-300)
    assert ef.max() < (1e-11 if prec == "f64" else 1e-3), ef.max()
