"""Inadmissible points (J <= 0, a non-finite or zero F, a non-finite dL/dP) where the kernels
form the kinematic scalars in batches: one point per lane for a warp's next four tiles of 8
points, kept in shared memory and read back by each point's group. The bad points sit at
the edges of those 32-point batches and tiles; each must come out NaN and counted, and no
other point may change: the update over all points equals, bit for bit, the update over
the good points alone, and matches the oracle there."""
import numpy as np
import pytest

import oracle
import workload as wl
from tests.parity import TOL, assert_close, blocks_rel, cm_to_pm, pm_to_cm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {"f64": torch.float64, "f32": torch.float32}
N = 1000
BAD = {0: "neg", 31: "nan", 32: "zero", 255: "inf", 256: "neg", 517: "nan", 999: "neg"}


@pytest.fixture(scope="module")
def pkg():
    import paper_2510_00884_gb300 as p
    p.build()
    return p


def with_bad_points(F):
    F = F.copy()
    for q, kind in BAD.items():
        if kind == "neg":
            F[q] = np.diag([1.0, 1.0, -1.0]).ravel()  # J = -1
        elif kind == "nan":
            F[q, 4] = np.nan
        elif kind == "inf":
            F[q, 2] = np.inf
        else:
            F[q] = 0.0
    return F


def update(pkg, spec, F_pm, prec):
    m = pkg.Model(spec, prec)
    psi, P, A, st = m.const_update(pm_to_cm(F_pm, DT[prec]), status=True)
    torch.cuda.synchronize()
    return psi.cpu().numpy(), cm_to_pm(P), cm_to_pm(A), st.cpu().numpy()


def check_update(pkg, spec, prec, seed, vs_oracle):
    rng = np.random.Generator(np.random.PCG64(seed))
    F = with_bad_points(wl.random_F(rng, N, 0.15))
    psi, P, A, st = update(pkg, spec, F, prec)
    bad = np.array(sorted(BAD))
    good = np.setdiff1d(np.arange(N), bad)
    assert st[0] == len(bad) and st[1] == bad[0], st
    assert np.isnan(P[bad]).all() and np.isnan(A[bad]).all() and np.isnan(psi[bad]).all()
    psi_g, P_g, A_g, st_g = update(pkg, spec, F[good], prec)
    assert st_g[0] == 0
    assert np.array_equal(P[good], P_g) and np.array_equal(A[good], A_g) and np.array_equal(psi[good], psi_g)
    if vs_oracle:
        Fin = np.asarray(F[good], dtype=np.float32 if prec == "f32" else np.float64).astype(np.float64)
        _, P_r, A_r = oracle.const_update(oracle.OracleModel(spec), Fin)
        assert_close(P[good], P_r, TOL[prec], f"good points P {prec}")
        assert_close(A[good], A_r, TOL[prec], f"good points A {prec}")


@pytest.mark.parametrize("net", [(wl.KIN_POLYCONVEX, 0, 16, 3, 0.0), (wl.KIN_ISO_SHIFTED, 0, 16, 2, 10.0),
                                 (wl.KIN_RAW, 1, 16, 2, 1.0)], ids=["ncm_w16l3", "iso_w16l2", "raw1_w16l2"])
def test_micnn_update_fp64_batched(pkg, net):
    """FP64 MICNN update on networks whose batch records fit beside their warps."""
    kin, nf, W, L, kappa = net
    rng = np.random.Generator(np.random.PCG64(700 + W + L + nf))
    spec = wl.make_model(rng, kin, nf, W=W, L=L, kappa=kappa, bias_std=0.1)
    check_update(pkg, spec, "f64", 710 + nf, vs_oracle=True)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("inner", ["cann", "gent_thomas"])
def test_closed_form_update_batched(pkg, inner, prec):
    """Closed-form inner functions: the batch runs in both precisions (FP64 scalars)."""
    rng = np.random.Generator(np.random.PCG64(720))
    spec = wl.make_cann(rng, std=0.1) if inner == "cann" else wl.GentThomasSpec()
    check_update(pkg, spec, prec, 721, vs_oracle=prec == "f64")


def test_micnn_backward_fp64_batched(pkg):
    """FP64 backward of the 2^20-point stress-loss network (d7 W32 L3, whose short batch
    records fit beside its slabs): bad F and non-finite dL/dP give NaN rows in dL/dF and
    nothing in dL/dtheta, which matches the oracle over the good points."""
    rng = np.random.Generator(np.random.PCG64(730))
    spec = wl.make_model(rng, wl.KIN_RAW, 2, W=32, L=3, kappa=0.0, bias_std=0.1)
    F = with_bad_points(wl.random_F(rng, N, 0.15))
    G = rng.normal(size=F.shape)
    gbad = [7, 128, 640]
    G[7, 0] = np.nan
    G[128, 8] = np.inf
    G[640, 5] = np.nan
    m = pkg.Model(spec, "f64")
    dF, dth = m.backward(pm_to_cm(F, torch.float64), pm_to_cm(G, torch.float64))
    torch.cuda.synchronize()
    dFh = cm_to_pm(dF)
    bad = np.array(sorted(list(BAD) + gbad))
    good = np.setdiff1d(np.arange(N), bad)
    assert np.isnan(dFh[bad]).all() and np.isfinite(dFh[good]).all()
    dF_r, dth_r, dth_abs = oracle.const_backward(oracle.OracleModel(spec), F[good], G[good], want_abs=True)
    assert_close(dFh[good], dF_r, TOL["f64"], "dF good points")
    e = blocks_rel(dth.cpu().numpy(), dth_r, spec, dth_abs)
    assert e.max() < 1e-12, e
