"""GPU parity of the bf16 tensor-core MLP path (hidden W x W layers in bf16 with fp32
accumulation) against the FP64 oracle at the bf16 tolerance (2e-2 on P and A, per point,
measure of tests/parity.py), with the FP32 path's error on the same inputs for context."""
import numpy as np
import pytest

import oracle
import workload as wl
from tests.parity import TOL, assert_close, cm_to_pm, pm_to_cm, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2510_00884_gb300 as p
    p.build()
    return p


CASES = [
    (wl.KIN_ISO_SHIFTED, 0, 64, 3, 10.0, 5003),
    (wl.KIN_ISO_SHIFTED, 0, 32, 2, 10.0, 1003),
    (wl.KIN_RAW, 2, 32, 3, 0.0, 2011),
    (wl.KIN_ISO_SHIFTED, 0, 64, 4, 3.0, 33),
    (wl.KIN_POLYCONVEX, 0, 32, 3, 0.0, 3001),
]


@pytest.mark.parametrize("case", CASES, ids=[f"k{c[0]}f{c[1]}w{c[2]}l{c[3]}n{c[5]}" for c in CASES])
def test_bf16_vs_oracle(pkg, case):
    kin, nf, W, L, kappa, n = case
    rng = np.random.Generator(np.random.PCG64(300 + W + L + nf))
    spec = wl.make_model(rng, kin, nf, W=W, L=L, kappa=kappa)
    F = wl.uniaxial_F(rng, n) if kin == wl.KIN_ISO_SHIFTED else wl.random_F(rng, n, 0.15)
    Fd = pm_to_cm(F, torch.float32)
    Fin = cm_to_pm(Fd).astype(np.float64)
    _, P_r, A_r = oracle.const_update(oracle.OracleModel(spec), Fin)
    mb = pkg.Model(spec, "bf16")
    psi, P, A, st = mb.const_update(Fd, status=True)
    torch.cuda.synchronize()
    assert int(st[0]) == 0
    assert_close(cm_to_pm(P), P_r, TOL["bf16"], "bf16 P")
    assert_close(cm_to_pm(A), A_r, TOL["bf16"], "bf16 A")
    # bf16 must be worse than fp32 but not absurdly: a sanity window on the median error
    e_bf = np.median(rel_err(cm_to_pm(A), A_r))
    m32 = pkg.Model(spec, "f32")
    _, P32, A32 = m32.const_update(Fd)
    e_32 = np.median(rel_err(cm_to_pm(A32), A_r))
    assert e_32 < e_bf < 2e-2


def test_bf16_edge_cases(pkg):
    rng = np.random.Generator(np.random.PCG64(310))
    spec = wl.make_model(rng, wl.KIN_ISO_SHIFTED, 0, W=64, L=3, kappa=10.0)
    mb = pkg.Model(spec, "bf16")
    F0 = torch.empty(9, 0, dtype=torch.float32, device="cuda")
    _, P0, _ = mb.const_update(F0)
    assert P0.shape == (9, 0)
    F = wl.uniaxial_F(rng, 40)
    F[5] = np.diag([1.0, 1.0, -0.5]).ravel()
    F[30, 2] = np.inf
    Fd = pm_to_cm(F, torch.float32)
    psi, P, A, st = mb.const_update(Fd, status=True)
    torch.cuda.synchronize()
    assert int(st[0]) == 2 and int(st[1]) == 5
    Pn = cm_to_pm(P)
    assert np.all(np.isnan(Pn[5])) and np.all(np.isnan(Pn[30]))
    good = np.setdiff1d(np.arange(40), [5, 30])
    _, P_r, _ = oracle.const_update(oracle.OracleModel(spec), cm_to_pm(Fd).astype(np.float64)[good])
    assert_close(Pn[good], P_r, TOL["bf16"], "bf16 good points")


def test_c2_full_size_sampled(pkg):
    """128^3 mesh worth of points (16,777,216, d3 W64 L3, the benchmark's launch): bf16 and
    fp32 paths on sampled points (strided + near J = 1 and J < 0.8) against the oracle."""
    w = wl.workload_c2()
    spec, F = w["model"], w["F"]
    n = F.shape[0]
    Fd = pm_to_cm(F, torch.float32)
    J = np.linalg.det(F.reshape(-1, 3, 3))
    idx = np.unique(np.concatenate([np.linspace(0, n - 1, 1500).astype(np.int64),
                                    np.nonzero(np.abs(J - 1) < 1e-3)[0][:300], np.nonzero(J < 0.8)[0][:300]]))
    Fin = cm_to_pm(Fd[:, torch.from_numpy(idx).cuda()]).astype(np.float64)
    _, P_r, A_r = oracle.const_update(oracle.OracleModel(spec), Fin)
    it = torch.from_numpy(idx).cuda()
    for prec in ("bf16", "f32"):
        m = pkg.Model(spec, prec)
        _, P, A, st = m.const_update(Fd, status=True)
        torch.cuda.synchronize()
        assert int(st[0]) == 0
        assert_close(P.index_select(1, it).cpu().numpy().T, P_r, TOL[prec], f"C2 {prec} P")
        assert_close(A.index_select(1, it).cpu().numpy().T, A_r, TOL[prec], f"C2 {prec} A")
        del P, A
        torch.cuda.empty_cache()


def test_bf16_tensor_memory_budget(pkg):
    """The tcgen05 kernel keeps d W accumulator columns and L W (F', F'') columns of tensor
    memory: d3 W64 L5 fills the 512 columns exactly and matches the oracle; L6 would need
    576 and is refused with UNSUPPORTED."""
    from paper_2510_00884_gb300 import _lib
    rng = np.random.Generator(np.random.PCG64(320))
    spec = wl.make_model(rng, wl.KIN_ISO_SHIFTED, 0, W=64, L=5, kappa=3.0)
    F = wl.uniaxial_F(rng, 389)
    Fd = pm_to_cm(F, torch.float32)
    _, P_r, A_r = oracle.const_update(oracle.OracleModel(spec), cm_to_pm(Fd).astype(np.float64))
    mb = pkg.Model(spec, "bf16")
    _, P, A, st = mb.const_update(Fd, status=True)
    torch.cuda.synchronize()
    assert int(st[0]) == 0
    assert_close(cm_to_pm(P), P_r, TOL["bf16"], "bf16 L5 P")
    assert_close(cm_to_pm(A), A_r, TOL["bf16"], "bf16 L5 A")
    big = pkg.Model(wl.make_model(rng, wl.KIN_ISO_SHIFTED, 0, W=64, L=6, kappa=3.0), "bf16")
    with pytest.raises(_lib.CommetError) as ei:
        big.const_update(Fd)
    assert ei.value.code == _lib.ERR_UNSUPPORTED
