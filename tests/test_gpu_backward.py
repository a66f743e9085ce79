"""GPU parity of the backward (adjoint) kernel: dL/dF and dL/dtheta against the FP64
oracle, central differences of the training loss, determinism and the autograd path."""
import numpy as np
import pytest

import oracle
import workload as wl
from tests.parity import TOL, assert_close, blocks_rel, cm_to_pm, pm_to_cm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {"f64": torch.float64, "f32": torch.float32}


@pytest.fixture(scope="module")
def pkg():
    import paper_2510_00884_gb300 as p
    p.build()
    return p


def oracle_dtheta_abs(spec, F, G):
    """sum_q |dL/dtheta of point q| per entry, from the oracle."""
    _, _, a = oracle.const_backward(oracle.OracleModel(spec), F, G, want_abs=True)
    return a


CASES = [(wl.KIN_RAW, 2, 32, 3, 0.0, 3001), (wl.KIN_ISO_SHIFTED, 0, 16, 2, 10.0, 2049),
         (wl.KIN_RAW, 1, 16, 4, 1.0, 777), (wl.KIN_RAW, 2, 32, 1, 2.0, 513), (wl.KIN_ISO_SHIFTED, 0, 32, 3, 5.0, 5),
         (wl.KIN_POLYCONVEX, 0, 16, 3, 0.0, 2500), (wl.KIN_POLYCONVEX, 0, 32, 2, 4.0, 301),
         (wl.KIN_POLYCONVEX, 0, 4, 3, 0.0, 777), (wl.KIN_ISO_SHIFTED, 0, 8, 2, 3.0, 1500)]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("case", CASES, ids=[f"k{c[0]}f{c[1]}w{c[2]}l{c[3]}n{c[5]}" for c in CASES])
def test_backward_vs_oracle(pkg, case, prec):
    kin, nf, W, L, kappa, n = case
    rng = np.random.Generator(np.random.PCG64(200 + W + L))
    spec = wl.make_model(rng, kin, nf, W=W, L=L, kappa=kappa, bias_std=0.1)
    F = wl.random_F(rng, n, 0.15)
    G = rng.normal(size=F.shape)
    m = pkg.Model(spec, prec)
    Fd, Gd = pm_to_cm(F, DT[prec]), pm_to_cm(G, DT[prec])
    dF, dth = m.backward(Fd, Gd)
    Fin, Gin = cm_to_pm(Fd).astype(np.float64), cm_to_pm(Gd).astype(np.float64)
    dF_r, dth_r = oracle.const_backward(oracle.OracleModel(spec), Fin, Gin)
    # dL/dF per point is G : A, compared like A; dL/dtheta block by block
    tol_F = TOL[prec]
    assert_close(cm_to_pm(dF), dF_r, tol_F, f"dF {prec}")
    tol_th = 1e-12 if prec == "f64" else 1e-4
    e = blocks_rel(dth.cpu().numpy().astype(np.float64), dth_r, spec, oracle_dtheta_abs(spec, Fin, Gin))
    assert e.max() < tol_th, e


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("nf", [0, 2])
def test_backward_w64_half_tile(pkg, nf, prec):
    """64-wide two-layer networks: their weights, gradient accumulators and point slabs
    fit in shared memory only at half the CTA tile, which the launch falls back to; the
    result matches the oracle like every other width (a ragged 1,001 points, biases set)."""
    rng = np.random.Generator(np.random.PCG64(400 + nf))
    kin = wl.KIN_RAW if nf else wl.KIN_ISO_SHIFTED
    spec = wl.make_model(rng, kin, nf, W=64, L=2, kappa=2.0, bias_std=0.1)
    F = wl.random_F(rng, 1001, 0.15)
    G = rng.normal(size=F.shape)
    m = pkg.Model(spec, prec)
    Fd, Gd = pm_to_cm(F, DT[prec]), pm_to_cm(G, DT[prec])
    dF, dth = m.backward(Fd, Gd)
    Fin, Gin = cm_to_pm(Fd).astype(np.float64), cm_to_pm(Gd).astype(np.float64)
    dF_r, dth_r = oracle.const_backward(oracle.OracleModel(spec), Fin, Gin)
    assert_close(cm_to_pm(dF), dF_r, TOL[prec], f"W64 dF {prec}")
    e = blocks_rel(dth.cpu().numpy().astype(np.float64), dth_r, spec, oracle_dtheta_abs(spec, Fin, Gin))
    assert e.max() < (1e-12 if prec == "f64" else 1e-4), e


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("case", [(wl.KIN_ISO_SHIFTED, 0, 3), (wl.KIN_RAW, 2, 3), (wl.KIN_POLYCONVEX, 0, 4)],
                         ids=["iso_l3", "fib2_l3", "poly_l4"])
def test_backward_w64_deep(pkg, case, prec):
    """64-wide networks with three or more layers (the precision workload's d3 W64 L3 and
    the paper's largest App. E model, W64 L4): their weights, gradient accumulators and
    point slabs do not fit in shared memory together, so the CTA accumulates into its
    workspace slice and reads the reverse pass's A_k from global memory; dL/dF and
    dL/dtheta match the oracle like every other width (a ragged 1,001 points, biases set),
    and the result is bitwise reproducible."""
    kin, nf, L = case
    rng = np.random.Generator(np.random.PCG64(410 + nf + L))
    spec = wl.make_model(rng, kin, nf, W=64, L=L, kappa=2.0 if kin != wl.KIN_POLYCONVEX else 0.0, bias_std=0.1)
    F = wl.random_F(rng, 1001, 0.15)
    G = rng.normal(size=F.shape)
    m = pkg.Model(spec, prec)
    Fd, Gd = pm_to_cm(F, DT[prec]), pm_to_cm(G, DT[prec])
    dF, dth = m.backward(Fd, Gd)
    dF2, dth2 = m.backward(Fd, Gd)
    assert torch.equal(dth, dth2) and torch.equal(dF, dF2)
    Fin, Gin = cm_to_pm(Fd).astype(np.float64), cm_to_pm(Gd).astype(np.float64)
    dF_r, dth_r, dth_abs = oracle.const_backward(oracle.OracleModel(spec), Fin, Gin, want_abs=True)
    assert_close(cm_to_pm(dF), dF_r, TOL[prec], f"W64 L{L} dF {prec}")
    e = blocks_rel(dth.cpu().numpy().astype(np.float64), dth_r, spec, dth_abs)
    assert e.max() < (1e-12 if prec == "f64" else 1e-4), e


def test_backward_c3_loss_central_differences(pkg):
    """C3 loss sum_q |P(F; theta) - P_target|^2 on 64 points: GPU dL/dtheta and dL/dF
    against central differences (h = 1e-6) of the GPU FP64 forward."""
    w = wl.workload_c3(n_qp=64)
    spec, F = w["model"], w["F"]
    t = w["target"]
    Fd = pm_to_cm(F, torch.float64)
    Pt = pkg.target_stress(Fd, spec.fibres, t["mu"], t["k1"], t["k2"], t["kappa"])
    m = pkg.Model(spec, "f64")
    _, P, _ = m.const_update(Fd, want_A=False)
    G = 2.0 * (P - Pt)
    dF, dth = m.backward(Fd, G)
    dth = dth.cpu().numpy()

    def loss(spec_, Fdev):
        _, PP, _ = pkg.Model(spec_, "f64").const_update(Fdev, want_A=False)
        return float(((PP - Pt) ** 2).sum().item())
    theta = spec.theta()
    h = 1e-6
    idx = np.unique(np.concatenate([np.arange(0, theta.size, 11), np.arange(theta.size - spec.W - spec.d,
                                                                               theta.size)]))
    fd = np.empty(idx.size)
    for t_i, i in enumerate(idx):
        e = np.zeros_like(theta)
        e[i] = h
        fd[t_i] = (loss(spec.with_theta(theta + e), Fd) - loss(spec.with_theta(theta - e), Fd)) / (2 * h)
    assert np.linalg.norm(dth[idx] - fd) / np.linalg.norm(fd) < 1e-6
    # dL/dF on a few entries
    dFn = dF.cpu().numpy()
    for (c, q) in [(0, 0), (4, 17), (8, 63), (1, 5), (6, 40)]:
        Fp, Fm = Fd.clone(), Fd.clone()
        Fp[c, q] += h
        Fm[c, q] -= h
        _, Pp, _ = m.const_update(Fp, want_A=False)
        _, Pm, _ = m.const_update(Fm, want_A=False)
        # the kernel's dL/dF is G : dP/dF of the model; the target is held at its value
        lp = float(((Pp - Pt) ** 2).sum().item())
        lm = float(((Pm - Pt) ** 2).sum().item())
        fdv = (lp - lm) / (2 * h)
        assert abs(dFn[c, q] - fdv) <= 1e-6 * max(1.0, abs(fdv))
    # and the oracle's gradient on the same points
    _, dth_r = oracle.const_backward(oracle.OracleModel(spec), F, cm_to_pm(G))
    assert np.linalg.norm(dth - dth_r) / np.linalg.norm(dth_r) < 1e-12


def test_backward_deterministic_and_linear(pkg):
    """Bitwise-identical results on repeat; the sum over two halves equals the whole."""
    rng = np.random.Generator(np.random.PCG64(31))
    spec = wl.workload_c1(n=1)["model"]
    n = 50_000
    F = wl.random_F(rng, n, 0.15)
    G = rng.normal(size=F.shape)
    m = pkg.Model(spec, "f64")
    Fd, Gd = pm_to_cm(F, torch.float64), pm_to_cm(G, torch.float64)
    _, t1 = m.backward(Fd, Gd)
    _, t2 = m.backward(Fd, Gd)
    assert torch.equal(t1, t2)
    h = n // 2
    _, ta = m.backward(Fd[:, :h].contiguous(), Gd[:, :h].contiguous())
    _, tb = m.backward(Fd[:, h:].contiguous(), Gd[:, h:].contiguous())
    assert torch.allclose(ta + tb, t1, rtol=1e-12, atol=1e-12 * t1.abs().max().item())


def test_autograd_function(pkg):
    """torch autograd through the forward (stress) and the adjoint kernel."""
    rng = np.random.Generator(np.random.PCG64(32))
    spec = wl.make_model(rng, wl.KIN_RAW, 2, W=32, L=3, kappa=0.0)
    m = pkg.Model(spec, "f64")
    F = pm_to_cm(wl.random_F(rng, 1000, 0.15), torch.float64).requires_grad_(True)
    sink = torch.zeros(m.n_params, dtype=torch.float64, device="cuda", requires_grad=True)
    P = pkg.ConstUpdateP.apply(F, sink, m)
    loss = (P ** 2).sum()
    loss.backward()
    dF_ref, dth_ref = m.backward(F.detach(), 2.0 * P.detach())
    assert torch.allclose(F.grad, dF_ref, rtol=0, atol=0)
    assert torch.allclose(sink.grad, dth_ref, rtol=0, atol=0)


def test_backward_c3_full_size_sampled(pkg):
    """1,048,576 points of the two-fibre network (the benchmark's backward launch, its
    whole persistent grid of per-CTA partial sums and the fixed-order reduction over
    them): sampled dL/dF against the oracle, and the whole dL/dtheta against the oracle
    over all 2^20 points, block by block at 1e-12 of sum_q |dtheta_q|."""
    w = wl.workload_c3()
    spec, F = w["model"], w["F"]
    t = w["target"]
    m = pkg.Model(spec, "f64")
    Fd = pm_to_cm(F, torch.float64)
    Pt = pkg.target_stress(Fd, spec.fibres, t["mu"], t["k1"], t["k2"], t["kappa"])
    _, P, _ = m.const_update(Fd, want_A=False)
    G = (2.0 * (P - Pt)).contiguous()
    dF, dth = m.backward(Fd, G)
    torch.cuda.synchronize()
    G_np = G.cpu().numpy().T.copy()
    dF_r, dth_r, dth_abs = oracle.const_backward(oracle.OracleModel(spec), F, G_np, want_abs=True)
    idx = np.unique(np.linspace(0, F.shape[0] - 1, 4000).astype(np.int64))
    it = torch.from_numpy(idx).cuda()
    assert_close(dF.index_select(1, it).cpu().numpy().T, dF_r[idx], 1e-12, "C3 dF")
    e = blocks_rel(dth.cpu().numpy(), dth_r, spec, dth_abs)
    assert e.max() < 1e-12, e
    # FP32 on the same points against the same oracle gradient
    m32 = pkg.Model(spec, "f32")
    dF32, dth32 = m32.backward(Fd.float(), G.float())
    torch.cuda.synchronize()
    Fin = Fd.float().double().cpu().numpy().T.copy()
    Gin = G.float().double().cpu().numpy().T.copy()
    dF_r32, dth_r32, dth_abs32 = oracle.const_backward(oracle.OracleModel(spec), Fin, Gin, want_abs=True)
    assert_close(dF32.index_select(1, it).double().cpu().numpy().T, dF_r32[idx], TOL["f32"], "C3 dF f32")
    e32 = blocks_rel(dth32.double().cpu().numpy(), dth_r32, spec, dth_abs32)
    assert e32.max() < 1e-4, e32
