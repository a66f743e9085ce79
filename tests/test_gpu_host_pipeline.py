"""The host-buffer entry point (commet_const_update_host): chunked copies in, kernels and
copies out on three streams give the device calls' results bit for bit, with ragged last
chunks, a chunk larger than the problem, stress-only and update-only forms, and every
precision."""
import numpy as np
import pytest

import workload as wl
from tests.parity import pm_to_cm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.float32}


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


def same(a, b):
    return a is None and b is None or torch.equal(a.cpu(), b.cpu())


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("chunk", [7, 60, 1000])
def test_with_mesh_matches_device_calls(pkg, prec, chunk):
    mesh = distorted(5, 4, 3, 900)
    rng = np.random.Generator(np.random.PCG64(901))
    spec = wl.make_model(rng, wl.KIN_RAW, 2, W=32, L=3, kappa=0.0)
    m = pkg.Model(spec, prec)
    gm = pkg.Mesh(mesh.X, mesh.conn)
    F = pm_to_cm(wl.random_F(rng, 8 * mesh.n_el, 0.15), DT[prec])
    psi, P, A = m.const_update(F)
    # the pipeline assembles the update's own (major-symmetric) tangent by its upper blocks
    f_e, K_e, _, _ = gm.elem_assemble(P, A, "f64" if prec == "f64" else "f32", symmetric=True)
    Fh = F.cpu().pin_memory()
    out = m.const_update_host(Fh, gm, chunk=chunk)
    torch.cuda.synchronize()
    for a, b in zip(out, (psi, P, A, f_e, K_e)):
        assert same(a, b)
    # stress only, no psi: f_e alone
    out2 = m.const_update_host(Fh, gm, chunk=chunk, want_A=False, want_psi=False)
    torch.cuda.synchronize()
    assert out2[0] is None and out2[2] is None and out2[4] is None
    _, P2, _ = m.const_update(F, want_A=False)
    f2, _, _, _ = gm.elem_assemble(P2, None, "f64" if prec == "f64" else "f32", want_K=False)
    assert same(out2[1], P2) and same(out2[3], f2)


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_update_only_matches_device_call(pkg, prec):
    rng = np.random.Generator(np.random.PCG64(902))
    if prec == "bf16":
        spec = wl.make_model(rng, wl.KIN_ISO_SHIFTED, 0, W=64, L=3, kappa=10.0)
        F = wl.uniaxial_F(rng, 1000)
    else:
        spec = wl.make_model(rng, wl.KIN_RAW, 2, W=32, L=3, kappa=0.0)
        F = wl.random_F(rng, 1000, 0.15)
    m = pkg.Model(spec, prec)
    Fd = pm_to_cm(F, DT[prec])
    ref = m.const_update(Fd)
    out = m.const_update_host(Fd.cpu().pin_memory(), chunk=333)
    torch.cuda.synchronize()
    for a, b in zip(out[:3], ref):
        assert same(a, b)
    assert out[3] is None and out[4] is None
    # pageable host memory works too (the copies then do not overlap)
    out3 = m.const_update_host(Fd.cpu(), chunk=128)
    torch.cuda.synchronize()
    assert same(out3[1], ref[1])


def test_host_pipeline_argument_checks(pkg):
    import ctypes as C
    from paper_2510_00884_gb300 import _lib
    rng = np.random.Generator(np.random.PCG64(903))
    m = pkg.Model(wl.make_model(rng, wl.KIN_RAW, 2, W=32, L=3, kappa=0.0), "f64")
    mesh = wl.structured_mesh(2)
    gm = pkg.Mesh(mesh.X, mesh.conn)
    lib = _lib.load()
    n = 8 * mesh.n_el
    F = torch.zeros(9, n, dtype=torch.float64).pin_memory()
    P = torch.zeros(9, n, dtype=torch.float64).pin_memory()
    fe = torch.zeros(24, mesh.n_el, dtype=torch.float64).pin_memory()
    need = int(lib.commet_const_update_host_workspace(m.handle, gm.handle, 4, 0))
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    p = lambda t: C.c_void_p(t.data_ptr())
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    # workspace too small
    assert lib.commet_const_update_host(m.handle, gm.handle, n, p(F), None, p(P), None, p(fe), None, p(ws),
                                        need - 256, 4, s) == _lib.ERR_INVALID_ARG
    # element tables without a mesh, n not 8 n_el, chunk 0
    assert lib.commet_const_update_host(m.handle, None, n, p(F), None, p(P), None, p(fe), None, p(ws), need, 4,
                                        s) == _lib.ERR_INVALID_ARG
    assert lib.commet_const_update_host(m.handle, gm.handle, n - 8, p(F), None, p(P), None, None, None, p(ws),
                                        need, 4, s) == _lib.ERR_INVALID_ARG
    assert lib.commet_const_update_host(m.handle, gm.handle, n, p(F), None, p(P), None, None, None, p(ws), need, 0,
                                        s) == _lib.ERR_INVALID_ARG
    assert lib.commet_const_update_host(m.handle, gm.handle, n, p(F), None, p(P), None, p(fe), None, p(ws), need, 4,
                                        s) == _lib.OK
    torch.cuda.synchronize()
