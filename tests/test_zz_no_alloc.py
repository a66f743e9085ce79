"""The backward entry point that allocates nothing (commet_const_backward_noalloc).

It serves callers whose host application owns all device memory and cannot give the
library a workspace: the per-CTA partial sums go to a fixed array inside the library.
This file is collected last so that a run stopping at the first failure has run every
other test before it; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import workload as wl
from tests.parity import assert_close, cm_to_pm, pm_to_cm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2510_00884_gb300 as p
    p.build()
    return p


def _call_noalloc(lib, m, F, G, dF, dth):
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.commet_const_backward_noalloc(m.handle, F.shape[1], C.c_void_p(F.data_ptr()),
                                             C.c_void_p(G.data_ptr()), C.c_void_p(dF.data_ptr()),
                                             C.c_void_p(dth.data_ptr()), s)


def test_noalloc_backward_matches_the_workspace_entry_point(pkg):
    from paper_2510_00884_gb300 import _lib
    lib = _lib.load()
    rng = np.random.Generator(np.random.PCG64(77))
    spec = wl.workload_c1(n=1)["model"]  # two-fibre d7 W32 L3 network
    m = pkg.Model(spec, "f64")
    n = 40_000
    F = pm_to_cm(wl.random_F(rng, n, 0.15), torch.float64)
    dF = torch.empty_like(F)
    dth = torch.empty(m.n_params, dtype=torch.float64, device="cuda")
    for call in range(2):
        # a different upstream gradient each call, so stale scratch would show
        G = pm_to_cm(rng.normal(size=(n, 9)), torch.float64)
        dF_ref, dth_ref = m.backward(F, G)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = _call_noalloc(lib, m, F, G, dF, dth)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        assert rc == _lib.OK, _lib.status_string(rc)
        if call == 1:
            assert free_after == free_before, "the call changed the device's free memory"
        assert_close(cm_to_pm(dF), cm_to_pm(dF_ref), 1e-12, f"call {call} dL/dF")
        g, r = dth.cpu().numpy(), dth_ref.cpu().numpy()
        assert np.linalg.norm(g - r) <= 1e-12 * np.linalg.norm(r), f"call {call} dL/dtheta"


def test_noalloc_backward_rejects_oversize_scratch(pkg):
    """A network whose partial sums exceed the fixed array is refused, launching nothing."""
    from paper_2510_00884_gb300 import _lib
    lib = _lib.load()
    rng = np.random.Generator(np.random.PCG64(78))
    spec = wl.make_model(rng, wl.KIN_ISO_SHIFTED, 0, W=64, L=3, kappa=1.0)
    m = pkg.Model(spec, "f64")
    need = lib.commet_const_backward_workspace(m.handle, 1 << 20)
    assert need > 8 * 1024 * 1024
    F = pm_to_cm(wl.random_F(rng, 1 << 20, 0.1), torch.float64)
    G = torch.zeros_like(F)
    dF = torch.full_like(F, 7.0)
    dth = torch.full((m.n_params,), 7.0, dtype=torch.float64, device="cuda")
    assert _call_noalloc(lib, m, F, G, dF, dth) == _lib.ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert bool((dth == 7.0).all()) and bool((dF == 7.0).all())
