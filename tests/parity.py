"""Shared helpers of the parity tests: the per-point relative error measure and layout
conversions between the library's component-major tables and the oracle's point-major
ones.

Error measure, per point (or element) and output X:
    e_q = |X_gpu,q - X_ref,q|_F / max(|X_ref,q|_F, 1e-3 * RMS_q |X_ref,q|_F)
The floor keeps points whose output is nearly zero from dominating. A comparison passes
when max_q e_q is below the tolerance: 1e-12 for FP64, 1e-5 for FP32, 2e-2 for BF16 on
P and A.
"""
import numpy as np

TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 2e-2}


def rel_err(gpu_pm: np.ndarray, ref_pm: np.ndarray, scale_pm=None) -> np.ndarray:
    """Per-row relative error of point-major arrays [n, k]. ``scale_pm`` (optional, [n, k])
    replaces the reference as the per-row scale where a subtraction in the method makes
    the result much smaller than the terms it is formed from."""
    g = np.asarray(gpu_pm, dtype=np.float64).reshape(gpu_pm.shape[0], -1)
    r = np.asarray(ref_pm, dtype=np.float64).reshape(ref_pm.shape[0], -1)
    nr = np.linalg.norm(r, axis=1)
    if scale_pm is not None:
        sc = np.asarray(scale_pm, dtype=np.float64).reshape(r.shape[0], -1)
        nr = np.maximum(nr, np.linalg.norm(sc, axis=1))
    floor = 1e-3 * np.sqrt(np.mean(nr ** 2)) if nr.size else 0.0
    return np.linalg.norm(g - r, axis=1) / np.maximum(np.maximum(nr, floor), 1e-300)


def assert_close(gpu_pm, ref_pm, tol, what="", scale_pm=None):
    e = rel_err(gpu_pm, ref_pm, scale_pm)
    assert np.all(np.isfinite(e)), f"{what}: non-finite error"
    worst = int(np.argmax(e)) if e.size else -1
    assert e.size == 0 or e.max() < tol, f"{what}: max rel err {e.max():.3e} at row {worst} (tol {tol})"
    return float(e.max()) if e.size else 0.0


def cm_to_pm(t) -> np.ndarray:
    """Component-major torch tensor [k, n] -> point-major numpy [n, k]."""
    return t.detach().cpu().numpy().T.copy()


def pm_to_cm(a, dtype, device="cuda"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a).T)).to(device=device, dtype=dtype).contiguous()
