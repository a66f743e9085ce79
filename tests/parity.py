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


def elem_geometry(mesh):
    """Oracle shape-function gradients dphi [n_el, 8 q, 8 I, 3] and weights w [n_el, 8]."""
    import oracle

    conn = np.asarray(mesh.conn)
    X = np.asarray(mesh.X)
    dphi = np.empty((conn.shape[0], 8, 8, 3))
    w = np.empty((conn.shape[0], 8))
    for e in range(conn.shape[0]):
        dphi[e], w[e] = oracle.hex8_gradients(X[conn[e]])
    return dphi, w


def _node_sum(mesh, per_el_node):
    """Sum per-element per-node values [n_el, 8] onto the nodes."""
    out = np.zeros(np.asarray(mesh.X).shape[0])
    np.add.at(out, np.asarray(mesh.conn).ravel(), np.asarray(per_el_node).ravel())
    return out


def _csr_of_node_blocks(mesh, blk, rowptr, col):
    """CSR values of per-element node-pair magnitudes blk [n_el, 8, 8] (the same value on
    each of the 3 x 3 dof pairs of a node pair), summed over elements."""
    import oracle

    K_mag = np.kron(blk, np.ones((3, 3)))  # [n_el, 24, 24]
    vals, missing = oracle.scatter_csr(mesh, K_mag, rowptr, col)
    assert missing == 0
    return vals


def assembly_scales(mesh, P_ref, A_ref, rowptr=None, col=None, geom=None):
    """Per-dof and per-CSR-entry magnitudes the assembled r and K are checked against.

    r[3I+i] = sum_e sum_q w_q P_iJ dphi_I,J and K[3I+i, 3K+k] = sum_e sum_q w_q dphi_I,J
    A_iJkL dphi_K,L (eq. r-quad / k-quad summed over elements). If every point's P and A
    are within a relative tolerance t in the Frobenius norm (the per-point measure above),
    every term moves by at most t |P_q|_F |dphi_I|_1 (resp. t |A_q|_F |dphi_I|_1
    |dphi_K|_1), so an entry of r (of K) is within t of
        s_r[3I+i]        = sum_e sum_q w_q |P_q|_F |dphi_I,q|_1,
        s_K[3I+i, 3K+k]  = sum_e sum_q w_q |A_q|_F |dphi_I,q|_1 |dphi_K,q|_1,
    to which the rounding of the sums adds a few units of the working precision times
    the same magnitudes. Rows are compared with ``rel_err(..., scale_pm=...)``: an entry
    whose element terms cancel (an interior r near equilibrium, an off-diagonal block)
    keeps the rounding of the terms it is made of. P_ref, A_ref are point-major, element
    e's points at rows 8e..8e+7. Returns s_r [3 n_nodes] and, given a CSR pattern, the
    CSR magnitudes [nnz]."""
    dphi, w = elem_geometry(mesh) if geom is None else geom
    n_el = dphi.shape[0]
    g1 = np.abs(dphi).sum(axis=3)  # [e][q][I]
    nP = np.linalg.norm(np.asarray(P_ref, dtype=np.float64).reshape(n_el, 8, 9), axis=2)
    s_r = np.repeat(_node_sum(mesh, np.einsum("eq,eqI->eI", w * nP, g1)), 3)
    if A_ref is None or rowptr is None:
        return s_r, None
    nA = np.linalg.norm(np.asarray(A_ref, dtype=np.float64).reshape(n_el, 8, 81), axis=2)
    blk = np.einsum("eq,eqI,eqK->eIK", w * nA, g1, g1)
    return s_r, _csr_of_node_blocks(mesh, blk, rowptr, col)


VOIGT_PAIRS = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))


def voigt_c_full_norm(c21):
    """Frobenius norm of the full 81-entry spatial tangent from its 21 Voigt values
    (upper triangle of the 6 x 6 matrix, row-major; minor and major symmetry)."""
    c21 = np.asarray(c21, dtype=np.float64).reshape(-1, 21)
    mult = []
    for I in range(6):
        for J in range(I, 6):
            nI = 1 if VOIGT_PAIRS[I][0] == VOIGT_PAIRS[I][1] else 2
            nJ = 1 if VOIGT_PAIRS[J][0] == VOIGT_PAIRS[J][1] else 2
            mult.append(nI * nJ * (1 if I == J else 2))
    return np.sqrt((c21 ** 2 * np.array(mult)).sum(axis=1))


def spatial_assembly_scales(mesh, F_pm, tau_pm, c_pm, rowptr, col):
    """The magnitudes of ``assembly_scales`` for the spatial eq. r-quad / k-quad:
    r[3I+i] = sum w tau_ij g_I,j and K[3I+i, 3K+k] = sum w (g_I,j c_ijkl g_K,l +
    delta_ik tau_jl g_I,j g_K,l) with the spatial gradients g = F^-T Grad(phi), so
        s_r = sum w |tau|_F |g_I|_1,   s_K = sum w (|c|_F + |tau|_F) |g_I|_1 |g_K|_1."""
    dphi, w = elem_geometry(mesh)
    n_el = dphi.shape[0]
    Finv = np.linalg.inv(np.asarray(F_pm, dtype=np.float64).reshape(n_el, 8, 3, 3))
    g = np.einsum("eqIJ,eqJj->eqIj", dphi, Finv)  # dphi_I/dx_j = dphi_I/dX_J (F^-1)_Jj
    g1 = np.abs(g).sum(axis=3)
    nt = np.linalg.norm(np.asarray(tau_pm, dtype=np.float64).reshape(n_el * 8, 6) * np.array([1, 1, 1, 2 ** .5, 2 ** .5, 2 ** .5]), axis=1).reshape(n_el, 8)
    nc = voigt_c_full_norm(c_pm).reshape(n_el, 8)
    s_r = np.repeat(_node_sum(mesh, np.einsum("eq,eqI->eI", w * nt, g1)), 3)
    blk = np.einsum("eq,eqI,eqK->eIK", w * (nc + nt), g1, g1)
    return s_r, _csr_of_node_blocks(mesh, blk, rowptr, col)


def adjoint_u_scale(mesh, dF_pm, geom=None):
    """Magnitude of du[I, i] = sum_e sum_q sum_J dF_iJ dphi_I,J (the transpose of the trial
    F): s[I, i] = sum_e sum_q sum_J |dF_iJ| |dphi_I,J|, the scale its rounding is
    measured against. Returns [n_nodes, 3]."""
    dphi, _ = elem_geometry(mesh) if geom is None else geom
    n_el = dphi.shape[0]
    a = np.abs(np.asarray(dF_pm, dtype=np.float64).reshape(n_el, 8, 3, 3))
    per = np.einsum("eqiJ,eqIJ->eIi", a, np.abs(dphi))
    out = np.zeros((np.asarray(mesh.X).shape[0], 3))
    np.add.at(out, np.asarray(mesh.conn).ravel(), per.reshape(-1, 3))
    return out


def csr_rows_rel_err(gpu_vals, ref_vals, scale_vals, rowptr, rows=None):
    """Per-row relative error of CSR values: |gpu_row - ref_row|_2 / |scale_row|_2 for the
    given rows (all if None). Every row is expected to hold at least one entry."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    rows = np.arange(rowptr.size - 1) if rows is None else np.asarray(rows, dtype=np.int64)
    lo, hi = rowptr[rows], rowptr[rows + 1]
    assert np.all(hi > lo), "empty CSR row"
    idx = np.concatenate([np.arange(a, b) for a, b in zip(lo, hi)]) if rows.size else np.zeros(0, np.int64)
    starts = np.concatenate([[0], np.cumsum(hi - lo)[:-1]]) if rows.size else np.zeros(0, np.int64)
    g = np.asarray(gpu_vals)[idx].astype(np.float64)
    r = np.asarray(ref_vals)[idx].astype(np.float64)
    s = np.asarray(scale_vals)[idx].astype(np.float64)
    if not rows.size:
        return np.zeros(0)
    d2 = np.add.reduceat((g - r) ** 2, starts)
    s2 = np.add.reduceat(s ** 2, starts)
    return np.sqrt(d2) / np.maximum(np.sqrt(s2), 1e-300)


def blocks_rel(g, r, spec, scale=None):
    """Relative error of each parameter block (W1, c1, A_k, B_k, c_k, a, b). dL/dtheta is
    a sum over points, so the error is measured against the sum of the magnitudes of the
    per-point terms (``scale`` = sum_q |dtheta_q|, the usual bound of a floating-point
    sum) when it is given: a block whose terms cancel has a small result but no smaller
    rounding error."""
    d, W, L = spec.d, spec.W, spec.L
    sizes = [W * d, W] + [W * W, W * d, W] * (L - 1) + [W, d]
    sc = r if scale is None else scale
    out, o = [], 0
    for n in sizes:
        a, b = g[o:o + n], r[o:o + n]
        out.append(np.linalg.norm(a - b) / max(np.linalg.norm(sc[o:o + n]), 1e-300))
        o += n
    return np.array(out)
