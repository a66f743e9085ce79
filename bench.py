"""Benchmark of the neural-constitutive hot path on one node (one rank per GPU).

A step is one pass of the hot path over one batch of the workload, with inputs resident
in HBM. Default workload (no flags) is `c1`: the 64^3 anisotropic mesh (262,144
elements, 2,097,152 points, two-fibre MICNN d7 W32 L3) in FP64, where a step is the
fused constitutive update (F -> Psi, P, A at every point) followed by the hex8 element
integrals (P, A -> f_int, K_e for every element). Other workloads:
  c0  8^3 cube: F from u, update, element integrals (FP64)
  c2  128^3 uniaxial points, d3 W64 L3: the update (FP32 or bf16 tensor-core MLP)
  c3  2^20 points of the c1 network: stress, loss gradient and the adjoint kernel
  c4  96^3 cantilever: fused Newton assembly u -> r, CSR K (FP32), with the unfused
      FP64 GPU path timed beside it
  ncm the paper's NCM (App. C): MICNN d3 W16 L3 without biases (675 parameters) on the
      polyconvex inputs (Ibar1 - 3, Ibar2^{3/2} - 3^{3/2}, (J - 1)^2), 64^3 mesh, c1's step
  cann the paper's CANN (exponents {1, 2} x {x, exp x}) on the same inputs, c1's step
  gt  the closed-form Gent-Thomas law (eq. gt), c1's step
  ickan an input-convex KAN (App. B; 3 -> 4 -> 4 -> 1, degree 4, 30 intervals), c1's step
  resid the gradient of a residual-based loss 1/2 |r_free|^2 (eq. loss) on a 64^3 cantilever:
      u -> F -> P -> r, then the adjoint chain to dL/dtheta and dL/du

Prints one JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle on the
host cores instead (a bounded sample of the same workload per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "qp constitutive updates/sec (P+tangent) and element assemblies/sec; % roofline"


# ------------------------------------------------------------------ work models

def update_macs(d: int, W: int, L: int) -> int:
    """Minimal exact multiply-adds per point of the forward update: network values
    W d + (L-1)(W^2 + W d), reverse adjoints (L-1) W^2 plus the gradient L W d,
    tangents (L-1) W^2 d, Hessian L W d(d+1)/2, rank-one part of A 9 d^2 + 81 d.
    Kinematics, activations and the structured terms of A are not counted."""
    macs = W * d + (L - 1) * (W * W + W * d)
    macs += (L - 1) * W * W + L * W * d
    macs += (L - 1) * W * W * d
    macs += L * W * d * (d + 1) // 2
    macs += 9 * d * d + 81 * d
    return macs


def algorithmic_flops_per_qp(d: int, W: int, L: int) -> int:
    return 2 * update_macs(d, W, L)


def backward_flops_per_qp(d: int, W: int, L: int) -> int:
    """Minimal multiply-adds (x2) per point of the backward: values and tangents along r
    2 [W d + (L-1)(W^2 + W d)], reverse of both 2 (L-1) W^2, weight-gradient outer
    products 2 [(L-1)(W^2 + W d) + W d], Hessian-vector and gradient sums 2 L W d, and
    r = G : dK/dF plus dL/dF's rank-one part 2 * 9 d."""
    macs = 2 * (W * d + (L - 1) * (W * W + W * d))
    macs += 2 * (L - 1) * W * W
    macs += 2 * ((L - 1) * (W * W + W * d) + W * d)
    macs += 2 * L * W * d
    macs += 2 * 9 * d
    return 2 * macs


# Multiply-adds per hex8 element of eq. r-quad / k-quad: per Gauss point and per row (I, i)
# of K_e, A contracted with the node's gradient (9 entries x 3) and then with every
# column's gradient (24 entries x 3), plus 3 for f_e: 24 x (27 + 72 + 3) per point, 8 points.
ELEM_MACS = 8 * 24 * (27 + 72 + 3)
# With a major-symmetric A (the update's own tangent), the upper node blocks only: per
# point the 24 rows' A contraction and f (27 + 3) and the 36 upper 3 x 3 blocks (27 each).
ELEM_MACS_SYM = 8 * (24 * (27 + 3) + 36 * 27)
PUSH_FORWARD_MACS = 21 * 15 + 6 * 3  # per point: c = F A F - delta tau (21 entries), tau = P F^T (6)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


def alu_peak_tflops(kind: str, n_sm: int, mhz: float) -> float:
    """FP64 / FP32 FMA peak from unit counts and clock: GB300 issues 2 DFMA or 128 FFMA
    per SM per clock (FP64 1.25 TFLOP/s nominal at 2070 MHz on 152 SMs)."""
    per_clk = 2 if kind == "f64" else 128
    return n_sm * per_clk * 2 * mhz * 1e6 / 1e12


def load_alu_peaks():
    """Measured FP64 / FP32 FMA rates and MUFU rates of this GPU from the committed probe
    summary (profiles/alu_peaks.json), or None."""
    p = os.path.join(ROOT, "profiles", "alu_peaks.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        return json.load(f)


def alu_peak(kind: str, n_sm: int, mhz: float):
    """(peak TFLOP/s, source) for an FP64 or FP32 kernel: the measured FMA rate when the
    probe summary is present, else the unit-count figure."""
    ap = load_alu_peaks()
    key = "f64_tflops" if kind == "f64" else "f32_tflops"
    derived = alu_peak_tflops(kind, n_sm, mhz)
    if ap and key in ap:
        return float(ap[key]), (f"measured {'DFMA' if kind == 'f64' else 'FFMA'} rate {ap[key]:.3g} TFLOP/s "
                                f"(profiles/alu_peaks.json, {ap.get('profile', '')}); unit-count figure "
                                f"{derived:.4g} at {mhz:.0f} MHz")
    return derived, (f"derived: {n_sm} SMs x {'2 DFMA' if kind == 'f64' else '128 FFMA'}/clk x 2 flop x "
                     f"{mhz:.0f} MHz (max SM clock)")


def mufu_peak_tops(n_sm: int, mhz: float):
    """Peak rate (T ops/s) of the softplus's MUFU mix, one ex2, one rcp and one lg2 per
    neuron: 3 / (1/r_ex2 + 1/r_rcp + 1/r_lg2) per SM per clock from the measured rates
    (else 16 per clock for each), and its source."""
    ap = load_alu_peaks()
    r = (ap or {}).get("mufu_per_sm_clk") or {}
    ex2, rcp, lg2 = float(r.get("ex2", 16.0)), float(r.get("rcp", 16.0)), float(r.get("lg2", 16.0))
    per_clk = 3.0 / (1.0 / ex2 + 1.0 / rcp + 1.0 / lg2)
    src = (f"measured MUFU ex2 {ex2:.3g}, rcp {rcp:.3g}, lg2 {lg2:.3g} per SM per clock (profiles/alu_peaks.json): "
           f"{per_clk:.3g} per clock for the mix" if r else "assumed 16 per SM per clock")
    return per_clk * n_sm * mhz * 1e6 / 1e12, src


def kernel_source_hash(files) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2510_00884_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, network: str, precision: str, src_hash: str, units: int):
    """Per-launch DRAM bytes of the kernel from the committed ncu summary, scaled from the
    captured case to `units` (points or elements); None when the kernel source changed
    since the capture."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        tab = json.load(f)
    e = tab.get(f"{kernel}|{network}|{precision}")
    if not e or e.get("src_hash") != src_hash:
        return None
    return e["dram_bytes"] * units / e["units"]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a region."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.path is None or not os.path.exists(self.path):
            return out
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                pw = float(parts[3]) if parts[3] not in ("", "[N/A]") else 0.0
                rows.append((float(parts[1]), float(parts[2]), pw, parts[5], parts[6], parts[7], parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return out
        out["sm_mhz"] = float(np.median([r[0] for r in rows]))
        out["sm_max_mhz"] = float(max(r[1] for r in rows))
        out["power_w_max"] = float(max(r[2] for r in rows))
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for n, v in zip(names, r[3:]):
                if v.lower() == "active":
                    reasons.add(n)
        out["reasons"] = sorted(reasons)
        out["samples"] = len(rows)
        return out


# ------------------------------------------------------------ multi-rank timing

def max_over_ranks(ms: float, dist=None, device=None) -> float:
    """The largest of the ranks' times (the job ends with its slowest rank); identity
    without a process group. ``device`` is where the reduction tensor lives (a CUDA device
    for NCCL, the CPU for gloo)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_rate(units_per_rank: int, world: int, steps: int, max_ms: float) -> float:
    """Whole-job throughput: every rank processes its own batch of units each step."""
    return world * units_per_rank * steps / (max_ms * 1e-3)


# ----------------------------------------------------------------- workloads

def make_workload(name: str, n: int | None = None, inner: str = "micnn"):
    import workload as wl
    kw = {} if n is None else ({"n_qp": n} if name == "c3" else {"n": n})
    if name == "c3":
        kw["inner"] = inner
    return {"c0": wl.workload_c0, "c1": wl.workload_c1, "c2": wl.workload_c2, "c3": wl.workload_c3,
            "c4": wl.workload_c4, "ncm": wl.workload_paper_ncm, "cann": wl.workload_cann,
            "gt": wl.workload_gent_thomas, "ickan": wl.workload_ickan, "resid": wl.workload_residual}[name](**kw)


def wl_sub(mesh, el):
    import workload as wl
    return wl.Mesh(X=mesh.X, conn=mesh.conn[el], n=mesh.n)


def oracle_residual_loss_gradient(oracle, m, sub, u, free):
    """The residual-loss gradient chain of the oracle on a (sub)mesh: u -> F -> P -> r,
    lam = free * r, then dL/dP, (dL/dF, dL/dtheta) and dL/du."""
    F = oracle.compute_F(sub, u)
    _, P, _ = oracle.const_update(m, F, want_A=False)
    f_e, _ = oracle.elem_assemble(sub, P, None, want_K=False)
    lam = free * oracle.scatter_residual(sub, f_e)
    G = oracle.residual_adjoint(sub, lam.reshape(-1, 3))
    dF, dth = oracle.const_backward(m, F, G)
    return oracle.compute_F_adjoint(sub, dF), dth


def special_points(F: np.ndarray, cap: int = 4096):
    """Indices of the points with |J - 1| < 1e-3 and of those with J < 0.8 (at most `cap`
    of each, evenly spread), where the cancellation in J - 1 and the strong compression
    test the reduced precisions."""
    J = np.linalg.det(F.reshape(-1, 3, 3))
    out = {}
    for key, sel in (("J_near_1", np.abs(J - 1.0) < 1e-3), ("J_below_0.8", J < 0.8)):
        idx = np.nonzero(sel)[0]
        if idx.size > cap:
            idx = idx[np.linspace(0, idx.size - 1, cap).astype(np.int64)]
        out[key] = idx
    return out


def cpu_baseline_leg(w, n_el_sample: int, with_elements: bool = True, spatial: bool = False):
    """The FP64 oracle on the host cores, timed on a fixed strided sample of the workload:
    every k-th element with its 8 points (update + element assembly), or every point of
    the backward workload (stress + loss + backward over all points). Besides the rate it
    returns the oracle's outputs on the sample, and (untimed) on the points of
    `special_points`, which the bench line's per-output error statement compares the GPU
    outputs with."""
    import oracle
    oracle.build()
    spec = w["model"]
    m = oracle.OracleModel(spec)
    res = {"outputs": {}, "special": {}}
    if "mesh" not in w:  # c3: the backward over every point (its gradient sums all of them)
        n = w["F"].shape[0]
        F = w["F"]
        tgt = oracle.OracleModel(None, inner=oracle.INNER_HGO, kin=1, fibres=spec.fibres, **w["target"])
        t0 = time.perf_counter()
        _, Pt, _ = oracle.const_update(tgt, F, want_A=False)
        _, P, _ = oracle.const_update(m, F, want_A=False)
        dF, dth, dth_abs = oracle.const_backward(m, F, 2.0 * (P - Pt), want_abs=True)
        secs = time.perf_counter() - t0
        res.update(qps=n / secs, eps=None, secs=secs, what=f"all {n} points, FP64 stress + loss + backward",
                   idx_qp=np.arange(n), idx_el=None)
        res["outputs"] = {"dL/dF": dF, "dL/dtheta": dth, "dL/dtheta_abs": dth_abs}
        return res
    mesh = w["mesh"]
    if "free" in w:  # the residual-loss gradient chain on a prefix of the mesh
        el = np.arange(min(n_el_sample // 16, mesh.n_el))
        sub = wl_sub(mesh, el)
        t0 = time.perf_counter()
        oracle_residual_loss_gradient(oracle, m, sub, w["u"], w["free"])
        secs = time.perf_counter() - t0
        res.update(qps=8 * el.size / secs, eps=el.size / secs, secs=secs,
                   what=f"first {el.size} elements and their {8 * el.size} points, FP64 residual-loss gradient chain",
                   idx_qp=None, idx_el=None)
        return res
    n_s = min(n_el_sample, mesh.n_el)
    el = np.linspace(0, mesh.n_el - 1, n_s).astype(np.int64) if n_s < mesh.n_el else np.arange(mesh.n_el)
    qp = (8 * el[:, None] + np.arange(8)).ravel()
    F = w["F"][qp] if "F" in w else oracle.compute_F(wl_sub(mesh, el), w["u"])
    t0 = time.perf_counter()
    psi, P, A = oracle.const_update(m, F)
    if with_elements:
        f_e, K_e = oracle.elem_assemble(mesh, P, A, el=el)
    secs = time.perf_counter() - t0
    stride = f"every {mesh.n_el // n_s}th element" if n_s < mesh.n_el else "every element"
    res.update(qps=8 * el.size / secs, eps=el.size / secs if with_elements else None, secs=secs,
               what=f"{stride} ({el.size} elements, {8 * el.size} points), FP64 update"
                    + (" + element assembly" if with_elements else ""),
               idx_qp=qp, idx_el=el if with_elements else None)
    res["outputs"] = {"psi": psi, "P": P, "A": A, "F": F}
    if with_elements:
        res["outputs"].update(f_e=f_e, K_e=K_e.reshape(-1, 576))
    if spatial:
        # the push-forward of the oracle's P and A (App. A.1) on the first 65,536 sampled points
        ns = min(65536, F.shape[0])
        tau, c = oracle.push_forward(F[:ns], P[:ns], A[:ns])
        res["outputs"].update(tau=tau, c=c, n_spatial=ns)
    if "F" in w:
        for key, idx in special_points(w["F"]).items():
            if idx.size:
                sp_psi, sp_P, sp_A = oracle.const_update(m, w["F"][idx])
                res["special"][key] = {"idx_qp": idx, "psi": sp_psi, "P": sp_P, "A": sp_A, "F": w["F"][idx]}
    return res


def z16_errors(gpu_pm: np.ndarray, ref_pm: np.ndarray, floor_of: str = "rms") -> dict:
    """Per-point (or per-element) relative error |X_gpu - X_ref|_F / max(|X_ref|_F,
    1e-3 RMS |X_ref|_F) over a sample: its maximum, 99th percentile and median. With
    floor_of = "median" the floor is 1e-3 of the median norm instead (heavy-tailed outputs,
    whose RMS a few points dominate)."""
    g = np.asarray(gpu_pm, dtype=np.float64).reshape(gpu_pm.shape[0], -1)
    r = np.asarray(ref_pm, dtype=np.float64).reshape(ref_pm.shape[0], -1)
    nr = np.linalg.norm(r, axis=1)
    if not nr.size:
        floor = 0.0
    elif floor_of == "median":
        floor = 1e-3 * float(np.median(nr))
    else:
        floor = 1e-3 * np.sqrt(np.mean(nr ** 2))
    e = np.linalg.norm(g - r, axis=1) / np.maximum(np.maximum(nr, floor), 1e-300)
    if not e.size:
        return {"n": 0}
    return {"n": int(e.size), "max": float(e.max()), "p99": float(np.percentile(e, 99)),
            "median": float(np.median(e))}


# --------------------------------------------------------------- our kernels

class Run:
    """Device buffers and the phases of one step for a workload."""

    def __init__(self, name, w, prec, dev, pkg, torch, spatial=False):
        self.name, self.w, self.prec, self.dev = name, w, prec, dev
        self.spatial = spatial
        dt = torch.float64 if prec == "f64" else torch.float32
        self.dt = dt
        spec = w["model"]
        self.spec = spec
        self.model = pkg.Model(spec, prec)
        self.mesh = w.get("mesh")
        mp = "f64" if prec == "f64" else "f32"
        if name in ("c1", "c2", "ncm", "cann", "gt", "ickan"):
            F_host = np.ascontiguousarray(w["F"].T)
            self.inputs_host = {"F": F_host}
            n = F_host.shape[1]
            self.n_qp, self.n_el = n, n // 8
            self.F = torch.from_numpy(F_host).to(device=dev, dtype=dt).contiguous()
            self.psi = torch.empty(n, dtype=dt, device=dev)
            if spatial:
                # Kirchhoff stress and spatial stiffness in Voigt form (6 + 21 values per point)
                self.P = torch.empty(6, n, dtype=dt, device=dev)
                self.A = torch.empty(21, n, dtype=dt, device=dev)
                self.phases = [("const_update_kernel", lambda: self.model.const_update_spatial(
                    self.F, out=(self.psi, self.P, self.A)))]
            else:
                self.P = torch.empty(9, n, dtype=dt, device=dev)
                self.A = torch.empty(81, n, dtype=dt, device=dev)
                self.phases = [("const_update_kernel",
                                lambda: self.model.const_update(self.F, out=(self.psi, self.P, self.A)))]
            self.outputs = [self.psi, self.P, self.A]
            if name in ("c1", "ncm", "cann", "gt", "ickan"):
                self.gmesh = pkg.Mesh(self.mesh.X, self.mesh.conn)
                self.f_e = torch.empty(24, self.n_el, dtype=dt, device=dev)
                self.K_e = torch.empty(576, self.n_el, dtype=dt, device=dev)
                self.outputs += [self.f_e, self.K_e]
                if spatial:
                    self.phases.append(("elem_spatial_kernel", lambda: self.gmesh.elem_assemble_spatial(
                        self.F, self.P, self.A, mp, out=(self.f_e, self.K_e, None, None))))
                else:
                    self.phases.append(("elem_assemble_kernel", lambda: self.gmesh.elem_assemble(
                        self.P, self.A, mp, out=(self.f_e, self.K_e, None, None), symmetric=True)))
            else:
                self.n_el = 0
            self.input_dev = {"F": self.F}
        elif name == "c0":
            self.gmesh = pkg.Mesh(self.mesh.X, self.mesh.conn)
            u_host = np.ascontiguousarray(w["u"].T)
            self.inputs_host = {"u": u_host}
            self.u = torch.from_numpy(u_host).to(device=dev, dtype=dt).contiguous()
            self.n_el = self.mesh.n_el
            self.n_qp = 8 * self.n_el
            n = self.n_qp
            self.Fb = torch.empty(9, n, dtype=dt, device=dev)
            self.psi = torch.empty(n, dtype=dt, device=dev)
            self.P = torch.empty(9, n, dtype=dt, device=dev)
            self.A = torch.empty(81, n, dtype=dt, device=dev)
            self.f_e = torch.empty(24, self.n_el, dtype=dt, device=dev)
            self.K_e = torch.empty(576, self.n_el, dtype=dt, device=dev)
            self.outputs = [self.psi, self.P, self.A, self.f_e, self.K_e]
            self.phases = [("compute_F_kernel", lambda: self.gmesh.compute_F(self.u, mp, out=self.Fb)),
                           ("const_update_kernel",
                            lambda: self.model.const_update(self.Fb, out=(self.psi, self.P, self.A))),
                           ("elem_assemble_kernel", lambda: self.gmesh.elem_assemble(
                               self.P, self.A, mp, out=(self.f_e, self.K_e, None, None), symmetric=True))]
            self.input_dev = {"u": self.u}
        elif name == "c3":
            F_host = np.ascontiguousarray(w["F"].T)
            n = F_host.shape[1]
            self.n_qp, self.n_el = n, 0
            self.F = torch.from_numpy(F_host).to(device=dev, dtype=dt).contiguous()
            t = w["target"]
            self.Pt = pkg.target_stress(self.F, spec.fibres, t["mu"], t["k1"], t["k2"], t["kappa"])
            self.inputs_host = {"F": F_host, "Pt": self.Pt.cpu().numpy()}
            self.P = torch.empty(9, n, dtype=dt, device=dev)
            self.G = torch.empty(9, n, dtype=dt, device=dev)
            nb = int(pkg._lib.load().commet_const_backward_workspace(self.model.handle, n))
            self.ws = torch.empty(max(1, nb), dtype=torch.uint8, device=dev)
            self.dF = torch.empty_like(self.F)
            self.dth = torch.empty(self.model.n_params, dtype=dt, device=dev)

            def bw():
                self.model.backward(self.F, self.G, workspace=self.ws, out=(self.dF, self.dth))

            def loss_grad():
                torch.sub(self.P, self.Pt, out=self.G)
                self.G.mul_(2.0)
            self.phases = [("const_update_kernel", lambda: self.model.const_update(
                               self.F, want_A=False, want_psi=False, out=(None, self.P, None))),
                           ("loss_gradient (torch elementwise)", loss_grad),
                           ("const_backward_kernel", bw)]
            self.outputs = [self.dF]
            self.input_dev = {"F": self.F, "Pt": self.Pt}
        elif name == "resid":
            # u -> F -> P (stress) -> r, then dL/dr -> dL/dP -> (dL/dF, dL/dtheta) -> dL/du
            self.gmesh = g = pkg.Mesh(self.mesh.X, self.mesh.conn, want_csr=True)
            u_host = np.ascontiguousarray(w["u"].T)
            self.inputs_host = {"u": u_host}
            self.u = torch.from_numpy(u_host).to(device=dev, dtype=dt).contiguous()
            self.free = torch.from_numpy(w["free"]).to(device=dev, dtype=dt)
            self.n_el = self.mesh.n_el
            self.n_qp = n = 8 * self.n_el
            self.Fb = torch.empty(9, n, dtype=dt, device=dev)
            self.P = torch.empty(9, n, dtype=dt, device=dev)
            self.r = torch.empty(3 * self.mesh.n_nodes, dtype=dt, device=dev)
            self.lam = torch.empty_like(self.r)
            self.G = torch.empty(9, n, dtype=dt, device=dev)
            self.dF = torch.empty_like(self.Fb)
            self.dth = torch.empty(self.model.n_params, dtype=dt, device=dev)
            self.du = torch.empty_like(self.u)
            nb = int(pkg._lib.load().commet_const_backward_workspace(self.model.handle, n))
            self.ws = torch.empty(max(1, nb), dtype=torch.uint8, device=dev)

            def lam_of_r():
                torch.mul(self.r, self.free, out=self.lam)
            self.phases = [("compute_F_kernel", lambda: g.compute_F(self.u, mp, out=self.Fb)),
                           ("const_update_kernel", lambda: self.model.const_update(
                               self.Fb, want_A=False, want_psi=False, out=(None, self.P, None))),
                           ("elem_assemble_kernel", lambda: g.elem_assemble(
                               self.P, None, mp, want_f=False, want_K=False, want_r=True, out=(None, None, self.r, None))),
                           ("loss_gradient (torch elementwise)", lam_of_r),
                           ("residual_adjoint_kernel", lambda: g.residual_adjoint(self.lam, mp, out=self.G)),
                           ("const_backward_kernel", lambda: self.model.backward(
                               self.Fb, self.G, workspace=self.ws, out=(self.dF, self.dth))),
                           ("compute_F_adjoint_kernel", lambda: g.compute_F_adjoint(self.dF, mp, out=self.du))]
            self.outputs = [self.du, self.dth]
            self.input_dev = {"u": self.u}
        elif name == "c4":
            self.gmesh = pkg.Mesh(self.mesh.X, self.mesh.conn, want_csr=True)
            u_host = np.ascontiguousarray(w["u"].T)
            self.inputs_host = {"u": u_host}
            self.u = torch.from_numpy(u_host).to(device=dev, dtype=dt).contiguous()
            self.n_el = self.mesh.n_el
            self.n_qp = 8 * self.n_el
            self.r = torch.empty(3 * self.mesh.n_nodes, dtype=dt, device=dev)
            self.Kv = torch.empty(self.gmesh.nnz, dtype=dt, device=dev)
            self.outputs = [self.r, self.Kv]
            self.phases = [("newton_kernel", lambda: pkg.newton_assemble(self.model, self.gmesh, self.u,
                                                                         out=(self.r, self.Kv)))]
            self.input_dev = {"u": self.u}
        else:
            raise SystemExit(f"unknown workload {name}")

    def step(self):
        for _, fn in self.phases:
            fn()

    def step_outputs(self):
        return [self.dF] if self.name == "c3" else self.outputs


def time_steps(run, torch, warmup: int, steps: int) -> float:
    """Mean ms per step of a Run on the current stream (CUDA events)."""
    for _ in range(warmup):
        run.step()
    stream = torch.cuda.current_stream()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(steps):
        run.step()
    t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / steps


def fp64_unfused_baseline(run, pkg, torch, dev, reps=2):
    """The unfused FP64 GPU path on the same mesh and field (compute_F, const_update,
    elem_assemble with the colour scatter): ms per pass."""
    spec, mesh = run.spec, run.mesh
    m64 = pkg.Model(spec, "f64")
    u = run.u.double()
    n = run.n_qp
    F = torch.empty(9, n, dtype=torch.float64, device=dev)
    P = torch.empty(9, n, dtype=torch.float64, device=dev)
    A = torch.empty(81, n, dtype=torch.float64, device=dev)
    r = torch.empty(3 * mesh.n_nodes, dtype=torch.float64, device=dev)
    Kv = torch.empty(run.gmesh.nnz, dtype=torch.float64, device=dev)

    def once():
        run.gmesh.compute_F(u, "f64", out=F)
        m64.const_update(F, want_psi=False, out=(None, P, A))
        run.gmesh.elem_assemble(P, A, "f64", want_f=False, want_K=False, out=(None, None, r, Kv), symmetric=True)
    once()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        once()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    del F, P, A, r, Kv
    torch.cuda.empty_cache()
    return ms


def launches_per_step(run) -> int:
    """Kernels of this library launched by one step (the torch elementwise op of c3 is not one)."""
    n = 0
    for name, _ in run.phases:
        if name == "newton_kernel":
            n += run.gmesh.n_colours
        elif name == "const_backward_kernel":
            n += 2
        elif name == "elem_assemble_kernel" and run.name == "resid":
            n += run.gmesh.n_colours
        elif name == "compute_F_adjoint_kernel":
            n += run.gmesh.n_colours
        elif not name.startswith("loss_gradient"):
            n += 1
    return n


def error_statement(run, leg, torch) -> dict | None:
    """Error of the step's outputs against the FP64 oracle per output, on the CPU-baseline
    sample (the oracle's outputs on the FP64 inputs, so the reduced precisions' rounding
    of F is part of their error): the per-point measure of z16_errors for psi, P, A (or
    tau, c) and per element for f_e, K_e; separately on the points with |J - 1| < 1e-3 and
    with J < 0.8; for the backward, dL/dF per point and dL/dtheta per parameter block
    against the sum of the magnitudes of its per-point terms."""
    out = leg.get("outputs") or {}
    if not out:
        return None

    def cols(t, idx):
        it = torch.from_numpy(np.asarray(idx, dtype=np.int64)).to(t.device)
        return t.index_select(1, it).double().cpu().numpy().T

    res = {"against": "FP64 oracle on the FP64 inputs", "measure": "per point |X - X_ref|_F / max(|X_ref|_F, "
           "1e-3 RMS|X_ref|_F): max, p99, median over the sample", "sample": leg["what"]}
    if run.name == "c3":
        spec = run.spec
        heavy = getattr(spec, "inner_name", "micnn") != "micnn"
        gdF = run.dF.double().cpu().numpy().T
        keep = np.isfinite(gdF).all(axis=1)
        n_drop = int((~keep).sum())
        res["dL/dF"] = z16_errors(gdF[keep], out["dL/dF"][keep], "median" if heavy else "rms")
        if heavy:
            res["dL/dF"]["floor"] = "1e-3 of the median norm (the CANN's exponential terms give a heavy tail)"
        if n_drop:
            # points the GPU left out (non-finite in this precision, reported as NaN): the
            # oracle's gradient is taken again over the kept points
            import oracle
            w = run.w
            m = oracle.OracleModel(spec)
            tgt = oracle.OracleModel(None, inner=oracle.INNER_HGO, kin=1, fibres=spec.fibres, **w["target"])
            F = w["F"][keep]
            _, Pt, _ = oracle.const_update(tgt, F, want_A=False)
            _, P, _ = oracle.const_update(m, F, want_A=False)
            _, dth_k, abs_k = oracle.const_backward(m, F, 2.0 * (P - Pt), want_abs=True)
            out = dict(out, **{"dL/dtheta": dth_k, "dL/dtheta_abs": abs_k})
            res["dL/dF"]["n_nonfinite_dropped"] = n_drop
        if getattr(spec, "inner_name", "micnn") == "micnn":
            d, W, L = spec.d, spec.W, spec.L
            sizes = [W * d, W] + [W * W, W * d, W] * (L - 1) + [W, d]
        else:
            sizes = [2 * spec.n] * spec.d  # the CANN's (w1, w2) of each input's terms
        g, r, a = run.dth.double().cpu().numpy(), out["dL/dtheta"], out["dL/dtheta_abs"]
        blk, o = [], 0
        for n in sizes:
            blk.append(float(np.linalg.norm(g[o:o + n] - r[o:o + n]) / max(np.linalg.norm(a[o:o + n]), 1e-300)))
            o += n
        res["dL/dtheta"] = {"blocks": len(blk), "max_block": max(blk),
                            "measure": "per block |dtheta - ref|_2 / |sum_q |dtheta_q||_2",
                            "rel_l2": float(np.linalg.norm(g - r) / np.linalg.norm(r))}
        return res
    iq = leg["idx_qp"]
    if run.spatial:
        ns = out.get("n_spatial", 0)
        if ns:
            res["tau"] = z16_errors(cols(run.P, iq[:ns]), out["tau"])
            res["c"] = z16_errors(cols(run.A, iq[:ns]), out["c"])
            res["spatial_points"] = int(ns)
        res["psi"] = z16_errors(cols(run.psi[None, :], iq), out["psi"][:, None])
    else:
        res["psi"] = z16_errors(cols(run.psi[None, :], iq), out["psi"][:, None])
        res["P"] = z16_errors(cols(run.P, iq), out["P"])
        res["A"] = z16_errors(cols(run.A, iq), out["A"])
    if "f_e" in out and leg.get("idx_el") is not None:
        res["f_e"] = z16_errors(cols(run.f_e, leg["idx_el"]), out["f_e"])
        res["K_e"] = z16_errors(cols(run.K_e, leg["idx_el"]), out["K_e"])
    if not run.spatial:
        for key, sp in leg.get("special", {}).items():
            res[key] = {"n": int(sp["idx_qp"].size), "P": z16_errors(cols(run.P, sp["idx_qp"]), sp["P"]),
                        "A": z16_errors(cols(run.A, sp["idx_qp"]), sp["A"])}
    return res


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2510_00884_gb300 as pkg

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    pkg.build()
    name = args.workload
    prec = args.precision or ("f32" if name == "c4" else "f64")
    w = make_workload(name, args.n, args.inner)
    if args.spatial and name not in ("c1", "c2", "ncm", "cann", "gt", "ickan"):
        raise SystemExit("--spatial applies to the c1, c2, ncm, cann, gt and ickan workloads")
    run = Run(name, w, prec, dev, pkg, torch, spatial=args.spatial)
    stream = torch.cuda.current_stream()
    dist = world > 1
    if dist:
        import torch.distributed as tdist

    def barrier():
        if dist:
            tdist.barrier()

    for _ in range(args.warmup):
        run.step()
    torch.cuda.synchronize()

    n_steps = args.steps
    nph = len(run.phases)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(nph + 1)] for _ in range(n_steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        barrier()
        torch.cuda.synchronize()
        t_start.record(stream)
        for s in range(n_steps):
            ev[s][0].record(stream)
            for p, (_, fn) in enumerate(run.phases):
                fn()
                ev[s][p + 1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
        barrier()
    total_ms = t_start.elapsed_time(t_end)
    phase_ms = [float(np.mean([e[p].elapsed_time(e[p + 1]) for e in ev])) for p in range(nph)]
    clocks = clk.summary()
    if dist:
        total_ms = max_over_ranks(total_ms, tdist, dev)
    ms_per_step = total_ms / n_steps
    qps = weak_scaling_rate(run.n_qp, world, n_steps, total_ms)
    eps = weak_scaling_rate(run.n_el, world, n_steps, total_ms) if run.n_el else None

    # ---- end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        pin_in = {k: torch.from_numpy(v).to(run.dt).pin_memory() for k, v in run.inputs_host.items()}
        outs = run.step_outputs()
        outs_h = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in outs]
        h2d = sum(t.numel() * t.element_size() for t in pin_in.values())
        d2h = sum(t.numel() * t.element_size() for t in outs_h)

        e2e_path = "device calls between pinned copies on one stream"
        if name in ("c1", "c2", "ncm", "cann", "gt", "ickan") and not args.spatial:
            # the host-buffer entry point: chunks copied in, computed and copied out on
            # three streams (commet_const_update_host)
            gm = getattr(run, "gmesh", None)
            # rows of at least 128 KB in the strided host copies (576 rows of K_e per chunk)
            chunk = (16384 if prec == "f64" else 32768) if gm is not None else 131072
            lib = pkg._lib.load()
            need = int(lib.commet_const_update_host_workspace(run.model.handle, gm.handle if gm else None, chunk, 1))
            ws_host = torch.empty(need, dtype=torch.uint8, device=dev)
            outs5 = tuple(outs_h) + (None,) * (5 - len(outs_h))
            e2e_path = f"commet_const_update_host, chunks of {chunk} {'elements' if gm is not None else 'points'}"

            def e2e_step():
                run.model.const_update_host(pin_in["F"], gm, out=outs5, chunk=chunk, workspace=ws_host)
        else:
            def e2e_step():
                for k, t in pin_in.items():
                    run.input_dev[k].copy_(t, non_blocking=True)
                run.step()
                for src, dst in zip(run.step_outputs(), outs_h):
                    dst.copy_(src, non_blocking=True)
        for _ in range(max(1, args.warmup)):
            e2e_step()
        torch.cuda.synchronize()
        n_e2e = max(1, min(n_steps, 5))
        barrier()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(n_e2e):
            e2e_step()
        t1.record(stream)
        torch.cuda.synchronize()
        barrier()
        e_ms = t0.elapsed_time(t1)
        if dist:
            e_ms = max_over_ranks(e_ms, tdist, dev)
        e2e = {"value": weak_scaling_rate(run.n_qp, world, n_e2e, e_ms), "unit": "qp/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": n_e2e,
               "ms_per_step": e_ms / n_e2e, "path": e2e_path}

    fp64_base = None
    if name in ("c1", "c2", "c3", "ncm", "cann", "gt", "ickan", "resid") and prec != "f64" and not args.no_baseline \
            and rank == 0:
        # the same step through the plain FP64 path of the same kernels
        run64 = Run(name, w, "f64", dev, pkg, torch, spatial=args.spatial)
        b_ms = time_steps(run64, torch, 2, 3)
        fp64_base = {"what": "same step, FP64 path", "ms_per_step": b_ms, "qp_per_s": run.n_qp / (b_ms * 1e-3),
                     "speedup_of_" + prec: b_ms / ms_per_step}
        del run64
        torch.cuda.empty_cache()
    if name == "c4" and not args.no_baseline and rank == 0:
        b_ms = fp64_unfused_baseline(run, pkg, torch, dev)
        fp64_base = {"what": "unfused FP64 GPU path (compute_F, const_update, elem_assemble + colour scatter)",
                     "ms_per_step": b_ms, "qp_per_s": run.n_qp / (b_ms * 1e-3),
                     "speedup_of_fused": b_ms / ms_per_step}

    if rank != 0:
        return None

    # ---- roofline of the dominant kernel
    peaks, peak_src = load_peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    spec = run.spec
    sW, sL = getattr(spec, "W", 0), getattr(spec, "L", 0)
    inner_name = getattr(spec, "inner_name", "micnn")
    net = f"d{spec.d}w{sW}l{sL}" if inner_name == "micnn" else f"{inner_name}_d{spec.d}"
    dom = int(np.argmax(phase_ms))
    kname = run.phases[dom][0]
    alu = "f64" if prec == "f64" else "f32"
    if kname == "const_update_kernel":
        per_qp = algorithmic_flops_per_qp(spec.d, sW, sL) + (2 * PUSH_FORWARD_MACS if args.spatial else 0)
        flops = per_qp * run.n_qp
        units = run.n_qp
        src = ["spatial.cu" if args.spatial else "const_update.cu", "update_kernel.cuh", "qp_body.cuh",
               "device_math.cuh"] + ([] if inner_name == "micnn" else ["closed_form.cuh"])
    elif kname == "const_backward_kernel":
        flops = backward_flops_per_qp(spec.d, sW, sL) * run.n_qp
        units, src = run.n_qp, ["backward.cu", "qp_body.cuh", "device_math.cuh", "closed_form.cuh"]
    elif kname == "newton_kernel":
        flops = (algorithmic_flops_per_qp(spec.d, sW, sL) * 8 + 2 * ELEM_MACS) * run.n_el
        units, src = run.n_el, ["newton.cu", "qp_body.cuh", "device_math.cuh"]
    else:
        # the FP64 material form runs the symmetric element kernel (the update's own tangent)
        sym = kname == "elem_assemble_kernel" and prec == "f64"
        flops = 2 * (ELEM_MACS_SYM if sym else ELEM_MACS) * run.n_el
        units, src = run.n_el, ["spatial.cu" if kname == "elem_spatial_kernel" else "elem.cu", "hex8.cuh"]
    peak, peak_source = alu_peak(alu, n_sm, mhz)
    bound = "alu"
    if prec == "bf16" and kname == "const_update_kernel":
        # the hidden W x W products run on the tensor cores: values, adjoints and the d
        # tangent channels of every hidden layer, 2 (L-1) W^2 (2 + d) flops per point
        flops = 2 * (sL - 1) * sW * sW * (2 + spec.d) * run.n_qp
        bound = "tensor"
        peak = float(peaks.get("bf16_tflops", 1900.0))
        peak_source = (f"bf16 dense matmul burst ({peak_src} peaks file); tcgen05.mma kind::f16, M 128, "
                       f"fp32 accumulate in tensor memory")
        src = ["bf16_update.cu", "umma.cuh", "device_math.cuh"]
    achieved = flops / (phase_ms[dom] * 1e-3) / 1e12
    bounds = None
    if prec == "bf16" and kname == "const_update_kernel":
        # the four ceilings of this kernel: tensor (the hidden products above), MUFU (exp,
        # reciprocal and log per neuron), FP32 (the algorithmic multiply-adds outside the
        # hidden products) and HBM (F in; psi, P, A out)
        sec = phase_ms[dom] * 1e-3
        mufu = 3 * sL * sW * run.n_qp
        f32_flops = algorithmic_flops_per_qp(spec.d, sW, sL) * run.n_qp - flops
        per_qp = (9 + 1 + (6 + 21 if args.spatial else 9 + 81)) * 4
        mufu_peak, mufu_src = mufu_peak_tops(n_sm, mhz)
        f32_peak, f32_src = alu_peak("f32", n_sm, mhz)
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        bounds = {
            "tensor": {"achieved_tflops": achieved, "peak": peak, "frac": achieved / peak},
            "mufu": {"achieved_tops": mufu / sec / 1e12, "peak": mufu_peak, "frac": mufu / sec / 1e12 / mufu_peak,
                     "ops_per_qp": 3 * sL * sW, "peak_source": mufu_src},
            "fp32": {"achieved_tflops": f32_flops / sec / 1e12, "peak": f32_peak,
                     "frac": f32_flops / sec / 1e12 / f32_peak, "peak_source": f32_src},
            "hbm": {"achieved_gbs": per_qp * run.n_qp / sec / 1e9, "peak": hbm,
                    "frac": per_qp * run.n_qp / sec / 1e9 / hbm, "bytes_per_qp": per_qp},
        }
    src_hash = kernel_source_hash(src)
    roofline = {"bound": bound, "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": ncu_traffic(kname, net, prec, src_hash, units),
                "peak_source": peak_source,
                "algorithmic_flops_per_launch": flops, "kernel_ms": phase_ms[dom],
                "frac_at_median_clock": (achieved / peak * mhz / clocks["sm_mhz"]) if clocks.get("sm_mhz") else None,
                "src_hash": src_hash}
    if bounds is not None:
        roofline["bounds"] = bounds
    if kname == "const_update_kernel" and getattr(spec, "inner_name", "micnn") != "micnn":
        # no network: the algorithmic work is the output stream (9 in, 1 + 9 + 81 or
        # 1 + 6 + 21 out per point), so the roofline is HBM
        es = 8 if prec == "f64" else 4
        per_qp = (9 + 1 + (6 + 21 if args.spatial else 9 + 81)) * es
        bts = per_qp * run.n_qp / (phase_ms[dom] * 1e-3) / 1e9
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        roofline = {"bound": "hbm", "kernel": kname, "achieved": bts, "peak": hbm, "unit": "GB/s",
                    "frac": bts / hbm, "traffic": ncu_traffic(kname, net, prec, src_hash, units),
                    "bytes_per_qp": per_qp, "src_hash": src_hash,
                    "peak_source": f"measured HBM copy ({peak_src} peaks file)", "kernel_ms": phase_ms[dom]}
    if kname == "const_backward_kernel" and getattr(spec, "inner_name", "micnn") != "micnn":
        # the CANN's backward: a few dozen operations per point around the forward's
        # closed form; the algorithmic work is the stream of F and G in and dL/dF out
        es = 8 if prec == "f64" else 4
        per_qp = 27 * es
        bts = per_qp * run.n_qp / (phase_ms[dom] * 1e-3) / 1e9
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        roofline = {"bound": "hbm", "kernel": kname, "achieved": bts, "peak": hbm, "unit": "GB/s",
                    "frac": bts / hbm, "traffic": ncu_traffic(kname, net, prec, src_hash, units),
                    "bytes_per_qp": per_qp, "src_hash": src_hash,
                    "peak_source": f"measured HBM copy ({peak_src} peaks file)", "kernel_ms": phase_ms[dom]}
    phases = {n_: ms for (n_, _), ms in zip(run.phases, phase_ms)}
    ek = "elem_spatial_kernel" if args.spatial else "elem_assemble_kernel"
    if ek in phases:
        es = 8 if prec == "f64" else 4
        el_ms = phases[ek]
        per_qp = 36 if args.spatial else 90  # F, tau, c  or  P, A
        roofline["elem_kernel"] = {"kernel": ek, "ms": el_ms, "bytes_per_el": (8 * per_qp + 600) * es,
                                   "achieved_gbs": run.n_el * (8 * per_qp + 600) * es / (el_ms * 1e-3) / 1e9,
                                   "hbm_peak_gbs": float(peaks.get("hbm_gbs", 6800.0)),
                                   "achieved_tflops": run.n_el * 2 * (ELEM_MACS if args.spatial or prec != "f64"
                                                                      else ELEM_MACS_SYM) / (el_ms * 1e-3) / 1e12}

    cpu = None
    errors = None
    if not args.no_cpu_baseline and world == 1:
        leg = cpu_baseline_leg(w, args.cpu_sample_el, with_elements=hasattr(run, "f_e"), spatial=args.spatial)
        cpu = {"value": leg["qps"], "unit": "qp/s", "cores": os.cpu_count() or 1, "kind": "oracle",
               "sample": f"{leg['what']} of {w['name']}, {leg['secs']:.1f} s", "elements_per_s": leg["eps"]}
        errors = error_statement(run, leg, torch)

    cfg = {"workload": w["name"], "n_qp": run.n_qp, "n_el": run.n_el, "network": (f"d{spec.d} W{sW} L{sL}" if getattr(spec, "inner_name", "micnn") == "micnn"
                                           else f"{spec.inner_name} d{spec.d}"),
           "precision": prec, "outputs": "tau, c (Voigt, spatial)" if args.spatial else "P, A (material)", "parallelism": f"replicas x{world} (independent meshes)",
           "l2": "inputs/outputs larger than L2 (129 MB) every step"}
    res = {
        "metric": METRIC, "value": qps, "unit": "qp/s", "n_gpus": world, "steps": n_steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": prec, "data": "synthetic (seeded; random non-negative MICNN weights)",
        "elements_per_s": eps, "phases_ms": phases, "config": cfg, "roofline": roofline, "cpu_baseline": cpu,
        "e2e": e2e, "gpu_launches": n_steps * launches_per_step(run), "clocks": clocks,
        "errors": errors,
    }
    if fp64_base is not None:
        res["fp64_unfused_gpu" if name == "c4" else "fp64_gpu"] = fp64_base
    return res


# ----------------------------------------------------------- reference arm

def run_reference(args):
    """The FP64 oracle on the host cores; each step is a bounded sample of the workload."""
    import oracle
    oracle.build()
    name = args.workload
    w = make_workload(name, args.n, args.inner)
    spec = w["model"]
    m = oracle.OracleModel(spec)
    if "free" in w:
        mesh = w["mesh"]
        n_el_s = min(args.ref_sample_el // 16, mesh.n_el)
        sub = wl_sub(mesh, np.arange(n_el_s))
        n_qp_s = 8 * n_el_s

        def step():
            oracle_residual_loss_gradient(oracle, m, sub, w["u"], w["free"])
        sample = f"first {n_el_s} elements / {n_qp_s} points of {w['name']} per step, FP64 residual-loss gradient"
    elif "mesh" in w:
        mesh = w["mesh"]
        n_el_s = min(args.ref_sample_el, mesh.n_el)
        el = np.arange(n_el_s)
        F = w["F"][: 8 * n_el_s] if "F" in w else oracle.compute_F(wl_sub(mesh, el), w["u"])
        n_qp_s = 8 * n_el_s

        def step():
            _, P, A = oracle.const_update(m, F)
            oracle.elem_assemble(mesh, P, A, el=el)
        sample = f"first {n_el_s} elements / {n_qp_s} points of {w['name']} per step, FP64 update + assembly"
    else:
        n_qp_s = min(8 * args.ref_sample_el, w["F"].shape[0])
        n_el_s = 0
        F = w["F"][:n_qp_s]
        tgt = oracle.OracleModel(None, inner=oracle.INNER_HGO, kin=1, fibres=spec.fibres, **w["target"])
        _, Pt, _ = oracle.const_update(tgt, F, want_A=False)

        def step():
            _, P, _ = oracle.const_update(m, F, want_A=False)
            oracle.const_backward(m, F, 2.0 * (P - Pt))
        sample = f"first {n_qp_s} points of {w['name']} per step, FP64 stress + backward"
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    secs = time.perf_counter() - t0
    qps = n_qp_s * args.steps / secs
    threads = os.cpu_count() or 1
    return {
        "impl": "reference", "metric": METRIC, "value": qps, "unit": "qp/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "elements_per_s": (n_el_s * args.steps / secs) if n_el_s else None,
        "config": {"workload": w["name"], "precision": "f64", "sample_qp": n_qp_s},
        "cpu_baseline": {"value": qps, "unit": "qp/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": qps, "unit": "qp/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# --------------------------------------------------------- twisting cube

def run_twist(args):
    """The FE benchmark of Sec. 4.3 on the GPU: a unit cube of n^3 hex8 elements (the paper's
    largest is 128^3, 6,440,067 dofs) clamped at x = 0; the x = 1 face is stretched by 1 and
    turned by half a turn in `--twist-steps` load steps. A timed step is the first load step
    solved from u = 0: a predictor that moves the fixed dofs through the system, then Newton
    iterations of FP64 assembly (u -> r, K), Dirichlet rows and columns, Jacobi-CG
    (rtol 1e-8) and the update, until |r_free| <= 1e-8 max(1, |r_free| after the predictor).
    Reports assembly and solve time separately, as the paper compares them."""
    import torch
    import workload as wl
    import paper_2510_00884_gb300 as pkg
    pkg.build()
    dev = torch.device("cuda", 0)
    n = args.n or 32
    mesh = wl.structured_mesh(n)
    spec = wl.workload_paper_ncm(n=1)["model"]
    gm = pkg.Mesh(mesh.X, mesh.conn, want_csr=True)
    model = pkg.Model(spec, "f64")
    dofs, vals = wl.twist_dirichlet(mesh, 1.0 / args.twist_steps)
    gm.set_dirichlet(dofs)
    u = torch.zeros(3, mesh.n_nodes, dtype=torch.float64, device=dev)
    assemble = pkg.Assembler(model, gm)  # FP64: separate update and element kernels
    du = torch.empty(3 * mesh.n_nodes, dtype=torch.float64, device=dev)
    ws = torch.empty(int(pkg._lib.load().commet_cg_workspace(gm.handle, 0)), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def load_step(times):
        # predictor (fixed dofs moved by their increment through the system), then Newton
        u.zero_()
        r0, newton, cg_its = None, 0, 0
        for it in range(30):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            r, Kv = assemble(u)
            gm.apply_dirichlet(r, Kv, delta=vals if it == 0 else None)
            e1.record(stream)
            if it > 0:
                rn = gm.norm2(r)
                r0 = rn if r0 is None else r0
                if rn <= 1e-8 * max(1.0, r0):
                    times["assembly"].append((e0, e1, None))
                    break
            _, n_cg, _ = gm.cg_solve(Kv, r, "f64", 1e-8, 50000, x=du, workspace=ws)
            gm.add_increment(du, -1.0, u)
            if it == 0:
                gm.set_dirichlet_values(vals, u)
            e2.record(stream)
            times["assembly"].append((e0, e1, e2))
            newton += 1
            cg_its += n_cg
        return newton, cg_its

    for _ in range(max(1, args.warmup)):
        load_step({"assembly": []})
    torch.cuda.synchronize()
    times = {"assembly": []}
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    its = [load_step(times) for _ in range(args.steps)]
    t1.record(stream)
    torch.cuda.synchronize()
    total = t0.elapsed_time(t1) / args.steps
    asm = sum(a.elapsed_time(b) for a, b, _ in times["assembly"]) / args.steps
    sol = sum(b.elapsed_time(c) for a, b, c in times["assembly"] if c is not None) / args.steps
    newton = its[0][0]
    res = {"metric": "twisting-cube load step (Sec. 4.3): Newton with GPU assembly and Jacobi-CG",
           "value": newton * 8 * mesh.n_el / (total * 1e-3), "unit": "assembled qp/s over the load step",
           "ms_per_load_step": total, "assembly_ms": asm, "solve_ms": sol, "newton_iterations": newton,
           "cg_iterations": its[0][1], "dofs": 3 * mesh.n_nodes, "n_el": mesh.n_el, "nnz": gm.nnz,
           "steps": args.steps, "warmup": args.warmup, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"twist_{n}cube", "network": "paper NCM d3 W16 L3 (675 parameters)",
                      "load": f"1/{args.twist_steps} of a unit stretch and a half turn", "cg_rtol": 1e-8}}
    print(json.dumps(res), flush=True)


# ------------------------------------------------------------------ sweeps

def run_sweep(args):
    """GPU analogues of the paper's material-point studies (one JSON line per case):
      size   model size (App. D): MICNN on the polyconvex inputs with L in {2, 3, 4} hidden
             layers and W in {2, 4, 8, 16, 32, 64} (W = 2 runs zero-padded to 4), plus the CANN
             and Gent-Thomas laws, at
             2^21 points per launch, P and A in FP64 and FP32 (and the bf16 tcgen05 MLP for
             W = 32, 64)
      batch  points per launch (the paper's batch size, Sec. 4.1) from 2^8 to 2^24 for the
             paper's NCM (3 x 16, 675 parameters), FP64 and FP32
    Each case: 3 warm-up launches, then the mean of `steps` launches timed with CUDA events."""
    import torch
    import workload as wl
    import paper_2510_00884_gb300 as pkg
    pkg.build()
    dev = torch.device("cuda", 0)
    peaks, _ = load_peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    rng = np.random.Generator(np.random.PCG64(11))

    def timed(model, F, out):
        for _ in range(3):
            model.const_update(F, out=out)
        s = torch.cuda.current_stream()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(s)
        for _ in range(args.steps):
            model.const_update(F, out=out)
        t1.record(s)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / args.steps

    def case(spec, label, n, prec, F_host):
        dt = torch.float64 if prec == "f64" else torch.float32
        F = torch.from_numpy(np.ascontiguousarray(F_host[:n].T)).to(device=dev, dtype=dt).contiguous()
        out = (torch.empty(n, dtype=dt, device=dev), torch.empty(9, n, dtype=dt, device=dev),
               torch.empty(81, n, dtype=dt, device=dev))
        try:
            m = pkg.Model(spec, prec)
            ms = timed(m, F, out)
        except pkg._lib.CommetError as e:
            print(json.dumps({"sweep": args.sweep, "case": label, "precision": prec, "n_qp": n, "error": str(e)}),
                  flush=True)
            return
        rec = {"sweep": args.sweep, "case": label, "precision": prec, "n_qp": n, "ms": ms,
               "qp_per_s": n / (ms * 1e-3), "n_params": m.n_params}
        if getattr(spec, "inner_name", "micnn") == "micnn" and prec == "bf16":
            # hidden products on the tensor cores against the bf16 matmul peak (headline),
            # with the MUFU and FP32 ceilings of the rest, as in the single-workload line
            sec = ms * 1e-3
            tc = 2 * (spec.L - 1) * spec.W * spec.W * (2 + spec.d) * n
            rest = algorithmic_flops_per_qp(spec.d, spec.W, spec.L) * n - tc
            tpk = float(peaks.get("bf16_tflops", 1900.0))
            mpk = mufu_peak_tops(n_sm, mhz)[0]
            fpk = alu_peak("f32", n_sm, mhz)[0]
            mufu = 3 * spec.L * spec.W * n / sec / 1e12
            rec.update({"bound": "tensor", "achieved_tflops": tc / sec / 1e12, "frac": tc / sec / 1e12 / tpk,
                        "mufu_frac": mufu / mpk, "fp32_frac": rest / sec / 1e12 / fpk})
        elif getattr(spec, "inner_name", "micnn") == "micnn":
            fl = algorithmic_flops_per_qp(spec.d, spec.W, spec.L) * n / (ms * 1e-3) / 1e12
            pk = alu_peak("f64" if prec == "f64" else "f32", n_sm, mhz)[0]
            rec.update({"bound": "alu", "achieved_tflops": fl, "frac": fl / pk})
        else:
            es = 8 if prec == "f64" else 4
            gbs = 100 * es * n / (ms * 1e-3) / 1e9
            rec.update({"bound": "hbm", "achieved_gbs": gbs, "frac": gbs / float(peaks.get("hbm_gbs", 6800.0))})
        del F, out, m
        torch.cuda.empty_cache()
        print(json.dumps(rec), flush=True)

    n_max = 1 << (24 if args.sweep == "batch" else 21)
    F_host = wl.random_F(rng, n_max, 0.15)
    if args.sweep == "size":
        for L in (2, 3, 4):
            for W in (2, 4, 8, 16, 32, 64):
                spec = wl.make_model(np.random.Generator(np.random.PCG64(100 * L + W)), wl.KIN_POLYCONVEX, 0,
                                     W=W, L=L, kappa=0.0)
                for prec in ("f64", "f32") + (("bf16",) if W >= 32 else ()):
                    case(spec, f"micnn L{L} W{W}", n_max, prec, F_host)
        for label, spec in (("cann (paper, 4 terms)", wl.make_cann(np.random.Generator(np.random.PCG64(9)))),
                            ("gent-thomas", wl.GentThomasSpec())):
            for prec in ("f64", "f32"):
                case(spec, label, n_max, prec, F_host)
    else:
        spec = wl.workload_paper_ncm(n=1)["model"]
        for prec in ("f64", "f32"):
            for e in range(8, 25, 2):
                case(spec, "paper NCM 3x16", 1 << e, prec, F_host)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["c0", "c1", "c2", "c3", "c4", "ncm", "cann", "gt", "ickan", "resid"],
                    default="c1")
    ap.add_argument("--n", type=int, default=None, help="mesh size per side (points for c3)")
    ap.add_argument("--inner", choices=["micnn", "cann"], default="micnn",
                    help="c3 only: the network (the C1 MICNN) or the paper's CANN")
    ap.add_argument("--precision", choices=["f64", "f32", "bf16"], default=None,
                    help="default: f64 (f32 for c4)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--spatial", action="store_true",
                    help="c1/c2/ncm: spatial Voigt outputs tau, c and the spatial element kernel")
    ap.add_argument("--no-baseline", action="store_true", help="skip the FP64 GPU timing beside a reduced-precision step (c4: the unfused FP64 path)")
    ap.add_argument("--twist", action="store_true",
                    help="the twisting-cube Newton benchmark of Sec. 4.3 (--n elements per side)")
    ap.add_argument("--twist-steps", type=int, default=20)
    ap.add_argument("--sweep", choices=["size", "batch"], default=None,
                    help="model-size or batch-size sweep of the update (one JSON line per case)")
    ap.add_argument("--cpu-sample-el", type=int, default=262144,
                    help="elements (c3: half the points) of the workload the CPU baseline runs on")
    ap.add_argument("--ref-sample-el", type=int, default=4096)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.sweep is not None:
        run_sweep(args)
        return
    if args.twist:
        run_twist(args)
        return
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
    res = run_ours(args, rank, world, local_rank)
    if rank == 0 and res is not None:
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
