"""Benchmark of the neural-constitutive hot path on one node (one rank per GPU).

A step is one pass of the whole hot path over the workload's batch, with inputs
resident in HBM: the fused constitutive update (F -> Psi, P, A for every quadrature
point) followed by the hex8 element integrals (P, A -> f_int, K_e for every element).
The default workload is the 64^3 anisotropic mesh (262,144 elements, 2,097,152 points,
two-fibre MICNN d7 W32 L3) in FP64.

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


# ------------------------------------------------------------------ helpers

def algorithmic_flops_per_qp(d: int, W: int, L: int) -> int:
    """Minimal exact work per point, in flops (2 per multiply-add), counted as stated in
    the design doc: network values W d + (L-1)(W^2 + W d), reverse adjoints (L-1) W^2 plus the
    gradient L W d, tangents (L-1) W^2 d, Hessian L W d(d+1)/2, and the rank-one part of A
    (9 d^2 + 81 d). Kinematics, activations and the structured terms of A are not counted."""
    macs = W * d + (L - 1) * (W * W + W * d)
    macs += (L - 1) * W * W + L * W * d
    macs += (L - 1) * W * W * d
    macs += L * W * d * (d + 1) // 2
    macs += 9 * d * d + 81 * d
    return 2 * macs


ELEM_FLOPS = 2 * 8 * (3 * 27 * 3 + 3 * 8 * 3 * 3)  # per element: 8 qp x (T3 + row contractions), MACs x 2


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


def kernel_source_hash(files) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2510_00884_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, network: str, precision: str, src_hash: str, n_qp: int):
    """Per-launch DRAM bytes of the kernel from the committed ncu summary, scaled from the
    captured case to n_qp points; None when the kernel source changed since the capture."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        tab = json.load(f)
    e = tab.get(f"{kernel}|{network}|{precision}")
    if not e or e.get("src_hash") != src_hash:
        return None
    return e["dram_bytes"] * n_qp / e["n_qp"]


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
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]) if parts[3] not in ("", "[N/A]") else 0.0,
                             parts[5], parts[6], parts[7], parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return out
        sm = np.array([r[0] for r in rows])
        out["sm_mhz"] = float(np.median(sm))
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


# ----------------------------------------------------------------- workloads

def make_workload(name: str, n: int | None = None):
    import workload as wl
    if name == "c1":
        return wl.workload_c1() if n is None else wl.workload_c1(n=n)
    if name == "c0":
        w = wl.workload_c0()
        return w
    raise SystemExit(f"unknown workload {name}")


def cpu_sample_rate(w, n_el_sample: int, threads: int):
    """Oracle throughput (qp/s through update + element assembly) on the first
    n_el_sample elements and their 8 n_el_sample points."""
    import oracle
    os.environ.setdefault("OMP_NUM_THREADS", str(threads))
    oracle.build()
    mesh, spec = w["mesh"], w["model"]
    el = np.arange(min(n_el_sample, mesh.n_el))
    F = w["F"][: 8 * el.size] if "F" in w else oracle.compute_F(mesh, w["u"])[: 8 * el.size]
    m = oracle.OracleModel(spec)
    t0 = time.perf_counter()
    _, P, A = oracle.const_update(m, F)
    t1 = time.perf_counter()
    oracle.elem_assemble(mesh, P, A, el=el)
    t2 = time.perf_counter()
    return 8 * el.size / (t2 - t0), el.size / (t2 - t0), t2 - t0


# --------------------------------------------------------------- our kernels

def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2510_00884_gb300 as pkg

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    pkg.build()
    w = make_workload(args.workload, args.n)
    prec = args.precision
    dt = torch.float64 if prec == "f64" else torch.float32
    spec, mesh = w["model"], w["mesh"]
    model = pkg.Model(spec, prec)
    gmesh = pkg.Mesh(mesh.X, mesh.conn)
    n_el = mesh.n_el
    if "F" in w:
        F_host = np.ascontiguousarray(w["F"].T)
    else:
        import torch as _t
        u = _t.from_numpy(np.ascontiguousarray(w["u"].T)).to(dev)
        F_host = gmesh.compute_F(u, "f64").cpu().numpy()
    n_qp = F_host.shape[1]
    F = torch.from_numpy(F_host).to(device=dev, dtype=dt).contiguous()
    psi = torch.empty(n_qp, dtype=dt, device=dev)
    P = torch.empty(9, n_qp, dtype=dt, device=dev)
    A = torch.empty(81, n_qp, dtype=dt, device=dev)
    f_e = torch.empty(24, n_el, dtype=dt, device=dev)
    K_e = torch.empty(576, n_el, dtype=dt, device=dev)
    stream = torch.cuda.current_stream()

    def step(Fin):
        model.const_update(Fin, out=(psi, P, A))
        gmesh.elem_assemble(P, A, prec, out=(f_e, K_e, None, None))

    dist = world > 1
    if dist:
        import torch.distributed as tdist

    def barrier():
        if dist:
            tdist.barrier()

    for _ in range(args.warmup):
        step(F)
    torch.cuda.synchronize()

    n_steps = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(n_steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        barrier()
        torch.cuda.synchronize()
        t_start.record(stream)
        for s in range(n_steps):
            ev[s][0].record(stream)
            model.const_update(F, out=(psi, P, A))
            ev[s][1].record(stream)
            gmesh.elem_assemble(P, A, prec, out=(f_e, K_e, None, None))
            ev[s][2].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
        barrier()
    total_ms = t_start.elapsed_time(t_end)
    cu_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    el_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in ev]))
    clocks = clk.summary()
    if dist:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / n_steps
    qps = world * n_qp * n_steps / (total_ms * 1e-3)
    eps = world * n_el * n_steps / (total_ms * 1e-3)

    # ---- end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        F_pin = torch.from_numpy(F_host).to(dt).pin_memory()
        outs_h = [torch.empty(t.shape, dtype=dt).pin_memory() for t in (psi, P, A, f_e, K_e)]
        h2d = F_pin.numel() * F_pin.element_size()
        d2h = sum(t.numel() * t.element_size() for t in outs_h)
        Fd = torch.empty_like(F)

        def e2e_step():
            Fd.copy_(F_pin, non_blocking=True)
            step(Fd)
            for src, dst in zip((psi, P, A, f_e, K_e), outs_h):
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
            t = torch.tensor([e_ms], device=dev, dtype=torch.float64)
            tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
            e_ms = float(t.item())
        e2e = {"value": world * n_qp * n_e2e / (e_ms * 1e-3), "unit": "qp/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": n_e2e,
               "ms_per_step": e_ms / n_e2e}

    if rank != 0:
        return None

    # ---- roofline of the dominant kernel (the fused constitutive update)
    peaks, peak_src = load_peaks()
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    flops_qp = algorithmic_flops_per_qp(spec.d, spec.W, spec.L)
    peak = alu_peak_tflops(prec, n_sm, float(peaks.get("sm_max_mhz", 2070.0)))
    achieved = flops_qp * n_qp / (cu_ms * 1e-3) / 1e12
    src_hash = kernel_source_hash(["const_update.cu", "device_math.cuh"])
    traffic = ncu_traffic("const_update_kernel", f"d{spec.d}w{spec.W}l{spec.L}", prec, src_hash, n_qp)
    roofline = {"bound": "alu", "kernel": "const_update_kernel", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "peak_source": f"derived: {n_sm} SMs x {'2 DFMA' if prec == 'f64' else '128 FFMA'}/clk x "
                               f"{peaks.get('sm_max_mhz', 2070.0):.0f} MHz (max SM clock, {peak_src} peaks file)",
                "algorithmic_flops_per_qp": flops_qp, "kernel_ms": cu_ms,
                "frac_at_median_clock": (achieved / peak * float(peaks.get("sm_max_mhz", 2070.0)) /
                                         clocks["sm_mhz"]) if clocks.get("sm_mhz") else None,
                "elem_kernel": {"ms": el_ms, "bytes_per_el": (8 * 90 + 600) * (8 if prec == "f64" else 4),
                                "achieved_gbs": n_el * (8 * 90 + 600) * (8 if prec == "f64" else 4) / (el_ms * 1e-3) / 1e9,
                                "hbm_peak_gbs": float(peaks.get("hbm_gbs", 6800.0)),
                                "achieved_tflops": n_el * ELEM_FLOPS / (el_ms * 1e-3) / 1e12}}

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        threads = os.cpu_count() or 1
        qps_cpu, eps_cpu, secs = cpu_sample_rate(w, args.cpu_sample_el, threads)
        cpu = {"value": qps_cpu, "unit": "qp/s", "cores": threads, "kind": "oracle",
               "sample": f"first {min(args.cpu_sample_el, n_el)} elements and their "
                         f"{8 * min(args.cpu_sample_el, n_el)} points of the same workload, FP64, "
                         f"update + element assembly, {secs:.1f} s",
               "elements_per_s": eps_cpu}

    return {
        "metric": METRIC, "value": qps, "unit": "qp/s", "n_gpus": world, "steps": n_steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": prec, "data": "synthetic (seeded; random non-negative MICNN weights)",
        "elements_per_s": eps,
        "config": {"workload": w["name"], "n_qp": n_qp, "n_el": n_el, "network": f"d{spec.d} W{spec.W} L{spec.L}",
                   "precision": prec, "parallelism": f"replicas x{world} (independent meshes)",
                   "l2": "inputs larger than L2: F %.0f MB, A %.0f MB per step" %
                         (9 * n_qp * F.element_size() / 1e6, 81 * n_qp * F.element_size() / 1e6)},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 2 * n_steps,
        "clocks": clocks,
    }


# ----------------------------------------------------------- reference arm

def run_reference(args):
    """The FP64 oracle on the host cores; each step is a bounded sample of the workload."""
    import oracle
    threads = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(threads))
    oracle.build()
    w = make_workload(args.workload, args.n)
    mesh, spec = w["mesh"], w["model"]
    n_el_s = min(args.ref_sample_el, mesh.n_el)
    el = np.arange(n_el_s)
    F = w["F"][: 8 * n_el_s] if "F" in w else oracle.compute_F(mesh, w["u"])[: 8 * n_el_s]
    m = oracle.OracleModel(spec)

    def step():
        _, P, A = oracle.const_update(m, F)
        oracle.elem_assemble(mesh, P, A, el=el)
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    secs = time.perf_counter() - t0
    qps = 8 * n_el_s * args.steps / secs
    sample = f"first {n_el_s} elements / {8 * n_el_s} points of {w['name']} per step, FP64"
    return {
        "impl": "reference", "metric": METRIC, "value": qps, "unit": "qp/s", "n_gpus": 0, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "elements_per_s": n_el_s * args.steps / secs,
        "config": {"workload": w["name"], "n_qp": 8 * mesh.n_el, "n_el": mesh.n_el, "precision": "f64",
                   "sample_el": n_el_s},
        "cpu_baseline": {"value": qps, "unit": "qp/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": qps, "unit": "qp/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c1")
    ap.add_argument("--n", type=int, default=None, help="mesh size per side (default: the workload's)")
    ap.add_argument("--precision", choices=["f64", "f32"], default="f64")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-el", type=int, default=65536)
    ap.add_argument("--ref-sample-el", type=int, default=4096)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
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
