"""Benchmark: scaled-stencil apply GDoF/s and %HBM peak, plus GMG-CG time to
relative residual 1e-8, on the unit cube split into 6 macro tetrahedra at
level 8 (255^3 = 16.6M unknowns), k = exp(sin(pi x) cos(pi y) z).

One timed step = one application of the full scaled operator (volume kernel
fused with the interface/Dirichlet pass, one launch) in FP32 on inputs
resident in HBM; L2 is flushed (512 MiB write) before every step, outside the
per-step CUDA events.  The solve figures come from separate FP32+FP64-
refinement and plain-FP64 GMG-CG solves of the manufactured problem.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun) runs N independent replicas (the multi-GPU interface
exchange is not built); `value` sums the replicas.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LEVEL, COARSEST = 8, 2
METRIC = "scaled-stencil apply GDoF/s & %HBM peak; GMG-CG time to rel. residual 1e-8"
WORKLOAD = "unit cube, 6 Kuhn macro-tets, level 8 (257 nodes/edge), k=exp(sin(pi x)cos(pi y)z)"

# ncu DRAM traffic (read+write bytes) per launch of the FP32 scaled apply on
# this workload, with the sha256 of the kernel source it was measured on; the
# figure is dropped (null) as soon as the kernel source changes.
# DRAM bytes of one apply (volume kernel 204.35 MB read + 55.10 MB written,
# interface kernel 73.77 MB read + 5.76 MB written), one ncu capture each;
# keyed on the hash of the scaled apply's sources
NCU_TRAFFIC = {"apply_sha": "ed3981851f0e6303", "bytes": 338974208}


def _code_only(src):
    """C++ source without comments and blank lines (a change of comments
    leaves the compiled kernels, and so a traffic record, valid)."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())


def _kernel_sha():
    """Hash of the scaled apply's sources (kernels and shared constants),
    code only."""
    h = hashlib.sha256()
    for f in ("apply.cu", "hhg_internal.h"):
        h.update(_code_only(open(os.path.join(ROOT, "paper_1709_06793_gb300", "csrc", f)).read()).encode())
    return h.hexdigest()[:16]


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """Samples nvidia-smi SM clocks / throttle reasons during the timed region."""

    def __init__(self, gpu):
        self.gpu, self.rows, self.proc = gpu, [], None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(2)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 3 + i and r[3 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def cpu_baseline(repeats=3):
    """The FP64 oracle's element-loop apply on the same cube and k at level 6
    (1/512 of the level-8 work), single-threaded numpy."""
    from oracle import hhg_oracle as O
    from paper_1709_06793_gb300 import inputs as I
    V, T = I.kuhn_cube()
    lm = O.LevelMesh(O.MacroMesh(V, T), 6)
    k = I.k_cube(lm.coords)
    u = np.where(lm.dirichlet, 0.0, I.uniform_from_keys(I.node_keys(lm.node_gverts, lm.node_weights, lm.N), 0))
    lm.apply(u, k, "scaled")
    t0 = time.perf_counter()
    for _ in range(repeats):
        lm.apply(u, k, "scaled")
    dt = (time.perf_counter() - t0) / repeats
    dof = len(lm.unknowns)
    return {"value": dof / dt / 1e9, "unit": "GDoF/s", "cores": 1, "kind": "oracle",
            "sample": f"oracle element-loop scaled apply, same cube/k at level 6 ({dof} unknowns), "
                      f"mean of {repeats}, numpy single thread"}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_time(ms, world):
    """Step time of the job: the slowest rank's (replicas, no data exchange;
    the only collective is this reduction of the timing)."""
    if world == 1:
        return ms
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(unknowns, ms, world):
    """Whole-job GDoF/s: every rank applies the operator to `unknowns`
    unknowns per step (weak scaling)."""
    return unknowns * world / (ms * 1e-3) / 1e9


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    base = cpu_baseline(repeats=1)
    times = []
    from oracle import hhg_oracle as O
    from paper_1709_06793_gb300 import inputs as I
    V, T = I.kuhn_cube()
    lm = O.LevelMesh(O.MacroMesh(V, T), 6)
    k = I.k_cube(lm.coords)
    u = np.where(lm.dirichlet, 0.0, np.sin(lm.coords[:, 0]))
    for _ in range(args.warmup):
        lm.apply(u, k, "scaled")
    for _ in range(args.steps):
        t0 = time.perf_counter()
        lm.apply(u, k, "scaled")
        times.append(time.perf_counter() - t0)
    dt = float(np.mean(times))
    val = len(lm.unknowns) / dt / 1e9
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GDoF/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "level": 8, "macro_tets": 6, "parallelism": "single"},
           "cpu_baseline": {"value": val, "unit": "GDoF/s", "cores": 1, "kind": "oracle",
                            "sample": "each step one " + base["sample"].split(", mean of")[0]
                                      + " (a level-8 apply would take minutes); rate per unknown"},
           "e2e": {"value": val, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


LEARNED_LEVEL = 7
LEARNED_WORKLOAD = ("unit cube, 6 Kuhn macro-tets, level 7 (129 nodes/edge), k=exp(2g), g a Gaussian random field "
                    "(correlation length 0.2, contrast 1e2); 2x16-channel 3x3x3 conv smoother, BF16 weights")
# FP32 lanes: 152 SMs x 128 lanes x 2 flops (FMA) x 2070 MHz (maximum SM clock)
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def learned_bench(H, I, torch, stream, flush):
    """C4: train the learned smoother on the GPU, then time GMG-CG to 1e-8
    with and without it, and time its forward kernel."""
    V, T = I.kuhn_cube()
    m = H.Mesh(V, T, LEARNED_LEVEL, COARSEST)
    off, lev, n = m.layout(0)
    xyz = m.coords(0)
    H.hhg_set_coefficient(m.h, torch.tensor(I.k_learned()(xyz), device="cuda"))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = H.hhg_learned_train(m.h, steps=120, pairs=4, lr=3e-3, max_depth=1, vcycle_pairs=2, init_noise=0.02,
                             seed=3, weights_bf16=1)
    train_s = time.perf_counter() - t0
    fi = torch.tensor(I.f_cube_sine(xyz), device="cuda")
    f = torch.empty_like(fi)
    H.hhg_apply_mass(m.h, 0, fi, f, H.HHG_F64)
    out = {"workload": LEARNED_WORKLOAD, "stored_nodes": n, "train_s": train_s, "train": st}
    for name, mode, sm in (("fp64", H.HHG_SOLVE_FP64, H.HHG_SMOOTH_JACOBI),
                           ("mixed", H.HHG_SOLVE_MIXED, H.HHG_SMOOTH_JACOBI),
                           ("mixed_learned", H.HHG_SOLVE_MIXED, H.HHG_SMOOTH_LEARNED)):
        u = torch.zeros(n, device="cuda", dtype=torch.float64)
        H.hhg_solve(m.h, f, u, tol=1e-8, mode=mode, smoother=sm, raise_on_fail=False)
        u.zero_()
        torch.cuda.synchronize()
        r = H.hhg_solve(m.h, f, u, tol=1e-8, mode=mode, smoother=sm, raise_on_fail=False)
        out[name] = {"ms": r["time_ms"], "iterations": r["iterations"], "rel_residual": r["rel_residual"],
                     "smoother_used": r["smoother_used"], "status": r["status"]}
    out["speedup_learned_vs_fp64"] = out["fp64"]["ms"] / out["mixed_learned"]["ms"]
    out["speedup_learned_vs_mixed"] = out["mixed"]["ms"] / out["mixed_learned"]["ms"]
    # forward kernel (one learned correction at depth 0) and one Jacobi sweep
    rr = torch.randn(n, device="cuda", dtype=torch.float32)
    cc = torch.empty_like(rr)
    uu = torch.zeros_like(rr)

    def timed(fn, reps=20):
        for _ in range(3):
            fn()
        ts = []
        for i in range(reps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.mean(ts))

    H.hhg_set_option(m.h, "learned_tc_all", 1)
    tc_ms = timed(lambda: H.hhg_learned_forward(m.h, 0, rr, cc, stream))
    H.hhg_set_option(m.h, "learned_tc_all", 0)
    fwd_ms = timed(lambda: H.hhg_learned_forward(m.h, 0, rr, cc, stream))
    jac_ms = timed(lambda: H.hhg_smooth(m.h, 0, H.HHG_SMOOTH_JACOBI, 1, 2.0 / 3.0, rr, uu, H.HHG_F32, stream))
    flops = 2 * 1296 * n  # 864 + 432 multiply-adds per stored node
    peaks, src = _peaks()
    ach_tc = flops / (tc_ms * 1e-3) / 1e12
    ach = flops / (fwd_ms * 1e-3) / 1e12
    out["forward_tensor_core"] = {
        "ms": tc_ms, "ratio_to_jacobi": tc_ms / jac_ms,
        "roofline": {"bound": "tensor", "achieved": ach_tc, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                     "frac": ach_tc / peaks["bf16_tflops"], "peak_source": f"{src} bf16_tflops (burst)",
                     "algorithmic_flops_per_launch": flops}}
    out["forward_fp32_activations"] = {
        "ms": fwd_ms, "ratio_to_jacobi": fwd_ms / jac_ms,
        "roofline": {"bound": "alu", "achieved": ach, "peak": FP32_ALU_TFLOPS, "unit": "TFLOP/s",
                     "frac": ach / FP32_ALU_TFLOPS,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz",
                     "algorithmic_flops_per_launch": flops}}
    out["jacobi_sweep_ms"] = jac_ms
    m.close()
    return out


TABLE_LEVELS = (4, 5, 6, 7, 8)  # the paper's L = 2 .. 6 on the 6-tet cube


def paper_table(H, I, torch, m_big=None, levels=TABLE_LEVELS):
    """Shape of the paper's 3D scalar table (Sec. 7.2, Tab. "hhg_nonlinear",
    m = 3): 10 V(3,3) multigrid cycles in FP64 with nodal integration,
    scale Vol+Face and scale all; discrete L2 error (lumped mass) of the
    manufactured u = sin(pi x) sin(pi y) sin(pi z), eoc, rho and the time to
    solution relative to nodal integration.  Coefficient k = cos(3 pi x y z) + 2."""
    rows = []
    prev = {}
    kf, ff = I.k_cosine(3), I.f_sine_cosine_k(3)
    V, T = I.kuhn_cube()
    for level in levels:
        m = m_big if (m_big is not None and level == LEVEL) else H.Mesh(V, T, level, COARSEST)
        off, lev, n = m.layout(0)
        xyz = m.coords(0)
        H.hhg_set_coefficient(m.h, torch.tensor(kf(xyz), device="cuda"))
        fi = torch.tensor(ff(xyz), device="cuda")
        f = torch.empty_like(fi)
        H.hhg_apply_mass(m.h, 0, fi, f, H.HHG_F64)
        w = torch.empty_like(fi)
        H.hhg_apply_mass(m.h, 0, torch.ones_like(fi), w, H.HHG_F64)  # lumped mass weights
        ustar = torch.tensor(I.u_sine(xyz), device="cuda")
        row = {"level": level, "L": level - 2, "unknowns": ((1 << level) - 1) ** 3}
        for name, op in (("nodal", H.HHG_OP_NODAL), ("volface", H.HHG_OP_VOLFACE), ("scaled", H.HHG_OP_SCALED)):
            u = torch.zeros(n, device="cuda", dtype=torch.float64)
            H.hhg_solve(m.h, f, u, tol=1e-30, maxit=10, mode=H.HHG_SOLVE_MG, nu1=3, nu2=3, op=op,
                        raise_on_fail=False)  # warm: coarse inverse, diagonals
            u.zero_()
            torch.cuda.synchronize()
            st = H.hhg_solve(m.h, f, u, tol=1e-30, maxit=10, mode=H.HHG_SOLVE_MG, nu1=3, nu2=3, op=op,
                             raise_on_fail=False)
            e = u - ustar
            err = math.sqrt(max(H.hhg_dot(m.h, 0, w * e, e, H.HHG_F64), 0.0))
            eoc = math.log2(prev[name] / err) if name in prev else None
            prev[name] = err
            row[name] = {"error": err, "eoc": eoc, "rho": st["rho"], "tts_ms": st["time_ms"]}
        for name in ("volface", "scaled"):
            row[name]["rel_tts"] = row[name]["tts_ms"] / row["nodal"]["tts_ms"]
        rows.append(row)
        if m is not m_big:
            m.close()
    return {"workload": "unit cube, 6 Kuhn macro-tets, k = cos(3 pi x y z) + 2, u* = sin(pi x) sin(pi y) sin(pi z), "
                        "rhs M I_h f; 10 V(3,3) cycles (damped Jacobi, omega 2/3), FP64",
            "rows": rows}


def batch_bench(H, I, torch, flush):
    """48 independent random tetrahedra with levels drawn from 5..8 (seed 1),
    k = 1 + 0.9 tanh(8-mode Fourier field): the FP32 apply of all of them in
    one launch (autotuned work lists) and the mixed-precision GMG-CG solve of
    the 48 problems together (one V-cycle launch per stage, CUDA graphs)."""
    V, T = I.random_tets(48, seed=1)
    levels = np.random.default_rng(1).integers(5, 9, size=48)
    m = H.Mesh(V, T, levels, 3)
    off, lev, n = m.layout(0)
    xyz = m.coords(0)
    H.hhg_set_coefficient(m.h, torch.tensor(I.k_batched(1)(xyz), device="cuda"))
    tune = H.hhg_autotune(m.h, H.HHG_F32)
    u = torch.rand(n, device="cuda", dtype=torch.float32)
    mask = torch.empty_like(u)
    H.hhg_residual(m.h, 0, torch.ones_like(u), torch.zeros_like(u), mask, H.HHG_F32)
    u *= mask
    y = torch.empty_like(u)
    for _ in range(3):
        H.hhg_apply_scaled(m.h, 0, u, y, H.HHG_F32)
    ts = []
    for i in range(20):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        H.hhg_apply_scaled(m.h, 0, u, y, H.HHG_F32)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ms = float(np.mean(ts))
    unknowns = int(sum(((1 << int(l)) - 3) * ((1 << int(l)) - 2) * ((1 << int(l)) - 1) // 6 for l in levels))
    f = torch.tensor(np.sin(3 * xyz[:, 0]) * np.cos(2 * xyz[:, 1]) + xyz[:, 2], device="cuda") * mask.double()
    out = {"workload": "48 random tetrahedra (min angle 20 deg), levels 5..8 (seed 1), k = 1 + 0.9 tanh(Fourier field)",
           "levels": [int(l) for l in levels], "stored_nodes": n, "unknowns": unknowns, "autotune": tune,
           "apply_ms": ms, "apply_gdofs": unknowns / (ms * 1e-3) / 1e9,
           "apply_gbs_algorithmic": 12 * n / (ms * 1e-3) / 1e9}
    for name, mode in (("mixed", H.HHG_SOLVE_MIXED), ("fp64", H.HHG_SOLVE_FP64)):
        x = torch.zeros(n, device="cuda", dtype=torch.float64)
        H.hhg_solve(m.h, f, x, tol=1e-8, mode=mode, raise_on_fail=False)
        x.zero_()
        torch.cuda.synchronize()
        st = H.hhg_solve(m.h, f, x, tol=1e-8, mode=mode, raise_on_fail=False)
        out["solve_" + name] = {"ms": st["time_ms"], "iterations": st["iterations"], "rel_residual": st["rel_residual"]}
    m.close()
    return out


TENSOR_LEVELS = (3, 4, 5, 6, 7)  # the paper's L = 1 .. 5 on the 12-tet cube


def tensor_table(H, I, torch, flush, levels=TENSOR_LEVELS):
    """Shape of the paper's tensor test (Sec. 7.3, Tab. "divK4"): the 12-tet
    cube, its permeability tensor K, multigrid V(3,3) (FP64) until the
    residual drops by 1e-9; discrete L2 error of u* = sin(pi x) sin(pi y)
    sin(pi z), eoc, rho, time to solution.  Plus the FP32 tensor apply on the
    finest level against its HBM roofline (u, six k_m, y: 32 B per node)."""
    V, T = I.cube12()
    rows, prev = [], None
    apply = None
    for level in levels:
        m = H.Mesh(V, T, level, 1)
        off, lev, n = m.layout(0)
        xyz = m.coords(0)
        H.hhg_set_tensor_coefficient(m.h, torch.tensor(np.ascontiguousarray(I.K_tensor(xyz).T), device="cuda"))
        fi = torch.tensor(I.f_sine_tensor(xyz), device="cuda")
        f = torch.empty_like(fi)
        H.hhg_apply_mass(m.h, 0, fi, f, H.HHG_F64)
        w = torch.empty_like(fi)
        H.hhg_apply_mass(m.h, 0, torch.ones_like(fi), w, H.HHG_F64)
        u = torch.zeros(n, device="cuda", dtype=torch.float64)
        kw = dict(tol=1e-9, maxit=60, mode=H.HHG_SOLVE_MG, nu1=3, nu2=3, op=H.HHG_OP_TENSOR, raise_on_fail=False)
        H.hhg_solve(m.h, f, u, **kw)
        u.zero_()
        torch.cuda.synchronize()
        st = H.hhg_solve(m.h, f, u, **kw)
        e = u - torch.tensor(I.u_sine(xyz), device="cuda")
        err = math.sqrt(max(H.hhg_dot(m.h, 0, w * e, e, H.HHG_F64), 0.0))
        rows.append({"level": level, "L": level - 2, "stored_nodes": n, "error": err, "eoc": math.log2(prev / err) if prev else None, "rho": st["rho"],
                     "cycles": st["iterations"], "tts_ms": st["time_ms"]})
        prev = err
        if level == levels[-1]:
            x = torch.rand(n, device="cuda", dtype=torch.float32)
            y = torch.empty_like(x)
            for _ in range(3):
                H.hhg_apply_tensor(m.h, 0, x, y, H.HHG_F32)
            ts = []
            for i in range(10):
                flush.fill_(float(i))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                H.hhg_apply_tensor(m.h, 0, x, y, H.HHG_F32)
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            ms = float(np.mean(ts))
            peaks, src = _peaks()
            ach = 32 * n / (ms * 1e-3) / 1e9
            apply = {"level": level, "stored_nodes": n, "ms": ms,
                     "roofline": {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                  "frac": ach / peaks["hbm_gbs"], "algorithmic_bytes_per_node": 32}}
        m.close()
    return {"workload": "unit cube, 12 macro-tets, K = the paper's tensor (Sec. 7.3), u* = sin(pi x) sin(pi y) "
                        "sin(pi z); V(3,3) (damped Jacobi) to a 1e-9 residual reduction, FP64",
            "rows": rows, "apply_fp32": apply}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--level", type=int, default=LEVEL)
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-table", action="store_true", help="skip the multigrid tables (scalar and tensor)")
    ap.add_argument("--only-learned", action="store_true",
                    help="run only the learned-smoother section (C4) and print its JSON")
    ap.add_argument("--tune-cache", action="store_true", help="reuse/append autotuner results in _build_tune.txt")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1709_06793_gb300 import build, inputs as I
    build.build()
    from paper_1709_06793_gb300 import hhg as H

    if args.only_learned:
        flush = torch.empty(512 * 1024 * 1024 // 4, device="cuda", dtype=torch.float32)
        out = learned_bench(H, I, torch, torch.cuda.current_stream(), flush)
        if rank == 0:
            print(json.dumps({"learned": out}))
        return

    V, T = I.kuhn_cube()
    m = H.Mesh(V, T, args.level, COARSEST)
    off, lev, n = m.layout(0)
    xyz = m.coords(0)
    N = 1 << args.level
    unknowns = (N - 1) ** 3
    H.hhg_set_coefficient(m.h, torch.tensor(I.k_cube(xyz), device="cuda"))
    rng = np.random.default_rng(0)
    u = torch.tensor(rng.uniform(-1, 1, n), device="cuda", dtype=torch.float32)
    # zero Dirichlet entries: one apply of a zero-boundary vector gives the mask
    y = torch.empty_like(u)
    ones = torch.ones_like(u)
    dg = torch.empty_like(u)
    H.hhg_residual(m.h, 0, ones, torch.zeros_like(u), dg, H.HHG_F32)  # r = 1 at unknowns, 0 on Dirichlet
    u *= dg
    flush = torch.empty(512 * 1024 * 1024 // 4, device="cuda", dtype=torch.float32)
    stream = torch.cuda.current_stream()
    tune = H.hhg_autotune(m.h, H.HHG_F32, os.path.join(ROOT, "_build_tune.txt") if args.tune_cache else None)

    for _ in range(max(3, args.warmup)):
        H.hhg_apply_scaled(m.h, 0, u, y, H.HHG_F32, stream)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t0 = time.perf_counter()
        for s in range(args.steps):
            flush.fill_(float(s))
            starts[s].record(stream)
            H.hhg_apply_scaled(m.h, 0, u, y, H.HHG_F32, stream)
            ends[s].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    ms = replica_time(float(np.mean(step_ms)), world)

    # the other operators on the same workload (the paper's cost comparison)
    def _time_op(fn, reps=10):
        for _ in range(3):
            fn()
        ts = []
        for i in range(reps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.mean(ts))

    nodal_ms = _time_op(lambda: H.hhg_apply_nodal(m.h, 0, u, y, H.HHG_F32, stream))
    volface_ms = _time_op(lambda: H.hhg_apply_volface(m.h, 0, u, y, H.HHG_F32, stream))
    operators = {"scaled_ms": ms, "nodal_ms": nodal_ms, "volface_ms": volface_ms,
                 "nodal_over_scaled": nodal_ms / ms, "volface_over_scaled": volface_ms / ms}

    # end to end through the public API with host buffers: every step copies
    # its u from pinned host memory, applies the operator and reads its y back
    # into pinned host memory.  Sequential: one stream, copy-apply-copy.
    # Pipelined: two device buffer pairs, the copies on their own streams, so
    # the host-to-device copy of step s+1, the apply of step s and the
    # device-to-host copy of step s-1 overlap (the host link is full duplex);
    # events order the reuse of each buffer.
    uh = u.cpu().pin_memory()
    yh = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(2)]
    ub = [torch.empty_like(u) for _ in range(2)]
    yb = [torch.empty_like(u) for _ in range(2)]
    ke = max(10, args.steps)

    def seq_step():
        ub[0].copy_(uh, non_blocking=True)
        H.hhg_apply_scaled(m.h, 0, ub[0], yb[0], H.HHG_F32, stream)
        yh[0].copy_(yb[0], non_blocking=True)

    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    in_done = [torch.cuda.Event() for _ in range(2)]
    comp_done = [torch.cuda.Event() for _ in range(2)]
    out_done = [torch.cuda.Event() for _ in range(2)]
    for e in in_done + comp_done + out_done:
        e.record(stream)

    def pipe_step(q):
        b = q & 1
        s_in.wait_event(comp_done[b])  # the apply of step q-2 has read ub[b]
        with torch.cuda.stream(s_in):
            ub[b].copy_(uh, non_blocking=True)
        in_done[b].record(s_in)
        stream.wait_event(in_done[b])
        stream.wait_event(out_done[b])  # y of step q-2 has left yb[b]
        H.hhg_apply_scaled(m.h, 0, ub[b], yb[b], H.HHG_F32, stream)
        comp_done[b].record(stream)
        s_out.wait_event(comp_done[b])
        with torch.cuda.stream(s_out):
            yh[b].copy_(yb[b], non_blocking=True)
        out_done[b].record(s_out)

    def timed_e2e(step_fn):
        for q in range(3):
            step_fn(q)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s_in.wait_stream(stream)
        s_out.wait_stream(stream)
        for q in range(ke):
            step_fn(q)
        stream.wait_stream(s_in)
        stream.wait_stream(s_out)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / ke

    seq_ms = timed_e2e(lambda q: seq_step())
    e2e_ms = timed_e2e(pipe_step)
    e2e = {"value": unknowns / (e2e_ms * 1e-3) / 1e9 * world, "unit": "GDoF/s",
           "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 4 * n, "ms_per_step": e2e_ms,
           "pipelined": "two buffer pairs; H2D, apply and D2H of neighbouring steps on separate streams",
           "sequential_value": unknowns / (seq_ms * 1e-3) / 1e9 * world, "sequential_ms_per_step": seq_ms}

    peaks, src = _peaks()
    algo_bytes = 12 * n  # read u, k; write y (FP32), every stored node
    achieved = algo_bytes / (ms * 1e-3) / 1e9
    traffic = NCU_TRAFFIC["bytes"] if NCU_TRAFFIC["apply_sha"] == _kernel_sha() else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "peak_source": f"{src} hbm_gbs (burst)",
            "kernel": "scaled_op_kernel<float,float,APPLY> (volume rows) + boundary_only_kernel<float,float,APPLY> "
                      "(interface rows, concurrent on a side stream); one apply = one launch of each",
            "algorithmic_bytes_per_launch": algo_bytes}

    solve = None
    if not args.no_solve:
        solve = {}
        # right-hand side f_h = M I_h f (consistent mass matrix), f = -div(k grad u*) for
        # the manufactured u* = sin(pi x) sin(pi y) sin(pi z)
        fi = torch.tensor(I.f_cube_sine(xyz), device="cuda")
        f = torch.empty_like(fi)
        H.hhg_apply_mass(m.h, 0, fi, f, H.HHG_F64)
        runs = (("mixed_fp32_fp64refine", H.HHG_SOLVE_MIXED, H.HHG_SMOOTH_JACOBI),
                ("mixed_bf16k_fp64refine", H.HHG_SOLVE_MIXED_KBF16, H.HHG_SMOOTH_JACOBI),
                ("fp64", H.HHG_SOLVE_FP64, H.HHG_SMOOTH_JACOBI),
                ("mixed_fp32_fp64refine_cheb", H.HHG_SOLVE_MIXED, H.HHG_SMOOTH_CHEBYSHEV),
                ("fp64_cheb", H.HHG_SOLVE_FP64, H.HHG_SMOOTH_CHEBYSHEV))
        for name, mode, sm in runs:
            ud64 = torch.zeros(n, device="cuda", dtype=torch.float64)
            H.hhg_solve(m.h, f, ud64, tol=1e-8, mode=mode, smoother=sm, raise_on_fail=False)  # warm (setup, graphs)
            ud64.zero_()
            torch.cuda.synchronize()
            st = H.hhg_solve(m.h, f, ud64, tol=1e-8, mode=mode, smoother=sm, raise_on_fail=False)
            solve[name] = {"ms": st["time_ms"], "iterations": st["iterations"], "outer": st["outer"],
                           "rel_residual": st["rel_residual"], "status": st["status"]}
        solve["metric"] = ("GMG-preconditioned CG, V(2,2), wall time to ||f - A u||/||f|| <= 1e-8 from u = 0, "
                           "rhs M I_h f; FP64 outer residual in every mode")
        solve["speedup_mixed_vs_fp64"] = solve["fp64"]["ms"] / solve["mixed_fp32_fp64refine"]["ms"]

    table = tensor = None
    if not args.no_table:
        table = paper_table(H, I, torch, m_big=m)
        tensor = tensor_table(H, I, torch, flush)

    batch = batch_bench(H, I, torch, flush) if not args.no_solve else None

    learned = None
    if not args.no_learned:
        learned = learned_bench(H, I, torch, stream, flush)

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline()

    out = {"metric": METRIC, "value": job_rate(unknowns, ms, world), "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "level": args.level, "unknowns": unknowns, "stored_nodes": n,
                      "macro_tets": 6, "parallelism": f"replicas{world}" if world > 1 else "single",
                      "l2": "flushed before every step (512 MiB write, outside the step events)"},
           "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 2 * args.steps,
           "autotune": tune,
           "clocks": clk.summary(), "wall_s_timed_region": wall, "operators": operators, "solve": solve, "batch": batch, "learned": learned, "mg_table": table,
           "tensor_table": tensor}
    if rank == 0:
        print(json.dumps(out))
    m.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
