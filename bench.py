"""Benchmark of the stencil-scaled P1 operator on hierarchical hybrid grids.

Headline workload (the large configuration): the unit cube split into 24
macro tetrahedra (body centre, face centres; each face cut into 4 triangles
coned to the centre), every one refined to level 9 (513 nodes per macro edge,
543,184,920 stored nodes, 535,300,095 unknowns), FP32 u and y with the
coefficient k = 1 + 0.5 sin(4 pi x) cos(4 pi y) sin(4 pi z) read as
bfloat16.

One timed step = one application of the scaled operator (Sec. 6.1) on inputs
resident in HBM: the volume kernel on the caller's stream and the interface
kernel on a forked side stream, joined before the step's end event (two
launches per step).  L2 is flushed (512 MiB write) before every step, outside
the step's CUDA events.  value = unique unknowns / step time (GDoF/s).

Also measured on the headline workload: the FP32-k and FP64 applies, the
nodal-integration apply (scaled vs nodal, Sec. 7.5), GMG-CG to relative
residual 1e-8 in FP32 with FP64 refinement (BF16 and FP32 k) against plain
FP64, each solution's energy-norm error against the FP64 discrete solution,
the shift of the discrete solution when k is rounded to bfloat16, end-to-end
applies from pinned host buffers next to the measured pinned-copy bandwidth,
and the FP64 / FP32 multiply-add peaks that bound the ALU-limited kernels.
Extra keys: the 6-tet cube at level 8 (FP32 k), the multigrid tables, the
48 random tetrahedra (independent, levels 5..8), 48 tetrahedra sharing
faces (one level) and the learned smoother.  cpu_baseline: the FP64
oracle on every host core (one process per core) on a smaller level of the
same workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun) runs N independent replicas of the headline measurement
(the path does not shard across GPUs); `value` sums the replicas.
"""
from __future__ import annotations

import argparse
import hashlib
import itertools
import json
import math
import os
import re
import subprocess
import sys
import threading
import time
from collections import Counter

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

COARSEST = 2
C5_LEVEL = 9
METRIC = "scaled-stencil apply GDoF/s & %HBM peak; GMG-CG time to rel. residual 1e-8"
WORKLOAD = ("unit cube, 24 macro-tets (body centre + face centres), level 9 (513 nodes/macro edge, 5.43e8 stored "
            "nodes), FP32 u/f/r, BF16 k, k=1+0.5 sin(4 pi x)cos(4 pi y)sin(4 pi z)")
C2_LEVEL = 8
C2_WORKLOAD = "unit cube, 6 Kuhn macro-tets, level 8 (257 nodes/edge), k=exp(sin(pi x)cos(pi y)z), FP32"
CPU_LEVEL = 4  # the oracle's apply sample of the headline workload (14,911 unknowns)
CPU_SOLVE_LEVEL = 5  # its GMG-CG sample (125,055 unknowns)

# ncu DRAM traffic (read + write bytes) of one scaled apply, with the hash of
# the kernel sources it was measured on; the figure is dropped (null) as soon
# as those sources change.  Captured on the 24-tet cube at level 8 (68,693,016
# stored nodes; the level-9 workload is too large to capture, so it is scaled
# kernel by kernel: the volume kernel by stored nodes, the interface kernel by
# interface copies), one kernel per ncu call (profiles/apply_bf16k_cube24_l8_traffic.md).
NCU_TRAFFIC = {
    # the column march with two column sets per lane (vkernel 2), the kernel
    # the autotuner picks for this workload
    "bf16k_cube24": {"sha": "047c2eeababe5719", "vkernel": 2,
                     "volume_bytes_per_node": (556425472 + 262863616) / 68693016,
                     "interface_bytes_per_copy": (307681024 + 41054208) / (24 * (257 * 258 * 259 // 6 - 255 * 254 * 253 // 6)),
                     "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, 24-tet cube level 8, "
                               "march_kernel<float,bf16,APPLY,2> and boundary_only_kernel captured in separate ncu runs, "
                               "scaled to this workload per kernel unit"},
}


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
    for f in ("apply.cu", "march.cu", "hhg_internal.h"):
        h.update(_code_only(open(os.path.join(ROOT, "paper_1709_06793_gb300", "csrc", f)).read()).encode())
    return h.hexdigest()[:16]


def interface_copies(T, level):
    """Stored copies on macro faces, edges and vertices: every tet's nodes
    minus its interior nodes."""
    N = 1 << level
    return len(T) * ((N + 1) * (N + 2) * (N + 3) // 6 - (N - 1) * (N - 2) * (N - 3) // 6)


def _traffic(dtype_name, n_stored, n_copies, vkernel=None):
    """DRAM bytes of one apply from the recorded per-unit counters, or None
    when the kernels changed since (source hash) or another volume kernel
    runs."""
    rec = NCU_TRAFFIC.get(dtype_name)
    if not rec or rec["sha"] != _kernel_sha() or (vkernel is not None and vkernel != rec.get("vkernel", vkernel)):
        return None, None
    return rec["volume_bytes_per_node"] * n_stored + rec["interface_bytes_per_copy"] * n_copies, rec["source"]


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def unknowns_of(T, level):
    """Unique unknowns of a conforming macro mesh, every tet at `level`
    (N = 2^level intervals per macro edge): the interior nodes of each macro
    tet, of each face shared by two tets, and of each edge and vertex off the
    boundary (the boundary is the union of the faces of one tet only; its
    nodes are Dirichlet nodes)."""
    N = 1 << level
    T = np.asarray(T)
    faces = Counter(tuple(sorted(f)) for t in T for f in itertools.combinations(t, 3))
    bfaces = [f for f, c in faces.items() if c == 1]
    bedges = {e for f in bfaces for e in itertools.combinations(f, 2)}
    bverts = {v for f in bfaces for v in f}
    edges = {tuple(sorted(e)) for t in T for e in itertools.combinations(t, 2)}
    verts = set(int(v) for v in T.ravel())
    n = len(T) * (N - 1) * (N - 2) * (N - 3) // 6
    n += sum(1 for c in faces.values() if c > 1) * (N - 1) * (N - 2) // 2
    n += len(edges - bedges) * (N - 1)
    n += len(verts - {int(v) for v in bverts})
    return n


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


# ----------------------------------------------------------------------------
# The oracle on the host cores (cpu_baseline leg and the reference arm): one
# spawned process per core, each applying the FP64 element-loop operator of
# the headline workload at a smaller level; throughput adds up over the
# processes.
# ----------------------------------------------------------------------------

_ORACLE_STATE = None


def _oracle_init(level):
    global _ORACLE_STATE
    from oracle import hhg_oracle as O
    from paper_1709_06793_gb300 import inputs as I
    V, T = I.cube24()
    lm = O.LevelMesh(O.MacroMesh(V, T), level)
    k = I.k_large(lm.coords)
    u = np.where(lm.dirichlet, 0.0, I.u_wave(lm.coords))
    _ORACLE_STATE = (lm, k, u)


def _oracle_apply(_):
    lm, k, u = _ORACLE_STATE
    t0 = time.perf_counter()
    lm.apply(u, k, "scaled")
    return time.perf_counter() - t0


def host_info():
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    info = {"nproc": cores, "cpu_count": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            key, _, val = line.partition(":")
            if key.strip() in ("Architecture", "CPU(s)", "Model name", "Thread(s) per core", "Core(s) per socket",
                               "Socket(s)", "CPU max MHz"):
                info[key.strip()] = val.strip()
    except Exception:
        info["lscpu"] = "unavailable"
    return info


class OraclePool:
    """One spawned worker per host core (numpy single-threaded in each), every
    worker holding the oracle's level mesh, k and u of the sample."""

    def __init__(self, level, procs=None):
        import multiprocessing as mp
        self.procs = procs or host_info()["nproc"]
        self.level = level
        saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for v in saved:
            os.environ[v] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_oracle_init, initargs=(level,))
        finally:
            for v, old in saved.items():
                if old is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = old

    def step(self):
        """One concurrent apply in every worker; returns the wall time."""
        t0 = time.perf_counter()
        self.pool.map(_oracle_apply, range(self.procs), chunksize=1)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_solve_sample(level, repeats=3):
    """The oracle's FP64 GMG-CG (V(2,2), assembled level matrices) on the
    headline workload at a smaller level, rhs M 1, to 1e-8; one process."""
    from oracle import hhg_oracle as O
    from paper_1709_06793_gb300 import inputs as I
    V, T = I.cube24()
    h = O.Hierarchy(V, T, level, COARSEST, k_func=I.k_large)
    fm = h.mesh[level]
    f = (fm.assemble_mass() @ np.ones(fm.n))[fm.unknowns]
    ts = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        x, it, hist = h.pcg(f, tol=1e-8)
        ts.append(time.perf_counter() - t0)
    return {"level": level, "unknowns": len(fm.unknowns), "ms": 1e3 * float(np.median(ts)), "iterations": it,
            "rel_residual": hist[-1], "cores": 1,
            "sample": f"oracle GMG-CG V(2,2) (scipy sparse level matrices) on the headline mesh and k at level {level}, "
                      f"rhs M 1, median of {repeats}, one process"}


def cpu_baseline(steps=20):
    """The oracle's apply on all host cores (rate per unknown, GDoF/s) at
    level CPU_LEVEL and its GMG-CG on one core at CPU_SOLVE_LEVEL, both on
    the headline workload."""
    pool = OraclePool(CPU_LEVEL)
    try:
        pool.step()  # warm (imports, first touches)
        ts = [pool.step() for _ in range(steps)]
    finally:
        pool.close()
    dt = float(np.median(ts))
    from paper_1709_06793_gb300 import inputs as I
    _, T = I.cube24()
    dof = unknowns_of(T, CPU_LEVEL)
    return {"value": pool.procs * dof / dt / 1e9, "unit": "GDoF/s", "cores": pool.procs, "kind": "oracle",
            "sample": f"{pool.procs} concurrent oracle element-loop scaled applies (FP64, one spawned process per "
                      f"core, numpy single-threaded), headline mesh and k at level {CPU_LEVEL} ({dof} unknowns "
                      f"each), median wall of {steps} rounds; rate per unknown",
            "host": host_info(), "solve": oracle_solve_sample(CPU_SOLVE_LEVEL)}


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
    """The oracle as the reference arm: every step one concurrent apply per
    host core on the headline workload at level CPU_LEVEL (a level-9 FP64
    element loop would take hours); rank 0 only."""
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    from paper_1709_06793_gb300 import inputs as I
    _, T = I.cube24()
    dof = unknowns_of(T, CPU_LEVEL)
    pool = OraclePool(CPU_LEVEL)
    try:
        for _ in range(max(1, args.warmup)):
            pool.step()
        times = [pool.step() for _ in range(args.steps)]
    finally:
        pool.close()
    dt = float(np.mean(times))
    val = pool.procs * dof / dt / 1e9
    sample = (f"each step {pool.procs} concurrent oracle element-loop scaled applies (FP64, one spawned process per "
              f"core), headline mesh and k at level {CPU_LEVEL} ({dof} unknowns each); rate per unknown")
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GDoF/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD.replace("level 9 (513 nodes/macro edge, 5.43e8 stored nodes)",
                                                   f"level {CPU_LEVEL} (oracle sample)"),
                      "level": CPU_LEVEL, "unknowns_per_process": dof, "processes": pool.procs,
                      "macro_tets": 24, "parallelism": "host processes"},
           "cpu_baseline": {"value": val, "unit": "GDoF/s", "cores": pool.procs, "kind": "oracle", "sample": sample,
                            "host": host_info()},
           "e2e": {"value": val, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return out


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
    sol, _, _ = solve_runs(H, torch, m, n, f, (("fp64", H.HHG_SOLVE_FP64, H.HHG_SMOOTH_JACOBI),
                                                ("mixed", H.HHG_SOLVE_MIXED, H.HHG_SMOOTH_JACOBI),
                                                ("mixed_learned", H.HHG_SOLVE_MIXED, H.HHG_SMOOTH_LEARNED)))
    out.update(sol)
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
        m = m_big if (m_big is not None and level == C2_LEVEL) else H.Mesh(V, T, level, COARSEST)
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
    sol, _, _ = solve_runs(H, torch, m, n, f, (("solve_mixed", H.HHG_SOLVE_MIXED, H.HHG_SMOOTH_JACOBI),
                                                ("solve_fp64", H.HHG_SOLVE_FP64, H.HHG_SMOOTH_JACOBI)))
    out.update(sol)
    m.close()
    return out


CONFORMING_LEVEL = 7


def conforming_batch_bench(H, I, torch, flush, level=CONFORMING_LEVEL):
    """48 tetrahedra that share faces (the unit cube as 2 x 2 x 2 half cubes
    of 6 Kuhn tetrahedra each, inner vertices moved at random), all at one
    level, k = 1 + 0.9 tanh(Fourier field): the batched apply of all 48 tets
    with the interface rows of their 72 shared faces, and the mixed-precision
    GMG-CG solve."""
    V, T = I.cube48()
    m = H.Mesh(V, T, level, 2)
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
    unknowns = unknowns_of(T, level)
    peaks, src = _peaks()
    f = torch.tensor(np.sin(3 * xyz[:, 0]) * np.cos(2 * xyz[:, 1]) + xyz[:, 2], device="cuda") * mask.double()
    out = {"workload": f"48 tetrahedra sharing faces (2 x 2 x 2 half cubes x 6 Kuhn tets, inner vertices jittered, "
                       f"seed 3), level {level}, k = 1 + 0.9 tanh(Fourier field)",
           "level": level, "stored_nodes": n, "unknowns": unknowns,
           "interface_copies": interface_copies(T, level), "autotune": tune,
           "apply_ms": ms, "apply_gdofs": unknowns / (ms * 1e-3) / 1e9,
           "apply_hbm_frac": 12 * unknowns / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"]}
    sol, _, _ = solve_runs(H, torch, m, n, f, (("solve_mixed", H.HHG_SOLVE_MIXED, H.HHG_SMOOTH_JACOBI),
                                                ("solve_fp64", H.HHG_SOLVE_FP64, H.HHG_SMOOTH_JACOBI)))
    out.update(sol)
    m.close()
    return out


TENSOR_LEVELS = (3, 4, 5, 6, 7)  # the paper's L = 1 .. 5 on the 12-tet cube


def tensor_apply_timed(H, m, n, level, torch, flush, reps=10):
    """FP32 tensor apply (the mesh's tensor coefficient set) against its HBM
    roofline: algorithmic bytes u, the six k_m and y (32 B per node); the
    kernel streams the seven edge weights instead of the six k_m (36 B per
    node), so the fraction is a lower bound of the kernel's own."""
    x = torch.rand(n, device="cuda", dtype=torch.float32)
    y = torch.empty_like(x)
    for _ in range(3):
        H.hhg_apply_tensor(m.h, 0, x, y, H.HHG_F32)
    ts = []
    for i in range(reps):
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
    return {"level": level, "stored_nodes": n, "ms": ms,
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": ach / peaks["hbm_gbs"], "algorithmic_bytes_per_node": 32,
                         "kernel_bytes_per_node": 36, "peak_source": f"{src} hbm_gbs (burst)"}}


def tensor_apply_only(H, I, torch, flush, level=TENSOR_LEVELS[-1]):
    """Only the FP32 tensor apply of the tensor table's finest level (the
    12-tet cube, the paper's K): the case its kernels are profiled on."""
    V, T = I.cube12()
    m = H.Mesh(V, T, level, 1)
    off, lev, n = m.layout(0)
    xyz = m.coords(0)
    H.hhg_set_tensor_coefficient(m.h, torch.tensor(np.ascontiguousarray(I.K_tensor(xyz).T), device="cuda"))
    out = tensor_apply_timed(H, m, n, level, torch, flush)
    m.close()
    return out


def tensor_table(H, I, torch, flush, levels=TENSOR_LEVELS):
    """Shape of the paper's tensor test (Sec. 7.3, Tab. "divK4"): the 12-tet
    cube, its permeability tensor K, multigrid V(3,3) (FP64) until the
    residual drops by 1e-9; discrete L2 error of u* = sin(pi x) sin(pi y)
    sin(pi z), eoc, rho, time to solution.  Plus the FP32 tensor apply on the
    finest level against its HBM roofline: algorithmic bytes u, the six k_m
    and y (32 B per node); the kernel streams the seven edge weights instead
    of the six k_m (36 B per node), so the fraction is a lower bound."""
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
            apply = tensor_apply_timed(H, m, n, level, torch, flush)
        m.close()
    return {"workload": "unit cube, 12 macro-tets, K = the paper's tensor (Sec. 7.3), u* = sin(pi x) sin(pi y) "
                        "sin(pi z); V(3,3) (damped Jacobi) to a 1e-9 residual reduction, FP64",
            "rows": rows, "apply_fp32": apply,
            "apply_fp32_next_level": tensor_apply_only(H, I, torch, flush, levels[-1] + 1)}



def events_ms(torch, stream, flush, fn, reps, warm=3):
    """Mean CUDA-event time of fn on `stream` over reps calls, L2 flushed
    before each (outside the events)."""
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
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


def alu_peaks(H, torch, stream):
    """Multiply-add peaks of this GPU from the library's probe kernel (8
    independent chains per thread, 8 blocks of 256 threads per SM), best of
    5 launches: FP64 fma, FP32 fma and packed FP32x2 fma, TFLOP/s."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = 8 * sms
    out = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    res = {"sms": sms, "blocks": blocks}
    for kind, name, iters in ((0, "fp64_fma_tflops", 2000), (1, "fp32_fma_tflops", 100000),
                              (2, "fp32x2_fma_tflops", 50000)):
        H.hhg_alu_probe(kind, blocks, iters, out, stream)
        ts, flops = [], 0.0
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            flops = H.hhg_alu_probe(kind, blocks, iters, out, stream)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        res[name] = flops / (min(ts) * 1e-3) / 1e12
    assert bool(torch.isfinite(out).all())
    res["fp32_best_tflops"] = max(res["fp32_fma_tflops"], res["fp32x2_fma_tflops"])
    return res


def energy_norm_sq(H, m, e, y):
    """e^T A e over unique unknowns (FP64 scaled operator)."""
    H.hhg_apply_scaled(m.h, 0, e, y, H.HHG_F64)
    return H.hhg_dot(m.h, 0, e, y, H.HHG_F64)


def solve_runs(H, torch, m, n, f, runs, tol=1e-8, ref_tol=1e-11):
    """Time GMG-CG for each (name, mode, smoother) to rel. residual `tol`
    from u = 0 (the second of two calls: the first, two iterations long,
    builds the coarse inverse, eigenvalue estimates and CUDA graphs), and
    state each solution's energy-norm error ||x - x*||_A / ||x*||_A against
    the FP64 discrete solution x* (FP32 GMG-CG with FP64 refinement to rel.
    residual ref_tol, the residual formed in FP64 with the FP64 k)."""
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    xref = torch.zeros_like(y)
    st = H.hhg_solve(m.h, f, xref, tol=ref_tol, mode=H.HHG_SOLVE_MIXED, max_outer=60, raise_on_fail=False)
    nref = math.sqrt(max(energy_norm_sq(H, m, xref, y), 0.0))
    out = {"reference": {"rel_residual": st["rel_residual"], "status": st["status"],
                         "what": f"x*: FP64 discrete solution, rel. residual <= {ref_tol:g} (FP64 outer residual)"}}
    for name, mode, sm in runs:
        x = torch.zeros_like(y)
        H.hhg_solve(m.h, f, x, tol=tol, maxit=2, mode=mode, smoother=sm, raise_on_fail=False)
        x.zero_()
        torch.cuda.synchronize()
        r = H.hhg_solve(m.h, f, x, tol=tol, mode=mode, smoother=sm, raise_on_fail=False)
        x -= xref
        err = math.sqrt(max(energy_norm_sq(H, m, x, y), 0.0)) / nref
        out[name] = {"ms": r["time_ms"], "iterations": r["iterations"], "outer": r["outer"],
                     "rel_residual": r["rel_residual"], "status": r["status"], "smoother_used": r["smoother_used"],
                     "energy_error_vs_fp64_solution": err}
        del x
    return out, xref, nref


def c5_setup(H, I, torch, level):
    V, T = I.cube24()
    m = H.Mesh(V, T, level, COARSEST)
    off, lev, n = m.layout(0)
    X = m.coords(0)
    k = torch.empty(n, dtype=torch.float64, device="cuda")
    u = torch.empty(n, dtype=torch.float32, device="cuda")
    step = 1 << 25
    for a in range(0, n, step):
        b = min(n, a + step)
        x = torch.from_numpy(X[a:b]).cuda()
        k[a:b] = I.k_large(x)
        u[a:b] = I.u_wave(x).float()
    del X, x
    H.hhg_set_coefficient(m.h, k)
    # zero the Dirichlet entries: the residual of f = 1, u = 0 is 1 at
    # unknowns and 0 on Dirichlet nodes
    mask = torch.empty_like(u)
    H.hhg_residual(m.h, 0, torch.ones_like(u), torch.zeros_like(u), mask, H.HHG_F32)
    u *= mask
    del mask
    return m, T, n, k, u


def e2e_measure(H, torch, m, u, n, unknowns, world, steps):
    """End to end through the public API with host buffers: every step copies
    its u from pinned host memory, applies the operator and reads y back into
    pinned host memory.  Pipelined: two device buffer pairs, the copies on
    their own streams, so the host-to-device copy of step s+1, the apply of
    step s and the device-to-host copy of step s-1 overlap (the host link is
    full duplex); events order the reuse of each buffer.  Beside it the
    pinned-copy bandwidth of the same byte count, one direction at a time and
    both at once (the pipelined step's lower bound)."""
    stream = torch.cuda.current_stream()
    uh = torch.empty(n, dtype=torch.float32, pin_memory=True)
    uh.copy_(u)
    yh = [torch.empty(n, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    ub = [torch.empty_like(u) for _ in range(2)]
    yb = [torch.empty_like(u) for _ in range(2)]
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    dt = H.HHG_F32_KBF16

    def copy_ms(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    def both():
        s_in.wait_stream(stream)
        s_out.wait_stream(stream)
        with torch.cuda.stream(s_in):
            ub[0].copy_(uh, non_blocking=True)
        with torch.cuda.stream(s_out):
            yh[1].copy_(yb[1], non_blocking=True)
        stream.wait_stream(s_in)
        stream.wait_stream(s_out)

    nbytes = 4 * n
    h2d_ms = copy_ms(lambda: ub[0].copy_(uh, non_blocking=True))
    d2h_ms = copy_ms(lambda: yh[0].copy_(yb[0], non_blocking=True))
    bidir_ms = copy_ms(both)
    pinned = {"bytes": nbytes, "h2d_gbs": nbytes / (h2d_ms * 1e-3) / 1e9, "d2h_gbs": nbytes / (d2h_ms * 1e-3) / 1e9,
              "both_directions_ms": bidir_ms,
              "both_directions_gbs_each": nbytes / (bidir_ms * 1e-3) / 1e9,
              "how": "torch copy_ between pinned host and device buffers of one step's u / y (cudaMemcpyAsync), "
                     "median of 3 (CUDA events); both directions at once on two streams"}

    in_done = [torch.cuda.Event() for _ in range(2)]
    comp_done = [torch.cuda.Event() for _ in range(2)]
    out_done = [torch.cuda.Event() for _ in range(2)]
    for e in in_done + comp_done + out_done:
        e.record(stream)

    def seq_step(q):
        ub[0].copy_(uh, non_blocking=True)
        H.hhg_apply_scaled(m.h, 0, ub[0], yb[0], dt, stream)
        yh[0].copy_(yb[0], non_blocking=True)

    def pipe_step(q):
        b = q & 1
        s_in.wait_event(comp_done[b])  # the apply of step q-2 has read ub[b]
        with torch.cuda.stream(s_in):
            ub[b].copy_(uh, non_blocking=True)
        in_done[b].record(s_in)
        stream.wait_event(in_done[b])
        stream.wait_event(out_done[b])  # y of step q-2 has left yb[b]
        H.hhg_apply_scaled(m.h, 0, ub[b], yb[b], dt, stream)
        comp_done[b].record(stream)
        s_out.wait_event(comp_done[b])
        with torch.cuda.stream(s_out):
            yh[b].copy_(yb[b], non_blocking=True)
        out_done[b].record(s_out)

    def timed(step_fn, ke):
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

    ke = max(5, min(steps, 20))
    seq_ms = timed(seq_step, ke)
    e2e_ms = timed(pipe_step, ke)
    ok = bool(torch.equal(yh[(ke - 1) & 1], yb[(ke - 1) & 1].cpu()))
    return {"value": job_rate(unknowns, e2e_ms, world), "unit": "GDoF/s",
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "ms_per_step": e2e_ms, "steps": ke,
            "pipelined": "two buffer pairs; H2D, apply and D2H of neighbouring steps on separate streams",
            "sequential_value": job_rate(unknowns, seq_ms, world), "sequential_ms_per_step": seq_ms,
            "pinned_copy": pinned,
            "bound_by_copies_value": job_rate(unknowns, bidir_ms, world),
            "frac_of_copy_bound": bidir_ms / e2e_ms, "result_read_back_intact": ok}


def c2_section(H, I, torch, stream, flush, steps):
    """The 6-tet cube at level 8, FP32 k (the medium configuration): the FP32
    scaled apply, nodal and Vol+Face applies, and the GMG-CG solves of the
    manufactured problem with their errors against the FP64 solution."""
    V, T = I.kuhn_cube()
    m = H.Mesh(V, T, C2_LEVEL, COARSEST)
    off, lev, n = m.layout(0)
    xyz = m.coords(0)
    unknowns = unknowns_of(T, C2_LEVEL)
    H.hhg_set_coefficient(m.h, torch.tensor(I.k_cube(xyz), device="cuda"))
    u = torch.tensor(np.random.default_rng(0).uniform(-1, 1, n), device="cuda", dtype=torch.float32)
    dg = torch.empty_like(u)
    H.hhg_residual(m.h, 0, torch.ones_like(u), torch.zeros_like(u), dg, H.HHG_F32)
    u *= dg
    y = torch.empty_like(u)
    tune = H.hhg_autotune(m.h, H.HHG_F32)
    ms = events_ms(torch, stream, flush, lambda: H.hhg_apply_scaled(m.h, 0, u, y, H.HHG_F32, stream), steps)
    nodal_ms = events_ms(torch, stream, flush, lambda: H.hhg_apply_nodal(m.h, 0, u, y, H.HHG_F32, stream), 10)
    volface_ms = events_ms(torch, stream, flush, lambda: H.hhg_apply_volface(m.h, 0, u, y, H.HHG_F32, stream), 10)
    peaks, src = _peaks()
    algo = 12 * unknowns
    traffic, tsrc = _traffic("f32_kuhn_cube", n, interface_copies(T, C2_LEVEL))
    out = {"workload": C2_WORKLOAD, "unknowns": unknowns, "stored_nodes": n, "autotune": tune,
           "apply_ms": ms, "apply_gdofs": unknowns / (ms * 1e-3) / 1e9,
           "roofline": {"bound": "hbm", "achieved": algo / (ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                        "unit": "GB/s", "frac": algo / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"], "traffic": traffic,
                        "traffic_source": tsrc, "algorithmic_bytes_per_launch": algo,
                        "peak_source": f"{src} hbm_gbs (burst)"},
           "nodal_ms": nodal_ms, "volface_ms": volface_ms, "nodal_over_scaled": nodal_ms / ms,
           "volface_over_scaled": volface_ms / ms}
    del u, y, dg
    # rhs f_h = M I_h f (consistent mass matrix), f = -div(k grad u*) for the
    # manufactured u* = sin(pi x) sin(pi y) sin(pi z)
    fi = torch.tensor(I.f_cube_sine(xyz), device="cuda")
    f = torch.empty_like(fi)
    H.hhg_apply_mass(m.h, 0, fi, f, H.HHG_F64)
    runs = (("mixed_fp32_fp64refine", H.HHG_SOLVE_MIXED, H.HHG_SMOOTH_JACOBI),
            ("mixed_bf16k_fp64refine", H.HHG_SOLVE_MIXED_KBF16, H.HHG_SMOOTH_JACOBI),
            ("mixed_bf16k_inner_fp64refine", H.HHG_SOLVE_MIXED_KBF16_INNER, H.HHG_SMOOTH_JACOBI),
            ("fp64", H.HHG_SOLVE_FP64, H.HHG_SMOOTH_JACOBI),
            ("mixed_fp32_fp64refine_cheb", H.HHG_SOLVE_MIXED, H.HHG_SMOOTH_CHEBYSHEV),
            ("fp64_cheb", H.HHG_SOLVE_FP64, H.HHG_SMOOTH_CHEBYSHEV))
    solve, _, _ = solve_runs(H, torch, m, n, f, runs)
    solve["metric"] = ("GMG-preconditioned CG, V(2,2), wall time to ||f - A u||/||f|| <= 1e-8 from u = 0, "
                       "rhs M I_h f; FP64 outer residual in every mode")
    solve["speedup_mixed_vs_fp64"] = solve["fp64"]["ms"] / solve["mixed_fp32_fp64refine"]["ms"]
    out["solve"] = solve
    return out, m


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--level", type=int, default=C5_LEVEL, help="level of the headline workload (9 = the contract)")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline only: skip the 6-tet cube, tables, batch and learned sections")
    ap.add_argument("--no-tune", action="store_true", help="skip the work-list autotuner (default segmentation)")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-table", action="store_true", help="skip the multigrid tables (scalar and tensor)")
    ap.add_argument("--only-learned", action="store_true",
                    help="run only the learned-smoother section (C4) and print its JSON")
    ap.add_argument("--only-tensor", action="store_true",
                    help="run only the FP32 tensor apply of the tensor table's finest level and print its JSON")
    ap.add_argument("--vkernel", type=int, choices=[0, 1, 2], default=None,
                    help="fix the volume kernel of the scaled apply instead of autotuning it (profiling)")
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

    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, device="cuda", dtype=torch.float32)
    if args.only_learned:
        out = learned_bench(H, I, torch, stream, flush)
        if rank == 0:
            print(json.dumps({"learned": out}))
        return
    if args.only_tensor:
        out = tensor_apply_only(H, I, torch, flush)
        if rank == 0:
            print(json.dumps({"tensor_apply_fp32": out}))
        return

    t_setup = time.perf_counter()
    m, T, n, k, u = c5_setup(H, I, torch, args.level)
    unknowns = unknowns_of(T, args.level)
    setup_s = time.perf_counter() - t_setup
    y = torch.empty_like(u)
    DT = H.HHG_F32_KBF16
    fixed = args.no_tune or args.vkernel is not None
    if args.vkernel is not None:
        H.hhg_set_option(m.h, "vkernel", args.vkernel)
    tune = None if fixed else H.hhg_autotune(m.h, DT)
    for _ in range(max(3, args.warmup)):
        H.hhg_apply_scaled(m.h, 0, u, y, DT, stream)
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
            H.hhg_apply_scaled(m.h, 0, u, y, DT, stream)
            ends[s].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    ms = replica_time(float(np.mean(step_ms)), world)

    peaks, src = _peaks()
    algo_bytes = 10 * unknowns  # read u (FP32), k (BF16); write y (FP32): every unknown once
    achieved = algo_bytes / (ms * 1e-3) / 1e9
    traffic, tsrc = _traffic("bf16k_cube24", n, interface_copies(T, args.level), int(H.hhg_get_option(m.h, "vkernel")))
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "traffic_source": tsrc,
            "peak_source": f"{src} hbm_gbs (burst)",
            "kernel": "volume kernel chosen by the autotuner (march_kernel<float,__nv_bfloat16,APPLY,P>, the column "
                      "march with P = 1 or 2 column sets per lane, or scaled_op_kernel, the tile march) + "
                      "boundary_only_kernel (interface rows, on a forked stream); achieved = algorithmic bytes / "
                      "CUDA-event time of the pair on the caller's stream",
            "algorithmic_bytes_per_launch": algo_bytes, "algorithmic_bytes_per_unknown": 10,
            "stored_node_bytes_fraction": 10 * n / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"]}

    out = {"metric": METRIC, "value": job_rate(unknowns, ms, world), "unit": "GDoF/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD if args.level == C5_LEVEL else
                      WORKLOAD.replace("level 9 (513 nodes/macro edge, 5.43e8 stored nodes)", f"level {args.level}"),
                      "level": args.level, "macro_tets": 24, "unknowns": unknowns, "stored_nodes": n,
                      "k_storage": "bf16", "vectors": "f32",
                      "parallelism": f"replicas{world}" if world > 1 else "single",
                      "l2": "flushed before every step (512 MiB write, outside the step events)"},
           "roofline": roof, "cpu_baseline": None, "e2e": None, "gpu_launches": 2 * args.steps,
           "autotune": tune, "clocks": clk.summary(), "wall_s_timed_region": wall, "setup_s": setup_s,
           "stored_nodes_per_s": n * world / (ms * 1e-3)}

    # the other operators on the same workload: FP32 k, the nodal-integration
    # apply (the paper's cost comparison), FP64 against the FP64-ALU peak
    tune32 = None if fixed else H.hhg_autotune(m.h, H.HHG_F32)
    f32_ms = events_ms(torch, stream, flush, lambda: H.hhg_apply_scaled(m.h, 0, u, y, H.HHG_F32, stream), 10)
    if tune is not None:
        H.hhg_set_option(m.h, "vkernel", tune["vkernel"])
        H.hhg_set_option(m.h, "kseg", tune["kseg"])
        H.hhg_set_option(m.h, "korder", tune["korder"])
    nodal_ms = events_ms(torch, stream, flush, lambda: H.hhg_apply_nodal(m.h, 0, u, y, DT, stream), 10)
    alu = alu_peaks(H, torch, stream)
    nodal_tf = 211 * unknowns / (nodal_ms * 1e-3) / 1e12
    ops = {"scaled_bf16k_ms": ms, "scaled_f32_ms": f32_ms, "autotune_f32": tune32,
           "scaled_f32_roofline": {"bound": "hbm", "achieved": 12 * unknowns / (f32_ms * 1e-3) / 1e9,
                                   "frac": 12 * unknowns / (f32_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                                   "algorithmic_bytes_per_unknown": 12},
           "nodal_bf16k_ms": nodal_ms, "nodal_over_scaled": nodal_ms / ms,
           "nodal_roofline": {"bound": "alu", "achieved": nodal_tf, "peak": alu["fp32_best_tflops"],
                              "unit": "TFLOP/s", "frac": nodal_tf / alu["fp32_best_tflops"],
                              "algorithmic_flops_per_unknown": 211,
                              "peak_source": "measured: the library's multiply-add probe, the faster of FP32 fma "
                                             "and packed FP32x2 fma",
                              "hbm_frac": algo_bytes / (nodal_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]}}
    out["alu_peaks"] = alu
    del y
    torch.cuda.empty_cache()

    if not args.no_solve and world == 1:
        ones = torch.ones(n, dtype=torch.float64, device="cuda")
        f = torch.empty_like(ones)
        H.hhg_apply_mass(m.h, 0, ones, f, H.HHG_F64)
        del ones
        # BF16 k throughout (the problem of the rounded k), BF16 k in the
        # inner solve only (the FP64-k problem), FP32 k, plain FP64
        runs = (("mixed_bf16k_fp64refine", H.HHG_SOLVE_MIXED_KBF16, H.HHG_SMOOTH_JACOBI),
                ("mixed_bf16k_inner_fp64refine", H.HHG_SOLVE_MIXED_KBF16_INNER, H.HHG_SMOOTH_JACOBI),
                ("mixed_fp32_fp64refine", H.HHG_SOLVE_MIXED, H.HHG_SMOOTH_JACOBI),
                ("fp64", H.HHG_SOLVE_FP64, H.HHG_SMOOTH_JACOBI))
        solve, xref, nref = solve_runs(H, torch, m, n, f, runs)
        solve["metric"] = ("GMG-preconditioned CG, V(2,2) damped Jacobi, wall time to ||f - A u||/||f|| <= 1e-8 "
                           "from u = 0, rhs M 1; FP64 outer residual in every mode")
        solve["speedup_mixed_bf16k_vs_fp64"] = solve["fp64"]["ms"] / solve["mixed_bf16k_fp64refine"]["ms"]
        solve["speedup_mixed_bf16k_inner_vs_fp64"] = solve["fp64"]["ms"] / solve["mixed_bf16k_inner_fp64refine"]["ms"]
        solve["speedup_mixed_fp32_vs_fp64"] = solve["fp64"]["ms"] / solve["mixed_fp32_fp64refine"]["ms"]
        # FP64 apply against the FP64-ALU peak (69 flops per unknown, Sec. 6.1's count)
        y64 = torch.empty_like(xref)
        f64_ms = events_ms(torch, stream, flush, lambda: H.hhg_apply_scaled(m.h, 0, xref, y64, H.HHG_F64, stream), 5)
        f64_tf = 69 * unknowns / (f64_ms * 1e-3) / 1e12
        ops["scaled_fp64_ms"] = f64_ms
        ops["scaled_fp64_roofline"] = {"bound": "alu", "achieved": f64_tf, "peak": alu["fp64_fma_tflops"],
                                       "unit": "TFLOP/s", "frac": f64_tf / alu["fp64_fma_tflops"],
                                       "algorithmic_flops_per_unknown": 69,
                                       "peak_source": "measured: the library's FP64 multiply-add probe",
                                       "hbm_frac": 24 * unknowns / (f64_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]}
        # how far the discrete solution moves when k is rounded to bfloat16
        # (the problem every BF16-k apply works on): ||x(k_bf16) - x*||_A / ||x*||_A
        H.hhg_set_coefficient(m.h, k.to(torch.bfloat16).to(torch.float64))
        xq = torch.zeros_like(xref)
        stq = H.hhg_solve(m.h, f, xq, tol=1e-11, mode=H.HHG_SOLVE_MIXED, max_outer=60, raise_on_fail=False)
        H.hhg_set_coefficient(m.h, k)
        xq -= xref
        solve["bf16_k_solution_shift"] = {
            "energy_rel": math.sqrt(max(energy_norm_sq(H, m, xq, y64), 0.0)) / nref,
            "max_abs_rel": float(xq.abs().max() / xref.abs().max()), "rel_residual_of_x_bf16": stq["rel_residual"],
            "what": "x(k_bf16): the discrete solution with k rounded to bfloat16 (RN), rel. residual <= 1e-11; "
                    "energy norm of the FP64-k operator"}
        out["solve"] = solve
        del xq, xref, y64, f
    out["operators"] = ops
    torch.cuda.empty_cache()

    if not args.no_e2e:
        out["e2e"] = e2e_measure(H, torch, m, u, n, unknowns, world, args.steps)
    m.close()
    del u, k
    torch.cuda.empty_cache()

    if world == 1 and not args.no_extras:
        c2, m2 = c2_section(H, I, torch, stream, flush, 50)
        out["c2"] = c2
        if not args.no_table:
            out["mg_table"] = paper_table(H, I, torch, m_big=m2)
            out["tensor_table"] = tensor_table(H, I, torch, flush)
        m2.close()
        if not args.no_solve:
            out["batch"] = batch_bench(H, I, torch, flush)
            out["batch_conforming"] = conforming_batch_bench(H, I, torch, flush)
        if not args.no_learned:
            out["learned"] = learned_bench(H, I, torch, stream, flush)

    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
