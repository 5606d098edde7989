#!/usr/bin/env python
"""Benchmark of the coupled Yee-FDTD + kinetic step on GB300.

One "step" is one full time step of the hot path (H stencil, kinetic delta-f
update + J moment + Ampere source term, E stencil with CPML and the soft
source) over the whole workload.  Default workload: 2-D TMz 4096 x 4096,
dx = lam0/20, 10-cell CPML, seeded Gaussian-density plasma cylinder of radius
512 cells (823 k plasma cells), 32 x 32 Cartesian velocity grid per cell
(1024 nodes, FP32 delta f = 3.4 GB), i.e. 8.4e8 phase-space nodes per step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

Prints one JSON line (rank 0).  N > 1 runs N independent replicas, one per
rank (weak scaling; no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcell-updates/s + phase-space updates/s at 1 GB300, % HBM roofline; closure vs kinetic"
UNIT = "Gcell-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="2d_tmz_4096_kinetic")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--engine", default="tcgen05", choices=["mma", "tcgen05"], help="closure MLP engine")
    ap.add_argument("--fused", type=int, default=0, choices=[0, 1],
                    help="2-D / 3-D FP32: fuse each E update with the next H update (default 0: separate passes)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the autotuner (the launch shapes come from the tuning cache, else the defaults)")
    ap.add_argument("--kin-shape", default="",
                    help="VPL,L[,BPS[,STAGES]]: force the kinetic kernel's launch shape after autotuning (profiling)")
    ap.add_argument("--decompose", action="store_true",
                    help="N > 1: split the grid along its slowest axis, one slab per rank, halos over NCCL "
                         "(strong scaling); N = 1 is the whole-grid path")
    ap.add_argument("--subdomains", type=int, default=0,
                    help="K > 1: run the grid as K slabs on this one GPU with halo copies (decomposition overhead)")
    ap.add_argument("--no-configs", action="store_true",
                    help="default workload at N = 1: skip the other configurations' entries (configs)")
    return ap.parse_args()


def cells_of(spec) -> int:
    g = spec["grid"]
    return int(g["nz"]) if g["ndim"] == 1 else int(g["nx"]) * int(g["ny"]) * (int(g["nz"]) if g["ndim"] == 3 else 1)


def make_spec(name: str):
    from fdtd_inputs import WORKLOADS
    return WORKLOADS[name]()


def reduce_max(x: float, world: int, device=None) -> float:
    """The largest x over the ranks of the job (x itself for a one-rank job):
    the job's time is its slowest rank's."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def step_launches(steps, mid_per_step, fused):
    """Kernels the solver launches for `steps` steps: 32-step graph replays,
    then one 16-, 8-, 4-, 2- and 1-step graph for each set bit of the
    remainder.  An n-step sequence runs H_0, per step the middle kernels and
    E, H for all but the last step, and one step-counter advance; each fused
    transition (an even number of the n - 1) makes E_k + H_{k+1} one launch."""
    def seq(n):
        f = (n - 1) - (n - 1) % 2 if fused else 0
        return mid_per_step * n + 2 * n - f + 1
    chunks, rem = divmod(steps, 32)
    return chunks * seq(32) + sum(seq(1 << b) for b in range(5) if rem >> b & 1)


def fused_in_steps(spec: dict, shapes: dict, option: int = 0) -> bool:
    """Whether the timed steps run the fused E + H pass: asked for by option
    (2-D / 3-D FP32), or chosen by the autotuner (2-D FP32, fused_rows > 0)."""
    f32 = spec["grid"].get("precision", "f32") == "f32"
    return (bool(option) and spec["grid"]["ndim"] >= 2 and f32) or shapes.get("fused_rows", 0) > 0


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: every rank processes units_per_rank in the job's time."""
    return world * units_per_rank / seconds


def sample_spec(name: str):
    """The bounded CPU sample of a workload: the same recipe with every length
    scaled down (same plasma fraction, velocity grid and precision choice)."""
    from fdtd_inputs import spec_1d_slab, spec_2d_cylinder, spec_3d_slab
    if name.startswith("2d_tmz_4096"):
        return spec_2d_cylinder(n=512, R=64), "2-D TMz 512x512, cylinder R=64 (all lengths / 8), 32x32 nodes"
    if name.startswith("3d_512"):
        return (spec_3d_slab(n=64, cpml=8, slab=(24, 40), src_k=12),
                "3-D 64^3, slab z in [24,40) (all lengths / 8), Nv=32")
    if name.startswith("3d_256"):
        spec = spec_3d_slab(n=32, cpml=4, slab=(12, 20), src_k=6, f_dtype="f32")
        if "f0evolve" in name:
            spec["plasma"].update(vgrid="speed3d", evolve_f0=1, mass_ratio=1.37e-5, tg_ev=0.026)
        return spec, "3-D 32^3, slab z in [12,20) (all lengths / 8), Nv=32"
    if name.startswith("batch1d"):
        from fdtd_inputs import batch_runs_1d
        return batch_runs_1d(nruns=8, seed=20221114), "8 of the 256 batched 1-D runs (same generator, seed)"
    return spec_1d_slab(), "1-D Nz=2000 slab (the full workload)"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          f"--id={self.gpu_id}", "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_uuid(dev) -> str:
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev)


# ------------------------------------------------------------- roofline data
def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def kinetic_src_sha(kernel: str = "k_kinetic") -> str:
    """Hash of the sources a kinetic kernel is built from (its ncu figures stay valid while it matches)."""
    files = {"k_kinetic_f0": ("kinetic.cu", "kinetic_row.cuh"),
             "k_kinetic_ring": ("kinetic_ring.cu", "kinetic_row.cuh", "async.cuh")}.get(
        kernel, ("kinetic_impl.cuh", "kinetic_row.cuh"))
    h = hashlib.sha1()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2211_05647_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


def ncu_traffic(kernel: str, workload: str, shape=None):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source and the same launch shape (vpl, l, ring stages)
    (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    sha = kinetic_src_sha(kernel)
    for ln in open(path):
        if ln.startswith("#") or not ln.strip():
            continue
        kv = dict(t.split("=", 1) for t in ln.split() if "=" in t)
        if kv.get("kernel") == kernel and kv.get("workload") == workload and kv.get("src_sha") == sha:
            got = (int(kv.get("vpl", 0)), int(kv.get("l", 0)), int(kv.get("stages", 0)))
            if shape is not None and got != tuple(shape):
                continue
            return float(kv["dram_bytes_per_launch"])
    return None


def batch_traffic(workload: str, steps_per_launch: int):
    """DRAM bytes per launch of the batched kernel from the committed ncu summary (bytes per step, taken
    on the current batch1d.cu / kinetic_row.cuh / async.cuh) times the steps a launch covers, else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    h = hashlib.sha1()
    for f in ("batch1d.cu", "kinetic_row.cuh", "async.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2211_05647_gb300", "csrc", f), "rb").read())
    sha = h.hexdigest()[:12]
    for ln in open(path):
        if ln.startswith("#") or not ln.strip():
            continue
        kv = dict(t.split("=", 1) for t in ln.split() if "=" in t)
        if kv.get("kernel") == "k_batch1d" and kv.get("workload") == workload and kv.get("src_sha") == sha:
            return float(kv["dram_bytes_per_step"]) * steps_per_launch
    return None


def kinetic_kernel(shapes: dict, evolve: bool):
    """The kinetic kernel a handle launches and its launch shape (vpl, l, ring stages)."""
    if evolve:
        return "k_kinetic_f0", None
    shape = (shapes["kin_vpl"], shapes["kin_l"], shapes.get("kin_stages", 0)) if shapes["kin_vpl"] else (8, 32, 0)
    return ("k_kinetic_ring" if shape[2] > 0 else "k_kinetic"), shape


# ---------------------------------------------------------------- oracle arm
def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_throughput(name: str, steps: int, warmup: int, budget_s: float | None, omp: bool = False):
    """Time the FP64 oracle on a bounded sample of the workload (omp: the
    all-core build of the same source).  Returns (Gcell-updates/s, phase-space
    updates/s, steps timed, sample text, cells, nodes)."""
    from oracle import oracle as O
    from tests.adapters import oracle_sim
    spec, text = sample_spec(name)
    specs = spec if isinstance(spec, list) else [spec]
    sims = [oracle_sim(O, sp, omp=omp) for sp in specs]
    for sim in sims:
        sim.step(warmup)
    n = 0
    t0 = time.perf_counter()
    while n < steps:
        for sim in sims:
            sim.step(1)
        n += 1
        if budget_s is not None and time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    cells = sum(cells_of(sp) for sp in specs)
    nodes = sum(sim.nslots * sim.nnode for sim in sims)
    return cells * n / dt / 1e9, nodes * n / dt, n, text, cells, nodes


# ------------------------------------------------- the other configurations
def _peak(key="hbm_gbs", fallback=6800.0):
    peaks = measured_peaks()
    return (peaks[key], f"MEASURED_PEAKS.json {key}") if peaks else (fallback, "fallback")


def _release():
    import torch
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def solver_config(workload: str, steps: int, warmup: int, autotune: bool, local: int) -> dict:
    """One single-grid workload: autotune (untimed), W warm-up steps, K steps
    timed with CUDA events on the solver stream, per-kernel launch times, the
    kinetic kernel's roofline and the step's algorithmic HBM fraction."""
    import torch
    from paper_2211_05647_gb300 import Solver
    spec = make_spec(workload)
    s = Solver.from_spec(spec, device=local)
    ns, nn = s.plasma_shape()
    cells = cells_of(spec)
    if autotune:
        s.autotune()
    shapes = s.launch_shapes()
    s.step(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    s.step(steps)
    e1.record(s.stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    kt = s.time_kernels(min(steps, 50))
    s.close()
    del s
    _release()
    fbytes = {"f32": 4, "bf16": 2, "f64": 8}[spec["plasma"]["f_dtype"]]
    evolve = bool(spec["plasma"].get("evolve_f0"))
    alg = 2 * fbytes * ns * nn * (2 if evolve else 1)
    peak, src = _peak()
    kname, kshape = kinetic_kernel(shapes, evolve)
    fb = 8 if spec["grid"].get("precision", "f32") == "f64" else 4
    ncomp = {1: 2, 2: 3, 3: 6}[spec["grid"]["ndim"]]
    step_alg = 2 * fb * ncomp * cells + alg
    ms_step = ms / steps
    achieved = alg / (kt["kinetic"] / 1e3) / 1e9
    return {"workload": workload, "steps": steps, "warmup": warmup, "ms_per_step": ms_step,
            "gcell_updates_per_s": cells * steps / (ms / 1e3) / 1e9,
            "phase_space_updates_per_s": ns * nn * steps / (ms / 1e3),
            "cells": cells, "plasma_cells": ns, "nodes_per_cell": nn, "f_dtype": spec["plasma"]["f_dtype"],
            "precision": spec["grid"].get("precision", "f32"), "kernel_ms": kt, "launch_shapes": shapes,
            # a 1-D grid (0.3 MB a step) stays in L2: its steps are bound by launch and L2 latency, not HBM
            "roofline": {"bound": "latency" if spec["grid"]["ndim"] == 1 else "hbm", "kernel": kname,
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "alg_bytes_per_launch": alg, "launch_ms": kt["kinetic"],
                         "traffic": ncu_traffic(kname, workload, kshape),
                         "peak_source": src},
            "step_hbm_frac_algorithmic": step_alg / (ms_step / 1e3) / 1e9 / peak,
            "gpu_launches": step_launches(steps, 1 if ns else 0, fused_in_steps(spec, shapes))}


def batch_config(workload: str, specs, steps: int, warmup: int, autotune: bool, local: int) -> dict:
    """Batched independent 1-D runs: one persistent launch per chunk of up to
    100 steps (graph replay); per-launch times with events between chunks."""
    import torch
    from paper_2211_05647_gb300 import Batch
    b = Batch(specs, device=local)
    tune = b.autotune() if autotune else None
    info = b.info()
    cells, nodes = info["cells"], info["nodes"]
    st = b.stream
    chunk = min(100, steps)
    rem = steps % chunk
    b.step(max(warmup, 1))
    b.step(chunk)                 # captures the chunk graph outside the timed region
    if rem:
        b.step(rem)
    torch.cuda.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps // chunk + 2)]
    evs[0].record(st)
    for i in range(steps // chunk):
        b.step(chunk)
        evs[i + 1].record(st)
    if rem:
        b.step(rem)
    e_end = torch.cuda.Event(enable_timing=True)
    e_end.record(st)
    torch.cuda.synchronize()
    ms = evs[0].elapsed_time(e_end)
    launch_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(steps // chunk)]
    b.close()
    del b
    _release()
    fdt = specs[0]["plasma"]["f_dtype"]
    fb = {"f32": 4, "bf16": 2, "f64": 8}[fdt]
    eb = 8 if specs[0]["grid"]["precision"] == "f64" else 4
    alg_step = 2 * eb * (2 * cells + len(specs)) + 2 * fb * nodes
    per_launch_ms = statistics.median(launch_ms) if launch_ms else ms
    achieved = alg_step * chunk / (per_launch_ms / 1e3) / 1e9
    peak, src = _peak()
    return {"workload": workload, "steps": steps, "warmup": warmup, "ms_per_step": ms / steps,
            "gcell_updates_per_s": cells * steps / (ms / 1e3) / 1e9,
            "phase_space_updates_per_s": nodes * steps / (ms / 1e3),
            "runs": len(specs), "cells": cells, "phase_space_nodes": nodes, "f_dtype": fdt,
            "clusters": info["clusters"], "ctas_per_cluster": info["cluster_ctas"], "steps_per_launch": chunk,
            "row_shape": tune,
            "roofline": {"bound": "hbm", "kernel": "k_batch1d", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": batch_traffic(workload, chunk),
                         "alg_bytes_per_launch": alg_step * chunk,
                         "launch_ms": per_launch_ms, "peak_source": src},
            "step_hbm_frac_algorithmic": alg_step / (ms / steps / 1e3) / 1e9 / peak,
            "gpu_launches": 2 * (steps // chunk + (1 if rem else 0))}


def closure_config(steps: int, warmup: int, engine: str, autotune: bool, local: int) -> dict:
    """Learned closure vs the kinetic solve on the same 8192^2 grid: the
    trained weights are the committed ones (paper_2211_05647_gb300/data,
    written by train_closure.py with the library's own training kernels).
    Each run does W warm-up steps, K steps timed with events, then the rest of
    the workload's 4000 steps untimed; the closure's fields after 4000 steps
    are compared with the kinetic run's (relative L2 per component)."""
    import numpy as np
    import torch
    from paper_2211_05647_gb300 import Solver
    from paper_2211_05647_gb300.train_closure import load
    w = load()
    spec = make_spec("2d_tmz_8192_closure")
    total = int(spec["steps"])
    cells = cells_of(spec)

    def run(with_closure):
        s = Solver.from_spec(spec, device=local)
        if with_closure:
            s.set_closure(w["params"], e_scale=w["e_scale"], j_scale=w["j_scale"], n_scale=w["n_scale"],
                          rho=w["rho"], beta=w["beta"], n_train_max=w["n_train_max"], engine=engine)
        if autotune:
            s.autotune()
        shape = s.closure_shape() if with_closure else s.plasma_shape()
        s.step(warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.step(steps)
        e1.record(s.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        s.step(max(total - warmup - steps, 0))
        fields = {f: s.read(f, device=False).astype(np.float64) for f in ("ez", "hx", "hy")}
        kt = s.time_kernels(20)
        shapes = s.launch_shapes()
        s.close()
        del s
        _release()
        return ms, fields, kt, shape, shapes

    def run_bf16_kinetic():
        # the kinetic solve with BF16-stored delta f (stochastic rounding), timed over the same K steps
        import copy
        sp = copy.deepcopy(spec)
        sp["plasma"]["f_dtype"] = "bf16"
        s = Solver.from_spec(sp, device=local)
        if autotune:
            s.autotune()
        s.step(warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.step(steps)
        e1.record(s.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        s.close()
        del s
        _release()
        return ms

    ms_c, f_c, kt_c, (n_kin, n_cl), sh_c = run(True)
    ms_k, f_k, kt_k, (ns_k, nn_k), sh_k = run(False)
    ms_kb = run_bf16_kinetic()
    err = {f: float(np.linalg.norm(f_c[f] - f_k[f]) / np.linalg.norm(f_k[f])) for f in f_c}
    flops = 2 * (17 * 128 + 128 * 128 + 128) * n_cl
    tpk, tsrc = _peak("bf16_tflops_sustained", 1700.0)
    hpk, _ = _peak()
    achieved = flops / (kt_c["closure"] / 1e3) / 1e12 if kt_c["closure"] > 0 else 0.0
    # closure step bytes: fields (24 B a cell) + per closure cell history ring (64 B read, 4 B write),
    # density, J state and E gather / scatter (16 B) + the kinetic fallback rows (8 B a node)
    ms_step_c = ms_c / steps
    step_alg = 24 * cells + 84 * n_cl + 8 * n_kin * nn_k
    return {"workload": "2d_tmz_8192_closure", "steps": steps, "warmup": warmup, "run_steps": total,
            "ms_per_step": ms_step_c, "gcell_updates_per_s": cells * steps / (ms_c / 1e3) / 1e9,
            "closure_engine": engine, "closure_cells": n_cl, "kinetic_fallback_cells": n_kin,
            "weights": {k: w["record"][k] for k in ("runs", "samples", "epochs", "batch") if k in w["record"]},
            "closure_vs_kinetic": {"kinetic_ms_per_step": ms_k / steps, "closure_ms_per_step": ms_step_c,
                                   "speedup": ms_k / ms_c, "field_rel_l2_after_run": err,
                                   "kinetic_gcell_updates_per_s": cells * steps / (ms_k / 1e3) / 1e9,
                                   "kinetic_phase_space_updates_per_s": ns_k * nn_k * steps / (ms_k / 1e3),
                                   # against the faster kinetic form, BF16-stored delta f
                                   "kinetic_bf16_ms_per_step": ms_kb / steps, "speedup_vs_bf16_kinetic": ms_kb / ms_c},
            "kernel_ms": {"closure_run": kt_c, "kinetic_run": kt_k},
            # kernel_ms times one unfused step; with the fused E + H pass in the timed steps the stencils take
            # the step time less the closure and kinetic-fallback kernels
            "stencil_ms_in_step": ms_step_c - kt_c["closure"] - kt_c["kinetic"],
            "launch_shapes": {"closure_run": sh_c, "kinetic_run": sh_k},
            "roofline": {"bound": "tensor", "kernel": "k_closure_tc" if engine == "tcgen05" else "k_closure",
                         "achieved": achieved, "peak": tpk, "unit": "TFLOP/s", "frac": achieved / tpk,
                         "traffic": None, "alg_flops_per_launch": flops, "launch_ms": kt_c["closure"],
                         "peak_source": tsrc},
            "step_hbm_frac_algorithmic": step_alg / (ms_step_c / 1e3) / 1e9 / hpk,
            "gpu_launches": step_launches(steps, 2 if n_kin else 1, fused_in_steps(spec, sh_c))}


def training_config(local: int, n: int = 1 << 20, batch: int = 4096, epochs: int = 3) -> dict:
    """Closure training throughput: `epochs` epochs of minibatch Adam
    (fdtd_mlp_train_epoch: gather, forward + backward on BF16 tensor-core
    tiles, Adam) over n seeded synthetic samples, timed with CUDA events after
    one untimed epoch."""
    import torch
    from paper_2211_05647_gb300 import MlpTrainer
    from paper_2211_05647_gb300 import closure as C
    g = torch.Generator(device="cpu").manual_seed(11)
    x = torch.randn(n, 17, generator=g).to(f"cuda:{local}")
    t = torch.randn(n, generator=g).to(f"cuda:{local}")
    tr = MlpTrainer(C.init_params(3, x.device), batch, lr=1e-3)
    nb = n // batch
    tr.epoch(x, t, 7, 0, 0, (epochs + 1) * nb)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for ep in range(1, epochs + 1):
        tr.epoch(x, t, 7, ep, ep * nb, (epochs + 1) * nb)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    samples = epochs * nb * batch
    # per sample: forward 2 (17*128 + 128*128 + 128), backward 2 (128*128 + 128*128 + 17*128) multiply-adds
    flop = 2 * (17 * 128 + 128 * 128 + 128) + 2 * (2 * 128 * 128 + 17 * 128)
    tf = samples * flop / (ms / 1e3) / 1e12
    pk, src = _peak("bf16_tflops_sustained", 1700.0)
    del x, t, tr
    _release()
    return {"samples_per_s": samples / (ms / 1e3), "ms_per_batch_step": ms / (epochs * nb), "batch": batch,
            "samples": n, "epochs_timed": epochs, "alg_flop_per_sample": flop, "tflops": tf,
            "roofline": {"bound": "tensor", "kernel": "k_mlp_train_tile", "achieved": tf, "peak": pk,
                         "unit": "TFLOP/s", "frac": tf / pk, "peak_source": src}}


def other_configs(args, local: int) -> dict:
    """The other configurations of the benchmark, each at its full size: the
    1-D FP64 slab (its full 2000 steps: a few microseconds each), the 3-D 512^3
    BF16 slab, the 256 batched 1-D runs (FP32 and BF16 delta f) and the
    learned closure against the kinetic solve at 8192^2."""
    out = {}
    auto = not args.no_autotune
    W, K = max(args.warmup, 3), args.steps
    jobs = [
        ("cfg1_1d_slab_fp64", lambda: solver_config("1d_slab_fp64", max(K, 2000), W, auto, local)),
        ("cfg3_3d_512_bf16", lambda: solver_config("3d_512_kinetic_bf16", K, W, auto, local)),
        ("cfg4_batch1d_256_f32", lambda: batch_config("batch1d_256_f32", make_spec("batch1d_256_f32"), K, W, auto,
                                                      local)),
        ("cfg4_batch1d_256_bf16", lambda: batch_config("batch1d_256_bf16", make_spec("batch1d_256_bf16"), K, W, auto,
                                                       local)),
        ("cfg5_closure_8192", lambda: closure_config(K, W, args.engine, auto, local)),
        ("closure_training", lambda: training_config(local)),
    ]
    clocks = ClockSampler(gpu_uuid(local))
    clocks.start()
    for name, job in jobs:
        t0 = time.perf_counter()
        try:
            out[name] = job()
        except Exception as exc:       # reported, not hidden: the entry says what failed
            out[name] = {"error": f"{type(exc).__name__}: {exc}"}
            _release()
        out[name]["wall_s"] = time.perf_counter() - t0
    out["clocks"] = clocks.stop()
    return out


def all_core_oracle():
    """(use the all-core oracle build?, threads it uses); the single-thread
    build when -fopenmp is not available."""
    try:
        from oracle import oracle as O
        O.build(omp=True)
        return True, O.threads(omp=True)
    except Exception:
        return False, 1


def cpu_baseline(workload: str) -> dict:
    """The oracle as it stands on the host cores: the all-core build (value)
    and the single-thread build beside it, each ~15 s of a bounded sample."""
    omp, cores = all_core_oracle()
    g, psr, n, text, _, _ = oracle_throughput(workload, 10 ** 6, 2, budget_s=15.0, omp=omp)
    g1, psr1, n1, _, _, _ = oracle_throughput(workload, 10 ** 6, 2, budget_s=15.0, omp=False)
    return {"value": g, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"{text}; {n} oracle steps in ~15 s on {cores} threads"
                      f"{'' if omp else ' (all-core build unavailable)'}",
            "phase_space_updates_per_s": psr,
            "single_thread": {"value": g1, "unit": UNIT, "cores": 1, "steps": n1, "phase_space_updates_per_s": psr1}}


# --------------------------------------------------------------------- main
def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))

    if args.impl == "reference":
        if rank != 0:
            return 0
        omp, cores = all_core_oracle()
        g, ps, n, text, cells, nodes = oracle_throughput(args.workload, args.steps, args.warmup, None, omp=omp)
        line = {"impl": "reference", "metric": METRIC, "value": g, "unit": UNIT, "n_gpus": args.gpus,
                "steps": n, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload, "sample": text},
                "phase_space_updates_per_s": ps,
                "cpu_baseline": {"value": g, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
                                 "sample": f"{text}; {n} oracle steps, {cores} threads"},
                "e2e": {"value": g, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2211_05647_gb300 import Solver

    if args.workload == "closure_training":
        r = training_config(local)
        if rank == 0:
            print(json.dumps({"metric": "closure training samples/s", "value": r["samples_per_s"],
                              "unit": "samples/s", "n_gpus": world, "steps": r["epochs_timed"], "warmup": 1,
                              "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                              "dtype": "bf16 operands, f32 accumulate", "data": "synthetic (seeded samples)",
                              "config": {"workload": args.workload, "batch": r["batch"], "samples": r["samples"]},
                              **{k: v for k, v in r.items() if k not in ("samples_per_s",)}}), flush=True)
        return 0
    spec = make_spec(args.workload)
    if (args.decompose and world > 1) or args.subdomains > 1:
        return decomposed_bench(args, spec, rank, world, local)
    if isinstance(spec, list):
        return batch_bench(args, spec, rank, world, local)
    if args.workload.endswith("_closure"):
        return closure_bench(args, spec, rank, world, local)
    if args.workload.endswith("_closure_cost"):
        return closure_cost_bench(args, spec, rank, world, local)
    s = Solver.from_spec(spec, device=local)
    ns, nn = s.plasma_shape()
    cells = cells_of(spec)
    st = s.stream
    s.set_option("fused_stencils", args.fused)
    tune = None if args.no_autotune else s.autotune()   # untimed: picks the launch shapes
    if args.kin_shape:
        v = [int(x) for x in args.kin_shape.split(",")] + [0, 0]
        s.set_option("kinetic_shape", v[3] * 10**9 + v[0] * 1000000 + v[1] * 1000 + v[2])
    shapes = s.launch_shapes()                           # the shapes in use (tuned, cached or default)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
            torch.cuda.synchronize()

    # warm-up (captures the step graphs)
    s.step(args.warmup)
    barrier()
    clocks = ClockSampler(gpu_uuid(local))
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    s.step(args.steps)
    e1.record(st)
    barrier()
    clk = clocks.stop()
    ms = reduce_max(e0.elapsed_time(e1), world, f"cuda:{local}")
    ms_step = ms / args.steps
    value = job_rate(cells * args.steps, world, ms / 1e3) / 1e9
    ps_rate = job_rate(ns * nn * args.steps, world, ms / 1e3)

    # per-kernel launch durations (eager launches with CUDA events on the solver's stream)
    kt = s.time_kernels(min(args.steps, 200))
    fused = fused_in_steps(spec, shapes, args.fused)

    # end-to-end through the public API: plasma density and initial fields from
    # pinned host memory, K steps, final fields and J back to pinned host memory
    s.reset()
    pol = {1: "ex", 2: "ez", 3: "ex"}[spec["grid"]["ndim"]]
    dens_h = torch.from_numpy(spec["plasma"]["density"]).pin_memory()
    outs = {1: ["ex", "hy", "j"], 2: ["ez", "hx", "hy", "j"], 3: ["ex", "ey", "ez", "hx", "hy", "hz", "j"]}[
        spec["grid"]["ndim"]]
    init = {n: torch.zeros(s.quantity_bytes(n) // (8 if s.precision == "f64" else 4),
                           dtype=torch.float64 if s.precision == "f64" else torch.float32).pin_memory()
            for n in outs if n != "j"}
    host_out = {n: torch.empty(init[n].shape, dtype=init[n].dtype, pin_memory=True) if n != "j" else
                torch.empty(ns, dtype=torch.float64 if s.precision == "f64" else torch.float32, pin_memory=True)
                for n in outs}
    barrier()
    # phase boundaries are synchronised so the window splits into set-up (plasma set-up from the host density:
    # upload, slot compaction, velocity tables, graph re-capture), field upload, steps and read-back
    t_e2e0 = time.perf_counter()
    p = dict(spec["plasma"])
    p["density"] = dens_h.numpy()
    s.set_plasma(**p)
    torch.cuda.synchronize()
    t_setup = time.perf_counter()
    qid = {"ex": 0, "ey": 1, "ez": 2, "hx": 3, "hy": 4, "hz": 5, "j": 6}
    for n, v in init.items():   # host -> device through the C ABI
        assert s.lib.fdtd_plasma_write_fields(s.h, qid[n], v.data_ptr(), v.numel() * v.element_size(), 0) == 0
    torch.cuda.synchronize()
    t_h2d = time.perf_counter()
    s.step(args.steps)
    torch.cuda.synchronize()
    t_steps = time.perf_counter()
    h2d = dens_h.numel() * 8 + sum(v.numel() * v.element_size() for v in init.values())
    d2h = 0
    for n in outs:
        o = host_out[n]
        rc = s.lib.fdtd_plasma_read_fields(s.h, qid[n], o.data_ptr(), o.numel() * o.element_size(), 0)
        assert rc == 0, rc
        d2h += o.numel() * o.element_size()
    torch.cuda.synchronize()
    t_end = time.perf_counter()
    t_e2e = t_end - t_e2e0
    e2e_breakdown_ms = {"setup_incl_density_h2d": (t_setup - t_e2e0) * 1e3, "fields_h2d": (t_h2d - t_setup) * 1e3,
                        "steps": (t_steps - t_h2d) * 1e3, "d2h": (t_end - t_steps) * 1e3}
    e2e_value = job_rate(cells * args.steps, world, reduce_max(t_e2e, world, f"cuda:{local}")) / 1e9

    if rank != 0:
        dist.destroy_process_group() if world > 1 else None
        return 0

    # roofline of the dominant kernel (the kinetic delta-f stream)
    fbytes = {"f32": 4, "bf16": 2, "f64": 8}[spec["plasma"]["f_dtype"]]
    evolve = bool(spec["plasma"].get("evolve_f0"))
    # read + write delta f once per node (and the F0 correction rows when F0 evolves)
    alg_bytes = 2 * fbytes * ns * nn * (2 if evolve else 1)
    achieved = alg_bytes / (kt["kinetic"] / 1e3) / 1e9
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    kname, kshape = kinetic_kernel(shapes, evolve)
    roof = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak,
            "traffic": ncu_traffic(kname, args.workload, kshape),
            "alg_bytes_per_launch": alg_bytes, "launch_ms": kt["kinetic"],
            "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback"}
    fb = 8 if s.precision == "f64" else 4
    ncomp = {1: 2, 2: 3, 3: 6}[spec["grid"]["ndim"]]
    step_alg = 2 * fb * ncomp * cells + alg_bytes

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if s.precision == "f32" else "f64",
            "data": "synthetic (seeded density field, Gaussian-modulated source)",
            "config": {"workload": args.workload, "grid": [spec["grid"]["nx"], spec["grid"]["ny"], spec["grid"]["nz"]],
                       "ndim": spec["grid"]["ndim"], "plasma_cells": ns, "nodes_per_cell": nn,
                       "f_dtype": spec["plasma"]["f_dtype"], "cpml_cells": spec["grid"]["cpml_cells"],
                       "l2": "inputs larger than L2 (delta f %.2f GB per GPU)" % (ns * nn * fbytes / 1e9),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "phase_space_updates_per_s": ps_rate,
            "step_hbm_frac_algorithmic": step_alg / (ms_step / 1e3) / 1e9 / peak,
            "kernel_ms": kt,
            # kernel_ms times one unfused step; with the fused pass (the option, or the autotuner's 2-D choice)
            # the timed steps fuse each E update with the next H update, so their stencil time is the step
            # time less the kinetic and closure kernels
            "fused_stencils": fused,
            "stencil_ms_in_step": ms_step - kt["kinetic"] - kt["closure"],
            "launch_shapes": dict(shapes, tuned=tune is not None),
            "roofline": roof,
            "gpu_launches": step_launches(args.steps, 1 if ns else 0, fused),
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
                    "d2h_bytes_per_step": d2h / args.steps, "breakdown_ms": e2e_breakdown_ms}}
    if world == 1 and not args.no_configs and args.workload == "2d_tmz_4096_kinetic":
        s.close()
        del s
        _release()
        line["configs"] = other_configs(args, local)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def closure_bench(args, spec, rank, world, local):
    """Learned J closure vs the kinetic solve on the same 8192^2 grid, with
    the committed trained weights (see closure_config)."""
    r = closure_config(args.steps, args.warmup, args.engine, not args.no_autotune, local)
    ms_c = reduce_max(r["ms_per_step"] * args.steps, world, f"cuda:{local}")
    if rank != 0:
        return 0
    cells = cells_of(spec)
    line = {"metric": METRIC, "value": job_rate(cells * args.steps, world, ms_c / 1e3) / 1e9, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_c / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 fields, bf16 MLP operands",
            "data": "synthetic (seeded density fields; weights trained on kinetic runs of seeded fields)",
            "config": {"workload": args.workload, "grid": [spec["grid"]["nx"], spec["grid"]["ny"]],
                       "closure_engine": args.engine, "closure_cells": r["closure_cells"],
                       "kinetic_fallback_cells": r["kinetic_fallback_cells"], "weights": r["weights"],
                       "l2": "inputs larger than L2"},
            "closure_vs_kinetic": r["closure_vs_kinetic"], "kernel_ms": r["kernel_ms"],
            "launch_shapes": r["launch_shapes"], "roofline": r["roofline"],
            "step_hbm_frac_algorithmic": r["step_hbm_frac_algorithmic"], "gpu_launches": r["gpu_launches"]}
    print(json.dumps(line), flush=True)
    return 0


def closure_cost_bench(args, spec, rank, world, local):
    """Inference cost of the learned closure: every plasma cell of the grid on
    the closure, seeded random weights (the cost does not depend on their
    values), K timed graph-replayed steps; roofline of the closure kernel against
    the sustained BF16 tensor peak."""
    import numpy as np
    import torch
    from paper_2211_05647_gb300 import Solver
    s = Solver.from_spec(spec, device=local)
    params = (np.random.default_rng(20221201).standard_normal(18945) * 0.05).astype(np.float32)
    s.set_closure(params, e_scale=1.0, j_scale=1e-3, n_scale=1e18, rho=0.9, n_train_max=1e30, beta=1e-21,
                  engine=args.engine)
    n_kin, n_cl = s.closure_shape()
    s.step(max(args.warmup, 3))
    torch.cuda.synchronize()
    clocks = ClockSampler(gpu_uuid(local))
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s.stream)
    s.step(args.steps)
    e1.record(s.stream)
    e1.synchronize()
    clk = clocks.stop()
    ms = reduce_max(e0.elapsed_time(e1), world, f"cuda:{local}")
    kt = s.time_kernels(min(args.steps, 50))
    if rank != 0:
        return 0
    cells = cells_of(spec)
    flops = 2 * (17 * 128 + 128 * 128 + 128) * n_cl
    peaks = measured_peaks()
    peak = peaks["bf16_tflops_sustained"] if peaks else 1700.0
    achieved = flops / (kt["closure"] / 1e3) / 1e12
    line = {"metric": METRIC, "value": job_rate(cells * args.steps, world, ms / 1e3) / 1e9, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 fields, bf16 MLP operands",
            "data": "synthetic (seeded density field, seeded random closure weights)",
            "config": {"workload": args.workload, "grid": [spec["grid"]["nx"], spec["grid"]["ny"]],
                       "closure_engine": args.engine, "closure_cells": n_cl, "kinetic_fallback_cells": n_kin,
                       "l2": "inputs larger than L2"},
            "kernel_ms": kt,
            "roofline": {"bound": "tensor", "kernel": "k_closure", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                         "alg_flops_per_launch": flops, "launch_ms": kt["closure"],
                         "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained" if peaks else "fallback"},
            "gpu_launches": step_launches(args.steps, 2 if n_kin else 1, fused_in_steps(spec, s.launch_shapes())),
            "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def decomposed_bench(args, spec, rank, world, local):
    """The grid split along its slowest axis: one slab per rank with halos sent
    to the neighbouring ranks (--decompose, N > 1: strong scaling, every rank's
    time is the job's), or K slabs on this GPU with device-to-device halos
    (--subdomains K: the decomposition's cost on one GPU).  Half steps run
    eagerly (a halo exchange sits between them); W warm-up steps, K timed."""
    import torch
    import torch.distributed as dist
    from paper_2211_05647_gb300.decomposed import DecomposedSolver, DistributedSolver
    cells = cells_of(spec)
    if args.subdomains > 1:
        d = DecomposedSolver(spec, parts=args.subdomains, device=local)
        stream, slabs, mode = d.stream, d.bounds, f"{args.subdomains} slabs on one GPU"
    else:
        d = DistributedSolver(spec, rank, world, device=local)
        stream, slabs, mode = d.sub.stream, d.bounds, f"{world} slabs, one per rank (NCCL halos)"
    d.step(args.warmup)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(gpu_uuid(local))
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    d.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = reduce_max(e0.elapsed_time(e1), world, f"cuda:{local}")
    subs = d.subs if args.subdomains > 1 else [d.sub]
    # per slab and step: H, the kinetic rows (slabs with plasma), E, the step counter
    launches = args.steps * sum(3 + (1 if sb.plasma_shape()[0] else 0) for sb in subs)
    d.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    line = {"metric": METRIC, "value": cells * args.steps / (ms / 1e3) / 1e9, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if args.subdomains <= 1 else "weak", "vs_baseline": None,
            "dtype": spec["grid"].get("precision", "f32"), "data": "synthetic (seeded density field)",
            "config": {"workload": args.workload, "decomposition": mode, "slabs": slabs,
                       "l2": "inputs larger than L2", "parallelism": mode},
            "gpu_launches": launches, "clocks": clk}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def batch_bench(args, specs, rank, world, local):
    """Batched independent 1-D runs: one persistent kernel launch per chunk of
    steps (graph replay), chunks of up to 100 steps."""
    import torch
    import torch.distributed as dist
    from paper_2211_05647_gb300 import Batch
    b = Batch(specs, device=local)
    tune = None if args.no_autotune else b.autotune()   # untimed: row shape of the persistent kernel
    info = b.info()
    cells, nodes = info["cells"], info["nodes"]
    st = b.stream
    chunk = min(100, args.steps)
    rem = args.steps % chunk
    b.step(max(args.warmup, 1))
    b.step(chunk)                 # captures the chunk graph outside the timed region
    if rem:
        b.step(rem)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(gpu_uuid(local))
    clocks.start()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps // chunk + 2)]
    evs[0].record(st)
    for i in range(args.steps // chunk):
        b.step(chunk)
        evs[i + 1].record(st)
    if rem:
        b.step(rem)
    e_end = torch.cuda.Event(enable_timing=True)
    e_end.record(st)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = evs[0].elapsed_time(e_end)
    launch_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps // chunk)]
    ms = reduce_max(ms, world, f"cuda:{local}")
    value = job_rate(cells * args.steps, world, ms / 1e3) / 1e9
    # e2e: creation from host specs (density upload), K steps, every run's E and J back to host
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b2 = Batch(specs, device=local)
    b2.step(args.steps)
    d2h = 0
    for r in range(b2.nruns):
        d2h += b2.read(r, "ex").nbytes + b2.read(r, "j").nbytes
    torch.cuda.synchronize()
    te = reduce_max(time.perf_counter() - t0, world, f"cuda:{local}")
    h2d = sum(sp["plasma"]["density"].nbytes for sp in specs)
    b2.close()
    if rank != 0:
        return 0
    fdt = specs[0]["plasma"]["f_dtype"]
    fb = {"f32": 4, "bf16": 2, "f64": 8}[fdt]
    eb = 8 if specs[0]["grid"]["precision"] == "f64" else 4
    alg_step = 2 * eb * (2 * cells + len(specs)) + 2 * fb * nodes
    per_launch_ms = statistics.median(launch_ms) if launch_ms else ms
    achieved = alg_step * chunk / (per_launch_ms / 1e3) / 1e9
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if eb == 4 else "f64", "data": "synthetic (seeded run sizes, slabs, densities)",
            "config": {"workload": args.workload, "runs": len(specs), "cells": cells, "phase_space_nodes": nodes,
                       "f_dtype": fdt, "clusters": info["clusters"], "ctas_per_cluster": info["cluster_ctas"], "steps_per_launch": chunk,
                       "row_shape": tune,
                       "l2": "inputs larger than L2 (delta f %.2f GB)" % (nodes * fb / 1e9),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "phase_space_updates_per_s": job_rate(nodes * args.steps, world, ms / 1e3),
            "roofline": {"bound": "hbm", "kernel": "k_batch1d", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": batch_traffic(args.workload, chunk),
                         "alg_bytes_per_launch": alg_step * chunk,
                         "launch_ms": per_launch_ms,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback"},
            "gpu_launches": 2 * (args.steps // chunk + (1 if rem else 0)),
            "clocks": clk,
            "e2e": {"value": job_rate(cells * args.steps, world, te) / 1e9, "unit": UNIT,
                    "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps}}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload)
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
