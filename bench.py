"""Benchmark: PCG solves of the hp-DG workloads through the C ABI.

Default line (`python bench.py`): the 2D hp-random workload - 32x32 base
squares refined at random (probability 0.3 per cell, depth <= 3, arbitrarily
irregular), degrees p ~ U{1..6}, SIPG with eta = 100, sine right-hand side (4
seeded modes), relative tolerance 1e-8, preconditioner B = B_B + B_C with one
AMG V-cycle on the LOR matrix.  A step is one complete PCG solve (every PCG
iteration runs the operator apply, the preconditioner and the vector
updates).  `value` is DOF-iterations per second of the mixed-precision solve
(FP32 preconditioner, FP64 operator / residual / dots), timed with CUDA
events around the solve's one graph launch; the FP64 solve is timed beside
it.  L2 is flushed (a 512 MiB write) before every timed step.

Beside it the same line carries
  roofline      the operator kernel (FP64-ALU bound) against the FP64 FMA peak
                measured in the same run, and `rooflines` for the trace
                kernel, the block solves and the whole preconditioner (HBM);
  oracle        the FP64 CPU oracle's solution of the same problem and the
                distance of the GPU's mixed and FP64 solutions to it;
  cpu_baseline  the oracle timed on the host cores (one thread and all cores);
  workloads     sub-lines with their own clocks: the same mesh with BR2, the
                16^3 cube workload, the same mesh carried onto a general
                quadrilateral and onto a curved domain (mapped elements),
                the hp-AMR sequences of the L-shape and internal-layer
                problems, the batched form (256
                problems x 4 right-hand sides in one launch) and a bounded
                sample of the served form.
--workload hp2d-br2 | hp2d-coef | hp2d-map | hp2d-curved | hp3d | batched | serving runs one of them as
the line.

--impl reference times the FP64 CPU oracle on the same workload (a bounded
sample of PCG iterations per step).  Multi-GPU: independent replicas (the
problem does not shard), one per rank.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# the CPU oracle legs choose their own thread count: keep numpy's BLAS on one
# thread unless the caller set it (set before numpy is first imported; the
# GPU path does no host BLAS work)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

WORKLOAD = "2D hp-random 32x32 base, prob 0.3, depth<=3, p~U{1..6}, SIPG eta=100, tol 1e-8, seed 0"
METRIC = "DOF-iters/s (PCG on the 2D hp-random workload, mixed FP32 preconditioner / FP64 outer)"
WORKLOAD_BR2 = ("2D hp-random 32x32 base, prob 0.3, depth<=3, p~U{1..6}, BR2 (eta = most sub-faces of one "
                "element), tol 1e-8, seed 0")
METRIC_BR2 = "DOF-iters/s (PCG on the 2D hp-random workload with BR2, mixed FP32 preconditioner / FP64 outer)"
WORKLOAD3 = ("3D hp-random 16^3 base, prob 0.2, depth<=2, p~U{1..5}, BR2 (eta = most sub-faces of one "
             "element), tol 1e-8, seed 0")
METRIC3 = "DOF-iters/s (PCG on the 3D hp-random workload, mixed FP32 preconditioner / FP64 outer)"
WORKLOADC = ("2D hp-random 32x32 base, prob 0.3, depth<=3, p~U{1..6}, coefficient a in {1, 20} by base-cell "
             "parity, SIPG eta=100 (times the larger a of the two sides), tol 1e-8, seed 0")
METRICC = ("DOF-iters/s (PCG on the 2D hp-random workload with a piecewise-constant coefficient, mixed FP32 "
           "preconditioner / FP64 outer)")
WORKLOADM = ("2D hp-random 32x32 base, prob 0.3, depth<=3, p~U{1..6}, carried by the bilinear map of the unit "
             "square onto the quadrilateral (0,0) (1.2,0.1) (0.15,0.95) (1.05,1.25), SIPG eta=100 "
             "(h = sqrt(area)), p+2 Gauss points, tol 1e-8, seed 0")
METRICM = ("DOF-iters/s (PCG on the 2D hp-random workload on mapped quadrilaterals, mixed FP32 preconditioner / "
           "FP64 outer)")
WORKLOADW = ("2D hp-random 32x32 base, prob 0.3, depth<=3, p~U{1..6}, carried by the curved map x = X + 0.06 "
             "sin(pi Y), y = Y + 0.04 sin(pi X) of the unit square (curved elements and faces), SIPG eta=100 "
             "(h = sqrt(area)), p+2 Gauss points, tol 1e-8, seed 0")
METRICW = ("DOF-iters/s (PCG on the 2D hp-random workload on curved elements, mixed FP32 preconditioner / "
           "FP64 outer)")
ORACLE_SAMPLE_ITERS = 20

# DRAM bytes (read + write) of one launch of a kernel on a workload, from the
# ncu captures summarised under profiles/.  Valid only for the sources they
# were taken on: a record reports null as soon as the hash of its sources
# differs from the one captured.
TRAFFIC = {
    "apply_kernel/hp2d": {"sources": ["paper_2009_01287_gb300/csrc/apply_kernel.cuh",
                                      "paper_2009_01287_gb300/csrc/apply_launch.cu",
                                      "paper_2009_01287_gb300/csrc/dg_internal.h",
                                      "paper_2009_01287_gb300/csrc/mesh.cpp"],
                          "sha256_16": "cc1d2ecc3337aba4", "bytes": 3550208},
    "apply3_kernel/hp3d": {"sources": ["paper_2009_01287_gb300/csrc/apply_kernel.cuh",
                                       "paper_2009_01287_gb300/csrc/apply3_kernel.cuh",
                                       "paper_2009_01287_gb300/csrc/apply_launch.cu",
                                       "paper_2009_01287_gb300/csrc/dg_internal.h",
                                       "paper_2009_01287_gb300/csrc/mesh3.cpp"],
                           "sha256_16": "83a21a1d591c4a38",
                           # captured on the same recipe at a 10^3 base (428,796 DOFs), scaled
                           # by the DOFs to the 16^3 workload (1,706,529 DOFs)
                           "bytes": 16861440 * 1706529 // 428796},
    "apply_map_kernel/hp2d-map": {"sources": ["paper_2009_01287_gb300/csrc/apply_map_kernel.cuh",
                                              "paper_2009_01287_gb300/csrc/apply_kernel.cuh",
                                              "paper_2009_01287_gb300/csrc/apply_launch.cu",
                                              "paper_2009_01287_gb300/csrc/dg_internal.h",
                                              "paper_2009_01287_gb300/csrc/mesh_map.cpp"],
                                  "sha256_16": "297ed5dbf05f2fa2", "bytes": 10816000},
}


def traffic(key: str):
    import hashlib
    rec = TRAFFIC.get(key)
    if rec is None or rec["bytes"] is None:
        return None
    h = hashlib.sha256()
    for f in rec["sources"]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return rec["bytes"] if h.hexdigest()[:16] == rec["sha256_16"] else None


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 9:
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def scope_model_flops(mesh) -> float:
    """FP64 flops of one operator apply by the scope table's model: 8(p+1)
    flop/DOF of sum-factorised volume work plus 64/(p+1) per DOF of face work
    (2D), i.e. 8 n^3 + 64 n per element of n = p+1 nodes per direction."""
    import numpy as np
    n = mesh.p.astype(np.float64) + 1.0
    return float(np.sum(8.0 * n ** 3 + 64.0 * n))


def trace_flops(mesh) -> float:
    """FP64 flops of the trace kernel: per side node the normal derivative, a
    contraction of length p+1 (2D: 4 (p+1)^2 FMAs per element; 3D: 6 (p+1)^3)."""
    import numpy as np
    n = mesh.p.astype(np.float64) + 1.0
    return float(np.sum(2.0 * (4.0 * n ** 2 if mesh.dim == 2 else 6.0 * n ** 3)))


# ---------------------------------------------------------------- GPU legs
class Ctx:
    def __init__(self, dev, stream):
        import torch
        self.torch = torch
        self.dev = dev
        self.stream = stream
        self.flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def events(self, n):
        return [self.torch.cuda.Event(enable_timing=True) for _ in range(n)]


def fp64_peak(B, ctx, iters: int = 40000) -> dict:
    tf = [B.dg_fp64_fma_probe(iters, ctx.stream)[0] for _ in range(3)]
    return {"tflops": max(tf), "runs": tf}


def time_solves(B, ctx, M, pc, b, x, tol, steps, warmup):
    torch = ctx.torch
    for _ in range(warmup):
        B.dg_pcg_solve(M.h, pc.h, b, x, tol, 5000, ctx.stream)
    ms, it = [], []
    for _ in range(steps):
        ctx.flush.fill_(1.0)
        torch.cuda.synchronize()
        info = B.dg_pcg_solve(M.h, pc.h, b, x, tol, 5000, ctx.stream)
        ms.append(info.solve_ms)
        it.append(info.iters)
    return ms, it


def operator_rooflines(B, ctx, M, mesh, peak_tf, peaks, three, tkey, mapped=False):
    """The operator kernel and the trace kernel, each timed alone with CUDA
    events (L2 flushed before every launch)."""
    torch = ctx.torch
    n = M.n_dofs
    xin = torch.randn(n, dtype=torch.float64, device=ctx.dev)
    yout = torch.empty_like(xin)
    for _ in range(5):
        B.dg_apply(M.h, xin, yout, ctx.stream)
    tr, ap = [], []
    for _ in range(30):
        ctx.flush.fill_(2.0)
        t = B.dg_apply_profile(M.h, xin, yout, ctx.stream)
        tr.append(t.trace_ms)
        ap.append(t.apply_ms)
    apply_ms, trace_ms = statistics.mean(ap), statistics.mean(tr)
    st = M.stats
    tfl = trace_flops(mesh)
    kfl = st.apply_flops - tfl
    ach = kfl / (apply_ms / 1e3) / 1e12
    name = ("apply3_kernel (BR2 operator on cubes, FP64)" if three else
            "apply_map_kernel (SIPG operator on mapped squares, FP64)" if mapped else
            "apply_kernel (SIPG operator, FP64)")
    model = ("FMAs of the kernel as formulated (x2), counted on the host from the mesh: volume 8 n^3, face "
             "terms 8 n (n + n_nb) per sub-face side, test-function normal derivatives 8 n^2 per element "
             "(n = p+1)")
    if mapped:
        model = ("FMAs of the kernel as formulated (x2), counted on the host from the mesh: volume at q = p+2 "
                 "Gauss points 4 n q (n + q) plus 24 q^2 for the geometric factors, per sub-face side and "
                 "Gauss point 6 (n + n_nb) + 60 (traces, geometry) and 6 n (side sums), test-function normal "
                 "derivatives 8 n^2 per element (n = p+1)")
    separable = not (three or mapped)
    main = {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak_tf, "unit": "TFLOP/s",
            "frac": ach / peak_tf, "traffic": traffic(tkey),
            "flops_per_launch": kfl, "launch_ms": apply_ms,
            "flops_model": model,
            "flops_scope_model_per_launch": scope_model_flops(mesh) if separable else None,
            "frac_scope_model": (scope_model_flops(mesh) / (apply_ms / 1e3) / 1e12 / peak_tf
                                  if separable else None),
            "algorithmic_bytes": st.apply_bytes,
            "hbm_gbs": st.apply_bytes / (apply_ms / 1e3) / 1e9,
            "hbm_frac": st.apply_bytes / (apply_ms / 1e3) / 1e9 / peaks["hbm_gbs"],
            "peak_source": "FP64 FMA-chain probe (dg_fp64_fma_probe) in this run; HBM of measured"}
    trace = {"kernel": "trace3_kernel" if three else "trace_kernel", "bound": "hbm",
             "launch_ms": trace_ms, "flops_per_launch": tfl,
             "note": "inside PCG the traces are written by the p-update kernel, not by this kernel"}
    # side traces: read x once, write u and dn at every side node
    import numpy as np
    npd = mesh.p.astype(np.float64) + 1.0
    side_nodes = float(np.sum(6.0 * npd ** 2 if three else 4.0 * npd))
    tb = 8.0 * n + 16.0 * side_nodes
    trace.update({"algorithmic_bytes": tb, "achieved": tb / (trace_ms / 1e3) / 1e9, "peak": peaks["hbm_gbs"],
                  "unit": "GB/s", "frac": tb / (trace_ms / 1e3) / 1e9 / peaks["hbm_gbs"]})
    return main, trace, apply_ms, trace_ms


def precond_rooflines(B, ctx, pc, peaks):
    torch = ctx.torch
    n = pc.mesh.n_dofs
    r = torch.randn(n, dtype=torch.float64, device=ctx.dev)
    z = torch.empty_like(r)
    for _ in range(3):
        B.dg_precond_apply(pc.h, r, z, ctx.stream)
    parts = {"blocks_ms": [], "restrict_ms": [], "lor_ms": [], "final_ms": [], "total_ms": []}
    for _ in range(30):
        ctx.flush.fill_(4.0)
        t = B.dg_precond_profile(pc.h, r, z, ctx.stream)
        for k in parts:
            parts[k].append(getattr(t, k))
    # the apply as the solve runs it (block solves beside the V-cycle)
    ev = ctx.events(60)
    for i in range(30):
        ctx.flush.fill_(4.0)
        ev[2 * i].record(ctx.stream)
        B.dg_precond_apply(pc.h, r, z, ctx.stream)
        ev[2 * i + 1].record(ctx.stream)
    torch.cuda.synchronize()
    concurrent = statistics.mean(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(30))
    m = {k: statistics.mean(v) for k, v in parts.items()}
    st = pc.stats
    hbm = peaks["hbm_gbs"]
    blocks = {"kernel": "block_solve_kernel (V_e block solves)", "bound": "hbm",
              "achieved": st.block_bytes / (m["blocks_ms"] / 1e3) / 1e9 if m["blocks_ms"] > 0 else None,
              "peak": hbm, "unit": "GB/s", "traffic": None, "algorithmic_bytes": st.block_bytes,
              "launch_ms": m["blocks_ms"]}
    if blocks["achieved"] is not None:
        blocks["frac"] = blocks["achieved"] / hbm
    whole = {"kernel": f"preconditioner z = B r ({st.kernels_per_apply} kernels, serial)", "bound": "hbm",
             "achieved": st.apply_bytes / (m["total_ms"] / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
             "frac": st.apply_bytes / (m["total_ms"] / 1e3) / 1e9 / hbm, "traffic": None,
             "algorithmic_bytes": st.apply_bytes, "launch_ms": m["total_ms"],
             "parts_ms": {k: m[k] for k in ("blocks_ms", "restrict_ms", "lor_ms", "final_ms")},
             "ms_with_blocks_beside_vcycle": concurrent}
    return blocks, whole, concurrent


def measure_single(B, ctx, mesh, rh, form, steps, warmup, peaks, peak_tf, tkey, three=False,
                   e2e=False, keep_x=False, tune=False, mapped=False):
    """Mixed and FP64 solves of one workload, its kernels' rooflines."""
    torch = ctx.torch
    opts64 = B.make_options(form=form, precision=B.DG_PREC_FP64, lor=B.DG_LOR_AMG)
    opts32 = B.make_options(form=form, precision=B.DG_PREC_MIXED, lor=B.DG_LOR_AMG)
    t0 = time.perf_counter()
    M = B.Mesh(mesh, B.make_options(form=form, precision=B.DG_PREC_FP64, lor=B.DG_LOR_AMG,
                                    tune_tiles=1 if tune else 0), ctx.stream)
    pc32 = B.Precond(M, opts32)
    setup_s = time.perf_counter() - t0
    pc64 = B.Precond(M, opts64)
    n = M.n_dofs
    b = torch.empty(n, dtype=torch.float64, device=ctx.dev)
    B.dg_rhs_sine(M.h, rh.amps, rh.waves, b, ctx.stream)
    x32 = torch.empty_like(b)
    x64 = torch.empty_like(b)
    clocks = ClockSampler(ctx.dev.index or 0).start()
    ms32, it32 = time_solves(B, ctx, M, pc32, b, x32, 1e-8, steps, warmup)
    ms64, it64 = time_solves(B, ctx, M, pc64, b, x64, 1e-8, steps, min(warmup, 2))
    main, trace, apply_ms, trace_ms = operator_rooflines(B, ctx, M, mesh, peak_tf, peaks, three, tkey, mapped)
    blocks, whole, pc_ms = precond_rooflines(B, ctx, pc32, peaks)
    out = {"n_dofs": n, "n_elems": int(M.stats.n_elems), "setup_s": setup_s,
           "iters_mixed": statistics.median(it32), "iters_fp64": statistics.median(it64),
           "time_to_tol_ms_mixed": statistics.median(ms32), "time_to_tol_ms_fp64": statistics.median(ms64),
           "dof_iters_per_s_mixed": n * sum(it32) / (sum(ms32) / 1e3),
           "dof_iters_per_s_fp64": n * sum(it64) / (sum(ms64) / 1e3),
           "phase_ms": {"iteration_mixed": statistics.median(ms32) / statistics.median(it32),
                        "operator_apply": apply_ms, "trace": trace_ms, "preconditioner_mixed": pc_ms},
           "roofline": main, "rooflines": [trace, blocks, whole],
           "precond": {"n_conforming": int(pc32.stats.n_conforming), "amg_levels": int(pc32.stats.n_levels),
                       "n_blocks": int(pc32.stats.n_blocks), "max_block": int(pc32.stats.max_block),
                       "kernels_per_apply": int(pc32.stats.kernels_per_apply),
                       "device_bytes": int(pc32.stats.device_bytes)}}
    ms = M.stats
    out["tiles"] = {"tuned": bool(ms.tiles_tuned),
                    "elements_per_tile_by_degree": None if three else list(ms.tile_elems)[1:],
                    "smem_budget_bytes": int(ms.tile_smem_budget) if three else None,
                    "apply_ms_fixed": ms.apply_ms_fixed if ms.tiles_tuned else None,
                    "apply_ms_tuned": ms.apply_ms_tuned if ms.tiles_tuned else None}
    if e2e:
        bh = b.cpu().pin_memory()
        xh = torch.zeros(n, dtype=torch.float64).pin_memory()
        t_e2e, it_e2e = [], []
        for _ in range(steps):
            ctx.flush.fill_(3.0)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            info = B.dg_pcg_solve_host(M.h, pc32.h, bh, xh, 1e-8, 5000, ctx.stream)
            t_e2e.append(time.perf_counter() - t1)
            it_e2e.append(info.iters)
        out["_e2e"] = (t_e2e, it_e2e)
    out["clocks"] = clocks.stop()
    out["_raw"] = (ms32, it32, ms64, it64)
    # the mixed solution's true relative residual with the FP64 operator
    rres = torch.empty_like(b)
    B.dg_apply(M.h, x32, rres, ctx.stream)
    torch.cuda.synchronize()
    out["true_rel_residual_mixed"] = float(torch.linalg.norm(rres - b) / torch.linalg.norm(b))
    if keep_x:
        out["_x"] = (x32.cpu().numpy(), x64.cpu().numpy())
    # operator, the preconditioner's kernels (the x / r update rides its final
    # kernel), the p update with the side traces
    out["kernels_per_iteration"] = 1 + int(pc32.stats.kernels_per_apply) + 1
    for h in (pc32, pc64, M):
        h.close()
    return out


def run_batched_leg(B, ctx, steps, warmup, n_problems=256, n_rhs=4, fp64=False, tune=True):
    """Batched workload: many uneven problems x several right-hand sides in
    one graph launch (every instance keeps its own PCG scalars)."""
    torch = ctx.torch
    from paper_2009_01287_gb300 import inputs
    meshes = [inputs.config3_problem(k)[0] for k in range(n_problems)]
    prec = B.DG_PREC_FP64 if fp64 else B.DG_PREC_MIXED
    t0 = time.perf_counter()
    bat = B.Batch(meshes, n_rhs=n_rhs, opts=B.make_options(precision=prec, tune_tiles=1 if tune else 0),
                  stream=ctx.stream)
    setup_s = time.perf_counter() - t0
    st = bat.stats
    tiles = {"tuned": bool(st.tiles_tuned), "elements_per_tile_by_degree": list(st.tile_elems)[1:],
             "fixed_rule": [min(16, 256 // (p + 1) ** 2) for p in range(1, 9)],
             "apply_ms_fixed": st.apply_ms_fixed if st.tiles_tuned else None,
             "apply_ms_tuned": st.apply_ms_tuned if st.tiles_tuned else None}
    b = torch.empty(bat.n_dofs, dtype=torch.float64, device=ctx.dev)
    bat.rhs_sine([inputs.sine_rhs(2, 1000 + i) for i in range(bat.n_inst)], b, ctx.stream)
    x = torch.empty_like(b)
    for _ in range(warmup):
        bat.solve(b, x, 1e-8, 5000, ctx.stream)
    clocks = ClockSampler(ctx.dev.index or 0).start()
    ms, dofit, iters = [], 0, []
    sizes = [int(bat.offsets[i + 1] - bat.offsets[i]) for i in range(bat.n_inst)]
    for _ in range(steps):
        torch.cuda.synchronize()
        res, t = bat.solve(b, x, 1e-8, 5000, ctx.stream)
        ms.append(t)
        dofit += sum(n * r.iters for n, r in zip(sizes, res))
        iters.append([r.iters for r in res])
    clk = clocks.stop()
    flat = [i for row in iters for i in row]
    bat.close()
    return {"workload": f"batched: {n_problems} 2D hp-random problems (base N log-uniform in [4,64], prob 0.3, "
                        f"depth<=3, p~U{{1..8}}, 1k-300k DOFs each) x {n_rhs} seeded sine RHS, SIPG eta=100, "
                        f"tol 1e-8, one graph launch per step",
            "metric": "DOF-iters/s", "value": dofit / (sum(ms) / 1e3), "ms_per_step": statistics.mean(ms),
            "instances": bat.n_inst, "total_dofs": bat.n_dofs,
            "dtype": "f64 (outer PCG, operator) + " + ("f64" if fp64 else "f32") + " (preconditioner)",
            "iters_min_median_max": [min(flat), statistics.median(flat), max(flat)], "setup_s": setup_s,
            "tiles": tiles, "l2": "vectors exceed L2 (no flush)", "clocks": clk}


def run_serving_leg(B, n_meshes, n_requests, rate, slots):
    from paper_2009_01287_gb300 import inputs, serve
    meshes = inputs.serving_meshes(n_meshes)
    reqs = serve.poisson_stream(n_requests, rate, meshes, seed=0)
    srv = serve.Server(slots=slots, precision=B.DG_PREC_MIXED)
    # resident state for every mesh first (setup is reported, not timed as latency)
    warm = [serve.Request(rid=10 ** 6 + j, arrival=0.0, mesh=m, rhs=inputs.sine_rhs(m.dim, 1))
            for j, m in enumerate(meshes)]
    t = time.perf_counter()
    srv.run(warm, realtime=False)
    setup_s = time.perf_counter() - t
    clocks = ClockSampler(0).start()
    t = time.perf_counter()
    res = srv.run(reqs, realtime=True)
    wall = time.perf_counter() - t
    clk = clocks.stop()
    rep = serve.report(res, wall)
    inflight, evictions = srv.max_inflight, srv.evictions
    srv.close()
    # sequential plain-FP64 loop over the same requests (one slot, FP64 preconditioner)
    seq = serve.Server(slots=1, precision=B.DG_PREC_FP64)
    seq.run(warm, realtime=False)
    t = time.perf_counter()
    res_seq = seq.run(reqs, realtime=True)
    rep_seq = serve.report(res_seq, time.perf_counter() - t)
    seq.close()
    sizes = sorted(m.n_dofs() for m in meshes)
    return {"workload": f"serving: {len(reqs)} requests, Poisson arrivals {rate}/s, {len(meshes)} distinct meshes "
                        f"(half squares, half cubes; DOFs log-uniform in [5k, 2M]: {sizes[0]}..{sizes[-1]}; "
                        f"p~U{{1..6}}), seeded sine RHS per request, tol 1e-8, {slots} slots, 2D SIPG / 3D BR2",
            "metric": "DOF-iters/s and p50/p99 latency", "value": rep["dof_iters_per_s"],
            "p50_latency_s": rep["p50_latency_s"], "p99_latency_s": rep["p99_latency_s"], "ok": rep["ok"],
            "requests": rep["requests"], "requests_3d": rep["requests_3d"], "wall_s": wall,
            "max_inflight": inflight, "evictions": evictions, "setup_s_all_meshes": setup_s,
            "sequential_fp64": rep_seq, "clocks": clk}


# ---------------------------------------------------------------- CPU oracle legs
def _oracle_problem(which: str, seed: int):
    from oracle import rhs, solver
    from paper_2009_01287_gb300 import inputs
    if which == "hp3d":
        mesh, rh = inputs.config2(seed, base=4)
        prob = solver.build_problem(mesh, form="br2")
    else:
        mesh, rh = (inputs.config1_coeff(seed) if which == "hp2d-coef" else
                    inputs.config1_mapped(seed) if which == "hp2d-map" else
                    inputs.config1_curved(seed) if which == "hp2d-curved" else inputs.config1(seed))
        prob = solver.build_problem(mesh, form="br2" if which == "hp2d-br2" else "sipg")
    pc = solver.Preconditioner(prob, lor="amg")
    b = rhs.load_vector(prob.space, rh.amps, rh.waves)
    return prob, pc, b


def _oracle_iters(prob, pc, b, iters: int) -> float:
    from oracle import solver
    t = time.perf_counter()
    solver.pcg(prob.A, b, pc.apply, 1e-30, iters)
    return time.perf_counter() - t


def oracle_leg_main(args):
    """Child process of the CPU baseline: the oracle on the workload, with
    the BLAS thread count its environment sets.  Writes a JSON summary (and
    the solution to tolerance when asked) to args.oracle_out."""
    import pickle

    import numpy as np
    cache = args.oracle_out + ".problem.pkl"
    t = time.perf_counter()
    if os.path.exists(cache):
        prob, pc, b = pickle.load(open(cache, "rb"))
    else:
        prob, pc, b = _oracle_problem(args.workload, args.seed)
        pickle.dump((prob, pc, b), open(cache, "wb"))
    setup_s = time.perf_counter() - t
    dt = _oracle_iters(prob, pc, b, ORACLE_SAMPLE_ITERS)
    out = {"n": int(prob.space.n), "sample_s": dt, "setup_s": setup_s,
           "threads": int(os.environ.get("OMP_NUM_THREADS", "1"))}
    if args.oracle_solve:
        from oracle import solver
        t = time.perf_counter()
        res = solver.pcg(prob.A, b, pc.apply, 1e-8, 5000)
        out.update({"solve_s": time.perf_counter() - t, "iters": res.iters, "rel_res": res.rel_res})
        np.save(args.oracle_out + ".x.npy", res.x)
    json.dump(out, open(args.oracle_out, "w"))


def cpu_baseline(workload: str, seed: int, solve: bool):
    """The oracle as it stands, on the GPU machine's host cores: 20 FP64 PCG
    iterations on one thread and on all cores (BLAS threads; scipy's sparse
    products are single-threaded), plus, when asked, its solve to 1e-8 on one
    thread (returned for the accuracy comparison)."""
    import numpy as np
    nproc = os.cpu_count() or 1
    tmp = tempfile.mkdtemp(prefix="dg_oracle_")
    outp = os.path.join(tmp, "leg.json")
    legs = {}
    for threads, do_solve in ((1, solve), (nproc, False)):
        env = dict(os.environ)
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[v] = str(threads)
        cmd = [sys.executable, os.path.abspath(__file__), "--oracle-leg", "--workload", workload,
               "--seed", str(seed), "--oracle-out", outp] + (["--oracle-solve"] if do_solve else [])
        subprocess.run(cmd, env=env, check=True, timeout=1800)
        legs[threads] = json.load(open(outp))
    n = legs[1]["n"]
    one, allc = legs[1], legs[nproc]
    cpu = platform.processor() or platform.machine()
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                cpu = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    sample = (f"{ORACLE_SAMPLE_ITERS} FP64 PCG iterations of the same workload" +
              (" on the same recipe with a 4^3 base" if workload == "hp3d" else "") +
              f" ({n} DOFs; setup untimed), scipy sparse + numpy")
    out = {"value": n * ORACLE_SAMPLE_ITERS / one["sample_s"], "unit": "DOF-iters/s", "cores": 1,
           "kind": "oracle", "sample": sample + ", one thread",
           "all_cores": {"value": n * ORACLE_SAMPLE_ITERS / allc["sample_s"], "cores": nproc,
                         "note": "BLAS on all cores; the sparse products stay single-threaded"},
           "nproc": nproc, "cpu": cpu, "setup_s": one["setup_s"]}
    x = None
    if solve:
        out["time_to_tol_s"] = one["solve_s"]
        out["iters"] = one["iters"]
        x = np.load(outp + ".x.npy")
    return out, x


# ---------------------------------------------------------------- main line
def run_ours(args):
    import numpy as np
    import torch

    from paper_2009_01287_gb300 import binding as B
    from paper_2009_01287_gb300 import inputs

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    ctx = Ctx(dev, torch.cuda.current_stream(dev))
    three = args.workload == "hp3d"
    coef = args.workload == "hp2d-coef"
    br2 = args.workload == "hp2d-br2"
    curved = args.workload == "hp2d-curved"
    mapped = args.workload == "hp2d-map" or curved
    if three:
        mesh, rh = inputs.config2(args.seed, base=args.base3)
    else:
        mesh, rh = (inputs.config1_coeff(args.seed) if coef else
                    inputs.config1_curved(args.seed) if curved else
                    inputs.config1_mapped(args.seed) if mapped else inputs.config1(args.seed))
    form = B.DG_FORM_BR2 if (three or br2) else B.DG_FORM_SIPG
    metric, workload = ((METRIC3, WORKLOAD3) if three else (METRICC, WORKLOADC) if coef else
                        (METRICW, WORKLOADW) if curved else (METRICM, WORKLOADM) if mapped else
                        (METRIC_BR2, WORKLOAD_BR2) if br2 else (METRIC, WORKLOAD))
    peaks, peak_kind = _peaks()
    probe = fp64_peak(B, ctx)
    if dist:
        dist.barrier()
    tkey = ("apply3_kernel/hp3d" if three else "apply_map_kernel/hp2d-map" if (mapped and not curved) else
            "none" if curved else
            "apply_kernel/hp2d" if not (coef or br2) else "none")
    res = measure_single(B, ctx, mesh, rh, form, args.steps, args.warmup, peaks, probe["tflops"], tkey,
                         three=three, e2e=True, keep_x=True, tune=args.tune_tiles, mapped=mapped)
    ms32, it32, ms64, it64 = res.pop("_raw")
    t_e2e, it_e2e = res.pop("_e2e")
    x32, x64 = res.pop("_x")
    from paper_2009_01287_gb300 import replicas
    n = res["n_dofs"]
    (t32, t64, te), dof_iters32 = replicas.aggregate(
        [sum(ms32) / 1e3, sum(ms64) / 1e3, sum(t_e2e)], n * sum(it32), device=dev)
    value = dof_iters32 / t32
    launches = sum(3 + res["precond"]["kernels_per_apply"] + it * res["kernels_per_iteration"] for it in it32)
    res["roofline"]["peak_fp64_probe_runs"] = probe["runs"]
    out = {
        "metric": metric,
        "value": value,
        "unit": "DOF-iters/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * t32 / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64 (outer PCG, operator) + f32 (preconditioner)",
        "data": "synthetic",
        "config": {"workload": workload, "n_dofs": n,
                   "n_elems": res["n_elems"], **res["precond"],
                   "parallelism": f"replicas x{ws}", "l2": "flushed (512 MiB write) before every step",
                   "timed": "CUDA events around each solve's one graph launch (copy of b, start, "
                            "while-loop of iterations, copy of x); no host round trip inside"},
        "iters_mixed": res["iters_mixed"],
        "iters_fp64": res["iters_fp64"],
        "time_to_tol_ms_mixed": res["time_to_tol_ms_mixed"],
        "time_to_tol_ms_fp64": res["time_to_tol_ms_fp64"],
        "dof_iters_per_s_fp64": ws * n * sum(it64) / t64,   # replicas: identical per rank
        "setup_s": res["setup_s"],
        "phase_ms": res["phase_ms"],
        "e2e": {"value": ws * n * sum(it_e2e) / te, "unit": "DOF-iters/s",
                "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n},
        "roofline": res["roofline"],
        "rooflines": res["rooflines"],
        "tiles": res["tiles"],
        "fp64_peak_tflops_measured": probe["tflops"],
        "gpu_launches": launches,
        "clocks": res["clocks"],
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cb, xo = cpu_baseline(args.workload, args.seed, solve=not three)
        out["cpu_baseline"] = cb
        if xo is not None:
            sc = float(np.abs(xo).max())
            out["oracle"] = {"iters": cb.get("iters"), "time_to_tol_s_one_thread": cb.get("time_to_tol_s"),
                             "rel_err_mixed": float(np.abs(x32 - xo).max()) / sc,
                             "rel_err_fp64": float(np.abs(x64 - xo).max()) / sc,
                             "norm": "max-norm of the difference over the max-norm of the oracle's solution"}
            out["oracle_rel_err_mixed"] = out["oracle"]["rel_err_mixed"]
    if rank == 0 and ws == 1 and not args.no_extras and args.workload == "hp2d":
        extras = {}

        def leg(name, fn):
            # a failing sub-line is recorded as such; the main line still prints
            try:
                extras[name] = fn()
            except Exception as exc:   # noqa: BLE001
                extras[name] = {"error": f"{type(exc).__name__}: {exc}"}

        def single(workload, mesh_rhs, form, traffic_key, **kw):
            mesh, rhs_ = mesh_rhs
            r = measure_single(B, ctx, mesh, rhs_, form, 3, 2, peaks, probe["tflops"], traffic_key, **kw)
            for k in ("_raw", "_e2e", "_x"):
                r.pop(k, None)
            return {"workload": workload, "metric": "DOF-iters/s", "value": r["dof_iters_per_s_mixed"], **r}

        leg("hp2d_br2", lambda: single(WORKLOAD_BR2, inputs.config1(args.seed), B.DG_FORM_BR2, "none"))
        leg("hp3d", lambda: single(WORKLOAD3, inputs.config2(args.seed), B.DG_FORM_BR2, "apply3_kernel/hp3d",
                                   three=True))
        leg("hp2d_map", lambda: single(WORKLOADM, inputs.config1_mapped(args.seed), B.DG_FORM_SIPG,
                                       "apply_map_kernel/hp2d-map", mapped=True))
        leg("hp2d_curved", lambda: single(WORKLOADW, inputs.config1_curved(args.seed), B.DG_FORM_SIPG, "none",
                                          mapped=True))
        for which in ("lshape", "layer"):   # the adaptive problems of Section 4.2
            leg(f"amr_{which}", lambda which=which: amr_leg(B, torch, which, 20))
        leg("batched", lambda: run_batched_leg(B, ctx, 2, 1))
        leg("serving", lambda: run_serving_leg(B, 8, 160, 200.0, 8))
        out["workloads"] = extras
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_serving(args):
    import torch
    from paper_2009_01287_gb300 import binding as B
    torch.cuda.set_device(0)
    leg = run_serving_leg(B, args.serve_meshes, args.serve_requests, args.serve_rate, args.serve_slots)
    out = {"metric": "p50/p99 solve latency and DOF-iters/s (continuous-batching server)",
           "value": leg["value"], "unit": "DOF-iters/s", "n_gpus": 1, "steps": 1, "warmup": 1,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64 (outer PCG, operator) + f32 (preconditioner)", "data": "synthetic",
           "config": {"workload": leg.pop("workload")}, **{k: v for k, v in leg.items() if k != "value"}}
    print(json.dumps(out))


def run_batched(args):
    import torch
    from paper_2009_01287_gb300 import binding as B
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    ctx = Ctx(dev, torch.cuda.current_stream(dev))
    leg = run_batched_leg(B, ctx, args.steps, args.warmup, args.batch_problems, args.batch_rhs, args.batch_fp64,
                          tune=not args.batch_fixed_tiles)
    out = {"metric": "DOF-iters/s (batched PCG, all instances in one graph launch)", "value": leg["value"],
           "unit": "DOF-iters/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": leg["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": leg["dtype"], "data": "synthetic",
           "config": {"workload": leg["workload"], "instances": leg["instances"], "total_dofs": leg["total_dofs"],
                      "l2": leg["l2"]},
           "iters_min_median_max": leg["iters_min_median_max"], "setup_s": leg["setup_s"], "tiles": leg["tiles"],
           "clocks": leg["clocks"]}
    print(json.dumps(out))


def amr_leg(B, torch, which: str, n_steps: int) -> dict:
    """The AMR sequence of one problem of Section 4.2 (`which`: "lshape" or
    "layer") through the C ABI: mixed-precision solves with B = B_B + B_C
    drive the refinement, and every step also solves with FP64 B~ = J_B + B_C
    for the iteration column the paper reports beside it."""
    from paper_2009_01287_gb300 import amr
    problem = amr.LSHAPE if which == "lshape" else amr.LAYER
    mixed = amr.library_solver(B, torch, precision=B.DG_PREC_MIXED, with_jacobi=False, problem=problem)
    b_tilde = amr.library_solver(B, torch, with_jacobi=True, problem=problem)

    def solve(mesh):
        x, info = mixed(mesh)
        info["iters_jacobi"] = b_tilde(mesh)[1]["iters_jacobi"]
        return x, info

    clocks = ClockSampler(0).start()
    t0 = time.perf_counter()
    recs = amr.run(solve, steps=n_steps, problem=problem)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    di = sum(r.n_dofs * r.iters for r in recs)
    ms = sum(r.solve_ms for r in recs)
    return {"workload": f"hp-AMR of the {problem.name}, {problem.initial().n_elems} p=1 squares to start, "
                        f"{n_steps} refinements, SIPG eta=100, tol 1e-8, weak Dirichlet data",
            "metric": "DOF-iters/s over the solves of the AMR sequence (mixed FP32 preconditioner / FP64 outer)",
            "value": di / (ms / 1e3), "wall_s_with_setup": wall,
            "table": [dataclasses.asdict(r) for r in recs], "clocks": clk}


def run_amr(args):
    """hp-adaptive refinement of the internal-layer or the L-shape problem (Section 4.2):
    `--amr-steps` refinements after the first solve, every solve through the C
    ABI (mixed-precision B = B_B + B_C, and FP64 B~ = J_B + B_C for the
    iteration column the paper reports beside it)."""
    import torch

    from paper_2009_01287_gb300 import binding as B
    torch.cuda.set_device(0)
    leg = amr_leg(B, torch, "lshape" if args.workload == "amr-lshape" else "layer", args.amr_steps)
    out = {"metric": leg["metric"], "value": leg["value"], "unit": "DOF-iters/s", "n_gpus": 1,
           "steps": len(leg["table"]), "warmup": 0, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64 (outer PCG, operator) + f32 (preconditioner)", "data": "synthetic",
           "config": {"workload": leg["workload"]}, "wall_s_with_setup": leg["wall_s_with_setup"],
           "table": leg["table"], "clocks": leg["clocks"]}
    print(json.dumps(out))


def run_reference_amr(args):
    """The oracle through the same AMR sequence (its own solves drive the
    marking): FP64 PCG with B = B_B + B_C per step, timed on one thread."""
    from oracle import rhs, solver

    from paper_2009_01287_gb300 import amr
    problem = amr.LSHAPE if args.workload == "amr-lshape" else amr.LAYER
    pcg_s = []

    def solve(mesh):
        prob = solver.build_problem(mesh)
        pc = solver.Preconditioner(prob, lor="amg")
        b = rhs.dirichlet_load(prob.space, problem.f, problem.u, 100.0)
        t = time.perf_counter()
        res = solver.pcg(prob.A, b, pc.apply, 1e-8, 20000)
        pcg_s.append(time.perf_counter() - t)
        return res.x, {"iters": res.iters, "n_blocks": len(prob.cs.blocks),
                       "max_block": max((len(bk) for bk in prob.cs.blocks), default=0)}

    recs = amr.run(solve, steps=args.amr_steps, problem=problem)
    di = sum(r.n_dofs * r.iters for r in recs)
    value = di / sum(pcg_s)
    sample = f"the {args.amr_steps}-step AMR sequence driven by the oracle's own solves, FP64 PCG timed"
    print(json.dumps({
        "impl": "reference", "metric": "DOF-iters/s over the solves of the AMR sequence", "value": value,
        "unit": "DOF-iters/s", "n_gpus": 1, "steps": len(recs), "warmup": 0, "ms_per_step": 1e3 * sum(pcg_s) / len(recs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"hp-AMR of the {problem.name}, {problem.initial().n_elems} p=1 squares to start, "
                               f"{args.amr_steps} refinements, SIPG eta=100, tol 1e-8, weak Dirichlet data"},
        "cpu_baseline": {"value": value, "unit": "DOF-iters/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "DOF-iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "table": [dataclasses.asdict(r) for r in recs]}))


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    if args.workload in ("amr-layer", "amr-lshape"):
        run_reference_amr(args)
        return
    if args.workload in ("batched", "serving"):
        print(json.dumps({"impl": "reference", "unavailable": f"the oracle has no {args.workload} form; "
                          "its single-problem PCG is timed by the hp2d, hp2d-br2, hp2d-coef, hp2d-map, hp2d-curved "
                          "and hp3d workloads"}))
        return
    three = args.workload == "hp3d"
    coef = args.workload == "hp2d-coef"
    br2 = args.workload == "hp2d-br2"
    mapped = args.workload == "hp2d-map"
    curved = args.workload == "hp2d-curved"
    metric, workload = ((METRIC3, WORKLOAD3) if three else (METRICC, WORKLOADC) if coef else
                        (METRICM, WORKLOADM) if mapped else (METRICW, WORKLOADW) if curved else
                        (METRIC_BR2, WORKLOAD_BR2) if br2 else (METRIC, WORKLOAD))
    prob, pc, b = _oracle_problem(args.workload, args.seed)
    for _ in range(args.warmup):
        _oracle_iters(prob, pc, b, ORACLE_SAMPLE_ITERS)
    times = [_oracle_iters(prob, pc, b, ORACLE_SAMPLE_ITERS) for _ in range(args.steps)]
    n = prob.space.n
    value = n * ORACLE_SAMPLE_ITERS * args.steps / sum(times)
    sample = f"{ORACLE_SAMPLE_ITERS} FP64 PCG iterations per step"
    if three:
        sample += f" on the same recipe with a 4^3 base ({n} DOFs)"
    out = {
        "impl": "reference",
        "metric": metric,
        "value": value,
        "unit": "DOF-iters/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload, "n_dofs": n},
        "cpu_baseline": {"value": value, "unit": "DOF-iters/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "DOF-iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="only the line's own workload")
    ap.add_argument("--workload", default="hp2d",
                    choices=["hp2d", "hp2d-br2", "hp2d-coef", "hp2d-map", "hp2d-curved", "hp3d", "batched",
                             "serving", "amr-layer", "amr-lshape"])
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-meshes", type=int, default=16)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--batch-problems", type=int, default=256)
    ap.add_argument("--batch-rhs", type=int, default=4)
    ap.add_argument("--batch-fp64", action="store_true")
    ap.add_argument("--batch-fixed-tiles", action="store_true", help="skip the tile tuner")
    ap.add_argument("--tune-tiles", action="store_true",
                    help="single-mesh workloads: let dg_mesh_create tune the operator's tiles")
    ap.add_argument("--base3", type=int, default=16,
                    help="cube workload: base grid per axis (16 is the workload; smaller for profiling captures)")
    ap.add_argument("--amr-steps", type=int, default=20, help="amr workloads: refinement steps")
    ap.add_argument("--oracle-leg", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--oracle-out", default="", help=argparse.SUPPRESS)
    ap.add_argument("--oracle-solve", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_leg:
        oracle_leg_main(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload in ("amr-layer", "amr-lshape"):
        run_amr(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
