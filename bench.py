"""Benchmark: PCG solves of the 2D hp-random workload through the C ABI.

Workload: 2D Poisson on [0,1]^2, 32x32 base squares refined at random
(probability 0.3 per cell, depth <= 3, arbitrarily irregular), degrees
p ~ U{1..6}, SIPG with eta = 100, sine right-hand side (4 seeded modes),
relative tolerance 1e-8; preconditioner B = B_B + B_C with one AMG V-cycle
on the LOR matrix.  A step is one complete PCG solve (every PCG iteration
runs the operator apply, the preconditioner and the vector updates).
`value` is DOF-iterations per second of the mixed-precision solve (FP32
preconditioner, FP64 operator / residual / dots); the FP64 solve is timed
beside it.  L2 is flushed (a 512 MiB write) before every timed step.

--workload hp2d-coef runs the same mesh with the piecewise-constant coefficient
a in {1, 20} of the random-refinement problem (Section 4.3); hp3d the cube
workload; batched and serving the B1 and V1 forms.

--impl reference times the FP64 CPU oracle on the same workload (a bounded
sample of PCG iterations per step).  Multi-GPU: independent replicas
(the problem does not shard), one per rank.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# the CPU oracle legs report one core: keep numpy's BLAS on one thread (set
# before numpy is first imported; the GPU path does no host BLAS work)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

WORKLOAD = "2D hp-random 32x32 base, prob 0.3, depth<=3, p~U{1..6}, SIPG eta=100, tol 1e-8, seed 0"
METRIC = "DOF-iters/s (PCG on the 2D hp-random workload, mixed FP32 preconditioner / FP64 outer)"
WORKLOAD3 = ("3D hp-random 16^3 base, prob 0.2, depth<=2, p~U{1..5}, BR2 (eta = most sub-faces of one "
             "element), tol 1e-8, seed 0")
METRIC3 = "DOF-iters/s (PCG on the 3D hp-random workload, mixed FP32 preconditioner / FP64 outer)"
WORKLOADC = ("2D hp-random 32x32 base, prob 0.3, depth<=3, p~U{1..6}, coefficient a in {1, 20} by base-cell "
             "parity, SIPG eta=100 (times the larger a of the two sides), tol 1e-8, seed 0")
METRICC = ("DOF-iters/s (PCG on the 2D hp-random workload with a piecewise-constant coefficient, mixed FP32 "
           "preconditioner / FP64 outer)")
ORACLE_SAMPLE_ITERS = 20

# DRAM bytes (read + write) of one apply_kernel launch on this workload, from
# the ncu capture summarised in profiles/apply_kernel_hp2d_32x32.md.  Valid
# only for the kernel and tile-building sources it was taken on: the line
# reports null traffic as soon as their hash differs.
APPLY_TRAFFIC = {"sources": ["paper_2009_01287_gb300/csrc/apply_kernel.cuh",
                             "paper_2009_01287_gb300/csrc/apply_launch.cu",
                             "paper_2009_01287_gb300/csrc/dg_internal.h",
                             "paper_2009_01287_gb300/csrc/mesh.cpp"],
                 "sha256_16": "74d388822a4cf47a", "bytes": 3548672 + 0}
# likewise for the 3D operator (profiles/apply3_kernel_hp3d_16cube.md)
APPLY3_TRAFFIC = {"sources": ["paper_2009_01287_gb300/csrc/apply_kernel.cuh",
                              "paper_2009_01287_gb300/csrc/apply3_kernel.cuh",
                              "paper_2009_01287_gb300/csrc/apply_launch.cu",
                              "paper_2009_01287_gb300/csrc/dg_internal.h",
                              "paper_2009_01287_gb300/csrc/mesh3.cpp"],
                  "sha256_16": "64366f7762b242cf", "bytes": 66824192 + 5452288}


def apply_traffic(three: bool = False):
    import hashlib
    rec = APPLY3_TRAFFIC if three else APPLY_TRAFFIC
    if rec["bytes"] is None:
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


def fp64_peak_tflops(sm_mhz: float) -> float:
    """FP64 FMA peak: 152 SMs x 2 FP64 FMA per SM per clock (GB300 nominal
    1.25 TFLOP/s at ~2.07 GHz), at the SM clock sampled under load."""
    return 152 * 2 * 2 * sm_mhz * 1e6 / 1e12


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
    stream = torch.cuda.current_stream(dev)
    three = args.workload == "hp3d"
    coef = args.workload == "hp2d-coef"
    if three:
        mesh, rh = inputs.config2(args.seed)
    else:
        mesh, rh = inputs.config1_coeff(args.seed) if coef else inputs.config1(args.seed)
    form = B.DG_FORM_BR2 if three else B.DG_FORM_SIPG
    opts64 = B.make_options(form=form, precision=B.DG_PREC_FP64, lor=B.DG_LOR_AMG)
    opts32 = B.make_options(form=form, precision=B.DG_PREC_MIXED, lor=B.DG_LOR_AMG)
    M = B.Mesh(mesh, opts64, stream)
    t0 = time.perf_counter()
    pc32 = B.Precond(M, opts32)
    setup_s = time.perf_counter() - t0
    pc64 = B.Precond(M, opts64)
    n = M.n_dofs
    b = torch.empty(n, dtype=torch.float64, device=dev)
    B.dg_rhs_sine(M.h, rh.amps, rh.waves, b, stream)
    x = torch.empty_like(b)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    tol, maxit = args.tol, 5000

    def solve(pc):
        return B.dg_pcg_solve(M.h, pc.h, b, x, tol, maxit, stream)

    for _ in range(args.warmup):
        solve(pc32)
        solve(pc64)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms32, it32, ms64, it64 = [], [], [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        info = solve(pc32)
        ms32.append(info.solve_ms)
        it32.append(info.iters)
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        info = solve(pc64)
        ms64.append(info.solve_ms)
        it64.append(info.iters)
    torch.cuda.synchronize()
    # dominant kernel: the operator apply, timed alone on the launching stream
    xin = torch.randn(n, dtype=torch.float64, device=dev)
    yout = torch.empty_like(xin)
    for _ in range(5):
        B.dg_apply(M.h, xin, yout, stream)
    napply = 50
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * napply)]
    for i in range(napply):
        flush.fill_(2.0)
        ev[2 * i].record(stream)
        B.dg_apply(M.h, xin, yout, stream)
        ev[2 * i + 1].record(stream)
    torch.cuda.synchronize()
    apply_ms = statistics.mean(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(napply))
    # the mixed preconditioner alone, timed the same way (phase breakdown)
    for i in range(napply):
        flush.fill_(4.0)
        ev[2 * i].record(stream)
        B.dg_precond_apply(pc32.h, xin, yout, stream)
        ev[2 * i + 1].record(stream)
    torch.cuda.synchronize()
    precond_ms = statistics.mean(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(napply))
    # end to end: host buffers in and out through the C ABI (pinned)
    bh = b.cpu().pin_memory()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory()
    t_e2e, it_e2e = [], []
    for _ in range(args.steps):
        flush.fill_(3.0)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        info = B.dg_pcg_solve_host(M.h, pc32.h, bh, xh, tol, maxit, stream)
        t_e2e.append(time.perf_counter() - t1)
        it_e2e.append(info.iters)
    clk = clocks.stop()
    from paper_2009_01287_gb300 import replicas
    (t32, t64, te), dof_iters32 = replicas.aggregate(
        [sum(ms32) / 1e3, sum(ms64) / 1e3, sum(t_e2e)], n * sum(it32), device=dev)
    value = dof_iters32 / t32
    stats = M.stats
    s32 = pc32.stats
    peaks, peak_kind = _peaks()
    sm_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp64_peak = fp64_peak_tflops(sm_mhz)
    achieved_tf = stats.apply_flops / (apply_ms / 1e3) / 1e12
    levels = s32.n_levels
    # preconditioner launches as the library reports them (restriction, two or
    # four kernels per AMG level, dense coarsest level, block solves, final)
    precond_kernels = int(s32.kernels_per_apply)
    # iteration: operator apply, x / r update, preconditioner, p update with traces
    kernels_per_iter = 1 + 1 + precond_kernels + 1
    launches = sum(2 + precond_kernels + it * kernels_per_iter for it in it32)  # + init, first p
    out = {
        "metric": METRIC3 if three else (METRICC if coef else METRIC),
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
        "config": {"workload": WORKLOAD3 if three else (WORKLOADC if coef else WORKLOAD), "n_dofs": n,
                   "n_elems": int(stats.n_elems),
                   "n_conforming": int(s32.n_conforming), "amg_levels": levels,
                   "n_blocks": int(s32.n_blocks), "max_block": int(s32.max_block),
                   "amg_plain_levels": [int(s32.level_plain[i]) for i in range(levels)],
                   "parallelism": f"replicas x{ws}", "l2": "flushed (512 MiB write) before every step"},
        "iters_mixed": statistics.median(it32),
        "iters_fp64": statistics.median(it64),
        "time_to_tol_ms_mixed": statistics.median(ms32),
        "time_to_tol_ms_fp64": statistics.median(ms64),
        "dof_iters_per_s_fp64": ws * n * sum(it64) / t64,   # replicas: identical per rank
        "setup_s": setup_s,
        "phase_ms": {"iteration_mixed": statistics.median(ms32) / statistics.median(it32),
                     "operator_apply": apply_ms, "preconditioner_mixed": precond_ms},
        "e2e": {"value": ws * n * sum(it_e2e) / te, "unit": "DOF-iters/s",
                "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n},
        "roofline": {"kernel": ("apply3_kernel (BR2 operator on cubes, FP64)" if three
                                else "apply_kernel (SIPG operator, FP64)"), "bound": "alu",
                     "achieved": achieved_tf, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": achieved_tf / fp64_peak, "traffic": None if coef else apply_traffic(three),
                     "algorithmic_bytes": stats.apply_bytes,
                     "flops_per_launch": stats.apply_flops, "launch_ms": apply_ms,
                     "hbm_gbs": stats.apply_bytes / (apply_ms / 1e3) / 1e9,
                     "hbm_frac": stats.apply_bytes / (apply_ms / 1e3) / 1e9 / peaks["hbm_gbs"],
                     "peak_source": f"FP64 FMA units x sampled SM clock; HBM {peak_kind}"},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        out["cpu_baseline"] = cpu_baseline3(args) if three else cpu_baseline(args, coef)
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


SERVE_WORKLOAD = ("serving: {n} requests, Poisson arrivals {rate}/s, {m} distinct 2D hp-random meshes "
                  "(DOFs log-uniform in [5k, 200k], prob 0.3, depth<=3, p~U{{1..6}}), seeded sine RHS per request, "
                  "tol 1e-8, {slots} slots")


def serve_meshes(m: int, seed: int = 0):
    """m distinct meshes with DOF targets log-uniform in [5k, 200k]."""
    import numpy as np
    from paper_2009_01287_gb300 import inputs
    rng = np.random.Generator(np.random.PCG64(777 + seed))
    out = []
    for j in range(m):
        target = math.exp(rng.uniform(math.log(5e3), math.log(2e5)))
        base = max(2, int(round(math.sqrt(target / 99.0))))
        out.append(inputs.random_refined_mesh(2, base, 3, 0.3, 1, 6, seed=9000 + j))
    return out


def run_serving(args):
    import torch

    from paper_2009_01287_gb300 import binding as B
    from paper_2009_01287_gb300 import serve

    torch.cuda.set_device(0)
    meshes = serve_meshes(args.serve_meshes)
    reqs = serve.poisson_stream(args.serve_requests, args.serve_rate, meshes, seed=0)
    # warm-up: resident state for every mesh (setup is reported, not timed as latency)
    srv = serve.Server(slots=args.serve_slots, precision=B.DG_PREC_MIXED)
    warm = [serve.Request(rid=10 ** 6 + j, arrival=0.0, mesh=m, rhs=reqs[0].rhs) for j, m in enumerate(meshes)]
    t = time.perf_counter()
    srv.run(warm, realtime=False)
    setup_s = time.perf_counter() - t
    clocks = ClockSampler(0)
    clocks.start()
    t = time.perf_counter()
    res = srv.run(reqs, realtime=True)
    wall = time.perf_counter() - t
    clk = clocks.stop()
    rep = serve.report(res, wall)
    srv.close()
    # sequential plain-FP64 loop over the same requests (one slot, FP64 preconditioner)
    seq = serve.Server(slots=1, precision=B.DG_PREC_FP64)
    seq.run(warm, realtime=False)
    t = time.perf_counter()
    res_seq = seq.run(reqs, realtime=True)
    wall_seq = time.perf_counter() - t
    rep_seq = serve.report(res_seq, wall_seq)
    seq.close()
    out = {
        "metric": "p50/p99 solve latency and DOF-iters/s (continuous-batching server)",
        "value": rep["dof_iters_per_s"],
        "unit": "DOF-iters/s",
        "n_gpus": 1,
        "steps": 1,
        "warmup": 1,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64 (outer PCG, operator) + f32 (preconditioner)",
        "data": "synthetic",
        "config": {"workload": SERVE_WORKLOAD.format(n=len(reqs), rate=args.serve_rate, m=len(meshes),
                                                     slots=args.serve_slots)},
        "p50_latency_s": rep["p50_latency_s"],
        "p99_latency_s": rep["p99_latency_s"],
        "ok": rep["ok"],
        "wall_s": wall,
        "max_inflight": srv.max_inflight,
        "sequential_fp64": rep_seq,
        "setup_s_all_meshes": setup_s,
        "clocks": clk,
    }
    print(json.dumps(out))


BATCH_WORKLOAD = ("batched: {n} 2D hp-random problems (base N log-uniform in [4,64], prob 0.3, depth<=3, "
                  "p~U{{1..8}}, 1k-300k DOFs each) x {r} seeded sine RHS, SIPG eta=100, tol 1e-8, one graph launch")


def run_batched(args):
    """Batched workload: many uneven problems x several right-hand sides in
    one graph launch (every instance keeps its own PCG scalars)."""
    import torch

    from paper_2009_01287_gb300 import binding as B
    from paper_2009_01287_gb300 import inputs

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    meshes = [inputs.config3_problem(k)[0] for k in range(args.batch_problems)]
    n_rhs = args.batch_rhs
    prec = B.DG_PREC_FP64 if args.batch_fp64 else B.DG_PREC_MIXED
    t0 = time.perf_counter()
    bat = B.Batch(meshes, n_rhs=n_rhs, opts=B.make_options(precision=prec), stream=stream)
    setup_s = time.perf_counter() - t0
    b = torch.empty(bat.n_dofs, dtype=torch.float64, device=dev)
    bat.rhs_sine([inputs.sine_rhs(2, 1000 + i) for i in range(bat.n_inst)], b, stream)
    x = torch.empty_like(b)
    for _ in range(args.warmup):
        bat.solve(b, x, args.tol, 5000, stream)
    clocks = ClockSampler(0)
    clocks.start()
    ms, dofit, iters = [], 0, []
    sizes = [int(bat.offsets[i + 1] - bat.offsets[i]) for i in range(bat.n_inst)]
    for _ in range(args.steps):
        torch.cuda.synchronize()
        res, t = bat.solve(b, x, args.tol, 5000, stream)
        ms.append(t)
        dofit += sum(n * r.iters for n, r in zip(sizes, res))
        iters.append([r.iters for r in res])
    clk = clocks.stop()
    flat = [i for row in iters for i in row]
    out = {
        "metric": "DOF-iters/s (batched PCG, all instances in one graph launch)",
        "value": dofit / (sum(ms) / 1e3),
        "unit": "DOF-iters/s",
        "n_gpus": 1,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": statistics.mean(ms),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64 (outer PCG, operator) + " + ("f64" if args.batch_fp64 else "f32") + " (preconditioner)",
        "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD.format(n=len(meshes), r=n_rhs), "instances": bat.n_inst,
                   "total_dofs": bat.n_dofs, "l2": "vectors exceed L2 (no flush)"},
        "iters_min_median_max": [min(flat), statistics.median(flat), max(flat)],
        "setup_s": setup_s,
        "clocks": clk,
    }
    print(json.dumps(out))


def _oracle_setup(seed: int, coef: bool = False):
    from oracle import rhs, solver
    from paper_2009_01287_gb300 import inputs
    mesh, rh = inputs.config1_coeff(seed) if coef else inputs.config1(seed)
    prob = solver.build_problem(mesh)
    pc = solver.Preconditioner(prob, lor="amg")
    b = rhs.load_vector(prob.space, rh.amps, rh.waves)
    return prob, pc, b


def _oracle_step(prob, pc, b, iters: int) -> float:
    from oracle import solver
    t = time.perf_counter()
    solver.pcg(prob.A, b, pc.apply, 1e-30, iters)
    return time.perf_counter() - t


def cpu_baseline3(args):
    """The oracle on a bounded sample of the 3D workload: the same refinement
    and degree recipe on a 4^3 base (25k DOFs; the full 16^3 mesh is beyond the
    oracle's setup), FP64 PCG iterations, one thread."""
    prob, pc, b = _oracle_setup3(args.seed)
    dt = _oracle_step(prob, pc, b, ORACLE_SAMPLE_ITERS)
    return {"value": prob.space.n * ORACLE_SAMPLE_ITERS / dt, "unit": "DOF-iters/s", "cores": 1,
            "kind": "oracle",
            "sample": f"{ORACLE_SAMPLE_ITERS} FP64 PCG iterations on the same recipe with a 4^3 base "
                      f"({prob.space.n} DOFs; setup untimed), scipy sparse + numpy, one thread"}


def cpu_baseline(args, coef: bool = False):
    prob, pc, b = _oracle_setup(args.seed, coef)
    dt = _oracle_step(prob, pc, b, ORACLE_SAMPLE_ITERS)
    return {"value": prob.space.n * ORACLE_SAMPLE_ITERS / dt, "unit": "DOF-iters/s", "cores": 1,
            "kind": "oracle",
            "sample": f"{ORACLE_SAMPLE_ITERS} FP64 PCG iterations of the same workload "
                      f"(setup untimed), scipy sparse + numpy, one thread"}


def _oracle_setup3(seed: int):
    """The 3D recipe on a 4^3 base (the full 16^3 mesh is beyond the oracle's setup)."""
    from oracle import rhs, solver
    from paper_2009_01287_gb300 import inputs
    mesh, rh = inputs.config2(seed, base=4)
    prob = solver.build_problem(mesh, form="br2")
    pc = solver.Preconditioner(prob, lor="amg")
    b = rhs.load_vector(prob.space, rh.amps, rh.waves)
    return prob, pc, b


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    if args.workload in ("batched", "serving"):
        print(json.dumps({"impl": "reference", "unavailable": f"the oracle has no {args.workload} form; "
                          "its single-problem PCG is timed by the hp2d, hp2d-coef and hp3d workloads"}))
        return
    three = args.workload == "hp3d"
    coef = args.workload == "hp2d-coef"
    prob, pc, b = _oracle_setup3(args.seed) if three else _oracle_setup(args.seed, coef)
    for _ in range(args.warmup):
        _oracle_step(prob, pc, b, ORACLE_SAMPLE_ITERS)
    times = [_oracle_step(prob, pc, b, ORACLE_SAMPLE_ITERS) for _ in range(args.steps)]
    n = prob.space.n
    value = n * ORACLE_SAMPLE_ITERS * args.steps / sum(times)
    sample = f"{ORACLE_SAMPLE_ITERS} FP64 PCG iterations per step"
    if three:
        sample += f" on the same recipe with a 4^3 base ({n} DOFs)"
    out = {
        "impl": "reference",
        "metric": METRIC3 if three else (METRICC if coef else METRIC),
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
        "config": {"workload": WORKLOAD3 if three else (WORKLOADC if coef else WORKLOAD), "n_dofs": n},
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
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="hp2d", choices=["hp2d", "hp2d-coef", "hp3d", "batched", "serving"])
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-meshes", type=int, default=16)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--batch-problems", type=int, default=256)
    ap.add_argument("--batch-rhs", type=int, default=4)
    ap.add_argument("--batch-fp64", action="store_true")
    args = ap.parse_args()
    if args.workload == "batched" and args.impl == "ours":
        run_batched(args)
        return
    if args.workload == "serving" and args.impl == "ours":
        run_serving(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
