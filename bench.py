#!/usr/bin/env python
"""Throughput benchmark of the float64 modal DG solver (2D Euler, SSP-RK3).

Metric: DOF-updates/s per RK stage = N * N_p * 4 * 3 * steps / time, on the
256 x 256 jittered periodic mesh (131,072 triangles) at p = 3 with the isentropic
vortex.  One benchmark step = one SSP-RK3 time step (three right-hand sides and
stage updates) followed by the conserved-totals reduction, i.e. every row of the
hot path, on inputs already resident in HBM.  L2 is flushed (256 MiB write)
between timed steps, outside the timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision fp64|tf32x3|tf32x1] [--method ssp_rk3|rk2|rk4]
  python bench.py --configs     the five stated workloads, one JSON line each
  python bench.py --sweep       mesh-size scaling (RK4, p = 1 and 4, 200 to 184,832 elements;
                                p = 1 also with the limiter)
  python bench.py --case NAME   a few untimed steps of one workload, for a profiler

With N = 1 the line also carries the tensor-core modes on the same workload
(throughput, speedup over float64 and state error against the float64 run) and
the adjoint/forward cost ratio on the 256 x 256, p = 2 workload.

Under torchrun (N > 1) every rank runs an independent replica of the workload on
its own GPU (the path is replicated, not sharded): value = all ranks' DOF
updates / the slowest rank's time.  --impl reference times the CPU oracle on
the host cores (rank 0 only): on one thread (the line's value) and as one
independent replica per core (cpu_all_cores).

With N = 1 the headline line also carries mixed_512_p4: the mixed-precision
workload (512 x 512 mesh, p = 4, perturbed vortex) in float64 and both
tensor-core modes, steady-state over 100 steps, with the state error of each
mode against float64 and the tensor-core element kernel's HBM roofline.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF-updates/s per RK stage, FP64 vs mixed at stated err; adjoint/forward ratio"
UNIT = "DOF-updates/s"
WORKLOAD = dict(name="isentropic vortex, 256x256 jittered periodic triangle mesh "
                     "(131072 elements), p=3, 4-point Gauss edges, SSP-RK3, CFL 0.3",
                n=256, p=3, ne=0, cfl=0.3)


def flops_element_per_elem(p: int, ne: int) -> float:
    """Float64 flops of one element-kernel launch per element, for the algorithm
    the kernel executes (sum factorisation on the collapsed volume grid and on
    the edges), counting an FMA as 2 flops and a multiply or add as 1:
      W = chi c                          2 N_p (p+1) 4
      U = P W (the a = 0 term, P_0 = 1, is a copy)
                                         2 (p+1)^2 p 4;
        p >= 3: on the mirror pairs of the Gauss-Legendre nodes, the sums
        over the even and the odd a and their sum and difference, and for p
        even the middle node alpha = 0 (P_a(0) = 0 for odd a)
                                         (p+1) h 4 (2 p + 2) [+ (p+1) 4 p]
      per volume point: 1/rho (4 FMA Newton steps), pressure, the Euler flux
      along row 1 of J^tau (H_beta = G_s) and along row 0 + (1+alpha)/2 row 1
      (H_alpha = G_r + (1+alpha)/2 G_s)  38
      the directions of H_alpha (2 FMAs each): once per alpha node and element
      for p >= 3                         4 (p+1); p <= 2: 4 per point
      Xa, Xb (Xa(0, .) = 0 without arithmetic, P_0' = 0); at p = 2-4 folded on
      the mirror pairs of the Gauss-Legendre nodes: per (ib, variable) 4 h
      additions (h = floor((p+1)/2) pairs; at p >= 3 formed in the point phase)
      and T = (2p+1) h (+ p+1 for p even, the middle node) products
                                         (p+1) 4 (2 T + 4 h);
      p = 1: 2 (p+1)^2 (2p+1) 4; p = 5 (every a, on the pair sums and
      differences): 4 (p+1)^2 h 4 + 16 h (p+1)
      V = chiA Xa + dchiB Xb (modes with a = 0: the Xb term only)
                                         (4 (N_p - p - 1) + 2 (p+1)) (p+1) 4
      lift sums per variable (face 0: omega P_a; faces 1, 2: F1 +/- F2)
                                         (2 (p+1) n_e + 2 n_e) 4
      lift per mode                      2 (1 + n_e) N_p 4
      stage update                       5 N_p 4
      next traces (face 0 from Z_a = sum_b chi_ab(-1) c_ab, then Z_0 +
      sum_{a>=1} P_a Z_a; faces 1, 2 from the sums over the modes of even and of
      odd first index, the constant mode's term chi_00 c_00 formed once)
                                         (2 N_p + 1 + n_e (2 p + 2 N_p)) 4"""
    NP = (p + 1) * (p + 2) // 2
    ND = p + 1
    h = ND // 2
    if 2 <= p <= 4:
        T = (2 * ND - 1) * h + (ND if ND % 2 else 0)
        x_phase = ND * 4 * (2 * T + 4 * h)
    elif p == 1:
        x_phase = 2 * ND * ND * (2 * ND - 1) * 4
    else:
        x_phase = 4 * ND * ND * h * 4 + 16 * h * ND
    if p >= 3:
        u_phase = ND * h * 4 * (2 * p + 2) + (ND * 4 * 2 * (p // 2) if ND % 2 else 0)
    else:
        u_phase = 2 * ND * ND * p * 4
    dirs = 4 * ND if p >= 3 else 4 * ND * ND
    return (2 * NP * ND * 4 + u_phase + 38 * ND * ND + dirs + x_phase + (4 * (NP - ND) + 2 * ND) * ND * 4
            + (2 * ND * ne + 2 * ne) * 4 + 2 * (1 + ne) * NP * 4 + 5 * NP * 4 + (2 * NP + 1 + ne * (2 * p + 2 * NP)) * 4)


def flops_element_direct_per_elem(p: int, ne: int, nq: int) -> float:
    """The same for the direct form on a rule of nq points (the symmetric
    rules): U = Phi c 2 nq N_p 4, per point 38 (the flux without H_alpha),
    V = Dr G_r + Ds G_s 4 nq N_p 4, the lift, update and traces as above."""
    NP = (p + 1) * (p + 2) // 2
    ND = p + 1
    return (2 * nq * NP * 4 + 38 * nq + 4 * nq * NP * 4
            + (2 * ND * ne + 2 * ne) * 4 + 2 * (1 + ne) * NP * 4 + 5 * NP * 4 + (2 * NP + 1 + ne * (2 * p + 2 * NP)) * 4)


def bytes_element_tc_per_elem(p: int, ne: int) -> float:
    """Algorithmic HBM bytes of one mixed-precision element-kernel launch per
    element, averaged over the three stages: stage input 8*4*N_p, u^n in two of
    three stages, the gathers of the three edges' float32 fluxes 4*4*3n_e and
    their float64 mean-mode integrals 3*4*8, geometry 64 B + face map 12 B, new
    state 8*4*N_p, new float32 traces 4*4*3n_e."""
    NP = (p + 1) * (p + 2) // 2
    NF = 3 * ne
    return 32 * NP + (2.0 / 3.0) * 32 * NP + 16 * NF + 96 + 76 + 32 * NP + 16 * NF


def hbm_peak():
    """Measured HBM copy bandwidth (GB/s) of the GB300s, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (measured copy)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def _src_hash(*names) -> str:
    """Hash of the code of the named sources with comments and blank lines taken
    out (a comment edit leaves the compiled kernel, and its traffic, as it was)."""
    import re
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_1601_07944_gb300", "csrc", n)) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        src = "\n".join(line.rstrip() for line in src.splitlines() if line.strip())
        h.update(src.encode())
    return h.hexdigest()[:16]


# DRAM bytes per launch of the element kernel (dram__bytes_read.sum +
# dram__bytes_write.sum) from one ncu capture, keyed by the hash of the code of
# the kernel's source files (dg_element.cu and the device headers, comments
# aside) it was taken on, and the volume rule when it is not the collapsed grid;
# a code change voids the entry.
TRAFFIC = {
    # k_element_sf<3,4,0>, stage-2 launch (reads u^n), 256x256 p=3 vortex (one ncu capture)
    "d9a87cb5b2bffedf": 119098624 + 43275520,
}


# Float64 thread instructions per element of one element-kernel launch
# (DFMA + DMUL + DADD: sm__sass_thread_inst_executed_op_d{fma,mul,add}_pred_on.sum
# over the elements) from one ncu capture, keyed like TRAFFIC.  The float64 pipe
# takes an FMA, a multiply or an add in the same issue slot, so these against
# the pipe's FMA rate (half the flop peak) tell how full the kernel keeps the
# pipe, whatever its mix of FMAs and single operations.
FP64_INST = {
    # k_element_sf<3,4,0>, stage-2 launch, 256x256 p=3 vortex: 1,512 DFMA + 289.2 DMUL
    # + 240.6 DADD per element (the stage-1 launch, without u^n, has 40 fewer)
    "d9a87cb5b2bffedf": 1512.0 + 289.1875 + 240.59375,
}


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _gpu_id_for_smi(local_rank: int) -> str:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return str(local_rank)


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


STAGES = {"ssp_rk3": 3, "rk2": 2, "rk4": 4}


def _dof_per_step(N: int, p: int, method: str = "ssp_rk3") -> int:
    """DOF updates of one time step: every stage updates all N N_p 4 unknowns."""
    return N * (p + 1) * (p + 2) // 2 * 4 * STAGES[method]


def slowest_rank_ms(ms: float, world: int, device: str = "cuda") -> float:
    """The timed region's duration of the slowest rank (all ranks call this)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as tdist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(dof_per_step_per_rank: int, steps: int, t_max_ms: float, world: int) -> float:
    """DOF updates per second of the whole job: every rank's replica advanced the
    same workload, and the job took as long as its slowest rank."""
    return world * dof_per_step_per_rank * steps / (t_max_ms * 1e-3)


def run_reference(args, world, rank):
    """The CPU oracle, as it stands, on a bounded sample of the workload."""
    if rank != 0:
        return
    import numpy as np  # noqa: F401

    import oracle
    from paper_1601_07944_gb300 import inputs as I
    oracle.build()
    p = WORKLOAD["p"]
    # calibrate on a 64x64 mesh of the same structure and order, then size the
    # sample so that warm-up + timed steps take about a minute
    n = 64
    mesh = I.periodic_mesh(n)
    o = oracle.OracleDG.from_mesh(mesh, p, n_edge_pts=WORKLOAD["ne"])
    c = o.project_ic(I.vortex)
    dt = I.fixed_dt(I.periodic_mesh(WORKLOAD["n"]), I.vortex, p, WORKLOAD["cfl"])
    t = time.perf_counter(); o.ssp_rk3(c, dt, 1); t1 = time.perf_counter() - t
    budget = 60.0
    per_elem_step = t1 / mesh.n_elem
    steps = args.steps + args.warmup
    while n < WORKLOAD["n"] and 4 * (2 * n * n) * per_elem_step * steps < budget:
        n *= 2
    mesh = I.periodic_mesh(n)
    o = oracle.OracleDG.from_mesh(mesh, p, n_edge_pts=WORKLOAD["ne"])
    c = o.project_ic(I.vortex)
    for _ in range(args.warmup):
        c = o.ssp_rk3(c, dt, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        c = o.ssp_rk3(c, dt, 1)
    el = time.perf_counter() - t0
    value = _dof_per_step(mesh.n_elem, p) * args.steps / el
    sample = ("oracle SSP-RK3 steps of the same vortex at p=3 on a %dx%d mesh (%d elements) of "
              "the same construction, 1 thread" % (n, n, mesh.n_elem))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded jittered periodic mesh, isentropic vortex)",
        "config": {"workload": WORKLOAD["name"], "sample": sample, "precision": "fp64"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        # the same oracle on every host core (one independent replica per core)
        "cpu_all_cores": cpu_all_cores(n, seconds=10.0),
    }
    print(json.dumps(line), flush=True)


def _oracle_worker(n, p, ne, cfl, vol_rule, seconds, q):
    """One replica of the oracle in its own process: whole SSP-RK3 steps of the
    n x n vortex workload for about `seconds`; puts (steps, elapsed) on q."""
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1601_07944_gb300 import inputs as I
    mesh = I.periodic_mesh(n)
    o = oracle.OracleDG.from_mesh(mesh, p, n_edge_pts=ne, vol_rule=vol_rule)
    c = o.project_ic(I.vortex)
    dt = I.fixed_dt(mesh, I.vortex, p, cfl)
    q.put("ready")
    steps, el = 0, 0.0
    while el < seconds or steps == 0:
        t = time.perf_counter()
        c = o.ssp_rk3(c, dt, 1)
        el += time.perf_counter() - t
        steps += 1
    q.put((steps, el))


def cpu_all_cores(n: int, seconds: float = 8.0, vol_rule: str = "collapsed"):
    """The oracle as it stands (single-threaded C) run as one independent replica
    per host core, in spawned processes (a process forked after the first CUDA call
    could hang): the whole host's throughput on the n x n workload, DOF-updates/s
    summed over the replicas, each timed over its own steps."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(n, WORKLOAD["p"], WORKLOAD["ne"], WORKLOAD["cfl"], vol_rule,
                                                       seconds, q)) for _ in range(cores)]
    for pr in procs:
        pr.start()
    got, ready = [], 0
    while len(got) < cores:
        item = q.get(timeout=600)
        if item == "ready":
            ready += 1
        else:
            got.append(item)
    for pr in procs:
        pr.join(timeout=60)
    dof = _dof_per_step(2 * n * n, WORKLOAD["p"])
    value = sum(dof * st / el for st, el in got)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d independent replicas (one per host core, spawned processes) of the single-threaded "
                      "oracle, each %d-%d whole SSP-RK3 steps of the %dx%d p=%d vortex (%s volume rule), "
                      "about %.0f s each" % (cores, min(g[0] for g in got), max(g[0] for g in got), n, n,
                                             WORKLOAD["p"], vol_rule, seconds)}


def cpu_baseline(seconds: float = 12.0, vol_rule: str = "collapsed"):
    """The oracle on the full workload mesh for as many whole steps as fit in about
    `seconds` (at least one), single-threaded."""
    import oracle
    from paper_1601_07944_gb300 import inputs as I
    oracle.build()
    mesh = I.periodic_mesh(WORKLOAD["n"])
    p = WORKLOAD["p"]
    o = oracle.OracleDG.from_mesh(mesh, p, n_edge_pts=WORKLOAD["ne"], vol_rule=vol_rule)
    c = o.project_ic(I.vortex)
    dt = I.fixed_dt(mesh, I.vortex, p, WORKLOAD["cfl"])
    steps, el = 0, 0.0
    while el < seconds or steps == 0:
        t = time.perf_counter()
        c = o.ssp_rk3(c, dt, 1)
        el += time.perf_counter() - t
        steps += 1
    return {"value": _dof_per_step(mesh.n_elem, p) * steps / el, "unit": UNIT, "cores": 1,
            "kind": "oracle",
            "sample": "%d full SSP-RK3 step(s) of the 256x256 p=3 workload (%s volume rule) on 1 host "
                      "thread (%.1f s)" % (steps, vol_rule, el)}


def mixed_modes(m, c0, dt, steps, flush, fp64_ms_per_step):
    """Throughput of the tensor-core modes on the same workload and their state
    error against the float64 GPU run after the same number of steps."""
    import numpy as np
    import torch
    stream = torch.cuda.current_stream()
    ref = c0.clone()
    m.rk_step(ref, dt, steps, precision="fp64")
    out = {}
    for prec in ("tf32x3", "tf32x1"):
        c = c0.clone()
        for _ in range(3):
            m.rk_step(c, dt, 1, precision=prec)
        torch.cuda.synchronize()
        ms = 0.0
        for _ in range(steps):
            flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
            a.record(stream); m.rk_step(c, dt, 1, precision=prec); m.conserved_totals(c); b.record(stream)
            torch.cuda.synchronize()
            ms += a.elapsed_time(b)
        m.device_status()
        x = c0.clone()
        m.rk_step(x, dt, steps, precision=prec)
        R, X = ref.cpu().numpy(), x.cpu().numpy()
        out[prec] = {"value": _dof_per_step(m.N, m.p) * steps / (ms * 1e-3), "ms_per_step": ms / steps,
                     "speedup_vs_fp64": fp64_ms_per_step / (ms / steps),
                     "rel_l2_vs_fp64": float(np.linalg.norm(X - R) / np.linalg.norm(R)),
                     "error_after_steps": steps}
    return out


def mixed_config3(steps: int = 100):
    """The mixed-precision workload as stated: the perturbed vortex on the 512x512
    mesh (524,288 elements) at p = 4, SSP-RK3.  For float64, 3xTF32 and 1xTF32: the
    steady-state rate over `steps` steps in one call (CUDA-graph replay; the
    252 MB state and its work arrays exceed L2, so nothing is flushed), the state
    error of each tensor-core mode against the float64 run after the same steps,
    and the per-launch times of the element and edge kernels from the library's
    CUDA events over 5 plain steps; for the tensor-core modes the element kernel's
    roofline against the measured HBM copy rate (algorithmic bytes per launch,
    bytes_element_tc_per_elem)."""
    import torch
    from paper_1601_07944_gb300 import dg, inputs as I
    n, p = 512, 4
    mesh = I.periodic_mesh(n)
    m = dg.Mesh.from_mesh(mesh, p)
    dt = I.fixed_dt(mesh, I.perturbed_vortex, p)
    c0 = m.project_function(I.perturbed_vortex)
    hbm, src = hbm_peak()
    out = {"workload": "perturbed vortex (Fourier perturbations 1e-2, wavenumbers 1-4), 512x512 jittered "
                       "periodic mesh (524288 elements), p=4, 5-point Gauss edges, SSP-RK3",
           "steps": steps, "timing": "one %d-step call (CUDA-graph replay), CUDA events; inputs exceed L2" % steps}
    ref = None
    fp64_ms = None
    for prec in ("fp64", "tf32x3", "tf32x1"):
        c = c0.clone()
        m.rk_step(c, dt, 17, precision=prec)                       # capture + warm the graph
        c = c0.clone()
        a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(); a.record()
        m.rk_step(c, dt, steps, precision=prec)
        b.record(); torch.cuda.synchronize()
        m.device_status()
        ms = a.elapsed_time(b) / steps
        if ref is None:
            ref, fp64_ms = c.clone(), ms
        w = c0.clone()
        m.set_timing(True)
        m.rk_step(w, dt, 5, precision=prec)
        kt = m.kernel_times()
        m.set_timing(False)
        el_n, el_ms = kt.get("element", (1, 0.0))
        fa_n, fa_ms = kt.get("face", (1, 0.0))
        rec = {"value": _dof_per_step(m.N, p) * steps / (ms * steps * 1e-3), "unit": UNIT, "ms_per_step": ms,
               "element_ms_per_launch": el_ms / el_n, "face_ms_per_launch": fa_ms / fa_n}
        if prec != "fp64":
            nbytes = bytes_element_tc_per_elem(p, m.ne) * m.N
            ach = nbytes / (el_ms / el_n * 1e-3) / 1e9
            rec.update({"speedup_vs_fp64": fp64_ms / ms,
                        "rel_l2_vs_fp64": float(torch.linalg.norm(c - ref) / torch.linalg.norm(ref)),
                        "error_after_steps": steps,
                        "roofline": {"bound": "hbm", "kernel": "k_element_tc (tcgen05, %s)" % prec,
                                     "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                                     "traffic": None, "peak_source": src, "bytes_per_launch": nbytes,
                                     "avg_launch_ms": el_ms / el_n}})
        out[prec] = rec
    del m
    return out


def paper_steppers(m, c0, dt, steps, flush):
    """Float64 throughput of the paper's own integrators (classic RK2 read as
    Heun's method, and RK4) on the same workload, per RK stage as the headline."""
    import torch
    stream = torch.cuda.current_stream()
    out = {}
    for method in ("rk2", "rk4"):
        c = c0.clone()
        for _ in range(3):
            m.rk_step(c, dt, 1, method=method)
        torch.cuda.synchronize()
        ms = 0.0
        for _ in range(steps):
            flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
            a.record(stream); m.rk_step(c, dt, 1, method=method); m.conserved_totals(c); b.record(stream)
            torch.cuda.synchronize()
            ms += a.elapsed_time(b)
        m.device_status()
        out[method] = {"value": _dof_per_step(m.N, m.p, method) * steps / (ms * 1e-3),
                       "stages": STAGES[method], "ms_per_step": ms / steps}
    return out


def run_sweep(precisions=("fp64",)):
    """Mesh-size scaling in the manner of the paper's scaling runs (Section 7.1:
    p = 1 for 10,000 steps and p = 4 for 1,000 steps, RK4, on meshes of 180 to
    184,320 elements): jittered periodic meshes of 200 to 184,832 elements, the
    perturbed vortex, classical RK4, device-timed whole runs (CUDA graphs).  At
    p = 1 the float64 runs are repeated with every stage limited (Section 7.2:
    the limiter's cost)."""
    import torch
    from paper_1601_07944_gb300 import _build, dg, inputs as I
    _build.build()
    dg.load()
    for p, steps in ((1, 10000), (4, 1000)):
        for n in (10, 20, 40, 80, 152, 160, 304):
            mesh = I.periodic_mesh(n)
            m = dg.Mesh.from_mesh(mesh, p)
            dt = I.fixed_dt(mesh, I.perturbed_vortex, p)
            c0 = m.project_function(I.perturbed_vortex)
            runs = [(prec, False) for prec in precisions]
            if p == 1 and "fp64" in precisions:
                runs.append(("fp64", True))
            for prec, limited in runs:
                m.set_limiter(limited)
                c = c0.clone()
                if limited:
                    m.limit(c)
                m.rk_step(c, dt, 17, precision=prec, method="rk4")     # capture + warm the graph
                a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize(); a.record()
                m.rk_step(c, dt, steps, precision=prec, method="rk4")
                b.record(); torch.cuda.synchronize()
                m.device_status()
                ms = a.elapsed_time(b)
                print(json.dumps({"sweep": "mesh size", "method": "rk4", "p": p, "n": n, "n_elem": m.N,
                                  "precision": prec, "limiter": limited, "steps": steps, "time_s": ms * 1e-3,
                                  "ms_per_step": ms / steps,
                                  "dof_updates_per_s": _dof_per_step(m.N, p, "rk4") * steps / (ms * 1e-3)}),
                      flush=True)
            m.set_limiter(False)
            if n == 152:
                # the paper's kernel runtime distribution of an RK4 step (its mesh E,
                # 46,080 elements): per-kernel CUDA-event times (plain launches, no graph)
                c = c0.clone()
                m.set_timing(True)
                m.rk_step(c, dt, 100, method="rk4")
                kt = m.kernel_times()
                m.set_timing(False)
                tot = sum(ms for _, ms in kt.values())
                print(json.dumps({"sweep": "kernel time split", "method": "rk4", "p": p, "n_elem": m.N,
                                  "steps": 100, "ms_per_step": tot / 100,
                                  "share": {k: round(ms / tot, 4) for k, (_, ms) in kt.items()}}), flush=True)
            del m
    # the kind of run behind the paper's only absolute throughput figures (its
    # double Mach reflection table: p = 1, classic RK2, Barth-Jespersen limiter on
    # 68,622 / 236,964 / 964,338 elements): here on jittered periodic meshes of
    # about those sizes with discontinuous data (density_steps), every stage limited
    for n, steps in ((185, 2000), (344, 1000), (694, 400)):
        mesh = I.periodic_mesh(n)
        m = dg.Mesh.from_mesh(mesh, 1)
        dt = I.fixed_dt(mesh, I.density_steps, 1)
        c = m.project_function(I.density_steps)
        m.set_limiter(True)
        m.limit(c)
        m.rk_step(c, dt, 17, method="rk2")
        a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(); a.record()
        m.rk_step(c, dt, steps, method="rk2")
        b.record(); torch.cuda.synchronize()
        m.device_status()
        ms = a.elapsed_time(b)
        print(json.dumps({"sweep": "p=1 RK2 limited (the paper's DMR kind of run)", "method": "rk2", "p": 1,
                          "n": n, "n_elem": m.N, "precision": "fp64", "limiter": True, "steps": steps,
                          "time_s": ms * 1e-3, "ms_per_step": ms / steps,
                          "dof_updates_per_s": _dof_per_step(m.N, 1, "rk2") * steps / (ms * 1e-3)}),
              flush=True)
        del m


def vortex_error(steps: int = 200):
    """The 256x256, p=3 workload as stated: 200 float64 SSP-RK3 steps from the
    vortex, then the L2 density error against the exact translated vortex."""
    import torch
    from paper_1601_07944_gb300 import dg, inputs as I
    mesh = I.periodic_mesh(WORKLOAD["n"])
    p = WORKLOAD["p"]
    m = dg.Mesh.from_mesh(mesh, p, n_edge_pts=WORKLOAD["ne"])
    c = m.project_function(I.vortex)
    dt = I.fixed_dt(mesh, I.vortex, p, WORKLOAD["cfl"])
    e0 = m.l2_error(c, lambda x, y: I.vortex(x, y, 0.0))
    m.rk_step(c, dt, steps)
    t = steps * dt
    e1 = m.l2_error(c, lambda x, y: I.vortex(x, y, t))
    return {"steps": steps, "final_time": t, "l2_density_error": e1, "l2_density_error_t0": e0,
            "note": "the vortex is not exactly periodic on [-5,5]^2 (velocity perturbation ~2.4e-5 "
                    "at the seams); part of the error comes from there"}


def adjoint_ratio(steps: int = 20, every: int = 10):
    """Cost of the discrete adjoint relative to the forward pass on the 256x256,
    p=2 differentiation workload: one dg_adjoint_step (stages recomputed) and one
    dg_adjoint_step_stages (stages given) against one dg_rk_step, and the
    checkpointed backward (recomputation included, stage values kept, the
    default) against its forward, and the same backward recomputing the stages."""
    import torch
    from paper_1601_07944_gb300 import autograd as AG, dg, inputs as I
    mesh = I.periodic_mesh(256)
    p = 2
    m = dg.Mesh.from_mesh(mesh, p)
    c0 = m.project_function(I.perturbed_vortex)
    dt = I.fixed_dt(mesh, I.perturbed_vortex, p)
    lam = torch.randn_like(c0)
    out = torch.empty_like(c0)
    c = c0.clone()
    m.rk_step(c, dt, 2); m.adjoint_step(c0, dt, lam, out=out)
    torch.cuda.synchronize()
    u1, u2 = torch.empty_like(c0), torch.empty_like(c0)
    m.rk_step_stages(c0.clone(), dt, u1, u2)
    m.adjoint_step_stages(c0, u1, u2, dt, lam, out=out)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record(); m.rk_step(c, dt, steps); e[1].record()
    for _ in range(steps):
        m.adjoint_step(c0, dt, lam, out=out)
    e[2].record()
    for _ in range(steps):
        m.adjoint_step_stages(c0, u1, u2, dt, lam, out=out)
    e[3].record(); torch.cuda.synchronize()
    fwd, adj, adj_s = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3])
    dJ = m.det_j()
    tgt = c0.clone()
    ratio = {}
    for keep in (True, False):
        for rep in range(2):                   # the first pass warms up torch's autograd path
            x = c0.clone().requires_grad_(True)
            torch.cuda.synchronize(); t0 = time.perf_counter()
            cT = AG.solve(m, x, dt, steps, every, keep_stages=keep)
            loss = AG.density_misfit(dJ, cT, tgt)
            torch.cuda.synchronize(); t1 = time.perf_counter()
            loss.backward()
            torch.cuda.synchronize(); t2 = time.perf_counter()
        ratio[keep] = (t2 - t1) / (t1 - t0)
    return {"workload": "perturbed vortex, 256x256 mesh, p=2, %d steps, checkpoint every %d" % (steps, every),
            "adjoint_step_over_rk_step": adj / fwd,
            "adjoint_step_stages_given_over_rk_step": adj_s / fwd,
            "backward_over_forward_with_recompute": ratio[True],
            "backward_over_forward_recomputing_stages": ratio[False],
            "rk_step_ms": fwd / steps, "adjoint_step_ms": adj / steps, "adjoint_step_stages_given_ms": adj_s / steps}


def run_rules(n: int = 256, steps: int = 100):
    """The two volume rules side by side (the collapsed (p+1)^2 grid and the
    symmetric degree-2p rule with the paper's point counts, Sections 4.3.2, 6.1): the
    perturbed vortex on the n x n mesh, p = 1..5, SSP-RK3, every precision,
    device-timed whole runs (CUDA graphs), plus the element kernel's time per
    launch from per-kernel events over 5 plain steps and the state difference
    between the rules after the run (float64)."""
    import torch
    from paper_1601_07944_gb300 import _build, dg, inputs as I
    _build.build()
    dg.load()
    mesh = I.periodic_mesh(n)
    for p in (1, 2, 3, 4, 5):
        dt = I.fixed_dt(mesh, I.perturbed_vortex, p)
        finals = {}
        for rule in ("collapsed", "symmetric"):
            m = dg.Mesh.from_mesh(mesh, p, vol_rule=rule)
            c0 = m.project_function(I.perturbed_vortex)
            for prec in ("fp64", "tf32x3", "tf32x1"):
                c = c0.clone()
                m.rk_step(c, dt, 17, precision=prec)                   # capture + warm the graph
                c = c0.clone()
                a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize(); a.record()
                m.rk_step(c, dt, steps, precision=prec)
                b.record(); torch.cuda.synchronize()
                m.device_status()
                ms = a.elapsed_time(b)
                if prec == "fp64":
                    finals[rule] = c
                w = c0.clone()
                m.set_timing(True)
                m.rk_step(w, dt, 5, precision=prec)
                kt = m.kernel_times()
                m.set_timing(False)
                el_n, el_ms = kt.get("element", (0, 0.0))
                line = {"rules": "volume rule", "p": p, "n_elem": m.N, "vol_rule": rule, "n_vol_pts": m.nq,
                        "precision": prec, "steps": steps, "ms_per_step": ms / steps,
                        "dof_updates_per_s": _dof_per_step(m.N, p) * steps / (ms * 1e-3),
                        "element_ms_per_launch": el_ms / max(1, el_n)}
                if prec == "fp64":
                    fl = (flops_element_direct_per_elem(p, m.ne, m.nq) if rule == "symmetric"
                          else flops_element_per_elem(p, m.ne)) * m.N
                    line["element_fp64_tflops"] = fl / (line["element_ms_per_launch"] * 1e-3) / 1e12
                print(json.dumps(line), flush=True)
            del m
        d = float(torch.linalg.norm(finals["symmetric"] - finals["collapsed"]) / torch.linalg.norm(finals["collapsed"]))
        print(json.dumps({"rules": "state difference", "p": p, "steps": steps,
                          "rel_l2_symmetric_vs_collapsed_fp64": d}), flush=True)


def run_case(name: str):
    """A few steps of one workload, untimed, for a profiler to capture: `mixed`
    (3xTF32, 256x256, p=3, vortex), `mixed512` (3xTF32, 512x512, p=4, perturbed
    vortex), `limiter` (float64 RK4 with every stage limited, 304x304, p=1,
    perturbed vortex), `adjoint` (two dg_adjoint_step calls, 256x256, p=2), `small`
    (the fused small-mesh stepper: two float64 RK4 calls of 100 steps each,
    10x10 (200 elements), p=1, perturbed vortex)."""
    import torch
    from paper_1601_07944_gb300 import _build, dg, inputs as I
    _build.build()
    dg.load()
    if name in ("mixed", "mixed512"):
        n, p, ic = (256, 3, I.vortex) if name == "mixed" else (512, 4, I.perturbed_vortex)
        mesh = I.periodic_mesh(n)
        m = dg.Mesh.from_mesh(mesh, p)
        c = m.project_function(ic)
        dt = I.fixed_dt(mesh, ic, p)
        for _ in range(2):
            m.rk_step(c, dt, 1, precision="tf32x3")
    elif name == "limiter":
        mesh = I.periodic_mesh(304)
        m = dg.Mesh.from_mesh(mesh, 1)
        dt = I.fixed_dt(mesh, I.perturbed_vortex, 1)
        c = m.project_function(I.perturbed_vortex)
        m.set_limiter(True)
        m.limit(c)
        for _ in range(3):
            m.rk_step(c, dt, 1, method="rk4")
    elif name == "adjoint":
        mesh = I.periodic_mesh(256)
        m = dg.Mesh.from_mesh(mesh, 2)
        dt = I.fixed_dt(mesh, I.perturbed_vortex, 2)
        c = m.project_function(I.perturbed_vortex)
        lam = m.project_function(lambda x, y: I.perturbed_vortex(x, y, seed=I.SEED_TARGET))
        out = torch.empty_like(c)
        for _ in range(2):
            m.adjoint_step(c, dt, lam, out=out)
    elif name == "small":
        mesh = I.periodic_mesh(10)
        m = dg.Mesh.from_mesh(mesh, 1)
        dt = I.fixed_dt(mesh, I.perturbed_vortex, 1)
        c = m.project_function(I.perturbed_vortex)
        for _ in range(2):
            m.rk_step(c, dt, 100, method="rk4")
    else:
        raise SystemExit("unknown case %r" % name)
    torch.cuda.synchronize()
    m.device_status()
    print(json.dumps({"case": name, "ok": True}), flush=True)


def run_configs():
    """Every workload of the five configurations as stated, one JSON line each
    (device-timed full runs; parity with the oracle is the tests' job)."""
    import numpy as np
    import torch
    from paper_1601_07944_gb300 import _build, autograd as AG, dg, inputs as I
    _build.build()
    dg.load()

    def timed_run(m, c, dt, steps, prec, chunk=None):
        chunk = chunk or steps
        a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(); a.record()
        done = 0
        while done < steps:
            k = min(chunk, steps - done)
            m.rk_step(c, dt, k, precision=prec)
            done += k
        b.record(); torch.cuda.synchronize()
        m.device_status()
        return a.elapsed_time(b)

    def emit(d):
        print(json.dumps(d), flush=True)

    precs = ("fp64", "tf32x3", "tf32x1")
    # 1: 16^2, p=1, vortex, 100 steps
    mesh = I.periodic_mesh(16); m = dg.Mesh.from_mesh(mesh, 1)
    dt = I.fixed_dt(mesh, I.vortex, 1)
    c0 = m.project_function(I.vortex); t0 = m.conserved_totals(c0)
    c = c0.clone(); timed_run(m, c, dt, 100, "fp64")
    c = c0.clone(); ms = timed_run(m, c, dt, 100, "fp64")
    emit({"config": 1, "workload": "vortex 16x16 (512 elements), p=1, 100 steps", "precision": "fp64",
          "ms_per_step": ms / 100, "dof_updates_per_s": _dof_per_step(m.N, 1) * 100 / (ms * 1e-3),
          "totals_rel_drift": (np.abs(m.conserved_totals(c) - t0) / np.abs(t0)).tolist(),
          "l2_density_error_vs_exact": m.l2_error(c, lambda x, y: I.vortex(x, y, 100 * dt))})
    # 2: 256^2, p=3, vortex, 200 steps, 4 and 3 edge points
    for ne in (0, 3):
        mesh = I.periodic_mesh(256); m = dg.Mesh.from_mesh(mesh, 3, n_edge_pts=ne)
        dt = I.fixed_dt(mesh, I.vortex, 3)
        c0 = m.project_function(I.vortex)
        ref = None
        for prec in precs:
            c = c0.clone(); timed_run(m, c, dt, 3, prec)
            c = c0.clone(); ms = timed_run(m, c, dt, 200, prec)
            if ref is None:
                ref = c.clone()
            emit({"config": 2, "workload": "vortex 256x256 (131072 elements), p=3, %d edge points, 200 steps"
                  % m.ne, "precision": prec, "ms_per_step": ms / 200,
                  "dof_updates_per_s": _dof_per_step(m.N, 3) * 200 / (ms * 1e-3),
                  "rel_l2_vs_fp64": float(torch.linalg.norm(c - ref) / torch.linalg.norm(ref)),
                  "l2_density_error_vs_exact": m.l2_error(c, lambda x, y: I.vortex(x, y, 200 * dt))})
        del m
    # 3: 512^2, p=4, perturbed vortex
    mesh = I.periodic_mesh(512); m = dg.Mesh.from_mesh(mesh, 4)
    dt = I.fixed_dt(mesh, I.perturbed_vortex, 4)
    c0 = m.project_function(I.perturbed_vortex)
    ref = None
    for prec in precs:
        c = c0.clone(); timed_run(m, c, dt, 3, prec)
        c = c0.clone(); ms = timed_run(m, c, dt, 100, prec)
        if ref is None:
            ref = c.clone()
        emit({"config": 3, "workload": "perturbed vortex 512x512 (524288 elements), p=4, 100 steps",
              "precision": prec, "ms_per_step": ms / 100,
              "dof_updates_per_s": _dof_per_step(m.N, 4) * 100 / (ms * 1e-3),
              "rel_l2_vs_fp64": float(torch.linalg.norm(c - ref) / torch.linalg.norm(ref))})
    del m
    # 4: 256^2, p=2, 400 steps, checkpoint every 20: forward vs checkpointed backward
    mesh = I.periodic_mesh(256); m = dg.Mesh.from_mesh(mesh, 2)
    dt = I.fixed_dt(mesh, I.perturbed_vortex, 2)
    c0 = m.project_function(I.perturbed_vortex)
    tgt = m.project_function(lambda x, y: I.perturbed_vortex(x, y, seed=I.SEED_TARGET))
    m.rk_step(tgt, dt, 400)
    dJ = m.det_j()
    for rep in range(2):
        x = c0.clone().requires_grad_(True)
        torch.cuda.synchronize(); w0 = time.perf_counter()
        loss = AG.density_misfit(dJ, AG.solve(m, x, dt, 400, 20), tgt)
        torch.cuda.synchronize(); w1 = time.perf_counter()
        loss.backward()
        torch.cuda.synchronize(); w2 = time.perf_counter()
    emit({"config": 4, "workload": "perturbed vortex 256x256, p=2, 400 steps, checkpoint every 20",
          "precision": "fp64", "forward_s": w1 - w0, "backward_s": w2 - w1,
          "backward_over_forward": (w2 - w1) / (w1 - w0), "loss": float(loss.item())})
    del m
    # 5: 1024^2, p=5, perturbed vortex, 100 steps: throughput and totals drift
    mesh = I.periodic_mesh(1024); m = dg.Mesh.from_mesh(mesh, 5)
    dt = I.fixed_dt(mesh, I.perturbed_vortex, 5)
    c0 = m.project_function(I.perturbed_vortex); t0 = m.conserved_totals(c0)
    ref = None
    for prec in precs:
        c = c0.clone(); timed_run(m, c, dt, 2, prec)
        c = c0.clone()
        m.set_timing(True)
        ms = timed_run(m, c, dt, 100, prec)
        kt = m.kernel_times(); m.set_timing(False)
        if ref is None:
            ref = c.clone()
        line = {"config": 5, "workload": "perturbed vortex 1024x1024 (2097152 elements, 176M DOF), p=5, 100 steps",
                "precision": prec, "ms_per_step": ms / 100,
                "dof_updates_per_s": _dof_per_step(m.N, 5) * 100 / (ms * 1e-3),
                "totals_rel_drift": (np.abs(m.conserved_totals(c) - t0) / np.abs(t0)).tolist(),
                "rel_l2_vs_fp64": float(torch.linalg.norm(c - ref) / torch.linalg.norm(ref)),
                "kernel_ms_per_launch": {k: v[1] / v[0] for k, v in kt.items()}}
        if prec != "fp64":
            el_ms = kt["element"][1] / kt["element"][0]
            hbm, _ = hbm_peak()
            line["element_hbm_frac"] = bytes_element_tc_per_elem(5, 6) * m.N / (el_ms * 1e-3) / 1e9 / hbm
        emit(line)


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    from paper_1601_07944_gb300 import _build, dg, inputs as I

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    dg.load()

    def barrier():
        if world > 1:
            import torch.distributed as tdist
            tdist.barrier()

    p, ne = WORKLOAD["p"], WORKLOAD["ne"]
    method = args.method
    mesh = I.periodic_mesh(WORKLOAD["n"])
    m = dg.Mesh.from_mesh(mesh, p, n_edge_pts=ne, vol_rule=args.vol_rule)
    ne = m.ne
    c = m.project_function(I.vortex)
    dt = I.fixed_dt(mesh, I.vortex, p, WORKLOAD["cfl"])
    dof_step = _dof_per_step(m.N, p, method)
    stream = torch.cuda.current_stream()

    fp64_peak, fp32_peak = dg.probe_fma_rate()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    prec = args.precision
    for _ in range(args.warmup):
        m.rk_step(c, dt, 1, precision=prec, method=method)
        m.conserved_totals(c)
    torch.cuda.synchronize()

    clocks = ClockSampler(_gpu_id_for_smi(local))
    clocks.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    m.set_timing(True)
    barrier()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    totals = None
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        starts[i].record(stream)
        m.rk_step(c, dt, 1, precision=prec, method=method)
        totals = m.conserved_totals(c)
        ends[i].record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - w0
    clk = clocks.stop()
    ktimes = m.kernel_times()
    m.set_timing(False)
    dev_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))

    t_max = slowest_rank_ms(dev_ms, world, "cuda")
    value = whole_job_value(dof_step, args.steps, t_max, world)

    # end to end through the host-buffer entry point: H2D, step, D2H every step
    e2e_steps = max(1, min(args.steps, 20))
    h = torch.empty(m.coef_shape, dtype=torch.float64).pin_memory()
    h.copy_(c.cpu())
    barrier()
    t0 = time.perf_counter()
    if method == "ssp_rk3":
        for _ in range(e2e_steps):
            m.rk_step_host(h, dt, 1, precision=prec)
    else:
        # the same copies around dg_rk_step_method (pinned host buffer, one stream)
        for _ in range(e2e_steps):
            c.copy_(h, non_blocking=True)
            m.rk_step(c, dt, 1, precision=prec, method=method)
            h.copy_(c, non_blocking=True)
            torch.cuda.current_stream().synchronize()
    e2e_s = time.perf_counter() - t0
    state_bytes = m.N * 4 * m.np * 8

    line = None
    if rank == 0:
        # each timed library call is one kernel, except dg_conserved_totals: two
        # kernels (per-block partial sums, then the fixed-order final sum)
        launches = sum(n for n, _ in ktimes.values()) + ktimes.get("totals", (0, 0.0))[0]
        el_n, el_ms = ktimes.get("element", (0, 0.0))
        avg_el_ms = el_ms / max(1, el_n)
        if prec == "fp64":
            if args.vol_rule == "symmetric":
                flops = flops_element_direct_per_elem(p, ne, m.nq) * m.N
            else:
                flops = flops_element_per_elem(p, ne) * m.N
            achieved = flops / (avg_el_ms * 1e-3) / 1e12
            khash = _src_hash("dg_element.cu", "dg_device.cuh", "dg_tcgen05.cuh")
            if args.vol_rule != "collapsed":
                khash += ":" + args.vol_rule
            roofline = {"bound": "alu", "kernel": "k_element_sf (float64 FMA pipe)",
                        "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                        "frac": achieved / fp64_peak if fp64_peak else None, "traffic": TRAFFIC.get(khash),
                        "peak_source": "measured live: dg_probe_fma_rate float64 FMA chain",
                        "flops_per_launch": flops, "avg_launch_ms": avg_el_ms}
            ipe = FP64_INST.get(khash)
            if ipe is not None and fp64_peak:
                ach_i = ipe * m.N / (avg_el_ms * 1e-3) / 1e12
                roofline["fp64_issue"] = {"inst_per_elem": ipe, "achieved": ach_i, "peak": fp64_peak / 2,
                                          "unit": "T float64 instructions/s", "frac": ach_i / (fp64_peak / 2)}
            else:
                roofline["fp64_issue"] = None
        else:
            nbytes = bytes_element_tc_per_elem(p, ne) * m.N
            achieved = nbytes / (avg_el_ms * 1e-3) / 1e9
            hbm, src = hbm_peak()
            roofline = {"bound": "hbm", "kernel": "k_element_tc (tcgen05, %s)" % prec,
                        "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                        "traffic": None, "peak_source": src, "bytes_per_launch": nbytes,
                        "avg_launch_ms": avg_el_ms}
        share = {k: round(ms / max(1e-12, sum(x for _, x in ktimes.values())), 4)
                 for k, (_, ms) in ktimes.items()}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else prec + " contractions, f64 flux/update",
            "data": "synthetic (seeded jittered periodic mesh, isentropic vortex)",
            "config": {"workload": WORKLOAD["name"] if method == "ssp_rk3"
                       else WORKLOAD["name"].replace("SSP-RK3", method.upper()),
                       "n_elem": m.N, "p": p, "n_edge_pts": ne, "method": method,
                       "n_vol_pts": m.nq, "vol_rule": args.vol_rule, "precision": prec, "dt": dt,
                       "l2": "flushed between timed steps (256 MiB write outside the timed events)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roofline,
            "kernel_share": share,
            "kernel_times_ms": {k: {"launches": n, "total_ms": ms} for k, (n, ms) in ktimes.items()},
            "fp32_fma_tflops": fp32_peak,
            "e2e": {"value": dof_step * e2e_steps / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes,
                    "entry": "dg_rk_step_host" if method == "ssp_rk3" else "dg_rk_step_method"},
            "gpu_launches": launches,
            "paper_context": "GTX 580 (Fermi, FP64), double Mach reflection, p=1, RK2 with limiter: "
                             "1.31e8-1.53e8 DOF-updates/s per stage, derived from the paper's runtime "
                             "table; another problem and machine, context only",
            "clocks": clk,
            "wall_s_timed_region": wall,
            "totals_last_step": [float(x) for x in totals] if totals is not None else None,
        }
        if world == 1 and not args.no_extras and prec == "fp64" and method == "ssp_rk3":
            c0 = m.project_function(I.vortex)
            line["mixed"] = mixed_modes(m, c0, dt, max(5, min(args.steps, 20)), flush, t_max / args.steps)
            line["paper_steppers"] = paper_steppers(m, c0, dt, max(5, min(args.steps, 20)), flush)
            line["adjoint"] = adjoint_ratio()
            line["vortex_200_steps"] = vortex_error()
            line["mixed_512_p4"] = mixed_config3()
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(vol_rule=args.vol_rule)
            line["cpu_all_cores"] = cpu_all_cores(WORKLOAD["n"] // 2, vol_rule=args.vol_rule)
    if world > 1:
        import torch.distributed as tdist
        tdist.barrier()
        tdist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--configs", action="store_true",
                    help="run the five stated workloads (one JSON line each) instead of the benchmark")
    ap.add_argument("--precision", choices=["fp64", "tf32x3", "tf32x1"], default="fp64",
                    help="arithmetic of the timed steps (the headline line is fp64)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the mixed-precision and adjoint measurements")
    ap.add_argument("--method", choices=sorted(STAGES), default="ssp_rk3",
                    help="time integrator of the timed steps (the headline line is ssp_rk3)")
    ap.add_argument("--vol-rule", choices=["collapsed", "symmetric"], default="collapsed",
                    help="volume rule of the timed workload (the headline line uses the collapsed grid)")
    ap.add_argument("--rules", action="store_true",
                    help="both volume rules at p=1..5 in every precision instead of the benchmark")
    ap.add_argument("--sweep", action="store_true",
                    help="mesh-size scaling runs (p=1 x 10000 and p=4 x 1000 RK4 steps) instead of the benchmark")
    ap.add_argument("--case", choices=["mixed", "mixed512", "limiter", "adjoint", "small"],
                    help="a few untimed steps of one workload (for a profiler) instead of the benchmark")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    world, rank, local = _dist()
    if args.case:
        if rank == 0:
            run_case(args.case)
        return
    if args.configs:
        if rank == 0:
            run_configs()
        return
    if args.sweep:
        if rank == 0:
            run_sweep((args.precision,))
        return
    if args.rules:
        if rank == 0:
            run_rules()
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
