#!/usr/bin/env python
"""Benchmark of the SMM hot path on one GB300 (replicas on N GPUs).

Workload: manufactured-solution transport on a curved mesh -- [0,1]^2,
128x128 quads of geometry order 3 moved by the seeded sinusoidal map
(amplitude 0.05), DG p=4 (25 dofs/element), level-symmetric S8 (40
ordinates), sigma_t = 1, scattering ratio 0.9, MMS angular source and MMS
inflow.  16,384,000 angular unknowns per sweep.

A step is one SMM outer iteration through the C ABI (smm_iterate with
max_outer = 1): FP64 sweep with cached local inverses, FP64 moments and
boundary correction, IP-SMM right-hand side, multigrid-preconditioned CG to
1e-12, successive-difference check.  value = angular unknowns swept per second of
whole steps (all ranks).  Inputs stay resident; L2 is flushed (256 MiB
write) between timed steps.  Also reported: the FP32-refined and on-the-fly
LU variants of the step, the time to a 1e-8 relative successive difference
for the plain method (FP64 on-the-fly LU sweep, block-Jacobi PCG) and the
chosen one, the oracle on the host cores (cpu_baseline), and an end-to-end
number with host buffers.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WL = dict(nx=128, m=3, p=4, sn=8, sigma_t=1.0, c=0.9, seed=0)
WL_NAME = "mms-curved-128x128-m3-p4-S8-c0.9"
METRIC = "sweep unknowns/s (elem*dof*angle)"
CPU_SAMPLE_NX = 16


def workload_inputs(nx, m, p, sn_omega, sigma_t, c, seed):
    import numpy as np

    import smm_workloads as W

    mesh = W.structured_mesh(nx, m=m, perturb_seed=seed)
    ne = mesh.n_elem
    st = np.full(ne, sigma_t)
    ss = st * c
    pos = W.dg_node_positions(mesh, p)
    fpos = W.face_node_positions(mesh, p, W.boundary_faces(mesh))
    q = np.stack([W.mms_source(pos[:, :, 0], pos[:, :, 1], o[0], o[1], sigma_t, sigma_t * c) for o in sn_omega])
    inflow = np.stack([W.mms_psi(fpos[:, :, 0], fpos[:, :, 1], o[0], o[1]) for o in sn_omega])
    return mesh, st, ss, q, inflow


# ---------------------------------------------------------------------------
# CPU oracle leg (runs in a child process with one BLAS/OpenMP thread)
# ---------------------------------------------------------------------------

def oracle_rate(seconds: float, nx: int) -> dict:
    """Time oracle outer steps G(varphi) (sweep + closures + RHS + direct IP
    solve) on an nx*nx mesh of the bench workload's kind for ~`seconds`."""
    import numpy as np

    from oracle.smm import SMMProblem
    from oracle.transport import Discretization

    from oracle.quadrature import level_symmetric_2d
    om, _ = level_symmetric_2d(WL["sn"])
    mesh, st, ss, q, inflow = workload_inputs(nx, WL["m"], WL["p"], om, WL["sigma_t"], WL["c"], WL["seed"])
    disc = Discretization(mesh.nodes, mesh.elem_nodes, WL["m"], WL["p"], WL["sn"], st, ss)
    prob = SMMProblem(disc, q, inflow)
    phi = np.zeros((disc.ne, disc.n))
    times = []
    t_end = time.perf_counter() + seconds
    while len(times) < 2 or time.perf_counter() < t_end:
        t0 = time.perf_counter()
        phi, _ = prob.G(phi)
        times.append(time.perf_counter() - t0)
    unknowns = disc.ne * disc.n * disc.nd
    med = statistics.median(times)
    return dict(value=unknowns / med, unit="unknowns/s", cores=1, kind="oracle", steps=len(times),
                seconds_per_step=med,
                sample=f"oracle outer steps (sweep+closures+RHS+direct IP solve) on a {nx}x{nx} mesh of the same "
                       f"kind (m={WL['m']}, p={WL['p']}, S{WL['sn']}, c={WL['c']}), median of {len(times)}")


def run_oracle_child(seconds: float, nx: int) -> dict:
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_rate(%f, %d)))" % (ROOT, seconds, nx))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode:
        return dict(error=r.stderr[-500:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_model() -> str:
    """The host CPU's model name (x86: "model name"; Arm: implementer and part)."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return "unknown"
    fields = {}
    for line in info:
        if ":" in line:
            k, v = line.split(":", 1)
            fields.setdefault(k.strip(), v.strip())
    if "model name" in fields:
        return fields["model name"]
    if "CPU part" in fields:
        return f"Arm implementer {fields.get('CPU implementer', '?')} part {fields['CPU part']}"
    return "unknown"


def run_oracle_all_cores(seconds: float, nx: int, cores: int | None = None) -> dict:
    """The same oracle sample on every host core at once: one single-threaded
    child per core, each timing its own copy; the rates add up (independent
    problems, as replicas)."""
    if cores is None:
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_rate(%f, %d)))" % (ROOT, seconds, nx))
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                              text=True, env=env) for _ in range(cores)]
    rates, err = [], None
    for pr in procs:
        try:
            out, e = pr.communicate(timeout=900)
        except subprocess.TimeoutExpired:
            pr.kill()
            out, e = pr.communicate()
        if pr.returncode:
            err = (e or "")[-500:] or f"exit status {pr.returncode}"
        else:
            rates.append(json.loads(out.strip().splitlines()[-1])["value"])
    if err is not None:
        return dict(error=err)
    return dict(value=sum(rates), unit="unknowns/s", cores=cores, kind="oracle", cpu=cpu_model(),
                sample=f"{cores} concurrent single-threaded copies of the cpu_baseline sample ({nx}x{nx} mesh, "
                       f"~{seconds:g} s each), rates summed")


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (getattr(self, "out", "") or "").splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=[], samples=0)
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), reasons=sorted(reasons), samples=len(sm))


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

# DRAM bytes (read + write) per launch measured by ncu for the current kernels
# on this workload (the cg_iteration, sweep-kernel and launch-list summaries for this workload); a key
# is dropped whenever the kernels it covers change.
NCU_TRAFFIC: dict = {"cg_iteration": 644.0e6, "sweep_kernel": 3882.6e6, "moments": 138.6e6}

# a timed step is outer iteration START_ITERATIONS + 1 from varphi^0 = 0
START_ITERATIONS = 3


def cached_sweep_bytes_per_task(p: int, word: int, angular: bool) -> float:
    """HBM bytes of one cached-inverse task: the n x n inverse, the n outputs
    (FP64 and, in the FP64 path, the FP32-pair copy), the angular source term
    M q_d (an FP32 pair per node) and two inflow traces."""
    n = (p + 1) ** 2
    return word * (n * n + 2 * n + 2 * (p + 1)) + (8 * n if angular else 0)


def moments_bytes_per_elem(n: int, nd: int) -> float:
    """HBM bytes of the moment reduction per element: psi as FP32 pairs read
    once (8 nd n) and six FP64 moments written (48 n)."""
    return 8 * nd * n + 48 * n


def mg_cg_bytes_per_iter(ne: int, n: int, nu0: int = 3) -> float:
    """HBM bytes of one multigrid-preconditioned CG iteration on the element
    blocks, with nu0 level-0 smoothing steps before and after the coarse
    correction (the library's default: 3).  The operator is stored as the n x n
    diagonal block plus four G x G face-coupling matrices per element
    (G = 2(p+1)): the FP64-accuracy product reads it once as FP32 pairs
    (8 (n^2 + 4 G^2) B); level 0 reads the FP32 block-Jacobi inverse in every
    smoothing step (2 nu0 * 4 n^2 B), the FP32 face couplings in the 2 nu0 - 1
    steps that start from a nonzero iterate and in the residual (2 nu0 * 16 G^2
    B), and, in the residual, the 4 x n matrix w4^T A_d that stands for the
    diagonal block in the element-corner sums (16 n B; a smoothing step needs no
    diagonal block because Pinv is its inverse); the Chebyshev recurrence reads
    the previous FP32 iterate in 2 nu0 - 3 steps; about 30 FP64 vector passes of
    n words.  The vertex and aggregation levels are < 2 % of the bytes and left
    out."""
    g = 2 * (int(round(n ** 0.5)))
    op = n * n + 4 * g * g
    prev = max(0, 2 * nu0 - 3)
    return ne * (8 * op + 2 * nu0 * 4 * n * n + 2 * nu0 * 16 * g * g + 16 * n + prev * 4 * n + 30 * n * 8)


def max_over_ranks(value: float, dist, device) -> float:
    """The largest of every rank's value (the slowest replica sets the job's
    time); the value itself when there is one rank (dist is None)."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args) -> None:
    import numpy as np
    import torch

    import paper_2304_07386_gb300 as P

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2304_07386_gb300 import build as B
    B.build()
    om, _ = P.smm_quadrature(WL["sn"])
    t_in = time.time()
    mesh, st, ss, q, inflow = workload_inputs(WL["nx"], WL["m"], WL["p"], om, WL["sigma_t"], WL["c"], WL["seed"])
    t_in = time.time() - t_in
    stream = torch.cuda.Stream()

    def create(precision, solver=None, precond=None, anderson=0, moment=None, tiles=1):
        opt = P.smm_default_options()
        opt.anderson_depth = anderson
        opt.sweep_tiles = tiles
        if moment is not None:
            opt.moment_discretization = moment
        opt.sweep_precision = precision
        opt.tol_cg = 1e-12
        if solver is not None:
            opt.sweep_solver = solver
        if precond is not None:
            opt.precond = precond
        if args.host_cg_loop:
            opt.cg_device_loop = 0
        t0 = time.time()
        h = P.smm_create(mesh.nodes, mesh.elem_nodes, WL["m"], WL["p"], WL["sn"], st, ss, q, inflow=inflow,
                         options=opt, stream=stream)
        return h, time.time() - t0

    h, t_setup = create(P.SMM_SWEEP_FP64)
    info = h.info()
    ne, n, nd = info.n_elem, info.n_dof_elem, info.n_ord
    unknowns = info.n_angular
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB
    phi = torch.zeros(ne * n, dtype=torch.float64, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    def step(handle, x):
        rc, s = P.smm_iterate(handle, x, 1e-300, 1, relative=True, raise_on_error=False)
        if rc not in (0, 7):
            raise P.SMMError(rc, P.load_library().smm_last_error().decode())
        return s

    # Every warm-up and timed step is the same outer iteration: the fourth one
    # from varphi^0 = 0 (varphi^3 is restored before each step, outside the
    # timed region), so the CG work per step does not drift as the iteration
    # converges and the number does not depend on --steps / --warmup.
    phi_start = torch.zeros_like(phi)
    with torch.cuda.stream(stream):
        for _ in range(START_ITERATIONS):
            step(h, phi_start)
        for _ in range(args.warmup):
            phi.copy_(phi_start)
            step(h, phi)
        barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        stats = []
        with ClockSampler(local) as clk:
            for k in range(args.steps):
                flush.fill_(float(k))
                phi.copy_(phi_start)
                ev[k][0].record(stream)
                stats.append(step(h, phi))
                ev[k][1].record(stream)
            barrier()
        step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = max_over_ranks(sum(step_ms) / len(step_ms), dist, "cuda")
    value = world * unknowns / (ms * 1e-3)

    def mean(key):
        return sum(s[key] for s in stats) / len(stats)

    ms_sweep, ms_res, ms_solve = mean("ms_sweep"), mean("ms_residual"), mean("ms_solve")
    cg_it = mean("cg_total")
    launches = int(sum(s["n_launches"] for s in stats))

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    tasks = ne * nd
    # the sweep phase also runs the source kernel: M (n^2), varphi and q (2n) read, M s written as pairs (n)
    sweep_bytes = tasks * cached_sweep_bytes_per_task(WL["p"], 8, True) + ne * 8 * (n * n + 3 * n)
    cg_bytes = mg_cg_bytes_per_iter(ne, n)
    mom_bytes = ne * moments_bytes_per_elem(n, nd)
    ms_mom = mean("ms_moments")
    ms_iter = ms_solve / cg_it if cg_it > 0 else 0.0

    def entry(bytes_per_launch, ms_per_launch, kernel, traffic_key, launches_per_step):
        gbs = bytes_per_launch / (ms_per_launch * 1e-3) / 1e9 if ms_per_launch > 0 else 0.0
        return dict(bound="hbm", achieved=gbs, peak=hbm, unit="GB/s", frac=gbs / hbm,
                    traffic=NCU_TRAFFIC.get(traffic_key), algorithmic_bytes=bytes_per_launch, ms=ms_per_launch,
                    launches_per_step=launches_per_step, kernel=kernel, peak_note=f"{hbm_src} copy bandwidth")

    rooflines = {
        "cg_iteration": entry(cg_bytes, ms_iter, "one flexible-CG iteration: 11 kernels (operator product; "
                              "V-cycle: first smoothing step with the CG update, 2 smoothing steps, residual, "
                              "cluster coarse cycle, prolongation, 2 smoothing steps, last smoothing step with the "
                              "dot products; direction), run inside one device-side graph loop",
                              "cg_iteration", cg_it),
        "sweep_kernel": entry(sweep_bytes, ms_sweep, "sweep_kernel<double, 4, SOURCE, cached inverse> "
                              "(plus the per-sweep source kernel)", "sweep_kernel", 1),
        "moments": entry(mom_bytes, ms_mom, "moments_df_kernel + beta_kernel", "moments", 1),
    }
    rooflines["cg_iteration"]["traffic_note"] = (
        "ncu DRAM bytes of the 11 kernels, captured before the direction update's launch grid changed from a "
        "grid-stride loop to one thread per unknown (same kernel code, each unknown read and written once either way)")
    # dominant: the largest device time per step
    dom = max(rooflines, key=lambda k: rooflines[k]["ms"] * rooflines[k]["launches_per_step"])
    roof = dict(rooflines[dom])

    # end to end through the C ABI with host buffers: H2D of varphi^k, one outer
    # step, D2H of varphi^{k+1}, all inside the timed region
    host = torch.zeros(ne * n, dtype=torch.float64).pin_memory()
    e2e_ms = []
    with torch.cuda.stream(stream):
        for k in range(max(2, args.steps)):
            flush.fill_(1.0)
            host.copy_(phi_start)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            phi.copy_(host, non_blocking=True)
            step(h, phi)
            host.copy_(phi, non_blocking=True)
            b.record(stream)
            b.synchronize()
            e2e_ms.append(a.elapsed_time(b))
    e2e = dict(value=world * unknowns / (max_over_ranks(statistics.mean(e2e_ms), dist, "cuda") * 1e-3),
               unit="unknowns/s",
               h2d_bytes_per_step=8 * ne * n, d2h_bytes_per_step=8 * ne * n)

    extra = {}
    if not args.quick:
        def time_steps(handle, nsteps=4):
            x = torch.zeros_like(phi)
            out = []
            with torch.cuda.stream(stream):
                for _ in range(2):
                    step(handle, x)
                torch.cuda.synchronize()
                for _ in range(nsteps):
                    flush.fill_(2.0)
                    a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    s_ = step(handle, x)
                    b2.record(stream)
                    b2.synchronize()
                    out.append((a.elapsed_time(b2), s_))
            msx = statistics.mean(t for t, _ in out)
            return dict(value=unknowns / (msx * 1e-3), ms_per_step=msx,
                        ms_sweep=statistics.mean(s_["ms_sweep"] for _, s_ in out),
                        ms_residual=statistics.mean(s_["ms_residual"] for _, s_ in out),
                        ms_solve=statistics.mean(s_["ms_solve"] for _, s_ in out))

        h32, _ = create(P.SMM_SWEEP_FP32_REFINED)
        extra["fp32_refined_step"] = time_steps(h32)
        h32.destroy()
        hlu, _ = create(P.SMM_SWEEP_FP64, solver=P.smm.SMM_SOLVER_LU)
        extra["fp64_lu_step"] = time_steps(hlu)
        hlu.destroy()

        def solve(precision, solver=None, precond=None, anderson=0, moment=None):
            hh, _ = create(precision, solver, precond, anderson, moment)
            x = torch.zeros_like(phi)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                rc, s_ = P.smm_iterate(hh, x, 1e-8, 200, relative=True, raise_on_error=False)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            hh.destroy()
            return dt, s_, rc, x

        tp, sp, rcp, xp = solve(P.SMM_SWEEP_FP64, P.smm.SMM_SOLVER_LU, P.smm.SMM_PRECOND_BLOCK_JACOBI)
        tc, sc, rcc, xc = solve(P.SMM_SWEEP_FP64)
        ta, sa, rca, xa = solve(P.SMM_SWEEP_FP64, anderson=2)
        t3, s3, rc3, x3 = solve(P.SMM_SWEEP_FP32_REFINED)
        # parallel block Jacobi sweep: shorter dependency chains, more outer steps
        bj = {}
        for tiles in (2, 4, 8):
            hb_, _ = create(P.SMM_SWEEP_FP64, tiles=tiles)
            levels = hb_.info().n_levels
            xb_ = torch.zeros_like(phi)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                rcb, sb_ = P.smm_iterate(hb_, xb_, 1e-8, 400, relative=True, raise_on_error=False)
            torch.cuda.synchronize()
            bj[f"tiles_{tiles}x{tiles}"] = dict(
                seconds=time.perf_counter() - t0, status=rcb, outer=sb_["outer_iterations"], levels=levels,
                ms_sweep_per_outer=sb_["ms_sweep"] / max(1, sb_["outer_iterations"]),
                cg_total=sb_["cg_total"], rel_diff_vs_exact_sweep=float((xb_ - xc).abs().max() / xc.abs().max()))
            hb_.destroy()
        extra["time_to_1e-8_block_jacobi"] = bj
        tg, sg, rcg, xg = solve(P.SMM_SWEEP_FP64, moment=P.smm.SMM_MOMENT_CG)
        extra["time_to_1e-8_cg_moments"] = dict(
            seconds=tg, outer=sg["outer_iterations"], cg_total=sg["cg_total"], status=rcg,
            ms_solve_per_outer=sg["ms_solve"] / max(1, sg["outer_iterations"]),
            rel_diff_vs_ip=float((xg - xc).abs().max() / xc.abs().max()),
            method="continuous finite element moment system (Sec. 5.1), FP64 cached sweep, V-cycle-preconditioned "
                   "CG on the continuous nodes; differs from the IP solution by the discretization error")
        extra["time_to_1e-8"] = dict(
            plain_s=tp, plain_outer=sp["outer_iterations"], plain_cg_total=sp["cg_total"], plain_status=rcp,
            plain="FP64 sweep with on-the-fly LU, element-block-Jacobi PCG, zero guess",
            chosen_s=tc, chosen_outer=sc["outer_iterations"], chosen_cg_total=sc["cg_total"], chosen_status=rcc,
            chosen="FP64 sweep with cached local inverses, multigrid PCG, zero guess",
            fp32_refined_s=t3, fp32_refined_outer=s3["outer_iterations"], fp32_refined_status=rc3,
            anderson2_s=ta, anderson2_outer=sa["outer_iterations"], anderson2_cg_total=sa["cg_total"],
            anderson2_status=rca, rel_diff_anderson2_vs_plain=float((xa - xp).abs().max() / xp.abs().max()),
            rel_diff_chosen_vs_plain=float((xc - xp).abs().max() / xp.abs().max()),
            rel_diff_fp32_vs_plain=float((x3 - xp).abs().max() / xp.abs().max()),
            learned_guess="see the learned_guess entry (network trained in the run on the learned-guess workload)")

    if not args.quick and args.batch > 0:
        extra["batched_sweep"] = run_batch(args.batch, stream)
    if not args.quick and args.learned > 0:
        extra["learned_guess"] = run_learned(args.learned, stream)
    if not args.quick:
        extra["thick_thin"] = run_thick_thin(stream)

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = run_oracle_child(args.cpu_seconds, CPU_SAMPLE_NX)
        cpu["cpu"] = cpu_model()
        cpu_all = run_oracle_all_cores(args.cpu_seconds, CPU_SAMPLE_NX)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (FP32 copies of the multigrid smoother blocks)", "data": "synthetic",
            "config": {"workload": WL_NAME, "n_elem": ne, "p": WL["p"], "geom_order": WL["m"], "sn": WL["sn"],
                       "n_ord": nd, "angular_unknowns": unknowns, "parallelism": f"replicas x{world}",
                       "l2": "flushed between timed steps (256 MiB write)", "sweep": "fp64, cached local inverses",
                       "step_state": f"outer iteration {START_ITERATIONS + 1} from varphi^0 = 0, restored before "
                                     "every step",
                       "moment_solve": "flexible CG, multigrid V-cycle with degree-3 Chebyshev level-0 smoothing", "cg_tol": 1e-12,
                       "cg_loop": "host-checked chunks" if args.host_cg_loop else "one device-side graph loop"},
            "roofline": roof, "roofline_all": rooflines, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all,
            "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary(),
            "phases_ms": dict(residual=ms_res, sweep=ms_sweep, moments=mean("ms_moments"), rhs=mean("ms_rhs"),
                              solve=ms_solve, cg_iters=cg_it),
            "sweep_only": dict(value=unknowns / ((ms_sweep + ms_res) * 1e-3), unit="unknowns/s",
                               note="sweep kernel (plus the per-sweep source kernel)"),
            "setup_s": t_setup, "inputs_s": t_in,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    h.destroy()
    if dist:
        dist.destroy_process_group()


def batch_problem(seed: int):
    """One problem of the uneven batched-instances workload (reduced mesh
    range): n ~ U{32..96}, p ~ U{1..4}, S_N ~ U{4,6,8,10,12}, sigma_t =
    10 exp(1.5 g) with g a unit Gaussian random field (correlation length 0.1),
    c ~ U[0.5, 0.99], q = 1 per steradian, vacuum, straight mesh."""
    import numpy as np

    import smm_workloads as W

    rng = np.random.default_rng(1000 + seed)
    nx = int(rng.integers(32, 97))
    p = int(rng.integers(1, 5))
    sn = int(rng.choice([4, 6, 8, 10, 12]))
    c = float(rng.uniform(0.5, 0.99))
    mesh = W.structured_mesh(nx, m=1)
    st = 10.0 * np.exp(1.5 * W.gaussian_random_field(nx, 0.1, seed))
    return mesh, p, sn, st, c * st, np.ones((mesh.n_elem, (p + 1) ** 2))


def run_batch(nprob: int, stream) -> dict:
    """Time one batched sweep of nprob uneven problems against the same
    problems swept one at a time (FP32-refined sweeps, cached inverses)."""
    import torch

    import paper_2304_07386_gb300 as P

    hs, unknowns = [], 0
    for i in range(nprob):
        mesh, p, sn, st, ss, q = batch_problem(i)
        opt = P.smm_default_options()
        opt.sweep_precision = P.SMM_SWEEP_FP32_REFINED
        hs.append(P.smm_create(mesh.nodes, mesh.elem_nodes, 1, p, sn, st, ss, q, options=opt, stream=stream))
        unknowns += hs[-1].info().n_angular
    b = P.smm.smm_batch_create(hs)
    sched = b.schedule()

    def timed(fn, reps=3):
        best = 1e300
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        return best

    with torch.cuda.stream(stream):
        tb = timed(lambda: P.smm.smm_batch_sweep(b))
        ts = timed(lambda: [P.smm_sweep(h) for h in hs])
    b.destroy()
    for h in hs:
        h.destroy()
    return dict(problems=nprob, angular_unknowns=unknowns, batched_s=tb, one_at_a_time_s=ts,
                batched_value=unknowns / tb, one_at_a_time_value=unknowns / ts, unit="unknowns/s",
                schedule=sched, note="wall time of smm_batch_sweep vs consecutive smm_sweep calls (each includes "
                                     "the FP64 residual, the FP32 correction sweep, moments and one sync)")


def run_learned(nx: int, stream, n_train: int = 128, n_test: int = 8, p: int = 2, sn: int = 8) -> dict:
    """Learned-guess workload (p=2, S8, log-normal sigma_t / sigma_s fields,
    piecewise-constant source maps, on an nx*nx grid of quads): train the
    library's network on n_train converged solutions the method produces,
    then time held-out solves to a 1e-8 relative difference: the plain GPU
    method (FP64 on-the-fly LU sweep, block-Jacobi PCG, zero guess), the
    chosen method with a zero guess, and the chosen method started from the
    network's proposal (guess_check on)."""
    import numpy as np
    import torch

    import paper_2304_07386_gb300 as P
    import smm_workloads as W
    from paper_2304_07386_gb300 import guess as G

    n = (p + 1) ** 2

    def make(seed, plain=False, check=False, anderson=0):
        mesh, st, ss, qe = W.learned_guess_problem(nx, seed)
        opt = P.smm_default_options()
        opt.tol_cg = 1e-12
        opt.guess_check = int(check)
        opt.anderson_depth = anderson
        if plain:
            opt.sweep_solver = P.smm.SMM_SOLVER_LU
            opt.precond = P.smm.SMM_PRECOND_BLOCK_JACOBI
        h = P.smm_create(mesh.nodes, mesh.elem_nodes, 1, p, sn, st, ss, np.repeat(qe[:, None], n, axis=1),
                         options=opt, stream=stream)
        return h, (st, ss, qe)

    def solve(h, tol, phi0=None):
        x = torch.zeros(nx * nx * n, dtype=torch.float64, device="cuda")
        if phi0 is not None:
            x.copy_(torch.as_tensor(phi0, device="cuda"))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            rc, s = P.smm_iterate(h, x, tol, 200, relative=True, raise_on_error=False)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, s, x

    t_gen = time.perf_counter()
    X, Y = [], []
    for seed in range(n_train):
        h, (st, ss, qe) = make(seed)
        _, _, x = solve(h, 1e-10)
        mom = torch.zeros(6 * nx * nx * n, dtype=torch.float64, device="cuda")
        P.smm_moments(h, mom)
        h.destroy()
        X.append(G.features(st, ss, qe, nx))
        Y.append(G.targets(x.cpu().numpy(), mom.cpu().numpy(), nx, n))
    t_gen = time.perf_counter() - t_gen
    X, Y = np.stack(X), np.stack(Y)
    xn, yn = G.Normalizer(X), G.Normalizer(Y)
    net = P.smm.Guess(nx, nx, 4 * n, 16, seed=0, stream=stream)
    t_train = time.perf_counter()
    with torch.cuda.stream(stream):
        losses = G.train(net, torch.as_tensor(xn.fwd(X), device="cuda"), torch.as_tensor(yn.fwd(Y), device="cuda"),
                         steps=1500, batch=16, lr=3e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t_train
    rows = []
    for seed in range(100_000, 100_000 + n_test):
        hp, _ = make(seed, plain=True)
        tp, sp, xp = solve(hp, 1e-8)
        hp.destroy()
        hz, (st, ss, qe) = make(seed)
        tz, sz, xz = solve(hz, 1e-8)
        hz.destroy()
        with torch.cuda.stream(stream):
            xg = torch.as_tensor(xn.fwd(G.features(st, ss, qe, nx)[None]), device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            phi0 = G.predict_phi(net, xg, yn, nx, n)
            t_inf = time.perf_counter() - t0
        hg, _ = make(seed, check=True)
        tg, sg, xgs = solve(hg, 1e-8, phi0)
        hg.destroy()
        ha, _ = make(seed, check=True, anderson=2)
        ta, sa, xa = solve(ha, 1e-8, phi0)
        ha.destroy()
        rows.append(dict(plain_s=tp, plain_outer=sp["outer_iterations"], zero_s=tz, zero_outer=sz["outer_iterations"],
                         guess_s=tg + t_inf, guess_outer=sg["outer_iterations"], rejected=sg["guess_rejected"],
                         guess_anderson2_s=ta + t_inf, guess_anderson2_outer=sa["outer_iterations"],
                         rel_diff_guess_vs_plain=float((xgs - xp).abs().max() / xp.abs().max())))
    mean = lambda k: float(np.mean([r[k] for r in rows]))
    return dict(grid=f"{nx}x{nx}", p=p, sn=sn, train_problems=n_train, test_problems=n_test,
                params=net.n_params, data_gen_s=t_gen, train_s=t_train, final_loss=float(np.mean(losses[-50:])),
                initial_loss=float(np.mean(losses[:10])),
                mean_plain_s=mean("plain_s"), mean_zero_guess_s=mean("zero_s"), mean_learned_s=mean("guess_s"),
                mean_learned_anderson2_s=mean("guess_anderson2_s"),
                mean_outer_plain=mean("plain_outer"), mean_outer_zero=mean("zero_outer"),
                mean_outer_learned=mean("guess_outer"), mean_outer_learned_anderson2=mean("guess_anderson2_outer"),
                rejected=int(sum(r["rejected"] for r in rows)),
                max_rel_diff_vs_plain=max(r["rel_diff_guess_vs_plain"] for r in rows),
                note="times to a 1e-8 relative successive difference, inference included; the plain method is the "
                     "FP64 on-the-fly LU sweep with block-Jacobi PCG and a zero guess")


def run_thick_thin(stream, nx: int = 256, blocks: int = 8, p: int = 3, sn: int = 12) -> dict:
    """Multi-material thick/thin workload: [0,8]^2, nx x nx straight quads, a
    seeded blocks x blocks layout of thick (sigma_t = 200, c = 0.999) and thin
    (sigma_t = 0.2, c = 0.5) cells, unit isotropic source in the lowest-index
    thin block, vacuum, p = 3, S12.  Time to a 1e-8 relative successive
    difference from zero, outer iterations and CG iterations per outer step,
    for the default method and with Anderson acceleration of depth 2."""
    import numpy as np
    import torch

    import paper_2304_07386_gb300 as P
    import smm_workloads as W

    mesh = W.structured_mesh(nx, m=1, domain=(0.0, 8.0, 0.0, 8.0))
    st, ss, blk, thick = W.block_materials(nx, blocks, 0)
    src_blk = int(np.flatnonzero(~thick)[0])
    n = (p + 1) ** 2
    q = np.repeat((blk == src_blk).astype(np.float64)[:, None], n, axis=1)
    out = dict(grid=f"{nx}x{nx}", p=p, sn=sn, thick_blocks=int(thick.sum()), blocks=blocks * blocks)
    for name, depth in (("default", 0), ("anderson2", 2)):
        opt = P.smm_default_options()
        opt.anderson_depth = depth
        h = P.smm_create(mesh.nodes, mesh.elem_nodes, 1, p, sn, st, ss, q, options=opt, stream=stream)
        info = h.info()
        x = torch.zeros(info.n_elem * info.n_dof_elem, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, s = P.smm_iterate(h, x, 1e-8, 200, relative=True, raise_on_error=False)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        out[name] = dict(seconds=dt, status=rc, outer=s["outer_iterations"],
                         cg_per_outer=s["cg_total"] / max(1, s["outer_iterations"]), cg_max=s["cg_max"],
                         angular_unknowns=int(info.n_angular))
        h.destroy()
    return out


def run_reference(args) -> None:
    """The oracle arm: the CPU oracle on the host cores, K timed steps of a
    bounded sample (one outer step each), after W warm-up steps."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    import numpy as np

    from oracle.quadrature import level_symmetric_2d
    from oracle.smm import SMMProblem
    from oracle.transport import Discretization

    om, _ = level_symmetric_2d(WL["sn"])
    nx = CPU_SAMPLE_NX
    mesh, st, ss, q, inflow = workload_inputs(nx, WL["m"], WL["p"], om, WL["sigma_t"], WL["c"], WL["seed"])
    disc = Discretization(mesh.nodes, mesh.elem_nodes, WL["m"], WL["p"], WL["sn"], st, ss)
    prob = SMMProblem(disc, q, inflow)
    phi = np.zeros((disc.ne, disc.n))
    for _ in range(args.warmup):
        phi, _ = prob.G(phi)
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        phi, _ = prob.G(phi)
        t.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(t)
    unknowns = disc.ne * disc.n * disc.nd
    value = unknowns / (ms * 1e-3)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    sample = (f"oracle outer steps on a {nx}x{nx} mesh of the bench workload's kind (m={WL['m']}, p={WL['p']}, "
              f"S{WL['sn']}); the full {WL['nx']}x{WL['nx']} workload is {(WL['nx'] // nx) ** 2}x larger")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": 0, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WL_NAME, "sample_mesh": f"{nx}x{nx}", "angular_unknowns": unknowns},
        "cpu_baseline": {"value": value, "unit": "unknowns/s", "cores": 1, "kind": "oracle",
                         "sample": sample, "cpu": cpu_model()},
        "e2e": {"value": value, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="skip the FP64 and time-to-solution extras")
    ap.add_argument("--host-cg-loop", action="store_true",
                    help="launch the CG iterations from the host in chunks instead of one device-side loop graph "
                         "(profiling runs: ncu does not see kernels inside conditional graph nodes)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--nx", type=int, default=WL["nx"], help="mesh size override (profiling runs)")
    ap.add_argument("--batch", type=int, default=24, help="problems in the batched-sweep measurement (0: skip)")
    ap.add_argument("--learned", type=int, default=32, help="element grid of the learned-guess measurement (0: skip)")
    args = ap.parse_args()
    WL["nx"] = args.nx
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
