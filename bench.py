#!/usr/bin/env python
"""Benchmark of the SMM hot path on one GB300 (replicas on N GPUs).

Workload (headline): multi-material thick/thin transport -- [0,8]^2, 256x256
straight quads, a seeded 8x8 layout of 1x1 blocks, each thick (sigma_t = 200,
scattering ratio 0.999) or thin (sigma_t = 0.2, ratio 0.5), a unit isotropic
source in the lowest-index thin block, vacuum boundaries; DG p=3 (16
dofs/element), level-symmetric S12 (84 ordinates): 88,080,384 angular
unknowns per sweep.

A step is one SMM outer iteration through the C ABI (smm_iterate with
max_outer = 1): the sweep with cached local inverses applied in FP32-pair
arithmetic and the moments formed in its epilogue, the IP-SMM right-hand
side, multigrid-preconditioned flexible CG to 1e-12, the successive-difference
check.  value = angular unknowns swept per second of whole steps (all ranks).
Inputs stay resident; L2 is flushed (256 MiB write) between timed steps.
Also reported: the sweep alone (sweep_unknowns_per_s), rooflines of its
kernels, the time to a 1e-8 relative successive difference, the curved
manufactured-solution workload, the FP32-refined sweep, batched uneven
problems, the learned-guess comparison, the oracle on the host cores
(cpu_baseline), and an end-to-end number through smm_iterate on a host array.
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

# headline workload: thick/thin contrast (the element size of the 256x256 mesh on [0,8]^2 is 1/32; a
# block is 32x32 elements)
WL = dict(nx=256, blocks=8, p=3, sn=12, seed=0, length=8.0)
WL_NAME = "thick-thin-256x256-p3-S12"
METRIC = "sweep unknowns/s (elem*dof*angle)"
# the oracle's sample: 16x16 elements of the same size and materials, 2x2 blocks of 8x8 elements
CPU_SAMPLE = dict(nx=16, blocks=2, length=0.5)
# the curved manufactured-solution workload of the extras
WL2 = dict(nx=128, m=3, p=4, sn=8, sigma_t=1.0, c=0.9, seed=0)
WL2_NAME = "mms-curved-128x128-m3-p4-S8-c0.9"


def thick_thin_inputs(nx, blocks, p, seed, length):
    """Mesh, sigma_t, sigma_s and the isotropic source [n_elem][n] of the
    thick/thin workload (vacuum boundaries)."""
    import numpy as np

    import smm_workloads as W

    mesh = W.structured_mesh(nx, m=1, domain=(0.0, length, 0.0, length))
    st, ss, blk, thick = W.block_materials(nx, blocks, seed)
    src_blk = int(np.flatnonzero(~thick)[0])
    q = np.repeat((blk == src_blk).astype(np.float64)[:, None], (p + 1) ** 2, axis=1)
    return mesh, st, ss, q, thick


def workload_sources(mesh, p, sn_omega, sigma_t, c):
    """Manufactured angular source and inflow of the curved MMS workload."""
    import numpy as np

    import smm_workloads as W

    pos = W.dg_node_positions(mesh, p)
    fpos = W.face_node_positions(mesh, p, W.boundary_faces(mesh))
    q = np.stack([W.mms_source(pos[:, :, 0], pos[:, :, 1], o[0], o[1], sigma_t, sigma_t * c) for o in sn_omega])
    inflow = np.stack([W.mms_psi(fpos[:, :, 0], fpos[:, :, 1], o[0], o[1]) for o in sn_omega])
    return q, inflow


def workload_inputs(nx, m, p, sn_omega, sigma_t, c, seed):
    import numpy as np

    import smm_workloads as W

    mesh = W.structured_mesh(nx, m=m, perturb_seed=seed)
    ne = mesh.n_elem
    st = np.full(ne, sigma_t)
    ss = st * c
    q, inflow = workload_sources(mesh, p, sn_omega, sigma_t, c)
    return mesh, st, ss, q, inflow


# ---------------------------------------------------------------------------
# CPU oracle leg (runs in a child process with one BLAS/OpenMP thread)
# ---------------------------------------------------------------------------

def oracle_rate(seconds: float, nx: int) -> dict:
    """Time oracle outer steps G(varphi) (sweep + closures + RHS + direct IP
    solve) on the thick/thin sample for ~`seconds`."""
    import numpy as np

    from oracle.smm import SMMProblem
    from oracle.transport import Discretization

    c = CPU_SAMPLE
    mesh, st, ss, q, _ = thick_thin_inputs(c["nx"], c["blocks"], WL["p"], WL["seed"], c["length"])
    disc = Discretization(mesh.nodes, mesh.elem_nodes, 1, WL["p"], WL["sn"], st, ss)
    prob = SMMProblem(disc, q)
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
                seconds_per_step=med, sample=cpu_sample_text(len(times)))


def cpu_sample_text(steps=None) -> str:
    c = CPU_SAMPLE
    return (f"oracle outer steps (sweep + closures + RHS + direct IP solve) on a {c['nx']}x{c['nx']} piece of the "
            f"thick/thin workload (same element size and materials, {c['blocks']}x{c['blocks']} blocks, p={WL['p']}, "
            f"S{WL['sn']})" + (f", median of {steps}" if steps else "") +
            f"; the full workload has {(WL['nx'] // c['nx']) ** 2}x the elements")


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

# DRAM bytes (read + write) per launch measured by ncu for the current kernels (profiles/): captured
# on the 128x128 piece of the headline workload (a quarter of its elements, to keep the capture small)
# and scaled x4, every kernel's bytes being proportional to the element count; a key is dropped
# whenever the kernels it covers change.  The CG iteration's entry (4 x 332,872,960 bytes) was dropped
# when its last level-0 step came to form its two block sums in one pass (a change of shared-memory
# reductions only) and stays out until it is captured again.
NCU_TRAFFIC: dict = {"sweep_kernel": 4 * 3268649728}

# a timed step is outer iteration START_ITERATIONS + 1 from varphi^0 = 0
START_ITERATIONS = 3


def sweep_bytes(ne: int, nd: int, p: int, angular: bool) -> float:
    """Algorithmic HBM bytes of one sweep launch of this design (FP64 cached
    mode): per (element, ordinate) task the n x n inverse as FP32 pairs
    (8 n^2), the n solution pairs written (8 n), two inflow traces of p+1
    pairs read (16 (p+1)) and, for an angular source, M q_d as pairs (8 n);
    per element M s as pairs (8 n), the flux re-read by the moment reduction
    (8 n nd) and six FP64 moments written (48 n)."""
    n = (p + 1) ** 2
    task = 8 * n * n + 8 * n + 16 * (p + 1) + (8 * n if angular else 0)
    return ne * nd * task + ne * (8 * n + 8 * n * nd + 48 * n)


def sweep_trace_bytes(ne: int, nd: int, p: int, m: int) -> float:
    """The sweep's algorithmic bytes per unit of work counted for a method
    that assembles every local system from geometry (no stored operators):
    per task four face traces of p+1 FP64 values (two inflow read, two
    outflow written); per element varphi (8 n), the control points
    (16 (m+1)^2) and the six moments (48 n)."""
    n = (p + 1) ** 2
    return ne * nd * 32 * (p + 1) + ne * (8 * n + 16 * (m + 1) ** 2 + 48 * n)


def sweep_fp32_ops(ne: int, nd: int, p: int) -> float:
    """FP32 instructions of the sweep's pair arithmetic per launch: a pair
    multiply-add (Dekker product, TwoSum, error accumulation) is 12 FP32
    instructions; a task forms n^2 of them for A^-1 b and about 2 n (p+1) for
    its two inflow faces; the moment reduction forms 6 n nd per element."""
    n = (p + 1) ** 2
    return 12.0 * (ne * nd * (n * n + 2 * n * (p + 1)) + ne * 6 * n * nd)


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


def load_peaks() -> tuple:
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        peaks = {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    src = "measured" if "hbm_gbs" in peaks else "fallback"
    return hbm, src


def load_tensor_peak() -> tuple:
    """(dense BF16 TFLOP/s burst, 'measured' | 'fallback')"""
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        peaks = {}
    return float(peaks.get("bf16_tflops", 1900.0)), ("measured" if "bf16_tflops" in peaks else "fallback")


# FP32 instruction issue of the whole GPU at the maximum SM clock: 152 SMs x 128 FP32 lanes x 2.07 GHz
FP32_ISSUE_PEAK = 152 * 128 * 2.07e9


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
    t_in = time.time()
    nx = args.nx
    mesh, st, ss, q, thick = thick_thin_inputs(nx, WL["blocks"], WL["p"], WL["seed"], WL["length"] * nx / WL["nx"])
    t_in = time.time() - t_in
    stream = torch.cuda.Stream()

    def create(precision=P.SMM_SWEEP_FP64, anderson=0, moment=None, solver=None, cg_adaptive=0.0):
        opt = P.smm_default_options()
        opt.anderson_depth = anderson
        opt.cg_tol_adaptive = cg_adaptive
        opt.sweep_precision = precision
        opt.tol_cg = 1e-12
        if moment is not None:
            opt.moment_discretization = moment
        if solver is not None:
            opt.sweep_solver = solver
        if args.host_cg_loop:
            opt.cg_device_loop = 0
        t0 = time.time()
        h = P.smm_create(mesh.nodes, mesh.elem_nodes, 1, WL["p"], WL["sn"], st, ss, q, options=opt, stream=stream)
        return h, time.time() - t0

    h, t_setup = create()
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
        rc, s_ = P.smm_iterate(handle, x, 1e-300, 1, relative=True, raise_on_error=False)
        if rc not in (0, 7):
            raise P.SMMError(rc, P.load_library().smm_last_error().decode())
        return s_

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
        return sum(s_[key] for s_ in stats) / len(stats)

    ms_sweep, ms_src, ms_solve, ms_rhs = mean("ms_sweep"), mean("ms_residual"), mean("ms_solve"), mean("ms_rhs")
    cg_it = mean("cg_total")
    launches = int(sum(s_["n_launches"] for s_ in stats))
    hbm, hbm_src = load_peaks()
    cg_bytes = mg_cg_bytes_per_iter(ne, n)
    ms_iter = ms_solve / cg_it if cg_it > 0 else 0.0

    def entry(amount, ms_per_launch, kernel, traffic_key, launches_per_step, bound="hbm", peak=hbm, unit="GB/s",
              scale=1e9, peak_note=None):
        ach = amount / (ms_per_launch * 1e-3) / scale if ms_per_launch > 0 else 0.0
        return dict(bound=bound, achieved=ach, peak=peak, unit=unit, frac=ach / peak,
                    traffic=NCU_TRAFFIC.get(traffic_key), algorithmic=amount, ms=ms_per_launch,
                    launches_per_step=launches_per_step, kernel=kernel,
                    peak_note=peak_note or f"{hbm_src} copy bandwidth")

    sweep_kernel = (f"sweep_kernel<double, {WL['p']}, SOURCE, cached inverse>: the wavefront tasks, then the "
                    "element moments after the grid-wide gate")
    rooflines = {
        "cg_iteration": entry(cg_bytes, ms_iter, "one flexible-CG iteration: the operator product and the "
                              "multigrid V-cycle (level-0 Chebyshev smoothing, cluster coarse cycle), run inside "
                              "one device-side graph loop", "cg_iteration", cg_it),
        "sweep_kernel": entry(sweep_bytes(ne, nd, WL["p"], False), ms_sweep, sweep_kernel, "sweep_kernel", 1),
        "sweep_kernel_trace_bytes": entry(sweep_trace_bytes(ne, nd, WL["p"], 1), ms_sweep, sweep_kernel,
                                          None, 1),
        "sweep_kernel_fp32_issue": entry(sweep_fp32_ops(ne, nd, WL["p"]), ms_sweep, sweep_kernel, None, 1,
                                         bound="alu", peak=FP32_ISSUE_PEAK / 1e12, unit="T FP32 instr/s",
                                         scale=1e12, peak_note="152 SMs x 128 FP32 lanes x 2.07 GHz (one "
                                                               "instruction per lane per clock)"),
    }
    rooflines["sweep_kernel_trace_bytes"]["note"] = (
        "the bytes of a sweep that re-assembles each local system from geometry: this design reads "
        "a cached inverse per task instead (far more bytes, no per-sweep factorization)")
    # dominant: the largest device time per step among the kernels' own entries
    dom = max(("cg_iteration", "sweep_kernel"),
              key=lambda k: rooflines[k]["ms"] * rooflines[k]["launches_per_step"])
    roof = dict(rooflines[dom])
    roof["traffic"] = NCU_TRAFFIC.get(dom)

    # end to end through the C ABI with a host array: smm_iterate copies varphi^k in,
    # runs one outer step and copies varphi^{k+1} back, all inside the timed call
    host = np.zeros(ne * n)
    start_host = phi_start.cpu().numpy()
    e2e_ms = []
    with torch.cuda.stream(stream):
        for k in range(max(2, args.steps)):
            flush.fill_(1.0)
            host[:] = start_host
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, _ = P.smm_iterate(h, host, 1e-300, 1, relative=True, raise_on_error=False)
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e = dict(value=world * unknowns / (max_over_ranks(statistics.median(e2e_ms), dist, "cuda") * 1e-3),
               unit="unknowns/s", h2d_bytes_per_step=8 * ne * n, d2h_bytes_per_step=8 * ne * n,
               note="smm_iterate on a host array (wall clock, median of the steps)")

    extra = {}
    if not args.quick:
        extra.update(run_extras(args, P, torch, stream, create, step, phi, flush, ms_sweep))
    h.destroy()
    if args.learned_full:
        # the two-million-parameter network on 128 x 128 problems: 2000 training and 200 held-out solutions
        extra["learned_guess_full"] = run_learned(128, stream, 2000, 200, widths=(64, 384), steps=args.learned_steps,
                                                  configs=("plain", "learned_guess", "adaptive_inner_tol", "chosen"))
    if args.batch_full > 0:
        extra["batched_full"] = run_batch_full(stream, args.batch_full)

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = run_oracle_child(args.cpu_seconds, CPU_SAMPLE["nx"])
        cpu["cpu"] = cpu_model()
        cpu_all = run_oracle_all_cores(args.cpu_seconds, CPU_SAMPLE["nx"])

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64 accuracy: sweep products and right-hand side in FP32 pairs (f32x2), moments, CG and "
                     "checks in f64, multigrid smoother blocks in f32",
            "data": "synthetic",
            "config": {"workload": WL_NAME, "n_elem": ne, "p": WL["p"], "geom_order": 1, "sn": WL["sn"],
                       "n_ord": nd, "angular_unknowns": unknowns, "thick_blocks": int(thick.sum()),
                       "parallelism": f"replicas x{world}", "l2": "flushed between timed steps (256 MiB write)",
                       "sweep": "cached local inverses applied as FP32-pair products; moments in the sweep kernel",
                       "step_state": f"outer iteration {START_ITERATIONS + 1} from varphi^0 = 0, restored before "
                                     "every step",
                       "moment_solve": "flexible CG, multigrid V-cycle with degree-3 Chebyshev level-0 smoothing",
                       "cg_tol": 1e-12,
                       "cg_loop": "host-checked chunks" if args.host_cg_loop else "one device-side graph loop"},
            "roofline": roof, "roofline_all": rooflines, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all,
            "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary(),
            "phases_ms": dict(source=ms_src, sweep_with_moments=ms_sweep, rhs=ms_rhs, solve=ms_solve,
                              cg_iters=cg_it),
            "sweep_unknowns_per_s": dict(value=unknowns / (ms_sweep * 1e-3), unit="unknowns/s",
                                         ms=ms_sweep, note="one sweep including the fused moments (the sweep "
                                                           "kernel alone), per angular unknown"),
            "setup_s": t_setup, "inputs_s": t_in,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def time_steps(P, torch, stream, handle, x, flush, step, nsteps=4):
    """Mean time of nsteps outer steps from the state after two steps from zero."""
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
    ms = statistics.mean(t for t, _ in out)
    return dict(ms_per_step=ms, ms_sweep=statistics.mean(s_["ms_sweep"] for _, s_ in out),
                ms_residual_or_source=statistics.mean(s_["ms_residual"] for _, s_ in out),
                ms_solve=statistics.mean(s_["ms_solve"] for _, s_ in out))


def run_extras(args, P, torch, stream, create, step, phi, flush, ms_sweep_default) -> dict:
    import numpy as np

    extra = {}
    info = None

    def solve(**kw):
        hh, _ = create(**kw)
        x = torch.zeros_like(phi)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            rc, s_ = P.smm_iterate(hh, x, 1e-8, 300, relative=True, raise_on_error=False)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        hh.destroy()
        return dict(seconds=dt, status=rc, outer=s_["outer_iterations"], cg_total=s_["cg_total"],
                    cg_per_outer=s_["cg_total"] / max(1, s_["outer_iterations"]),
                    ms_sweep_per_outer=s_["ms_sweep"] / max(1, s_["outer_iterations"])), x

    d0, x0 = solve()
    da, xa = solve(anderson=2)
    da["rel_diff_vs_default"] = float((xa - x0).abs().max() / x0.abs().max())
    dc, xc = solve(moment=P.smm.SMM_MOMENT_CG)
    dc["rel_diff_vs_ip"] = float((xc - x0).abs().max() / x0.abs().max())
    dc["method"] = ("continuous finite element moment system (Sec. 5.1); differs from the IP solution by the "
                    "discretization error")
    # inexact moment solves: each to max(1e-12, 1e-2 x the previous step's relative difference)
    di, xi = solve(cg_adaptive=1e-2)
    di["rel_diff_vs_default"] = float((xi - x0).abs().max() / x0.abs().max())
    dai, xai = solve(anderson=2, cg_adaptive=1e-2)
    dai["rel_diff_vs_default"] = float((xai - x0).abs().max() / x0.abs().max())
    extra["time_to_1e-8"] = dict(workload=WL_NAME, default=d0, anderson2=da, cg_moment_system=dc,
                                 adaptive_inner_tol=di, anderson2_adaptive_inner_tol=dai,
                                 note="from varphi^0 = 0 to a 1e-8 relative successive difference; wall time "
                                      "of smm_iterate, setup excluded; adaptive_inner_tol: moment solves to "
                                      "max(1e-12, 1e-2 d_{k-1}) instead of 1e-12 (options.cg_tol_adaptive)")
    # the FP32-refined sweep (FP64 transport residual + FP32 correction sweep) on the same workload
    h32, _ = create(precision=P.SMM_SWEEP_FP32_REFINED)
    extra["fp32_refined_step"] = time_steps(P, torch, stream, h32, torch.zeros_like(phi), flush, step)
    h32.destroy()
    if args.cfg2:
        extra["mms_curved"] = run_mms_curved(P, torch, stream, flush, step)
    if args.batch > 0:
        extra["batched_sweep"] = run_batch(args.batch, stream)
    if args.learned > 0:
        extra["learned_guess"] = run_learned(args.learned, stream, args.learned_train, args.learned_test)
    return extra


def run_mms_curved(P, torch, stream, flush, step) -> dict:
    """The curved manufactured-solution workload (128x128 quads of geometry
    order 3, p = 4, S8, c = 0.9, MMS source and inflow): one outer step and
    the sweep alone."""
    om, _ = P.smm_quadrature(WL2["sn"])
    mesh, st, ss, q, inflow = workload_inputs(WL2["nx"], WL2["m"], WL2["p"], om, WL2["sigma_t"], WL2["c"],
                                              WL2["seed"])
    opt = P.smm_default_options()
    opt.tol_cg = 1e-12
    h = P.smm_create(mesh.nodes, mesh.elem_nodes, WL2["m"], WL2["p"], WL2["sn"], st, ss, q, inflow=inflow,
                     options=opt, stream=stream)
    info = h.info()
    x = torch.zeros(info.n_elem * info.n_dof_elem, dtype=torch.float64, device="cuda")
    r = time_steps(P, torch, stream, h, x, flush, step)
    r.update(workload=WL2_NAME, angular_unknowns=int(info.n_angular),
             value=info.n_angular / (r["ms_per_step"] * 1e-3),
             sweep_unknowns_per_s=info.n_angular / (r["ms_sweep"] * 1e-3), unit="unknowns/s")
    x.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        rc, s_ = P.smm_iterate(h, x, 1e-8, 300, relative=True, raise_on_error=False)
    torch.cuda.synchronize()
    r["time_to_1e-8"] = dict(seconds=time.perf_counter() - t0, status=rc, outer=s_["outer_iterations"],
                             cg_total=s_["cg_total"])
    h.destroy()
    # the same problem on the more strongly curved mesh (wave numbers up to 3 at amplitude 0.05 of the
    # domain): faces turn enough for grazing ordinates to cross them both ways, so the upwind graphs
    # have cycles, which are lagged.  Lagged inflow converges by one trip around a cycle per outer
    # step, damped by the cycle's optical path: in the thin medium (sigma_t = 1, cells 1/128 mfp) that
    # is slow, so it runs a bounded number of steps and reports the difference reached; the same mesh
    # with sigma_t = 100 runs to 1e-8.
    import numpy as np

    import smm_workloads as W
    mesh = W.structured_mesh(WL2["nx"], m=WL2["m"], perturb_seed=WL2["seed"], wave_max=3, scale_by_k=False)
    r["strongly_curved_cycles_lagged"] = {}
    # (the thin medium also with Anderson acceleration of depth 5: the lagged inflow converges linearly,
    # with a few slow modes, which is what Anderson mixing removes)
    for key, sig, max_outer, depth in (("sigma_t=1", WL2["sigma_t"], 100, 0), ("sigma_t=1_anderson5", WL2["sigma_t"], 100, 5),
                                       ("sigma_t=100", 100.0, 300, 0)):
        q, inflow = workload_sources(mesh, WL2["p"], om, sig, WL2["c"])
        stl = np.full(mesh.n_elem, sig)
        opt.anderson_depth = depth
        h = P.smm_create(mesh.nodes, mesh.elem_nodes, WL2["m"], WL2["p"], WL2["sn"], stl, stl * WL2["c"], q,
                         inflow=inflow, options=opt, stream=stream)
        info = h.info()
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            rc, s_ = P.smm_iterate(h, x, 1e-8, max_outer, relative=True, raise_on_error=False)
        torch.cuda.synchronize()
        r["strongly_curved_cycles_lagged"][key] = dict(
            seconds=time.perf_counter() - t0, status=rc, outer=s_["outer_iterations"], max_outer=max_outer,
            last_rel_diff=s_["last_rel_diff"], cg_total=s_["cg_total"], lagged_face_ordinates=int(info.n_lagged),
            levels=int(info.n_levels), ms_sweep_per_outer=s_["ms_sweep"] / max(1, s_["outer_iterations"]))
        h.destroy()
    opt.anderson_depth = 0
    return r


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
    problems swept one at a time (the default sweep: cached inverses applied
    in FP32-pair arithmetic, moments in the sweep kernel)."""
    import torch

    import paper_2304_07386_gb300 as P

    hs, unknowns = [], 0
    for i in range(nprob):
        mesh, p, sn, st, ss, q = batch_problem(i)
        opt = P.smm_default_options()
        opt.precond = P.smm.SMM_PRECOND_BLOCK_JACOBI  # only sweeps are timed: skip the multigrid setup
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
                schedule=sched, note="wall time of one smm_batch_sweep launch vs consecutive smm_sweep calls (each "
                                     "with its source kernel, sweep kernel and one host sync); best of 3")


def batch_full_problem(seed: int):
    """One problem of the uneven batched-instances workload at its full size:
    n ~ U{32..192}, p ~ U{1..4}, S_N ~ U{4,6,8,10,12}, sigma_t = 10 exp(1.5 g)
    with g a unit Gaussian random field (correlation length 0.1), c ~
    U[0.5, 0.99], q = 1 per steradian, vacuum, straight mesh."""
    import numpy as np

    import smm_workloads as W

    rng = np.random.default_rng(5000 + seed)
    nx = int(rng.integers(32, 193))
    p = int(rng.integers(1, 5))
    sn = int(rng.choice([4, 6, 8, 10, 12]))
    c = float(rng.uniform(0.5, 0.99))
    mesh = W.structured_mesh(nx, m=1)
    st = 10.0 * np.exp(1.5 * W.gaussian_random_field(nx, 0.1, 5000 + seed))
    return mesh, p, sn, st, c * st, np.ones((mesh.n_elem, (p + 1) ** 2))


def run_batch_full(stream, nprob: int = 256, wave_bytes: float = 150e9) -> dict:
    """All nprob uneven problems solved to a 1e-8 relative successive
    difference with the default FP64-accuracy method (cached pair inverses,
    multigrid CG).  Their cached inverses together exceed the GPU's memory, so
    the problems go in waves whose estimated device footprint stays below
    wave_bytes; each wave is created, iterated as one batch (one sweep launch
    per outer step for all its problems) and destroyed."""
    import numpy as np
    import torch

    import paper_2304_07386_gb300 as P

    def footprint(nx, p, sn):
        n, nd, ne = (p + 1) ** 2, sn * (sn + 2) // 2, nx * nx
        return ne * nd * (8 * n * n + 8 * n + 16) + ne * 48 * 1024

    specs = []
    for i in range(nprob):
        rng = np.random.default_rng(5000 + i)
        nx, p = int(rng.integers(32, 193)), int(rng.integers(1, 5))
        sn = int(rng.choice([4, 6, 8, 10, 12]))
        specs.append((i, footprint(nx, p, sn)))
    waves, cur, used = [], [], 0.0
    for i, b in specs:
        if cur and used + b > wave_bytes:
            waves.append(cur)
            cur, used = [], 0.0
        cur.append(i)
        used += b
    waves.append(cur)
    total_unknowns, t_setup, t_iter, outer, converged, statuses = 0, 0.0, 0.0, [], 0, []
    for wave in waves:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hs = []
        for i in wave:
            mesh, p, sn, st, ss, q = batch_full_problem(i)
            opt = P.smm_default_options()
            opt.tol_cg = 1e-12
            hs.append(P.smm_create(mesh.nodes, mesh.elem_nodes, 1, p, sn, st, ss, q, options=opt, stream=stream))
        b = P.smm.smm_batch_create(hs)
        phis = [torch.zeros(h.info().n_elem * h.info().n_dof_elem, dtype=torch.float64, device="cuda") for h in hs]
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        status = 0
        try:
            with torch.cuda.stream(stream):
                stats = P.smm.smm_batch_iterate(b, phis, 1e-8, 300, relative=True)
        except P.smm.SMMError as ex:  # e.g. a problem not converged in 300 steps
            status, stats = ex.status, []
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        t_setup += t1 - t0
        t_iter += t2 - t1
        statuses.append(status)
        for h in hs:
            total_unknowns += h.info().n_angular
        for s_ in stats:
            outer.append(s_["outer_iterations"])
            converged += int(s_["last_rel_diff"] <= 1e-8)
        b.destroy()
        for h in hs:
            h.destroy()
        del phis
        torch.cuda.empty_cache()
    return dict(problems=nprob, waves=len(waves), problems_per_wave=[len(w) for w in waves],
                angular_unknowns_per_sweep=total_unknowns, setup_s=t_setup, iterate_s=t_iter,
                outer_mean=float(np.mean(outer)) if outer else None, outer_max=max(outer) if outer else None,
                converged=converged, wave_status=statuses,
                note="time to a 1e-8 relative difference for every problem, batched per wave (setup excluded)")


def network_flops(nx: int, n_out: int, c1: int, c2: int) -> float:
    """Algorithmic FLOPs of one sample's forward pass (2 per multiply-add over
    the real channels of every layer; the half-resolution layers on nx/2)."""
    full, half = nx * nx, (nx // 2) ** 2
    macs = 9 * 3 * c1 * full + 9 * c1 * c2 * half + 9 * c2 * c2 * half + 9 * c2 * c1 * full + \
        9 * 2 * c1 * c1 * full + c1 * n_out * full
    return 2.0 * macs


def run_learned(nx: int, stream, n_train: int = 192, n_test: int = 16, p: int = 2, sn: int = 8,
                widths=(24, 32), steps: int = 1500, configs=None) -> dict:
    """Learned-guess workload (p=2, S8, log-normal sigma_t / sigma_s fields,
    piecewise-constant source maps, on an nx*nx grid of quads): train the
    library's network on n_train converged solutions the method produces,
    then solve n_test held-out problems to a 1e-8 relative difference.

    plain: each problem on its own with the library's default FP64-accuracy
    path (cached inverses, multigrid CG) from the zero guess.  chosen: all
    problems in one batched iteration (one sweep launch per outer step for
    all of them), each started from the network's proposal (guess_check on)
    with Anderson acceleration of depth 2 and inexact moment solves (to
    1e-2 of the previous relative difference).  The ablations switch one
    ingredient at a time.  Times are wall times of the solves (network
    inference included, handle setup excluded)."""
    import numpy as np
    import torch

    import paper_2304_07386_gb300 as P
    import smm_workloads as W
    from paper_2304_07386_gb300 import guess as G

    n = (p + 1) ** 2

    def make(seed, check=False, anderson=0, adaptive=0.0):
        mesh, st, ss, qe = W.learned_guess_problem(nx, seed)
        opt = P.smm_default_options()
        opt.tol_cg = 1e-12
        opt.guess_check = int(check)
        opt.anderson_depth = anderson
        opt.cg_tol_adaptive = adaptive
        h = P.smm_create(mesh.nodes, mesh.elem_nodes, 1, p, sn, st, ss, np.repeat(qe[:, None], n, axis=1),
                         options=opt, stream=stream)
        return h, (st, ss, qe)

    def zeros():
        return torch.zeros(nx * nx * n, dtype=torch.float64, device="cuda")

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            r = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, r

    t_gen = time.perf_counter()
    X, Y = [], []
    for seed in range(n_train):
        h, (st, ss, qe) = make(seed)
        x = zeros()
        with torch.cuda.stream(stream):
            P.smm_iterate(h, x, 1e-10, 300, relative=True, raise_on_error=False)
        h.destroy()
        X.append(G.features(st, ss, qe, nx))
        Y.append(G.targets(x.cpu().numpy(), nx, n))
    t_gen = time.perf_counter() - t_gen
    X, Y = np.stack(X), np.stack(Y)
    xn, yn = G.Normalizer(X), G.Normalizer(Y)
    c1, c2 = widths
    net = P.smm.Guess(nx, nx, n, 16, seed=0, stream=stream, c1=c1, c2=c2)
    Xd, Yd = torch.as_tensor(xn.fwd(X), device="cuda"), torch.as_tensor(yn.fwd(Y), device="cuda")
    t_train = time.perf_counter()
    with torch.cuda.stream(stream):
        losses = G.train(net, Xd, Yd, steps=steps, batch=16, lr=3e-3 if c2 <= 64 else 1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t_train
    # the network's passes alone on a resident batch of 16 (CUDA events on the network's stream):
    # forward, and forward + backward (gradients, no update)
    fl = network_flops(nx, n, c1, c2)
    xb, yb = Xd[:16].contiguous(), Yd[:16].contiguous()
    out = torch.zeros((16, n, nx, nx), dtype=torch.float32, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    with torch.cuda.stream(stream):
        for _ in range(3):
            net.forward(xb, out)
        ev[0].record(stream)
        for _ in range(10):
            net.forward(xb, out)
        ev[1].record(stream)
        for _ in range(3):
            net.gradients(xb, yb)
        ev[2].record(stream)
        for _ in range(10):
            net.gradients(xb, yb)
        ev[3].record(stream)
    torch.cuda.synchronize()
    ms_fwd = ev[0].elapsed_time(ev[1]) / 10
    ms_fb = ev[2].elapsed_time(ev[3]) / 10
    peak_tensor, peak_src = load_tensor_peak()
    network = dict(widths=[c1, c2], params=net.n_params, batch=16, forward_ms=ms_fwd, forward_backward_ms=ms_fb,
                   forward_tflops=16 * fl / ms_fwd * 1e-9, forward_backward_tflops=16 * 3 * fl / ms_fb * 1e-9,
                   train_steps=steps, train_step_tflops_wall=steps * 16 * 3 * fl / t_train * 1e-12,
                   roofline=dict(bound="tensor", achieved=16 * 3 * fl / ms_fb * 1e-9, peak=peak_tensor,
                                 unit="TFLOP/s", frac=16 * 3 * fl / ms_fb * 1e-9 / peak_tensor, peak_source=peak_src,
                                 note="algorithmic FLOPs (real channels, forward x 3 for forward + backward) of the "
                                      "mma.sync BF16 implicit-GEMM passes over their measured time (loss, "
                                      "repacking and reductions included), against the measured cuBLAS BF16 peak"))

    seeds = list(range(100_000, 100_000 + n_test))

    def proposals(infos):
        out = []
        for st, ss, qe in infos:
            xg = torch.as_tensor(xn.fwd(G.features(st, ss, qe, nx)[None]), device="cuda")
            out.append(torch.as_tensor(G.predict_phi(net, xg, yn, nx, n), device="cuda"))
        return out

    def singles(check, anderson, learned, adaptive=0.0):
        hs = [make(sd, check=check, anderson=anderson, adaptive=adaptive) for sd in seeds]
        xs = [zeros() for _ in seeds]

        def run():
            if learned:
                for x, g in zip(xs, proposals([i for _, i in hs])):
                    x.copy_(g)
            st_ = []
            for (h, _), x in zip(hs, xs):
                rc, s_ = P.smm_iterate(h, x, 1e-8, 300, relative=True, raise_on_error=False)
                st_.append((rc, s_))
            return st_
        dt, st_ = timed(run)
        for h, _ in hs:
            h.destroy()
        return dt, st_, xs

    def batched(check, anderson, learned, adaptive=0.0):
        hs = [make(sd, check=check, anderson=anderson, adaptive=adaptive) for sd in seeds]
        b = P.smm.smm_batch_create([h for h, _ in hs])
        xs = [zeros() for _ in seeds]

        def run():
            if learned:
                for x, g in zip(xs, proposals([i for _, i in hs])):
                    x.copy_(g)
            return P.smm.smm_batch_iterate(b, xs, 1e-8, 300, relative=True)
        dt, st_ = timed(run)
        b.destroy()
        for h, _ in hs:
            h.destroy()
        return dt, [(0, s_) for s_ in st_], xs

    rows = {}
    ref = None
    for name, fn, kw in (("plain", singles, dict(check=False, anderson=0, learned=False)),
                         ("batched", batched, dict(check=False, anderson=0, learned=False)),
                         ("learned_guess", singles, dict(check=True, anderson=0, learned=True)),
                         ("anderson2", singles, dict(check=False, anderson=2, learned=False)),
                         ("adaptive_inner_tol", singles, dict(check=False, anderson=0, learned=False, adaptive=1e-2)),
                         ("chosen", batched, dict(check=True, anderson=2, learned=True, adaptive=1e-2))):
        if configs is not None and name not in configs:
            continue
        dt, st_, xs = fn(**kw)
        if ref is None:
            ref = xs
        rows[name] = dict(seconds=dt, mean_outer=float(np.mean([s_["outer_iterations"] for _, s_ in st_])),
                          rejected=int(sum(s_["guess_rejected"] for _, s_ in st_)),
                          all_converged=all(rc == 0 for rc, _ in st_),
                          max_rel_diff_vs_plain=max(float((x - r).abs().max() / r.abs().max())
                                                    for x, r in zip(xs, ref)))
    return dict(grid=f"{nx}x{nx}", p=p, sn=sn, train_problems=n_train, test_problems=n_test,
                params=net.n_params, network=network, data_gen_s=t_gen, train_s=t_train,
                final_loss=float(np.mean(losses[-50:])),
                initial_loss=float(np.mean(losses[:10])), **rows,
                speedup_chosen_vs_plain=(rows["plain"]["seconds"] / rows["chosen"]["seconds"]
                                         if "plain" in rows and "chosen" in rows else None),
                note="wall time to a 1e-8 relative successive difference for all held-out problems; plain = the "
                     "default FP64-accuracy method one problem at a time from zero; chosen = learned guess "
                     "(guess_check) + one batched sweep launch per outer step + Anderson depth 2 + moment "
                     "solves to max(1e-12, 1e-2 x the previous relative difference)")


def run_network_passes(batch: int, nx: int = 128, n_out: int = 9, widths=(64, 384)) -> None:
    """The learned guess's network alone (the two-million-parameter widths on
    nx x nx grids): forward, forward + backward (gradients), and a training
    step (gradients + Adam), each 3 warm-up and 10 timed calls with CUDA events
    on the network's stream, on seeded normal inputs and targets resident on
    the GPU.  Prints one JSON line."""
    import torch

    import paper_2304_07386_gb300 as P
    from paper_2304_07386_gb300 import build as B
    B.build()
    c1, c2 = widths
    stream = torch.cuda.current_stream()
    net = P.smm.Guess(nx, nx, n_out, batch, seed=0, stream=stream, c1=c1, c2=c2)
    gen = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(batch, 3, nx, nx, device="cuda", generator=gen)
    t = torch.randn(batch, n_out, nx, nx, device="cuda", generator=gen)
    out = torch.zeros(batch, n_out, nx, nx, device="cuda")
    fl = network_flops(nx, n_out, c1, c2)
    peak, src = load_tensor_peak()
    res = dict(grid=f"{nx}x{nx}", batch=batch, widths=[c1, c2], params=net.n_params)
    for name, fn, mult in (("forward", lambda: net.forward(x, out), 1),
                           ("forward_backward", lambda: net.gradients(x, t), 3),
                           ("train_step", lambda: net.train_step(x, t, 1e-4), 3)):
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(10):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 10
        tf = batch * mult * fl / ms * 1e-9
        res[name] = dict(ms=ms, tflops=tf, frac_of_bf16_peak=tf / peak)
    res["peak_tflops"] = peak
    res["peak_source"] = src
    print(json.dumps({"network_passes": res}))


def run_reference(args) -> None:
    """The oracle arm: the CPU oracle on the host cores, K timed steps of a
    bounded sample of the headline workload (one outer step each), after W
    warm-up steps."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    import numpy as np

    from oracle.smm import SMMProblem
    from oracle.transport import Discretization

    c = CPU_SAMPLE
    mesh, st, ss, q, _ = thick_thin_inputs(c["nx"], c["blocks"], WL["p"], WL["seed"], c["length"])
    disc = Discretization(mesh.nodes, mesh.elem_nodes, 1, WL["p"], WL["sn"], st, ss)
    prob = SMMProblem(disc, q)
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
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "unknowns/s", "n_gpus": 0, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WL_NAME, "sample_mesh": f"{c['nx']}x{c['nx']}", "angular_unknowns": unknowns},
        "cpu_baseline": {"value": value, "unit": "unknowns/s", "cores": 1, "kind": "oracle",
                         "sample": cpu_sample_text(), "cpu": cpu_model()},
        "e2e": {"value": value, "unit": "unknowns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="the headline line only (no extras)")
    ap.add_argument("--host-cg-loop", action="store_true",
                    help="launch the CG iterations from the host in chunks instead of one device-side loop graph "
                         "(profiling runs: ncu does not see kernels inside conditional graph nodes)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--nx", type=int, default=WL["nx"], help="mesh size override (profiling runs)")
    ap.add_argument("--no-cfg2", dest="cfg2", action="store_false", help="skip the curved MMS workload")
    ap.add_argument("--batch", type=int, default=24, help="problems in the batched-sweep measurement (0: skip)")
    ap.add_argument("--learned", type=int, default=64, help="element grid of the learned-guess measurement (0: skip)")
    ap.add_argument("--learned-train", type=int, default=192, help="training problems of the learned guess")
    ap.add_argument("--learned-test", type=int, default=16, help="held-out problems of the learned guess")
    ap.add_argument("--learned-full", action="store_true",
                    help="the learned guess at full size (128x128, p = 2, S8, 2000 training and 200 held-out "
                         "problems, the two-million-parameter network; opt-in: about a quarter of an hour; also "
                         "with --quick)")
    ap.add_argument("--learned-steps", type=int, default=3000, help="training steps of --learned-full")
    ap.add_argument("--batch-full", type=int, default=0,
                    help="problems of the full-size uneven batched workload solved to 1e-8 in memory-sized waves "
                         "(opt-in: about ten minutes for 256)")
    ap.add_argument("--network-passes", type=int, default=0,
                    help="time only the learned guess's two-million-parameter network on 128x128 grids at this "
                         "batch (forward, forward + backward, training step) and exit")
    args = ap.parse_args()
    if args.network_passes > 0:
        run_network_passes(args.network_passes)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
