#!/usr/bin/env python
"""Benchmark of the fully explicit projection timestep on GB300.

One step = one full FP64 timestep (Sec. 2, Eqs. 3-7) on the 512 x 384 x 512 channel (Lx = 2 pi,
Ly = 2, Lz = pi, tanh stretching 2.0): the two stages of Heun's RK2 momentum predictor (central
advection and diffusion, nu = 1/550, body force 2 nu), then the projection: the divergence of u*
fused into the forward x-FFT, the forward z-FFT, the PDD wall-normal solves (P = 8, exact
reduced system), the (0, 0) mode, the inverse z- and x-FFTs, and the gradient correction.
Input: laminar Poiseuille profile plus seeded N(0, 0.1^2) noise (seed 1), no-penetration walls,
dt = 1e-4.

Metric: grid points per second of whole timesteps (Gpts/s) and ms/timestep; the Poisson solve's
own throughput (the projection's kernels) is reported beside it.  The fields (2.4 GB of velocity,
2.4 GB of stage scratch, 0.8 GB spectrum) are far larger than the 129 MB L2, so no flush is
needed between steps.

--impl reference times the CPU oracle (numpy, FP64) on a bounded sample of the same workload.
Under torchrun every rank runs an independent replica (the path is replicas-only on this pool).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

CASE = W.CHANNEL_512
PDD_PARTS = 8
DT = 1e-4
NU = 1.0 / 550.0
FX = 2.0 * NU      # body force that keeps u = 1 - y^2 steady in the continuum
METRIC = ("Poisson solve Gpts/s & ms/timestep (FP64 full timestep: RK2 momentum predictor + "
          "projection = divergence + FFT/PDD solve + gradient)")
UNIT = "Gpts/s"


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu if isinstance(gpu, int) else (str(gpu) if str(gpu).startswith("GPU-") else f"GPU-{gpu}")
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------- ranks
def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over all ranks (identity without an initialised process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = device if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world: int, points_per_rank: int, ms_per_step: float) -> float:
    """Whole-job Gpts/s of N independent replicas timed by the slowest rank."""
    return world * points_per_rank / (ms_per_step * 1e-3) / 1e9


# ------------------------------------------------------------------------------- roofline model
def kernel_model(name: str, nx: int, ny: int, nz: int):
    """Algorithmic HBM bytes and FFT flops of one launch of each FP64 projection kernel.

    N = nx ny nz real points, Ns = (nx/2 + 1) ny nz complex modes (16 bytes each in FP64).
    FFT flops use the 5 n log2 n convention for an n-point complex transform (2.5 n log2 n
    for an n-point real transform).
    """
    N = nx * ny * nz
    Ns = (nx // 2 + 1) * ny * nz
    plane = nx * nz
    if name == "fwd_x_div":    # read u, v (ny+1 planes), w; write the half spectrum
        return 8 * (3 * N + plane) + 16 * Ns, 2.5 * N * math.log2(nx)
    if name in ("fft_z_fwd", "fft_z_inv"):
        return 32 * Ns, 5.0 * Ns * math.log2(nz)
    if name == "tridiag_pdd":
        return 32 * Ns, 0.0
    if name == "inv_x":        # read the half spectrum, write p
        return 16 * Ns + 8 * N, 2.5 * N * math.log2(nx)
    if name == "gradient":     # read p, u, v, w; write u, v, w
        return 8 * N + 2 * 8 * (3 * N + plane), 0.0
    if name == "momentum_1":   # read u, v, w; write u_bar
        return 2 * 8 * (3 * N + plane), momentum_flops_per_point(1) * N
    if name == "momentum_2":   # read u_bar (stencil) and u (pointwise); write u_star
        return 3 * 8 * (3 * N + plane), momentum_flops_per_point(2) * N
    return 0, 0.0


def momentum_flops_per_point(stage: int) -> float:
    """Algorithmic FP64 flops per grid point of one Heun stage (Eqs. 3, 5, 6), counted from the
    discrete operators (an FMA is 2 flops), with every face or edge flux evaluated once and shared
    by the two cells (or the two momentum equations) it serves:

    * advection, divergence form with two-point averages, per component: the flux on its own face
      ((a + b)/2 squared: add, two multiplies = 3) and half of each of the two edge fluxes it
      shares with another component (two averages and a product with the 1/4 folded in: 4, half
      of it per equation: 2 + 2), then the divergence of the three fluxes (three differences
      scaled by 1/dx, 1/dy_j, 1/dz and summed: 3 + 3 + 2 = 8): 15;
    * diffusion: x and z second differences ((p+ + p-) - 2 p scaled: 3 each), the stretched-y
      difference (c_j (p+ - p) - a_j (p - p-): 4), their sum (2) and the factor nu (1): 13;
    * the body force (x component only: 1 flop per point in total) and the Heun update
      (stage 1: u + dt R, one FMA = 2 per component; stage 2: (u + u_bar + dt R)/2, one FMA, one
      add and a multiply = 4 per component).
    Three components: 3 (15 + 13) + 1 + (6 or 12) = 91 (stage 1) or 97 (stage 2)."""
    per_component = 15 + 13
    heun = 2 if stage == 1 else 4
    return 3 * per_component + 1 + 3 * heun


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except (OSError, ValueError):
        return {}


# DRAM bytes (read + write) of one fwd_x launch, from an ncu capture of the same kernel on the
# 256x192x256 projection, scaled by the number of points (x 8.0) to the 512x384x512 launch; the
# capture also shows the FP64 pipe 86 % busy.  Valid for the kernel as captured.
FWD_X_FP64_TRAFFIC = {"bytes": 3.05e9, "ncu_fp64_pipe_active_pct": 85.9,
                      "source": "ncu capture at 256x192x256 scaled x8 by points"}

# DRAM traffic of the momentum stages from an ncu capture of the same kernels on the 256x192x256
# timestep, scaled by the number of points (x 8.0) to the 512x384x512 launches; the capture shows
# the FP64 pipe 89 % busy.  Valid for the kernel as captured.
KERNEL_TRAFFIC = {
    "momentum_1": {"bytes": 4.58e9, "ncu_fp64_pipe_active_pct": 88.9,
                   "source": "ncu capture at 256x192x256 scaled x8 by points"},
    "momentum_2": {"bytes": 7.00e9, "ncu_fp64_pipe_active_pct": 89.1,
                   "source": "ncu capture at 256x192x256 scaled x8 by points"},
}

# ------------------------------------------------------------------------------- CPU oracle
SAMPLE_NX, SAMPLE_NZ = 64, 64   # the oracle's sample: the bench's wall-normal grid on a 64 x 64 plane


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_sample(seconds: float = 12.0):
    """Time the CPU oracle's full timestep on a sample of the workload (same Ny, stretching, dt).

    The sample keeps the wall-normal grid (Ny = 384, tanh 2.0) and shrinks the periodic plane
    to 64 x 64; the oracle is repeated until about `seconds` have passed.  Returns Gpts/s and the
    seconds per sample timestep.
    """
    import oracle
    nx, nz = SAMPLE_NX, SAMPLE_NZ
    faces = W.tanh_faces(CASE.ny, CASE.stretch)
    g = oracle.Grid(nx, nz, faces, CASE.lx, CASE.lz)
    sample = W.ChannelCase("sample", nx, CASE.ny, nz, CASE.stretch)
    u, v, w = W.poiseuille_plus_noise(1, sample)
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.timestep(g, u, v, w, DT, NU, FX)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    pts = reps * nx * nz * CASE.ny
    return {"value": pts / el / 1e9, "s_per_step": el / reps, "reps": reps, "seconds": el}


def _oracle_worker(seconds):
    return oracle_sample(seconds)


def cpu_baseline(seconds: float = 12.0):
    """The oracle as it stands, timed on the host: one process, then one process per core (spawned,
    each single-threaded, all running the same sample at once; the whole-host throughput is the sum).
    """
    import multiprocessing as mp
    ncores = os.cpu_count() or 1
    one = oracle_sample(seconds)
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(ncores) as pool:
            res = pool.map(_oracle_worker, [seconds] * ncores)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    total = sum(r["value"] for r in res)
    return {"value": total, "unit": UNIT, "cores": ncores, "kind": "oracle", "cpu": cpu_model(),
            "single_thread_value": one["value"],
            "sample": f"oracle.timestep (RK2 predictor + projection) on {SAMPLE_NX}x{CASE.ny}x{SAMPLE_NZ} (same "
                      f"Ny=384 tanh 2.0 wall-normal grid), numpy FP64 FFT + extended-precision Thomas; one "
                      f"process: {one['reps']} steps in {one['seconds']:.1f} s; then {ncores} single-threaded "
                      f"processes at once for ~{seconds:.0f} s each, throughput summed"}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample(seconds=0.5)
    steps = [oracle_sample(seconds=4.0) for _ in range(args.steps)]
    value = statistics.median(s["value"] for s in steps)
    s_step = statistics.median(s["s_per_step"] for s in steps)
    sample = (f"oracle.timestep on {SAMPLE_NX}x{CASE.ny}x{SAMPLE_NZ} (the bench's Ny=384 tanh 2.0 wall-normal "
              f"grid on a 64x64 plane), 1 thread; each step = repeated sample timesteps for ~4 s")
    cfg = config_dict()
    cfg["reference_sample"] = {"grid": [SAMPLE_NX, CASE.ny, SAMPLE_NZ], "note": "the oracle runs this sample; "
                               "value is its Gpts/s, ms_per_step the sample's time per timestep"}
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": s_step * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": cfg,
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu": cpu_model(),
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def config_dict():
    return {"workload": f"{CASE.name} FP64 full timestep (RK2 predictor + projection)",
            "grid": [CASE.nx, CASE.ny, CASE.nz],
            "pdd_parts": PDD_PARTS, "tridiag": "PDD, exact reduced system", "dt": DT, "nu": NU, "fx": FX,
            "input": "Poiseuille 1-y^2 + N(0,0.1^2) seed 1, walls v=0",
            "l2": "no flush: fields 2.4 GB (+2.4 GB stage scratch) >> 129 MB L2", "parallelism": "replicas"}


# ------------------------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_2104_08863_gb300 import build as b
    b.build()
    import paper_2104_08863_gb300 as P

    faces = W.tanh_faces(CASE.ny, CASE.stretch)
    mk = lambda flags: P.Plan(CASE.nx, CASE.ny, CASE.nz, faces, CASE.lx, CASE.lz, precision=P.PP_FP64,
                              tridiag=P.PT_PDD_EXACT, pdd_parts=PDD_PARTS, flags=flags, device=dev)
    plan = mk(0)                         # the timed loop: no per-launch events
    u0, v0, w0 = W.poiseuille_plus_noise(1, CASE)
    u, v, w = (torch.from_numpy(a).to(dev) for a in (u0, v0, w0))
    p = torch.empty(CASE.ny, CASE.nz, CASE.nx, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    fp64_gflops = P.fp64_fma_rate(dev)   # the FP64 roofline denominator, measured now on this GPU

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    scratch = (torch.empty_like(u), torch.empty_like(v), torch.empty_like(w))
    for _ in range(args.warmup):
        plan.timestep(u, v, w, DT, NU, FX, p_out=p, scratch=scratch)
    launches_per_step = plan.last_launch_count
    barrier()
    clocks = ClockSampler(torch.cuda.get_device_properties(dev).uuid if hasattr(
        torch.cuda.get_device_properties(dev), "uuid") else local)
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        plan.timestep(u, v, w, DT, NU, FX, p_out=p, scratch=scratch)
    e1.record(stream)
    barrier()
    ms_total = e0.elapsed_time(e1)
    clk = clocks.stop()
    ms_step = max_over_ranks(ms_total / args.steps, dev)
    value = replica_throughput(world, CASE.npoints, ms_step)

    # per-kernel device times: a second pass of the same steps on a plan that records an event pair
    # around every launch (untimed for the headline), continuing from the same state
    tplan = mk(P.POISSON_TIMING)
    stage = {}
    for it in range(args.steps + 1):
        tplan.timestep(u, v, w, DT, NU, FX, p_out=p, scratch=scratch)
        rec = tplan.stage_times()
        if it == 0:
            continue   # the timing plan's first step warms its events
        for name, ms in rec:
            stage.setdefault(name, []).append(ms)
    del tplan
    proj_ms = sum(sum(vs) for k, vs in stage.items() if not k.startswith("momentum")) / args.steps
    mom_ms = sum(sum(vs) for k, vs in stage.items() if k.startswith("momentum")) / args.steps
    poisson = {"gpts": replica_throughput(world, CASE.npoints, max_over_ranks(proj_ms, dev)),
               "projection_ms": proj_ms, "momentum_ms": mom_ms,
               "note": "sums of per-launch event times of a second pass of the same steps"}

    # dominant kernel and its roofline
    totals = {k: sum(vs) for k, vs in stage.items()}
    dom = max(totals, key=totals.get)
    launches = len(stage[dom])
    avg_ms = totals[dom] / launches
    nbytes, flops = kernel_model(dom, CASE.nx, CASE.ny, CASE.nz)
    peaks = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    t_hbm = nbytes / (hbm_peak * 1e9)
    t_alu = flops / (fp64_gflops * 1e9)
    if t_alu > t_hbm:
        achieved = flops / (avg_ms * 1e-3) / 1e12
        tr = FWD_X_FP64_TRAFFIC if dom == "fwd_x_div" else KERNEL_TRAFFIC.get(dom)
        roof = {"bound": "alu", "achieved": achieved, "peak": fp64_gflops / 1e3, "unit": "TFLOP/s",
                "frac": achieved / (fp64_gflops / 1e3), "traffic": tr["bytes"] if tr else None,
                "traffic_source": tr["source"] if tr else None,
                "ncu_fp64_pipe_active_pct": tr["ncu_fp64_pipe_active_pct"] if tr else None, "kernel": dom,
                "peak_source": "FP64 FMA throughput measured in this run by the library's diagnostics kernel "
                               "(poisson_fp64_fma_rate, 2 flops per FMA)",
                "flops_per_point": flops / CASE.npoints,
                "flops_source": "algorithmic count of the discrete operators (bench.momentum_flops_per_point)",
                "hbm_achieved_gbs": nbytes / (avg_ms * 1e-3) / 1e9}
    else:
        achieved = nbytes / (avg_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None, "kernel": dom,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    roof["avg_launch_ms"] = avg_ms
    share = {k: round(v / sum(totals.values()), 4) for k, v in sorted(totals.items(), key=lambda kv: -kv[1])}

    # end to end through the host-buffer C-ABI entry point (pinned host memory)
    uh, vh, wh = (torch.from_numpy(a).pin_memory() for a in (u0, v0, w0))
    ph = torch.empty(CASE.ny, CASE.nz, CASE.nx, dtype=torch.float64).pin_memory()
    staging = (u, v, w, p)
    plan.timestep_host(uh, vh, wh, DT, NU, FX, staging, scratch, p_h=ph)
    e2e_steps = max(1, min(args.steps, 5))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        plan.timestep_host(uh, vh, wh, DT, NU, FX, staging, scratch, p_h=ph)
    barrier()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dev)
    h2d = 8 * (3 * CASE.npoints + CASE.nx * CASE.nz)
    d2h = h2d + 8 * CASE.npoints
    del uh, vh, wh, ph, staging, scratch, u, v, w, p, plan
    torch.cuda.empty_cache()

    forms = precision_forms(dev) if (world == 1 and not args.no_forms) else None
    ts_forms = timestep_forms(dev) if (world == 1 and not args.no_forms) else None
    batch = batch_form(dev) if (world == 1 and not args.no_forms) else None
    cpu = cpu_baseline() if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_dict(),
               "roofline": roof, "kernel_share": share, "poisson_solve": poisson,
               "cpu_baseline": cpu,
               "e2e": {"value": world * CASE.npoints / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "steps": e2e_steps},
               "gpu_launches": launches_per_step * args.steps, "clocks": clk, "precision_forms": forms,
               "timestep_forms": ts_forms, "batch_form": batch}
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


def timestep_forms(dev, steps: int = 5, warmup: int = 3):
    """The bench timestep in FP64 and in the FP32-refined form (double-float momentum and
    divergence on FP32 pairs, two-correction Poisson solve) on the 512 x 384 x 512 channel.

    Both start from the bench's initial state; after one timestep the refined form's velocity and
    pressure are compared with the FP64 form's (max |difference| / max |FP64|).  Each form is
    then timed over `steps` further timesteps with CUDA events (stage times from a separate pass).
    """
    import torch
    import paper_2104_08863_gb300 as P
    faces = W.tanh_faces(CASE.ny, CASE.stretch)
    u0, v0, w0 = W.poiseuille_plus_noise(1, CASE)
    out = {"workload": f"{CASE.name} full timestep from the bench's initial state"}
    ref = None
    for name, prec in (("fp64", P.PP_FP64), ("fp32_refined", P.PP_FP32_REFINED)):
        kw = dict(tridiag=P.PT_PDD_EXACT, pdd_parts=PDD_PARTS) if prec == P.PP_FP64 else dict(refine_steps=2)
        mk = lambda flags: P.Plan(CASE.nx, CASE.ny, CASE.nz, faces, CASE.lx, CASE.lz, precision=prec, flags=flags,
                                  device=dev, **kw)
        plan = mk(0)
        u, v, w = (torch.from_numpy(a).to(dev) for a in (u0, v0, w0))
        p = torch.empty(CASE.ny, CASE.nz, CASE.nx, dtype=torch.float64, device=dev)
        scratch = (torch.empty_like(u), torch.empty_like(v), torch.empty_like(w))
        plan.timestep(u, v, w, DT, NU, FX, p_out=p, scratch=scratch)
        snap = [t.clone() for t in (u, v, w, p)]
        for _ in range(warmup):
            plan.timestep(u, v, w, DT, NU, FX, p_out=p, scratch=scratch)
        stream = torch.cuda.current_stream(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(steps):
            plan.timestep(u, v, w, DT, NU, FX, p_out=p, scratch=scratch)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        del plan
        tplan = mk(P.POISSON_TIMING)   # stage times from a separate pass with per-launch events
        stage = {}
        tplan.timestep(u, v, w, DT, NU, FX, p_out=p, scratch=scratch)
        for _ in range(2):
            tplan.timestep(u, v, w, DT, NU, FX, p_out=p, scratch=scratch)
            for k, t in tplan.stage_times():
                stage[k] = stage.get(k, 0.0) + t / 2
        del tplan
        entry = {"ms_per_timestep": ms, "gpts_s": CASE.npoints / (ms * 1e-3) / 1e9,
                 "stage_ms": {k: round(x, 4) for k, x in sorted(stage.items(), key=lambda kv: -kv[1])}}
        if ref is None:
            ref = snap
        else:
            vel = max(float((a - b).abs().max()) / float(b.abs().max()) for a, b in zip(snap[:3], ref[:3]))
            entry["maxrel_velocity_vs_fp64"] = vel
            entry["maxrel_pressure_vs_fp64"] = float((snap[3] - ref[3]).abs().max()) / float(ref[3].abs().max())
        out[name] = entry
        del u, v, w, p, scratch, snap
        torch.cuda.empty_cache()
    return out


GOLDEN_1536 = os.path.join(ROOT, "tests", "golden", "channel1536_seed2_modes.json")


def golden_modes_1536():
    """The oracle's solutions of sampled (kx, kz) modes for the seed-2 random-divergence rhs of the
    1536 x 768 x 1024 channel, stored by tests/golden/make_golden_1536.py (no oracle code runs here)."""
    d = json.load(open(GOLDEN_1536))
    return [(m["kx"], m["kz"], np.array([complex(re, im) for re, im in m["P"]])) for m in d["modes"]]


def mode_coeffs_gpu(p, kx, kz):
    """sum_{k,i} p[j,k,i] e^{-2 pi i (kz k / Nz + kx i / Nx)} for every row j, on the device (analysis)."""
    import torch
    ny, nz, nx = p.shape
    ax = -2.0 * math.pi * kx * torch.arange(nx, dtype=torch.float64, device=p.device) / nx
    az = -2.0 * math.pi * kz * torch.arange(nz, dtype=torch.float64, device=p.device) / nz
    pd = p.double()
    xr, xi = pd @ torch.cos(ax), pd @ torch.sin(ax)            # (ny, nz)
    cz, sz = torch.cos(az), torch.sin(az)
    re = xr @ cz - xi @ sz
    im = xr @ sz + xi @ cz
    return (re + 1j * im).cpu().numpy()


# Algorithmic HBM bytes per grid point of the precision forms at 1536x768x1024: FP64 plain 48
# (58.0 GB: read f, write and read F, write and read P, write p), FP32 plain 24 (29.0 GB), FP32
# with one FP64-residual correction 80 (96.7 GB: both solves, the FP64 rhs read twice, the FP32
# pressure written and read back, the FP64 pressure written).
FORM_MODEL_BYTES_PER_POINT = {"fp64": 48, "fp32": 24, "fp32_refined_1": 80}


def precision_forms(dev, steps: int = 5, warmup: int = 3):
    """FP64 plain vs FP32 vs FP32-refined Poisson solves on the 1536 x 768 x 1024 channel.

    Right-hand side: the divergence D(u, v, w) of the seed-2 N(0, 1) staggered velocity
    (workloads.random_velocity(2, ...), the same numbers the oracle's stored modes were computed
    from), formed on the device by poisson_divergence; the solve removes its dy-weighted mean.  Each
    form is timed with CUDA events over `steps` solves (stage times from a separate pass with
    per-launch events).  Its error is stated against the oracle (maxrel_vs_oracle: the largest
    difference of the result's 2-D DFT at the stored modes, every row, over max|p| Nx Nz) and
    against the plain FP64 GPU solve (maxrel_vs_fp64: max |p - p_FP64| / max |p_FP64|).
    """
    import torch
    import paper_2104_08863_gb300 as P
    case = W.CHANNEL_1536
    faces = W.tanh_faces(case.ny, case.stretch)
    golden = golden_modes_1536()
    hbm_peak = float(measured_peaks().get("hbm_gbs", 6800.0))
    plans = {}
    mk = lambda prec, rs, flags=0: P.Plan(case.nx, case.ny, case.nz, faces, case.lx, case.lz, precision=prec,
                                          fp64_low_modes=4, refine_steps=max(rs, 1), flags=flags, device=dev)
    plans["fp64"] = mk(P.PP_FP64, 0)
    uvw = [torch.from_numpy(a).to(dev) for a in W.random_velocity(2, case.nx, case.ny, case.nz)]
    f = plans["fp64"].divergence(*uvw, dt=1.0)
    del uvw
    torch.cuda.empty_cache()
    out = {"workload": f"{case.name} Poisson solve, rhs D(u, v, w) of the seed-2 N(0,1) velocity",
           "grid": [case.nx, case.ny, case.nz],
           "oracle_modes": [[kx, kz] for kx, kz, _ in golden]}
    ref = None
    forms = [("fp64", P.PP_FP64, 0), ("fp32", P.PP_FP32, 0), ("fp32_refined_1", P.PP_FP32_REFINED, 1),
             ("fp32_refined_2", P.PP_FP32_REFINED, 2)]
    stream = torch.cuda.current_stream(dev)
    for name, prec, steps_r in forms:
        plan = plans.pop(name, None) or mk(prec, steps_r)
        rhs = f.float() if prec == P.PP_FP32 else f
        p = torch.empty_like(rhs)
        for _ in range(warmup):
            plan.solve(rhs, out=p)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(steps):
            plan.solve(rhs, out=p)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        del plan
        tplan = mk(prec, steps_r, P.POISSON_TIMING)
        tplan.solve(rhs, out=p)
        stage = {}
        for _ in range(2):
            tplan.solve(rhs, out=p)
            for k, t in tplan.stage_times():
                stage[k] = stage.get(k, 0.0) + t / 2
        del tplan
        entry = {"ms": ms, "gpts_s": case.npoints / (ms * 1e-3) / 1e9,
                 "stage_ms": {k: round(v, 4) for k, v in sorted(stage.items(), key=lambda kv: -kv[1])}}
        if name in FORM_MODEL_BYTES_PER_POINT:
            model = FORM_MODEL_BYTES_PER_POINT[name] * case.npoints
            achieved = model / (ms * 1e-3) / 1e9
            entry["hbm_roofline"] = {"model_bytes": model, "achieved_gbs": achieved, "peak_gbs": hbm_peak,
                                     "frac": achieved / hbm_peak,
                                     "model": "six-transfer algorithmic bytes of the form (read f, write and "
                                              "read the spectrum twice, write p; the refined form adds the "
                                              "residual pass and the correction solve)",
                                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
        pmax = float(p.abs().max())
        worst = 0.0
        for kx, kz, want in golden:
            got = mode_coeffs_gpu(p, kx, kz)
            worst = max(worst, float(np.max(np.abs(got - want))) / (pmax * case.nx * case.nz))
        entry["maxrel_vs_oracle"] = worst
        if ref is None:
            ref = p.clone()
            scale = float(ref.abs().max())
        else:
            entry["maxrel_vs_fp64"] = float((p.double() - ref).abs().max()) / scale
        out[name] = entry
        del p
        torch.cuda.empty_cache()
    out["library_reference"] = library_reference(dev, f, ref, case)
    return out


def _cusparse_lib():
    import ctypes
    import torch
    cands = [os.path.join(os.path.dirname(torch.__file__), "lib", "libcusparse.so.12"), "libcusparse.so.12",
             "/usr/local/cuda/lib64/libcusparse.so.12", "libcusparse.so"]
    for c in cands:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


def library_reference(dev, f64, ref, case, steps: int = 3, warmup: int = 2):
    """Reference point from vendor libraries: the same FP32 Poisson solve with cuFFT (torch.fft) for
    the x and z transforms and cuSPARSE's batched tridiagonal solver (cusparseCgtsvInterleavedBatch,
    Thomas algorithm, whose interleaved layout is the spectrum's: row j of system b at j B + b) for
    the wall-normal systems.  Stages are timed with CUDA events (the diagonals, which the solver
    overwrites, are restored outside the timed region).  The error is taken against the FP64 solve
    with the x-z mean profile (the singular (0, 0) mode, regularised here) removed from both."""
    import ctypes
    import torch
    lib = _cusparse_lib()
    if lib is None:
        return {"unavailable": "libcusparse not found"}
    nx, ny, nz = case.nx, case.ny, case.nz
    m1 = nx // 2 + 1
    nb = nz * m1
    y = np.asarray(W.tanh_faces(ny, case.stretch))
    dy = np.diff(y)
    h = np.diff(0.5 * (y[1:] + y[:-1]))
    a = np.zeros(ny)
    c = np.zeros(ny)
    a[1:] = 1.0 / (dy[1:] * h)
    c[:-1] = 1.0 / (dy[:-1] * h)
    lamx = -(4.0 / (case.lx / nx) ** 2) * np.sin(np.pi * np.arange(m1) / nx) ** 2
    lamz = -(4.0 / (case.lz / nz) ** 2) * np.sin(np.pi * np.arange(nz) / nz) ** 2
    lam = torch.from_numpy((lamz[:, None] + lamx[None, :]).reshape(-1)).to(dev)
    diag = (torch.from_numpy(-(a + c)).to(dev)[:, None] + lam[None, :]).to(torch.complex64)
    diag[:, 0] -= 1.0   # regularise the singular (0, 0) system; its mode is compared away
    del lam
    sub = torch.from_numpy(a).to(dev, torch.complex64)[:, None].expand(ny, nb).contiguous()
    sup = torch.from_numpy(c).to(dev, torch.complex64)[:, None].expand(ny, nb).contiguous()
    dl, d, du = sub.clone(), diag.clone(), sup.clone()
    handle = ctypes.c_void_p()
    if lib.cusparseCreate(ctypes.byref(handle)) != 0:
        return {"unavailable": "cusparseCreate failed"}
    stream = torch.cuda.current_stream(dev)
    lib.cusparseSetStream(handle, ctypes.c_void_p(stream.cuda_stream))
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    f32 = f64.float()
    X = torch.fft.fft(torch.fft.rfft(f32, dim=2), dim=1).contiguous()
    size = ctypes.c_size_t(0)
    st = lib.cusparseCgtsvInterleavedBatch_bufferSizeExt(handle, 0, ny, ptr(dl), ptr(d), ptr(du), ptr(X), nb,
                                                          ctypes.byref(size))
    if st != 0:
        lib.cusparseDestroy(handle)
        return {"unavailable": f"cusparseCgtsvInterleavedBatch_bufferSizeExt status {st}"}
    work = torch.empty(max(int(size.value), 16), dtype=torch.uint8, device=dev)
    tm = {"cufft_forward_ms": 0.0, "cusparse_gtsv_ms": 0.0, "cufft_inverse_ms": 0.0}
    p = None
    for it in range(warmup + steps):
        dl.copy_(sub)
        d.copy_(diag)
        du.copy_(sup)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        torch.cuda.synchronize(dev)
        ev[0].record(stream)
        X = torch.fft.fft(torch.fft.rfft(f32, dim=2), dim=1).contiguous()
        ev[1].record(stream)
        st = lib.cusparseCgtsvInterleavedBatch(handle, 0, ny, ptr(dl), ptr(d), ptr(du), ptr(X), nb, ptr(work))
        ev[2].record(stream)
        p = torch.fft.irfft(torch.fft.ifft(X, dim=1), n=nx, dim=2)
        ev[3].record(stream)
        torch.cuda.synchronize(dev)
        if st != 0:
            lib.cusparseDestroy(handle)
            return {"unavailable": f"cusparseCgtsvInterleavedBatch status {st}"}
        if it >= warmup:
            for k, (e0, e1) in zip(tm, ((ev[0], ev[1]), (ev[1], ev[2]), (ev[2], ev[3]))):
                tm[k] += e0.elapsed_time(e1) / steps
    lib.cusparseDestroy(handle)

    def strip(q):
        return q - q.mean(dim=(1, 2), keepdim=True)

    err = float((strip(p.double()) - strip(ref)).abs().max() / strip(ref).abs().max())
    out = {k: round(v, 3) for k, v in tm.items()}
    out["ms"] = round(sum(tm.values()), 3)
    out["maxrel_vs_fp64_without_mode00"] = err
    out["note"] = "unofficial reference point: FP32, textbook Thomas in cuSPARSE, no FP64 low modes"
    del dl, d, du, sub, sup, diag, X, p, work, f32
    torch.cuda.empty_cache()
    return out


def batch_form(dev, steps: int = 5, warmup: int = 2, tune: bool = True):
    """64 uneven FP32 solves (default_rng(5) sizes): sequential plain solves vs one batched graph launch.

    Right-hand sides: seeded N(0, 1) fields drawn on the device.  Reports aggregate Gpts/s of
    both, the batch's kernel launches replayed per graph launch, and the autotuner's choices.
    """
    import torch
    import paper_2104_08863_gb300 as P
    cases = W.batch_instances(5, 64)
    total = sum(c.npoints for c in cases)
    specs = [dict(nx=c.nx, ny=c.ny, nz=c.nz, y_faces=W.tanh_faces(c.ny, c.stretch)) for c in cases]
    gen = torch.Generator(device=dev)
    gen.manual_seed(5)
    rhs = [torch.randn(c.ny, c.nz, c.nx, dtype=torch.float32, device=dev, generator=gen) for c in cases]
    outs = [torch.empty_like(r) for r in rhs]
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        for _ in range(warmup):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / steps

    plans = [P.Plan(c.nx, c.ny, c.nz, sp["y_faces"], precision=P.PP_FP32, device=dev) for c, sp in zip(cases, specs)]
    ms_seq = timed(lambda: [pl.solve(r, out=o) for pl, r, o in zip(plans, rhs, outs)])
    del plans
    bb = P.BatchPlan(specs, precision=P.PP_FP32, device=dev)
    ms_branches = timed(lambda: bb.solve(rhs, out=outs))
    branch_kernels = bb.last_launch_count
    del bb
    bp = P.BatchPlan(specs, precision=P.PP_FP32, device=dev, persistent=True)
    ms_batch = timed(lambda: bp.solve(rhs, out=outs))
    out = {"workload": "64 uneven FP32 Poisson solves, sizes from default_rng(5)", "points": total,
           "sequential_ms": ms_seq, "sequential_gpts_s": total / (ms_seq * 1e-3) / 1e9,
           "graph_branches_ms": ms_branches, "graph_branches_gpts_s": total / (ms_branches * 1e-3) / 1e9,
           "graph_branches_kernels": branch_kernels,
           "persistent_ms": ms_batch, "persistent_gpts_s": total / (ms_batch * 1e-3) / 1e9,
           "persistent_kernels_per_graph_launch": bp.last_launch_count,
           "persistent_status": bp.device_status()}
    del bp
    if tune:
        t0 = time.perf_counter()
        bt, strat = P.tune_batch(specs, precision=P.PP_FP32, device=dev)
        tune_s = time.perf_counter() - t0
        ms_tuned = timed(lambda: bt.solve(rhs, out=outs))
        best = min(strat, key=strat.get)
        out.update({"batched_tuned_ms": ms_tuned, "batched_tuned_gpts_s": total / (ms_tuned * 1e-3) / 1e9,
                    "autotune_s": tune_s, "autotune_strategy": best,
                    "autotune_strategy_ms": {k: round(v, 4) for k, v in strat.items()},
                    "tuned_parts_hist": {str(k): sum(1 for t in bt.tuned if t[0] == k)
                                         for k in sorted(set(t[0] for t in bt.tuned))}})
        del bt
    torch.cuda.empty_cache()
    return out


def pdd_study(dev):
    """Truncated PDD (Sec. 2.2: framed entries of Z dropped) against the exact reduced system.

    Part 1 (CPU, oracle, one wall-normal system): the truncation error of a single mode as a
    function of sigma = -(lambda_x + lambda_z) on the 384-row (tanh 2.0) and 768-row (tanh 2.2)
    grids for several P, against the Thomas solution; the paper's condition is that the dropped
    spike ends fall below machine accuracy.  Part 2 (GPU): whole solves on the 512x384x512 (FP64)
    and 1536x768x1024 (FP32) channels, max |p_trunc - p_exact| / max |p_exact| and times.
    """
    import oracle
    import torch
    import paper_2104_08863_gb300 as P
    out = {"per_sigma": {}, "solves": {}}
    rng = np.random.default_rng(12)
    for ny, s in ((384, 2.0), (768, 2.2)):
        g = oracle.Grid(8, 8, W.tanh_faces(ny, s))
        a, c = g.lower, g.upper
        d = rng.standard_normal(ny) + 1j * rng.standard_normal(ny)
        rows = {}
        for parts in (4, 8, 16, 32):
            errs = {}
            for sigma in (1e0, 1e1, 1e2, 1e3, 1e4, 1e5):
                diag = -(a + c) - sigma
                x = oracle.thomas(a, diag, c, d)
                xt = oracle.pdd(a, diag, c, d, parts, truncated=True)
                errs[f"{sigma:.0e}"] = float(np.max(np.abs(xt - x)) / np.max(np.abs(x)))
            rows[f"P={parts} (m={ny // parts})"] = errs
        out["per_sigma"][f"ny={ny} tanh {s}"] = rows
    gen = torch.Generator(device=dev)
    for case, prec, parts_list in ((CASE, P.PP_FP64, (4, 8, 16)), (W.CHANNEL_1536, P.PP_FP32, (8, 16, 32))):
        faces = W.tanh_faces(case.ny, case.stretch)
        gen.manual_seed(2)
        dtype = torch.float64 if prec == P.PP_FP64 else torch.float32
        f = torch.randn(case.ny, case.nz, case.nx, dtype=dtype, device=dev, generator=gen)
        res = {}
        for parts in parts_list:
            sol = {}
            for tri in (P.PT_PDD_EXACT, P.PT_PDD_TRUNCATED):
                plan = P.Plan(case.nx, case.ny, case.nz, faces, case.lx, case.lz, precision=prec, tridiag=tri,
                              pdd_parts=parts, flags=P.POISSON_TIMING, device=dev)
                p = torch.empty_like(f)
                plan.solve(f, out=p)
                plan.solve(f, out=p)
                tri_ms = sum(ms for k, ms in plan.stage_times() if k.startswith("tridiag"))
                sol[tri] = (p, tri_ms)
                del plan
            pe, pt = sol[P.PT_PDD_EXACT][0], sol[P.PT_PDD_TRUNCATED][0]
            res[f"P={parts}"] = {"maxrel_trunc_vs_exact": float((pt - pe).abs().max() / pe.abs().max()),
                                 "tridiag_ms_exact": sol[P.PT_PDD_EXACT][1],
                                 "tridiag_ms_truncated": sol[P.PT_PDD_TRUNCATED][1]}
            del sol, pe, pt
            torch.cuda.empty_cache()
        out["solves"][f"{case.name} {'FP64' if prec == P.PP_FP64 else 'FP32'}"] = res
        del f
    return out


PROFILE_CASES = {
    # name: (case, precision, refine_steps, kind) with kind "timestep", "projection" or "solve"
    "fp64_timestep_256": (W.CHANNEL_256, 0, 0, "timestep"),
    "fp64_timestep_512": (W.CHANNEL_512, 0, 0, "timestep"),
    "fp32_refined_timestep_256": (W.CHANNEL_256, 2, 2, "timestep"),
    "fp64_projection_256": (W.CHANNEL_256, 0, 0, "projection"),
    "fp64_projection_512": (W.CHANNEL_512, 0, 0, "projection"),
    "fp32_solve_512": (W.CHANNEL_512, 1, 0, "solve"),
    "fp32_refined_solve_512": (W.CHANNEL_512, 2, 1, "solve"),
    # the 768-row wall-normal grid of the 1536x768x1024 precision form on a 256x256 plane
    "fp32_refined_solve_256x768x256": (W.ChannelCase("channel_256x768x256_tanh2.2", 256, 768, 256, 2.2), 2, 1,
                                       "solve"),
    # the 1536-point x lines of the 1536x768x1024 precision form on a 96x128 (y, z) section
    "fp32_refined_solve_1536x96x128": (W.ChannelCase("channel_1536x96x128_tanh2.2", 1536, 96, 128, 2.2), 2, 1,
                                       "solve"),
    # the full 1536 x 1024 planes of the precision form at 64 rows (a fifth entry would add plan flags)
    "fp32_refined_solve_1536x64x1024": (W.ChannelCase("channel_1536x64x1024_tanh2.2", 1536, 64, 1024, 2.2), 2, 1,
                                        "solve"),
    # the precision form itself (launch lists only: one metric pass)
    "fp32_refined_solve_1536x768x1024": (W.CHANNEL_1536, 2, 1, "solve"),
    # the 64 uneven FP32 solves of the batched form as one persistent work-queue launch
    "batch64_persistent": (None, 1, 0, "batch"),
}


def profile_case(name: str, repeats: int = 2):
    """Run a named case `repeats` times without timing (for ncu captures of single kernels)."""
    import torch
    from paper_2104_08863_gb300 import build as b
    b.build()
    import paper_2104_08863_gb300 as P
    case, prec, steps, kind = PROFILE_CASES[name][:4]
    extra = PROFILE_CASES[name][4] if len(PROFILE_CASES[name]) > 4 else 0
    dev = torch.device("cuda", 0)
    if kind == "batch":
        cases = W.batch_instances(5, 64)
        specs = [dict(nx=c.nx, ny=c.ny, nz=c.nz, y_faces=W.tanh_faces(c.ny, c.stretch)) for c in cases]
        gen = torch.Generator(device=dev)
        gen.manual_seed(5)
        rhs = [torch.randn(c.ny, c.nz, c.nx, dtype=torch.float32, device=dev, generator=gen) for c in cases]
        bp = P.BatchPlan(specs, precision=P.PP_FP32, device=dev, persistent=True)
        outs = [torch.empty_like(r) for r in rhs]
        for _ in range(repeats):
            bp.solve(rhs, out=outs)
        torch.cuda.synchronize(dev)
        print(json.dumps({"profile_case": name, "launches_per_call": bp.last_launch_count}))
        return
    faces = W.tanh_faces(case.ny, case.stretch)
    parts = PDD_PARTS if (prec == P.PP_FP64 and case.ny % PDD_PARTS == 0) else 0
    plan = P.Plan(case.nx, case.ny, case.nz, faces, case.lx, case.lz, precision=prec, pdd_parts=parts,
                  refine_steps=max(steps, 1), flags=extra, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(0)
    dtype = torch.float32 if prec == P.PP_FP32 else torch.float64
    if kind in ("projection", "timestep"):
        u = torch.randn(case.ny, case.nz, case.nx, dtype=dtype, device=dev, generator=gen)
        v = torch.randn(case.ny + 1, case.nz, case.nx, dtype=dtype, device=dev, generator=gen)
        w = torch.randn(case.ny, case.nz, case.nx, dtype=dtype, device=dev, generator=gen)
        v[0].zero_()
        v[-1].zero_()
        scratch = (torch.empty_like(u), torch.empty_like(v), torch.empty_like(w))
        for _ in range(repeats):
            if kind == "timestep":
                plan.timestep(u, v, w, DT, NU, FX, scratch=scratch)
            else:
                plan.project(u, v, w, DT)
    else:
        f = torch.randn(case.ny, case.nz, case.nx, dtype=dtype, device=dev, generator=gen)
        p = torch.empty_like(f)
        for _ in range(repeats):
            plan.solve(f, out=p)
    torch.cuda.synchronize(dev)
    print(json.dumps({"profile_case": name, "launches_per_call": plan.last_launch_count}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the 1536x768x1024 precision-form comparison")
    ap.add_argument("--forms-only", action="store_true")
    ap.add_argument("--batch-only", action="store_true", help="only the 64-instance batched form")
    ap.add_argument("--pdd-study", action="store_true", help="truncated vs exact PDD (Sec. 2.2) study")
    ap.add_argument("--profile", choices=sorted(PROFILE_CASES), help="run a named case for ncu, no timing")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.profile:
        profile_case(args.profile)
    elif args.impl == "reference":
        run_reference(args)
    elif args.pdd_study:
        import torch
        from paper_2104_08863_gb300 import build as b
        b.build()
        print(json.dumps(pdd_study(torch.device("cuda", 0))))
    elif args.batch_only:
        import torch
        from paper_2104_08863_gb300 import build as b
        b.build()
        print(json.dumps(batch_form(torch.device("cuda", 0))))
    elif args.forms_only:
        import torch
        from paper_2104_08863_gb300 import build as b
        b.build()
        dev = torch.device("cuda", 0)
        print(json.dumps({"precision_forms": precision_forms(dev), "timestep_forms": timestep_forms(dev)}))
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
