"""Benchmark of the hybrid lattice Boltzmann hot path on GB300.

Workload (the throughput configuration of the method): D2Q9 spinodal
decomposition on a 1024 x 1024 periodic lattice, FP32-deviation populations,
a = -0.1, b = 0.1, kappa = 0.14, tau = 1, Gamma = 0.5, OC stencil (N = 0.3,
Q = 2.5), m = 4 FD substeps, phi uniform in [-0.01, 0.01] (splitmix64, seed
0), n = 1, u = 0; 20000 LB steps.

One timed "step" of this benchmark is one call lbm_step(h, 1000): 1000 LB
steps of the whole hot path (stencil force, collide/stream, FD update), so the
default --steps 20 covers the configuration's 20000 LB steps.  L2 is flushed
(a 256 MiB write) between timed steps.  Metric: MLUPS = sites x LB steps /
seconds / 1e6, whole job.

--impl reference times the FP64 CPU oracle (single thread) on the same
workload, each step one LB step of the 1024 x 1024 lattice.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L = 1024
LB_PER_STEP = 1000
CFG = dict(a=-0.1, b=0.1, kappa=0.14, tau=1.0, Gamma=0.5, N=0.3, Q=2.5)
M_SUB = 4
# algorithmic bytes per site of the collide kernel (FP32 deviations):
# populations read + written (2 x 9 x 4 B) and phi read (4 B)
COLLIDE_BYTES_PER_SITE = 76
# floating-point operations per site and FD substep of Eqs. 32-36 as printed:
# advection 13 (two central differences, two upwind differences, four products,
# three sums, phi - dt tend), diffusion 28 (three 5-point Laplacians at 6, the
# cube 2, a L1 + b L2 - kappa L3 and phih + dt Gamma (.) 8)
FD_FLOPS_PER_SITE_SUBSTEP = 41
# FP32 pipe peak of a GB300: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu --set full capture of the 1024^2 workload
# (profiles/collide2d_fd2d_spinodal1024.md), valid for the kernels captured
# there: the FD block kernel with 4 substeps, 96-row regions and 16 warps
# (consecutive rows per warp, psi fused), and the TMA collide kernel with the
# packed-pair collision (launch-shape variant 5).  ncu flushes the caches
# before a captured launch: these are cold-cache figures.
NCU_TRAFFIC_1024 = {"fd": ((128, 96, 4, 2), 12.648448e6), "collide": (5, 41.977856e6 + 2.784768e6)}
# the same collide kernel (variant 5) captured on 2048^2 (4.19 M sites; the
# lattice no longer fits L2): 168.389120 MB read + 129.996032 MB written per
# launch = 71.2 B/site; the 4096^2 line scales it by the site count
NCU_TRAFFIC_COLLIDE_2048 = (5, 168.389120e6 + 129.996032e6)
METRIC = "MLUPS (D2Q9 hybrid LB + FD step)"
WORKLOAD = "spinodal-1024x1024-d2q9-f32dev"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def whole_job_mlups(ms_local, world, site_updates_per_rank, dist=None, device="cuda"):
    """Whole-job throughput of `world` replicas: every rank did
    site_updates_per_rank lattice updates; the job took the slowest rank's
    time (the maximum over ranks).  Returns (MLUPS, that time in ms)."""
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return world * site_updates_per_rank / (ms_max / 1000.0) / 1e6, ms_max


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        med = statistics.median(sm)
        # a median well below the maximum with no reason active points to a
        # clock lock left by someone else: such a run is taken again
        return {"sm_mhz": med, "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "below_max_without_reason": bool(med < 0.9 * max(mx) and not reasons)}


def make_inputs(seed, side=None):
    from paper_0902_3921_gb300 import inputs as I
    side = side or L
    phi = I.spinodal(2, side, side, seed=seed)
    n, u = I.rest(2, side, side)
    return n, phi, u


def cpu_identity():
    """This host's logical CPU count and model name (lscpu, else /proc/cpuinfo)."""
    import platform
    import subprocess
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "model": model, "machine": platform.machine()}


def cpu_oracle_mlups(steps=1, seed=0, threads=1):
    """The FP64 oracle as it stands, `steps` LB steps of the 1024^2 workload
    on `threads` threads (0: all cores; its OpenMP site loops give the same
    bits for any count).  Returns (MLUPS, seconds, threads used)."""
    import oracle as O
    O.build()
    used = O.set_threads(threads)
    op = O.Params(Lx=L, Ly=L, m=M_SUB, **CFG)
    n, phi, u = make_inputs(seed)
    st = O.State.create(op, n, phi, u)
    t0 = time.perf_counter()
    st.run(steps)
    dt = time.perf_counter() - t0
    O.set_threads(0)
    return L * L * steps / dt / 1e6, dt, used


def cpu_baseline_line(single_steps):
    """The oracle on one thread and on all host cores (about 10-20 s of CPU
    work on the 16-core host of the GPU machine): the all-core figure is the
    baseline, the single-thread one is reported beside it."""
    m1, dt1, _ = cpu_oracle_mlups(single_steps, threads=1)
    steps_all = 4 * single_steps
    mn, dtn, used = cpu_oracle_mlups(steps_all, threads=0)
    return {"value": mn, "unit": "MLUPS", "cores": used, "kind": "oracle",
            "sample": f"{steps_all} LB steps of the 1024x1024 workload on {used} threads ({dtn:.1f} s)",
            "single_thread": {"value": m1, "unit": "MLUPS", "cores": 1,
                              "sample": f"{single_steps} LB steps of the same workload ({dt1:.1f} s)"},
            "host": cpu_identity()}


def run_reference(args, rank, world):
    if rank != 0:
        return
    times = []
    cores = 1
    for k in range(args.warmup + args.steps):
        mlups, dt, cores = cpu_oracle_mlups(1, seed=k, threads=0)
        if k >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = L * L * args.steps / total / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice": [L, L],
                       "lb_steps_per_timed_step": 1,
                       "note": f"FP64 CPU oracle on {cores} threads (OpenMP site loops), one LB step "
                               "per timed step"},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} LB steps of the 1024x1024 workload",
                             "host": cpu_identity()},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local):
    import torch
    from paper_0902_3921_gb300 import build as B
    from paper_0902_3921_gb300 import lbm

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    if dist is not None:
        dist.barrier()
    lib = lbm.load_library()
    stream = torch.cuda.Stream()
    side = args.lattice
    params = lbm.LbmParams(Lx=side, Ly=side, fd_substeps=M_SUB, precision=lbm.LBM_F32DEV,
                           **CFG)
    S = params.S
    n, phi, u = make_inputs(seed=rank, side=side)
    lat = lbm.Lattice(params, stream=stream.cuda_stream)
    lbm.lbm_set_graphs(lat.handle, not args.no_graphs)
    lat.init_fields(n, phi, u)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        if dist is not None:
            dist.barrier()

    # warm-up (also builds and caches the CUDA graphs)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            lat.step(LB_PER_STEP)
        lat.synchronize()
    # timed region: device-resident state, K x lbm_step(1000), L2 flushed between
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                lat.step(LB_PER_STEP)
                ev[k][1].record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    value, ms_max = whole_job_mlups(ms, world, S * LB_PER_STEP * args.steps, dist, "cuda")
    tuning = lbm.lbm_tuning(lat.handle)
    if args.quick:
        # profiling runs: the timed region only
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "MLUPS",
                              "lattice": side, "quick": True, "tuning": tuning}), flush=True)
        lat.close()
        return

    # kernel timing region: the same steps, each kernel bracketed by events
    lbm.lbm_set_kernel_timing(lat.handle, True)
    lbm.lbm_kernel_times(lat.handle, reset=True)
    with torch.cuda.stream(stream):
        lat.step(2000)
    kt = lbm.lbm_kernel_times(lat.handle, reset=True)
    lbm.lbm_set_kernel_timing(lat.handle, False)
    coll_ms, coll_n = kt["collide"]
    fd_ms, fd_n = kt["fd"]
    coll_avg_s = coll_ms / coll_n / 1000.0
    fd_avg_s = fd_ms / max(fd_n, 1) / 1000.0
    fd_launches_per_step = max(fd_n, 1) / 2000.0
    achieved = COLLIDE_BYTES_PER_SITE * S / coll_avg_s / 1e9
    peak, peak_kind = measured_peak()
    shape_fd = (tuning["fd_tile_width"], tuning["fd_rows_per_warp"], tuning["fd_substeps_per_launch"],
                tuning["fd_cols_per_lane"])
    traffic_fd = NCU_TRAFFIC_1024["fd"][1] if side == 1024 and shape_fd == NCU_TRAFFIC_1024["fd"][0] else None
    traffic_coll = (NCU_TRAFFIC_1024["collide"][1]
                    if side == 1024 and tuning["collide_sites_per_thread"] == NCU_TRAFFIC_1024["collide"][0]
                    else None)
    roof_collide = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": traffic_coll,
                    "kernel": "collide2d (stencil force + collide + stream)",
                    "bytes_per_site": COLLIDE_BYTES_PER_SITE, "avg_launch_us": coll_avg_s * 1e6,
                    "peak_kind": peak_kind, "share_of_step": coll_ms / (coll_ms + fd_ms)}
    # FLOPs of one launch: the m substeps of an LB step spread over its launches
    fd_flops_launch = FD_FLOPS_PER_SITE_SUBSTEP * M_SUB * S / fd_launches_per_step
    fd_tflops = fd_flops_launch / fd_avg_s / 1e12
    fd_note = ("counts the useful flops only (164 a site and LB step); the kernel is bound by the "
               "shared-memory pipe and issue latency, not the FP32 units")
    if traffic_fd is not None:
        fd_note += (": ncu of this launch shape at 1024^2 shows 60 % L1/shared-memory throughput, "
                    "44 % of cycles issuing and 6.78 M warp instructions a launch (0.34 of the "
                    "issue rate over its duration), with 12 B/site of DRAM traffic")
    roof_fd = {"bound": "alu", "achieved": fd_tflops, "peak": FP32_PEAK_TFLOPS, "note": fd_note,
               "unit": "TFLOP/s", "frac": fd_tflops / FP32_PEAK_TFLOPS, "traffic": traffic_fd,
               "kernel": "fd2d (m = 4 FD substeps of Eqs. 32-36)",
               "flops_per_site": FD_FLOPS_PER_SITE_SUBSTEP * M_SUB,
               "launches_per_lb_step": fd_launches_per_step,
               "avg_launch_us": fd_avg_s * 1e6, "peak_kind": "derived (unit counts x clock)",
               "share_of_step": fd_ms / (coll_ms + fd_ms)}
    # the same kernels inside the graph-timed step: their event times above
    # are taken on eager launches (each bracketed by events), which sum to
    # more than the graph step (launch gaps); the in-step figures
    # share the graph step's time in the proportion of the event times
    graph_lb_us = ms_max / (args.steps * LB_PER_STEP) * 1000.0
    eager_lb_us = (coll_ms + fd_ms) / 2000.0 * 1000.0
    share_c = coll_ms / (coll_ms + fd_ms)
    c_in = share_c * graph_lb_us
    f_in = (1.0 - share_c) * graph_lb_us / fd_launches_per_step
    roof_collide.update({"in_step_us": c_in,
                         "frac_in_step": COLLIDE_BYTES_PER_SITE * S / (c_in * 1e-6) / 1e9 / peak})
    roof_fd.update({"in_step_us": f_in,
                    "frac_in_step": fd_flops_launch / (f_in * 1e-6) / 1e12 / FP32_PEAK_TFLOPS})
    kernel_times = {"graph_lb_step_us": graph_lb_us, "eager_lb_step_us": eager_lb_us,
                    "graph_over_eager": graph_lb_us / eager_lb_us,
                    "collide_us_per_lb_step_eager": coll_ms / 2000.0 * 1000.0,
                    "fd_us_per_lb_step_eager": fd_ms / 2000.0 * 1000.0,
                    "note": "avg_launch_us: CUDA events around eager launches; in_step_us: the graph-timed "
                            "step split in the proportion of those times (they add up to the step)"}
    dominant, other = (roof_fd, roof_collide) if fd_ms > coll_ms else (roof_collide, roof_fd)

    # end to end through the C ABI with host buffers: H2D of the inputs from
    # pinned memory, 1000 LB steps, D2H of n, phi, u*
    pin = {k: torch.empty(S, dtype=torch.float64).pin_memory() for k in
           ("n", "phi", "ux", "uy", "on", "ophi", "oux", "ouy")}
    pin["n"].numpy()[:] = n.reshape(-1)
    pin["phi"].numpy()[:] = phi.reshape(-1)
    pin["ux"].numpy()[:] = u[0].reshape(-1)
    pin["uy"].numpy()[:] = u[1].reshape(-1)
    import ctypes
    P = {k: ctypes.cast(v.data_ptr(), ctypes.POINTER(ctypes.c_double)) for k, v in pin.items()}
    e2e_steps = max(2, min(args.steps, 5))
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        rc = lib.lbm_init_fields(lat.handle, P["n"], P["phi"], P["ux"], P["uy"], None)
        rc |= lib.lbm_step(lat.handle, LB_PER_STEP)
        rc |= lib.lbm_moments(lat.handle, P["on"], P["ophi"], P["oux"], P["ouy"], None)
        if rc:
            raise RuntimeError(lbm.lbm_last_error(lat.handle))
    t_e2e = time.perf_counter() - t0
    te = torch.tensor([t_e2e], dtype=torch.float64, device="cuda")
    if dist is not None:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = world * S * LB_PER_STEP * e2e_steps / float(te.item()) / 1e6

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline_line(args.cpu_sample_steps)
        sub = max(1, tuning["fd_substeps_per_launch"])
        fd_launches = (M_SUB + sub - 1) // sub
        gpu_launches = args.steps * LB_PER_STEP * (1 + fd_launches)
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if side == L else f"spinodal-{side}x{side}-d2q9-f32dev",
                       "lattice": [side, side], "lb_steps_per_timed_step":
                       LB_PER_STEP, "fd_substeps": M_SUB, "precision": "f32 deviations",
                       "params": CFG, "l2": "flushed (256 MiB write) between timed steps",
                       "tuning": tuning,
                       "parallelism": f"replicas x{world}"},
            "roofline": dominant,
            "roofline_other_kernel": other,
            "step_roofline": step_roofline(value),
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "MLUPS",
                    "h2d_bytes_per_step": 4 * 8 * S, "d2h_bytes_per_step": 4 * 8 * S,
                    "lb_steps_per_step": LB_PER_STEP},
            "gpu_launches": gpu_launches,
            "clocks": clocks.summary(),
            "kernel_times": kernel_times,
        }
        if side == L and not args.no_large:
            line["large_lattice"] = large_lattice(args.large_side, stream)
            line["f16_storage"] = {"1024": f16_storage(side, 2000, stream),
                                   str(args.large_side): f16_storage(args.large_side, 200, stream)}
        if side == L and not args.no_forms:
            line["forms"] = other_forms(local, rank, stream)
        print(json.dumps(line), flush=True)
    lat.close()
    if dist is not None:
        dist.destroy_process_group()


def other_forms(local, rank, stream):
    """Short, bounded runs of the other forms of the path, on the same GPU:
    the 512-instance batch (200 LB steps), the 256^3 D3Q19 drop (FP32 and
    FP16 deviations, 3 x 10 LB steps) and the learned surrogate (forward pass
    on 2048^2, and the trained network's speedup at fixed error from
    t = 2000 to 16000)."""
    out = {"batched": batched_form(200, local, rank, stream),
           "drop3d": drop3d_form(D3_SIDE, 3, 2, local, stream)}
    fwd, net, x0, x1 = surrogate_forward(400, 3, local, rank, stream)
    net.close()
    del x0, x1
    fwd["fixed_error"] = surrogate_fixed_error(SURR_SIDE)
    out["surrogate"] = fwd
    return out


# algorithmic bytes of one FD launch per site: phi read and written, u* read
FD_BYTES_PER_SITE_LAUNCH = 16

# bytes per site and LB step the method must carry between steps (FP32
# deviations): populations read and written (9 x 4 x 2) and phi (4 x 2)
STEP_BYTES_PER_SITE = 80


def step_roofline(mlups):
    """The whole step against the measured copy bandwidth: MLUPS x 80 B."""
    peak, kind = measured_peak()
    ach = mlups * 1e6 * STEP_BYTES_PER_SITE / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "bytes_per_site": STEP_BYTES_PER_SITE, "peak_kind": kind,
            "note": "u* (16 B/site written and read between the two kernels) is not counted"}


def f16_storage(side, lb_steps, stream):
    """The same workload with FP16 deviation storage (scale 2^10; FP32
    arithmetic): whole-step MLUPS over lb_steps LB steps after as many
    warm-up steps, and the collide kernel's per-launch event time against
    its 40 B/site (populations 9 x 2 B read and written, phi 4 B)."""
    import torch
    from paper_0902_3921_gb300 import inputs as I
    from paper_0902_3921_gb300 import lbm

    S = side * side
    lat = lbm.Lattice(lbm.LbmParams(Lx=side, Ly=side, fd_substeps=M_SUB, precision=lbm.LBM_F16DEV, **CFG),
                      stream=stream.cuda_stream)
    n, u = I.rest(2, side, side)
    lat.init_fields(n, I.spinodal(2, side, side, seed=0), u)
    del n, u
    with torch.cuda.stream(stream):
        lat.step(lb_steps)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        t0.record(stream)
        lat.step(lb_steps)
        t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    lbm.lbm_set_kernel_timing(lat.handle, True)
    lbm.lbm_kernel_times(lat.handle, reset=True)
    with torch.cuda.stream(stream):
        lat.step(min(lb_steps, 200))
    kt = lbm.lbm_kernel_times(lat.handle, reset=True)
    tuning = lbm.lbm_tuning(lat.handle)
    lat.close()
    (cms, cn), (fms, fn) = kt["collide"], kt["fd"]
    c_s = cms / cn / 1000.0
    peak, peak_kind = measured_peak()
    ach = 40 * S / c_s / 1e9
    return {"lattice": [side, side], "value": S * lb_steps / (ms / 1000.0) / 1e6, "unit": "MLUPS",
            "lb_steps_timed": lb_steps, "precision": "f16 deviations (scale 2^10), f32 arithmetic",
            "tuning": tuning,
            "collide": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                        "avg_launch_us": c_s * 1e6, "bytes_per_site": 40, "peak_kind": peak_kind},
            "fd_avg_launch_us": fms / fn * 1000.0}


def large_lattice(side, stream):
    """The same scheme on side^2 (default 4096^2, 1.5 GB of populations: far
    beyond L2), where the collide kernel is HBM-bound: whole-step MLUPS over
    3 x 100 LB steps and both kernels' per-launch event times."""
    import torch
    from paper_0902_3921_gb300 import inputs as I
    from paper_0902_3921_gb300 import lbm

    S = side * side
    lat = lbm.Lattice(lbm.LbmParams(Lx=side, Ly=side, fd_substeps=M_SUB, precision=lbm.LBM_F32DEV, **CFG),
                      stream=stream.cuda_stream)
    n, u = I.rest(2, side, side)
    lat.init_fields(n, I.spinodal(2, side, side, seed=0), u)
    del n, u
    with torch.cuda.stream(stream):
        lat.step(100)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        t0.record(stream)
        for _ in range(3):
            lat.step(100)
        t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    lbm.lbm_set_kernel_timing(lat.handle, True)
    lbm.lbm_kernel_times(lat.handle, reset=True)
    with torch.cuda.stream(stream):
        lat.step(100)
    kt = lbm.lbm_kernel_times(lat.handle, reset=True)
    tuning = lbm.lbm_tuning(lat.handle)
    lat.close()
    (cms, cn), (fms, fn) = kt["collide"], kt["fd"]
    c_s = cms / cn / 1000.0
    peak, peak_kind = measured_peak()
    ach = COLLIDE_BYTES_PER_SITE * S / c_s / 1e9
    value = S * 300 / (ms / 1000.0) / 1e6
    return {"lattice": [side, side], "value": value, "unit": "MLUPS",
            "lb_steps_timed": 300, "tuning": tuning, "step_roofline": step_roofline(value),
            "collide": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                        "avg_launch_us": c_s * 1e6, "bytes_per_site": COLLIDE_BYTES_PER_SITE,
                        "peak_kind": peak_kind,
                        "traffic": (NCU_TRAFFIC_COLLIDE_2048[1] * S / 2048 ** 2
                                    if tuning["collide_sites_per_thread"] == NCU_TRAFFIC_COLLIDE_2048[0] else None),
                        "traffic_note": "ncu capture on 2048^2 scaled by the site count"},
            "fd_avg_launch_us": fms / fn * 1000.0, "fd_launches_per_lb_step": fn / 100.0,
            # each FD launch reads phi and u* and writes phi: 16 B/site
            "fd": {"bound": "hbm", "achieved": FD_BYTES_PER_SITE_LAUNCH * S / (fms / fn / 1000.0) / 1e9,
                   "peak": peak, "unit": "GB/s",
                   "frac": FD_BYTES_PER_SITE_LAUNCH * S / (fms / fn / 1000.0) / 1e9 / peak,
                   "avg_launch_us": fms / fn * 1000.0, "bytes_per_site": FD_BYTES_PER_SITE_LAUNCH,
                   "kernel": f"fd2d (tile {tuning['fd_tile_width']}: 1 = y-marching wavefront)",
                   "peak_kind": peak_kind}}


def batched_form(steps, local, rank, stream):
    """512 independent drops (sides 32..256, half pushed by g_x = 1e-5 for the
    first 2000 of 6000 steps) advanced together, FP32 deviations, `steps` LB
    steps timed after as many warm-up steps, on the path the library chose at
    creation (the persistent kernel, one launch per LB step, or the tiled path,
    the collide over the tiles of all instances and m/2 wavefront FD launches
    over their strips; either captured in a CUDA graph); compared with the
    plain kernels on one square lattice of (about) the same number of sites,
    timed the same way."""
    import torch
    from paper_0902_3921_gb300 import inputs as I
    from paper_0902_3921_gb300 import lbm

    desc = I.batch_instances(512, seed=rank)
    insts = [(d["side"], d["side"], (1e-5 if d["forced"] else 0.0, 0.0),
              2000 if d["forced"] else 0) for d in desc]
    common = lbm.LbmParams(precision=lbm.LBM_F32DEV, fd_substeps=M_SUB, **CFG)
    b = lbm.Batch(common, insts, stream=stream.cuda_stream)
    xi = (2 * CFG["kappa"] / -CFG["a"]) ** 0.5
    for k, d in enumerate(desc):
        phi = I.drop(2, d["side"], d["side"], R=d["R"], phi0=1.0, xi=xi)
        n, u = I.rest(2, d["side"], d["side"])
        b.init_fields(k, n, phi, u)
    sites = b.shape()["sites"]
    b.step(steps)  # warm-up, captures the graph
    b.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        with torch.cuda.stream(stream):
            t0.record(stream)
            b.step(steps)
            t1.record(stream)
        torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    value = sites * steps / (ms / 1000.0) / 1e6
    shape = b.shape()
    b.close()
    # the plain kernels on one lattice with the same number of sites
    side = int(round(sites ** 0.5 / 16.0)) * 16
    lat = lbm.Lattice(lbm.LbmParams(Lx=side, Ly=side, fd_substeps=M_SUB, precision=lbm.LBM_F32DEV, **CFG),
                      stream=stream.cuda_stream)
    n, u = I.rest(2, side, side)
    lat.init_fields(n, I.spinodal(2, side, side, seed=rank), u)
    del n, u
    with torch.cuda.stream(stream):
        lat.step(steps)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        t0.record(stream)
        lat.step(steps)
        t1.record(stream)
    torch.cuda.synchronize()
    plain = side * side * steps / (t0.elapsed_time(t1) / 1000.0) / 1e6
    lat.close()
    peak, kind = measured_peak()
    return {"value": value, "unit": "MLUPS", "instances": 512, "sites": sites, "lb_steps_timed": steps,
            "ms": ms, "shape": shape, "path": "tiled" if shape["threads"] == 0 else "persistent",
            "launches_per_lb_step": 2 + M_SUB // 2 if shape["threads"] == 0 else 1,
            "step_roofline": {"bound": "hbm", "achieved": value * STEP_BYTES_PER_SITE / 1e3, "peak": peak,
                              "unit": "GB/s", "frac": value * STEP_BYTES_PER_SITE / 1e3 / peak,
                              "bytes_per_site": STEP_BYTES_PER_SITE, "peak_kind": kind},
            "plain_equal_sites": {"lattice": [side, side], "value": plain, "unit": "MLUPS"},
            "vs_plain_equal_sites": value / plain, "clocks": clocks.summary()}


def run_batched(args, rank, world, local):
    """512 independent drops (sides 32..256, half pushed by g_x = 1e-5 for the
    first 2000 of 6000 steps) advanced together on the path the library chose
    (persistent kernel or tiled launches, in a graph), against 512 plain
    lattices stepped one launch sequence each, same GPU, FP32."""
    import torch
    from paper_0902_3921_gb300 import build as B
    from paper_0902_3921_gb300 import inputs as I
    from paper_0902_3921_gb300 import lbm

    torch.cuda.set_device(local)
    B.build()
    lbm.load_library()
    desc = I.batch_instances(512, seed=rank)
    insts = [(d["side"], d["side"], (1e-5 if d["forced"] else 0.0, 0.0),
              2000 if d["forced"] else 0) for d in desc]
    common = lbm.LbmParams(precision=lbm.LBM_F32DEV, fd_substeps=M_SUB, **CFG)
    stream = torch.cuda.Stream()
    b = lbm.Batch(common, insts, stream=stream.cuda_stream)
    xi = (2 * CFG["kappa"] / -CFG["a"]) ** 0.5
    fields = []
    for k, d in enumerate(desc):
        phi = I.drop(2, d["side"], d["side"], R=d["R"], phi0=1.0, xi=xi)
        n, u = I.rest(2, d["side"], d["side"])
        fields.append((n, phi, u))
        b.init_fields(k, n, phi, u)
    sites = b.shape()["sites"]
    steps = args.batch_steps
    b.step(steps)  # warm-up, captures the graph for this (t0, nsteps)
    b.synchronize()
    for k, f in enumerate(fields):
        b.init_fields(k, *f)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        with torch.cuda.stream(stream):
            t0.record(stream)
            b.step(steps)
            t1.record(stream)
        torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    value = sites * steps / (ms / 1000.0) / 1e6
    shape = b.shape()
    b.close()
    # the same instances as plain lattices, one lbm_step per lattice and step
    os.environ["HLBM_TUNING"] = "4,16,2,0,0"
    lats = []
    for k, (Lx, Ly, g, fs) in enumerate(insts):
        lat = lbm.Lattice(lbm.LbmParams(Lx=Lx, Ly=Ly, fd_substeps=M_SUB, precision=lbm.LBM_F32DEV,
                                        g=(g[0], g[1], 0.0), force_steps=fs, **CFG),
                          stream=stream.cuda_stream)
        lbm.lbm_set_graphs(lat.handle, False)
        lat.init_fields(*fields[k])
        lats.append(lat)
    del os.environ["HLBM_TUNING"]
    plain_steps = args.plain_steps
    with torch.cuda.stream(stream):
        for lat in lats:
            lat.step(1)
    torch.cuda.synchronize()
    t0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(plain_steps):
            for lat in lats:
                lat.step(1)
    t1.record(stream)
    torch.cuda.synchronize()
    ms_plain = t0.elapsed_time(t1)
    plain = sites * plain_steps / (ms_plain / 1000.0) / 1e6
    for lat in lats:
        lat.close()
    if rank == 0:
        print(json.dumps({
            "metric": "MLUPS (512 independent D2Q9 hybrid lattices)", "value": value,
            "unit": "MLUPS", "n_gpus": world, "steps": steps, "ms_per_step": ms / steps,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched-512-drops-sides32-256", "sites": sites,
                       "instances": 512, "shape": shape, "fd_substeps": M_SUB},
            "plain_per_instance": {"value": plain, "unit": "MLUPS", "steps": plain_steps,
                                   "launches_per_step": 512 * 2},
            "speedup_vs_plain": value / plain, "clocks": clocks.summary()}), flush=True)


D3_SIDE = 256
D3_CFG = dict(CFG, N=1 / 6, Q=1 / 3)  # the 3D stencil weights of the 3D drop tests
D3_LB_PER_STEP = 10
# algorithmic bytes per site: D3Q19 populations read + written, phi read
D3_COLLIDE_BYTES = {"f32": 2 * 19 * 4 + 4, "f16": 2 * 19 * 2 + 4}
# FD3d per substep: phi read + written, u* (3 components) read (the fused
# minimum; the three-pass kernels also write and re-read phih and psi)
D3_FD_BYTES = 4 + 4 + 12
D3_M = 8
# whole-step algorithmic bytes per site: populations read and written, phi
# read and written (FP32: 19 x 4 x 2 + 8; FP16 deviations: 19 x 2 x 2 + 8)
D3_STEP_BYTES = {"f32": 160, "f16": 84}


def drop3d_form(side, steps, warmup, local, stream):
    """D3Q19 drop on a side^3 periodic lattice (R = 48 side/256, centred), FP32
    and FP16 deviations, m = 8 FD substeps; one timed step = lbm_step(10).
    Returns {"f32": ..., "f16": ...} with MLUPS, rooflines and clocks."""
    import torch
    from paper_0902_3921_gb300 import inputs as I
    from paper_0902_3921_gb300 import lbm

    S3 = side
    S = S3 ** 3
    xi = (2 * D3_CFG["kappa"] / -D3_CFG["a"]) ** 0.5
    phi0 = (-D3_CFG["a"] / D3_CFG["b"]) ** 0.5
    phi = I.drop(3, S3, S3, S3, R=48 * S3 / 256, phi0=phi0, xi=xi)
    n, u = I.rest(3, S3, S3, S3)
    out = {}
    peak, peak_kind = measured_peak()
    for name, prec in (("f32", lbm.LBM_F32DEV), ("f16", lbm.LBM_F16DEV)):
        lat = lbm.Lattice(lbm.LbmParams(dims=3, Lx=S3, Ly=S3, Lz=S3, precision=prec, **D3_CFG),
                          stream=stream.cuda_stream)
        lat.init_fields(n, phi, u)
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                lat.step(D3_LB_PER_STEP)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clocks:
            with torch.cuda.stream(stream):
                t0.record(stream)
                for _ in range(steps):
                    lat.step(D3_LB_PER_STEP)
                t1.record(stream)
            torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / steps
        value = S * D3_LB_PER_STEP / (ms / 1000.0) / 1e6
        lbm.lbm_set_kernel_timing(lat.handle, True)
        lbm.lbm_kernel_times(lat.handle, reset=True)
        with torch.cuda.stream(stream):
            lat.step(D3_LB_PER_STEP)
        kt = lbm.lbm_kernel_times(lat.handle, reset=True)
        lbm.lbm_set_kernel_timing(lat.handle, False)
        (cms, cn), (fms, fn) = kt["collide"], kt["fd"]
        if S3 in (128, 256) and os.environ.get("HLBM_FD3_FUSED_ADV"):
            fd_kind = "fd3p (m = 8 substeps, one kernel each: advection, psi and the new phi)"
        elif S3 in (128, 256):
            fd_kind = "fd3d (m = 8 substeps, each an advection pass and a fused psi / new-phi pass)"
        else:
            fd_kind = "fd3d (m = 8 substeps, three passes each: phih, psi, phi)"
        c_s, f_s = cms / cn / 1000.0, fms / fn / 1000.0  # f_s: all FD launches of one LB step
        ac = D3_COLLIDE_BYTES[name] * S / c_s / 1e9
        af = D3_M * D3_FD_BYTES * S / f_s / 1e9
        roof_c = {"bound": "hbm", "achieved": ac, "peak": peak, "unit": "GB/s", "frac": ac / peak,
                  "traffic": None, "kernel": "collide3d", "bytes_per_site": D3_COLLIDE_BYTES[name],
                  "avg_launch_us": c_s * 1e6, "peak_kind": peak_kind, "share_of_step": cms / (cms + fms)}
        roof_f = {"bound": "hbm", "achieved": af, "peak": peak, "unit": "GB/s", "frac": af / peak,
                  "traffic": None,
                  "kernel": fd_kind,
                  "bytes_per_site": D3_M * D3_FD_BYTES, "avg_launch_us": f_s * 1e6,
                  "note": f"avg_launch_us covers all FD launches of one LB step ({fn} launches)",
                  "peak_kind": peak_kind, "share_of_step": fms / (cms + fms)}
        dom, oth = (roof_c, roof_f) if cms >= fms else (roof_f, roof_c)
        step_bytes = D3_STEP_BYTES[name]
        out[name] = {"lattice": [S3, S3, S3], "value": value, "unit": "MLUPS", "ms_per_step": ms,
                     "lb_steps_per_timed_step": D3_LB_PER_STEP, "timed_steps": steps,
                     "step_roofline": {"bound": "hbm", "achieved": value * step_bytes / 1e3, "peak": peak,
                                       "unit": "GB/s", "frac": value * step_bytes / 1e3 / peak,
                                       "bytes_per_site": step_bytes, "peak_kind": peak_kind},
                     "roofline": dom, "roofline_other_kernel": oth,
                     "clocks": clocks.summary(), "launches_per_step": (cn + fn)}
        lat.close()
    return out


def run_drop3d(args, rank, world, local):
    """D3Q19 drop on a 256^3 periodic lattice (R = 48, centred), FP32 and FP16
    deviations, m = 8 FD substeps; one timed step = lbm_step(10)."""
    import torch
    from paper_0902_3921_gb300 import build as B
    from paper_0902_3921_gb300 import inputs as I
    from paper_0902_3921_gb300 import lbm

    torch.cuda.set_device(local)
    B.build()
    lbm.load_library()
    S3 = args.side3d
    stream = torch.cuda.Stream()
    out = drop3d_form(S3, args.steps, args.warmup, local, stream)
    xi = (2 * D3_CFG["kappa"] / -D3_CFG["a"]) ** 0.5
    phi0 = (-D3_CFG["a"] / D3_CFG["b"]) ** 0.5
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        import oracle as O
        O.build()
        op = O.Params(dims=3, Lx=64, Ly=64, Lz=64, m=8, **D3_CFG)
        p64 = I.drop(3, 64, 64, 64, R=12, phi0=phi0, xi=xi)
        n64, u64 = I.rest(3, 64, 64, 64)
        st = O.State.create(op, n64, p64, u64)
        tc = time.perf_counter()
        st.run(2)
        dt = time.perf_counter() - tc
        cpu = {"value": 64 ** 3 * 2 / dt / 1e6, "unit": "MLUPS", "cores": 1, "kind": "oracle",
               "sample": f"2 LB steps of a 64^3 drop ({dt:.1f} s, single thread)"}
    if rank == 0:
        f32 = out["f32"]
        print(json.dumps({
            "metric": "MLUPS (D3Q19 hybrid LB + FD step)", "value": f32["value"], "unit": "MLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": f32["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"drop3d-{S3}^3-d3q19", "lattice": [S3, S3, S3], "R": 48 * S3 // 256,
                       "lb_steps_per_timed_step": D3_LB_PER_STEP, "fd_substeps": 8,
                       "precision": "f32 deviations",
                       "l2": "working set (5.4 GB FP32 populations) exceeds L2"},
            "roofline": f32["roofline"], "roofline_other_kernel": f32["roofline_other_kernel"],
            "fp16_deviations": {"value": out["f16"]["value"], "unit": "MLUPS",
                                "roofline": out["f16"]["roofline"],
                                "roofline_other_kernel": out["f16"]["roofline_other_kernel"]},
            "cpu_baseline": cpu, "gpu_launches": f32["launches_per_step"] * args.steps,
            "clocks": f32["clocks"]}), flush=True)


SURR_SIDE = 2048
SURR_WINDOW = 50  # LB steps one forward pass replaces
# algorithmic bytes per pixel of one 32 -> 32 convolution layer: BF16 input
# and output activations, 32 channels each; FLOPs per pixel 2 x 9 x 32 x 32
CONV_BYTES_PER_PX = 128
CONV_FLOPS_PER_PX = 2 * 9 * 32 * 32
# DRAM bytes of one 32 -> 32 layer launch at 2048^2 from one ncu capture
# (profiles/conv_tc_surrogate2048.md)
NCU_TRAFFIC_CONV_2048 = 278.498816e6 + 222.286080e6


def cpu_surrogate_forward(side=64, reps=1):
    """The FP64 reference network (oracle/surrogate.py) on a side^2 lattice:
    pixels per second of one forward pass (single thread)."""
    from oracle import surrogate as OS
    rng = np.random.default_rng(0)
    chans = [4] + [32] * 5 + [4]
    params = [(rng.standard_normal((co, 3, 3, ci)) * 0.1, np.zeros(co)) for ci, co in zip(chans[:-1], chans[1:])]
    x = rng.standard_normal((1, side, side, 4))
    t = time.perf_counter()
    for _ in range(reps):
        OS.forward(params, x)
    dt = time.perf_counter() - t
    return side * side * reps / dt, dt


def surrogate_forward(steps, warmup, local, rank, stream):
    """The learned surrogate's step, x_{t+50} = x_t + Net(x_t), on the 2048^2
    inference lattice: six periodic 3x3 convolutions (4 -> 32 -> ... -> 32 ->
    4), BF16 weights and activations, FP32 accumulation on the tcgen05 tensor
    cores.  Weights are random (throughput does not depend on their values).
    value = lattice updates per second the forward pass stands in for
    (2048^2 sites x 50 LB steps per pass).  Returns (result dict, net, x0,
    x1); the caller closes the net."""
    import torch
    from paper_0902_3921_gb300 import lbm

    S = SURR_SIDE
    P = S * S
    net = lbm.Net(32, 6, seed=1)
    net.set_normalisation([0.0, 0.0, 0.0, 0.0], [0.6, 2e-3, 2e-3, 3e-3], [0.05, 1e-3, 1e-3, 1e-3])
    g = torch.Generator(device="cuda").manual_seed(rank)
    x0 = (0.5 * torch.randn(P * 4, device="cuda", generator=g)).contiguous()
    x1 = torch.empty_like(x0)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            net.forward(x0.data_ptr(), 1, S, S, x1.data_ptr(), stream=stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    steps = max(steps, 400)  # about 0.3 s, long enough for the clock samples
    with ClockSampler(local) as clocks:
        with torch.cuda.stream(stream):
            t0.record(stream)
            for _ in range(steps):
                net.forward(x0.data_ptr(), 1, S, S, x1.data_ptr(), stream=stream.cuda_stream)
            t1.record(stream)
        torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    value = P * SURR_WINDOW / (ms / 1000.0) / 1e6
    layer_ms = net.layer_times(x0.data_ptr(), 1, S, S, reps=max(3, steps // 20),
                               stream=stream.cuda_stream)
    dom = max(range(1, 5), key=lambda l: layer_ms[l])  # a 32 -> 32 layer
    conv_s = layer_ms[dom] / 1000.0
    achieved = CONV_BYTES_PER_PX * P / conv_s / 1e9
    hbm_peak, hbm_kind = measured_peak()
    tensor_tflops = CONV_FLOPS_PER_PX * P / conv_s / 1e12
    # measured BF16 burst throughput of a cuBLAS GEMM, else the 1.9 PFLOP/s
    # fallback measured on a GB300 before
    bf16_peak, bf16_kind = 1900.0, "fallback"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = json.load(f).get("bf16_tflops")
        if v:
            bf16_peak, bf16_kind = float(v), "measured"
    except (OSError, ValueError):
        pass
    res = {"value": value, "unit": "MLUPS-equivalent", "ms_per_forward": ms, "forwards_timed": steps,
           "lattice": [S, S], "window_lb_steps": SURR_WINDOW,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                        "frac": achieved / hbm_peak,
                        "traffic": NCU_TRAFFIC_CONV_2048 if S == 2048 else None,
                        "kernel": f"conv_tc layer {dom} (32 -> 32, tcgen05)",
                        "bytes_per_px": CONV_BYTES_PER_PX, "avg_launch_us": layer_ms[dom] * 1000.0,
                        "peak_kind": hbm_kind,
                        "tensor": {"achieved": tensor_tflops, "peak": bf16_peak, "unit": "TFLOP/s",
                                   "frac": tensor_tflops / bf16_peak, "peak_kind": bf16_kind}},
           "layer_us": [v * 1000.0 for v in layer_ms], "clocks": clocks.summary()}
    return res, net, x0, x1


def run_surrogate(args, rank, world, local):
    """The surrogate workload: the forward pass (surrogate_forward), end to end
    from pinned host memory, the plain scheme timed on the same lattice beside
    it, and the trained network's speedup at fixed error."""
    import torch
    from paper_0902_3921_gb300 import build as B
    from paper_0902_3921_gb300 import inputs as I
    from paper_0902_3921_gb300 import lbm

    torch.cuda.set_device(local)
    B.build()
    lbm.load_library()
    S = SURR_SIDE
    P = S * S
    stream = torch.cuda.Stream()
    fwd, net, x0, x1 = surrogate_forward(args.steps, args.warmup, local, rank, stream)
    value, ms, steps, layer_ms = fwd["value"], fwd["ms_per_forward"], fwd["forwards_timed"], fwd["layer_us"]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    # e2e: pinned host state in, prediction out, every step
    hx0 = torch.empty(P * 4, dtype=torch.float32, pin_memory=True)
    hx0.copy_(x0.cpu())
    hx1 = torch.empty_like(hx0, pin_memory=True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(args.steps):
            x0.copy_(hx0, non_blocking=True)
            net.forward(x0.data_ptr(), 1, S, S, x1.data_ptr(), stream=stream.cuda_stream)
            hx1.copy_(x1, non_blocking=True)
        e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1) / args.steps
    net.close()
    # the plain scheme on the same lattice: 50 LB steps per window
    lat = lbm.Lattice(lbm.LbmParams(Lx=S, Ly=S, fd_substeps=M_SUB, precision=lbm.LBM_F32DEV, **CFG),
                      stream=stream.cuda_stream)
    phi = I.spinodal(2, S, S, seed=rank, amp=0.01)
    n, u = I.rest(2, S, S)
    lat.init_fields(n, phi, u)
    with torch.cuda.stream(stream):
        lat.step(SURR_WINDOW)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        t0.record(stream)
        lat.step(SURR_WINDOW * 4)
        t1.record(stream)
    torch.cuda.synchronize()
    ms_plain = t0.elapsed_time(t1) / 4
    plain = P * SURR_WINDOW / (ms_plain / 1000.0) / 1e6
    lat.close()
    fixed = None if args.no_fixed_error else surrogate_fixed_error(S)
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        pxs, secs = cpu_surrogate_forward(side=256, reps=3)
        cpu = {"value": pxs * SURR_WINDOW / 1e6, "unit": "MLUPS-equivalent", "cores": 1, "kind": "oracle",
               "sample": f"three FP64 forward passes of the same network on a 256x256 lattice ({secs:.1f} s)"}
    if rank == 0:
        print(json.dumps({
            "metric": "MLUPS-equivalent of the surrogate step (2048^2, 50 LB steps per pass)",
            "value": value, "unit": "MLUPS", "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "surrogate-2048x2048-6x3x3conv-32ch", "pixels": P,
                       "window_lb_steps": SURR_WINDOW, "layers": 6, "channels": 32,
                       "l2": "activations (256 MiB per 32-channel layer) exceed L2"},
            "roofline": fwd["roofline"],
            "layer_us": layer_ms,
            "plain_scheme": {"value": plain, "unit": "MLUPS", "lattice": [S, S]},
            "speedup_vs_plain_per_window": value / plain,
            "fixed_error": fixed,
            "cpu_baseline": cpu,
            "e2e": {"value": P * SURR_WINDOW / (ms_e2e / 1000.0) / 1e6, "unit": "MLUPS",
                    "h2d_bytes_per_step": P * 16, "d2h_bytes_per_step": P * 16},
            "gpu_launches": 8 * steps,
            "clocks": fwd["clocks"]}), flush=True)


SURR_WEIGHTS = os.path.join(ROOT, "paper_0902_3921_gb300", "weights", "surrogate_32ch6_spinodal.npz")


def surrogate_fixed_error(side):
    """The trained network (paper_0902_3921_gb300/weights, trained on 512^2
    spinodal trajectories, t = 2000 ... 12000) against the plain scheme on
    the side^2 spinodal lattice (seed 1000) from t = 2000 to 16000, windows of
    50 LB steps with the residual check: wall-clock speedup and the errors of
    L(t) and S(k) at t = 4000, 8000, 16000."""
    import numpy as np
    from paper_0902_3921_gb300 import lbm
    from paper_0902_3921_gb300 import surrogate as SG

    if not os.path.exists(SURR_WEIGHTS):
        return None
    z = np.load(SURR_WEIGHTS)
    net = lbm.Net(32, 6, seed=0)
    net.set_params(z["params"])
    nrm = z["normalisation"]
    net.set_normalisation(nrm[0], nrm[1], nrm[2])
    res = SG.evaluate(net, side, checkpoints=(4000, 8000, 16000))
    net.close()
    rows = res["checkpoints"]
    return {"speedup": res["speedup"], "t": [2000, 16000], "lattice": [side, side], "seed": 1000,
            "windows": sum(r["windows"] for r in rows), "fallbacks": res["fallbacks"],
            "L_rel_err": [abs(r["L_surrogate"] - r["L_plain"]) / r["L_plain"] for r in rows],
            "S_rel_l2": [r["S_rel_l2"] for r in rows], "checkpoints": [r["t"] for r in rows],
            "ms_plain": res["ms_plain"], "ms_surrogate": res["ms_surrogate"],
            "weights": os.path.relpath(SURR_WEIGHTS, ROOT)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample-steps", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lattice", type=int, default=L,
                    help="lattice side (the workload is 1024; other sides are for profiling)")
    ap.add_argument("--no-large", action="store_true", help="skip the 4096^2 (--large-side) line")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the batched, 3D and surrogate sub-results of the default line")
    ap.add_argument("--large-side", type=int, default=4096)
    ap.add_argument("--quick", action="store_true",
                    help="timed region only (no kernel timing, e2e or CPU baseline)")
    ap.add_argument("--no-graphs", action="store_true", help="launch kernels one by one")
    ap.add_argument("--workload", default="spinodal", choices=["spinodal", "batched", "surrogate", "drop3d"])
    ap.add_argument("--batch-steps", type=int, default=200)
    ap.add_argument("--side3d", type=int, default=D3_SIDE,
                    help="3D lattice side (the workload is 256; smaller sides are for profiling)")
    ap.add_argument("--plain-steps", type=int, default=10)
    ap.add_argument("--no-fixed-error", action="store_true",
                    help="surrogate workload: skip the trained network's speedup-at-fixed-error run")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batched":
        run_batched(args, rank, world, local)
    elif args.workload == "surrogate":
        run_surrogate(args, rank, world, local)
    elif args.workload == "drop3d":
        run_drop3d(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
