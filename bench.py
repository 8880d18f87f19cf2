"""Throughput benchmark of the colour-gradient LBM step (MLUPS = million fluid-node updates/s).

Default workload: the batched parameter sweep -- 64 displacement channels, widths W drawn
from U{40..200} (seed 0), lengths 10 W, velocity inlet / pressure outlet, walls top and
bottom, (M, Ca, theta) drawn from the grids M in {1,5,20,50,100}, Ca in {0.01,0.05,0.1},
theta in {30,...,150} deg -- in FP32.  One benchmark step = one time step of all 64
channels (one launch per kernel for the whole batch).  The state (about 1.5 GB) is far
larger than the 129 MB L2, so no flush is needed; smaller workloads flush L2 before every
timed step and are timed per step with CUDA events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--precision P]
    python bench.py --impl reference ...      # the FP64 CPU oracle on the host cores

Under torchrun each rank runs its own batch (weak scaling, no collective on the data path);
rank 0 prints one JSON line.
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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_1707_00198_gb300 import inputs as I  # noqa: E402

L2_BYTES = 129 * 2 ** 20
STORE_BYTES = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}
DTYPE = {"fp64": "f64", "fp32": "f32", "fp16": "f16-store/f32-math", "bf16": "bf16-store/f32-math"}


# ----------------------------------------------------------------------------- workloads
def workload(name: str, rank: int = 0, lattices: int = 64):
    """The synthetic workload of one rank.  The batched sweep gives every rank the same
    channel widths (equal work: weak scaling) with its own draw of (M, Ca, theta); the
    single-lattice workloads are replicas."""
    if name == "batched_sweep":
        return I.channel_sweep(lattices, seed=0, param_seed=rank if rank else None), \
            f"{lattices} displacement channels, W~U{{40..200}}, L=10W, (M,Ca,theta) grids"
    if name == "capillary":
        g, p = I.config_capillary()
        return ([g], [p]), "capillary filling 1200x80, d=40, L=800, theta=30deg, sigma=1e-2"
    if name == "fingering":
        g, p = I.config_fingering(M=1.0, Ca=0.05, theta_deg=90.0, seed=0)
        return ([g], [p]), "displacement channel 2000x102, M=1, Ca=0.05, theta=90deg"
    if name == "fingering_grid":
        return I.fingering_grid(), "75 displacement channels 2000x102, the full (M, Ca, theta) grid"
    if name == "static_droplet":
        g, p = I.config_static_droplet()
        return ([g], [p]), "static droplet 100x50, R=20, theta=60deg"
    if name == "roofline_box":
        g = I.two_wall_box(8192, 4096, bands=8, noise=1e-3, seed=0)
        return ([g], [I.Params(sigma=0.01, theta=math.radians(60))]), "two-wall box 8192x4096, 8 colour bands"
    raise SystemExit(f"unknown workload {name}")


def reference_sample(geoms, prms):
    """A bounded sample of the workload for the CPU oracle: the first lattice cropped to a
    100-node-long section (same width, boundaries and parameters)."""
    g, p = geoms[0], prms[0]
    if g.bc_x == "inout":
        g2 = I.displacement_channel(W=g.ny - 2, L=min(100, g.nx), x_I=min(25.0, g.nx / 4), seed=7)
    else:
        nx = min(100, g.nx)
        bc_x = g.bc_x
        solid = g.solid[:, :nx].copy()
        if bc_x == "closed":
            solid[:, -1] = 1
        g2 = I.Geometry(nx, g.ny, solid, g.rhoN0[:, :nx].copy(), bc_x=bc_x, bc_y=g.bc_y)
    return g2, p


def fluid_nodes(geoms) -> int:
    return int(sum(int((g.solid == 0).sum()) for g in geoms))


# ----------------------------------------------------------------------------- helpers
def reduce_over_ranks(ms: float, nf: int, ws: int, device: str):
    """(max over ranks of the timed region in ms, fluid nodes summed over ranks)."""
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    n = torch.tensor([float(nf)], dtype=torch.float64, device=device)
    if ws > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(n)
    return float(t.item()), int(round(n.item()))


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            r = [c.strip() for c in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def kernel_source_digest() -> str:
    """Digest of the kernel sources' code: // comments and whitespace are left out, so that a
    comment edit does not invalidate counters taken from the same code."""
    h = hashlib.sha256()
    for f in ("lbcg_kernels.cu", "lbcg_device.cuh", "lbcg_geom.h"):
        text = open(os.path.join(ROOT, "paper_1707_00198_gb300", "csrc", f), encoding="utf-8").read()
        code = "\n".join(" ".join(line.split("//", 1)[0].split()) for line in text.splitlines())
        h.update(code.encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, n_fluid: int):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, scaled by fluid
    nodes, or None if the kernel source changed since the counters were taken."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))[kernel]
    except Exception:
        return None
    if rec.get("src_digest") != kernel_source_digest() or "dram_bytes_per_fluid_node" not in rec:
        return None
    return rec["dram_bytes_per_fluid_node"] * n_fluid


def recorded_counter(kernel: str, key: str):
    """A per-fluid-node figure of `kernel` recorded from ncu in profiles/ncu_traffic.json, or
    None if it is absent or the kernel source changed since the counters were taken."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))[kernel]
    except Exception:
        return None
    if rec.get("src_digest") != kernel_source_digest() or key not in rec:
        return None
    return rec[key]


def fp64_rate_tflops(n: int = 4096, reps: int = 3) -> float:
    """Measured FP64 rate of this GPU: cuBLAS DGEMM (torch.matmul of two float64 n x n
    matrices), best of `reps`, CUDA events, 2 n^3 flops."""
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b
    return 2 * n ** 3 / (best / 1e3) / 1e12


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the CPU-baseline record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_oracle_rate(geoms, prms, budget_s: float = 15.0, max_steps: int = 100000):
    """Time the FP64 oracle (as it stands) on a bounded sample; returns (MLUPS, steps, nodes, cores)."""
    from oracle import lbcg_oracle as O
    g, p = reference_sample(geoms, prms)
    lat = O.make_lattice(g, p.theta)
    fR, fB = O.init_state(lat, g.rhoN0, p.rho0, p)
    nf = int((g.solid == 0).sum())
    t0 = time.perf_counter()
    fR, fB = O.run(lat, p, fR, fB, 2)
    per = (time.perf_counter() - t0) / 2
    n = int(max(3, min(max_steps, budget_s / max(per, 1e-6))))
    t0 = time.perf_counter()
    O.run(lat, p, fR, fB, n)
    dt = time.perf_counter() - t0
    return nf * n / dt / 1e6, n, (g.nx, g.ny, nf), torch.get_num_threads()


def c_step_rate(g, p, threads: int, budget_s: float = 2.0, steps: int = 0, warmup: int = 1):
    """Time the plain C/OpenMP step (oracle/lbcg_cpu.c, as it stands) on lattice g with the given
    number of threads (0 = all).  Returns (MLUPS, steps timed, seconds)."""
    from oracle import cpu_step as CS
    C = CS.CpuLattice(g, p)
    f = C.init_state()
    f = C.run(*f, warmup, threads=threads)
    nf = int((g.solid == 0).sum())
    if steps <= 0:
        t0 = time.perf_counter()
        f = C.run(*f, 1, threads=threads)
        steps = int(max(2, min(100000, budget_s / max(time.perf_counter() - t0, 1e-6))))
    t0 = time.perf_counter()
    C.run(*f, steps, threads=threads)
    dt = time.perf_counter() - t0
    C.close()
    return nf * steps / dt / 1e6, steps, dt


def cpu_baseline_record(geoms, prms, desc):
    """The CPU baseline: the C step on the first lattice of the workload, on all host cores
    (the reported value) and on one core, plus the same for the static-droplet (100 x 50) and
    fingering (2000 x 102, M = 1, Ca = 0.05, theta = 90 deg) configurations, and the PyTorch
    oracle's rate on a section for context.  About 20 s of CPU time."""
    from oracle import cpu_step as CS
    g, p = geoms[0], prms[0]
    cores = len(os.sched_getaffinity(0))
    v_all, n_all, _ = c_step_rate(g, p, cores)
    v_one, _, _ = c_step_rate(g, p, 1)
    cfg = {}
    for name, (gg, pp) in (("static_droplet_100x50", I.config_static_droplet()),
                           ("fingering_2000x102", I.config_fingering(M=1.0, Ca=0.05, theta_deg=90.0))):
        cfg[name] = {"all_cores": c_step_rate(gg, pp, cores)[0], "one_core": c_step_rate(gg, pp, 1, budget_s=1.0)[0]}
    ov, on, (sx, sy, snf), ocores = cpu_oracle_rate(geoms, prms, budget_s=4.0)
    return {"value": v_all, "unit": "MLUPS", "cores": CS.threads_used(cores), "kind": "oracle",
            "impl": "plain C/OpenMP FP64 step (oracle/lbcg_cpu.c)", "cpu_model": cpu_model(),
            "cores_available": cores, "one_core": v_one,
            "sample": f"{n_all} FP64 steps of the first lattice ({g.nx}x{g.ny}, {int((g.solid == 0).sum())} fluid "
                      f"nodes) of: {desc}",
            "configs_MLUPS": cfg,
            "pytorch_oracle": {"value": ov, "cores": ocores,
                               "sample": f"{on} steps of a {sx}x{sy} section ({snf} fluid nodes)"}}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The reference arm: the plain C/OpenMP step of oracle/ (as it stands) on the host cores,
    each step one step of the first lattice of the workload."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import cpu_step as CS
    (geoms, prms), desc = workload(args.workload, rank=0, lattices=args.lattices)
    g, p = geoms[0], prms[0]
    cores = len(os.sched_getaffinity(0))
    nf = int((g.solid == 0).sum())
    v, n, dt = c_step_rate(g, p, cores, steps=args.steps, warmup=args.warmup)
    sample = f"the first lattice ({g.nx}x{g.ny}, {nf} fluid nodes) of: {desc}"
    line = {"impl": "reference", "metric": "MLUPS", "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "precision": "fp64 (CPU, plain C/OpenMP)"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": CS.threads_used(cores), "kind": "oracle",
                             "impl": "plain C/OpenMP FP64 step (oracle/lbcg_cpu.c)", "cpu_model": cpu_model(),
                             "cores_available": cores, "sample": sample},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- our arm
AUTOTUNE_PROBE = 20   # launches per candidate schedule in lbcg_autotune


def timed_steps(lat, stream, K, flush_buf):
    """K steps; returns total device ms (per-step events when flushing L2 between steps).
    Without flushing the K steps are one lbcg_step call, which replays the handle's CUDA graph
    of 32 steps."""
    if flush_buf is None:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.step(K)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with torch.cuda.stream(stream):
        for k in range(K):
            flush_buf.add_(1)
            evs[k][0].record(stream)
            lat.step(1)
            evs[k][1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs)


def measure_form(geoms, prms, precision, K, W, stream, with_profile=False, ty=0):
    from paper_1707_00198_gb300 import lbcg
    lat = lbcg.Lattice(geoms, prms, precision, stream=stream.cuda_stream)
    if ty:
        lat.set_tile(ty)
    else:
        lat.autotune(AUTOTUNE_PROBE)
    lat.step(W)
    torch.cuda.synchronize()
    flush = None
    if lat.state_bytes < 2 * L2_BYTES:
        flush = torch.zeros(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    if with_profile:
        lbcg.lbcg_profile(lat.h, True)
    ms = timed_steps(lat, stream, K, flush)
    kt = None
    if with_profile:
        kt = lbcg.lbcg_kernel_times(lat.h)
        lbcg.lbcg_profile(lat.h, False)
    return lat, ms, kt, flush is not None


def sequential_rate(lbcg, geoms, prms, precision: str, K: int, W: int, stream) -> dict:
    """The same channels as independent single-lattice handles, stepped one after another
    (each with the schedule lbcg_autotune picks for it and CUDA-graph replay): the baseline
    the batched launch is compared with."""
    hs = [lbcg.Lattice(g, p, precision, stream=stream.cuda_stream) for g, p in zip(geoms, prms)]
    try:
        for L in hs:
            L.autotune(AUTOTUNE_PROBE)
            L.step(W)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for L in hs:
                L.step(K)
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    finally:
        for L in hs:
            L.close()
    nf = fluid_nodes(geoms)
    return {"MLUPS": nf * K / (ms / 1e3) / 1e6, "steps": K, "handles": len(geoms),
            "schedules": "each handle's own lbcg_autotune choice"}


def config_rates(lbcg, stream, K: int = 640) -> dict:
    """MLUPS of single lattices at the paper's configuration sizes, each on the schedule
    lbcg_autotune picks for it and replayed from its CUDA graph: the static droplet (100x50,
    FP64), capillary filling (1200x80, FP32) and the fingering channel (2000x102, M=1, Ca=0.05,
    theta=90 deg; FP32, FP16 and BF16 storage).  Their states fit in L2 and are not flushed
    between steps, so these are L2-resident rates."""
    cases = [("static_droplet_100x50", I.config_static_droplet(), ("fp64",)),
             ("capillary_1200x80", I.config_capillary(), ("fp64", "fp32")),
             ("fingering_2000x102", I.config_fingering(M=1.0, Ca=0.05, theta_deg=90.0), ("fp32", "fp16", "bf16"))]
    out = {"l2": "resident (states of 0.7-30 MB, not flushed)", "steps": K}
    for name, (g, p), precs in cases:
        nf = int((g.solid == 0).sum())
        for prec in precs:
            L = lbcg.Lattice(g, p, prec, stream=stream.cuda_stream)
            try:
                L.autotune(AUTOTUNE_PROBE)
                L.step(64)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                L.step(K)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                out[f"{name}_{prec}"] = {"MLUPS": nf * K / (ms / 1e3) / 1e6, "us_per_step": ms / K * 1e3,
                                         "schedule": f"tiles 32x{L.schedule}" if L.schedule else
                                         f"y-sweep, {L.sweep_rows or 'automatic'}-row segments"}
            finally:
                L.close()
    return out


def fingering_grid_rates(lbcg, stream, K: int = 320, W: int = 10) -> dict:
    """MLUPS of the viscous-fingering study run as one batch -- a 2000x102 channel for each of
    the 75 (M, Ca, theta) points of the grids (15.3 M fluid nodes) -- in FP32 and the two 16-bit
    storage forms, each on the schedule lbcg_autotune picks and replayed from its CUDA graph.
    The states (1.1-2.2 GB) are larger than L2."""
    geoms, prms = I.fingering_grid()
    nf = fluid_nodes(geoms)
    out = {"lattices": len(geoms), "fluid_nodes": nf, "steps": K, "l2": "inputs larger than L2"}
    for prec in ("fp32", "fp16", "bf16"):
        L, ms, _, _ = measure_form(geoms, prms, prec, K, W, stream)
        try:
            out[prec] = {"MLUPS": nf * K / (ms / 1e3) / 1e6, "ms_per_step": ms / K,
                         "hbm_gbs_alg": 36 * STORE_BYTES[prec] * nf * K / (ms / 1e3) / 1e9,
                         "schedule": f"tiles 32x{L.schedule}" if L.schedule else
                         f"y-sweep, {L.sweep_rows or 'automatic'}-row segments"}
        finally:
            L.close()
    return out


def observable_errors(lbcg, stream) -> dict:
    """Error of each storage form's observables against an FP64 run of the same case: the
    sessile droplet (100x50, theta 60 deg) after 2000 steps -- contact angle and colour masses --
    and a fingering channel (400x42, M=5, Ca=0.05, theta=60 deg) after 4000 steps -- finger-tip
    position, finger length and contact-line speed over the last 2000 steps."""
    gd, pd = I.config_static_droplet()
    gf, pf = I.displacement_channel(W=40, L=400, x_I=40.0, seed=0), I.fingering_params(5.0, 0.05, 60.0)

    def droplet(prec):
        L = lbcg.Lattice(gd, pd, prec, stream=stream.cuda_stream)
        try:
            o0 = L.observables(wall_y=0.5)
            L.step(2000)
            o = L.observables(wall_y=0.5)
        finally:
            L.close()
        return o["theta_deg"], o["mass_R"], o["mass_B"], o0["mass_R"]

    def finger(prec):
        L = lbcg.Lattice(gf, pf, prec, stream=stream.cuda_stream)
        try:
            L.step(2000)
            a = L.observables()
            L.step(2000)
            b = L.observables()
        finally:
            L.close()
        return b["x_tip"], b["x_tip"] - b["x_cl"], (b["x_cl"] - a["x_cl"]) / 2000.0

    ref_d, ref_f = droplet("fp64"), finger("fp64")
    out = {"reference": {"theta_deg": ref_d[0], "x_tip": ref_f[0], "finger_length": ref_f[1], "dS_dt": ref_f[2]}}
    for prec in ("fp32", "fp16", "bf16"):
        d, f = droplet(prec), finger(prec)
        out[prec] = {"theta_deg_err": d[0] - ref_d[0], "mass_R_rel_err": (d[1] - ref_d[1]) / ref_d[1],
                     "x_tip_rel_err": (f[0] - ref_f[0]) / ref_f[0], "finger_length_err": f[1] - ref_f[1],
                     "dS_dt_rel_err": (f[2] - ref_f[2]) / ref_f[2]}
    return out


def adjoint_rate(lbcg, stream, T: int, K: int, precision: str = "fp32", reverse: str = "fp64"):
    """Wall time of lbcg_adjoint (forward with checkpoints + reverse sweep) for the finger
    length of a 400x42 displacement channel, M=10, Ca=0.05, theta=60 deg; the forward steps
    and checkpoints in `precision`, the reverse sweep in `reverse`."""
    g, p = I.config_adjoint()
    L = lbcg.Lattice(g, p, precision, stream=stream.cuda_stream)
    try:
        L.adjoint(2 * K, K, reverse_fp32=reverse == "fp32")   # warm-up: first launches, allocations
        L.close()
        L = lbcg.Lattice(g, p, precision, stream=stream.cuda_stream)
        sched = L.autotune(AUTOTUNE_PROBE)   # the forward steps' schedule (the state is kept)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = L.adjoint(T, K, reverse_fp32=reverse == "fp32")
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
    except Exception as e:  # noqa: BLE001 -- reported, not hidden
        return {"error": str(e)}
    finally:
        L.close()
    nf = int((g.solid == 0).sum())
    return {"workload": f"displacement channel {g.nx}x{g.ny}, M=10, Ca=0.05, theta=60deg, J = finger length",
            "precision": f"{precision} forward, {reverse} reverse", "steps": T, "checkpoint": K, "seconds": t,
            "forward_schedule": f"tiles 32x{sched}" if sched else "y-sweep",
            "s_per_step": t / T,
            "mlups_forward_plus_reverse": nf * T / t / 1e6, "J": out["J"], "dJ_dtheta": out["dtheta"],
            "dJ_dsigma": out["dsigma"], "dJ_dnu_R": out["dnu_R"], "dJ_dnu_B": out["dnu_B"],
            "timing": "host clock around the whole call (it synchronises)"}


def run_ours(args):
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__ as ge
    ge.build()
    from paper_1707_00198_gb300 import lbcg

    (geoms, prms), desc = workload(args.workload, rank=rank, lattices=args.lattices)
    nf = fluid_nodes(geoms)
    nodes = sum(g.nx * g.ny for g in geoms)
    stream = torch.cuda.Stream()
    s_bytes = STORE_BYTES[args.precision]

    # ---- timed region: K steps of the whole batch, kernels timed with events on the stream
    clocks = Clocks(local)
    lat = lbcg.Lattice(geoms, prms, args.precision, stream=stream.cuda_stream)
    if args.ty:
        lat.set_tile(args.ty)
    elif args.rows:
        lat.set_sweep(args.rows)
    else:
        lat.autotune(AUTOTUNE_PROBE)   # sweep segment heights and tile shapes, on the initial state
    sched, rows = lat.schedule, lat.sweep_rows
    lat.step(args.warmup)
    torch.cuda.synchronize()
    flush = torch.zeros(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda") if lat.state_bytes < 2 * L2_BYTES \
        else None
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = lat.step_launches
    ms = timed_steps(lat, stream, args.steps, flush)
    torch.cuda.synchronize()
    launches = lat.step_launches - launches0   # kernel launches of the timed region, graph nodes counted
    clk = clocks.stop()
    if ws > 1:
        torch.distributed.barrier()
    # kernel durations: a separate pass with an event around each kernel (direct launches)
    Kp = min(args.steps, 200)
    lbcg.lbcg_profile(lat.h, True)
    ms_prof = timed_steps(lat, stream, Kp, flush)
    kms, ksteps = lbcg.lbcg_kernel_times(lat.h)
    lbcg.lbcg_profile(lat.h, False)
    ms_max, nf_total = reduce_over_ranks(ms, nf, ws, "cuda")
    value = nf_total * args.steps / (ms_max / 1e3) / 1e6
    obs = lbcg.lbcg_observables(lat.h, 0, lbcg.obs_spec(ny=geoms[0].ny), raise_on_diverged=False)

    # ---- roofline of the dominant kernel (k_step)
    step_ms = kms[1] / max(ksteps, 1)
    alg_bytes = 36 * s_bytes * nf
    achieved = alg_bytes / (step_ms / 1e3) / 1e9
    peaks = measured_peaks()
    peak, peak_src = (peaks["hbm_gbs"], "measured") if peaks and "hbm_gbs" in peaks else (6800.0, "fallback")
    if sched:
        kname = f"k_step<{args.precision},ty{sched}>"
    else:
        kname = "k_sweep<fp64>" if args.precision == "fp64" else f"k_sweepf<{args.precision}>"
    traffic = recorded_traffic(kname, nf)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": kname, "peak_source": peak_src,
            "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": step_ms,
            "kernel_ms_share": {"k_wall": kms[0] / ms_prof, "step kernel": kms[1] / ms_prof},
            "kernel_ms_source": f"separate pass of {Kp} steps launched as the graph's branches, CUDA events "
                                "around each kernel; per step, the time during which at least one branch's "
                                "kernel of that kind ran (union of the event intervals)"}
    flops_node = recorded_counter(kname, "fp64_flops_per_fluid_node") if args.precision == "fp64" else None
    if flops_node is not None:
        # the FP64 sweep is bound by FP64 arithmetic, not by memory: its roofline is the FP64
        # flops it executes (DFMA counted twice, DADD and DMUL once; from ncu) against the
        # measured DGEMM rate (GB300's FP64 units: 1.25 TFLOP/s nominal)
        fp64_peak = fp64_rate_tflops()
        ach = flops_node * nf / (step_ms / 1e3) / 1e12
        roof.update({"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach / fp64_peak,
                     "peak_source": "measured: cuBLAS DGEMM 4096^3 through torch.matmul, best of 3",
                     "fp64_flops_per_fluid_node": flops_node, "hbm_achieved_gbs": achieved,
                     "hbm_frac": achieved / peak})
    whole_gbs = alg_bytes * args.steps / (ms / 1e3) / 1e9

    # ---- end to end through the C ABI with host buffers (pinned): upload state, step, download
    sb = lat.state_bytes
    pin = torch.empty(sb, dtype=torch.uint8, pin_memory=True)
    lbcg.lbcg_download_state(lat.h, pin.data_ptr(), sb)
    Ke = max(3, min(args.steps, 20))
    lbcg.lbcg_step_host(lat.h, pin.data_ptr(), pin.data_ptr(), sb, 1)   # untimed: its streams and events
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(Ke):
        lbcg.lbcg_step_host(lat.h, pin.data_ptr(), pin.data_ptr(), sb, 1)
    torch.cuda.synchronize()
    te = time.perf_counter() - t0
    e2e = {"value": nf * Ke / te / 1e6 * (nf_total / nf), "unit": "MLUPS", "h2d_bytes_per_step": sb,
           "d2h_bytes_per_step": sb, "steps": Ke,
           "path": "lbcg_step_host per step: the whole state from pinned host memory, one step, the "
                   "whole state back, the copies of 8 lattice groups overlapping their steps"}
    lat.close()

    # ---- the other storage forms on the same workload, the same number of timed steps, each with
    # the roofline of its step kernel (algorithmic bytes / CUDA-event kernel time)
    forms = {}
    if not args.no_forms:
        for prec in ("fp32", "fp16", "bf16"):
            if prec == args.precision:
                forms[prec] = {"MLUPS": value / ws, "ms_per_step": ms / args.steps, "steps": args.steps,
                               "hbm_gbs_alg": whole_gbs,
                               "roofline": {"kernel": kname, "avg_launch_ms": step_ms, "achieved": achieved,
                                            "peak": peak, "frac": achieved / peak, "unit": "GB/s"}}
                continue
            L2, msf, _, _ = measure_form(geoms, prms, prec, args.steps, args.warmup, stream, ty=args.ty)
            lbcg.lbcg_profile(L2.h, True)
            timed_steps(L2, stream, Kp, None)
            kf, kn = lbcg.lbcg_kernel_times(L2.h)
            lbcg.lbcg_profile(L2.h, False)
            sched_f = L2.schedule
            L2.close()
            kms_f = kf[1] / max(kn, 1)
            alg_f = 36 * STORE_BYTES[prec] * nf
            forms[prec] = {"MLUPS": nf * args.steps / (msf / 1e3) / 1e6, "ms_per_step": msf / args.steps,
                           "steps": args.steps,
                           "hbm_gbs_alg": alg_f * args.steps / (msf / 1e3) / 1e9,
                           "roofline": {"kernel": f"k_step<{prec},ty{sched_f}>" if sched_f else f"k_sweepf<{prec}>",
                                        "avg_launch_ms": kms_f, "achieved": alg_f / (kms_f / 1e3) / 1e9,
                                        "peak": peak, "frac": alg_f / (kms_f / 1e3) / 1e9 / peak, "unit": "GB/s"}}

    # ---- batched launch against the same channels as sequential single-lattice runs
    seq = None
    if rank == 0 and args.workload == "batched_sweep" and not args.no_forms:
        seq = sequential_rate(lbcg, geoms, prms, args.precision, max(10, args.steps // 10), args.warmup, stream)
        seq["batched_MLUPS"] = value / ws
        seq["batched_speedup"] = seq["batched_MLUPS"] / seq["MLUPS"]

    # ---- observable error of the storage forms against FP64 (rank 0)
    obs_err = observable_errors(lbcg, stream) if (rank == 0 and not args.no_forms) else None
    # ---- single lattices at the paper's configuration sizes (rank 0)
    cfg_rates = config_rates(lbcg, stream) if (rank == 0 and not args.no_forms) else None
    grid_rates = fingering_grid_rates(lbcg, stream) if (rank == 0 and not args.no_forms) else None

    # ---- the discrete adjoint on the 400x42 channel (FP64, rank 0)
    adj = None
    if rank == 0 and not args.no_adjoint:
        adj = adjoint_rate(lbcg, stream, args.adjoint_steps, args.adjoint_checkpoint, "fp32", "fp32")
        adj["fp32_fp64_reverse"] = adjoint_rate(lbcg, stream, args.adjoint_steps, args.adjoint_checkpoint, "fp32", "fp64")
        adj["fp64"] = adjoint_rate(lbcg, stream, args.adjoint_steps, args.adjoint_checkpoint, "fp64", "fp64")

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N=1 only)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline_record(geoms, prms, desc)

    if rank == 0:
        line = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
                "config": {"workload": args.workload, "description": desc, "lattices": len(geoms), "nodes": nodes,
                           "schedule": (f"tiles 32x{sched}" if sched else
                                        "y-sweep, 124-column strips, " +
                                        (f"{rows}-row segments" if rows else "automatic segment height")) +
                           ("" if (args.ty or args.rows) else " (chosen by lbcg_autotune)"),
                           "fluid_nodes_per_gpu": nf, "precision": args.precision,
                           "state_bytes": sb, "l2": "flushed before every timed step" if flush is not None
                           else "inputs larger than L2", "mlups_counts": "fluid-node updates"},
                "hbm_gbs_alg": whole_gbs, "hbm_frac_alg": whole_gbs / peak,
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
                "forms": forms, "observable_error_vs_fp64": obs_err, "batched_vs_sequential": seq,
                "config_sizes": cfg_rates, "fingering_grid_batch": grid_rates, "adjoint": adj,
                "nonfinite_lattice0": obs.get("nonfinite", None)}
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default="batched_sweep",
                    choices=("batched_sweep", "fingering_grid", "capillary", "fingering", "static_droplet",
                             "roofline_box"))
    ap.add_argument("--precision", default="fp32", choices=("fp64", "fp32", "fp16", "bf16"))
    ap.add_argument("--lattices", type=int, default=64, help="channels of the batched sweep")
    ap.add_argument("--ty", type=int, default=0, help="tile height of k_step (4, 8, 16; 0 = default)")
    ap.add_argument("--rows", type=int, default=0,
                    help="y-sweep with this many rows per strip segment instead of lbcg_autotune's choice")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--adjoint-steps", type=int, default=4000)
    ap.add_argument("--adjoint-checkpoint", type=int, default=200)
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
