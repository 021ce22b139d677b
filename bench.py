#!/usr/bin/env python3
"""Benchmark of the LBM hot path on GB300: MLUPS and fraction of the HBM roofline.

Workload (one "step" = one lbm_step: boundary/ghost fill + fused stream-collide sweep):
  D3Q19 TRT (Lambda = 3/16, tau = 1), 256^3 channel, no-slip bounce-back walls in y
  (halfway, solid ghost layers), periodic x and z, body force (1e-6, 0, 0), rest start.
  Headline variant: FP32 storage (two-grid unless --variant says otherwise); the other
  variants (FP64 / FP32 x two-grid / AA) are reported under "variants".

Timing: W untimed warm-up steps, then K steps bracketed by a barrier and a device
synchronisation, measured with CUDA events on the library's stream; max over ranks.  The
state (2 x 2.6 GB for FP32 two-grid) is far larger than L2 (129 MB), so no L2 flush is
needed between steps.  Per-kernel device times come from the library's own event tracing
(lbm_enable_timing / lbm_read_timing) on the same stream.

--impl reference times the CPU oracle (the plain FP64 C program the parity tests use) on
a bounded sample of the same workload: each step is one oracle time step of a
256 x 256 x d slab of the channel (periodic in z, identical per-cell work), d <= 8 chosen so
that the run takes about a minute.

Multi-GPU: every rank runs an independent replica of the workload on its own GPU (the
path is not sharded); value = total lattice updates of all ranks / max time.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SHAPE = (256, 256, 256)
FORCE = (1e-6, 0.0, 0.0)
OMEGA = 1.0
LAMBDA = 3.0 / 16.0
METRIC = "MLUPS (lattice updates per second) of the fused stream-collide step and % of HBM roofline"
WORKLOAD = "D3Q19 TRT (Lambda=3/16, tau=1) channel 256^3, no-slip walls in y, periodic x/z, body force 1e-6"
VARIANTS = {
    "fp32-twogrid": ("FP32", "TWO_GRID", "TRT"),
    "fp32-aa": ("FP32", "AA", "TRT"),
    "fp64-twogrid": ("FP64", "TWO_GRID", "TRT"),
    "fp64-aa": ("FP64", "AA", "TRT"),
    "fp16dev-twogrid": ("FP16_DEV", "TWO_GRID", "TRT"),
    "fp16dev-aa": ("FP16_DEV", "AA", "TRT"),
    "bf16dev-twogrid": ("BF16_DEV", "TWO_GRID", "TRT"),
    "fp32-mrt-twogrid": ("FP32", "TWO_GRID", "MRT"),
    "fp64-mrt-twogrid": ("FP64", "TWO_GRID", "MRT"),
}
# MRT variants: shear rate omega, third order omega- (Lambda), bulk and fourth-order rates below
# (the fifth and sixth groups exist on D3Q27 only)
MRT_RATES = (1.4, 1.2, 1.0, 1.0)
# stated error of each variant: the channel after ERROR_STEPS steps against the oracle's column
ERROR_STEPS = 2000
ERROR_SHAPE = (32, 256, 32)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------------------------------
# distributed plumbing (one process per GPU; replicas)
# ---------------------------------------------------------------------------------------
def dist_setup(backend=None):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            return rank, world, local
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(local)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(value: float, world: int) -> float:
    """Max of a float over ranks (timing: the slowest rank defines the step time)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(units_per_rank: float, seconds_per_rank: float, world: int):
    """Whole-job throughput: units of all ranks / max time over ranks."""
    tmax = reduce_max(seconds_per_rank, world)
    return units_per_rank * world / tmax, tmax


# ---------------------------------------------------------------------------------------
# measurement helpers
# ---------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.strip()]
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except (ValueError, IndexError):
                continue
            for k, n in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip().lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def sweep_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1909_13772_gb300", "csrc")
    for name in ("sweep.cu", "cell.cuh", "cumulant.cuh", "kernels.cuh", "lattice.cuh", "select.cuh"):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# FP64 pipe of one GB300: ncu's peak for DFMA-pipe thread-instructions is 2 per clock per SM;
# x 152 SMs x 2,070 MHz (maximum SM clock) = 629.3 G thread-instructions/s (derived, not measured).
FP64_PIPE_PEAK_GINST = 2 * 152 * 2.070


def recorded_fp64_ops(variant: str):
    """FP64-pipe thread-instructions (DADD + DFMA + DMUL) per cell of one sweep launch from a
    committed ncu summary taken on the current sweep source (a line 'FP64OPS variant=<v>
    per_cell=<n> source=<hash>')."""
    cur = sweep_source_hash()
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")) + glob.glob(os.path.join(ROOT, "profiles", "*.txt")):
        with open(path) as fh:
            for line in fh:
                m = re.search(r"FP64OPS variant=(\S+) per_cell=([0-9.eE+]+) source=([0-9a-f]+)", line)
                if m and m.group(1) == variant and m.group(3) == cur:
                    return float(m.group(2))
    return None


def fp64_pipe(variant: str, cells: int, sweep_ms: float):
    """The FP64 sweep against the FP64 pipe (it is bound there, not by HBM): recorded
    instructions per cell x cells / sweep time over the derived peak; None without a record."""
    per_cell = recorded_fp64_ops(variant)
    if per_cell is None or sweep_ms <= 0:
        return None
    achieved = per_cell * cells / (sweep_ms / 1e3) / 1e9
    return {"per_cell": per_cell, "achieved": round(achieved, 1), "peak": round(FP64_PIPE_PEAK_GINST, 1),
            "unit": "G FP64 thread-instructions/s", "frac": round(achieved / FP64_PIPE_PEAK_GINST, 4),
            "peak_source": "derived: 2 per clock per SM x 152 SMs x 2,070 MHz"}


def closure_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1909_13772_gb300", "csrc")
    for name in ("closure.cu", "closure.hpp", "cell.cuh", "cumulant.cuh", "kernels.cuh", "lattice.cuh", "select.cuh"):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_instructions(kernel: str):
    """Thread-instructions per cell of a kernel from a committed ncu summary, if it was taken on
    the current closure source (a line 'INSTR kernel=<k> per_cell=<n> source=<hash>')."""
    cur = closure_source_hash()
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        with open(path) as fh:
            for line in fh:
                m = re.search(r"INSTR kernel=(\S+) per_cell=([0-9.eE+]+) source=([0-9a-f]+)", line)
                if m and m.group(1) == kernel and m.group(3) == cur:
                    return float(m.group(2))
    return None


def recorded_traffic(variant: str):
    """DRAM bytes per sweep launch from a committed ncu summary, if it was taken on the
    current sweep source (a line 'TRAFFIC variant=<v> bytes_per_launch=<n> source=<hash>')."""
    cur = sweep_source_hash()
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")) + glob.glob(os.path.join(ROOT, "profiles", "*.txt")):
        with open(path) as fh:
            for line in fh:
                m = re.search(r"TRAFFIC variant=(\S+) bytes_per_launch=([0-9.eE+]+) source=([0-9a-f]+)", line)
                if m and m.group(1) == variant and m.group(3) == cur:
                    return float(m.group(2))
    return None


# ---------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------
def make_sim(lbm, storage, pattern, stream, tile=None, collision="TRT", shape=SHAPE):
    p = lbm.make_params(stencil=lbm.D3Q19, collision=getattr(lbm, collision), storage=getattr(lbm, storage),
                        pattern=getattr(lbm, pattern), omega=OMEGA, magic_lambda=LAMBDA, force=FORCE,
                        periodic=(1, 0, 1), mrt_rates=MRT_RATES if collision == "MRT" else None)
    sim = lbm.Simulation(p, [((0, 0, 0), shape)], stream=stream)
    if tile:
        sim.set_tile(*tile)
    # y faces default to no-slip: walls at y = -1/2 and y = 255.5
    return sim


def time_variant(lbm, variant, steps, warmup, world, tile=None, min_seconds=0.0, max_repeats=200):
    """W warm-up steps, then the timed region of exactly K steps (CUDA events on the library's
    stream, barrier and device synchronisation on both sides), repeated until min_seconds of
    timed work have run (at most max_repeats times; once when min_seconds is 0) so that the
    clock sampler sees the GPU under load; the reported time is the median repeat."""
    import torch
    storage, pattern, collision = VARIANTS[variant]
    stream = torch.cuda.Stream()
    sim = make_sim(lbm, storage, pattern, stream.cuda_stream, tile, collision)
    from paper_1909_13772_gb300 import inputs
    rho, u = inputs.rest(SHAPE)
    sim.init(0, rho, u)
    info = sim.info()
    sim.step(warmup)
    torch.cuda.synchronize()
    lbm.lbm_read_timing(sim.ctx, reset=True)
    lbm.lbm_enable_timing(sim.ctx, True)
    sampler = ClockSampler(torch.cuda.current_device())
    times, launches, spent = [], 0, 0.0
    while True:
        barrier(world)
        launches0 = sim.launches()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        start.record(stream)
        sim.step(steps)
        end.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        launches = sim.launches() - launches0
        times.append(start.elapsed_time(end))
        spent += times[-1] / 1e3
        if spent >= min_seconds or len(times) >= max_repeats:
            break
    clocks = sampler.stop()
    lbm.lbm_enable_timing(sim.ctx, False)
    kt = lbm.lbm_read_timing(sim.ctx, reset=True)
    ms = statistics.median(times)
    diag = sim.reduce()
    sim.close()
    del stream
    cells = info["cells"]
    bpp = info["bytes_per_pdf"]
    lups_per_s, tmax = aggregate(cells * steps, ms / 1e3, world)
    sweep_ms = kt["sweep"][0] / max(1, kt["sweep"][1])
    fill_ms = kt["fill"][0] / max(1, kt["fill"][1])
    alg_bytes = 2 * 19 * bpp * info["fluid_cells"]  # per sweep launch
    return {
        "mlups": lups_per_s / 1e6, "ms_per_step": tmax * 1e3 / steps, "sweep_ms": sweep_ms, "fill_ms": fill_ms,
        "sweep_share": kt["sweep"][0] / max(1e-9, kt["sweep"][0] + kt["fill"][0]),
        "sweep_gbs": alg_bytes / (sweep_ms / 1e3) / 1e9, "alg_bytes_per_sweep": alg_bytes, "launches": launches,
        "clocks": clocks, "info": info, "finite": diag["nonfinite"] == 0, "mass": diag["mass"],
        "repeats": len(times),
    }


def variant_error(lbm, variant, steps=ERROR_STEPS):
    """The variant's stated error against the oracle: the channel run from rest for `steps` steps
    on a 32 x 256 x 32 box (the flow is x- and z-invariant and every column does the same
    arithmetic, so its columns are bit for bit those of the 256^3 run) against the oracle's
    column after the same steps (tests/golden/channel_column_2000.txt, written by its committed
    generator from the oracle alone).  Normwise errors of the PDFs, of the deviations f_i - w_i
    and of the velocity u_x(y)."""
    import importlib.util
    import torch
    spec = importlib.util.spec_from_file_location(
        "make_channel_column", os.path.join(ROOT, "tests", "golden", "make_channel_column.py"))
    rec = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(rec)
    if steps != rec.STEPS or tuple(MRT_RATES[:2]) != (rec.MRT_BULK, rec.MRT_FOURTH):
        return None
    storage, pattern, collision = VARIANTS[variant]
    want = rec.read()[collision.lower()]  # [q, y]
    stream = torch.cuda.Stream()
    sim = make_sim(lbm, storage, pattern, stream.cuda_stream, None, collision, ERROR_SHAPE)
    try:
        from paper_1909_13772_gb300 import inputs
        rho, u = inputs.rest(ERROR_SHAPE)
        sim.init(0, rho, u)
        sim.step(steps)
        got = sim.pdfs_region(0, (ERROR_SHAPE[0] // 2, 0, ERROR_SHAPE[2] // 2), (1, ERROR_SHAPE[1], 1))[:, 0, :, 0]
    finally:
        sim.close()
    c, w, _ = lbm.lbm_stencil_table(19)
    cx = c[:, 0].astype(np.float64)
    ug, uw = cx @ got / got.sum(0), cx @ want / want.sum(0)
    dev = want - w[:, None]
    return {"steps": steps, "pdf": float(np.abs(got - want).max() / np.abs(want).max()),
            "deviation": float(np.abs(got - want).max() / np.abs(dev).max()),
            "u": float(np.abs(ug - uw).max() / np.abs(uw).max()),
            "against": "oracle column after %d steps (tests/golden/channel_column_2000.txt)" % steps}


def time_diag_sweep(lbm, variant, calls=40):
    """The sweep that ends every lbm_step call (and every step of the e2e leg) computes the step
    diagnostics; its mean time over `calls` one-step calls against the plain sweep's mean over
    one call of `calls` steps, both from the library's event tracing."""
    import torch
    from paper_1909_13772_gb300 import inputs
    storage, pattern, collision = VARIANTS[variant]
    stream = torch.cuda.Stream()
    sim = make_sim(lbm, storage, pattern, stream.cuda_stream, None, collision)
    try:
        rho, u = inputs.rest(SHAPE)
        sim.init(0, rho, u)
        sim.step(4)
        torch.cuda.synchronize()
        lbm.lbm_enable_timing(sim.ctx, True)
        for _ in range(calls):
            lbm.lbm_step(sim.ctx, 1)
        torch.cuda.synchronize()
        d = lbm.lbm_read_timing(sim.ctx)
        lbm.lbm_step(sim.ctx, calls)  # calls - 1 plain sweeps and one with diagnostics
        torch.cuda.synchronize()
        p = lbm.lbm_read_timing(sim.ctx)
    finally:
        sim.close()
    diag = d["sweep"][0] / d["sweep"][1]
    plain = (p["sweep"][0] - diag) / (p["sweep"][1] - 1)
    return {"diag_ms": round(diag, 4), "plain_ms": round(plain, 4), "ratio": round(diag / plain, 3), "calls": calls}


def time_e2e(lbm, variant, steps, world):
    """Same metric through the C ABI with host buffers: host->device upload of the initial
    macroscopic fields, K x (lbm_step + read-back of the step's diagnostics -- mass, momentum,
    energy, max speed), device->host download of the final fields, all inside the timed
    region.  Every step's record is read on the host; it is posted after its step and taken
    after the next step has been issued, so the GPU does not wait for the host's read.  The
    host buffers are page-locked, so the library's kernels read and write them directly.  The
    timed region (upload, steps, download) runs 3 times (5 for short runs); the median run is
    reported."""
    import torch
    from paper_1909_13772_gb300 import inputs
    storage, pattern, collision = VARIANTS[variant]
    stream = torch.cuda.Stream()
    sim = make_sim(lbm, storage, pattern, stream.cuda_stream, None, collision)
    rho, u = inputs.rest(SHAPE)
    # pinned host buffers, kept alive (the NumPy views below do not own them)
    pinned = [torch.from_numpy(rho).pin_memory(), torch.from_numpy(u).pin_memory(),
              torch.empty(rho.shape, dtype=torch.float64).pin_memory(),
              torch.empty(u.shape, dtype=torch.float64).pin_memory()]
    rho_h, u_h, rho_o, u_o = (t.numpy() for t in pinned)
    sim.init(0, rho_h, u_h)  # allocates and builds lists outside the timed region
    sim.step(2)
    lbm.lbm_get_macroscopic(sim.ctx, 0, rho_o, u_o)  # first use of the output buffers, untimed
    torch.cuda.synchronize()
    runs = []
    for _ in range(3 if steps >= 1000 else 5):  # the median run is reported
        barrier(world)
        t0 = time.perf_counter()
        lbm.lbm_init_macroscopic(sim.ctx, 0, rho_h, u_h)
        t1 = time.perf_counter()
        pending = None
        for _ in range(steps):
            lbm.lbm_step(sim.ctx, 1)
            ticket = lbm.lbm_step_diagnostics_post(sim.ctx)
            if pending is not None:
                lbm.lbm_step_diagnostics_take(sim.ctx, pending)
            pending = ticket
        if pending is not None:
            lbm.lbm_step_diagnostics_take(sim.ctx, pending)
        t2 = time.perf_counter()
        lbm.lbm_get_macroscopic(sim.ctx, 0, rho_o, u_o)
        t3 = time.perf_counter()
        runs.append((t3 - t0, t1 - t0, t2 - t1, t3 - t2))
    barrier(world)
    runs.sort()
    dt, up, mid, down = runs[len(runs) // 2]
    parts = {"upload_and_init_ms": round(up * 1e3, 3), "steps_ms": round(mid * 1e3, 3),
             "download_ms": round(down * 1e3, 3), "runs": len(runs),
             "run_ms": [round(r[0] * 1e3, 3) for r in runs]}
    cells = sim.info()["cells"]
    sim.close()
    del pinned
    lups, _ = aggregate(cells * steps, dt, world)
    n = rho.size
    return {"value": lups / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": int(4 * n * 8 / steps),
            "d2h_bytes_per_step": int((4 * n * 8) / steps + 64), "steps": steps, "breakdown": parts,
            "per_call": ("fields up once, %d x (lbm_step(1) + step diagnostics read back, each record taken "
                         "after the next step was issued), fields down once") % steps}


def cpu_baseline(min_seconds=10.0, max_steps=200, single_seconds=5.0):
    """The oracle as it stands, on the host cores, on a 256 x 256 x 8 slab of the channel; and on
    one core (the same slab, fewer steps)."""
    import oracle
    from paper_1909_13772_gb300 import inputs
    shape = (SHAPE[0], SHAPE[1], 8)
    p = oracle.OracleParams(shape=shape, q=19, collision=oracle.TRT, omega=OMEGA, magic_lambda=LAMBDA, force=FORCE,
                            periodic=(1, 0, 1), face_kind=(1, 1, 1, 1, 1, 1))
    rho, u = inputs.rest(shape)
    cells = shape[0] * shape[1] * shape[2]

    def rate(limit, cap):
        f = oracle.run(p, oracle.init(p, rho, u), 1)
        steps, t = 0, 0.0
        while steps == 0 or (t < limit and steps < cap):
            t0 = time.perf_counter()
            f = oracle.run(p, f, 1)
            t += time.perf_counter() - t0
            steps += 1
        return steps, t

    cores = oracle.get_threads()
    steps, t = rate(min_seconds, max_steps)
    oracle.set_threads(1)
    try:
        s1, t1 = rate(single_seconds, max_steps)
    finally:
        oracle.set_threads(cores)
    return {"value": cells * steps / t / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": "%d oracle steps of a 256x256x8 slab of the channel (FP64, D3Q19 TRT, walls in y)" % steps,
            "single_thread": {"value": cells * s1 / t1 / 1e6, "unit": "MLUPS", "cores": 1,
                              "sample": "%d oracle steps of the same slab on one core" % s1}}


def _oracle_rate(p, rho, u, flags=None, min_seconds=10.0, max_steps=2000):
    """Steps of the oracle as it stands from (rho, u), one at a time after one untimed step,
    until min_seconds have passed or max_steps were run (at least one): (steps, seconds)."""
    import oracle
    kw = {} if flags is None else {"flags": flags}
    f = oracle.run(p, oracle.init(p, rho, u, **kw), 1, **kw)
    steps, t = 0, 0.0
    while steps == 0 or (t < min_seconds and steps < max_steps):
        t0 = time.perf_counter()
        f = oracle.run(p, f, 1, **kw)
        t += time.perf_counter() - t0
        steps += 1
    return steps, t


def cpu_baseline_turbulence(min_seconds=10.0, n=64):
    """The oracle on the n^3 member of the decaying-turbulence family (D3Q27 TRT tau = 0.52,
    FP64; the size at which the oracle checks the family's FP64 reference run)."""
    import oracle
    from paper_1909_13772_gb300 import inputs
    rho, u = inputs.turbulence(n, seed=1909, kmax=min(32, n // 2), umax=0.05)
    p = oracle.OracleParams(shape=(n, n, n), q=27, collision=oracle.TRT, omega=1 / 0.52, magic_lambda=LAMBDA,
                            periodic=(1, 1, 1))
    steps, t = _oracle_rate(p, rho, u, min_seconds=min_seconds)
    return {"value": round(n ** 3 * steps / t / 1e6, 3), "unit": "MLUPS", "cores": oracle.get_threads(),
            "kind": "oracle", "sample": "%d oracle steps of the %d^3 member of the family (FP64, D3Q27 TRT)" % (steps, n)}


def cpu_baseline_porous(min_seconds=10.0, nb=4):
    """The oracle on the mini-bed: the porous-bed generator at nb^3 blocks (same seeds, spheres,
    inlet/outlet, D3Q19 TRT tau = 0.8), as one flagged domain, FP64."""
    import oracle
    from paper_1909_13772_gb300 import inputs
    _, shape, _ = inputs.rectilinear_blocks(nb=(nb, nb, nb), lo=16, hi=64, seed=4096)
    flags = inputs.sphere_packing(shape, radius=8.0, porosity=0.40, seed=7)
    p = oracle.OracleParams(shape=shape, q=19, collision=oracle.TRT, omega=1 / 0.8, magic_lambda=LAMBDA,
                            periodic=(0, 1, 1), face_kind=(oracle.VELOCITY, oracle.PRESSURE, 1, 1, 1, 1),
                            face_u=((0.02, 0.0, 0.0),) + ((0.0, 0.0, 0.0),) * 5, face_rho=(1.0,) * 6)
    rho, u = inputs.rest(shape)
    steps, t = _oracle_rate(p, rho, u, flags=flags, min_seconds=min_seconds)
    fluid = int((flags == 0).sum())
    return {"value": round(fluid * steps / t / 1e6, 3), "unit": "MFLUPS", "cores": oracle.get_threads(),
            "kind": "oracle", "sample": "%d oracle steps of the %d^3-block mini-bed (%d x %d x %d cells, %d fluid; FP64)"
                                        % (steps, nb, shape[0], shape[1], shape[2], fluid)}


def run_ours(args):
    import torch
    rank, world, local = dist_setup()
    from paper_1909_13772_gb300 import lbm
    lbm.load_library()
    head = args.variant
    res = time_variant(lbm, head, args.steps, args.warmup, world, min_seconds=args.min_seconds)
    variants = {}
    if not args.headline_only:
        for v in VARIANTS:
            if v == head:
                variants[v] = res
            else:
                k = max(10, min(args.steps, 200 if v.startswith("fp64") else args.steps))
                variants[v] = time_variant(lbm, v, k, args.warmup, world)
            variants[v]["error"] = variant_error(lbm, v)
    diag_sweep = time_diag_sweep(lbm, head)
    e2e = time_e2e(lbm, head, args.steps, world)
    cpu = cpu_baseline() if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None
    peak, peak_kind = measured_peaks()
    traffic = recorded_traffic(head)
    roof = {"bound": "hbm", "achieved": round(res["sweep_gbs"], 1), "peak": peak, "unit": "GB/s",
            "frac": round(res["sweep_gbs"] / peak, 4), "traffic": traffic,
            "kernel": "k_sweep (fused stream-collide, %s)" % head,
            "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind if peak_kind == "measured" else "fallback",
            "alg_bytes_per_launch": res["alg_bytes_per_sweep"], "sweep_ms": round(res["sweep_ms"], 4),
            "sweep_share_of_step": round(res["sweep_share"], 4)}
    fp64 = fp64_pipe(head, res["info"]["cells"], res["sweep_ms"]) if head.startswith("fp64") else None
    if fp64 is not None:
        # bound by the FP64 pipe: that is the roofline; the HBM figures stay beside it
        roof = {"bound": "alu", "achieved": fp64["achieved"], "peak": fp64["peak"], "unit": fp64["unit"],
                "frac": fp64["frac"], "traffic": traffic, "kernel": roof["kernel"],
                "peak_source": fp64["peak_source"], "fp64_per_cell": fp64["per_cell"],
                "hbm": {"achieved": roof["achieved"], "peak": peak, "unit": "GB/s", "frac": roof["frac"]},
                "alg_bytes_per_launch": roof["alg_bytes_per_launch"], "sweep_ms": roof["sweep_ms"],
                "sweep_share_of_step": roof["sweep_share_of_step"]}
    out = {
        "metric": METRIC, "value": round(res["mlups"], 1), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(res["ms_per_step"], 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "fp16dev": "f16 (deviation storage, f32 arithmetic)",
                  "bf16dev": "bf16 (deviation storage, f32 arithmetic)"}[head.split("-")[0]],
        "data": "synthetic (rest state, body-force driven; no dataset)",
        "config": {"workload": WORKLOAD, "variant": head, "shape": list(SHAPE), "stencil": "D3Q19",
                   "collision": "TRT", "magic_lambda": LAMBDA, "omega": OMEGA,
                   "cells_per_gpu": res["info"]["cells"], "parallelism": "replicas" if world > 1 else "single",
                   "l2": "no flush: state of %.1f GB per array >> 129 MB L2" % (
                       res["info"]["cells"] * 19 * res["info"]["bytes_per_pdf"] / 1e9)},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "diagnostics_sweep": diag_sweep,
        "gpu_launches": res["launches"],
        "clocks": res["clocks"],
        "timing": {"repeats": res["repeats"], "value_from": "median of the repeats of the K-step timed region "
                                                            "(each bracketed by barrier + synchronize)"},
        "stated_error": variants.get(head, {}).get("error"),
        "variants": {k: dict({"mlups": round(v["mlups"], 1), "sweep_gbs": round(v["sweep_gbs"], 1),
                              "frac_hbm": round(v["sweep_gbs"] / peak, 4), "ms_per_step": round(v["ms_per_step"], 4),
                              "sweep_ms": round(v["sweep_ms"], 4), "fill_ms": round(v["fill_ms"], 4),
                              "collision": VARIANTS[k][2], "error_vs_oracle": v.get("error")},
                             **({"fp64_pipe": fp64_pipe(k, v["info"]["cells"], v["sweep_ms"])}
                                if k.startswith("fp64") else {}))
                     for k, v in variants.items()},
    }
    if world == 1 and not args.no_workloads:
        out["workloads"] = measure_workloads(args)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def measure_porous(args):
    """Block-structured porous bed: 16^3 = 4096 blocks with edges log-uniform in [16, 64]
    (default_rng(4096)), Boolean sphere packing R = 8, porosity 0.40 (default_rng(7)),
    velocity inlet u = (0.02, 0, 0) at x-, pressure outlet rho = 1 at x+, periodic y/z,
    D3Q19 TRT FP32, tau = 0.8.  Metric: MFLUPS (updates of fluid cells per second)."""
    import torch
    rank, world, local = dist_setup()
    from paper_1909_13772_gb300 import inputs, lbm
    lbm.load_library()
    t0 = time.perf_counter()
    nbk = args.porous_blocks
    blocks, shape, _ = inputs.rectilinear_blocks(nb=(nbk, nbk, nbk), lo=16, hi=64, seed=4096)
    flags = inputs.sphere_packing(shape, radius=8.0, porosity=0.40, seed=7)
    t_geom = time.perf_counter() - t0
    storage, pattern = VARIANTS[args.variant][:2]
    p = lbm.make_params(stencil=lbm.D3Q19, collision=lbm.TRT, storage=getattr(lbm, storage),
                        pattern=getattr(lbm, pattern), omega=1 / 0.8, magic_lambda=LAMBDA, periodic=(0, 1, 1))
    stream = torch.cuda.Stream()
    sim = lbm.Simulation(p, blocks, stream=stream.cuda_stream)
    sim.set_face(0, 0, lbm.VELOCITY, (0.02, 0.0, 0.0), 1.0)
    sim.set_face(0, 1, lbm.PRESSURE, (0.0, 0.0, 0.0), 1.0)
    t0 = time.perf_counter()
    for b, (o, sz) in enumerate(sim.blocks):
        sub = flags[o[2]:o[2] + sz[2], o[1]:o[1] + sz[1], o[0]:o[0] + sz[0]]
        sim.set_boundary(b, sub if sub.any() else None)
    info = sim.info()
    t_plan = time.perf_counter() - t0
    t0 = time.perf_counter()
    for b, (o, sz) in enumerate(sim.blocks):
        rho, u = inputs.rest(sz)
        sim.init(b, rho, u)
    t_init = time.perf_counter() - t0
    if args.per_block:
        lbm.lbm_set_batching(sim.ctx, False)
    if args.ghost:
        lbm.lbm_set_in_place(sim.ctx, False)
    sparse = bool(getattr(args, "sparse", False))
    if sparse:
        lbm.lbm_set_sparse(sim.ctx, True)
    tuned = None
    if args.autotune and not sparse:
        tuned = lbm.lbm_autotune(sim.ctx, 10)
    sim.step(args.warmup)
    torch.cuda.synchronize()
    barrier(world)
    # per-kernel times from the library's tracing (plain launches)
    lbm.lbm_read_timing(sim.ctx, reset=True)
    lbm.lbm_enable_timing(sim.ctx, True)
    sim.step(min(args.steps, 50))
    lbm.lbm_enable_timing(sim.ctx, False)
    kt = lbm.lbm_read_timing(sim.ctx, reset=True)
    if args.graph:
        lbm.lbm_set_graph(sim.ctx, True)
        sim.step(3)  # capture
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    sim.step(args.steps)
    end.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = start.elapsed_time(end)
    diag = sim.step_diagnostics()
    sim.close()
    fluid = info["fluid_cells"]
    flups, tmax = aggregate(fluid * args.steps, ms / 1e3, world)
    sweep_ms = kt["sweep"][0] / max(1, kt["sweep"][1])
    fill_ms = kt["fill"][0] / max(1, kt["fill"][1])
    bpp = info["bytes_per_pdf"]
    alg = 2 * 19 * bpp * fluid
    table = 4 * 18 * fluid if sparse else 0  # the list layout's pull table, read once per step
    peak, peak_kind = measured_peaks()
    out = {"metric": "MFLUPS (fluid-cell lattice updates per second), porous bed", "value": round(flups / 1e6, 1),
           "unit": "MFLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(tmax * 1e3 / args.steps, 4), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": args.variant, "data": "synthetic (seeded sphere packing)",
           "config": {"workload": "porous bed, %d uneven blocks (%d^3, edges log-uniform 16..64), spheres R=8, "
                                  "porosity 0.40, velocity inlet 0.02 / pressure outlet, D3Q19 TRT tau=0.8"
                                  % (nbk ** 3, nbk),
                      "domain": list(shape), "cells": info["cells"], "fluid_cells": fluid, "tiles": info["tiles"],
                      "links": list(info["links"]), "ghost_slots": info["ghost_slots"],
                      "ghost_runs": info["ghost_runs"], "setup_s": {"geometry": round(t_geom, 1),
                                                                    "lists": round(t_plan, 1),
                                                                    "init": round(t_init, 1)}},
           "roofline": {"bound": "hbm", "achieved": round(alg / (sweep_ms / 1e3) / 1e9, 1), "peak": peak,
                        "unit": "GB/s", "frac": round(alg / (sweep_ms / 1e3) / 1e9 / peak, 4), "traffic": None,
                        "kernel": "k_sweep (fluid cells only)", "sweep_ms": round(sweep_ms, 4),
                        "fill_ms": round(fill_ms, 4), "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind,
                        "bytes": "fluid PDF bytes 2 Q s per fluid cell" + (" (plus the list table, 4 (Q - 1) B per fluid "
                                                                           "cell: frac_with_table)" if sparse else ""),
                        "frac_with_table": round((alg + table) / (sweep_ms / 1e3) / 1e9 / peak, 4) if sparse else None},
           # the time a step spends outside its kernels: launch gaps (graph replay when --graph)
           "launch_gap_ms_per_step": round(tmax * 1e3 / args.steps - sweep_ms - fill_ms, 4),
           "cpu_baseline": (cpu_baseline_porous(min_seconds=getattr(args, "cpu_seconds", 10.0))
                            if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None),
           "clocks": clocks, "finite": diag["nonfinite"] == 0, "max_speed": diag["max_speed"],
           "graph": bool(args.graph), "autotuned_tile": list(tuned[0]) if tuned else None,
           "autotuned_in_place": tuned[2] if tuned else None,
           "launch": "one sweep launch per block" if args.per_block else "one batched sweep launch",
           "layout": "fluid-cell list (lbm_set_sparse)" if sparse else "dense blocks",
           "neighbours": ("in place where faces match" if (tuned[2] if tuned else not args.ghost)
                          else "ghost-layer copies")}
    return out


def measure_tgv(args):
    """C1, the correctness configuration: 2-D Taylor-Green vortex extruded in z on a 32^3 fully
    periodic box, D3Q19 SRT tau = 0.6, FP64, u0 = 0.01.  The state (two 4.7 MB arrays) lives in
    L2, so the step rate is reported without a roofline fraction.  With the tile picked by
    lbm_autotune, times K steps for both patterns, launched plainly and as CUDA-graph replays of
    step pairs; fits the vortex's decay
    rate over the timed steps (after a 20-step start-up transient) against 2 nu k^2; times the
    oracle on the full configuration (100 steps) on the host cores."""
    import math
    import torch
    rank, world, local = dist_setup()
    from paper_1909_13772_gb300 import inputs, lbm
    lbm.load_library()
    n, tau, u0 = 32, 0.6, 0.01
    shape = (n, n, n)
    cells = n ** 3
    rho, u = inputs.taylor_green(n, u0=u0)
    k = 2.0 * math.pi / n
    nu = (tau - 0.5) / 3.0
    X, Y = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    mode = np.cos(k * X) * np.sin(k * Y)

    def amplitude(v):
        return float((v[0] * mode[None]).sum() / (mode * mode).sum() / n)

    runs = {}
    for pattern in ("TWO_GRID", "AA"):
        for graph in (False, True):
            p = lbm.make_params(stencil=lbm.D3Q19, collision=lbm.SRT, storage=lbm.FP64,
                                pattern=getattr(lbm, pattern), omega=1.0 / tau, periodic=(1, 1, 1))
            stream = torch.cuda.Stream()
            sim = lbm.Simulation(p, [((0, 0, 0), shape)], stream=stream.cuda_stream)
            sim.init(0, rho, u)
            tuned = lbm.lbm_autotune(sim.ctx, 10)  # restores the state; picks tile and neighbour mode
            if graph:
                lbm.lbm_set_graph(sim.ctx, True)
            sim.step(max(20, args.warmup))
            torch.cuda.synchronize()
            a0 = amplitude(sim.macroscopic(0)[1])
            barrier(world)
            launches0 = sim.launches()
            # the K-step timed region, repeated until the clock sampler has seen the GPU under
            # load for a while (its 15-us steps are far shorter than one 200-ms sample); the
            # time is the median repeat, the decay rate that of the first
            sampler = ClockSampler(torch.cuda.current_device())
            times, spent, a1, launches = [], 0.0, None, 0
            while True:
                start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                start.record(stream)
                sim.step(args.steps)
                end.record(stream)
                torch.cuda.synchronize()
                times.append(start.elapsed_time(end))
                spent += times[-1] / 1e3
                if a1 is None:
                    launches = sim.launches() - launches0
                    a1 = amplitude(sim.macroscopic(0)[1])
                if spent >= getattr(args, "tgv_min_seconds", 0.8) or len(times) >= 5000:
                    break
            clocks = sampler.stop()
            ms = statistics.median(times)
            sim.close()
            lups, tmax = aggregate(cells * args.steps, ms / 1e3, world)
            runs["%s%s" % (pattern.lower().replace("_", ""), "-graph" if graph else "")] = {
                "mlups": round(lups / 1e6, 1), "ms_per_step": round(tmax * 1e3 / args.steps, 5),
                "decay_rate_vs_2nuk2": round(-math.log(a1 / a0) / args.steps / (2 * nu * k * k), 5),
                "launches": launches, "autotuned_tile": list(tuned[0]), "autotuned_in_place": tuned[2],
                "clocks": clocks, "repeats": len(times)}
    best = max(runs, key=lambda r: runs[r]["mlups"])
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        op = oracle.OracleParams(shape=shape, q=19, collision=oracle.SRT, omega=1.0 / tau)
        f = oracle.init(op, rho, u)
        t0 = time.perf_counter()
        oracle.run(op, f, 100)
        t = time.perf_counter() - t0
        cpu = {"value": round(cells * 100 / t / 1e6, 3), "unit": "MLUPS", "cores": oracle.get_threads(),
               "kind": "oracle", "sample": "the full configuration: 100 oracle steps of the 32^3 vortex (FP64)"}
    out = {"metric": "MLUPS of the Taylor-Green correctness configuration (L2-resident: no roofline fraction)",
           "value": runs[best]["mlups"], "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": max(20, args.warmup), "ms_per_step": runs[best]["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (analytic vortex)",
           "config": {"workload": "2-D Taylor-Green vortex extruded in z, 32^3 periodic, D3Q19 SRT tau=0.6, "
                                  "u0=0.01, FP64", "value_from": best},
           "roofline": None,
           "roofline_note": "L2-resident (two 4.7 MB arrays in the 129 MB L2): no HBM roofline; the FP64 "
                            "sweep's own bound, the FP64 pipe, is reported on the channel's fp64 variants",
           "cpu_baseline": cpu, "gpu_launches": runs[best]["launches"],
           "clocks": runs[best]["clocks"], "variants": runs}
    return out


def _spectrum(u):
    """Shell-averaged kinetic-energy spectrum E(k), k = 1..n/2, of a periodic u[3, z, y, x]."""
    n = u.shape[-1]
    uh = np.stack([np.fft.rfftn(u[a]) for a in range(3)]) / n ** 3
    e = 0.5 * (np.abs(uh) ** 2).sum(axis=0)
    e[..., 1:] *= 2.0  # half spectrum along x: count the conjugate modes
    kf = np.fft.fftfreq(n, d=1.0 / n)
    kr = np.fft.rfftfreq(n, d=1.0 / n)
    KZ, KY, KX = np.meshgrid(kf, kf, kr, indexing="ij")
    shell = np.rint(np.sqrt(KX * KX + KY * KY + KZ * KZ)).astype(int)
    return np.bincount(shell.ravel(), weights=e.ravel(), minlength=n)[1:n // 2 + 1]


def measure_turbulence(args):
    """Decaying turbulence, D3Q27 TRT (Lambda = 3/16), tau = 0.52, periodic box, random-phase
    solenoidal k^(-5/3) start (default_rng(1909), shells 1..32, max|u| = 0.05), rho = 1.
    Throughput: 512^3 for each storage variant, and for the cumulant collision (Sec. 5.1.1,
    shear rate 1/tau, every other rate 1) in FP32.  Error: the same run at the error-study size
    for the configured steps in every variant, compared field by field with the GPU FP64 run of
    the same collision."""
    import torch
    rank, world, local = dist_setup()
    from paper_1909_13772_gb300 import inputs, lbm
    lbm.load_library()
    variants = [("FP64", "f64"), ("FP32", "f32"), ("FP16_DEV", "f16-dev"), ("BF16_DEV", "bf16-dev"),
                ("FP64", "f64-cumulant"), ("FP32", "f32-cumulant")]
    chosen = getattr(args, "turb_variants", None)
    if chosen:
        keep = set(chosen.split(","))
        perf_variants = [v for v in variants if v[1] in keep]
        # the error study always carries the FP64 reference of each chosen collision
        keep |= {"f64-cumulant" if k.endswith("cumulant") else "f64" for k in keep}
        variants = [v for v in variants if v[1] in keep]
    else:
        perf_variants = variants
    stream = torch.cuda.Stream()

    def make(n, storage, name=""):
        coll = lbm.CUMULANT if name.endswith("cumulant") else lbm.TRT
        p = lbm.make_params(stencil=lbm.D3Q27, collision=coll, storage=getattr(lbm, storage), pattern=lbm.AA,
                            omega=1 / 0.52, magic_lambda=LAMBDA, periodic=(1, 1, 1))
        return lbm.Simulation(p, [((0, 0, 0), (n, n, n))], stream=stream.cuda_stream)

    # throughput at 512^3
    n_perf = args.turb_size
    perf_steps = getattr(args, "turb_perf_steps", None) or min(args.steps, 200)
    tiled = bool(getattr(args, "turb_tile", False)) and n_perf % 2 == 0
    t0 = time.perf_counter()
    if tiled:
        # the (n/2)^3 member repeated 2 x 2 x 2 (periodic, so a valid start of the same family up
        # to the missing odd modes); the sweep's cost does not depend on the field
        rho, u = inputs.turbulence(n_perf // 2, seed=1909, kmax=min(32, n_perf // 4), umax=0.05)
        rho, u = np.tile(rho, (2, 2, 2)), np.tile(u, (1, 2, 2, 2))
    else:
        rho, u = inputs.turbulence(n_perf, seed=1909, kmax=32, umax=0.05)
    t_gen = time.perf_counter() - t0
    perf = {}
    peak, peak_kind = measured_peaks()
    sampler = ClockSampler(torch.cuda.current_device())
    for storage, name in perf_variants:
        if storage == "FP64" and not args.turb_fp64_perf:
            continue
        sim = make(n_perf, storage, name)
        sim.init(0, rho, u)
        sim.step(args.warmup)
        torch.cuda.synchronize()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        sim.step(perf_steps)
        end.record(stream)
        torch.cuda.synchronize()
        ms = start.elapsed_time(end) / perf_steps
        info = sim.info()
        sim.close()
        alg = 2 * 27 * info["bytes_per_pdf"] * info["cells"]
        perf[name] = {"mlups": round(info["cells"] / (ms / 1e3) / 1e6, 1), "ms_per_step": round(ms, 4),
                      "gbs": round(alg / (ms / 1e3) / 1e9, 1), "frac_hbm": round(alg / (ms / 1e3) / 1e9 / peak, 4)}
    clocks = sampler.stop()
    del rho, u
    # per-field error at the error-study size
    n = args.turb_err_size
    rho, u = inputs.turbulence(n, seed=1909, kmax=32, umax=0.05)
    fields = {}
    for storage, name in variants:
        sim = make(n, storage, name)
        sim.init(0, rho, u)
        d0 = sim.reduce()
        sim.step(args.steps)
        r, v = sim.macroscopic(0)
        d1 = sim.reduce()
        sim.close()
        fields[name] = (r, v, d0, d1)
    spectra = {k: _spectrum(fields[k][1]) for k in ("f64", "f64-cumulant") if k in fields}
    err = {}
    for name, (r, v, d0, d1) in fields.items():
        ref = "f64-cumulant" if name.endswith("cumulant") else "f64"
        r64, v64, d064, d164 = fields[ref]
        e64 = spectra[ref]
        e = _spectrum(v)
        err[name] = {
            "rho": float(np.abs(r - r64).max() / np.abs(r64 - 1.0).max()),
            "u": float(np.abs(v - v64).max() / np.abs(v64).max()),
            "kinetic_energy": float(d1["kinetic_energy"] / d164["kinetic_energy"] - 1.0),
            "spectrum_l2": float(np.sqrt(((e - e64) ** 2).sum() / (e64 ** 2).sum())),
            "mass_drift": float(d1["mass"] / d0["mass"] - 1.0),
            "momentum_drift": float(max(abs(a - b) for a, b in zip(d1["momentum"], d0["momentum"])) / d0["mass"]),
        }
    out = {"metric": "MLUPS per storage variant and per-field error vs the FP64 run, decaying turbulence",
           "value": perf.get("f32", {}).get("mlups"), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "higher_is_better": True, "data": "synthetic (seeded random-phase field)",
           "config": {"workload": "D3Q27 TRT tau=0.52 periodic decaying turbulence, k^-5/3 random-phase start, "
                                  "max|u| = 0.05, AA pattern (and the cumulant collision, shear 1/tau, other "
                                  "rates 1)", "throughput_size": n_perf,
                      "throughput_steps": perf_steps, "error_size": n, "error_steps": args.steps,
                      "generator_s": round(t_gen, 1),
                      "throughput_field": ("the %d^3 member repeated 2x2x2" % (n_perf // 2)) if tiled else
                      "the %d^3 member" % n_perf,
                      "error_reference": "the GPU FP64 run of the same start and collision (its kernels match "
                                         "the oracle to 1e-12: TRT on the 64^3 member over 2,000 steps, the "
                                         "cumulant collision on the 32^3 member over 300)"},
           "roofline": ({"bound": "hbm", "achieved": perf["f32"]["gbs"], "peak": peak, "unit": "GB/s",
                         "frac": perf["f32"]["frac_hbm"], "traffic": None,
                         "kernel": "k_sweep D3Q27 FP32 AA (one launch per step)",
                         "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind} if "f32" in perf else None),
           "roofline_cumulant": ({"bound": "hbm", "achieved": perf["f32-cumulant"]["gbs"], "peak": peak, "unit": "GB/s",
                                  "frac": perf["f32-cumulant"]["frac_hbm"], "traffic": None,
                                  "kernel": "k_sweep D3Q27 FP32 AA, cumulant collision (one launch per step)",
                                  "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind}
                                 if "f32-cumulant" in perf else None),
           "clocks": clocks, "throughput": perf, "error_vs_fp64": err,
           "cumulant_vs_trt_fp64": ({"u": float(np.abs(fields["f64-cumulant"][1] - fields["f64"][1]).max()
                                                / np.abs(fields["f64"][1]).max()),
                                     "spectrum_l2": float(np.sqrt(((spectra["f64-cumulant"] - spectra["f64"]) ** 2).sum()
                                                                  / (spectra["f64"] ** 2).sum()))}
                                    if len(spectra) == 2 else None),
           "cpu_baseline": (cpu_baseline_turbulence(min_seconds=getattr(args, "cpu_seconds", 10.0))
                            if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None)}
    return out


def measure_closure(args):
    """Locally varying relaxation (learned closure, C5 coarse grid): D3Q19 TRT tau0 = 0.502,
    FP32 storage, AA pattern, periodic N^3 box of decaying turbulence (random-phase k^(-5/3)
    start, default_rng(9), shells 1..N/4, max|u| = 0.1).  Each step once with the constant
    rate, once with Smagorinsky (C_s = 0.17) and once with the tensor-core network fused into
    the collision.  Value: MLUPS of the network step at 128^3; roofline of the network sweep
    there against instruction issue, its bound (instructions per cell from the committed ncu
    summary of the same source)."""
    import torch
    rank, world, local = dist_setup()
    from paper_1909_13772_gb300 import closure_study, inputs, lbm
    lbm.load_library()
    stream = torch.cuda.Stream()
    net = closure_study.init_params(0, 100.0, 300.0, 1e-3)
    sizes = [int(v) for v in args.closure_sizes.split(",")]
    kinds = [k for k in ("trt", "smagorinsky", "mlp") if k in args.closure_kinds.split(",")]
    res = {}
    for n in sizes:
        rho, u = inputs.turbulence(n, seed=9, kmax=n // 4, umax=0.1)
        for name in kinds:
            p = lbm.make_params(stencil=lbm.D3Q19, collision=lbm.TRT, storage=lbm.FP32, pattern=lbm.AA,
                                omega=1 / 0.502, magic_lambda=LAMBDA, periodic=(1, 1, 1))
            sim = lbm.Simulation(p, [((0, 0, 0), (n, n, n))], stream=stream.cuda_stream)
            if name == "smagorinsky":
                sim.set_closure(lbm.CLOSURE_SMAGORINSKY, cs=0.17)
            elif name == "mlp":
                sim.set_closure(lbm.CLOSURE_MLP, mlp_params=net)
            sim.init(0, rho, u)
            sim.step(args.warmup)
            torch.cuda.synchronize()
            barrier(world)
            lbm.lbm_read_timing(sim.ctx, reset=True)
            lbm.lbm_enable_timing(sim.ctx, True)
            sim.step(min(args.steps, 50))
            lbm.lbm_enable_timing(sim.ctx, False)
            kt = lbm.lbm_read_timing(sim.ctx, reset=True)
            torch.cuda.synchronize()
            # the K-step timed region, repeated until the clock sampler has seen the GPU under
            # load (the median repeat is the time); the state is re-initialised every 25 repeats,
            # before the constant-rate run at this tau can reach its divergence
            sampler = ClockSampler(torch.cuda.current_device())
            times, spent, finite = [], 0.0, True
            while True:
                if times and len(times) % 25 == 0:
                    sim.init(0, rho, u)
                start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                start.record(stream)
                sim.step(args.steps)
                end.record(stream)
                torch.cuda.synchronize()
                times.append(start.elapsed_time(end))
                spent += times[-1] / 1e3
                if len(times) % 25 == 0 or spent >= getattr(args, "closure_min_seconds", 0.8):
                    finite = finite and sim.step_diagnostics()["nonfinite"] == 0
                if spent >= getattr(args, "closure_min_seconds", 0.8) or len(times) >= 2000:
                    break
            clocks = sampler.stop()
            ms = statistics.median(times)
            sim.close()
            ups, tmax = aggregate(n ** 3 * args.steps, ms / 1e3, world)
            sweep_ms = kt["sweep"][0] / max(1, kt["sweep"][1])
            res["%s-%d" % (name, n)] = {"mlups": round(ups / 1e6, 1), "ms_per_step": round(tmax * 1e3 / args.steps, 4),
                                        "sweep_ms": round(sweep_ms, 4), "finite": finite,
                                        "clocks": clocks, "repeats": len(times)}
        del rho, u
    n = sizes[0]
    peak_hbm, peak_kind = measured_peaks()
    if "mlp" not in kinds:
        return {"metric": "closure step timings", "variants": res}
    sweep_ms = res["mlp-%d" % n]["sweep_ms"]
    clocks = res["mlp-%d" % n]["clocks"]
    sm_clock = (clocks or {}).get("sm_max_mhz") or 2070.0
    # the network sweep is bound by instruction issue: four schedulers per SM, one warp
    # instruction (32 thread-instructions) each per clock
    issue_peak = 4 * 32 * 152 * sm_clock * 1e6 / 1e12  # T thread-instructions/s
    per_cell = recorded_instructions("closure-mlp-aa-%d" % n)
    issue_ach = per_cell * n ** 3 / (sweep_ms / 1e3) / 1e12 if per_cell else None
    alg_bytes = 2 * 19 * 4 * n ** 3
    mma_flops = 2 * (16 * 32 + 32 * 32 + 32 * 8) * n ** 3  # padded MMA shapes per cell
    out = {"metric": "MLUPS of the learned-closure step (tensor-core network fused into the collision)",
           "value": res["mlp-%d" % n]["mlups"], "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": res["mlp-%d" % n]["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32 (network bf16 x bf16 -> f32)",
           "data": "synthetic (seeded random-phase turbulence)",
           "config": {"workload": "learned closure, D3Q19 TRT tau0=0.502 periodic %d^3 decaying turbulence, "
                                  "FP32 AA, 7-32-32-1 SiLU network" % n, "sizes": sizes,
                      "l2": "no flush: %d^3 FP32 state %d MB vs 129 MB L2" % (n, 19 * 4 * n ** 3 // 10 ** 6)},
           "roofline": {"bound": "alu", "achieved": round(issue_ach, 3) if issue_ach else None,
                        "peak": round(issue_peak, 3), "unit": "T thread-instructions/s (issue)",
                        "frac": round(issue_ach / issue_peak, 4) if issue_ach else None,
                        "traffic": None, "kernel": "k_closure_sweep<network>, AA pair at %d^3" % n,
                        "peak_source": "4 schedulers x 32 lanes per clock per SM x 152 SMs x max SM clock",
                        "instructions_per_cell": per_cell,
                        "sweep_ms": round(sweep_ms, 4),
                        "hbm_gbs": round(alg_bytes / (sweep_ms / 1e3) / 1e9, 1),
                        "hbm_frac": round(alg_bytes / (sweep_ms / 1e3) / 1e9 / peak_hbm, 4),
                        "tensor_tflops": round(mma_flops / (sweep_ms / 1e3) / 1e12, 2)},
           "cost_vs_constant_rate": {k: round(res["mlp-%d" % k]["ms_per_step"] / res["trt-%d" % k]["ms_per_step"], 3)
                                     for k in sizes if "trt" in kinds},
           "variants": res, "clocks": res["mlp-%d" % n]["clocks"],
           "cpu_baseline": (cpu_baseline_closure(net, min_seconds=getattr(args, "cpu_seconds", 10.0))
                            if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None)}
    return out


def cpu_baseline_closure(net, min_seconds=10.0, n=32):
    """The oracle with the network closure (FP64 network, BF16 weights) on an n^3 member of the
    closure workload's turbulence family."""
    import oracle
    from paper_1909_13772_gb300 import inputs
    rho, u = inputs.turbulence(n, seed=9, kmax=n // 4, umax=0.1)
    p = oracle.OracleParams(shape=(n, n, n), q=19, collision=oracle.TRT, omega=1 / 0.502, magic_lambda=LAMBDA,
                            periodic=(1, 1, 1))
    cl = dict(kind=oracle.MLP, mlp=net)
    f = oracle.run(p, oracle.init(p, rho, u), 1, closure=cl)
    steps, t = 0, 0.0
    while steps == 0 or (t < min_seconds and steps < 2000):
        t0 = time.perf_counter()
        f = oracle.run(p, f, 1, closure=cl)
        t += time.perf_counter() - t0
        steps += 1
    return {"value": round(n ** 3 * steps / t / 1e6, 3), "unit": "MLUPS", "cores": oracle.get_threads(),
            "kind": "oracle", "sample": "%d oracle steps with the network closure on the %d^3 member (FP64)"
                                        % (steps, n)}



def cpu_baseline_refine(min_seconds=5.0):
    """The oracle's refined run on a 48 x 8 x 8 coarse box with its last 16 columns refined."""
    import oracle
    from paper_1909_13772_gb300 import inputs
    shape, a = (48, 8, 8), 32
    p = oracle.OracleParams(shape=shape, q=19, collision=oracle.TRT, omega=1 / 0.6, magic_lambda=LAMBDA,
                            periodic=(1, 1, 1))
    pf = oracle.refine_fine_params(p, a, shape[0])
    rc, uc = inputs.random_state(shape, seed=61, rho_amp=0.01, u_amp=0.02)
    rf, uf = inputs.random_state(pf.shape, seed=62, rho_amp=0.01, u_amp=0.02)
    fc, ff = oracle.refine_init(p, a, shape[0], rc, uc, rf, uf)
    fc, ff = oracle.refine_run(p, a, shape[0], fc, ff, 1)
    steps, t = 0, 0.0
    while steps == 0 or t < min_seconds:
        t0 = time.perf_counter()
        fc, ff = oracle.refine_run(p, a, shape[0], fc, ff, 1)
        t += time.perf_counter() - t0
        steps += 1
    ups = a * 64 + 2 * int(np.prod(pf.shape))  # cell updates per coarse step
    return {"value": round(ups * steps / t / 1e6, 3), "unit": "MLUPS", "cores": oracle.get_threads(), "kind": "oracle",
            "sample": "%d coarse steps of a 48x8x8 coarse box with its last 16 columns refined 2:1 (FP64, D3Q19 TRT)"
                      % steps}


def measure_refine(args):
    """Static 2:1 refinement: a periodic 256 x 128 x 128 coarse box (D3Q19 TRT tau_c = 0.6, FP32,
    two-grid) whose last 64 columns are refined (fine block 128 x 256 x 256, two fine steps per
    coarse step), started from a seeded random state on both grids.  Value: cell updates per
    second (coarse updates + two per fine cell and coarse step), each coarse step a CUDA-graph
    replay; the sweeps' share from a separate traced pass."""
    import torch
    rank, world, local = dist_setup()
    from paper_1909_13772_gb300 import inputs, lbm, refine
    lbm.load_library()
    shape, a = (256, 128, 128), 192
    nx, ny, nz = shape
    stream = torch.cuda.Stream()
    params = lbm.make_params(stencil=19, collision=lbm.TRT, storage=lbm.FP32, omega=1 / 0.6, magic_lambda=LAMBDA)
    run = refine.RefinedRun(params, shape, a, stream=stream.cuda_stream)
    try:
        rc, uc = inputs.random_state((a, ny, nz), seed=61, rho_amp=0.01, u_amp=0.02)
        rf, uf = inputs.random_state((2 * (nx - a), 2 * ny, 2 * nz), seed=62, rho_amp=0.01, u_amp=0.02)
        run.init(rc, uc, rf, uf)
        run.step(args.warmup)
        torch.cuda.synchronize()
        d0 = run.reduce()
        launches0 = run.coarse.launches() + run.fine.launches()
        # the K-step timed region, repeated until the clock sampler has seen the GPU under load;
        # the time is the median repeat
        sampler = ClockSampler(torch.cuda.current_device())
        torch.cuda.synchronize()
        times, spent, launches = [], 0.0, None
        while True:
            start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            start.record(stream)
            run.step(args.steps)
            end.record(stream)
            torch.cuda.synchronize()
            times.append(start.elapsed_time(end))
            spent += times[-1] / 1e3
            if launches is None:
                launches = run.coarse.launches() + run.fine.launches() - launches0
            if spent >= 0.8 or len(times) >= 500:
                break
        clocks = sampler.stop()
        ms = statistics.median(times) / args.steps
        nrep = len(times)
        d1 = run.reduce()
        # the sweeps' own times from a traced pass (tracing runs the launches one by one, not
        # as the graph replay of the timed region)
        for s in (run.coarse, run.fine):
            lbm.lbm_read_timing(s.ctx, reset=True)
            lbm.lbm_enable_timing(s.ctx, True)
        run.step(args.steps)
        torch.cuda.synchronize()
        kt = [lbm.lbm_read_timing(s.ctx, reset=True) for s in (run.coarse, run.fine)]
        for s in (run.coarse, run.fine):
            lbm.lbm_enable_timing(s.ctx, False)
    finally:
        run.close()
    nc, nf = a * ny * nz, 2 * (nx - a) * 4 * ny * nz
    ups = nc + 2 * nf
    sweep_ms = (kt[0]["sweep"][0] + kt[1]["sweep"][0]) / args.steps
    alg = 2 * 19 * 4 * ups  # PDF bytes of the sweeps per coarse step
    peak, peak_kind = measured_peaks()
    gbs = alg / (sweep_ms / 1e3) / 1e9
    return {"metric": "MLUPS of the 2:1 refined step (coarse and fine cell updates per second)",
            "value": round(ups / (ms / 1e3) / 1e6, 1), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded random state on both grids)",
            "config": {"workload": "static 2:1 refinement, periodic 256x128x128 coarse box, last 64 columns "
                                   "refined (fine 128x256x256), D3Q19 TRT tau_c = 0.6, FP32 two-grid",
                       "coarse_cells": nc, "fine_cells": nf, "updates_per_coarse_step": ups},
            "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(gbs / peak, 4), "traffic": None,
                         "kernel": "k_sweep of both grids (3 launches per coarse step)",
                         "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind},
            "sweep_share_of_step": round(sweep_ms / ms, 4),
            "transfers_ms_per_step": round(ms - sweep_ms, 4),
            "launch": "CUDA-graph replay of each coarse step (3 transfers, 3 sweeps)",
            "mass_drift": d1["mass"] / d0["mass"] - 1.0,
            "mass_drift_steps": args.steps * nrep, "timing": {"repeats": nrep, "value_from": "median repeat"},
            "gpu_launches": launches, "clocks": clocks,
            "cpu_baseline": cpu_baseline_refine() if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None}


def _print_rank0(out):
    if int(os.environ.get("RANK", "0")) == 0:
        print(json.dumps(out), flush=True)


def run_porous(args):
    _print_rank0(measure_porous(args))


def run_tgv(args):
    _print_rank0(measure_tgv(args))


def run_turbulence(args):
    _print_rank0(measure_turbulence(args))


def run_closure(args):
    _print_rank0(measure_closure(args))


def run_refine(args):
    _print_rank0(measure_refine(args))


def measure_workloads(args):
    """The other configurations, each with its own metric, roofline, oracle figure and clocks,
    sized to keep the default run within a few minutes (one GPU): C1 the 32^3 Taylor-Green
    vortex (FP64, the full configuration); C3 D3Q27 decaying turbulence (throughput of the FP32
    and 16-bit storages at 512^3, per-field errors of every storage against the FP64 run at 128^3
    after 2,000 steps); C4 the 4096-block porous bed (autotuned tile and neighbour mode, CUDA-graph
    replay); C5 the learned closure on the 128^3 coarse grid (constant rate, Smagorinsky,
    network)."""
    import copy
    out = {}

    def sub(**kw):
        a = copy.copy(args)
        for k, v in kw.items():
            setattr(a, k, v)
        return a

    k = args.steps
    jobs = [
        ("c1_taylor_green", measure_tgv, sub(steps=max(100, k), cpu_seconds=5.0)),
        ("c3_turbulence", measure_turbulence, sub(steps=2000, turb_size=512, turb_err_size=128,
                                                  turb_perf_steps=min(max(k, 20), 100), turb_tile=True,
                                                  turb_fp64_perf=False, cpu_seconds=5.0)),
        ("c4_porous_bed", measure_porous, sub(steps=min(max(k, 20), 100), graph=True, autotune=False,
                                              per_block=False, ghost=False, porous_blocks=16, cpu_seconds=5.0,
                                              variant="fp32-twogrid", sparse=True)),
        ("c4_porous_bed_dense", measure_porous, sub(steps=min(max(k, 20), 100), graph=True, autotune=True,
                                                    per_block=False, ghost=False, porous_blocks=16,
                                                    no_cpu_baseline=True, variant="fp32-twogrid", sparse=False)),
        ("c5_closure", measure_closure, sub(steps=min(max(k, 20), 100), closure_sizes="128",
                                            closure_kinds="trt,smagorinsky,mlp", cpu_seconds=5.0)),
        ("refinement", measure_refine, sub(steps=min(max(k, 20), 100))),
    ]
    for name, fn, a in jobs:
        t0 = time.perf_counter()
        try:
            out[name] = fn(a)
        except Exception as e:  # a failing workload is reported, the headline line still prints
            out[name] = {"error": "%s: %s" % (type(e).__name__, e)}
        out[name]["wall_s"] = round(time.perf_counter() - t0, 1)
        log("workload %s: %.1f s" % (name, out[name]["wall_s"]))
    return out

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    import oracle
    from paper_1909_13772_gb300 import inputs
    # slab depth: about a minute of oracle work at ~17 MLUPS for the requested steps
    depth = int(max(1, min(8, round(60.0 * 17e6 / (max(1, args.steps) * SHAPE[0] * SHAPE[1])))))
    shape = (SHAPE[0], SHAPE[1], depth)
    p = oracle.OracleParams(shape=shape, q=19, collision=oracle.TRT, omega=OMEGA, magic_lambda=LAMBDA, force=FORCE,
                            periodic=(1, 0, 1), face_kind=(1, 1, 1, 1, 1, 1))
    rho, u = inputs.rest(shape)
    f = oracle.init(p, rho, u)
    f = oracle.run(p, f, args.warmup)
    t0 = time.perf_counter()
    f = oracle.run(p, f, args.steps)
    dt = time.perf_counter() - t0
    cells = shape[0] * shape[1] * shape[2]
    v = cells * args.steps / dt / 1e6
    sample = ("each step: one oracle time step of a 256x256x%d slab of the channel (FP64, D3Q19 TRT); "
              "slab depth sized so that the whole run stays near a minute" % shape[2])
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "MLUPS", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (rest state, body-force driven; no dataset)",
           "config": {"workload": WORKLOAD, "variant": args.variant, "shape": list(SHAPE), "sample_shape": list(shape)},
           "cpu_baseline": {"value": round(v, 3), "unit": "MLUPS", "cores": oracle.get_threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(v, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--variant", choices=list(VARIANTS), default="fp32-twogrid")
    ap.add_argument("--headline-only", action="store_true", help="skip the other variants")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--graph", action="store_true", help="porous: replay step pairs as CUDA graphs")
    ap.add_argument("--autotune", action="store_true",
                    help="porous: pick the sweep tile and the neighbour mode with lbm_autotune")
    ap.add_argument("--per-block", action="store_true", help="porous: one sweep launch per block (comparison)")
    ap.add_argument("--ghost", action="store_true", help="porous: ghost-layer copies instead of in-place neighbours")
    ap.add_argument("--sparse", action="store_true", help="porous: the fluid-cell list layout of the two-grid sweep")
    ap.add_argument("--workload", choices=["channel", "porous", "turbulence", "closure", "tgv", "refine"],
                    default="channel",
                    help="channel: the 256^3 benchmark (default); porous: the 4096-block porous bed; "
                         "tgv: the 32^3 Taylor-Green correctness configuration; "
                         "turbulence: D3Q27 decaying turbulence, storage variants and their errors; "
                         "closure: constant rate vs Smagorinsky vs the learned closure; "
                         "refine: the static 2:1 refined box")
    ap.add_argument("--porous-blocks", type=int, default=16, help="porous: blocks per axis (16: 4096 blocks)")
    ap.add_argument("--closure-sizes", default="128,256", help="closure: box sizes; the first is the value's")
    ap.add_argument("--closure-kinds", default="trt,smagorinsky,mlp", help="closure: which steps to time")
    ap.add_argument("--turb-size", type=int, default=512)
    ap.add_argument("--turb-err-size", type=int, default=256)
    ap.add_argument("--turb-fp64-perf", action="store_true")
    ap.add_argument("--turb-variants", default=None,
                    help="comma-separated subset of f64,f32,f16-dev,bf16-dev,f64-cumulant,f32-cumulant")
    ap.add_argument("--no-workloads", action="store_true",
                    help="channel: leave out the records of the other configurations (C1, C3, C4, C5)")
    ap.add_argument("--min-seconds", type=float, default=2.0,
                    help="channel: repeat the K-step timed region until this much timed work has run "
                         "(the clock sampler needs load); the value is the median repeat")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "porous":
        run_porous(args)
    elif args.workload == "turbulence":
        run_turbulence(args)
    elif args.workload == "closure":
        run_closure(args)
    elif args.workload == "tgv":
        run_tgv(args)
    elif args.workload == "refine":
        run_refine(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
