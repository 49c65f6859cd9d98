"""Benchmark of the ventilation-flow time step on GB300: Gcell-updates/s and fraction of the HBM roofline.

Workload (one step = every row of the hot path: RK4 stages, divergence, 4 iterations of the FFT Poisson solve,
projection, filter, FP64 reductions): the single room of 256 x 128 x 128 cells (10 x 5 x 5 m, 2-cell walls, a
5x5-cell inlet duct forced to 1 m/s and the opposite outlet), FP32 bulk with FP64 reductions every step.  The
state (about 0.3 GB) is larger than L2, so no flush is needed between steps.

Our arm prints one JSON line with the device-timed throughput, the end-to-end throughput through the C ABI with
host buffers (also with every step's record read before the next step), the roofline of the dominant kernel
(per-kernel CUDA-event times from vf_profile_steps), the FP64 form's throughput, one FFT Poisson solve against
cuFFT, the large-room, batch, serving and next-row legs, clocks sampled during the timed region and the oracle
timed on the host cores (one process per core, and one full-size step on one core).

``--impl reference`` times the FP64 CPU oracle as it stands on every host core (the only other place this script
runs it), on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcell-updates/s per step & % HBM roofline"
UNIT = "Gcell-updates/s"

# Algorithmic bytes per cell of each kernel phase in FP32 (F = 4 bytes per value, 1 byte of mask per pass that
# reads it): what each launch must read and write at least once.
F32 = 4
PHASE_BYTES_PER_CELL = {
    "stage1": 8 * F32 + 1,       # read q_n (4 values), write q2 (4), mask
    "stage2": 12 * F32 + 1,      # read q2 (stencil), q_n; write q3; mask
    "stage3": 12 * F32 + 1,      # read q3 (stencil), q_n; write q4; mask
    "stage4": 20 * F32 + 1,      # read q4 (stencil), q_n, q2, q3; write q*; mask
    "div": 4 * F32,              # read u*, v*, w*; write r
    "fft_x_fwd": 2 * F32,        # read f; write the half spectrum (N/2 complex = N F bytes)
    "fft_y_fwd": 2 * F32,        # read + write the spectrum
    "fft_z_solve": 2 * F32,
    "fft_y_inv": 2 * F32,
    "fft_x_inv": 2 * F32,        # read the spectrum, write p
    "fft_yz_solve": 2 * F32,     # read + write the spectrum once (y, z transforms and division in shared memory)
    "poisson_rhs": None,         # touches only the cells next to solids (about 1 in 9 here): not a roofline row
    "project": 7 * F32 + 1,      # read u*, v*, w*, p, mask; write u, v, w
    "filter": 8 * F32 + 1,       # read u, v, w, c, mask; write 4 fields
    "reduce": 4 * F32 + 1,       # read u, v, w, c, mask
    "adjust_dt": None,           # one thread: the dynamic time step's control block
    "particles": None,           # per particle, not per cell
}
# kernel function of each phase (phases of one function are one roofline row)
PHASE_KERNEL = {"stage1": "k_stage", "stage2": "k_stage", "stage3": "k_stage", "stage4": "k_stage",
                "div": "k_div", "fft_x_fwd": "k_fft_x_fwd", "fft_x_inv": "k_fft_x_inv", "fft_y_fwd": "k_fft_y",
                "fft_y_inv": "k_fft_y", "fft_z_solve": "k_fft_z_solve", "fft_yz_solve": "k_fft_yz_solve",
                "project": "k_project", "filter": "k_filter", "reduce": "k_reduce_state"}
# Byte model of one step with the kernels fused as far as the method allows (121F+9 per cell with n = 4 Poisson
# iterations: RK4 with an accumulator, divergence, four Poisson iterations, projection fused with the filter),
# used for the step-level roofline fraction.
STEP_MODEL_BYTES_PER_CELL_FP32 = 121 * F32 + 9


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu_index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("VF_BENCH_GLOO") is None else "gloo")
    return world, rank, local


def dist_max(value, world):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def code_text(text):
    """Source text without its comments, whitespace runs collapsed: what the compiler reads of it."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def source_digest(path, end_marker=None):
    """SHA-256 of the code of a source file (comments and layout aside), or of its text up to the first line that
    starts with ``end_marker`` (the part a kernel and the helpers above it are compiled from); None when the file or
    the marker is missing."""
    full = os.path.join(ROOT, path)
    if not os.path.exists(full):
        return None
    data = open(full, encoding="utf-8").read()
    if end_marker:
        cut = data.find("\n" + end_marker)
        if cut < 0:
            return None
        data = data[:cut + 1]
    return hashlib.sha256(code_text(data).encode()).hexdigest()


def traffic_record(kernel, tiles):
    """DRAM bytes per launch of ``kernel`` from the committed ncu summary, if taken on the current source of the
    kernel (and of everything above it in its file, and the shared headers) with the same launch tiles."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    entries = rec.get("kernels", {}).get(kernel)
    if not entries:
        return None
    if isinstance(entries, dict):
        entries = [entries]
    for entry in entries:   # one capture per launch tiling
        if any(tiles.get(key) != value for key, value in (entry.get("tiles") or {}).items()):
            continue
        digest = source_digest(entry["source"], entry.get("source_end_marker"))
        if digest is None or digest != entry.get("source_sha256"):
            return None
        for hdr, hdr_digest in (entry.get("headers") or {}).items():
            if source_digest(hdr) != hdr_digest:
                return None
        return entry["dram_bytes_per_launch"] * entry.get("scale_to_full", 1.0)
    return None


def fp64_flop_record():
    """FP64 floating-point operations per cell and step of the FP64 step (DADD + DMUL + 2 DFMA thread
    instructions counted by ncu over one step of the 256x128x128 room), if counted on the current sources."""
    path = os.path.join(ROOT, "profiles", "fp64_flops.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    for src, digest in rec.get("sources", {}).items():
        if source_digest(src) != digest:
            return None
    return rec.get("flops_per_cell_step")


def cpu_baseline_oracle(room, precision_note, steps=1):
    """The FP64 oracle timed on the host cores over ``steps`` full steps of the same room."""
    from oracle import flow as F
    from paper_2204_02107_gb300 import rooms
    prm = F.Params(nx=room.nx, ny=room.ny, nz=room.nz, lx=room.lx, ly=room.ly, lz=room.lz, nu=rooms.NU_AIR,
                   dt=room.dt, u_set=(room.u_in, 0.0, 0.0), c_set=0.0, filter=True, n_pressure_iters=4)
    geom = F.Geometry(room.beta, room.S, room.room)
    st = F.zero_state(prm, c=room.initial_c())
    t0 = time.perf_counter()
    for _ in range(steps):
        st, _ = F.step(st, geom, prm)
    dt = time.perf_counter() - t0
    single = {"value": room.cells * steps / dt / 1e9, "unit": UNIT, "cores": 1,
              "sample": f"{steps} full FP64 step(s) of the {room.nx}x{room.ny}x{room.nz} room ({precision_note}); "
                        f"numpy element-wise ops and numpy.fft run on one core"}
    # every host core: one copy of a 128x64x64 room of the same construction per core, 3 timed steps after 1
    procs = host_cores()
    try:
        value, _ = oracle_all_cores((128, 64, 64), 3, 1, procs)
    except Exception as e:   # keep the measured single-core figure rather than lose the line
        return {"value": single["value"], "unit": UNIT, "cores": 1, "kind": "oracle", "sample": single["sample"],
                "all_cores_error": repr(e)}
    return {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"{procs} independent copies (one process per host core, one thread each) of the room "
                      f"construction at 128x64x64 (1/8 of the cells), 3 full FP64 steps each ({precision_note}) "
                      f"after 1 warm-up step, timed from a common barrier to the slowest process",
            "single_core_full_size": single}


def oracle_room(nx, ny, nz):
    """The oracle's inputs for the single-room construction at nx x ny x nz (filter on, 4 pressure iterations)."""
    from oracle import flow as F
    from paper_2204_02107_gb300 import rooms
    room = rooms.single_room(nx, ny, nz)
    prm = F.Params(nx=room.nx, ny=room.ny, nz=room.nz, lx=room.lx, ly=room.ly, lz=room.lz, nu=rooms.NU_AIR,
                   dt=room.dt, u_set=(room.u_in, 0.0, 0.0), c_set=0.0, filter=True, n_pressure_iters=4)
    return room, prm, F.Geometry(room.beta, room.S, room.room), F.zero_state(prm, c=room.initial_c())


def oracle_worker(shape, steps, warmup, barrier, queue):
    """One host process: warm-up oracle steps, a barrier shared by every process, then ``steps`` timed steps; puts
    the elapsed seconds of the timed steps (or the error) on the queue."""
    try:
        from oracle import flow as F
        room, prm, geom, st = oracle_room(*shape)
        for _ in range(warmup):
            st, _ = F.step(st, geom, prm)
        barrier.wait(timeout=900)
        t0 = time.perf_counter()
        for _ in range(steps):
            st, _ = F.step(st, geom, prm)
        queue.put(("ok", time.perf_counter() - t0))
    except Exception as e:   # reported by the parent
        queue.put(("error", repr(e)))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_all_cores(shape, steps, warmup, procs):
    """The oracle as it stands, one independent copy of the room per host core (spawned processes, one thread
    each), the timed steps started together after a barrier: whole-host cell-updates/s = procs x cells x steps /
    the slowest process's time, like the max over ranks of the GPU arm."""
    import multiprocessing as mp
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    ctx = mp.get_context("spawn")
    barrier, queue = ctx.Barrier(procs), ctx.Queue()
    ps = [ctx.Process(target=oracle_worker, args=(shape, steps, warmup, barrier, queue)) for _ in range(procs)]
    for p in ps:
        p.start()
    import queue as queue_mod
    results = []
    while len(results) < procs:   # a process that dies without reporting ends the wait
        try:
            results.append(queue.get(timeout=1.0))
        except queue_mod.Empty:
            if not any(p.is_alive() for p in ps) and queue.empty():
                for p in ps:
                    p.join(timeout=1)
                raise RuntimeError("an oracle process exited without a result")
    for p in ps:
        p.join(timeout=60)
    errors = [r[1] for r in results if r[0] != "ok"]
    if errors:
        raise RuntimeError(f"oracle process failed: {errors[0]}")
    el = max(r[1] for r in results)
    cells = shape[0] * shape[1] * shape[2]
    return procs * cells * steps / el / 1e9, el


def pick_oracle_sample(steps_total, budget_s, slowdown):
    """Largest room of the ladder whose steps_total oracle steps fit budget_s, estimated from one timed step of the
    smallest room scaled by cells and by ``slowdown`` (per-cell cost falls with size, so the estimate errs long)."""
    from oracle import flow as F
    ladder = [(128, 64, 64), (64, 32, 32), (32, 16, 16)]
    room, prm, geom, st = oracle_room(*ladder[-1])
    st, _ = F.step(st, geom, prm)
    t0 = time.perf_counter()
    F.step(st, geom, prm)
    per_cell = (time.perf_counter() - t0) / room.cells
    for shape in ladder:
        if per_cell * slowdown * shape[0] * shape[1] * shape[2] * steps_total <= budget_s:
            return shape
    return ladder[-1]


def run_reference(args):
    """--impl reference: the oracle on every host core (one copy of the sample room per core), on a bounded sample
    of the workload sized so that the warm-up and timed steps end within a few minutes."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    procs = host_cores()
    budget_s = 150.0
    pick = pick_oracle_sample(args.steps + args.warmup, budget_s, slowdown=2.0)   # 2: cores share memory
    try:
        value, el = oracle_all_cores(pick, args.steps, args.warmup, procs)
    except Exception as e:   # one process in this one instead of no line
        print(f"all-core oracle run failed ({e!r}); timing this process alone", file=sys.stderr)
        from oracle import flow as F
        procs = 1
        room, prm, geom, st = oracle_room(*pick)
        for _ in range(args.warmup):
            st, _ = F.step(st, geom, prm)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            st, _ = F.step(st, geom, prm)
        el = time.perf_counter() - t0
        value = room.cells * args.steps / el / 1e9
    cells = pick[0] * pick[1] * pick[2]
    frac = cells / (256 * 128 * 128)
    sample = (f"each step {procs} independent full FP64 oracle steps (one process per host core) of the same room "
              f"construction at {pick[0]}x{pick[1]}x{pick[2]} ({frac:.4g} of the cells of the 256x128x128 room; "
              f"the largest of 128x64x64, 64x32x32, 32x16x16 whose {args.steps} + {args.warmup} steps fit about "
              f"{budget_s:.0f} s); numpy, one thread per process")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"single room 256x128x128 (sampled at {pick[0]}x{pick[1]}x{pick[2]}, "
                                   f"one copy per host core)", "cells": cells * procs,
                       "parallelism": f"{procs} host processes (host oracle)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def time_grid_steps(g, steps, stream, reduce_every=1):
    import torch
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    g.step(steps, reduce_every=reduce_every)
    end.record(stream)
    end.synchronize()
    return start.elapsed_time(end) / 1e3


def bench_large_room(stream, steps):
    """512 x 256 x 256 room (partition wall with doorway, two duct pairs, 20 seeded boxes, U_in = 0.1 m/s), FP32."""
    from paper_2204_02107_gb300 import native, rooms
    room = rooms.large_room()
    g = native.room_grid(room, precision="fp32", stream=stream.cuda_stream, history_capacity=max(16, steps + 3))
    g.autotune(reps=5)
    g.step(3, reduce_every=1)
    g.sync()
    sec = time_grid_steps(g, steps, stream)
    g.close()
    return {"workload": "large room 512x256x256, FP32 bulk + FP64 reductions every step, n = 4",
            "value": room.cells * steps / sec / 1e9, "unit": UNIT, "ms_per_step": sec * 1e3 / steps,
            "steps": steps, "cells": room.cells,
            "step_roofline_frac": STEP_MODEL_BYTES_PER_CELL_FP32 * room.cells * steps / sec / 1e9 / measured_peaks()[0]}


def bench_batch(stream, steps):
    """64 rooms of uneven size (64^3 .. 192x96x96, 0-10 boxes, U_in in [0.1, 1] m/s) advanced together."""
    import torch
    from paper_2204_02107_gb300 import native, rooms
    rs = rooms.batch_rooms(64)
    b = native.Batch(max_slots=64, hbm_budget_bytes=120 << 30, reduce_every=1, stream=stream.cuda_stream,
                     autotune=5)
    total = 0
    for r in rs:
        b.add(native.room_desc(r, precision="fp32", history_capacity=max(16, steps + 3)), r.beta, r.S,
              (r.u_in, 0.0, 0.0), 0.0, steps + 3, room=r.room, c0=r.initial_c())
        total += r.cells
    b.step(3)
    b.sync()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    b.step(steps)
    end.record(stream)
    end.synchronize()
    sec = start.elapsed_time(end) / 1e3
    info = b.info()
    b.close()
    return {"workload": "64 rooms 64^3..192x96x96 in one batch graph per step, FP32 bulk + FP64 reductions, "
                        "tiles autotuned per room shape on admission",
            "value": total * steps / sec / 1e9, "unit": UNIT, "ms_per_batch_step": sec * 1e3 / steps,
            "steps": steps, "rooms": len(rs), "cells": total, "bytes_in_use": info["bytes_in_use"]}


def bench_next_rows(stream, steps):
    """The single room with the paper's other modes: a dynamic time step (maximum Courant number 0.2, started
    from a developed jet), the inlet as a tanh window of Eq. 5, and one million Lagrangian particles."""
    import torch
    from paper_2204_02107_gb300 import native, rooms
    room = rooms.single_room(256, 128, 128)
    cells = room.cells
    out = {}

    def timed(g, n):
        g.step(3, reduce_every=1)
        g.sync()
        sec = time_grid_steps(g, n, stream)
        return sec

    # dynamic time step: develop the jet first so the Courant limit binds
    g = native.room_grid(room, precision="fp32", stream=stream.cuda_stream, courant_max=0.2,
                         history_capacity=max(16, steps + 400))
    g.step(300, reduce_every=0)
    sec = timed(g, steps)
    hist = g.history(steps)
    ph = g.profile_steps(5, reduce_every=1)
    g.close()
    out["dynamic_dt"] = {"value": cells * steps / sec / 1e9, "unit": UNIT, "ms_per_step": sec * 1e3 / steps,
                         "courant_max": 0.2, "dt_mean_s": float(np.mean([h["dt"] for h in hist])),
                         "dt_fixed_s": room.dt, "adjust_us": ph["adjust_dt"][0] / ph["adjust_dt"][1] * 1e3}
    # tanh inlet window over the duct
    g = native.room_grid(room, precision="fp32", stream=stream.cuda_stream)
    h = (room.lx / room.nx, room.ly / room.ny, room.lz / room.nz)
    ys, zs = np.nonzero(room.S.any(axis=2).T)
    center = (0.5 * h[0], 0.5 * (ys.min() + ys.max()) * h[1], 0.5 * (zs.min() + zs.max()) * h[2])
    g.set_inflow_tanh(center, (3 * h[0], 5 * h[1], 5 * h[2]), (2.0, 3.0, 3.0), (room.u_in, 0.0, 0.0), 0.0)
    sec = timed(g, steps)
    g.close()
    out["tanh_inlet"] = {"value": cells * steps / sec / 1e9, "unit": UNIT, "ms_per_step": sec * 1e3 / steps}
    # particles: one million, sizes 1-100 um, uniformly in the fluid
    n = 1 << 20
    rng = np.random.default_rng(12)
    fluid = np.argwhere(room.beta.astype(bool))
    cellsel = fluid[rng.integers(0, len(fluid), n)]
    pos = (cellsel[:, ::-1] + rng.uniform(-0.45, 0.45, (n, 3))) * np.array(h)
    pos = np.mod(pos, np.array([room.lx, room.ly, room.lz]))
    g = native.room_grid(room, precision="fp32", stream=stream.cuda_stream)
    g.set_particles(pos, np.zeros((n, 3)), rng.uniform(1e-6, 100e-6, n))
    sec = timed(g, steps)
    ph = g.profile_steps(5, reduce_every=1)
    g.close()
    p_us = ph["particles"][0] / ph["particles"][1] * 1e3
    # per particle: read x, y, z, u, v, w, d and the state (60 B), write x, y, z, u, v, w (48 B); the eight
    # sampled 4-vectors come from the field, mostly through L2
    p_bytes = 108.0
    out["particles"] = {"value": cells * steps / sec / 1e9, "unit": UNIT, "ms_per_step": sec * 1e3 / steps,
                        "particles": n, "particle_kernel_us": p_us,
                        "particle_updates_per_s": n / (p_us * 1e-6),
                        "particle_kernel_gb_s": n * p_bytes / (p_us * 1e-6) / 1e9,
                        "bytes_per_particle": p_bytes}
    return out


def bench_cube_wake(stream, cells_per_h=30, warm=24000, meas=12000, every=5, fevery=50):
    """Cube-in-channel validation (Sec. 3.1.2, Tab. 2): Strouhal number of the vortex street from the transverse
    velocity at a wake probe (upward zero crossings), mean drag coefficient from the immersed-boundary force on the
    obstacle, FP32, 30 cells per obstacle side; throughput over the development steps."""
    import torch
    from paper_2204_02107_gb300 import native, rooms
    cc = rooms.cube_channel(cells_per_h)
    g = native.Grid(cc.nx, cc.ny, cc.nz, cc.lx, cc.ly, cc.lz, nu=cc.nu, dt=cc.dt, precision="fp32",
                    history_capacity=16, stream=stream.cuda_stream)
    g.set_mask(cc.beta)
    g.set_inflow_field(cc.S, cc.targets)
    g.set_force_region(cc.cube)
    rng = np.random.default_rng(1)
    g.set_field("u", cc.u_init)
    g.set_field("v", 0.01 * rng.standard_normal(cc.shape) * (cc.beta > 0))
    sec = time_grid_steps(g, warm, stream, reduce_every=0)
    dst = torch.empty(cc.cells, dtype=torch.float32, device="cuda")
    pz, py, px = cc.probe
    pidx = px + cc.nx * (py + cc.ny * pz)
    probe = torch.empty(meas // every, dtype=torch.float32, device="cuda")
    forces = []
    with torch.cuda.stream(stream):
        for k in range(meas // every):
            g.step(every, reduce_every=0)
            native.lib().vf_read_field(g._h, native.FIELDS["v"], native.C.c_void_p(dst.data_ptr()), 0,
                                       native.VF_DEVICE)
            probe[k] = dst[pidx]
            if (k * every) % fevery == 0:
                forces.append(g.region_force())
    g.sync()
    g.close()
    sig = probe.double().cpu().numpy()
    t = (np.arange(len(sig)) + 1) * every * cc.dt
    s = sig - sig.mean()
    zc = [t[i] - s[i] * (t[i + 1] - t[i]) / (s[i + 1] - s[i]) for i in range(len(s) - 1) if s[i] < 0 <= s[i + 1]]
    st = cc.h_obstacle / (float(np.mean(np.diff(zc))) * cc.u_bulk) if len(zc) > 2 else None
    cd = 2.0 * float(np.mean([f[0] for f in forces])) / (cc.u_bulk ** 2 * cc.h_obstacle * cc.lz)
    return {"workload": f"cube in channel {cc.nx}x{cc.ny}x{cc.nz} (2D flow, periodic z), {cells_per_h} cells per "
                        f"obstacle side, Re_ob = 84, FP32", "value": cc.cells * warm / sec / 1e9, "unit": UNIT,
            "strouhal": st, "drag_coefficient": cd, "periods_measured": len(zc) - 1,
            "paper_table2_30_cells": {"strouhal": 0.2097, "drag_coefficient": 3.12}}


def bench_serve(n_requests, fp64_sample=12):
    """Serving (Poisson arrivals, 4 requests per second, seed 5; grids 64^3..256x128x128, inflow 0.1 or 1 m/s,
    200-2000 steps, random masks; 120 GB budget) by continuous batching in FP32: the real-time trace for latency,
    the same trace with every request visible at t = 0 for capacity (solves per hour with the queue never empty),
    and the GPU's cell-update rate while serving.  The one-at-a-time FP64 server is timed on the first
    ``fp64_sample`` requests (the whole trace would take about ten minutes in FP64), against the FP32 server on the
    same requests, both saturated; ACH of those requests from both servers is compared."""
    from paper_2204_02107_gb300 import rooms, serve
    reqs = rooms.request_trace(count=n_requests, seed=5, rate_per_s=4.0, step_range=(200, 2000))

    def served(requests, realtime):
        srv = serve.Server(hbm_budget_bytes=120 << 30, max_slots=64, chunk_steps=25, precision="fp32")
        t0 = time.perf_counter()
        res = srv.run(requests, realtime=realtime)
        wall = time.perf_counter() - t0
        srv.close()
        return res, wall

    rt, _ = served(reqs, True)
    at_zero = [dict(r, arrival_s=0.0) for r in reqs]      # saturated: every request waiting from t = 0
    sat, sat_wall = served(at_zero, False)
    sample = [dict(r, arrival_s=0.0) for r in sorted(reqs, key=lambda r: r["arrival_s"])[:fp64_sample]]
    sat_sample, sample_wall = served(sample, False)
    t0 = time.perf_counter()
    base = serve.run_one_at_a_time(sample, precision="fp64", realtime=False)
    base_wall = time.perf_counter() - t0
    by_id = {r.id: r for r in base}
    rel = [abs(r.ach_per_hour - by_id[r.id].ach_per_hour) / abs(by_id[r.id].ach_per_hour) for r in sat
           if r.id in by_id and by_id[r.id].ach_per_hour]
    fp32_sample_sph = len(sat_sample) / sample_wall * 3600.0
    fp64_sample_sph = len(base) / base_wall * 3600.0
    return {"workload": f"{n_requests} requests, Poisson arrivals 4/s (seed 5), grids 64^3..256x128x128, "
                        f"200-2000 steps, inflow 0.1 or 1 m/s, random masks, 120 GB budget",
            "continuous_batching_fp32_realtime": serve.summarize(rt),
            "continuous_batching_fp32_saturated": dict(serve.summarize(sat, makespan_s=sat_wall),
                                                        note="every request visible at t = 0; latency from t = 0"),
            "single_room_gcell_updates_per_s_for_context": None,
            "fp64_sample": {"requests": len(base), "one_at_a_time_fp64_solves_per_hour": fp64_sample_sph,
                            "continuous_batching_fp32_solves_per_hour": fp32_sample_sph,
                            "fp32_served_over_fp64": fp32_sample_sph / fp64_sample_sph,
                            "one_at_a_time_fp64": serve.summarize(base, makespan_s=base_wall),
                            "note": f"the first {len(base)} requests of the trace, all visible at t = 0, served "
                                    "one at a time in FP64 and by continuous batching in FP32"},
            "ach_rel_diff_max": max(rel) if rel else None,
            "ach_within_half_percent": (max(rel) <= 5e-3) if rel else None}


def bench_fft_vs_cufft(stream, nx=256, ny=128, nz=128, lengths=(10.0, 5.0, 5.0), reps=50):
    """One FFT Poisson solve of the room's grid (Sec. 2.2: forward 3D FFT, division by lambda with the null modes
    set to 0, inverse 3D FFT), FP32: the library's own kernels (vf_poisson_solve) against cuFFT doing the same
    solve through torch.fft (R2C, a multiply by 1/lambda, C2R).  A timed comparison only: the step never calls
    cuFFT."""
    import torch
    from paper_2204_02107_gb300 import native
    lx, ly, lz = lengths
    g = native.Grid(nx, ny, nz, lx, ly, lz, nu=1.6e-5, dt=1e-2, precision="fp32", stream=stream.cuda_stream)
    gen = torch.Generator(device="cuda").manual_seed(11)
    f = torch.randn((nz, ny, nx), generator=gen, device="cuda", dtype=torch.float32)
    p = torch.empty_like(f)
    # eigenvalues of D o G on the R2C half spectrum, shape (nz, ny, nx/2 + 1); the eight null modes -> 0
    h = (lx / nx, ly / ny, lz / nz)
    kz = torch.arange(nz, device="cuda", dtype=torch.float64).view(nz, 1, 1)
    ky = torch.arange(ny, device="cuda", dtype=torch.float64).view(1, ny, 1)
    kx = torch.arange(nx // 2 + 1, device="cuda", dtype=torch.float64).view(1, 1, nx // 2 + 1)
    lam = -(torch.sin(2 * math.pi * kx / nx) ** 2 / h[0] ** 2 + torch.sin(2 * math.pi * ky / ny) ** 2 / h[1] ** 2
            + torch.sin(2 * math.pi * kz / nz) ** 2 / h[2] ** 2)
    inv_lam = torch.where(lam.abs() > 1e-9 * lam.abs().max(), 1.0 / lam, torch.zeros_like(lam)).float()

    def ours():
        g.poisson_solve(f, p)

    def cufft():
        fh = torch.fft.rfftn(f)
        fh.mul_(inv_lam)
        return torch.fft.irfftn(fh, s=(nz, ny, nx))

    def timed(fn):
        for _ in range(5):
            fn()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for _ in range(reps):
            fn()
        end.record(stream)
        end.synchronize()
        return start.elapsed_time(end) / reps * 1e3

    with torch.cuda.stream(stream):
        t_ours = timed(ours)
        t_cufft = timed(cufft)
        ref = cufft()
        ours()
        torch.cuda.current_stream().synchronize()
        diff = float((p - ref).norm() / ref.norm())
    g.close()
    return {"workload": f"one FFT Poisson solve, {nx}x{ny}x{nz}, FP32 (forward FFT, 1/lambda, inverse FFT)",
            "ours_us": t_ours, "cufft_us": t_cufft, "cufft_over_ours": t_cufft / t_ours, "rel_l2_diff": diff,
            "cufft_path": "torch.fft.rfftn, multiply by 1/lambda, torch.fft.irfftn on the same stream"}


def e2e_run(room, precision, steps, stream, per_step=False):
    """End to end through the C ABI with pinned host buffers: grid creation, mask / inflow / region / scalar
    upload, ``steps`` steps with a reduction record each, then the records and all five fields read back.
    per_step: every step is its own vf_step(1) followed by vf_history(1), which copies that step's record to the
    host and so waits for the step (a caller monitoring every step)."""
    import torch
    from paper_2204_02107_gb300 import native
    n = room.cells

    def pinned(arr, dtype):
        t = torch.empty(arr.size, dtype=dtype, pin_memory=True)
        t.numpy()[:] = arr.ravel()
        return t.numpy()

    beta = pinned(room.beta, torch.uint8)
    S = pinned(room.S, torch.uint8)
    region = pinned(room.room, torch.uint8)
    c0 = pinned(room.initial_c().astype(np.float32), torch.float32)
    outs = [torch.empty(n, dtype=torch.float32, pin_memory=True).numpy() for _ in range(5)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = native.Grid(room.nx, room.ny, room.nz, room.lx, room.ly, room.lz, nu=1.6e-5, dt=room.dt,
                    precision=precision, stream=stream.cuda_stream, history_capacity=max(16, steps))
    t_create = time.perf_counter()
    g.set_mask(beta)
    g.set_inflow(S, (room.u_in, 0.0, 0.0), 0.0)
    g.set_region(region)
    g.set_field("c", c0)
    g.sync()
    t_upload = time.perf_counter()
    if per_step:
        hist = []
        for _ in range(steps):
            g.step(1, reduce_every=1)
            hist += g.history(1)
    else:
        g.step(steps, reduce_every=1)
        hist = g.history(steps)
    t_steps = time.perf_counter()
    for name, out in zip(("u", "v", "w", "c", "p"), outs):
        native.lib().vf_read_field(g._h, native.FIELDS[name], native.C.c_void_p(out.ctypes.data), 0,
                                   native.VF_HOST)
    g.sync()
    el = time.perf_counter() - t0
    g.close()
    h2d = 3 * n + 4 * n
    d2h = 5 * 4 * n + len(hist) * native.C.sizeof(native.VfReduce) + (8 * steps if per_step else 8)
    what = ("create grid + upload mask, forcing region, room region, scalar (pinned host) + steps with per-step FP64 "
            "reductions + read back the reduction records and u, v, w, c, p")
    if per_step:
        what += "; each step launched alone and its record read back (a host wait) before the next"
    return {"value": n * steps / el / 1e9, "unit": UNIT, "h2d_bytes_per_step": h2d / steps,
            "d2h_bytes_per_step": d2h / steps, "seconds": el,
            "seconds_by_part": {"create_grid": t_create - t0, "upload_inputs": t_upload - t_create,
                                "steps_and_records": t_steps - t_upload, "read_fields": t0 + el - t_steps},
            "steps": steps, "records_read": len(hist),
            "last_record_step": hist[-1]["step"] if hist else None, "what": what}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=100)
    ap.add_argument("--extra-steps", type=int, default=30, help="timed steps of the large-room and batch legs")
    ap.add_argument("--serve-requests", type=int, default=256, help="requests of the serving leg (0: skip)")
    ap.add_argument("--no-extras", action="store_true", help="skip the large-room, batch and serving legs")
    ap.add_argument("--extras", default="large_room,batch,next_rows,cube_wake,serve",
                    help="comma list of the extra legs to run (large_room, batch, next_rows, cube_wake, serve)")
    ap.add_argument("--no-autotune", action="store_true", help="launch with the default tiles")
    ap.add_argument("--tiles", default=None, help="z-chunks stage,div,project,filter (skips the autotuner)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    from paper_2204_02107_gb300 import native, rooms
    native.lib()

    room = rooms.single_room(256, 128, 128)
    stream = torch.cuda.Stream()
    g = native.room_grid(room, precision="fp32", stream=stream.cuda_stream)
    if args.tiles:
        g.set_tiles(*[int(v) for v in args.tiles.split(",")])
        tiles, tiles_source = g.tiles(), "given"
    elif args.no_autotune:
        tiles, tiles_source = g.tiles(), "defaults"
    else:
        tiles, tiles_source = g.autotune(reps=20), "autotuned before warm-up"
    cells = room.cells
    launches_per_step = None   # counted from the profiled steps below

    g.step(args.warmup, reduce_every=1)
    g.sync()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0]) if \
        os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local
    with ClockSampler(gpu_index) as clocks:
        time.sleep(0.3)
        dist_barrier(world)
        torch.cuda.synchronize()
        start.record(stream)
        g.step(args.steps, reduce_every=1)
        end.record(stream)
        end.synchronize()
        torch.cuda.synchronize()
        dist_barrier(world)
    ms = start.elapsed_time(end)
    ms_max = dist_max(ms, world)
    hist = g.history(16)
    value = world * cells * args.steps / (ms_max / 1e3) / 1e9

    # per-kernel durations (CUDA events after every launch on the grid's stream)
    prof_steps = max(3, min(args.steps, 20))
    phases = g.profile_steps(prof_steps, reduce_every=1)
    peak, peak_kind = measured_peaks()
    per_kernel = {}
    for name, (tot_ms, nl) in phases.items():
        avg_s = tot_ms / nl / 1e3
        bpc = PHASE_BYTES_PER_CELL.get(name)
        per_kernel[name] = {"launches": nl, "avg_us": avg_s * 1e6, "share": None,
                            "algorithmic_gb_s": None if bpc is None else bpc * cells / avg_s / 1e9}
    total_ms = sum(t for t, _ in phases.values())
    for name, (tot_ms, _) in phases.items():
        per_kernel[name]["share"] = tot_ms / total_ms
    # dominant kernel: phases grouped by the kernel function that runs them (the four RK4 stages are one kernel,
    # k_stage), ranked by total time; achieved = its algorithmic bytes over its time, per launch
    groups = {}
    for name, (tot_ms, nl) in phases.items():
        bpc = PHASE_BYTES_PER_CELL.get(name)
        if bpc is None:
            continue
        kname = PHASE_KERNEL.get(name, name)
        g_ms, g_n, g_b = groups.get(kname, (0.0, 0, 0.0))
        groups[kname] = (g_ms + tot_ms, g_n + nl, g_b + bpc * cells * nl)
    dominant = max(groups, key=lambda k: groups[k][0])
    g_ms, g_n, g_b = groups[dominant]
    achieved = (g_b / g_n) / (g_ms / g_n / 1e3) / 1e9
    traffic = traffic_record(dominant, tiles)
    step_s = ms_max / 1e3 / args.steps
    step_gbs = STEP_MODEL_BYTES_PER_CELL_FP32 * cells / step_s / 1e9
    # the bytes this implementation's kernels must move per cell-step (every phase's algorithmic bytes times its
    # launches per step; the Eq. 9 correction, which touches only the cells next to solids, is left out)
    actual_bpc = sum(PHASE_BYTES_PER_CELL[name] * nl / prof_steps for name, (_, nl) in phases.items()
                     if PHASE_BYTES_PER_CELL.get(name) is not None)
    actual_gbs = actual_bpc * cells / step_s / 1e9

    # FP64 form of the same step (parity path)
    g64 = native.room_grid(room, precision="fp64", stream=stream.cuda_stream)
    tiles64 = g64.tiles() if (args.no_autotune or args.tiles) else g64.autotune(reps=5)
    g64.step(3, reduce_every=1)
    g64.sync()
    s64, e64 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s64.record(stream)
    g64.step(args.fp64_steps, reduce_every=1)
    e64.record(stream)
    e64.synchronize()
    fp64_ms = s64.elapsed_time(e64)
    # one more step inside an NVTX range: the range ncu's FP64 instruction count is taken over
    torch.cuda.nvtx.range_push("fp64_step")
    g64.step(1, reduce_every=1)
    g64.sync()
    torch.cuda.nvtx.range_pop()
    g64.close()
    fp64_peak = native.measure_fp64_rate()
    fp64_flops = fp64_flop_record()
    fp64_achieved = None if fp64_flops is None else fp64_flops * cells / (fp64_ms / args.fp64_steps / 1e3) / 1e9

    e2e = e2e_run(room, "fp32", args.steps, stream)
    try:
        e2e_each = e2e_run(room, "fp32", min(args.steps, 500), stream, per_step=True)
    except Exception as e:   # an extra figure: never costs the line
        e2e_each = {"error": repr(e)}
    g.close()
    extras = {"fft_vs_cufft": bench_fft_vs_cufft(stream)}
    legs = set() if args.no_extras else {x.strip() for x in args.extras.split(",") if x.strip()}
    if legs and world == 1:
        if "large_room" in legs:
            extras["large_room"] = bench_large_room(stream, args.extra_steps)
        if "batch" in legs:
            extras["batch"] = bench_batch(stream, args.extra_steps)
        if "next_rows" in legs:
            extras["next_rows"] = bench_next_rows(stream, max(args.extra_steps, 100))
        if "cube_wake" in legs:
            extras["cube_wake"] = bench_cube_wake(stream)
        if "serve" in legs and args.serve_requests > 0:
            extras["serve"] = bench_serve(args.serve_requests)
            extras["serve"]["single_room_gcell_updates_per_s_for_context"] = value

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "single room 256x128x128 (10x5x5 m, 2-cell walls, 5x5 duct, U_in = 1 m/s), "
                               "FP32 bulk + FP64 reductions every step, filter on, 4 pressure iterations",
                   "cells": cells, "global_cells": cells * world, "precision": "fp32_mixed",
                   "l2": "state 0.3 GB > 126 MB L2: inputs larger than L2, no flush",
                   "parallelism": "one independent room per GPU" if world > 1 else "single GPU",
                   "tiles": tiles, "tiles_source": tiles_source},
        "roofline": {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": g_b / g_n, "launches_per_step": g_n / prof_steps,
                     "avg_launch_us": g_ms / g_n * 1e3},
        "step_roofline": {"model_bytes_per_cell": STEP_MODEL_BYTES_PER_CELL_FP32, "achieved_gb_s": step_gbs,
                          "frac": step_gbs / peak, "peak_kind": peak_kind,
                          "actual_bytes_per_cell": actual_bpc, "actual_achieved_gb_s": actual_gbs,
                          "actual_frac": actual_gbs / peak},
        "kernels": per_kernel,
        "fp64": {"value": cells * args.fp64_steps / (fp64_ms / 1e3) / 1e9, "unit": UNIT,
                 "ms_per_step": fp64_ms / args.fp64_steps, "steps": args.fp64_steps, "tiles": tiles64,
                 "roofline": {"bound": "fp64_alu", "unit": "GFLOP/s", "achieved": fp64_achieved,
                              "peak": fp64_peak, "peak_kind": "measured FP64 FMA rate of this device",
                              "frac": None if fp64_achieved is None else fp64_achieved / fp64_peak,
                              "flops_per_cell_step": fp64_flops}},
        "e2e": e2e,
        "e2e_result_read_every_step": e2e_each,
        "gpu_launches": int(round(sum(n for _, n in phases.values()) / prof_steps)) * args.steps,
        "clocks": clocks.summary(),
        "last_record": {k: hist[-1][k] for k in ("step", "ke", "c_room", "div_max", "u_max")} if hist else None,
    }
    line.update(extras)
    if world == 1 and rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_oracle(room, "FP64, filter on, 4 pressure iterations")
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
