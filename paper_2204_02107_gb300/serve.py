"""Continuous-batching server for ventilation-scenario requests.

Requests (room grid, mask, inflow speed, step count) arrive over time.  The server keeps every admitted room on
the device in a batch (``native.Batch``): between chunks of batch steps it admits waiting requests as long as a
free slot and the device-memory budget allow, the rooms of one chunk run concurrently in one CUDA graph launch per
step, and finished rooms are read out (the per-step reduction history, the air changes per hour fitted from the
mean scalar, the Wells-Riley risk) and released.  A request's result is computed exactly as if the room ran alone.

The comparison server, ``run_one_at_a_time``, takes the same requests first-come first-served, one grid at a time.
"""
from __future__ import annotations

import collections
import dataclasses
import os
import time

import numpy as np

from . import native, rooms


@dataclasses.dataclass
class Result:
    id: int
    arrival_s: float
    start_s: float
    finish_s: float
    cells: int
    steps: int
    ach_per_hour: float
    c_mean_final: float
    risk_30min: float

    @property
    def latency_s(self):
        return self.finish_s - self.arrival_s


def room_result(req, grid, room, arrival, start, finish):
    """Read a finished room: ACH from the log-slope of the room-mean scalar (Sec. 3.3.2) and the 30-minute
    Wells-Riley risk of 100 quanta in the room volume at that ACH (Eqs. 17-18)."""
    hist = grid.history(req["steps"])
    t = np.array([h["t"] for h in hist])
    cm = np.array([h["c_room"] / h["v_room"] for h in hist])
    ach = native.ach_log_slope(t, cm) if len(t) >= 2 and np.all(cm > 0) else float("nan")
    v_room = hist[-1]["v_room"] if hist else float("nan")
    _, risk = native.wells_riley(100.0 / v_room, 1.2, max(ach, 0.0), 0.5) if np.isfinite(ach) else (0.0, float("nan"))
    return Result(req["id"], arrival, start, finish, room.cells, req["steps"], ach, float(cm[-1]) if len(cm) else
                  float("nan"), risk)


class Server:
    """Continuous batching over a ``native.Batch``."""

    def __init__(self, hbm_budget_bytes=120 << 30, max_slots=64, chunk_steps=50, precision="fp32", autotune=0,
                 tile_cache_path=None):
        """autotune > 0: the first room of each shape is autotuned with that many reps when admitted.
        tile_cache_path: a JSON tile cache (``native.tile_cache_save``) loaded now if the file exists and written
        back by close(), so tuned tiles outlive the server."""
        self.tile_cache_path = tile_cache_path
        if tile_cache_path is not None and os.path.exists(tile_cache_path):
            native.tile_cache_load(tile_cache_path)
        self.batch = native.Batch(max_slots=max_slots, hbm_budget_bytes=hbm_budget_bytes, reduce_every=1,
                                  autotune=autotune)
        self.chunk = chunk_steps
        self.precision = precision
        self.max_slots = max_slots

    def close(self):
        self.batch.close()
        if self.tile_cache_path is not None:
            native.tile_cache_save(self.tile_cache_path)

    def run(self, requests, realtime=True):
        """Serve a trace (dicts from ``rooms.request_trace``); returns the list of Results in completion order.

        realtime=True: a request becomes visible at its arrival time on the wall clock; False: all requests are
        visible at once (arrival times still define latency).

        Admission overlaps the GPU: a chunk of batch steps is launched first, then the waiting requests are admitted
        into the free slots while it runs (a new room's uploads go through its own stream, never behind the running
        rooms), and they join the batch from the next chunk on."""
        pending = collections.deque(sorted(requests, key=lambda r: r["arrival_s"]))
        waiting = collections.deque()
        active = {}                               # slot -> (request, room, start time)
        results = []
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0
        c_dtype = np.float32 if self.precision != "fp64" else np.float64

        def arrivals():
            now = clock()
            while pending and (not realtime or pending[0]["arrival_s"] <= now):
                req = pending.popleft()
                waiting.append((req, rooms.request_room(req)))

        def admit():
            # in arrival order while slots and memory allow
            while waiting:
                req, room = waiting[0]
                desc = native.room_desc(room, precision=self.precision, history_capacity=max(16, req["steps"]))
                try:
                    slot = self.batch.add(desc, room.beta, room.S, (room.u_in, 0.0, 0.0), 0.0, req["steps"],
                                          room=room.room, c0=room.initial_c(c_dtype))
                except native.VentflowError as e:
                    if e.code == native.VF_ENOMEM and active:
                        break                     # wait for running rooms to free memory
                    raise
                waiting.popleft()
                active[slot] = (req, room, clock())

        while pending or waiting or active:
            arrivals()
            if not active:
                admit()
                if not active:
                    if pending:
                        time.sleep(max(0.0, min(0.05, pending[0]["arrival_s"] - clock())))
                    continue
            self.batch.step(self.chunk)           # launched; the GPU runs it while the host admits
            arrivals()
            admit()
            for slot in self.batch.poll():        # waits for the chunk
                req, room, start = active.pop(slot)
                results.append(room_result(req, self.batch.grid(slot), room, req["arrival_s"], start, clock()))
                self.batch.remove(slot)
        return results


def run_one_at_a_time(requests, precision="fp64", realtime=True):
    """First-come first-served, one grid at a time (the comparison server)."""
    results = []
    t0 = time.perf_counter()
    clock = lambda: time.perf_counter() - t0
    for req in sorted(requests, key=lambda r: r["arrival_s"]):
        if realtime:
            while clock() < req["arrival_s"]:
                time.sleep(min(0.05, req["arrival_s"] - clock()))
        start = clock()
        room = rooms.request_room(req)
        g = native.room_grid(room, precision=precision, history_capacity=max(16, req["steps"]))
        g.step(req["steps"], reduce_every=1)
        g.sync()
        results.append(room_result(req, g, room, req["arrival_s"], start, clock()))
        g.close()
    return results


def summarize(results, makespan_s=None):
    lat = np.array([r.latency_s for r in results])
    if makespan_s is None:
        makespan_s = max(r.finish_s for r in results) - min(r.arrival_s for r in results)
    cells_steps = sum(r.cells * r.steps for r in results)
    return {"requests": len(results), "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "makespan_s": makespan_s,
            "solves_per_hour": len(results) / makespan_s * 3600.0,
            "gcell_updates_per_s": cells_steps / makespan_s / 1e9}
