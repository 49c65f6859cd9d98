"""Continuous batching on the host, without a GPU: the server's admission, chunked stepping and read-out run against
a stand-in batch that keeps the library's admission rules (a free slot and the memory budget counted in
vf_grid_bytes) and whose rooms record an exact exponential decay of the room-mean scalar.  Every request must be
served once, admitted in arrival order, never beyond the budget or the slots, and the air changes per hour read out
from a finished room must be its decay rate (Sec. 3.3.2's log-slope through the library's host metrics)."""
import math

import numpy as np
import pytest

from oracle import ventilation as V
from paper_2204_02107_gb300 import native, rooms, serve


def decay_rate_per_hour(desc, u_set):
    """The stand-in room's ACH, fixed by its description (distinct per size and inflow)."""
    return 0.5 + desc.nx / 64.0 + 3.0 * u_set[0]


class FakeGrid:
    def __init__(self, rec):
        self.rec = rec

    def history(self, max_records=None):
        r = self.rec
        v_room = 12.5
        k = r["ach"] / 3600.0
        out = [{"t": s * r["dt"], "c_room": v_room * math.exp(-k * s * r["dt"]), "v_room": v_room}
               for s in range(1, r["done"] + 1)]
        return out if max_records is None else out[-max_records:]


class FakeBatch:
    def __init__(self, max_slots, hbm_budget_bytes, reduce_every=1, **kw):
        self.max_slots, self.budget = max_slots, hbm_budget_bytes
        self.rooms = {}
        self.in_use = 0
        self.peak_bytes = 0
        self.peak_rooms = 0
        self.admitted = []          # (nx, u_in) in admission order
        FakeBatch.last = self

    def add(self, desc, beta, S, u_set, c_set, steps, room=None, c0=None):
        need = native.grid_bytes(desc)
        free = [s for s in range(self.max_slots) if s not in self.rooms]
        if not free or self.in_use + need > self.budget:
            raise native.VentflowError(native.VF_ENOMEM, "stand-in batch full")
        slot = free[0]
        self.rooms[slot] = {"need": need, "steps": steps, "done": 0, "dt": desc.dt, "reported": False,
                            "ach": decay_rate_per_hour(desc, u_set)}
        self.in_use += need
        self.peak_bytes = max(self.peak_bytes, self.in_use)
        self.peak_rooms = max(self.peak_rooms, len(self.rooms))
        self.admitted.append((desc.nx, u_set[0]))
        return slot

    def step(self, n):
        for r in self.rooms.values():
            r["done"] = min(r["steps"], r["done"] + n)

    def poll(self):
        out = [s for s, r in self.rooms.items() if r["done"] >= r["steps"] and not r["reported"]]
        for s in out:
            self.rooms[s]["reported"] = True
        return out

    def grid(self, slot):
        return FakeGrid(self.rooms[slot])

    def remove(self, slot):
        self.in_use -= self.rooms.pop(slot)["need"]

    def close(self):
        pass


def trace(count=12):
    return rooms.request_trace(count=count, seed=5, sizes=[(64, 64, 64), (96, 64, 64), (128, 64, 64)],
                               step_range=(60, 400))


def one_room_bytes(req):
    return native.grid_bytes(native.room_desc(rooms.request_room(req), precision="fp32",
                                              history_capacity=max(16, req["steps"])))


@pytest.mark.parametrize("rooms_in_budget,max_slots", [(2.5, 64), (100.0, 3), (1.0, 64)])
def test_every_request_served_within_budget_and_slots(monkeypatch, rooms_in_budget, max_slots):
    monkeypatch.setattr(native, "Batch", FakeBatch)
    reqs = trace()
    biggest = max(one_room_bytes(r) for r in reqs)
    budget = int(rooms_in_budget * biggest)
    srv = serve.Server(hbm_budget_bytes=budget, max_slots=max_slots, chunk_steps=50)
    results = srv.run(reqs, realtime=False)
    fb = FakeBatch.last
    srv.close()
    assert sorted(r.id for r in results) == [r["id"] for r in reqs]
    assert fb.peak_bytes <= budget and fb.peak_rooms <= max_slots and fb.in_use == 0 and not fb.rooms
    if rooms_in_budget >= 2 and max_slots >= 2:
        assert fb.peak_rooms >= 2                    # rooms really overlap
    # admission in arrival order (first come, first admitted)
    by_arrival = sorted(reqs, key=lambda r: r["arrival_s"])
    assert fb.admitted == [(r["nx"], r["u_in"]) for r in by_arrival]
    starts = {r.id: r.start_s for r in results}
    order = [starts[r["id"]] for r in by_arrival]
    assert order == sorted(order)
    for res in results:
        req = reqs[res.id]
        room = rooms.request_room(req)
        desc = native.room_desc(room)
        want = decay_rate_per_hour(desc, (req["u_in"], 0.0, 0.0))
        assert res.ach_per_hour == pytest.approx(want, rel=1e-9)
        assert res.steps == req["steps"] and res.cells == room.cells
        assert res.finish_s >= res.start_s
        q = V.wells_riley_dose(100.0 / 12.5, 1.2, want, 0.5)
        assert res.risk_30min == pytest.approx(V.infection_probability(q), rel=1e-9)


def test_room_over_the_whole_budget_is_an_error(monkeypatch):
    monkeypatch.setattr(native, "Batch", FakeBatch)
    reqs = trace(3)
    srv = serve.Server(hbm_budget_bytes=min(one_room_bytes(r) for r in reqs) - 1, max_slots=4)
    with pytest.raises(native.VentflowError) as e:
        srv.run(reqs, realtime=False)
    assert e.value.code == native.VF_ENOMEM
    srv.close()


def test_summary_counts_and_percentiles():
    res = [serve.Result(i, arrival_s=float(i), start_s=float(i), finish_s=float(i) + 1.0 + i, cells=1000, steps=10,
                        ach_per_hour=1.0, c_mean_final=0.5, risk_30min=0.01) for i in range(5)]
    s = serve.summarize(res)
    assert s["requests"] == 5
    assert s["p50_latency_s"] == pytest.approx(3.0)
    assert s["p99_latency_s"] == pytest.approx(np.percentile([1, 2, 3, 4, 5], 99))
    assert s["makespan_s"] == pytest.approx(9.0)       # first arrival 0, last finish 4 + 5
    assert s["solves_per_hour"] == pytest.approx(5 / 9.0 * 3600)
    assert s["gcell_updates_per_s"] == pytest.approx(5 * 1000 * 10 / 9.0 / 1e9)


def test_server_keeps_its_tuned_tiles_across_restarts(monkeypatch, tmp_path):
    monkeypatch.setattr(native, "Batch", FakeBatch)
    native.tile_cache_clear()
    path = str(tmp_path / "tiles.json")
    tiles = {"zc_stage": 8, "zc_div": 16, "zc_project": 8, "zc_filter": 32, "fft_x": 1, "fft_y": 0, "fft_z": 2}
    srv = serve.Server(tile_cache_path=path)             # no file yet: nothing to load
    native.tile_cache_insert(96, 64, 64, "fp32", tiles)  # what an admission autotune leaves in the cache
    srv.close()                                          # writes the cache
    native.tile_cache_clear()
    srv = serve.Server(tile_cache_path=path)             # a restarted server loads it
    assert native.tile_cache_lookup(96, 64, 64, "fp32") == tiles
    srv.close()
    native.tile_cache_clear()
