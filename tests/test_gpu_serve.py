"""Continuous-batching server: every request's result equals the same room run alone (bitwise fields, same ACH),
requests arriving while others run are admitted between chunks, and a tight memory budget defers admission
without failing."""
import numpy as np
import pytest

from paper_2204_02107_gb300 import native, rooms, serve
from gpu_helpers import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def small_trace(n=6, seed=11):
    sizes = [(40, 24, 20), (48, 30, 18), (32, 32, 16), (64, 32, 32)]
    return rooms.request_trace(count=n, seed=seed, rate_per_s=50.0, sizes=sizes, step_range=(5, 25))


def test_served_results_equal_solo_runs(torch):
    reqs = small_trace()
    srv = serve.Server(hbm_budget_bytes=4 << 30, max_slots=4, chunk_steps=4)
    results = srv.run(reqs, realtime=True)
    srv.close()
    assert sorted(r.id for r in results) == [r["id"] for r in reqs]
    solo = {r.id: r for r in serve.run_one_at_a_time(reqs, precision="fp32", realtime=False)}
    for r in results:
        s = solo[r.id]
        assert r.steps == s.steps and r.cells == s.cells
        assert r.ach_per_hour == s.ach_per_hour          # same arithmetic alone and in the mix
        assert r.c_mean_final == s.c_mean_final
        assert r.latency_s > 0


def test_fields_bitwise_in_mix(torch):
    """A room admitted into a busy batch ends with the same fields as alone."""
    reqs = small_trace(n=3, seed=5)
    b = native.Batch(max_slots=3, hbm_budget_bytes=4 << 30, reduce_every=1)
    slots = {}
    for i, req in enumerate(reqs):
        room = rooms.request_room(req)
        slots[req["id"]] = (b.add(native.room_desc(room), room.beta, room.S, (room.u_in, 0, 0), 0.0, req["steps"],
                                  room=room.room, c0=room.initial_c()), room, req)
        b.step(3)                                   # the next room arrives while this one runs
    b.step(100)
    assert len(b.poll()) == 3
    for slot, room, req in slots.values():
        g = native.room_grid(room, precision="fp32")
        g.step(req["steps"], reduce_every=1)
        for n in ("u", "v", "w", "c", "p"):
            assert np.array_equal(b.grid(slot).read_field(n), g.read_field(n))
        g.close()
    b.close()


def test_budget_defers_admission(torch):
    reqs = small_trace(n=5, seed=3)
    biggest = max(native.grid_bytes(native.room_desc(rooms.request_room(r), history_capacity=max(16, r["steps"])))
                  for r in reqs)
    srv = serve.Server(hbm_budget_bytes=biggest + 1, max_slots=4, chunk_steps=5)
    results = srv.run(reqs, realtime=False)
    srv.close()
    assert len(results) == len(reqs)
    summ = serve.summarize(results)
    assert summ["p99_latency_s"] >= summ["p50_latency_s"] > 0
