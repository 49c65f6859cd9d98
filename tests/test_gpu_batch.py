"""Batched rooms (vf_batch_*): rooms of uneven size advanced by one graph launch per batch step.

A room's fields must be bitwise identical alone (its own grid, vf_step) and in the mix; admission follows the
memory budget exactly (vf_grid_bytes equals what a grid allocates); finished rooms stop at their target step."""
import numpy as np
import pytest

from paper_2204_02107_gb300 import native, rooms
from gpu_helpers import FIELD_NAMES, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def case_rooms():
    return [
        (rooms.make_room(40, 24, 20, h=0.05, boxes=[(12, 16, 6, 10, 2, 8)], u_in=1.0), 9),
        (rooms.make_room(48, 30, 18, h=0.05, boxes=[(20, 26, 12, 20, 2, 9)], u_in=0.4), 6),
        (rooms.make_room(32, 32, 16, h=0.05, u_in=0.7), 12),
    ]


def alone(room, steps, precision):
    g = native.room_grid(room, precision=precision)
    g.step(steps, reduce_every=1)
    out = {n: g.read_field(n) for n in FIELD_NAMES + ("p",)}
    last = g.history()[-1] if steps else None
    g.close()
    return out, last


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_room_alone_equals_room_in_mix(torch, precision):
    cases = case_rooms()
    b = native.Batch(max_slots=4, hbm_budget_bytes=8 << 30, reduce_every=1)
    slots = []
    for room, steps in cases:
        desc = native.room_desc(room, precision=precision)
        slots.append(b.add(desc, room.beta, room.S, (room.u_in, 0, 0), 0.0, steps, room=room.room,
                           c0=room.initial_c()))
    b.step(100)           # more than any target: every room stops at its own step count
    done = sorted(b.poll())
    assert done == sorted(slots)
    info = b.info()
    assert info["done"] == 3 and info["active"] == 0 and info["batch_steps"] == max(s for _, s in cases)
    for (room, steps), slot in zip(cases, slots):
        ref, last = alone(room, steps, precision)
        g = b.grid(slot)
        assert g.info()["step"] == steps
        for n in FIELD_NAMES + ("p",):
            assert np.array_equal(g.read_field(n), ref[n]), (slot, n)
        rec = g.history()[-1]
        assert rec["step"] == steps and rec["ke"] == last["ke"] and list(rec["hist"]) == list(last["hist"])
    b.close()


def test_admission_by_budget_and_slot_reuse(torch):
    cases = case_rooms()
    descs = [native.room_desc(r, precision="fp32") for r, _ in cases]
    need = [native.grid_bytes(d) for d in descs]
    b = native.Batch(max_slots=2, hbm_budget_bytes=need[0] + need[1] - 1, reduce_every=0)
    r0, s0 = cases[0]
    slot0 = b.add(descs[0], r0.beta, r0.S, (r0.u_in, 0, 0), 0.0, s0)
    assert b.info()["bytes_in_use"] == need[0]
    r1, s1 = cases[1]
    with pytest.raises(native.VentflowError) as ei:
        b.add(descs[1], r1.beta, r1.S, (r1.u_in, 0, 0), 0.0, s1)
    assert ei.value.code == native.VF_ENOMEM
    assert b.info()["bytes_in_use"] == need[0]
    b.step(s0)
    assert b.poll() == [slot0]
    b.remove(slot0)
    assert b.info()["bytes_in_use"] == 0
    slot1 = b.add(descs[1], r1.beta, r1.S, (r1.u_in, 0, 0), 0.0, s1)
    b.step(s1)
    assert b.poll() == [slot1]
    b.close()


def test_grid_bytes_matches_allocation(torch):
    for room, _ in case_rooms():
        for precision in ("fp32", "fp64"):
            desc = native.room_desc(room, precision=precision)
            g = native.room_grid(room, precision=precision)
            assert g.info()["device_bytes"] == native.grid_bytes(desc)
            g.close()


def test_rooms_added_while_others_run(torch):
    """Continuous batching: a room admitted after others have started still matches its solo run bitwise."""
    cases = case_rooms()
    b = native.Batch(max_slots=3, hbm_budget_bytes=8 << 30, reduce_every=1)
    (ra, sa), (rb, sb) = cases[0], cases[2]
    slot_a = b.add(native.room_desc(ra), ra.beta, ra.S, (ra.u_in, 0, 0), 0.0, sa, room=ra.room, c0=ra.initial_c())
    b.step(4)
    slot_b = b.add(native.room_desc(rb), rb.beta, rb.S, (rb.u_in, 0, 0), 0.0, sb, room=rb.room, c0=rb.initial_c())
    b.step(50)
    assert sorted(b.poll()) == sorted([slot_a, slot_b])
    for (room, steps), slot in (((ra, sa), slot_a), ((rb, sb), slot_b)):
        ref, _ = alone(room, steps, "fp32")
        g = b.grid(slot)
        for n in FIELD_NAMES:
            assert np.array_equal(g.read_field(n), ref[n]), (slot, n)
    b.close()


def test_grids_created_large_then_small_both_run(torch):
    """Kernel shared-memory limits are process-wide: a smaller grid created later must not break a larger one."""
    big = rooms.make_room(64, 64, 64, h=0.05, u_in=1.0)
    small = rooms.make_room(40, 24, 20, h=0.05, u_in=1.0)
    g1 = native.room_grid(big, precision="fp64")
    g2 = native.room_grid(small, precision="fp32")
    g1.step(2)
    g2.step(2)
    g1.sync()
    g2.sync()
    assert g1.info()["step"] == 2 and np.isfinite(g1.read_field("u")).all()
    g1.close()
    g2.close()
