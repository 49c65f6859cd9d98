"""Scalar budget of the step on the GPU (Eqs. 3-4 in flux form, the room inventory of Sec. 3.3).

Every record vf_step writes carries the RK4-weighted forcing inventory (all fluid cells and the room cells), the
scalar that leaves the room through its openings, the scalar the re-mask after the filter removes from solids and
the filter's change of the room inventory.  These are compared with the oracle's budget of the same steps, and
the GPU's own records must close: the change of the total inventory equals forcing minus mask loss, the change of
the room inventory equals room forcing minus outflow plus the filter's room change.
"""
import numpy as np
import pytest

from oracle import flow as F
from gpu_helpers import gpu_grid, load_state, require_gpu, room_case

pytestmark = pytest.mark.gpu

TERMS = (("budget_forcing", "forcing"), ("budget_forcing_room", "forcing_room"), ("budget_outflow", "outflow"),
         ("budget_mask_loss", "mask_loss"), ("budget_filter_room", "filter_room"))


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def closure(prev, rec):
    """Residuals of the two balances between consecutive records (scaled by nothing: c m^3)."""
    total = rec["c_total"] - prev["c_total"] - (rec["budget_forcing"] - rec["budget_mask_loss"])
    room = rec["c_room"] - prev["c_room"] - (rec["budget_forcing_room"] - rec["budget_outflow"]
                                             + rec["budget_filter_room"])
    return total, room


def run_both(torch, precision, room_with_inlet=False, filter=True, steps=6):
    room, prm, geom, st0 = room_case(48, 30, 18, boxes=[(20, 26, 12, 20, 2, 9), (30, 34, 4, 8, 2, 5)], seed=11,
                                     filter=filter)
    region = np.maximum(room.room, room.S) if room_with_inlet else room.room
    geom = F.Geometry(room.beta, room.S, region)
    if precision == "fp32":
        st0 = F.State(*(getattr(st0, n).astype(np.float32).astype(np.float64) for n in ("u", "v", "w", "c")),
                      np.zeros(prm.shape), 0.0, 0)
    rec0 = F.reductions(st0, geom, prm)
    _, recs = F.run(st0.copy(), geom, prm, steps, with_budget=True)
    g = gpu_grid(prm, room.beta, room.S, region, precision)
    load_state(g, st0, prm, as_fp32=(precision == "fp32"))
    g.step(steps, reduce_every=1)
    hist = g.history()
    g.close()
    assert len(hist) == steps
    return rec0, recs, hist


@pytest.mark.parametrize("room_with_inlet", [False, True])
def test_budget_fp64_matches_oracle_and_closes(torch, room_with_inlet):
    rec0, recs, hist = run_both(torch, "fp64", room_with_inlet=room_with_inlet)
    scale = rec0["c_total"]
    for want, got in zip(recs, hist):
        for key, okey in TERMS:
            assert got[key] == pytest.approx(want[okey], rel=1e-10, abs=1e-13 * scale), key
    assert abs(hist[-1]["budget_outflow"]) > 1e-6 * scale       # the jet carries scalar out of the room
    assert abs(hist[-1]["budget_forcing"]) > 1e-6 * scale
    assert hist[-1]["budget_mask_loss"] != 0.0 and hist[-1]["budget_filter_room"] != 0.0
    assert (hist[-1]["budget_forcing_room"] != 0.0) == room_with_inlet
    prev = {"c_total": rec0["c_total"], "c_room": rec0["c_room"]}
    for rec in hist:
        total, room = closure(prev, rec)
        assert abs(total) < 1e-12 * scale and abs(room) < 1e-12 * scale, (total, room)
        prev = rec


def test_budget_fp64_filter_off(torch):
    """filter off: the standalone reduction carries the stage terms; nothing is lost to the re-mask"""
    rec0, recs, hist = run_both(torch, "fp64", filter=False, steps=3)
    scale = rec0["c_total"]
    for want, got in zip(recs, hist):
        for key, okey in TERMS:
            assert got[key] == pytest.approx(want[okey], rel=1e-10, abs=1e-13 * scale), key
        assert got["budget_mask_loss"] == 0.0 and got["budget_filter_room"] == 0.0
    prev = {"c_total": rec0["c_total"], "c_room": rec0["c_room"]}
    for rec in hist:
        total, room = closure(prev, rec)
        assert abs(total) < 1e-12 * scale and abs(room) < 1e-12 * scale
        prev = rec


def test_budget_fp32(torch):
    """FP32 fields with FP64 reductions: the budget terms within the FP32 field error of the oracle's, and the
    records close to the float rounding of the inventories"""
    rec0, recs, hist = run_both(torch, "fp32", room_with_inlet=True)
    scale = rec0["c_total"]
    for want, got in zip(recs, hist):
        for key, okey in TERMS:
            assert got[key] == pytest.approx(want[okey], rel=1e-4, abs=1e-7 * scale), key
    prev = {"c_total": rec0["c_total"], "c_room": rec0["c_room"]}
    for rec in hist:
        total, room = closure(prev, rec)
        assert abs(total) < 1e-6 * scale and abs(room) < 1e-6 * scale, (total, room)
        prev = rec


def test_budget_records_only_on_recorded_steps(torch):
    """on-demand reductions carry no step budget; a step without a record leaves the next record's terms its own"""
    room, prm, geom, st0 = room_case(40, 24, 20, boxes=[(12, 16, 6, 10, 2, 8)], seed=5)
    _, recs = F.run(st0.copy(), geom, prm, 4, with_budget=True)
    g = gpu_grid(prm, room.beta, room.S, room.room, "fp64")
    load_state(g, st0, prm)
    assert all(g.reductions()[k] == 0.0 for k, _ in TERMS)
    g.step(4, reduce_every=2)
    hist = g.history()
    g.close()
    assert [h["step"] for h in hist] == [2, 4]
    for want, got in zip((recs[1], recs[3]), hist):
        for key, okey in TERMS:
            assert got[key] == pytest.approx(want[okey], rel=1e-10, abs=1e-13 * recs[0]["c_total"]), key
