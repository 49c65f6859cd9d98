"""Launch tiles (z-chunks per kernel family) and the autotuner.

A tile changes how the stencil kernels are split into CTAs, never what a cell computes: the fields after any
number of steps are bitwise the same under every tiling, including chunks that leave a ragged last chunk along z
and chunks larger than nz.  The reductions are summed per CTA, so only their last bits may follow the filter's
chunk; the histogram is exact.  The autotuner writes scratch arrays only and its choice is cached per shape; on the
generic FFT path it also picks the FFT radix schedules, which change the rounding order only."""
import numpy as np
import pytest

from oracle import flow as F
from paper_2204_02107_gb300 import native, rooms
from gpu_helpers import FIELD_NAMES, field_errors, gpu_grid, load_state, read_state, rel_l2, require_gpu
from gpu_helpers import room_case as oracle_case

pytestmark = pytest.mark.gpu

ALL = FIELD_NAMES + ("p",)
DEFAULT = {"zc_stage": 4, "zc_div": 32, "zc_project": 8, "zc_filter": 16, "fft_x": 0, "fft_y": 0, "fft_z": 0}
ZC = ("zc_stage", "zc_div", "zc_project", "zc_filter")
# Reductions under another filter chunk are summed in another order.  FP32: the kinetic energy is a plain float sum
# of at most 64 non-negative terms per thread before the float-float and FP64 stages, so its relative change is
# below 64 * 2^-24 < 4e-6; the scalar inventories are compensated (float-float) sums, good to ~2^-44 of the sum.
# FP64: plain double sums, ~64 * 2^-53 per thread.
REL = {"fp32": {"ke": 4e-6, "c_total": 1e-10, "c_room": 1e-10, "c2_room": 1e-10},
       "fp64": {"ke": 1e-12, "c_total": 1e-12, "c_room": 1e-12, "c2_room": 1e-12}}
TILINGS = [(4, 4, 4, 4), (8, 8, 8, 16), (16, 32, 4, 8), (32, 16, 32, 32), (64, 64, 64, 64), (12, 20, 36, 5)]


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


BOXES = [(14, 20, 6, 12, 2, 9), (30, 36, 10, 18, 4, 12)]


def room_case():
    # nz = 20: chunks 8, 12, 16, 36 leave a ragged last chunk; 32 and 64 exceed nz
    return rooms.make_room(48, 24, 20, h=0.05, boxes=BOXES, u_in=0.8)


def run(room, precision, tiles, steps=12):
    g = native.room_grid(room, precision=precision)
    if tiles is not None:
        g.set_tiles(*tiles)
    g.step(steps, reduce_every=1)
    out = {n: g.read_field(n) for n in ALL}
    hist = g.history()
    g.close()
    return out, hist


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_fields_bitwise_under_every_tiling(torch, precision):
    room = room_case()
    ref, ref_hist = run(room, precision, (8, 8, 8, 16))
    for tiles in TILINGS:
        out, hist = run(room, precision, tiles)
        for n in ALL:
            assert np.array_equal(out[n], ref[n]), (tiles, n)
        assert len(hist) == len(ref_hist)
        for a, b in zip(hist, ref_hist):
            assert a["step"] == b["step"] and np.array_equal(a["hist"], b["hist"])
            assert a["hist_under"] == b["hist_under"] and a["hist_over"] == b["hist_over"]
            for key, rel in REL[precision].items():
                assert a[key] == pytest.approx(b[key], rel=rel, abs=1e-300), (tiles, key)
            assert a["v_room"] == b["v_room"]         # a count of cells times the cell volume
            assert a["div_max"] == b["div_max"] and a["u_max"] == b["u_max"]


def test_small_tiles_against_oracle_fp64(torch):
    """The smallest and largest chunks, FP64, against the oracle over 20 steps."""
    room, prm, geom, st0 = oracle_case(48, 24, 20, boxes=BOXES, u_in=0.8)
    ref, _ = F.run(st0.copy(), geom, prm, 20)
    for tiles in [(4, 4, 4, 4), (64, 64, 64, 64)]:
        g = gpu_grid(prm, room.beta, room.S, room.room, "fp64")
        load_state(g, st0, prm)
        g.set_tiles(*tiles)
        g.step(20)
        errs = field_errors(read_state(g, prm), ref)
        g.close()
        assert max(errs.values()) <= 1e-11, (tiles, errs)


def test_set_tiles_rejects_out_of_range(torch):
    room = room_case()
    g = native.room_grid(room, precision="fp32")
    before = g.tiles()
    for bad in [(3, 8, 8, 16), (8, 65, 8, 16), (8, 8, 0, 16), (8, 8, 8, -4)]:
        with pytest.raises(native.VentflowError) as ei:
            g.set_tiles(*bad)
        assert ei.value.code == native.VF_EINVAL
        assert g.tiles() == before
    g.step(2)            # still usable
    g.sync()
    g.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_autotune_keeps_state_and_caches_choice(torch, precision):
    native.tile_cache_clear()
    room = room_case()
    g = native.room_grid(room, precision=precision)
    g.step(5, reduce_every=1)
    before = {n: g.read_field(n) for n in ALL}
    hist_before = g.history()
    info_before = g.info()
    chosen = g.autotune(reps=3)
    assert {chosen[k] for k in ZC} <= {4, 8, 16, 32}
    assert g.tiles() == chosen
    assert native.tile_cache_lookup(room.nx, room.ny, room.nz, precision) == chosen
    for n in ALL:
        assert np.array_equal(g.read_field(n), before[n]), n
    assert g.info()["step"] == info_before["step"] and g.info()["t"] == info_before["t"]
    hist_after = g.history()
    assert len(hist_after) == len(hist_before)
    assert [h["ke"] for h in hist_after] == [h["ke"] for h in hist_before]
    # stepping on: the same fields as a grid that never autotuned and switches to the chosen FFT schedules after
    # the same 5 steps (the z-chunks change no field value; another FFT schedule only the rounding order)
    g.step(7, reduce_every=1)
    tuned = {n: g.read_field(n) for n in ALL}
    g.close()
    native.tile_cache_clear()
    g2 = native.room_grid(room, precision=precision)
    g2.step(5, reduce_every=1)
    g2.set_tiles(8, 8, 8, 16, chosen["fft_x"], chosen["fft_y"], chosen["fft_z"])
    g2.step(7, reduce_every=1)
    for n in ALL:
        assert np.array_equal(g2.read_field(n), tuned[n]), n
    g2.close()
    untuned, _ = run(room, precision, None, steps=12)
    for n in ALL:
        assert rel_l2(tuned[n], untuned[n]) < (1e-12 if precision == "fp64" else 1e-5), n


def test_new_grid_takes_cached_tiles(torch):
    native.tile_cache_clear()
    room = room_case()
    g = native.room_grid(room, precision="fp32")
    assert g.tiles() == DEFAULT
    chosen = g.autotune(reps=2)
    g.close()
    g2 = native.room_grid(room, precision="fp32")
    assert g2.tiles() == chosen
    g2.close()
    g3 = native.room_grid(room, precision="fp64")        # another precision: not cached
    assert g3.tiles() == DEFAULT
    g3.close()
    native.tile_cache_clear()
    assert native.tile_cache_lookup(room.nx, room.ny, room.nz, "fp32") is None


def test_batch_autotunes_on_admission_and_matches_alone(torch):
    native.tile_cache_clear()
    cases = [(rooms.make_room(40, 24, 20, h=0.05, boxes=[(12, 16, 6, 10, 2, 8)], u_in=1.0), 9),
             (rooms.make_room(32, 32, 16, h=0.05, u_in=0.7), 6)]
    b = native.Batch(max_slots=3, hbm_budget_bytes=4 << 30, reduce_every=1, autotune=2)
    slots = []
    for room, steps in cases:
        slots.append(b.add(native.room_desc(room), room.beta, room.S, (room.u_in, 0, 0), 0.0, steps,
                           room=room.room, c0=room.initial_c()))
        assert native.tile_cache_lookup(room.nx, room.ny, room.nz, "fp32") is not None
    b.step(50)
    assert sorted(b.poll()) == sorted(slots)
    for (room, steps), slot in zip(cases, slots):
        g = native.room_grid(room, precision="fp32")      # takes the cached tiles, as the room in the batch did
        assert g.tiles() == b.grid(slot).tiles()
        g.step(steps, reduce_every=1)
        for n in ALL:
            assert np.array_equal(g.read_field(n), b.grid(slot).read_field(n)), n
        assert g.history()[-1]["ke"] == b.grid(slot).history()[-1]["ke"]
        g.close()
    b.close()
    native.tile_cache_clear()
