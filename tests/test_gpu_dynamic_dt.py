"""Dynamic time step (Sec. 2.4, AdjustDt: the user sets the maximum Courant number).

The device chooses dt = min(dt_max, courant_max / sigma) before every step from the Courant rate of the state the
step starts from; the tests compare fields, the dt sequence and the time with the oracle's adaptive run, check that
a cap that never binds gives the fixed-dt run bitwise, and that graphs, restarts and batches keep the arithmetic."""
import numpy as np
import pytest

from oracle import flow as F
from paper_2204_02107_gb300 import native
from gpu_helpers import FIELD_NAMES, field_errors, gpu_grid, load_state, read_state, require_gpu, room_case

pytestmark = pytest.mark.gpu

FP64_BAR = 1e-11
FP32_BAR = 1e-5
CMAX = 0.3


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


CASES = [((48, 30, 18), [(20, 26, 12, 20, 2, 9)]),               # generic FFT passes
         ((64, 32, 32), [(20, 26, 8, 14, 2, 12)])]                # register FFT passes


@pytest.mark.parametrize("shape,boxes", CASES)
def test_adaptive_fp64_vs_oracle(torch, shape, boxes):
    room, prm, geom, st0 = room_case(*shape, boxes=boxes, seed=5)
    ref, recs, dt_last = F.run_adaptive(st0.copy(), geom, prm, 40, CMAX)
    dts = [r["dt"] for r in recs]
    assert min(dts) < prm.dt and len(set(dts)) > 10          # the limit binds and moves
    g = gpu_grid(prm, room.beta, room.S, room.room, "fp64", courant_max=CMAX)
    load_state(g, st0, prm)
    g.step(40, reduce_every=1)
    errs = field_errors(read_state(g, prm.with_(dt=dt_last)), ref)
    assert max(errs.values()) < FP64_BAR, errs
    hist = g.history()
    assert len(hist) == 40
    for h, r in zip(hist, recs):
        assert h["dt"] == pytest.approx(r["dt"], rel=1e-13)
        assert h["t"] == pytest.approx(r["t"], rel=1e-13)
        assert h["ke"] == pytest.approx(r["ke"], rel=1e-10)
    assert g.info()["t"] == pytest.approx(recs[-1]["t"], rel=1e-13)
    g.close()


def test_adaptive_fp32_one_step(torch):
    room, prm, geom, st0 = room_case(64, 32, 32, boxes=[(20, 26, 8, 14, 2, 12)], seed=8)
    st32 = F.State(*(getattr(st0, n).astype(np.float32).astype(np.float64) for n in ("u", "v", "w", "c")),
                   np.zeros(prm.shape), 0.0, 0)
    ref, recs, dt_last = F.run_adaptive(st32.copy(), geom, prm, 1, CMAX)
    assert recs[0]["dt"] < prm.dt
    g = gpu_grid(prm, room.beta, room.S, room.room, "fp32", courant_max=CMAX)
    load_state(g, st32, prm, as_fp32=True)
    g.step(1, reduce_every=1)
    errs = field_errors(read_state(g, prm.with_(dt=dt_last)), ref)
    assert max(errs.values()) < FP32_BAR, errs
    assert g.history()[-1]["dt"] == pytest.approx(recs[0]["dt"], rel=1e-6)
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cap_that_never_binds_is_the_fixed_run(torch, precision):
    """With a Courant limit far above the flow's, every step takes dt_max; the device computes the dt constants
    with the host's formulas, so the fields are bitwise those of the fixed-dt grid."""
    room, prm, geom, st0 = room_case(40, 24, 20, boxes=[(12, 16, 6, 10, 2, 8)], seed=2)
    out = {}
    for cm in (0.0, 1e9):
        g = gpu_grid(prm, room.beta, room.S, room.room, precision, courant_max=cm)
        load_state(g, st0, prm, as_fp32=precision == "fp32")
        g.step(12, reduce_every=1)
        out[cm] = {n: g.read_field(n) for n in FIELD_NAMES + ("p",)}
        if cm > 0:
            assert all(h["dt"] == prm.dt for h in g.history())
        g.close()
    for n in FIELD_NAMES + ("p",):
        assert np.array_equal(out[0.0][n], out[1e9][n]), n


def test_graph_and_direct_launch_identical(torch, monkeypatch):
    room, prm, geom, st0 = room_case(40, 24, 20, boxes=[(12, 16, 6, 10, 2, 8)], seed=6)
    out = {}
    for mode in ("graph", "direct"):
        if mode == "direct":
            monkeypatch.setenv("VF_NO_GRAPH", "1")
        g = gpu_grid(prm, room.beta, room.S, room.room, "fp32", courant_max=CMAX)
        load_state(g, st0, prm, as_fp32=True)
        g.step(15, reduce_every=3)
        out[mode] = ({n: g.read_field(n) for n in FIELD_NAMES + ("p",)}, [h["dt"] for h in g.history()])
        g.close()
    for n in FIELD_NAMES + ("p",):
        assert np.array_equal(out["graph"][0][n], out["direct"][0][n]), n
    assert out["graph"][1] == out["direct"][1]


def test_restart_bitwise(torch):
    """Save after 6 adaptive steps, restore into a new grid (its Courant rate is recomputed from the restored
    fields), 6 more steps: bitwise the 12-step run, and the same time."""
    room, prm, geom, st0 = room_case(40, 24, 20, boxes=[(12, 16, 6, 10, 2, 8)], seed=4)
    g = gpu_grid(prm, room.beta, room.S, room.room, "fp64", courant_max=CMAX)
    load_state(g, st0, prm)
    g.step(12)
    full = {n: g.read_field(n) for n in FIELD_NAMES + ("p",)}
    t_full = g.info()["t"]
    g.close()
    g1 = gpu_grid(prm, room.beta, room.S, room.room, "fp64", courant_max=CMAX)
    load_state(g1, st0, prm)
    g1.step(6)
    saved = {n: g1.read_field(n) for n in FIELD_NAMES + ("p",)}
    info = g1.info()
    g1.close()
    g2 = gpu_grid(prm, room.beta, room.S, room.room, "fp64", courant_max=CMAX)
    for n, a in saved.items():
        g2.set_field(n, a)
    g2.set_time(info["t"], info["step"])
    g2.step(6)
    for n in FIELD_NAMES + ("p",):
        assert np.array_equal(g2.read_field(n), full[n]), n
    assert g2.info()["t"] == t_full and g2.info()["step"] == 12
    g2.close()


def test_time_is_the_sum_of_the_steps(torch):
    room, prm, geom, st0 = room_case(32, 32, 16, seed=9)
    g = gpu_grid(prm, room.beta, room.S, room.room, "fp32", courant_max=CMAX)
    load_state(g, st0, prm, as_fp32=True)
    g.step(20, reduce_every=1)
    hist = g.history()
    t = 0.0
    for h in hist:
        t += h["dt"]
        assert h["t"] == t
    assert g.info()["t"] == t
    g.close()


def test_room_in_batch_equals_alone(torch):
    """A room starting at rest: dt_max until the inflow jet makes the Courant limit (0.1) bind."""
    room, prm, geom, st0 = room_case(40, 24, 20, boxes=[(12, 16, 6, 10, 2, 8)])
    cmax = 0.1
    desc = native.room_desc(room, precision="fp32", courant_max=cmax)
    b = native.Batch(max_slots=2, hbm_budget_bytes=2 << 30, reduce_every=1)
    slot = b.add(desc, room.beta, room.S, (room.u_in, 0, 0), 0.0, 25, room=room.room, c0=room.initial_c())
    b.step(40)
    assert b.poll() == [slot]
    g = native.room_grid(room, precision="fp32", courant_max=cmax)
    g.step(25, reduce_every=1)
    for n in FIELD_NAMES + ("p",):
        assert np.array_equal(b.grid(slot).read_field(n), g.read_field(n)), n
    dts = [h["dt"] for h in g.history()]
    assert [h["dt"] for h in b.grid(slot).history()] == dts
    assert dts[0] == prm.dt and min(dts) < prm.dt
    g.close()
    b.close()
