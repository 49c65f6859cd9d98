"""Smooth source mask of Eq. 5 on the GPU: the window is evaluated on the device and drives the forcing terms.

A room whose inlet is a tanh window instead of the binary patch is compared with the oracle (which builds the
window with its own Eq. 5 code) over 100 FP64 steps and one FP32 step; the same window passed as values gives the
same flow; returning to a binary region gives the binary run bitwise."""
import numpy as np
import pytest

from oracle import flow as F
from gpu_helpers import FIELD_NAMES, field_errors, gpu_grid, load_state, read_state, require_gpu, room_case

pytestmark = pytest.mark.gpu

FP64_BAR = 1e-11
FP32_BAR = 1e-5


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def window(room, prm):
    """Eq. 5 window over the inlet duct: centred between the two wall cells at x = 0, 1, over the duct in y, z."""
    h = prm.h
    ys, zs = np.nonzero(room.S.any(axis=2).T)           # duct cells (y, z)
    cy, cz = 0.5 * (ys.min() + ys.max()) * h[1], 0.5 * (zs.min() + zs.max()) * h[2]
    center = (0.5 * h[0], cy, cz)
    width = (3.0 * h[0], 5.0 * h[1], 5.0 * h[2])
    sharp = (2.0, 3.0, 3.0)
    return center, width, sharp


@pytest.mark.parametrize("shape,boxes", [((48, 30, 18), [(20, 26, 12, 20, 2, 9)]),
                                         ((64, 32, 32), [(20, 26, 8, 14, 2, 12)])])
def test_tanh_inlet_fp64_100_steps(torch, shape, boxes):
    room, prm, _, st0 = room_case(*shape, boxes=boxes)
    center, width, sharp = window(room, prm)
    S = F.tanh_source_mask(prm, center, width, sharp)
    geom = F.Geometry(room.beta, S, room.room)
    ref, recs = F.run(st0.copy(), geom, prm, 100)
    g = gpu_grid(prm, room.beta, room.S, room.room, "fp64")
    g.set_inflow_tanh(center, width, sharp, prm.u_set, prm.c_set)
    load_state(g, st0, prm)
    g.step(100, reduce_every=100)
    errs = field_errors(read_state(g, prm), ref)
    assert max(errs.values()) < FP64_BAR, errs
    assert np.max(np.abs(read_state(g, prm).u)) > 0.3          # the smooth jet is there
    last = g.history()[-1]
    assert last["c_total"] == pytest.approx(recs[-1]["c_total"], rel=1e-10)
    g.close()


def test_tanh_inlet_fp32_one_step(torch):
    room, prm, _, st0 = room_case(64, 32, 32, boxes=[(20, 26, 8, 14, 2, 12)], seed=3)
    center, width, sharp = window(room, prm)
    geom = F.Geometry(room.beta, F.tanh_source_mask(prm, center, width, sharp), room.room)
    st32 = F.State(*(getattr(st0, n).astype(np.float32).astype(np.float64) for n in ("u", "v", "w", "c")),
                   np.zeros(prm.shape), 0.0, 0)
    ref, _ = F.step(st32.copy(), geom, prm)
    g = gpu_grid(prm, room.beta, room.S, room.room, "fp32")
    g.set_inflow_tanh(center, width, sharp, prm.u_set, prm.c_set)
    load_state(g, st32, prm, as_fp32=True)
    g.step(1)
    errs = field_errors(read_state(g, prm), ref)
    assert max(errs.values()) < FP32_BAR, errs
    g.close()


def test_values_equal_device_window_and_binary_restores(torch):
    room, prm, _, st0 = room_case(40, 24, 20, boxes=[(12, 16, 6, 10, 2, 8)], seed=1)
    center, width, sharp = window(room, prm)
    S = F.tanh_source_mask(prm, center, width, sharp)
    out = {}
    for mode in ("tanh", "values", "binary_after", "binary"):
        g = gpu_grid(prm, room.beta, room.S, room.room, "fp64")
        if mode == "tanh":
            g.set_inflow_tanh(center, width, sharp, prm.u_set, prm.c_set)
        elif mode == "values":
            g.set_inflow_values(S, prm.u_set, prm.c_set)
        elif mode == "binary_after":
            g.set_inflow_tanh(center, width, sharp, prm.u_set, prm.c_set)
            g.set_inflow(room.S, prm.u_set, prm.c_set)
        load_state(g, st0, prm)
        g.step(20)
        out[mode] = {n: g.read_field(n) for n in FIELD_NAMES + ("p",)}
        g.close()
    for n in FIELD_NAMES + ("p",):
        a, b = out["tanh"][n], out["values"][n]
        assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.max(np.abs(b))), n
        assert np.array_equal(out["binary_after"][n], out["binary"][n]), n
