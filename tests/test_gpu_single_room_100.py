"""FP64 parity of the full-size single room over 100 steps, at the benchmark's launch configuration.

The 256 x 128 x 128 room (10 x 5 x 5 m, 2-cell walls, one duct pair, U_in = 1 m/s, filter on, 4 pressure
iterations) starts from rest with stale air.  The oracle's state after 100 steps is stored at 8 k sampled cells (a
seeded draw over the room plus the inlet jet's region) with its full-field norms and last record, by
``tests/golden/make_single_room_fp64_100.py``, which calls only the oracle: about ten minutes of host time that a
GPU run does not repeat.  The GPU runs the same 100 steps through the C ABI and must match within 1e-11 relative
L2 on the sample of every field, and its last record and scalar budget the oracle's.
"""
import os

import numpy as np
import pytest

from oracle import flow as F
from paper_2204_02107_gb300 import native, rooms
from gpu_helpers import gpu_grid, load_state, require_gpu

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "single_room_fp64_100.npz")
FP64_BAR = 1e-11


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def test_single_room_fp64_100_steps(torch):
    ref = np.load(GOLDEN)
    steps = int(ref["steps"])
    room = rooms.single_room(256, 128, 128)
    prm = F.Params(nx=room.nx, ny=room.ny, nz=room.nz, lx=room.lx, ly=room.ly, lz=room.lz, nu=rooms.NU_AIR,
                   dt=room.dt, u_set=(room.u_in, 0.0, 0.0), c_set=0.0, filter=True, n_pressure_iters=4)
    g = gpu_grid(prm, room.beta, room.S, room.room, "fp64")
    load_state(g, F.zero_state(prm, c=room.initial_c()), prm)
    g.step(steps, reduce_every=steps)
    idx = ref["idx"]
    for name in ("u", "v", "w", "c", "p"):
        full = g.read_field(name)
        got = full.ravel()[idx]
        want = ref[name]
        err = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert err < FP64_BAR, (name, err)
        assert abs(np.linalg.norm(full) - float(ref[name + "_norm"])) < FP64_BAR * float(ref[name + "_norm"]), name
    assert np.max(np.abs(ref["u"])) > 0.5                 # the inlet jet is in the sample
    last = g.history()[-1]
    g.close()
    assert last["step"] == steps
    for key in ("ke", "c_total", "c_room", "c2_room", "v_room", "u_max", "div_l2"):
        assert last[key] == pytest.approx(float(ref["rec_" + key]), rel=1e-10), key
    scale = float(ref["rec_c_total"])
    for key, okey in (("budget_forcing", "forcing"), ("budget_forcing_room", "forcing_room"),
                      ("budget_outflow", "outflow"), ("budget_mask_loss", "mask_loss"),
                      ("budget_filter_room", "filter_room")):
        assert last[key] == pytest.approx(float(ref["rec_" + okey]), rel=1e-9, abs=1e-13 * scale), key
