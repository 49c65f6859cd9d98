"""Parity at the benchmark's full size and launch configuration: the 256 x 128 x 128 room, one step from a masked
random state that is exactly representable in float, through the FP64 path (1e-11) and the FP32 path (1e-5),
against one oracle step.  Also host-side fault injection: a failing allocation is reported, not hidden."""
import numpy as np
import pytest

from oracle import flow as F
from paper_2204_02107_gb300 import native, rooms
from gpu_helpers import FIELD_NAMES, field_errors, gpu_grid, load_state, read_state, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def test_single_room_full_size_one_step(torch):
    room = rooms.single_room(256, 128, 128)
    prm = F.Params(nx=room.nx, ny=room.ny, nz=room.nz, lx=room.lx, ly=room.ly, lz=room.lz, nu=rooms.NU_AIR,
                   dt=room.dt, u_set=(room.u_in, 0.0, 0.0), c_set=0.0, filter=True, n_pressure_iters=4)
    geom = F.Geometry(room.beta, room.S, room.room)
    u, v, w = rooms.random_fields(prm.shape, 23, count=3, scale=0.3, beta=room.beta)
    f32 = lambda a: a.astype(np.float32).astype(np.float64)
    st = F.State(f32(u), f32(v), f32(w), f32(room.initial_c()), np.zeros(prm.shape))
    ref, rec = F.step(st.copy(), geom, prm)
    for precision, bar in (("fp64", 1e-11), ("fp32", 1e-5)):
        g = gpu_grid(prm, room.beta, room.S, room.room, precision)
        load_state(g, st, prm, as_fp32=(precision == "fp32"))
        g.step(1, reduce_every=1)
        out = read_state(g, prm)
        errs = field_errors(out, ref)
        assert max(errs.values()) < bar, (precision, errs)
        last = g.history()[-1]
        for key in ("ke", "c_room", "c2_room", "v_room", "c_total"):
            assert last[key] == pytest.approx(rec[key], rel=bar * 10), (precision, key)
        if precision == "fp64":
            assert list(last["hist"]) == list(rec["hist"])
        solid = room.beta == 0
        for n in FIELD_NAMES:
            assert np.all(getattr(out, n)[solid] == 0.0)
        g.close()


def test_allocation_failure_is_reported(torch, monkeypatch):
    """Inject a failure at the n-th device allocation of a grid (host-side): vf_create_grid returns VF_ENOMEM and
    leaves nothing behind; the next grid works."""
    room = rooms.make_room(40, 24, 20, h=0.05)
    for n in (1, 5, 23):
        monkeypatch.setenv("VF_FAULT_ALLOC_AT", str(n))
        with pytest.raises(native.VentflowError) as ei:
            native.room_grid(room, precision="fp32")
        assert ei.value.code == native.VF_ENOMEM
    monkeypatch.delenv("VF_FAULT_ALLOC_AT")
    g = native.room_grid(room, precision="fp32")
    g.step(2)
    g.sync()
    g.close()


def test_step_before_mask_is_a_state_error(torch):
    g = native.Grid(16, 16, 16, 1.0, 1.0, 1.0, nu=1e-3, dt=1e-3)
    with pytest.raises(native.VentflowError) as ei:
        g.step(1)
    assert ei.value.code == native.VF_ESTATE
    g.close()
