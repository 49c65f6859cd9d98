"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: FP64 path within 1e-11 relative L2 per field after 100 steps; FP32 path (FP32 fields, FP64 reductions)
within 1e-5 relative L2 per field for one step from an identical state; masking and histogram counts exact.
Sizes span several 32 x 8 x 16 CTA tiles with ragged tails and every FFT radix (2, 3, 4, 5, 8).
"""
import math

import numpy as np
import pytest

from oracle import flow as F
from paper_2204_02107_gb300 import native, rooms
from gpu_helpers import (FIELD_NAMES, field_errors, gpu_grid, load_state, read_state, rel_l2, require_gpu,
                         room_case)

pytestmark = pytest.mark.gpu

FP64_BAR = 1e-11
FP32_BAR = 1e-5


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def test_taylor_green_fp64_100_steps(torch):
    """Config: Taylor-Green 32^3 on [0, 2 pi)^3, nu = 0.01, dt = 1e-3, 100 steps, FP64, no mask, filter off."""
    n = 32
    prm = F.Params(nx=n, ny=n, nz=n, lx=2 * math.pi, ly=2 * math.pi, lz=2 * math.pi, nu=0.01, dt=1e-3,
                   filter=False, n_pressure_iters=1)
    u, v, w = rooms.taylor_green(n)
    st0 = F.State(u, v, w, np.zeros(prm.shape), np.zeros(prm.shape))
    geom = F.open_geometry(prm)
    ref, recs = F.run(st0.copy(), geom, prm, 100)
    g = gpu_grid(prm, np.ones(prm.shape), np.zeros(prm.shape), np.ones(prm.shape), "fp64")
    load_state(g, st0, prm)
    e0 = g.reductions()["ke"]
    g.step(100, reduce_every=1)
    out = read_state(g, prm)
    errs = field_errors(out, ref)
    assert max(errs.values()) < FP64_BAR, errs
    hist = g.history()
    assert len(hist) == 100 and hist[-1]["step"] == 100
    amp = math.sqrt(hist[-1]["ke"] / e0)
    assert abs(amp - math.exp(-3 * prm.nu * 0.1)) / math.exp(-3 * prm.nu * 0.1) < 1e-4
    assert max(r["div_max"] for r in hist) < 1e-12
    assert hist[-1]["ke"] == pytest.approx(recs[-1]["ke"], rel=1e-12)
    g.close()


@pytest.mark.parametrize("fft_path", ["plane", "tile"])
@pytest.mark.parametrize("shape,boxes", [
    ((40, 24, 20), [(12, 16, 6, 10, 2, 8)]),
    ((48, 30, 18), [(20, 26, 12, 20, 2, 9), (30, 34, 4, 8, 2, 5)]),
    ((64, 32, 32), [(20, 26, 8, 14, 2, 12), (40, 46, 18, 26, 2, 9)]),   # register FFT path on the plane layout
])
def test_masked_room_fp64_100_steps(torch, monkeypatch, shape, boxes, fft_path):
    """Walls, inlet/outlet duct, boxes, forcing, filter, 4 pressure iterations: 100 steps vs the oracle, with the
    y-z transforms done per kx plane in shared memory or as separate tile passes."""
    if fft_path == "tile":
        monkeypatch.setenv("VF_TILE_FFT", "1")
    room, prm, geom, st0 = room_case(*shape, boxes=boxes)
    ref, recs = F.run(st0.copy(), geom, prm, 100)
    g = gpu_grid(prm, room.beta, room.S, room.room, "fp64")
    load_state(g, st0, prm)
    g.step(100, reduce_every=10)
    out = read_state(g, prm)
    errs = field_errors(out, ref)
    assert max(errs.values()) < FP64_BAR, errs
    assert np.max(np.abs(out.u)) > 0.5          # the inflow jet is there
    solid = room.beta == 0
    for n in FIELD_NAMES:
        assert np.all(getattr(out, n)[solid] == 0.0)
    hist = g.history()
    assert [h["step"] for h in hist] == list(range(10, 101, 10))
    last = hist[-1]
    for key in ("ke", "c_total", "c_room", "c2_room", "v_room", "div_l2", "div_max", "u_max"):
        assert last[key] == pytest.approx(recs[-1][key], rel=1e-10, abs=1e-300), key
    g.close()


@pytest.mark.parametrize("shape", [(40, 24, 20), (64, 36, 30), (64, 32, 32), (72, 36, 36), (96, 48, 48),
                                   (80, 40, 40)])
def test_fp32_one_step_from_identical_state(torch, shape):
    """FP32 bulk: one step from a state that is exactly representable in float, compared with the oracle (the
    last three shapes on the register FFT's 2-3-5 lengths: 9 x 4, 12 x 4 and 20 x 2 points)."""
    room, prm, geom, st0 = room_case(*shape, boxes=[(10, 14, 6, 12, 2, 8)], seed=17)
    st, _ = F.run(st0, geom, prm, 3)
    st32 = F.State(*(getattr(st, n).astype(np.float32).astype(np.float64) for n in ("u", "v", "w", "c")),
                   (st.p / prm.dt).astype(np.float32).astype(np.float64) * prm.dt, st.t, st.step)
    ref, rec = F.step(st32.copy(), geom, prm)
    g = gpu_grid(prm, room.beta, room.S, room.room, "fp32")
    if shape[1] == shape[2] and shape[1] in (36, 48, 40):
        assert g.fft_path() == "register_plane"
    load_state(g, st32, prm, as_fp32=True)
    g.step(1)
    out = read_state(g, prm)
    errs = field_errors(out, ref)
    assert max(errs.values()) < FP32_BAR, errs
    red = g.reductions()
    for key in ("ke", "c_total", "c_room", "c2_room", "v_room"):
        assert red[key] == pytest.approx(rec[key], rel=1e-5), key
    g.close()


@pytest.mark.parametrize("fft_path", ["plane", "tile"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", [(8, 8, 8), (10, 12, 16), (20, 30, 18), (40, 10, 50), (72, 36, 20), (256, 8, 8),
                                   (16, 128, 128)])
def test_poisson_solve_matches_oracle(torch, monkeypatch, precision, shape, fft_path):
    """vf_poisson_solve (forward 3D FFT, division by lambda, inverse) against the oracle's numpy.fft solve, with
    the y-z transforms per kx plane or as tile passes (a 128 x 128 plane exceeds shared memory in FP64, so that
    case takes the tile path in both settings)."""
    if fft_path == "tile":
        monkeypatch.setenv("VF_TILE_FFT", "1")
    nx, ny, nz = shape
    prm = F.Params(nx=nx, ny=ny, nz=nz, lx=nx * 0.1, ly=ny * 0.07, lz=nz * 0.13, nu=0.0, dt=1.0)
    rng = np.random.default_rng(nx * 10007 + ny * 101 + nz)
    f = rng.standard_normal(prm.shape)
    ref = F.poisson_fft_solve(f, prm)
    g = native.Grid(nx, ny, nz, prm.lx, prm.ly, prm.lz, nu=0.0, dt=1.0, precision=precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    fd = torch.tensor(f, dtype=dt, device="cuda")
    pd = torch.empty_like(fd)
    g.poisson_solve(fd, pd)
    g.sync()
    got = pd.double().cpu().numpy()
    if precision == "fp32":
        ref = F.poisson_fft_solve(f.astype(np.float32).astype(np.float64), prm)
    err = rel_l2(got, ref)
    assert err < (1e-13 if precision == "fp64" else 2e-6), err
    g.close()


def test_reductions_and_histogram_exact(torch):
    """Reductions of a loaded state: sums to round-off, histogram counts exactly equal to the oracle's."""
    room, prm, geom, st0 = room_case(40, 24, 20, boxes=[(12, 16, 6, 10, 2, 8)], seed=5)
    rng = np.random.default_rng(9)
    c = rng.uniform(-0.1, 1.1, size=prm.shape) * room.beta
    st = F.State(st0.u, st0.v, st0.w, c, st0.p)
    ref = F.reductions(st, geom, prm)
    g = gpu_grid(prm, room.beta, room.S, room.room, "fp64")
    load_state(g, st, prm)
    red = g.reductions()
    assert list(red["hist"]) == list(ref["hist"])
    assert red["hist_under"] == ref["hist_under"] and red["hist_over"] == ref["hist_over"]
    for key in ("ke", "c_total", "c_room", "c2_room", "v_room", "div_l2", "div_max", "u_max"):
        assert red[key] == pytest.approx(ref[key], rel=1e-12), key
    g.close()
    g32 = gpu_grid(prm, room.beta, room.S, room.room, "fp32")
    st32 = F.State(*(getattr(st, n).astype(np.float32).astype(np.float64) for n in ("u", "v", "w", "c")), st.p)
    load_state(g32, st32, prm, as_fp32=True)
    red32 = g32.reductions()
    ref32 = F.reductions(st32, geom, prm)
    # float stencil of the divergence differs from the double one by float rounding; sums are compensated
    for key in ("ke", "c_total", "c_room", "c2_room", "v_room"):
        assert red32[key] == pytest.approx(ref32[key], rel=1e-7), key
    assert list(red32["hist"]) == list(ref32["hist"])
    g32.close()


def test_nonfinite_detected(torch):
    room, prm, geom, st0 = room_case(16, 16, 16, seed=3)
    g = gpu_grid(prm, room.beta, room.S, room.room, "fp32")
    u = st0.u.copy()
    u[5, 5, 5] = np.nan
    g.set_field("u", u)
    with pytest.raises(native.VentflowError) as ei:
        g.reductions()
    assert ei.value.code == native.VF_ENONFINITE
    g.close()


def test_graph_and_direct_launch_identical(torch, monkeypatch):
    """The captured CUDA graph replays exactly the launches of the direct path (bitwise equal results)."""
    room, prm, geom, st0 = room_case(40, 24, 20, boxes=[(12, 16, 6, 10, 2, 8)], seed=2)
    outs = []
    for no_graph in (False, True):
        if no_graph:
            monkeypatch.setenv("VF_NO_GRAPH", "1")
        g = gpu_grid(prm, room.beta, room.S, room.room, "fp32")
        load_state(g, st0, prm)
        g.step(7, reduce_every=3)
        outs.append((read_state(g, prm), g.history()))
        g.close()
    for n in FIELD_NAMES:
        assert np.array_equal(getattr(outs[0][0], n), getattr(outs[1][0], n))
    assert [h["ke"] for h in outs[0][1]] == [h["ke"] for h in outs[1][1]]


def test_restart_bitwise(torch):
    """Checkpoint/resume: 5 steps + save/restore + 5 steps equals 10 steps bitwise."""
    room, prm, geom, st0 = room_case(40, 24, 20, boxes=[(12, 16, 6, 10, 2, 8)], seed=4)
    g = gpu_grid(prm, room.beta, room.S, room.room, "fp64")
    load_state(g, st0, prm)
    g.step(10)
    full = read_state(g, prm)
    g.close()
    g1 = gpu_grid(prm, room.beta, room.S, room.room, "fp64")
    load_state(g1, st0, prm)
    g1.step(5)
    saved = {n: g1.read_field(n) for n in FIELD_NAMES + ("p",)}
    info = g1.info()
    g1.close()
    g2 = gpu_grid(prm, room.beta, room.S, room.room, "fp64")
    for n, a in saved.items():
        g2.set_field(n, a)
    g2.set_time(info["t"], info["step"])
    g2.step(5)
    out = read_state(g2, prm)
    for n in FIELD_NAMES:
        assert np.array_equal(getattr(out, n), getattr(full, n)), n
    assert g2.info()["step"] == 10
    g2.close()
