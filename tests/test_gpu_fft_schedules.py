"""Radix schedules of the generic FFT passes (Sec. 2.2's FFT Poisson solve) and their autotuning.

Every candidate schedule of every axis must give the oracle's numpy.fft solve (FP64 1e-13, FP32 2e-6 relative L2,
the bars of the other Poisson parity tests), with the (y, z) transforms per kx plane or as tile passes; a masked room
stepped with non-default schedules must stay within the FP64 parity bar after 100 steps; the autotuner must pick
valid schedules, cache them with the z-chunks, and a grid created later must take them (and step bitwise like the
tuned grid)."""
import numpy as np
import pytest

from oracle import flow as F
from paper_2204_02107_gb300 import native, rooms
from gpu_helpers import field_errors, gpu_grid, load_state, read_state, rel_l2, require_gpu, room_case

pytestmark = pytest.mark.gpu

# generic-path shapes (nx/2, ny, nz not all 16 x 2^k): lengths with 2, 3 and 5 factors in every axis
SHAPES = [(48, 40, 36), (80, 24, 20), (40, 72, 48)]


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def schedule_counts(shape):
    nx, ny, nz = shape
    return [len(native.fft_schedules(n)) for n in (nx // 2, ny, nz)]


@pytest.mark.parametrize("fft_path", ["plane", "tile"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", SHAPES)
def test_every_schedule_matches_oracle(torch, monkeypatch, precision, shape, fft_path):
    if fft_path == "tile":
        monkeypatch.setenv("VF_TILE_FFT", "1")
    nx, ny, nz = shape
    prm = F.Params(nx=nx, ny=ny, nz=nz, lx=nx * 0.1, ly=ny * 0.07, lz=nz * 0.13, nu=0.0, dt=1.0)
    rng = np.random.default_rng(nx * 131 + ny * 17 + nz)
    f = rng.standard_normal(prm.shape)
    if precision == "fp32":
        f = f.astype(np.float32).astype(np.float64)
    ref = F.poisson_fft_solve(f, prm)
    g = native.Grid(nx, ny, nz, prm.lx, prm.ly, prm.lz, nu=0.0, dt=1.0, precision=precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    fd = torch.tensor(f, dtype=dt, device="cuda")
    bar = 1e-13 if precision == "fp64" else 2e-6
    counts = schedule_counts(shape)
    assert max(counts) >= 3
    trials = [(0, 0, 0), tuple(c - 1 for c in counts)]
    for axis in range(3):
        for c in range(1, counts[axis]):
            idx = [0, 0, 0]
            idx[axis] = c
            trials.append(tuple(idx))
    for idx in trials:
        g.set_tiles(4, 32, 8, 16, *idx)
        assert [g.tiles()[k] for k in ("fft_x", "fft_y", "fft_z")] == list(idx)
        pd = torch.full_like(fd, float("nan"))
        g.poisson_solve(fd, pd)
        g.sync()
        err = rel_l2(pd.double().cpu().numpy(), ref)
        assert err < bar, (idx, err)
    g.close()


def test_set_tiles_rejects_unknown_schedule(torch):
    g = native.Grid(48, 40, 36, 4.8, 2.8, 4.68, nu=0.0, dt=1.0, precision="fp64")
    counts = schedule_counts((48, 40, 36))
    before = g.tiles()
    for idx in ((counts[0], 0, 0), (0, counts[1], 0), (0, 0, counts[2]), (-1, 0, 0)):
        with pytest.raises(native.VentflowError) as e:
            g.set_tiles(4, 32, 8, 16, *idx)
        assert e.value.code == native.VF_EINVAL
    g.close()
    g = native.Grid(48, 40, 36, 4.8, 2.8, 4.68, nu=0.0, dt=1.0, precision="fp64")
    assert g.tiles() == before
    g.close()


@pytest.mark.parametrize("fft_path", ["plane", "tile"])
def test_masked_room_fp64_100_steps_other_schedules(torch, monkeypatch, fft_path):
    """The masked-room parity case with the last candidate schedule on every axis."""
    if fft_path == "tile":
        monkeypatch.setenv("VF_TILE_FFT", "1")
    shape = (48, 30, 18)
    room, prm, geom, st0 = room_case(*shape, boxes=[(20, 26, 12, 20, 2, 9), (30, 34, 4, 8, 2, 5)])
    ref, _ = F.run(st0.copy(), geom, prm, 100)
    g = gpu_grid(prm, room.beta, room.S, room.room, "fp64")
    idx = [c - 1 for c in schedule_counts(shape)]
    assert max(idx) >= 2
    g.set_tiles(4, 32, 8, 16, *idx)
    load_state(g, st0, prm)
    g.step(100, reduce_every=10)
    errs = field_errors(read_state(g, prm), ref)
    assert max(errs.values()) < 1e-11, errs
    g.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_autotune_picks_and_caches_schedules(torch, precision):
    native.tile_cache_clear()
    room = rooms.make_room(48, 40, 36, h=0.05, boxes=[(14, 20, 6, 12, 2, 9)], u_in=0.8)
    g = native.room_grid(room, precision=precision)
    g.step(3, reduce_every=1)
    before = {n: g.read_field(n) for n in ("u", "v", "w", "c", "p")}
    chosen = g.autotune(reps=2)
    counts = schedule_counts((48, 40, 36))
    for k, c in zip(("fft_x", "fft_y", "fft_z"), counts):
        assert 0 <= chosen[k] < c, (k, chosen)
    assert g.tiles() == chosen
    assert native.tile_cache_lookup(48, 40, 36, precision) == chosen
    for n, arr in before.items():                   # the autotuner writes scratch arrays only
        assert np.array_equal(g.read_field(n), arr), n
    g.step(5, reduce_every=1)
    tuned = {n: g.read_field(n) for n in before}
    g.close()
    g2 = native.room_grid(room, precision=precision)  # takes the cached chunks and schedules
    assert g2.tiles() == chosen
    g2.set_tiles(4, 32, 8, 16, 0, 0, 0)                # the tuned grid's first 3 steps ran the defaults
    g2.step(3, reduce_every=1)
    g2.set_tiles(*(chosen[k] for k in ("zc_stage", "zc_div", "zc_project", "zc_filter", "fft_x", "fft_y", "fft_z")))
    g2.step(5, reduce_every=1)
    for n in before:
        assert np.array_equal(g2.read_field(n), tuned[n]), n
    g2.close()
    native.tile_cache_clear()


def test_register_path_grid_keeps_indices_unused(torch):
    """A grid on the register FFT path stores schedule indices but its solve does not change with them."""
    nx, ny, nz = 64, 32, 32
    prm = F.Params(nx=nx, ny=ny, nz=nz, lx=6.4, ly=2.24, lz=4.16, nu=0.0, dt=1.0)
    f = np.random.default_rng(5).standard_normal(prm.shape)
    g = native.Grid(nx, ny, nz, prm.lx, prm.ly, prm.lz, nu=0.0, dt=1.0, precision="fp64")
    fd = torch.tensor(f, dtype=torch.float64, device="cuda")
    p0 = torch.empty_like(fd)
    g.poisson_solve(fd, p0)
    g.set_tiles(4, 32, 8, 16, *[c - 1 for c in schedule_counts((nx, ny, nz))])
    p1 = torch.empty_like(fd)
    g.poisson_solve(fd, p1)
    g.sync()
    assert torch.equal(p0, p1)
    g.close()
