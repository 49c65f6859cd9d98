"""Register-resident FFT passes of the Poisson solve: every axis R G long with G threads of R values per
transform (lengths 16 G, G in 1, 2, 4, 8, 16, in both precisions; in FP32 also the 2-3-5 lengths 36, 40, 48, 60,
72, 80, 96 of the batch rooms, whose R-point DFTs are split at compile time into 2-, 3-, 4-, 5-, 8- and 16-point
ones, with G threads also where G does not divide R).

The solve is checked against the oracle's numpy.fft solve for every shape, and whole masked-room steps (the Eq. 9
correction kernel followed by the register passes) against the generic mixed-radix passes (VF_GENERIC_FFT).  The
masked-room parity tests against the oracle include register-path shapes."""
import numpy as np
import pytest

from oracle import flow as F
from paper_2204_02107_gb300 import native
from gpu_helpers import FIELD_NAMES, gpu_grid, load_state, rel_l2, require_gpu, room_case

pytestmark = pytest.mark.gpu

# (nx, ny, nz): G of x (nx / 32), y and z (n / 16); in FP32 the x lengths 32 and 64 run as 4 x 8 and 8 x 8
SHAPES = [(32, 16, 16),      # 1 1 1
          (64, 32, 64),      # 2 2 4
          (128, 64, 32),     # 4 4 2
          (256, 128, 128),   # 8 8 8
          (512, 256, 16),    # 16 16 1
          (32, 16, 256),     # 1 1 16
          (64, 128, 16)]     # 2 8 1

# FP32 2-3-5 shapes: (R, G) of x (nx / 2) and of y = z; 9 x 4, 15 x 4 and 9 x 8 have more threads than divide R
SHAPES_235 = [(72, 36, 36),      # (9, 4) (9, 4)
              (80, 40, 40),      # (20, 2) (20, 2)
              (96, 48, 48),      # (12, 4) (12, 4)
              (120, 60, 60),     # (15, 4) (15, 4)
              (144, 72, 72),     # (9, 8) (9, 8)
              (160, 80, 80),     # (20, 4) (20, 4)
              (192, 96, 96),     # (24, 4) (24, 4)
              (128, 72, 72),     # (16, 4) (9, 8)
              (72, 64, 64),      # (9, 4) (16, 4)
              (64, 80, 80),      # (16, 2) (20, 4)
              (120, 96, 96)]     # (15, 4) (24, 4)


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


@pytest.mark.parametrize("mode", ["plane", "tile"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", SHAPES)
def test_poisson_solve_all_g(torch, monkeypatch, precision, shape, mode):
    """mode "plane": the whole (y, z) plane of a kx in shared memory where it fits (else tiles anyway);
    "tile": y passes and z tiles forced."""
    if mode == "tile":
        monkeypatch.setenv("VF_REG_TILE", "1")
    nx, ny, nz = shape
    prm = F.Params(nx=nx, ny=ny, nz=nz, lx=nx * 0.1, ly=ny * 0.07, lz=nz * 0.13, nu=0.0, dt=1.0)
    rng = np.random.default_rng(nx * 7919 + ny * 31 + nz)
    f = rng.standard_normal(prm.shape)
    g = native.Grid(nx, ny, nz, prm.lx, prm.ly, prm.lz, nu=0.0, dt=1.0, precision=precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    fd = torch.tensor(f, dtype=dt, device="cuda")
    pd = torch.empty_like(fd)
    # (the FP64 256 x 128 plane exceeds the shared memory of one CTA: tiles in both modes)
    too_big = precision == "fp64" and (ny, nz) == (128, 128)
    assert g.fft_path() == ("register_tile" if mode == "tile" or too_big else "register_plane")
    g.poisson_solve(fd, pd)
    g.sync()
    got = pd.double().cpu().numpy()
    g.close()
    if precision == "fp32":
        f = f.astype(np.float32).astype(np.float64)
    ref = F.poisson_fft_solve(f, prm)
    err = rel_l2(got, ref)
    assert err < (1e-13 if precision == "fp64" else 2e-6), err


def poisson_case(torch, shape, precision, seed_extra=0):
    nx, ny, nz = shape
    prm = F.Params(nx=nx, ny=ny, nz=nz, lx=nx * 0.1, ly=ny * 0.07, lz=nz * 0.13, nu=0.0, dt=1.0)
    rng = np.random.default_rng(nx * 7919 + ny * 31 + nz + seed_extra)
    f = rng.standard_normal(prm.shape)
    g = native.Grid(nx, ny, nz, prm.lx, prm.ly, prm.lz, nu=0.0, dt=1.0, precision=precision)
    return prm, f, g


@pytest.mark.parametrize("shape", SHAPES_235)
def test_poisson_solve_235_fp32(torch, shape):
    """FP32 register transforms of 2-3-5 lengths (whole (y, z) planes) against the oracle's numpy.fft solve; the
    same lengths in FP64 take the generic passes."""
    prm, f, g = poisson_case(torch, shape, "fp32")
    assert g.fft_path() == "register_plane"
    fd = torch.tensor(f, dtype=torch.float32, device="cuda")
    pd = torch.empty_like(fd)
    g.poisson_solve(fd, pd)
    g.sync()
    got = pd.double().cpu().numpy()
    g.close()
    ref = F.poisson_fft_solve(f.astype(np.float32).astype(np.float64), prm)
    err = rel_l2(got, ref)
    assert err < 2e-6, err
    _, _, g64 = poisson_case(torch, shape, "fp64")
    assert g64.fft_path() == "generic"
    g64.close()


def test_235_unequal_plane_takes_generic(torch):
    """a 2-3-5 length in y or z needs ny = nz on the register path; otherwise the generic passes run"""
    for shape in ((144, 72, 96), (128, 64, 72)):
        _, _, g = poisson_case(torch, shape, "fp32")
        assert g.fft_path() == "generic", shape
        g.close()


@pytest.mark.parametrize("shape", [(144, 72, 72), (120, 96, 96), (72, 64, 64)])
def test_register_235_room_matches_generic_passes(torch, monkeypatch, shape):
    """20 FP32 steps of a masked room through the 2-3-5 register passes and the generic ones"""
    nx, ny, nz = shape
    room, prm, geom, st0 = room_case(nx, ny, nz, boxes=[(nx // 4, nx // 4 + 8, 10, 20, 2, 12),
                                                        (nx // 2, nx // 2 + 12, ny // 2, ny // 2 + 10, 2, 8)],
                                     seed=nx + ny)
    out = {}
    for path in ("register", "generic"):
        monkeypatch.delenv("VF_GENERIC_FFT", raising=False)
        if path == "generic":
            monkeypatch.setenv("VF_GENERIC_FFT", "1")
        g = gpu_grid(prm, room.beta, room.S, room.room, "fp32")
        assert g.fft_path() == ("register_plane" if path == "register" else "generic")
        load_state(g, st0, prm, as_fp32=True)
        g.step(20)
        out[path] = {n: g.read_field(n) for n in FIELD_NAMES + ("p",)}
        g.close()
    for n in FIELD_NAMES + ("p",):
        assert rel_l2(out["register"][n], out["generic"][n]) < 2e-5, n


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_register_path_matches_generic_passes(torch, monkeypatch, precision):
    """20 steps of a masked 128 x 64 x 32 room through the register passes (plane and tile mode) and the generic
    ones."""
    room, prm, geom, st0 = room_case(128, 64, 32, boxes=[(30, 40, 10, 20, 2, 12), (70, 90, 30, 44, 2, 8)], seed=7)
    out = {}
    for path in ("register", "register_tile", "generic"):
        monkeypatch.delenv("VF_REG_TILE", raising=False)
        if path == "register_tile":
            monkeypatch.setenv("VF_REG_TILE", "1")
        if path == "generic":
            monkeypatch.setenv("VF_GENERIC_FFT", "1")
        g = gpu_grid(prm, room.beta, room.S, room.room, precision)
        load_state(g, st0, prm, as_fp32=precision == "fp32")
        g.step(20)
        out[path] = {n: g.read_field(n) for n in FIELD_NAMES + ("p",)}
        g.close()
    bar = 1e-12 if precision == "fp64" else 2e-5
    for n in FIELD_NAMES + ("p",):
        for path in ("register", "register_tile"):
            assert rel_l2(out[path][n], out["generic"][n]) < bar, (path, n)


def test_masked_room_fp64_100_steps_tile_mode(torch, monkeypatch):
    """The register path with y passes and z tiles (forced) against the oracle over 100 FP64 steps."""
    from gpu_helpers import field_errors, read_state
    monkeypatch.setenv("VF_REG_TILE", "1")
    room, prm, geom, st0 = room_case(64, 32, 32, boxes=[(20, 26, 8, 14, 2, 12), (40, 46, 18, 26, 2, 9)])
    ref, _ = F.run(st0.copy(), geom, prm, 100)
    g = gpu_grid(prm, room.beta, room.S, room.room, "fp64")
    load_state(g, st0, prm)
    g.step(100)
    errs = field_errors(read_state(g, prm), ref)
    g.close()
    assert max(errs.values()) < 1e-11, errs


def test_masked_room_fp64_4_thread_groups(torch):
    """FP64 register passes with 4-thread groups on every axis (128 x 64 x 64: x 64 = 16 x 4, y = z 64 = 16 x 4; the
    groups on adjacent lanes, strides from the quarter-warp bank model) against the oracle over 40 steps."""
    from gpu_helpers import field_errors, read_state
    room, prm, geom, st0 = room_case(128, 64, 64, boxes=[(30, 40, 10, 20, 2, 12), (70, 90, 30, 44, 2, 8)], seed=9)
    ref, _ = F.run(st0.copy(), geom, prm, 40)
    g = gpu_grid(prm, room.beta, room.S, room.room, "fp64")
    assert g.fft_path() == "register_plane"
    load_state(g, st0, prm)
    g.step(40)
    errs = field_errors(read_state(g, prm), ref)
    g.close()
    assert max(errs.values()) < 1e-11, errs
