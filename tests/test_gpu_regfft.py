"""Register-resident FFT passes of the Poisson solve (every axis 16 G long, G in 1, 2, 4, 8, 16).

The solve is checked against the oracle's numpy.fft solve for every G on every axis, and whole masked-room steps
(the Eq. 9 correction kernel followed by the register passes) against the generic mixed-radix passes
(VF_GENERIC_FFT).  The masked-room parity tests against the oracle include register-path shapes."""
import numpy as np
import pytest

from oracle import flow as F
from paper_2204_02107_gb300 import native
from gpu_helpers import FIELD_NAMES, gpu_grid, load_state, rel_l2, require_gpu, room_case

pytestmark = pytest.mark.gpu

# (nx, ny, nz): G of x (nx / 32), y and z (n / 16)
SHAPES = [(32, 16, 16),      # 1 1 1
          (64, 32, 64),      # 2 2 4
          (128, 64, 32),     # 4 4 2
          (256, 128, 128),   # 8 8 8
          (512, 256, 16),    # 16 16 1
          (32, 16, 256),     # 1 1 16
          (64, 128, 16)]     # 2 8 1


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
    g.poisson_solve(fd, pd)
    g.sync()
    got = pd.double().cpu().numpy()
    g.close()
    if precision == "fp32":
        f = f.astype(np.float32).astype(np.float64)
    ref = F.poisson_fft_solve(f, prm)
    err = rel_l2(got, ref)
    assert err < (1e-13 if precision == "fp64" else 2e-6), err


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
