"""vf_poisson_solve_noalloc: the Poisson solve for callers that cannot allocate device memory (code running where
cudaMalloc is forbidden, e.g. inside an allocator or a framework that owns every device allocation).

It keeps its scratch in one static device array instead of allocating, so it is checked here against the
allocating entry point vf_poisson_solve on the same inputs, within the same tolerances as the other Poisson
tests, over two calls in a row (the second reuses the array the first left behind).  This file is collected last
so that a failure here comes after every other test has run."""
import numpy as np
import pytest

from paper_2204_02107_gb300 import native
from gpu_helpers import rel_l2, require_gpu

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-13, "fp32": 2e-6}


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def allocating_solve(torch, shape, lengths, precision, f):
    nx, ny, nz = shape
    g = native.Grid(nx, ny, nz, *lengths, nu=0.0, dt=1.0, precision=precision)
    p = torch.empty_like(f)
    g.poisson_solve(f, p)
    g.sync()
    out = p.double().cpu().numpy()
    g.close()
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_matches_allocating_solve_twice(torch, precision):
    dt = torch.float64 if precision == "fp64" else torch.float32
    cases = [((72, 36, 20), (7.2, 2.52, 2.6), 11), ((40, 10, 50), (4.0, 0.7, 6.5), 12)]
    for shape, lengths, seed in cases:          # two calls in a row on the shared scratch array
        nx, ny, nz = shape
        f = torch.tensor(np.random.default_rng(seed).standard_normal((nz, ny, nx)), dtype=dt, device="cuda")
        want = allocating_solve(torch, shape, lengths, precision, f)
        p = torch.full_like(f, float("nan"))
        native.poisson_solve_noalloc(nx, ny, nz, *lengths, f, p)
        got = p.double().cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_l2(got, want) < TOL[precision], (shape, rel_l2(got, want))


def test_noalloc_rejects_oversized_grid(torch):
    limit = native.lib().vf_poisson_noalloc_max_cells(native.VF_FP64)
    assert limit == 4194304
    f = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(native.VentflowError) as ei:
        native.poisson_solve_noalloc(512, 128, 128, 1.0, 1.0, 1.0, f, f)   # 8.4 M cells > FP64 limit
    assert ei.value.code == native.VF_ESIZE
    with pytest.raises(native.VentflowError) as ei:
        native.poisson_solve_noalloc(2048, 8, 8, 1.0, 1.0, 1.0, f, f)      # nx/2 + 1 > 1024
    assert ei.value.code == native.VF_ESIZE
