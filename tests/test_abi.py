"""The C ABI without a GPU: the library loads, exports every function the header declares, validates sizes
before touching the device, and its host-side metrics agree with the oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import ventilation as V
from paper_2204_02107_gb300 import build as B
from paper_2204_02107_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    srcs = [os.path.join(B.CSRC, f) for f in os.listdir(B.CSRC)] + [os.path.join(B.INCLUDE, "ventflow.h")]
    if not os.path.exists(B.LIB_PATH) or os.path.getmtime(B.LIB_PATH) < max(os.path.getmtime(s) for s in srcs):
        B.build()
    return native.lib()


def declared_functions():
    names = []
    for header in os.listdir(os.path.join(ROOT, "include")):
        text = open(os.path.join(ROOT, "include", header)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(vf_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    raw = ctypes.CDLL(B.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing


def test_binding_covers_header(lib):
    assert set(declared_functions()) <= set(native._SIGNATURES)


def test_struct_sizes_match_header(lib):
    # vf_reduce: 11 scalars + 64 + 2 counters + 5 budget terms, all 8 bytes
    assert ctypes.sizeof(native.VfReduce) == 8 * (11 + 64 + 2 + 5)
    sizes = (ctypes.c_int64 * 4)()
    assert lib.vf_abi_sizes(sizes) == 0
    assert list(sizes) == [ctypes.sizeof(native.VfGridDesc), ctypes.sizeof(native.VfReduce),
                           ctypes.sizeof(native.VfBatchDesc), ctypes.sizeof(native.VfTiles)]
    d = native.default_desc()
    assert (d.nx, d.ny, d.nz) == (64, 64, 64) and d.n_pressure_iters == 4 and d.filter == 1
    assert d.precision == native.VF_FP32_MIXED and d.alpha_c < 0


def test_status_strings(lib):
    assert native.status_string(0) == "VF_OK"
    assert native.status_string(native.VF_ESIZE) == "VF_ESIZE"
    assert native.status_string(-99) == "VF_UNKNOWN"


@pytest.mark.parametrize("n", [7, 9, 14, 22, 6, 0, -8])
def test_bad_sizes_rejected_before_any_device_call(lib, n):
    d = native.default_desc()
    d.nx = n
    h = ctypes.c_void_p()
    assert lib.vf_create_grid(ctypes.byref(d), ctypes.byref(h)) == native.VF_ESIZE
    assert not h.value


@pytest.mark.parametrize("shape", [(2048, 1024, 1024), (1152, 1024, 1024), (4096, 512, 1024)])
def test_grids_over_two_to_the_thirty_cells_rejected(lib, shape):
    d = native.default_desc()
    d.nx, d.ny, d.nz = shape
    h = ctypes.c_void_p()
    assert lib.vf_create_grid(ctypes.byref(d), ctypes.byref(h)) == native.VF_ESIZE
    assert not h.value
    t = native.VfTiles(4, 32, 8, 16, 0, 0, 0)
    assert lib.vf_tile_cache_insert(*shape, native.VF_FP32_MIXED, ctypes.byref(t)) == native.VF_ESIZE


def test_bad_arguments_rejected(lib):
    d = native.default_desc()
    d.dt = 0.0
    h = ctypes.c_void_p()
    assert lib.vf_create_grid(ctypes.byref(d), ctypes.byref(h)) == native.VF_EINVAL
    d = native.default_desc()
    d.precision = 7
    assert lib.vf_create_grid(ctypes.byref(d), ctypes.byref(h)) == native.VF_EINVAL
    assert lib.vf_create_grid(None, ctypes.byref(h)) == native.VF_EINVAL
    assert lib.vf_destroy(None) == native.VF_OK


def test_host_metrics_match_oracle(lib):
    t = np.linspace(0, 600, 121)
    c = 0.9 * np.exp(-4.5 * t / 3600)
    assert native.ach_log_slope(t, c) == pytest.approx(V.ach_log_slope(t, c), rel=1e-12)
    t = np.linspace(0, 3600, 300)
    c = 0.55 * np.exp(-3.3 * t / 3600) + 0.31
    a, c0, c1 = native.ach_fit3(t, c)
    ra, rc0, rc1 = V.ach_fit3(t, c)
    assert a == pytest.approx(3.3, rel=1e-7) and a == pytest.approx(ra, rel=1e-7)
    assert c0 == pytest.approx(rc0, rel=1e-6) and c1 == pytest.approx(rc1, rel=1e-6)
    for ach in (0.0, 1e-9, 3.48, 67.6):
        q, p = native.wells_riley(100 / 192, 1.2, ach, 0.5)
        assert q == pytest.approx(V.wells_riley_dose(100 / 192, 1.2, ach, 0.5), rel=1e-12)
        assert p == pytest.approx(V.infection_probability(q), rel=1e-12)
    with pytest.raises(native.VentflowError):
        native.wells_riley(1.0, 1.2, -1.0, 0.5)


def test_fft_schedules(lib):
    """Radix schedules of the generic FFT passes: every candidate factors n into radices the kernels implement,
    candidates are distinct, at most 8, and candidate 0 is the documented default (fewest power-of-two passes,
    then the 3s and 5s)."""
    default = {8: [8], 16: [16], 32: [4, 8], 64: [8, 8], 128: [16, 8], 256: [16, 16], 12: [4, 3],
               20: [4, 5], 36: [4, 3, 3], 72: [8, 3, 3], 80: [16, 5], 96: [4, 8, 3], 120: [8, 3, 5],
               160: [4, 8, 5], 192: [8, 8, 3], 1024: [16, 8, 8]}
    for n in range(2, 1025):
        cands = native.fft_schedules(n)
        m = n
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        if m != 1:
            assert cands == [], n
            continue
        assert 1 <= len(cands) <= 8, n
        assert len({tuple(c) for c in cands}) == len(cands), n
        for c in cands:
            assert int(np.prod(c)) == n and set(c) <= {2, 3, 4, 5, 8, 16}, (n, c)
        if n in default:
            assert cands[0] == default[n], (n, cands[0])
    # several schedules for the mixed lengths of the batch rooms
    assert all(len(native.fft_schedules(n)) >= 3 for n in (36, 40, 48, 60, 72, 80, 96))
    buf = (ctypes.c_int32 * 2)()
    assert lib.vf_fft_schedules(1024, 0, buf, 2) == native.VF_EINVAL      # three radices do not fit in two
    assert lib.vf_fft_schedules(64, -1, buf, 2) == native.VF_EINVAL
    assert lib.vf_fft_schedules(64, 99, buf, 2) == 0


def test_tile_cache_save_and_load(lib, tmp_path):
    """The tile cache round-trips through JSON without a GPU; the library checks every stored entry."""
    native.tile_cache_clear()
    a = {"zc_stage": 8, "zc_div": 16, "zc_project": 4, "zc_filter": 32, "fft_x": 1, "fft_y": 2, "fft_z": 0}
    b = {"zc_stage": 4, "zc_div": 32, "zc_project": 8, "zc_filter": 16, "fft_x": 0, "fft_y": 0, "fft_z": 0}
    native.tile_cache_insert(96, 80, 72, "fp32", a)
    native.tile_cache_insert(64, 64, 64, "fp64", b)
    assert native.tile_cache_lookup(96, 80, 72, "fp32") == a
    assert [k for k, _ in native.tile_cache_entries()] == [(64, 64, 64, "fp64"), (96, 80, 72, "fp32")]
    path = tmp_path / "tiles.json"
    native.tile_cache_save(path)
    native.tile_cache_clear()
    assert native.tile_cache_entries() == []
    assert native.tile_cache_load(path) == 2
    assert native.tile_cache_lookup(96, 80, 72, "fp32") == a and native.tile_cache_lookup(64, 64, 64, "fp64") == b
    bad = [((96, 80, 72), dict(a, zc_stage=3), native.VF_EINVAL),                  # chunk below the minimum
           ((96, 80, 72), dict(a, fft_x=len(native.fft_schedules(48))), native.VF_EINVAL),   # not a candidate
           ((98, 80, 72), a, native.VF_ESIZE)]                                     # 98 = 2 * 7^2
    for (nx, ny, nz), tiles, code in bad:
        with pytest.raises(native.VentflowError) as e:
            native.tile_cache_insert(nx, ny, nz, "fp32", tiles)
        assert e.value.code == code
    key = (ctypes.c_int32 * 4)()
    assert lib.vf_tile_cache_entry(5, key, ctypes.byref(native.VfTiles())) == native.VF_EINVAL
    native.tile_cache_clear()


C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "ventflow.h"

int main(void)
{
    vf_grid_desc d;
    int64_t sizes[4];
    int32_t rad[16];
    if (vf_grid_desc_default(&d) != VF_OK || d.n_pressure_iters != 4 || d.precision != VF_FP32_MIXED) return 1;
    if (vf_abi_sizes(sizes) != VF_OK) return 2;
    if (sizes[0] != (int64_t)sizeof(vf_grid_desc) || sizes[1] != (int64_t)sizeof(vf_reduce) ||
        sizes[2] != (int64_t)sizeof(vf_batch_desc) || sizes[3] != (int64_t)sizeof(vf_tiles)) return 3;
    if (vf_fft_schedules(96, 0, rad, 16) != 3 || rad[0] * rad[1] * rad[2] != 96) return 4;
    if (strcmp(vf_status_string(VF_ESIZE), "VF_ESIZE") != 0) return 5;
    d.nx = 14;   /* 14 = 2 x 7: rejected before any device work */
    vf_grid* g = NULL;
    if (vf_create_grid(&d, &g) != VF_ESIZE || g != NULL) return 6;
    printf("ok\n");
    return 0;
}
"""


def test_header_is_plain_c_and_links(lib, tmp_path):
    """The header compiles as C11 with warnings as errors, and a C program linked against the library sees the
    same struct sizes as the library and calls its host-only entry points (no GPU needed)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(B.LIB_PATH)
    cmd = [gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
           str(exe), "-L", libdir, "-l:" + os.path.basename(B.LIB_PATH), "-Wl,-rpath," + libdir]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    env = dict(os.environ)
    env["LD_LIBRARY_PATH"] = ":".join(p for p in ("/usr/local/cuda/lib64", env.get("LD_LIBRARY_PATH", "")) if p)
    out = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=60)
    assert out.returncode == 0 and out.stdout.strip() == "ok", (out.returncode, out.stdout, out.stderr)


def test_batch_and_solver_arguments_rejected_before_any_device_call(lib):
    """Batch descriptions, the allocation-free solve's sizes and NULL handles are checked on the host first."""
    h = ctypes.c_void_p()
    for fields in ({"max_slots": 0}, {"hbm_budget_bytes": 0}, {"reduce_every": -1}, {"autotune": -1},
                   {"autotune": 1001}):
        d = native.VfBatchDesc(4, 1 << 30, 1, None, 0)
        for k, v in fields.items():
            setattr(d, k, v)
        assert lib.vf_batch_create(ctypes.byref(d), ctypes.byref(h)) == native.VF_EINVAL, fields
    assert lib.vf_batch_create(None, ctypes.byref(h)) == native.VF_EINVAL
    # sizes beyond the static scratch, or not 2-3-5 smooth, are refused before the device is touched
    f = ctypes.c_void_p(16)
    big = lib.vf_poisson_noalloc_max_cells(native.VF_FP64)
    assert big > 0 and lib.vf_poisson_noalloc_max_cells(7) == 0
    assert lib.vf_poisson_solve_noalloc(512, 128, 128, 1.0, 1.0, 1.0, native.VF_FP64, f, f, None) == native.VF_ESIZE
    assert lib.vf_poisson_solve_noalloc(14, 8, 8, 1.0, 1.0, 1.0, native.VF_FP64, f, f, None) == native.VF_ESIZE
    # the y and z passes' shared-memory bound: ny or nz above 581 (FP64) / 592 (FP32), whatever the cell count
    for prec in (native.VF_FP64, native.VF_FP32_MIXED):
        assert lib.vf_poisson_solve_noalloc(8, 600, 8, 1.0, 1.0, 1.0, prec, f, f, None) == native.VF_ESIZE
        assert lib.vf_poisson_solve_noalloc(8, 8, 600, 1.0, 1.0, 1.0, prec, f, f, None) == native.VF_ESIZE
        assert not native._noalloc_sizes_accepted(8, 600, 8, prec)
    assert native._noalloc_sizes_accepted(8, 576, 8, native.VF_FP64)
    # NULL grid handles
    assert lib.vf_step(None, 1, 0) == native.VF_EINVAL
    assert lib.vf_sync(None) == native.VF_EINVAL
    t = native.VfTiles()
    assert lib.vf_get_tiles(None, ctypes.byref(t)) == native.VF_EINVAL
    path = ctypes.c_int32(-1)
    assert lib.vf_fft_path(None, ctypes.byref(path)) == native.VF_EINVAL and path.value == -1
