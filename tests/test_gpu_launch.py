"""Programmatic dependent launch (opt-in with VF_PDL=1) changes when a kernel is scheduled, never what it computes:
20 steps of a masked room with its reductions every step, FP32 and FP64, give bitwise the same fields and records
with and without it.  The setting is read once per process, so the opt-in run is a child process."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2204_02107_gb300 import native, rooms
from gpu_helpers import FIELD_NAMES, require_gpu

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
RECORD_KEYS = ("ke", "div_l2", "div_max", "u_max", "c_total", "c_room", "c2_room", "v_room")


def run_case(out_path):
    """20 steps of a 64 x 32 x 32 room with one box and a random initial velocity, in both precisions."""
    room = rooms.make_room(64, 32, 32, h=0.05, boxes=[(20, 26, 8, 14, 2, 12)], u_in=1.0)
    u, v, w = rooms.random_fields(room.beta.shape, 5, count=3, scale=0.2, beta=room.beta)
    out = {}
    for precision in ("fp32", "fp64"):
        g = native.room_grid(room, precision=precision, history_capacity=32)
        for name, arr in (("u", u), ("v", v), ("w", w)):
            g.set_field(name, arr.astype(np.float32) if precision == "fp32" else arr)
        g.step(20, reduce_every=1)
        for name in FIELD_NAMES + ("p",):
            out[f"{precision}_{name}"] = g.read_field(name)
        recs = g.history()
        for key in RECORD_KEYS:
            out[f"{precision}_rec_{key}"] = np.array([r[key] for r in recs])
        out[f"{precision}_rec_hist"] = np.array([r["hist"] for r in recs])
        g.close()
    np.savez(out_path, **out)


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def test_programmatic_launch_is_bitwise_neutral(torch, tmp_path):
    plain = tmp_path / "plain.npz"
    pdl = tmp_path / "pdl.npz"
    run_case(plain)
    env = dict(os.environ, VF_PDL="1", PYTHONPATH=os.pathsep.join([ROOT, HERE, os.environ.get("PYTHONPATH", "")]))
    code = f"import test_gpu_launch as t; t.run_case({str(pdl)!r})"
    res = subprocess.run([sys.executable, "-c", code], cwd=HERE, env=env, capture_output=True, text=True,
                         timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    a, b = np.load(plain), np.load(pdl)
    assert sorted(a.files) == sorted(b.files)
    for key in a.files:
        assert np.array_equal(a[key], b[key]), key
