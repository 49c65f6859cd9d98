"""Shared helpers of the GPU tests: build-on-demand of the library, and running the same case through the CUDA
path (via the C ABI) and through the oracle."""
import os

import numpy as np
import pytest

from oracle import flow as F
from paper_2204_02107_gb300 import build as B
from paper_2204_02107_gb300 import native, rooms

FIELD_NAMES = ("u", "v", "w", "c")


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    srcs = [os.path.join(B.CSRC, f) for f in os.listdir(B.CSRC)] + [os.path.join(B.INCLUDE, "ventflow.h")]
    if not os.path.exists(B.LIB_PATH) or os.path.getmtime(B.LIB_PATH) < max(os.path.getmtime(s) for s in srcs):
        B.build()
    native.lib()
    return torch


def params_of(prm_kw):
    return F.Params(**prm_kw)


def gpu_grid(prm: F.Params, geom_beta, geom_S, geom_room, precision, **kw):
    g = native.Grid(prm.nx, prm.ny, prm.nz, prm.lx, prm.ly, prm.lz, nu=prm.nu, dt=prm.dt, alpha_c=prm.alpha_c,
                    tau_f=prm.tau_f, body_force=prm.body_force, n_pressure_iters=prm.n_pressure_iters,
                    filter=prm.filter, precision=precision, **kw)
    g.set_mask(np.asarray(geom_beta, dtype=np.uint8))
    g.set_inflow(np.asarray(geom_S, dtype=np.uint8), prm.u_set, prm.c_set)
    g.set_region(np.asarray(geom_room, dtype=np.uint8))
    return g


def load_state(g, state: F.State, prm: F.Params, as_fp32=False):
    for name in FIELD_NAMES:
        arr = getattr(state, name)
        g.set_field(name, arr.astype(np.float32) if as_fp32 else arr)
    g.set_field("p", (state.p / prm.dt).astype(np.float32) if as_fp32 else state.p / prm.dt)
    g.set_time(state.t, state.step)


def read_state(g, prm: F.Params):
    f = {n: g.read_field(n) for n in FIELD_NAMES}
    return F.State(f["u"], f["v"], f["w"], f["c"], g.read_field("p") * prm.dt)


def rel_l2(a, b, norm=None):
    den = np.linalg.norm(b) if norm is None else norm
    if den == 0:
        return float(np.linalg.norm(a - b))
    return float(np.linalg.norm(a - b) / den)


def field_errors(gpu: F.State, ref: F.State):
    """Relative L2 error per field; fields whose reference norm is ~0 (w of Taylor-Green) are normalised by the
    velocity norm."""
    vel_norm = np.sqrt(sum(np.linalg.norm(getattr(ref, n)) ** 2 for n in ("u", "v", "w")))
    out = {}
    for n in FIELD_NAMES + ("p",):
        a, b = getattr(gpu, n), getattr(ref, n)
        nb = np.linalg.norm(b)
        if n in ("u", "v", "w") and nb < 1e-6 * vel_norm:
            out[n] = rel_l2(a, b, vel_norm)
        elif nb == 0:
            out[n] = float(np.linalg.norm(a))
        else:
            out[n] = rel_l2(a, b)
    return out


def room_case(nx, ny, nz, boxes=(), h=0.05, u_in=1.0, filter=True, n_iters=4, seed=None):
    room = rooms.make_room(nx, ny, nz, h=h, boxes=boxes, u_in=u_in)
    prm = F.Params(nx=nx, ny=ny, nz=nz, lx=room.lx, ly=room.ly, lz=room.lz, nu=rooms.NU_AIR, dt=room.dt,
                   u_set=(room.u_in, 0.0, 0.0), c_set=0.0, filter=filter, n_pressure_iters=n_iters)
    geom = F.Geometry(room.beta, room.S, room.room)
    st = F.zero_state(prm, c=room.initial_c())
    if seed is not None:
        u, v, w = rooms.random_fields(prm.shape, seed, count=3, scale=0.2, beta=room.beta)
        st = F.State(u, v, w, st.c, st.p)
    return room, prm, geom, st
