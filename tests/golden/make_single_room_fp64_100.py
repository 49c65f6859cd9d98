"""Writes single_room_fp64_100.npz: the FP64 oracle's state of the 256 x 128 x 128 single room after 100 steps,
at a seeded sample of cells, with the full-field norms and the last step's reductions and scalar budget.

The case is the single room as configured for the benchmark (10 x 5 x 5 m, 2-cell walls, one 5 x 5-cell duct pair,
U_in = 1 m/s, dt = 0.25 dx / U_in, filter on, 4 pressure iterations), started from rest with stale air (c = 1 in
the fluid, 0 in the forcing region and the solids).  Only the oracle and the seeded input generators are called,
so every stored value comes from the oracle.  About ten minutes of one host core:

    python tests/golden/make_single_room_fp64_100.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import flow as F  # noqa: E402
from paper_2204_02107_gb300 import rooms  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "single_room_fp64_100.npz")
STEPS = 100
SAMPLE_SEED = 100
RECORD_KEYS = ("ke", "c_total", "c_room", "c2_room", "v_room", "u_max", "div_max", "div_l2", "forcing",
               "forcing_room", "outflow", "mask_loss", "filter_room")


def case():
    room = rooms.single_room(256, 128, 128)
    prm = F.Params(nx=room.nx, ny=room.ny, nz=room.nz, lx=room.lx, ly=room.ly, lz=room.lz, nu=rooms.NU_AIR,
                   dt=room.dt, u_set=(room.u_in, 0.0, 0.0), c_set=0.0, filter=True, n_pressure_iters=4)
    geom = F.Geometry(room.beta, room.S, room.room)
    return room, prm, geom, F.zero_state(prm, c=room.initial_c())


def sample_cells(prm):
    """4096 cells drawn over the whole room and 4096 over the inlet jet's region (x < 48, y and z within 16 cells
    of the duct axis), as linear indices x + nx (y + ny z)."""
    rng = np.random.default_rng(SAMPLE_SEED)
    n = prm.nx * prm.ny * prm.nz
    everywhere = rng.choice(n, size=4096, replace=False)
    x = rng.integers(0, 48, size=4096)
    y = rng.integers(prm.ny // 2 - 16, prm.ny // 2 + 16, size=4096)
    z = rng.integers(prm.nz // 2 - 16, prm.nz // 2 + 16, size=4096)
    jet = x + prm.nx * (y + prm.ny * z)
    return np.unique(np.concatenate([everywhere, jet]))


def main():
    room, prm, geom, st = case()
    rec = None
    for s in range(STEPS):
        st, rec = F.step(st, geom, prm, with_budget=(s == STEPS - 1))
    idx = sample_cells(prm)
    fields = {"u": st.u, "v": st.v, "w": st.w, "c": st.c, "p": F.physical_pressure(st, prm)}
    out = {"idx": idx, "steps": np.array(STEPS)}
    for name, f in fields.items():
        out[name] = f.ravel()[idx]
        out[name + "_norm"] = np.array(np.linalg.norm(f))
    for key in RECORD_KEYS:
        out["rec_" + key] = np.array(rec[key])
    np.savez_compressed(OUT, **out)
    print(f"wrote {OUT}: {idx.size} cells")


if __name__ == "__main__":
    main()
