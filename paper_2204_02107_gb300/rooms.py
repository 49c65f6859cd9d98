"""Seeded synthetic inputs: room geometries (binary masks), initial fields and request traces.

This module builds inputs only: masks from walls, ducts, doorways and boxes, the Taylor-Green initial field,
seeded random fields and arrival traces.  It holds none of the flow method's arithmetic, so the CUDA path, the
CPU oracle, the tests and the benchmark can all draw the same inputs from it.

The paper's rooms exist only as figures (Sec. 3.3, Tab. 3), so these rooms stand in for them with the paper's
scales: 2-cell solid walls, 5x5-cell square ducts (0.195 m at dx = 0.0390625 m), a forcing region S in the inlet
wall opening and a plain opening in the opposite wall (the periodic wrap joins them, the paper's option A of
Sec. 2.1), floor-standing boxes as furniture, and a partition wall with a doorway.

Arrays have shape (nz, ny, nx) (x fastest in memory); masks are uint8 with 1 = fluid / in region.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

DX_ROOM = 0.0390625          # 10 m / 256 cells
NU_AIR = 1.6e-5              # Tab. 3
DUCT_CELLS = 5


def smooth235(n):
    """True if n is even, >= 8 and has no prime factor other than 2, 3 and 5."""
    if n < 8 or n % 2:
        return False
    for p in (2, 3, 5):
        while n % p == 0:
            n //= p
    return n == 1


@dataclass
class Room:
    """A room case: sizes, masks and the inflow set point."""

    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    lz: float
    beta: np.ndarray                  # uint8 (nz, ny, nx): 1 fluid, 0 solid
    S: np.ndarray                     # uint8: 1 in the inlet forcing region
    room: np.ndarray                  # uint8: 1 for cells counted in the room inventory / histogram
    u_in: float = 1.0
    inflow_area: float = 0.0          # m^2, total inlet cross-section
    name: str = "room"
    meta: dict = field(default_factory=dict)

    @property
    def h(self):
        return self.lx / self.nx

    @property
    def dt(self):
        """Fixed time step 0.25 dx / U_in."""
        return 0.25 * self.h / self.u_in

    @property
    def cells(self):
        return self.nx * self.ny * self.nz

    def initial_c(self, dtype=np.float64):
        """Stale air c = 1 in fluid cells, 0 in solids and in the forcing region (exact 0 / 1 in any dtype: an FP32
        grid can take float32, half the bytes to form and upload)."""
        return self.beta.astype(dtype) * (np.asarray(1.0, dtype) - self.S.astype(dtype))


def _empty_box(nx, ny, nz, wall):
    beta = np.zeros((nz, ny, nx), dtype=np.uint8)
    beta[wall:nz - wall, wall:ny - wall, wall:nx - wall] = 1
    return beta


def make_room(nx, ny, nz, h=DX_ROOM, wall=2, ducts=((None, None),), duct=DUCT_CELLS, boxes=(), partition=None,
              u_in=1.0, name="room"):
    """Closed box with ``wall``-cell solid walls, inlet/outlet duct pairs through the x walls, optional solid
    boxes (cell ranges, half-open) and an optional partition wall with a doorway.

    Each duct pair: cells (y in yc +- duct//2, z in zc +- duct//2) are opened in the x = 0..wall-1 wall (fluid,
    S = 1) and in the x = nx-wall..nx-1 wall (fluid, S = 0).  ``None`` centres mean the middle of the wall.
    ``partition`` = (x0, thickness, door_width, door_height): solid slab at x0..x0+thickness-1 with a doorway of
    door_width cells centred in y, from the floor up to door_height cells."""
    beta = _empty_box(nx, ny, nz, wall)
    S = np.zeros_like(beta)
    half = duct // 2
    for yc, zc in ducts:
        yc = ny // 2 if yc is None else yc
        zc = nz // 2 if zc is None else zc
        ys = slice(yc - half, yc - half + duct)
        zs = slice(zc - half, zc - half + duct)
        beta[zs, ys, 0:wall] = 1
        S[zs, ys, 0:wall] = 1
        beta[zs, ys, nx - wall:nx] = 1
    for (x0, x1, y0, y1, z0, z1) in boxes:
        beta[z0:z1, y0:y1, x0:x1] = 0
    if partition is not None:
        x0, thick, dw, dh = partition
        beta[wall:nz - wall, wall:ny - wall, x0:x0 + thick] = 0
        y0 = ny // 2 - dw // 2
        beta[wall:wall + dh, y0:y0 + dw, x0:x0 + thick] = 1
    S &= beta
    room = beta.copy()
    room[:, :, 0:wall] = 0
    room[:, :, nx - wall:nx] = 0
    area = len(ducts) * (duct * h) ** 2
    return Room(nx, ny, nz, nx * h, ny * h, nz * h, beta, S, room, u_in=u_in, inflow_area=area, name=name)


def random_boxes(rng, count, nx, ny, nz, h, wall=2, side_m=(0.3, 1.5), keep_clear=(), clear_m=1.0,
                 max_tries=1000):
    """``count`` floor-standing axis-aligned boxes with sides uniform in ``side_m`` metres, kept ``clear_m`` away
    (in x and y) from the points in ``keep_clear`` (cell coordinates (x, y)) and inside the walls."""
    boxes = []
    lo_cells = max(1, int(round(side_m[0] / h)))
    hi_cells = max(lo_cells, int(round(side_m[1] / h)))
    clear = int(math.ceil(clear_m / h))
    tries = 0
    while len(boxes) < count and tries < max_tries:
        tries += 1
        sx, sy, sz = (int(rng.integers(lo_cells, hi_cells + 1)) for _ in range(3))
        sx = min(sx, nx - 2 * wall - 2)
        sy = min(sy, ny - 2 * wall - 2)
        sz = min(sz, nz - 2 * wall - 2)
        if min(sx, sy, sz) < 1:
            continue
        x0 = int(rng.integers(wall + 1, nx - wall - sx))
        y0 = int(rng.integers(wall + 1, ny - wall - sy))
        z0 = wall
        ok = True
        for (cx, cy) in keep_clear:
            if x0 - clear <= cx < x0 + sx + clear and y0 - clear <= cy < y0 + sy + clear:
                ok = False
                break
        if ok:
            boxes.append((x0, x0 + sx, y0, y0 + sy, z0, z0 + sz))
    return boxes


def single_room(nx=256, ny=128, nz=128, u_in=1.0):
    """Single 10 x 5 x 5 m room, 2-cell walls, one 5x5-cell duct pair at the centre of the x walls, U_in = 1 m/s."""
    return make_room(nx, ny, nz, h=DX_ROOM * 256 / nx, u_in=u_in, name=f"single room {nx}x{ny}x{nz}")


def large_room(nx=512, ny=256, nz=256, seed=3, u_in=0.1, n_boxes=20):
    """Large 20 x 10 x 10 m room: partition wall at mid-x with a doorway, two duct pairs, seeded furniture."""
    h = DX_ROOM * 512 / nx
    rng = np.random.default_rng(seed)
    ducts = ((ny // 4, 3 * nz // 4), (3 * ny // 4, 3 * nz // 4))
    clear_pts = [(x, y) for (y, _) in ducts for x in (2, nx - 3)]
    boxes = random_boxes(rng, n_boxes, nx, ny, nz, h, keep_clear=clear_pts)
    partition = (nx // 2, 2, max(2, int(round(26 * nx / 512))), max(2, int(round(51 * nz / 256))))
    return make_room(nx, ny, nz, h=h, ducts=ducts, boxes=boxes, partition=partition, u_in=u_in,
                     name=f"large room {nx}x{ny}x{nz}")


BATCH_NX = (64, 72, 80, 96, 120, 128, 144, 160, 192)
BATCH_NYZ = (64, 72, 80, 96)


def batch_rooms(count=64, seed=4, nx_set=BATCH_NX, nyz_set=BATCH_NYZ):
    """``count`` rooms of uneven sizes (nx >= ny = nz), each with walls, one duct pair, 0-10 seeded boxes and
    U_in uniform in [0.1, 1] m/s, at dx = 0.0390625 m."""
    rng = np.random.default_rng(seed)
    rooms = []
    for i in range(count):
        nyz = int(rng.choice(nyz_set))
        nx = int(rng.choice([n for n in nx_set if n >= nyz]))
        u_in = float(rng.uniform(0.1, 1.0))
        nb = int(rng.integers(0, 11))
        clear_pts = [(2, nyz // 2), (nx - 3, nyz // 2)]
        boxes = random_boxes(rng, nb, nx, nyz, nyz, DX_ROOM, side_m=(0.3, 1.0), keep_clear=clear_pts, clear_m=0.5)
        rooms.append(make_room(nx, nyz, nyz, h=DX_ROOM, boxes=boxes, u_in=u_in, name=f"batch room {i}"))
    return rooms


def request_trace(count=256, seed=5, rate_per_s=4.0, sizes=None, step_range=(200, 2000)):
    """Poisson-arrival ventilation requests: list of dicts (arrival_s, nx, ny, nz, u_in, steps, n_boxes, seed)."""
    rng = np.random.default_rng(seed)
    if sizes is None:
        sizes = [(nx, n, n) for n in BATCH_NYZ for nx in BATCH_NX if nx >= n] + [(256, 128, 128)]
    t = 0.0
    reqs = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate_per_s))
        nx, ny, nz = sizes[int(rng.integers(0, len(sizes)))]
        reqs.append(dict(id=i, arrival_s=t, nx=nx, ny=ny, nz=nz, u_in=float(rng.choice([0.1, 1.0])),
                         steps=int(rng.integers(step_range[0], step_range[1] + 1)),
                         n_boxes=int(rng.integers(0, 11)), seed=int(rng.integers(0, 2 ** 31 - 1))))
    return reqs


def request_room(req):
    """The room of one request from ``request_trace``."""
    rng = np.random.default_rng(req["seed"])
    nx, ny, nz = req["nx"], req["ny"], req["nz"]
    boxes = random_boxes(rng, req["n_boxes"], nx, ny, nz, DX_ROOM, side_m=(0.3, 1.0),
                         keep_clear=[(2, ny // 2), (nx - 3, ny // 2)], clear_m=0.5)
    return make_room(nx, ny, nz, h=DX_ROOM, boxes=boxes, u_in=req["u_in"], name=f"request {req['id']}")


def taylor_green(n=32, length=2.0 * math.pi):
    """Taylor-Green initial velocity u = sin x cos y cos z, v = -cos x sin y cos z, w = 0 on [0, L)^3, cell
    centres at i * L / n.  Returns (u, v, w) of shape (n, n, n)."""
    x = np.arange(n) * (length / n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    u = np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -np.cos(X) * np.sin(Y) * np.cos(Z)
    w = np.zeros_like(u)
    return u, v, w


def random_fields(shape, seed, count=4, scale=1.0, beta=None):
    """``count`` seeded standard-normal fields of ``shape`` times ``scale``, zeroed where beta == 0."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        f = scale * rng.standard_normal(shape)
        if beta is not None:
            f = f * (beta > 0)
        out.append(f)
    return out


def random_mask(shape, seed, solid_fraction=0.2, n_boxes=4):
    """Seeded random geometry for small parity cases: a few solid boxes plus scattered solid cells, as uint8."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    beta = np.ones(shape, dtype=np.uint8)
    for _ in range(n_boxes):
        sx, sy, sz = (int(rng.integers(1, max(2, n // 3))) for n in (nx, ny, nz))
        x0, y0, z0 = int(rng.integers(0, nx)), int(rng.integers(0, ny)), int(rng.integers(0, nz))
        xs = (np.arange(sx) + x0) % nx
        ys = (np.arange(sy) + y0) % ny
        zs = (np.arange(sz) + z0) % nz
        beta[np.ix_(zs, ys, xs)] = 0
    beta[rng.random(shape) < solid_fraction * 0.1] = 0
    return beta


@dataclass
class CubeChannel:
    """The cube-in-channel case of Sec. 3.1.2 (Tab. 1, right column), made periodic in z with nz cells so that the
    3D solver computes the 2D flow: a channel of width D = 2 pi between solid walls, a square obstacle of side
    h = D/6 centred at (1.2 D, D/2), a forcing strip at the left end imposing the parabolic profile
    U(y) = U_max 4 eta (1 - eta) (eta = distance from the lower wall / D), obstacle Reynolds number
    Re_ob = U_b h / nu with U_b = 2/3 U_max.  Cell sizes are h / cells_per_h in x and y; nx and ny are the
    nearest 2-3-5 smooth sizes to the paper's 8.8 D x 1.1 D (walls at least 0.05 D thick)."""

    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    lz: float
    beta: np.ndarray
    S: np.ndarray
    targets: tuple          # (u_set, v_set, w_set, c_set) per cell
    cube: np.ndarray        # uint8 mask of the obstacle's cells
    u_init: np.ndarray      # the parabolic profile in the channel, 0 in solids
    nu: float
    dt: float
    h_obstacle: float
    u_bulk: float
    probe: tuple            # (z, y, x) of the wake probe, 2 h behind the obstacle on the centre line
    wall: int
    cells_per_h: int

    @property
    def cells(self):
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


def cube_channel(cells_per_h=30, nz=8, u_max=1.0, re_ob=84.0, courant=0.2, force_width_h=0.5):
    D = 2.0 * math.pi
    c = int(cells_per_h)
    dx = D / 6.0 / c
    width = 6 * c                                   # channel cells
    wall = int(math.ceil(0.05 * width))
    while not smooth235(width + 2 * wall):
        wall += 1
    ny = width + 2 * wall
    nx = int(math.ceil(8.8 * width))
    while not smooth235(nx):
        nx += 1
    shape = (nz, ny, nx)
    beta = np.ones(shape, dtype=np.uint8)
    beta[:, :wall, :] = 0
    beta[:, wall + width:, :] = 0
    cube = np.zeros(shape, dtype=np.uint8)
    x0 = int(round(1.2 * width - c / 2))
    y0 = wall + (width - c) // 2
    cube[:, y0:y0 + c, x0:x0 + c] = 1
    beta[cube == 1] = 0
    # parabolic profile across the channel, the walls' surfaces half a cell outside the first fluid centres
    eta = (np.arange(ny) - (wall - 0.5)) / width
    prof = np.where((eta > 0.0) & (eta < 1.0), u_max * 4.0 * eta * (1.0 - eta), 0.0)
    u_prof = np.broadcast_to(prof[None, :, None], shape).astype(np.float64) * (beta > 0)
    S = np.zeros(shape, dtype=np.float64)
    nf = max(2, int(round(force_width_h * c)))
    S[:, wall:wall + width, :nf] = 1.0
    zero = np.zeros(shape)
    targets = (u_prof * (S > 0), zero, zero, zero)
    u_b = 2.0 / 3.0 * u_max
    h = D / 6.0
    nu = u_b * h / re_ob
    probe = (nz // 2, wall + width // 2, x0 + 3 * c)
    return CubeChannel(nx, ny, nz, nx * dx, ny * dx, nz * dx, beta, S, targets, cube, u_prof, nu,
                       courant * dx / u_max, h, u_b, probe, wall, c)
