"""Plain FP64 CPU oracle of the DNSLABIB incompressible-flow time step (Korhonen et al., arXiv 2204.02107).

TEST INFRASTRUCTURE ONLY. This module is imported by ``tests/``, by ``__graft_entry__.smoke()`` and by the CPU
baseline leg of ``bench.py``; the library path never imports, links or runs it.  It shares no code with the CUDA
path: both sides only meet at the seeded input arrays.

Everything here is written for a reader who checks it against the paper by eye: numpy float64, one operator per
function, ``np.roll`` for the periodic neighbours, ``numpy.fft`` as the FFT primitive, no fusion, no blocking.

Array convention: every field is a float64 array of shape (nz, ny, nx), so C order gives the linear cell index
``x + nx*(y + ny*z)``.  Array axis 2 is x, axis 1 is y, axis 0 is z.  Cell centres sit at ``x_i = i*dx`` on a
periodic domain of length ``lx = nx*dx`` (likewise for y and z).

Readings of the paper that this file commits to (each is restated where it is used):
  * Classic four-stage RK4 (Butcher nodes 0, 1/2, 1/2, 1; weights 1/6, 1/3, 1/3, 1/6) for u, v, w and c, with no
    pressure term inside the stages and one projection per step (Sec. 2.1).
  * Collocated central differences: delta f = (f[i+1] - f[i-1]) / (2h), delta2 f = (f[i+1] - 2 f[i] + f[i-1]) / h^2.
    The FFT solver inverts the symbol of D o G, i.e. lambda = -sum_j sin^2(2 pi k_j / n_j) / h_j^2; the eight modes
    with every k_j in {0, n_j/2} have lambda = 0 and get p_hat = 0 (Sec. 2.2, Eq. 9).
  * Every stored field is exactly zero in solid cells: stage right-hand sides are multiplied by beta and the
    projection writes u = beta (u* - grad p) (Sec. 2.1, Eq. 4 and the remark that velocities are multiplied by beta).
  * Scalar transport in flux form with face weight beta_f = beta_i beta_{i+1} on both the convective and the
    diffusive flux, so no flux crosses a fluid/solid face (Eq. 3 and the Neumann condition in Eq. 4).
  * Sixth-order filter phi + sum_i pi^-6 S6_i phi with S6 = (1, -6, 15, -20, 15, -6, 1), i.e. gamma = dx^6 / pi^6
    applied to the 7-point sixth difference; applied after the projection to u, v, w, c, then re-masked (Eq. 6).
  * tau_f <= 0 means tau_f = dt.  The reported pressure is the internal p divided by dt (u = u* - grad p has no dt).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
import math

import numpy as np

# array axis of each physical direction: x -> 2, y -> 1, z -> 0
AXES = (2, 1, 0)

# 7-point sixth difference (1, -6, 15, -20, 15, -6, 1) = (E - 2 + E^-1)^3, offsets -3..3 (Eq. 6)
S6_COEFFS = (1.0, -6.0, 15.0, -20.0, 15.0, -6.0, 1.0)

HIST_BINS = 64


@dataclass(frozen=True)
class Params:
    """Case parameters of one grid (Sec. 2.4: the SetParameters / CreateGeometry inputs)."""

    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    lz: float
    nu: float
    dt: float
    alpha_c: float | None = None      # None -> nu (Schmidt number 1; the paper does not give alpha_c)
    tau_f: float = 0.0                # <= 0 -> dt
    body_force: tuple = (0.0, 0.0, 0.0)
    u_set: tuple = (0.0, 0.0, 0.0)
    c_set: float = 0.0
    n_pressure_iters: int = 4         # the paper's hard-coded n (Sec. 2.2)
    filter: bool = True

    @property
    def h(self):
        return (self.lx / self.nx, self.ly / self.ny, self.lz / self.nz)

    @property
    def cell_volume(self):
        hx, hy, hz = self.h
        return hx * hy * hz

    @property
    def tau(self):
        return self.tau_f if self.tau_f > 0.0 else self.dt

    @property
    def alpha(self):
        return self.nu if self.alpha_c is None else self.alpha_c

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def with_(self, **kw):
        return replace(self, **kw)


@dataclass
class State:
    """Fields of one grid: velocity, scalar, pressure (internal, = dt * p_phys / rho), time and step count."""

    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    c: np.ndarray
    p: np.ndarray
    t: float = 0.0
    step: int = 0

    def copy(self):
        return State(self.u.copy(), self.v.copy(), self.w.copy(), self.c.copy(), self.p.copy(), self.t, self.step)


@dataclass
class Geometry:
    """Binary masks (Sec. 2.1): beta = 1 fluid / 0 solid, S = 1 forcing region / 0 elsewhere, room = cells that
    count for the room inventory, volume and histogram."""

    beta: np.ndarray
    S: np.ndarray
    room: np.ndarray = field(default=None)

    def __post_init__(self):
        self.beta = np.asarray(self.beta, dtype=np.float64)
        self.S = np.asarray(self.S, dtype=np.float64)
        if self.room is None:
            self.room = self.beta.copy()
        self.room = np.asarray(self.room, dtype=np.float64)


# ----------------------------------------------------------------------------------------------------------------
# Difference operators (Sec. 2.1: second-order central differences)
# ----------------------------------------------------------------------------------------------------------------

def shift(f, offset, axis):
    """Periodic neighbour: shift(f, +1, axis)[i] = f[i+1]."""
    return np.roll(f, -offset, axis)


def delta(f, axis, h):
    """Central first difference (f[i+1] - f[i-1]) / (2h)."""
    return (shift(f, 1, axis) - shift(f, -1, axis)) / (2.0 * h)


def delta2(f, axis, h):
    """Central second difference (f[i+1] - 2 f[i] + f[i-1]) / h^2."""
    return (shift(f, 1, axis) - 2.0 * f + shift(f, -1, axis)) / (h * h)


def sixth_difference(f, axis):
    """Undivided 7-point sixth difference sum_m S6[m] f[i+m], m = -3..3 (Eq. 6 with dx^6 folded into gamma)."""
    out = np.zeros_like(f)
    for m, coef in zip(range(-3, 4), S6_COEFFS):
        out += coef * shift(f, m, axis)
    return out


# ----------------------------------------------------------------------------------------------------------------
# Stage right-hand sides (Eqs. 2-4)
# ----------------------------------------------------------------------------------------------------------------

def momentum_rhs(u, v, w, geom: Geometry, prm: Params):
    """Right-hand side of Eq. 2 without the pressure gradient, masked by beta.

    Convection in skew-symmetric form 1/2 [ d_j(u_j u_i) + u_j d_j u_i ] (Sec. 2.1), diffusion nu sum_j d2_j u_i,
    relaxation forcing S (u_set,i - u_i) / tau_f, body force b_i; the sum is multiplied by beta (Eq. 4).
    """
    vel = (u, v, w)
    h = prm.h
    out = []
    for i in range(3):
        ui = vel[i]
        conv = np.zeros_like(ui)
        diff = np.zeros_like(ui)
        for j in range(3):
            uj = vel[j]
            conv += 0.5 * (delta(uj * ui, AXES[j], h[j]) + uj * delta(ui, AXES[j], h[j]))
            diff += delta2(ui, AXES[j], h[j])
        rhs = -conv + prm.nu * diff + geom.S * (prm.u_set[i] - ui) / prm.tau + prm.body_force[i]
        out.append(geom.beta * rhs)
    return out


def scalar_rhs(c, u, v, w, geom: Geometry, prm: Params):
    """Right-hand side of Eq. 3, masked by beta.

    Flux form: the face value at i+1/2 along direction j is F = beta_i beta_{i+1} * (u_j c |_i + u_j c |_{i+1}) / 2
    and the diffusive flux is alpha_c beta_i beta_{i+1} (c_{i+1} - c_i) / h_j, so nothing crosses a fluid/solid face
    (dc/dn = 0 at solids, Eq. 4).  Forcing S (c_set - c) / tau_f.
    """
    vel = (u, v, w)
    h = prm.h
    total = np.zeros_like(c)
    for j in range(3):
        ax = AXES[j]
        beta_face = geom.beta * shift(geom.beta, 1, ax)              # weight of face i+1/2
        uc = vel[j] * c
        conv_flux = beta_face * 0.5 * (uc + shift(uc, 1, ax))       # F_{i+1/2}
        diff_flux = beta_face * (shift(c, 1, ax) - c) / h[j]         # beta_f dc/dx_j at i+1/2
        total += -(conv_flux - shift(conv_flux, -1, ax)) / h[j]
        total += prm.alpha * (diff_flux - shift(diff_flux, -1, ax)) / h[j]
    total += geom.S * (prm.c_set - c) / prm.tau
    return geom.beta * total


def stage_rhs(q, geom, prm):
    """(k_u, k_v, k_w, k_c) at stage state q = (u, v, w, c)."""
    ku, kv, kw = momentum_rhs(q[0], q[1], q[2], geom, prm)
    kc = scalar_rhs(q[3], q[0], q[1], q[2], geom, prm)
    return [ku, kv, kw, kc]


RK4_NODES = (0.0, 0.5, 0.5, 1.0)
RK4_WEIGHTS = (1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0)


def room_outflow_rate(c, u, v, w, geom: Geometry, prm: Params):
    """Rate at which the scalar leaves the room region through its boundary (the outlet and inlet openings of a
    ventilated room, Sec. 3.3): over every face between a room cell and a cell outside the room, the face flux of
    Eq. 3 in the flux form of scalar_rhs -- convective beta_f (u_j c |_i + u_j c |_{i+1}) / 2 minus diffusive
    alpha_c beta_f (c_{i+1} - c_i) / h_j -- times the face area dV / h_j, counted positive out of the room."""
    vel = (u, v, w)
    h = prm.h
    room = geom.room
    total = 0.0
    for j in range(3):
        ax = AXES[j]
        beta_face = geom.beta * shift(geom.beta, 1, ax)
        uc = vel[j] * c
        flux = beta_face * (0.5 * (uc + shift(uc, 1, ax)) - prm.alpha * (shift(c, 1, ax) - c) / h[j])  # i -> i+1
        room_next = shift(room, 1, ax)
        # +1 where the face leads out of the room (i inside, i+1 outside), -1 where it leads in
        sign = room * (1.0 - room_next) - (1.0 - room) * room_next
        total += prm.cell_volume / h[j] * float(np.sum(sign * flux))
    return total


def rk4_predictor(q, geom, prm, record=None):
    """Classic RK4 over (u, v, w, c) with no pressure term inside the stages: returns q* (Sec. 2.1).

    If ``record`` is a dict, the scalar budget terms of the step are stored in it, each the RK-weighted sum
    dt * sum_s b_s X_s over the four stage states: 'forcing', the inventory the relaxation source adds
    (X_s = sum_cells beta S (c_set - c_s) / tau_f dV); 'forcing_room', the same over the room cells; 'outflow',
    what leaves the room through its boundary (X_s = room_outflow_rate at stage state s)."""
    dt = prm.dt
    ks = []
    stage_q = q
    for s in range(4):
        if s > 0:
            stage_q = [qn + RK4_NODES[s] * dt * k for qn, k in zip(q, ks[-1])]
        ks.append(stage_rhs(stage_q, geom, prm))
        if record is not None:
            src = geom.beta * geom.S * (prm.c_set - stage_q[3]) / prm.tau
            weight = dt * RK4_WEIGHTS[s]
            record['forcing'] = record.get('forcing', 0.0) + weight * float(np.sum(src)) * prm.cell_volume
            record['forcing_room'] = (record.get('forcing_room', 0.0)
                                      + weight * float(np.sum(geom.room * src)) * prm.cell_volume)
            record['outflow'] = record.get('outflow', 0.0) + weight * room_outflow_rate(
                stage_q[3], stage_q[0], stage_q[1], stage_q[2], geom, prm)
    return [qn + dt * sum(b * k[f] for b, k in zip(RK4_WEIGHTS, ks)) for f, qn in enumerate(q)]


# ----------------------------------------------------------------------------------------------------------------
# Pressure (Sec. 2.2, Eqs. 7-9)
# ----------------------------------------------------------------------------------------------------------------

def divergence(u, v, w, prm: Params):
    """Discrete divergence D u = sum_j delta_j u_j."""
    h = prm.h
    return delta(u, AXES[0], h[0]) + delta(v, AXES[1], h[1]) + delta(w, AXES[2], h[2])


def wavenumbers(n):
    """Integer wavenumbers k = 0..n-1 in numpy.fft order (k and k - n are the same mode)."""
    return np.arange(n)


def laplacian_symbol(prm: Params):
    """lambda(k) = -sum_j sin^2(2 pi k_j / n_j) / h_j^2: the Fourier symbol of D o G with central D and G.

    Shape (nz, ny, nx), numpy.fft ordering on each axis."""
    hx, hy, hz = prm.h
    lx = np.sin(2.0 * np.pi * wavenumbers(prm.nx) / prm.nx) ** 2 / hx ** 2
    ly = np.sin(2.0 * np.pi * wavenumbers(prm.ny) / prm.ny) ** 2 / hy ** 2
    lz = np.sin(2.0 * np.pi * wavenumbers(prm.nz) / prm.nz) ** 2 / hz ** 2
    return -(lz[:, None, None] + ly[None, :, None] + lx[None, None, :])


def null_modes(prm: Params):
    """Boolean (nz, ny, nx): the eight modes with every k_j in {0, n_j/2}, where the symbol is exactly zero."""
    def on_axis(n):
        k = wavenumbers(n)
        return (k == 0) | (2 * k == n)
    return on_axis(prm.nz)[:, None, None] & on_axis(prm.ny)[None, :, None] & on_axis(prm.nx)[None, None, :]


def poisson_fft_solve(f, prm: Params):
    """p = FFT^-1[ FFT(f) / lambda ] with p_hat = 0 on the null modes (forward FFT, division by the discrete
    Laplacian eigenvalues, inverse FFT)."""
    lam = laplacian_symbol(prm)
    null = null_modes(prm)
    fhat = np.fft.fftn(f)
    safe = np.where(null, 1.0, lam)
    phat = np.where(null, 0.0, fhat / safe)
    return np.fft.ifftn(phat).real


def pressure_rhs(r, pk, geom: Geometry, prm: Params):
    """Right-hand side of Eq. 9: f = D u* + sum_j delta_j((1 - beta) delta_j p^k), by central differences."""
    h = prm.h
    solid = 1.0 - geom.beta
    f = r.copy()
    for j in range(3):
        f += delta(solid * delta(pk, AXES[j], h[j]), AXES[j], h[j])
    return f


def pressure_iterations(r, p0, geom, prm: Params, n=None):
    """Iterate Eq. 9 n times from p^0 (the previous step's pressure)."""
    n = prm.n_pressure_iters if n is None else n
    p = p0
    for _ in range(n):
        p = poisson_fft_solve(pressure_rhs(r, p, geom, prm), prm)
    return p


def project(ustar, vstar, wstar, p, geom: Geometry, prm: Params):
    """Velocity correction u = beta (u* - grad p) with central grad (Eq. 8, masked by beta)."""
    h = prm.h
    return [geom.beta * (us - delta(p, AXES[i], h[i])) for i, us in enumerate((ustar, vstar, wstar))]


# ----------------------------------------------------------------------------------------------------------------
# Filter (Eq. 6)
# ----------------------------------------------------------------------------------------------------------------

def filter6(f, geom: Geometry):
    """phi_bar = beta (phi + sum_i pi^-6 S6_i phi): gamma_i = dx_i^6 / pi^6 times the 7-point sixth difference
    divided by dx_i^6, summed over the three axes, then re-masked."""
    out = f.copy()
    for ax in AXES:
        out += sixth_difference(f, ax) / math.pi ** 6
    return geom.beta * out


# ----------------------------------------------------------------------------------------------------------------
# Reductions (Sec. 3.3: mean CO2, its spread, the CO2 distribution; divergence and energy diagnostics)
# ----------------------------------------------------------------------------------------------------------------

def histogram(c, room):
    """64 bins over c in [0, 1] for room cells: bin = min(floor(64 c), 63); c < 0 and c > 1 go to separate
    under/over counters.  Returns (counts[64], under, over)."""
    vals = c[room > 0.5]
    under = int(np.count_nonzero(vals < 0.0))
    over = int(np.count_nonzero(vals > 1.0))
    inside = vals[(vals >= 0.0) & (vals <= 1.0)]
    bins = np.minimum(np.floor(inside * HIST_BINS).astype(np.int64), HIST_BINS - 1)
    counts = np.bincount(bins, minlength=HIST_BINS)
    return counts, under, over


def reductions(state: State, geom: Geometry, prm: Params, div_velocity=None):
    """Diagnostics of a state, all in FP64.  The divergence is that of ``div_velocity`` (u, v, w) when given,
    else of the state's velocity."""
    dV = prm.cell_volume
    u, v, w, c = state.u, state.v, state.w, state.c
    div = divergence(*(div_velocity if div_velocity is not None else (u, v, w)), prm)
    counts, under, over = histogram(c, geom.room)
    room = geom.room
    return {
        't': state.t,
        'step': state.step,
        'ke': 0.5 * dV * float(np.sum(u * u + v * v + w * w)),
        'div_max': float(np.max(np.abs(div))),
        'div_l2': math.sqrt(dV * float(np.sum(div * div))),
        'u_max': float(max(np.max(np.abs(u)), np.max(np.abs(v)), np.max(np.abs(w)))),
        'c_total': dV * float(np.sum(c)),
        'c_room': dV * float(np.sum(room * c)),
        'c2_room': dV * float(np.sum(room * c * c)),
        'v_room': dV * float(np.sum(room)),
        'hist': counts,
        'hist_under': under,
        'hist_over': over,
    }


# ----------------------------------------------------------------------------------------------------------------
# One time step (Sec. 2.4 main loop: RK4 momentum + scalar, projection, filter)
# ----------------------------------------------------------------------------------------------------------------

def step(state: State, geom: Geometry, prm: Params, with_budget=False):
    """Advance one time step; returns (new_state, record).

    Order: RK4 predictor on (u, v, w, c) -> r = D u* -> n iterations of Eq. 9 warm-started from the previous p ->
    u = beta (u* - grad p) -> sixth-order filter of u, v, w, c and re-mask (if enabled) -> reductions of the new
    state, whose divergence entries are those of the projected velocity (before the filter)."""
    budget = {} if with_budget else None
    q = [state.u, state.v, state.w, state.c]
    us, vs, ws, cs = rk4_predictor(q, geom, prm, record=budget)
    r = divergence(us, vs, ws, prm)
    p = pressure_iterations(r, state.p, geom, prm)
    u, v, w = project(us, vs, ws, p, geom, prm)
    projected = (u, v, w)
    c = cs
    if budget is not None:
        budget['c_star_total'] = prm.cell_volume * float(np.sum(cs))
    if prm.filter:
        if budget is not None:
            # what the filter adds before the re-mask: removed again in solids, kept in the room's fluid cells
            change = sum(sixth_difference(cs, ax) for ax in AXES) / math.pi ** 6
            budget['mask_loss'] = prm.cell_volume * float(np.sum((1.0 - geom.beta) * (cs + change)))
            budget['filter_room'] = prm.cell_volume * float(np.sum(geom.room * geom.beta * change))
        u, v, w, c = (filter6(f, geom) for f in (u, v, w, c))
    elif budget is not None:
        budget['mask_loss'] = 0.0
        budget['filter_room'] = 0.0
    new = State(u, v, w, c, p, state.t + prm.dt, state.step + 1)
    # the step's divergence diagnostic measures the projection: D u right after it, before the filter (Sec. 2.2)
    rec = reductions(new, geom, prm, div_velocity=projected)
    if budget is not None:
        rec.update(budget)
    return new, rec


def run(state: State, geom: Geometry, prm: Params, n_steps: int, with_budget=False):
    """n_steps steps; returns (final state, list of per-step records)."""
    recs = []
    for _ in range(n_steps):
        state, rec = step(state, geom, prm, with_budget=with_budget)
        recs.append(rec)
    return state, recs


# ----------------------------------------------------------------------------------------------------------------
# Force of the immersed boundary on a solid region (the cube-in-channel drag of Sec. 3.1.2)
# ----------------------------------------------------------------------------------------------------------------

def region_force(state: State, geom: Geometry, prm: Params, region):
    """Rate at which the mask removes momentum from the cells of `region` (per unit density): the unmasked
    right-hand side of Eq. 2 there, -convection + nu diffusion + forcing + body force - grad(p/rho), summed
    over the region times the cell volume.  The fluid pushes the body with this force (the drag along the flow
    when the region is an obstacle).  The pressure is the physical p/rho = p/dt of the internal one."""
    vel = (state.u, state.v, state.w)
    h = prm.h
    p_phys = state.p / prm.dt
    region = np.asarray(region, dtype=bool)
    out = []
    for i in range(3):
        ui = vel[i]
        conv = np.zeros_like(ui)
        diff = np.zeros_like(ui)
        for j in range(3):
            uj = vel[j]
            conv += 0.5 * (delta(uj * ui, AXES[j], h[j]) + uj * delta(ui, AXES[j], h[j]))
            diff += delta2(ui, AXES[j], h[j])
        rhs = (-conv + prm.nu * diff + geom.S * (prm.u_set[i] - ui) / prm.tau + prm.body_force[i]
               - delta(p_phys, AXES[i], h[i]))
        out.append(prm.cell_volume * float(np.sum(rhs[region])))
    return out


# ----------------------------------------------------------------------------------------------------------------
# Smooth source mask (Eq. 5): a window of widths W_j centred at c_j with tanh edges of sharpness B_j
# ----------------------------------------------------------------------------------------------------------------

def tanh_window_factor(d, half_width, sharpness):
    """One axis of Eq. 5: (1 - tanh(B [d / (W/2) - (W/2) / d])) / 2 for the distance d >= 0 to the centre; at d = 0
    the bracket tends to minus infinity and the factor to its limit 1."""
    d = np.asarray(d, dtype=np.float64)
    out = np.ones_like(d)
    nz = d > 0.0
    arg = sharpness * (d[nz] / half_width - half_width / d[nz])
    out[nz] = 0.5 * (1.0 - np.tanh(arg))
    return out


def tanh_source_mask(prm: Params, center, width, sharpness):
    """S(x, y, z) of Eq. 5 on the cell centres x_i = i h_x (likewise y, z).  The paper does not say how the
    distance |x - x_c| meets the periodic boundary; this takes the minimum-image distance, so the mask is
    continuous across the wrap (the same as the plain distance for a window away from the box faces)."""
    lengths = (prm.lx, prm.ly, prm.lz)
    S = np.ones(prm.shape)
    for j, ax in enumerate(AXES):
        n = prm.shape[ax]
        coord = np.arange(n) * prm.h[j]
        d = np.abs(coord - center[j])
        d = np.minimum(d, lengths[j] - d)
        f = tanh_window_factor(d, 0.5 * width[j], sharpness[j])
        shape = [1, 1, 1]
        shape[ax] = n
        S = S * f.reshape(shape)
    return S


# ----------------------------------------------------------------------------------------------------------------
# Dynamic time step (Sec. 2.4: the user sets the maximum Courant number and AdjustDt adapts dt as the flow evolves)
# ----------------------------------------------------------------------------------------------------------------

def courant_rate(state: State, prm: Params):
    """sigma = max over cells of sum_j |u_j| / h_j, so that the advective Courant number of a step is dt * sigma.
    The paper names the maximum Courant number as the control but not its form; this is the three-dimensional
    advective one (the sum over axes, the stricter of the usual choices)."""
    hx, hy, hz = prm.h
    return float(np.max(np.abs(state.u) / hx + np.abs(state.v) / hy + np.abs(state.w) / hz))


def adjust_dt(state: State, prm: Params, courant_max: float):
    """The time step for the next step from the current velocity: dt = min(prm.dt, courant_max / sigma); prm.dt
    is the upper bound (and the step used while the fluid is at rest)."""
    sigma = courant_rate(state, prm)
    if sigma == 0.0:
        return prm.dt
    return min(prm.dt, courant_max / sigma)


def run_adaptive(state: State, geom: Geometry, prm: Params, n_steps: int, courant_max: float):
    """n_steps steps, each with dt = adjust_dt(current state).  The internal pressure carries a factor dt
    (u = u* - grad p has none), so the warm start is rescaled by dt_new / dt_old when dt changes: the physical
    pressure p / dt the next solve starts from is the one the previous step produced.  The incoming state's
    pressure is taken to be relative to prm.dt.  Returns (final state, records with 'dt', dt of the last step)."""
    recs = []
    dt_prev = prm.dt
    for _ in range(n_steps):
        dt = adjust_dt(state, prm, courant_max)
        if dt != dt_prev:
            state = State(state.u, state.v, state.w, state.c, state.p * (dt / dt_prev), state.t, state.step)
        state, rec = step(state, geom, prm.with_(dt=dt))
        rec['dt'] = dt
        recs.append(rec)
        dt_prev = dt
    return state, recs, dt_prev


def physical_pressure(state: State, prm: Params):
    """p / rho in physical units: the internal p carries a factor dt because u = u* - grad p has none."""
    return state.p / prm.dt


def zero_state(prm: Params, c=None):
    z = np.zeros(prm.shape)
    return State(z.copy(), z.copy(), z.copy(), z.copy() if c is None else np.asarray(c, dtype=np.float64), z.copy())


def open_geometry(prm: Params):
    """beta = 1 everywhere, no forcing region."""
    return Geometry(np.ones(prm.shape), np.zeros(prm.shape))
