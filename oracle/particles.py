"""Plain FP64 CPU oracle of the Lagrangian particles of DNSLABIB (Sec. 2.3: one-way coupled, drag and gravity,
implicit Euler).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and never by the library, with which it shares no code.

Equations of motion (Sec. 2.3):  du_p/dt = (C_d / tau_p)(u_f - u_p) + g,  tau_p = rho_p d^2 / (18 rho_f nu),
Re_p = |u_f - u_p| d / nu,  C_d = 1 + Re_p^(2/3) / 6,  dx_p/dt = u_p.

Readings of the paper taken here:
  * d is the particle size that enters tau_p.  The paper calls it the radius, but its sedimentation times
    (36 / 9 / 1 min from 1.5 m for 5 / 10 / 30 um) follow with d the diameter, rho_p = 1000, rho_f = 1.2 kg/m^3.
  * Implicit Euler with the drag coefficient taken from the relative velocity at the start of the step (the drag is
    linear in u_p once C_d is fixed): u_p' = (u_p + a u_f + dt g) / (1 + a), a = dt C_d / tau_p; then x_p' = x_p + dt u_p'.
  * u_f is the fluid velocity at the end of the flow step, interpolated trilinearly between the eight cell centres
    around x_p (cell centres at i h, periodic).
  * Positions wrap periodically.  A particle whose new position lies in a solid cell (nearest cell centre with
    beta = 0) is deposited: it keeps its previous position, its velocity becomes 0 and it never moves again.
"""
from __future__ import annotations

import numpy as np

from .flow import Params


def trilinear(f, prm: Params, pos):
    """Field f (array (nz, ny, nx) on the cell centres) at the points pos (array (n, 3): x, y, z)."""
    h = prm.h
    dims = (prm.nx, prm.ny, prm.nz)
    lo, frac = [], []
    for j in range(3):
        s = pos[:, j] / h[j]
        i0 = np.floor(s)
        frac.append(s - i0)
        lo.append(i0.astype(np.int64) % dims[j])
    out = np.zeros(pos.shape[0])
    for cz in (0, 1):
        wz = frac[2] if cz else 1.0 - frac[2]
        iz = (lo[2] + cz) % dims[2]
        for cy in (0, 1):
            wy = frac[1] if cy else 1.0 - frac[1]
            iy = (lo[1] + cy) % dims[1]
            for cx in (0, 1):
                wx = frac[0] if cx else 1.0 - frac[0]
                ix = (lo[0] + cx) % dims[0]
                out += (wx * wy * wz) * f[iz, iy, ix]
    return out


def relaxation_time(d, rho_p, rho_f, nu):
    """tau_p = rho_p d^2 / (18 rho_f nu) (Sec. 2.3)."""
    return rho_p * d * d / (18.0 * rho_f * nu)


def drag_coefficient(re):
    """C_d = 1 + Re_p^(2/3) / 6 (Sec. 2.3)."""
    return 1.0 + np.power(re, 2.0 / 3.0) / 6.0


def nearest_cell(pos, prm: Params):
    h = prm.h
    dims = (prm.nx, prm.ny, prm.nz)
    return [np.floor(pos[:, j] / h[j] + 0.5).astype(np.int64) % dims[j] for j in range(3)]


def particle_step(pos, vel, d, deposited, u, v, w, beta, prm: Params, dt, rho_p, rho_f, gravity):
    """One implicit-Euler step of every particle; returns (pos, vel, deposited), new arrays."""
    pos = np.asarray(pos, dtype=np.float64)
    vel = np.asarray(vel, dtype=np.float64)
    uf = np.stack([trilinear(u, prm, pos), trilinear(v, prm, pos), trilinear(w, prm, pos)], axis=1)
    rel = uf - vel
    re = np.sqrt(np.sum(rel * rel, axis=1)) * d / prm.nu
    a = dt * drag_coefficient(re) / relaxation_time(d, rho_p, rho_f, prm.nu)
    g = np.asarray(gravity, dtype=np.float64)
    new_vel = (vel + a[:, None] * uf + dt * g[None, :]) / (1.0 + a)[:, None]
    new_pos = pos + dt * new_vel
    lengths = np.array([prm.lx, prm.ly, prm.lz])
    new_pos = np.mod(new_pos, lengths[None, :])
    ix, iy, iz = nearest_cell(new_pos, prm)
    hits = beta[iz, iy, ix] == 0.0
    stop = deposited | hits
    new_pos = np.where(stop[:, None], pos, new_pos)
    new_vel = np.where(stop[:, None], 0.0, new_vel)
    return new_pos, new_vel, stop


def terminal_velocity(d, rho_p, rho_f, nu, g=9.81):
    """v* = g tau_p (Sec. 2.3, the Stokes limit C_d -> 1)."""
    return g * relaxation_time(d, rho_p, rho_f, nu)
