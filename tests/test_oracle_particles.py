"""Pins of the oracle's Lagrangian particles (Sec. 2.3).

Fixed by: the interpolation's exactness on cell values and on linear fields; the paper's printed sedimentation
times; the closed form of the implicit-Euler recurrence; relaxation to a uniform flow; deposition on a floor; the
drag law at Reynolds numbers with integer 2/3 powers and one step at a slip Reynolds number of 27."""
import json
import os

import numpy as np
import pytest

from oracle import flow as F
from oracle import particles as P

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
NU = 1.6e-5
RHO_P, RHO_F = 1000.0, 1.2


def prm_box(nx=12, ny=10, nz=16, h=0.25):
    return F.Params(nx=nx, ny=ny, nz=nz, lx=nx * h, ly=ny * h, lz=nz * h, nu=NU, dt=0.01)


def test_trilinear_at_cell_centres_and_on_linear_fields():
    prm = prm_box()
    rng = np.random.default_rng(0)
    f = rng.standard_normal(prm.shape)
    idx = np.stack([rng.integers(0, n, 20) for n in (prm.nx, prm.ny, prm.nz)], axis=1)
    pos = idx * np.array(prm.h)
    assert np.array_equal(P.trilinear(f, prm, pos), f[idx[:, 2], idx[:, 1], idx[:, 0]])
    # a linear field is reproduced exactly between the centres (away from the periodic seam)
    x = np.arange(prm.nx) * prm.h[0]
    y = np.arange(prm.ny) * prm.h[1]
    z = np.arange(prm.nz) * prm.h[2]
    lin = 0.3 + 1.7 * x[None, None, :] - 0.4 * y[None, :, None] + 2.2 * z[:, None, None]
    pts = np.stack([rng.uniform(0, (n - 1) * hh, 50) for n, hh in zip((prm.nx, prm.ny, prm.nz), prm.h)], axis=1)
    expect = 0.3 + 1.7 * pts[:, 0] - 0.4 * pts[:, 1] + 2.2 * pts[:, 2]
    assert np.allclose(P.trilinear(lin, prm, pts), expect, rtol=0, atol=1e-12)


def test_paper_sedimentation_times():
    sed = GOLDEN["sedimentation"]
    for d_um, printed in zip(sed["diameters_um"], sed["sedimentation_time_min_printed"]):
        v = P.terminal_velocity(d_um * 1e-6, RHO_P, RHO_F, NU)
        minutes = sed["height_m"] / v / 60.0
        assert abs(minutes - printed) / printed < 0.05, (d_um, minutes)


def test_still_air_fall_time_matches_sedimentation_time():
    """A 10 um particle released at rest in still air falls 1.5 m in h / v* (dt = 1 s >> tau_p: implicit Euler is
    stable and sits on the terminal velocity, to the small Re_p correction of C_d)."""
    prm = F.Params(nx=8, ny=8, nz=8, lx=4.0, ly=4.0, lz=4.0, nu=NU, dt=1.0)
    zero = np.zeros(prm.shape)
    d = np.array([10e-6])
    pos = np.array([[2.0, 2.0, 3.0]])
    vel = np.zeros((1, 3))
    dep = np.zeros(1, dtype=bool)
    v_star = P.terminal_velocity(d[0], RHO_P, RHO_F, NU)
    steps = int(round(1.5 / v_star))
    for _ in range(steps):
        pos, vel, dep = P.particle_step(pos, vel, d, dep, zero, zero, zero, np.ones(prm.shape), prm, 1.0, RHO_P,
                                        RHO_F, (0.0, 0.0, -9.81))
    # C_d - 1 = Re^(2/3) / 6 = 0.24 % at Re_p = 1.8e-3 slows the fall; the step count rounds h / v* to 0.06 %
    assert abs((3.0 - pos[0, 2]) - 1.5) / 1.5 < 5e-3
    assert vel[0, 2] == pytest.approx(-v_star, rel=3e-3)


def test_implicit_euler_recurrence_closed_form():
    """From rest in still air: u_n = u_inf (1 - (1 + a)^-n), u_inf = g tau_p / C_d, a = dt C_d / tau_p (C_d held
    fixed by the tiny particle Reynolds number)."""
    prm = prm_box()
    zero = np.zeros(prm.shape)
    d = np.array([5e-6])                           # Re_p <= 2.2e-4: C_d - 1 <= 6e-4
    tau = P.relaxation_time(d[0], RHO_P, RHO_F, NU)
    dt = 0.2 * tau
    pos, vel, dep = np.array([[1.0, 1.0, 2.0]]), np.zeros((1, 3)), np.zeros(1, dtype=bool)
    a = dt / tau
    for n in range(1, 6):
        pos, vel, dep = P.particle_step(pos, vel, d, dep, zero, zero, zero, np.ones(prm.shape), prm, dt, RHO_P,
                                        RHO_F, (0.0, 0.0, -9.81))
        expect = -9.81 * tau * (1.0 - (1.0 + a) ** (-n))
        assert vel[0, 2] == pytest.approx(expect, rel=1e-3)


def test_relaxes_to_uniform_flow():
    prm = prm_box()
    U = (0.4, -0.1, 0.05)
    u, v, w = (np.full(prm.shape, c) for c in U)
    d = np.array([20e-6, 50e-6])
    pos, vel, dep = np.array([[1.0, 1.0, 1.0], [2.0, 0.5, 3.0]]), np.zeros((2, 3)), np.zeros(2, dtype=bool)
    for _ in range(200):
        pos, vel, dep = P.particle_step(pos, vel, d, dep, u, v, w, np.ones(prm.shape), prm, 0.01, RHO_P, RHO_F,
                                        (0.0, 0.0, 0.0))
    assert np.allclose(vel, np.array(U)[None, :], rtol=0, atol=1e-12)


def test_deposits_on_a_floor():
    prm = prm_box()
    beta = np.ones(prm.shape)
    beta[0:2, :, :] = 0.0                          # solid floor, z = 0, 1
    zero = np.zeros(prm.shape)
    d = np.array([100e-6])
    pos, vel, dep = np.array([[1.0, 1.0, 1.2]]), np.zeros((1, 3)), np.zeros(1, dtype=bool)
    for _ in range(400):
        pos, vel, dep = P.particle_step(pos, vel, d, dep, zero, zero, zero, beta, prm, 0.01, RHO_P, RHO_F,
                                        (0.0, 0.0, -9.81))
    assert dep[0] and np.all(vel == 0.0)
    k = int(np.floor(pos[0, 2] / prm.h[2] + 0.5))
    assert beta[k, 4, 4] == 1.0 and pos[0, 2] < 0.7    # stopped in the last fluid cell above the floor


def test_drag_law_special_values():
    """C_d = 1 + Re_p^(2/3) / 6 (Sec. 2.3) at Reynolds numbers whose 2/3 power is an integer: Stokes drag at 0,
    5/3 at 8, 5/2 at 27, 1 + 100/6 at 1000 (a wrong exponent or coefficient misses all but the first)."""
    re = np.array([0.0, 8.0, 27.0, 1000.0])
    assert P.drag_coefficient(re) == pytest.approx([1.0, 5.0 / 3.0, 2.5, 1.0 + 100.0 / 6.0], rel=1e-14)


def test_step_uses_drag_at_the_start_of_step_slip():
    """A particle at rest in a uniform stream whose slip Reynolds number is 27: one implicit Euler step gives
    u_p' = a U / (1 + a) with a = dt C_d / tau_p and C_d = 5/2 taken at the starting slip (the reading of Sec. 2.3's
    implicit Euler with a nonlinear drag); dropping the Re correction (C_d = 1) or taking C_d at the new slip
    fails this."""
    prm = prm_box()
    d = 100e-6
    U = 27.0 * NU / d                               # slip Reynolds number U d / nu = 27
    u = np.full(prm.shape, U)
    zero = np.zeros(prm.shape)
    tau = RHO_P * d * d / (18.0 * RHO_F * NU)       # Sec. 2.3's relaxation time
    dt = 0.05 * tau
    a = dt * 2.5 / tau
    pos, vel, dep = P.particle_step(np.array([[1.0, 1.0, 2.0]]), np.zeros((1, 3)), np.array([d]),
                                    np.zeros(1, dtype=bool), u, zero, zero, np.ones(prm.shape), prm, dt, RHO_P,
                                    RHO_F, (0.0, 0.0, 0.0))
    assert vel[0, 0] == pytest.approx(a * U / (1.0 + a), rel=1e-12)
    assert vel[0, 1] == 0.0 and vel[0, 2] == 0.0
    assert pos[0, 0] == pytest.approx(1.0 + dt * a * U / (1.0 + a), rel=1e-12)
