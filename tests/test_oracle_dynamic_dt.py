"""Pins of the oracle's dynamic time step (Sec. 2.4: the maximum Courant number is the control, AdjustDt adapts dt).

Fixed by closed forms and invariants: the Courant rate of a single moving cell, the time step of a uniform flow
(an exact steady solution of the discrete step), dt at rest, the cap, and the warm-start rescale (a hydrostatic
fluid at rest stays at rest across a change of dt only when the internal pressure is rescaled)."""
import numpy as np
import pytest

from oracle import flow as F


def box(nx=8, ny=12, nz=10, **kw):
    base = dict(nx=nx, ny=ny, nz=nz, lx=0.8, ly=1.5, lz=0.7, nu=1e-3, dt=0.05, filter=True)
    base.update(kw)
    return F.Params(**base)


def test_courant_rate_single_cell():
    prm = box()
    st = F.zero_state(prm)
    hx, hy, hz = prm.h
    st.u[3, 4, 5], st.v[3, 4, 5], st.w[3, 4, 5] = -0.3, 0.2, 0.9
    st.u[1, 1, 1] = 0.01                         # a slower cell elsewhere
    assert F.courant_rate(st, prm) == pytest.approx(0.3 / hx + 0.2 / hy + 0.9 / hz, rel=1e-15)


def test_uniform_flow_dt_closed_form_and_steady():
    """A uniform velocity in a fully fluid periodic box is an exact steady solution (every central difference of a
    constant is zero); dt = courant_max / (|U|/hx + |V|/hy + |W|/hz) at every step and t advances by it."""
    prm = box(filter=True)
    U = (0.7, -0.2, 0.1)
    st = F.State(np.full(prm.shape, U[0]), np.full(prm.shape, U[1]), np.full(prm.shape, U[2]),
                 np.linspace(0.0, 1.0, np.prod(prm.shape)).reshape(prm.shape), np.zeros(prm.shape))
    geom = F.open_geometry(prm)
    hx, hy, hz = prm.h
    cmax = 0.35
    expect = cmax / (0.7 / hx + 0.2 / hy + 0.1 / hz)
    assert expect < prm.dt
    end, recs, dt_last = F.run_adaptive(st, geom, prm, 5, cmax)
    assert [r['dt'] for r in recs] == [expect] * 5 and dt_last == expect
    assert end.t == pytest.approx(5 * expect, rel=1e-15)
    for a, b in ((end.u, st.u), (end.v, st.v), (end.w, st.w)):
        assert np.max(np.abs(a - b)) <= 1e-15


def test_rest_and_cap_use_the_given_dt():
    prm = box()
    geom = F.open_geometry(prm)
    rest = F.zero_state(prm)
    assert F.adjust_dt(rest, prm, 0.5) == prm.dt
    # a slow flow: the Courant limit is far above prm.dt, so every step takes prm.dt and the run is the fixed one
    rng = np.random.default_rng(4)
    st = F.State(*(1e-3 * rng.standard_normal(prm.shape) for _ in range(3)), np.ones(prm.shape),
                 np.zeros(prm.shape))
    a, ra, _ = F.run_adaptive(st.copy(), geom, prm, 3, 1e6)
    b, rb = F.run(st.copy(), geom, prm, 3)
    assert all(r['dt'] == prm.dt for r in ra)
    for n in ("u", "v", "w", "c", "p"):
        assert np.array_equal(getattr(a, n), getattr(b, n))


def test_courant_number_of_each_step_is_the_maximum():
    """From a random flow the chosen dt times the Courant rate of the state it starts from is courant_max."""
    prm = box(dt=1.0)
    geom = F.open_geometry(prm)
    rng = np.random.default_rng(11)
    st = F.State(*(0.5 * rng.standard_normal(prm.shape) for _ in range(3)), np.ones(prm.shape), np.zeros(prm.shape))
    cmax = 0.3
    for _ in range(3):
        dt = F.adjust_dt(st, prm, cmax)
        assert dt * F.courant_rate(st, prm) == pytest.approx(cmax, rel=1e-14)
        st, _ = F.step(st, geom, prm.with_(dt=dt))


def test_warm_start_rescale_keeps_hydrostatic_rest():
    """Fluid at rest under gravity between solid layers: after reaching the steady state at dt1 the internal
    pressure is dt1 times the hydrostatic p/rho.  Stepping on with dt2 from p * dt2/dt1 keeps the fluid at rest up
    to the O(dt^2) stage terms; from the unscaled p the solve misses the new balance by the factor dt2/dt1."""
    prm = F.Params(nx=8, ny=16, nz=8, lx=8.0, ly=16.0, lz=8.0, nu=0.2, dt=0.05, body_force=(0.0, -1.0, 0.0),
                   filter=False)
    beta = np.ones(prm.shape)
    beta[:, 0:2, :] = 0.0
    geom = F.Geometry(beta, np.zeros(prm.shape))
    st, recs = F.run(F.zero_state(prm), geom, prm, 300)
    assert recs[-1]['u_max'] < 1e-14
    dt2 = 0.03
    scaled = F.State(st.u, st.v, st.w, st.c, st.p * (dt2 / prm.dt), st.t, st.step)
    _, with_rescale = F.step(scaled, geom, prm.with_(dt=dt2))
    _, without = F.step(st, geom, prm.with_(dt=dt2))
    assert without['u_max'] > 1e-3
    assert with_rescale['u_max'] < 1e-2 * without['u_max']
