"""Lagrangian particles (Sec. 2.3) on the GPU against the oracle.

Particles advected by the FP64 flow of a masked room, a still-air sedimentation run against the paper's times,
deposition on a solid floor, FP32 sampling, and the dynamic time step driving the particles."""
import numpy as np
import pytest

from oracle import flow as F
from oracle import particles as P
from gpu_helpers import gpu_grid, load_state, require_gpu, room_case

pytestmark = pytest.mark.gpu

RHO_P, RHO_F, G = 1000.0, 1.2, (0.0, 0.0, -9.81)


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def seeded_particles(room, prm, n, seed):
    """n particles in fluid cells at least 3 cells from any solid, sizes 1-100 um (the paper's classes)."""
    rng = np.random.default_rng(seed)
    beta = room.beta.astype(bool)
    inner = beta.copy()
    for ax in range(3):
        for sft in (-3, -2, -1, 1, 2, 3):
            inner &= np.roll(beta, sft, axis=ax)
    cells = np.argwhere(inner)[rng.choice(int(inner.sum()), n, replace=False)]
    h = np.array(prm.h)
    pos = (cells[:, ::-1] + rng.uniform(-0.5, 0.5, (n, 3))) * h
    vel = rng.normal(0.0, 0.05, (n, 3))
    size = np.concatenate([rng.uniform(90e-6, 100e-6, n // 5), rng.uniform(10e-6, 30e-6, n - n // 5 - n // 4),
                           rng.uniform(1e-6, 10e-6, n // 4)])
    return pos, vel, size


def oracle_run(st, geom, prm, pos, vel, size, steps):
    dep = np.zeros(len(size), dtype=bool)
    for _ in range(steps):
        st, _ = F.step(st, geom, prm)
        pos, vel, dep = P.particle_step(pos, vel, size, dep, st.u, st.v, st.w, geom.beta, prm, prm.dt, RHO_P, RHO_F, G)
    return pos, vel, dep


@pytest.mark.parametrize("shape,boxes", [((48, 30, 18), [(20, 26, 12, 20, 2, 9)]),
                                         ((64, 32, 32), [(20, 26, 8, 14, 2, 12)])])
def test_particles_in_room_flow_fp64(torch, shape, boxes):
    room, prm, geom, st0 = room_case(*shape, boxes=boxes, seed=3)
    pos0, vel0, size = seeded_particles(room, prm, 400, seed=7)
    ref_pos, ref_vel, ref_dep = oracle_run(st0.copy(), geom, prm, pos0, vel0, size, 40)
    g = gpu_grid(prm, room.beta, room.S, room.room, "fp64")
    load_state(g, st0, prm)
    g.set_particles(pos0, vel0, size, RHO_P, RHO_F, G)
    g.step(40)
    pos, vel, dep = g.particles()
    g.close()
    assert np.array_equal(dep, ref_dep)
    assert np.max(np.abs(pos - ref_pos)) < 1e-11
    assert np.max(np.abs(vel - ref_vel)) < 1e-10
    assert np.max(np.abs(pos - pos0)) > 1e-3                 # they moved


def test_still_air_sedimentation(torch):
    """5, 10 and 30 um particles released at rest 1.5 m above the floor of an open box of still air: after the
    paper's sedimentation time of each (h / v*) it has fallen 1.5 m (to the C_d correction)."""
    prm = F.Params(nx=16, ny=16, nz=16, lx=4.0, ly=4.0, lz=4.0, nu=1.6e-5, dt=1.0, filter=False)
    geom = F.open_geometry(prm)
    size = np.array([5e-6, 10e-6, 30e-6])
    pos0 = np.array([[1.0, 1.0, 3.0], [2.0, 2.0, 3.0], [3.0, 3.0, 3.0]])
    g = gpu_grid(prm, geom.beta, geom.S, geom.room, "fp64")
    g.set_particles(pos0, np.zeros((3, 3)), size, RHO_P, RHO_F, G)
    steps = int(round(1.5 / P.terminal_velocity(30e-6, RHO_P, RHO_F, prm.nu)))    # about a minute
    g.step(steps)
    pos, vel, dep = g.particles()
    g.close()
    ref_pos, ref_vel, _ = oracle_run(F.zero_state(prm), geom, prm, pos0, np.zeros((3, 3)), size, steps)
    assert np.max(np.abs(pos - ref_pos)) < 1e-12 and not dep.any()
    v_star = P.terminal_velocity(size, RHO_P, RHO_F, prm.nu)
    # C_d = 1 + Re^(2/3)/6 slows the 30 um particle by 2.2 % (Re_p = 0.048), the smaller ones by less
    assert abs((3.0 - pos[2, 2]) - 1.5) / 1.5 < 3e-2                  # the 30 um particle fell 1.5 m
    assert np.allclose(-vel[:, 2], v_star, rtol=3e-2)


def test_deposition_on_floor(torch):
    prm = F.Params(nx=16, ny=16, nz=16, lx=1.6, ly=1.6, lz=1.6, nu=1.6e-5, dt=0.01, filter=False)
    beta = np.ones(prm.shape)
    beta[0:2, :, :] = 0.0
    geom = F.Geometry(beta, np.zeros(prm.shape))
    size = np.array([100e-6, 80e-6, 2e-6])
    pos0 = np.array([[0.4, 0.4, 0.35], [0.8, 0.8, 0.5], [1.2, 1.2, 0.3]])
    g = gpu_grid(prm, beta, geom.S, geom.room, "fp64")
    g.set_particles(pos0, np.zeros((3, 3)), size, RHO_P, RHO_F, G)
    g.step(300)
    pos, vel, dep = g.particles()
    g.close()
    ref_pos, ref_vel, ref_dep = oracle_run(F.zero_state(prm), geom, prm, pos0, np.zeros((3, 3)), size, 300)
    assert list(dep) == list(ref_dep) == [True, True, False]
    assert np.max(np.abs(pos - ref_pos)) < 1e-12 and np.all(vel[dep] == 0.0)


def test_particles_fp32_flow(torch):
    room, prm, geom, st0 = room_case(64, 32, 32, boxes=[(20, 26, 8, 14, 2, 12)], seed=5)
    st32 = F.State(*(getattr(st0, n).astype(np.float32).astype(np.float64) for n in ("u", "v", "w", "c")),
                   np.zeros(prm.shape), 0.0, 0)
    pos0, vel0, size = seeded_particles(room, prm, 200, seed=2)
    ref_pos, ref_vel, _ = oracle_run(st32.copy(), geom, prm, pos0, vel0, size, 1)
    g = gpu_grid(prm, room.beta, room.S, room.room, "fp32")
    load_state(g, st32, prm, as_fp32=True)
    g.set_particles(pos0, vel0, size, RHO_P, RHO_F, G)
    g.step(1)
    pos, vel, _ = g.particles()
    g.close()
    # the drag runs in float: velocities to FP32 rounding, positions to dt times that
    vbar = 1e-5 * max(1.0, np.max(np.abs(ref_vel)))
    assert np.max(np.abs(vel - ref_vel)) < vbar
    assert np.max(np.abs(pos - ref_pos)) < prm.dt * vbar


def test_particles_with_dynamic_dt(torch):
    room, prm, geom, st0 = room_case(40, 24, 20, boxes=[(12, 16, 6, 10, 2, 8)], seed=4)
    pos0, vel0, size = seeded_particles(room, prm, 100, seed=3)
    cmax = 0.3
    st, recs, _ = F.run_adaptive(st0.copy(), geom, prm, 1, cmax)     # the dt sequence, step by step below
    st = st0.copy()
    pos, vel, dep = pos0, vel0, np.zeros(len(size), dtype=bool)
    dt_prev = prm.dt
    for _ in range(15):
        dt = F.adjust_dt(st, prm, cmax)
        st = F.State(st.u, st.v, st.w, st.c, st.p * (dt / dt_prev), st.t, st.step)
        st, _ = F.step(st, geom, prm.with_(dt=dt))
        pos, vel, dep = P.particle_step(pos, vel, size, dep, st.u, st.v, st.w, geom.beta, prm, dt, RHO_P, RHO_F, G)
        dt_prev = dt
    g = gpu_grid(prm, room.beta, room.S, room.room, "fp64", courant_max=cmax)
    load_state(g, st0, prm)
    g.set_particles(pos0, vel0, size, RHO_P, RHO_F, G)
    g.step(15)
    gpos, gvel, gdep = g.particles()
    g.close()
    assert np.array_equal(gdep, dep)
    assert np.max(np.abs(gpos - pos)) < 1e-11
