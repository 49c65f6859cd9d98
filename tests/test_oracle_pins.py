"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: closed-form Fourier symbols of the central
difference operators, exact RK4 amplification factors of linear problems, a brute-force dense least-squares
projection, the Taylor-Green decay, the Poiseuille profile, conservation identities and brute-force counts.
A plausible mistake in the oracle (a dropped 1/2, a wrong sign, a swapped axis, a wrong RK weight) fails one.
"""
import math

import numpy as np
import pytest

from oracle import flow as F
from paper_2204_02107_gb300 import rooms


def rk4_poly(z):
    """Stability polynomial of classic RK4."""
    return 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24


def grid_coords(prm):
    hx, hy, hz = prm.h
    z, y, x = np.meshgrid(np.arange(prm.nz) * hz, np.arange(prm.ny) * hy, np.arange(prm.nx) * hx, indexing="ij")
    return x, y, z


BASE = F.Params(nx=24, ny=20, nz=18, lx=2.4, ly=3.0, lz=1.8, nu=0.0, dt=1e-2, filter=False, n_pressure_iters=1)


# ---------------------------------------------------------------- operators: exact symbols on Fourier modes

@pytest.mark.parametrize("d", [0, 1, 2])
@pytest.mark.parametrize("k", [1, 3, 7])
def test_delta_symbols(d, k):
    prm = BASE
    coords = grid_coords(prm)
    n = (prm.nx, prm.ny, prm.nz)[d]
    h = prm.h[d]
    L = (prm.lx, prm.ly, prm.lz)[d]
    kk = 2 * math.pi * k / L
    theta = kk * h
    phase = kk * coords[d] + 0.3
    f = np.cos(phase)
    ax = F.AXES[d]
    np.testing.assert_allclose(F.delta(f, ax, h), -np.sin(theta) / h * np.sin(phase), atol=1e-12)
    np.testing.assert_allclose(F.delta2(f, ax, h), -4 * np.sin(theta / 2) ** 2 / h ** 2 * f, atol=1e-9)
    np.testing.assert_allclose(F.sixth_difference(f, ax), -64 * np.sin(theta / 2) ** 6 * f, atol=1e-11)
    # the other two axes see a constant
    for other in range(3):
        if other != d:
            assert np.max(np.abs(F.delta(f, F.AXES[other], prm.h[other]))) < 1e-12
    assert n > 2 * k


def test_filter_symbol():
    """Eq. 6 with gamma = dx^6/pi^6: a Fourier mode is multiplied by 1 - 64/pi^6 sum_j sin^6(theta_j/2)."""
    prm = BASE
    x, y, z = grid_coords(prm)
    kx, ky, kz = 5, 2, 9
    th = [2 * math.pi * k / n for k, n in zip((kx, ky, kz), (prm.nx, prm.ny, prm.nz))]
    f = np.cos(2 * math.pi * (kx * x / prm.lx + ky * y / prm.ly + kz * z / prm.lz))
    g = F.open_geometry(prm)
    expect = (1 - 64 / math.pi ** 6 * sum(math.sin(t / 2) ** 6 for t in th)) * f
    np.testing.assert_allclose(F.filter6(f, g), expect, atol=1e-13)
    # Nyquist along all three axes: damped but not reversed (symbol 1 - 3*64/pi^6 ~ 0.80)
    nyq = np.cos(math.pi * (np.arange(prm.nx)[None, None, :] + np.arange(prm.ny)[None, :, None]
                            + np.arange(prm.nz)[:, None, None]))
    ratio = F.filter6(nyq, g) / nyq
    np.testing.assert_allclose(ratio, 1 - 3 * 64 / math.pi ** 6, atol=1e-13)


# ---------------------------------------------------------------- skew-symmetric convection conserves energy

def test_skew_symmetric_convection_conserves_energy():
    """sum_cells u . N(u) = 0 for a random, non-solenoidal periodic field (summation by parts of the skew form)."""
    prm = BASE.with_(nu=0.0)
    g = F.open_geometry(prm)
    u, v, w = rooms.random_fields(prm.shape, seed=11, count=3)
    k = F.momentum_rhs(u, v, w, g, prm)
    dot = sum(float(np.sum(a * b)) for a, b in zip((u, v, w), k))
    scale = sum(float(np.sum(np.abs(a * b))) for a, b in zip((u, v, w), k))
    assert abs(dot) < 1e-13 * scale
    # the divergence form alone (a plausible mistake) does not conserve energy
    h = prm.h
    div_only = [sum(F.delta(uj * ui, F.AXES[j], h[j]) for j, uj in enumerate((u, v, w))) for ui in (u, v, w)]
    dot2 = sum(float(np.sum(a * b)) for a, b in zip((u, v, w), div_only))
    assert abs(dot2) > 1e-6 * scale


# ---------------------------------------------------------------- RK4 on exactly linear problems

def one_step(prm, geom, u, v, w, c):
    st = F.State(u.copy(), v.copy(), w.copy(), c.copy(), np.zeros(prm.shape))
    new, _ = F.step(st, geom, prm)
    return new


@pytest.mark.parametrize("d", [0, 1, 2])
def test_rk4_scalar_diffusion_amplification(d):
    """u = 0: c = cos mode diffuses linearly, so one step multiplies it by R4(z), z = alpha dt * symbol(delta2)."""
    alpha = 0.7
    prm = BASE.with_(nu=alpha, alpha_c=alpha, dt=0.0)
    h = prm.h[d]
    n = (prm.nx, prm.ny, prm.nz)[d]
    k = 3
    theta = 2 * math.pi * k / n
    sym = -4 * math.sin(theta / 2) ** 2 / h ** 2
    dt = -1.7 / (alpha * sym)              # z = -1.7: far from 1, separates RK4 from other tableaux
    prm = prm.with_(dt=dt)
    coords = grid_coords(prm)
    c = np.cos(2 * math.pi * k * coords[d] / (prm.lx, prm.ly, prm.lz)[d])
    z0 = np.zeros(prm.shape)
    new = one_step(prm, F.open_geometry(prm), z0, z0, z0, c)
    np.testing.assert_allclose(new.c, rk4_poly(-1.7) * c, atol=1e-12)
    assert np.all(new.u == 0) and np.all(new.p == 0)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_rk4_scalar_advection_amplification(d):
    """Uniform velocity U along axis d: c = Re(e^{i k x}) advects linearly; flux form gives the central symbol."""
    U = 2.0
    nu = 0.05
    prm = BASE.with_(nu=nu, alpha_c=nu)
    h = prm.h[d]
    n = (prm.nx, prm.ny, prm.nz)[d]
    k = 2
    theta = 2 * math.pi * k / n
    dt = 0.9 * h / U
    prm = prm.with_(dt=dt)
    z = -1j * U * dt * math.sin(theta) / h - nu * dt * 4 * math.sin(theta / 2) ** 2 / h ** 2
    coords = grid_coords(prm)
    ph = 2 * math.pi * k * coords[d] / (prm.lx, prm.ly, prm.lz)[d]
    c = np.cos(ph)
    vel = [np.zeros(prm.shape) for _ in range(3)]
    vel[d][:] = U
    new = one_step(prm, F.open_geometry(prm), *vel, c)
    expect = np.real(rk4_poly(z) * np.exp(1j * ph))
    np.testing.assert_allclose(new.c, expect, atol=1e-13)
    np.testing.assert_allclose((new.u, new.v, new.w)[d], U, atol=1e-13)


@pytest.mark.parametrize("d,e", [(0, 1), (1, 2), (2, 0), (0, 2)])
def test_rk4_momentum_advection_diffusion_amplification(d, e):
    """u_d = U, u_e = cos(k x_d): the skew form reduces to U delta_d u_e (linear); D u = 0 so no pressure acts."""
    U = 1.5
    nu = 0.02
    prm = BASE.with_(nu=nu)
    h = prm.h[d]
    n = (prm.nx, prm.ny, prm.nz)[d]
    k = 4
    theta = 2 * math.pi * k / n
    dt = 0.8 * h / U
    prm = prm.with_(dt=dt, n_pressure_iters=2)
    z = -1j * U * dt * math.sin(theta) / h - nu * dt * 4 * math.sin(theta / 2) ** 2 / h ** 2
    coords = grid_coords(prm)
    ph = 2 * math.pi * k * coords[d] / (prm.lx, prm.ly, prm.lz)[d]
    vel = [np.zeros(prm.shape) for _ in range(3)]
    vel[d][:] = U
    vel[e] = np.cos(ph)
    new = one_step(prm, F.open_geometry(prm), *vel, np.zeros(prm.shape))
    out = (new.u, new.v, new.w)
    np.testing.assert_allclose(out[e], np.real(rk4_poly(z) * np.exp(1j * ph)), atol=1e-12)
    np.testing.assert_allclose(out[d], U, atol=1e-12)
    assert np.max(np.abs(new.p)) < 1e-12


def test_forcing_and_body_force():
    """Uniform fields, S = 1 everywhere: (q - q_set) is multiplied by R4(-dt/tau_f); a body force adds b dt."""
    prm = BASE.with_(nu=0.01, dt=0.01, tau_f=0.02, u_set=(0.4, -0.2, 0.1), c_set=0.25)
    g = F.Geometry(np.ones(prm.shape), np.ones(prm.shape))
    one = np.ones(prm.shape)
    new = one_step(prm, g, 1.0 * one, 2.0 * one, -1.0 * one, 0.9 * one)
    R = rk4_poly(-prm.dt / prm.tau_f)
    for got, q0, qs in zip((new.u, new.v, new.w, new.c), (1.0, 2.0, -1.0, 0.9), (0.4, -0.2, 0.1, 0.25)):
        np.testing.assert_allclose(got, qs + R * (q0 - qs), atol=1e-14)
    # tau_f <= 0 means tau_f = dt: R4(-1) = 3/8
    prm2 = prm.with_(tau_f=0.0)
    new2 = one_step(prm2, g, one, one, one, one)
    np.testing.assert_allclose(new2.u, 0.4 + 0.375 * (1 - 0.4), atol=1e-14)
    prm3 = BASE.with_(dt=0.05, body_force=(0.3, 0.0, -0.6))
    new3 = one_step(prm3, F.open_geometry(prm3), 0 * one, 0 * one, 0 * one, 0 * one)
    np.testing.assert_allclose(new3.u, 0.3 * 0.05, atol=1e-15)
    np.testing.assert_allclose(new3.w, -0.6 * 0.05, atol=1e-15)


# ---------------------------------------------------------------- Poisson solve

def test_poisson_manufactured_modes():
    """p = random combination of non-null modes, f = lambda(k) p_k mode by mode (closed form) -> solve returns p;
    and D(G p) equals that f (the symbol is the one of the central operators)."""
    prm = F.Params(nx=12, ny=10, nz=18, lx=1.2, ly=2.0, lz=0.9, nu=0.0, dt=1.0)
    rng = np.random.default_rng(3)
    x, y, z = grid_coords(prm)
    p = np.zeros(prm.shape)
    f = np.zeros(prm.shape)
    hx, hy, hz = prm.h
    for _ in range(6):
        k = (int(rng.integers(0, prm.nx)), int(rng.integers(0, prm.ny)), int(rng.integers(0, prm.nz)))
        if all(kk == 0 or 2 * kk == n for kk, n in zip(k, (prm.nx, prm.ny, prm.nz))):
            continue
        a, ph = rng.standard_normal(), rng.uniform(0, 2 * math.pi)
        mode = a * np.cos(2 * math.pi * (k[0] * x / prm.lx + k[1] * y / prm.ly + k[2] * z / prm.lz) + ph)
        lam = -sum(math.sin(2 * math.pi * kk / n) ** 2 / hh ** 2
                   for kk, n, hh in zip(k, (prm.nx, prm.ny, prm.nz), (hx, hy, hz)))
        if abs(lam) < 1e-9:        # a mode that is null for D o G although not one of the eight (cannot happen)
            continue
        p += mode
        f += lam * mode
    got = F.poisson_fft_solve(f, prm)
    np.testing.assert_allclose(got, p, atol=1e-12 * np.max(np.abs(p)))
    dg = sum(F.delta(F.delta(p, F.AXES[j], prm.h[j]), F.AXES[j], prm.h[j]) for j in range(3))
    np.testing.assert_allclose(dg, f, atol=1e-11 * np.max(np.abs(f)))


def test_poisson_null_modes_dropped():
    """The eight modes with k_j in {0, n_j/2} are in the null space of D o G and get p_hat = 0."""
    prm = F.Params(nx=8, ny=10, nz=6, lx=1.0, ly=1.0, lz=1.0, nu=0.0, dt=1.0)
    ix = np.arange(prm.nx)[None, None, :]
    iy = np.arange(prm.ny)[None, :, None]
    iz = np.arange(prm.nz)[:, None, None]
    total = np.zeros(prm.shape)
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                total = total + np.cos(math.pi * (a * ix + b * iy + c * iz)) * np.ones(prm.shape)
    assert np.max(np.abs(F.poisson_fft_solve(total, prm))) < 1e-14
    assert F.null_modes(prm).sum() == 8


# ---------------------------------------------------------------- beta-iteration vs brute-force projection

def central_gradient_matrix(shape, h):
    """Dense (3N x N) matrix of the periodic central gradient, built from index arithmetic alone."""
    nz, ny, nx = shape
    N = nx * ny * nz
    G = np.zeros((3 * N, N))

    def idx(x, y, z):
        return (x % nx) + nx * ((y % ny) + ny * (z % nz))

    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = idx(x, y, z)
                G[i, idx(x + 1, y, z)] += 0.5 / h[0]
                G[i, idx(x - 1, y, z)] -= 0.5 / h[0]
                G[N + i, idx(x, y + 1, z)] += 0.5 / h[1]
                G[N + i, idx(x, y - 1, z)] -= 0.5 / h[1]
                G[2 * N + i, idx(x, y, z + 1)] += 0.5 / h[2]
                G[2 * N + i, idx(x, y, z - 1)] -= 0.5 / h[2]
    return G


def masked_projection_case(shape=(8, 10, 8), seed=21):
    nz, ny, nx = shape
    prm = F.Params(nx=nx, ny=ny, nz=nz, lx=nx * 0.1, ly=ny * 0.1, lz=nz * 0.1, nu=0.0, dt=1.0)
    beta = rooms.random_mask(prm.shape, seed=seed, n_boxes=3).astype(np.float64)
    g = F.Geometry(beta, np.zeros(prm.shape))
    us = rooms.random_fields(prm.shape, seed=seed + 1, count=3, beta=beta)
    return prm, g, us


def test_beta_iteration_converges_to_least_squares_projection():
    """With central D = -G^T, Eq. 7 masked is the normal equation of min_p |beta G p - u*|, so the converged
    iteration of Eq. 9 must give the same corrected velocity as a dense least-squares solve."""
    prm, g, (us, vs, ws) = masked_projection_case()
    N = us.size
    G = central_gradient_matrix(prm.shape, prm.h)
    B = np.tile(g.beta.ravel(), 3)
    ustar = np.concatenate([us.ravel(), vs.ravel(), ws.ravel()])
    p_ls, *_ = np.linalg.lstsq(B[:, None] * G, B * ustar, rcond=None)
    u_ls = B * (ustar - G @ p_ls)
    r = F.divergence(us, vs, ws, prm)
    p = F.pressure_iterations(r, np.zeros(prm.shape), g, prm, n=600)
    u_it = np.concatenate([a.ravel() for a in F.project(us, vs, ws, p, g, prm)])
    np.testing.assert_allclose(u_it, u_ls, atol=1e-10 * np.max(np.abs(u_ls)))
    # the projected field is divergence-free (up to round-off) and zero in solids
    ui = [u_it[k * N:(k + 1) * N].reshape(prm.shape) for k in range(3)]
    assert np.max(np.abs(F.divergence(*ui, prm))) < 1e-9 * np.max(np.abs(r))
    assert np.all(ui[0][g.beta == 0] == 0)


def test_beta_iteration_residual_decreases():
    """The divergence left by n iterations decreases with n (the paper uses n = 4)."""
    prm, g, (us, vs, ws) = masked_projection_case(seed=5)
    r = F.divergence(us, vs, ws, prm)
    res = []
    for n in (1, 2, 4, 8, 16):
        p = F.pressure_iterations(r, np.zeros(prm.shape), g, prm, n=n)
        u = F.project(us, vs, ws, p, g, prm)
        res.append(np.sqrt(np.sum(F.divergence(*u, prm) ** 2)))
    assert all(b < a for a, b in zip(res, res[1:])), res


def test_unmasked_projection_divergence_free():
    """beta = 1, random u*: one iteration is exact; max|D u| * h / max|u| at round-off."""
    prm = F.Params(nx=16, ny=12, nz=10, lx=1.6, ly=1.2, lz=1.0, nu=0.0, dt=1.0)
    g = F.open_geometry(prm)
    us = rooms.random_fields(prm.shape, seed=8, count=3)
    p = F.pressure_iterations(F.divergence(*us, prm), np.zeros(prm.shape), g, prm, n=1)
    u = F.project(*us, p, g, prm)
    assert np.max(np.abs(F.divergence(*u, prm))) * prm.h[0] / np.max(np.abs(u[0])) < 1e-12


# ---------------------------------------------------------------- whole steps

def test_taylor_green_decay():
    """Taylor-Green on a periodic 32^3 grid of [0, 2 pi)^3, nu = 0.01, dt = 1e-3, 100 steps: the amplitude
    sqrt(E/E0) follows exp(-3 nu t) (Stokes decay of |k|^2 = 3) to 1e-4, and the field stays divergence-free."""
    n = 32
    prm = F.Params(nx=n, ny=n, nz=n, lx=2 * math.pi, ly=2 * math.pi, lz=2 * math.pi, nu=0.01, dt=1e-3,
                   filter=False, n_pressure_iters=1)
    u, v, w = rooms.taylor_green(n)
    st = F.State(u, v, w, np.zeros(prm.shape), np.zeros(prm.shape))
    g = F.open_geometry(prm)
    e0 = F.reductions(st, g, prm)['ke']
    st, recs = F.run(st, g, prm, 100)
    amp = math.sqrt(recs[-1]['ke'] / e0)
    expect = math.exp(-3 * prm.nu * st.t)
    assert abs(amp - expect) / expect < 1e-4
    assert abs(amp - expect) / expect > 1e-7          # the discrete operator is not the continuous one
    assert max(r['div_max'] for r in recs) < 1e-12


def channel_case(ny=16, b=1e-3, nu=0.05):
    prm = F.Params(nx=8, ny=ny, nz=8, lx=8.0, ly=float(ny), lz=8.0, nu=nu, dt=0.2 / nu, body_force=(b, 0.0, 0.0),
                   filter=False, n_pressure_iters=4)
    beta = np.ones(prm.shape)
    beta[:, 0, :] = 0.0        # solid rows at y = 0 and y = ny-1: walls D = (ny-1) h apart
    beta[:, ny - 1, :] = 0.0
    g = F.Geometry(beta, np.zeros(prm.shape))
    y = np.arange(ny) * prm.h[1]
    D = (ny - 1) * prm.h[1]
    profile = b / (2 * nu) * y * (D - y)
    U = np.broadcast_to(profile[None, :, None], prm.shape) * beta
    return prm, g, U


def test_poiseuille_fixed_point():
    """the analytic channel profile U(y) = (b/2nu) y (D - y) (Sec. 3.1.1) is a discrete steady state: central
    second differences are exact on quadratics and the walls sit where U = 0."""
    prm, g, U = channel_case()
    z = np.zeros(prm.shape)
    st, _ = F.run(F.State(U.copy(), z.copy(), z.copy(), z.copy(), z.copy()), g, prm, 3)
    assert np.max(np.abs(st.u - U)) < 1e-10 * np.max(U)
    assert np.max(np.abs(st.v)) == 0 and np.max(np.abs(st.w)) == 0


def test_poiseuille_transient_reaches_profile():
    """Started from rest, the channel approaches the analytic profile; after enough steps the relative error is
    below the paper's printed 1e-5 (Sec. 3.1.1); the bulk velocity obeys Re = b D^3 / (12 nu^2) within O(h^2)."""
    prm, g, U = channel_case()
    z = np.zeros(prm.shape)
    st = F.State(z.copy(), z.copy(), z.copy(), z.copy(), z.copy())
    D = (prm.ny - 1) * prm.h[1]
    decay = prm.nu * (math.pi / D) ** 2                 # slowest mode
    n_steps = int(math.ceil(math.log(1e6) / (decay * prm.dt)))
    st, _ = F.run(st, g, prm, n_steps)
    err = np.max(np.abs(st.u - U)) / np.max(U)
    assert err < 1e-5
    b = prm.body_force[0]
    ub_discrete = float(np.mean(U[0, 1:prm.ny - 1, 0])) * (prm.ny - 2) / (prm.ny - 1)
    ub_formula = b * D ** 2 / (12 * prm.nu)
    assert abs(ub_discrete - ub_formula) / ub_formula < 0.05


def small_room_case(seed=2, nx=40, ny=24, nz=20, steps=0):
    room = rooms.make_room(nx, ny, nz, h=0.05, boxes=[(12, 16, 6, 10, 2, 8)], u_in=1.0)
    prm = F.Params(nx=nx, ny=ny, nz=nz, lx=room.lx, ly=room.ly, lz=room.lz, nu=1.6e-5, dt=room.dt,
                   u_set=(room.u_in, 0.0, 0.0), c_set=0.0, filter=True, n_pressure_iters=4)
    g = F.Geometry(room.beta, room.S, room.room)
    st = F.zero_state(prm, c=room.initial_c())
    return prm, g, st


def test_masking_exact_zero_in_solids():
    """u, v, w, c are exactly zero in every solid cell after every step."""
    prm, g, st = small_room_case()
    solid = g.beta == 0
    for _ in range(5):
        st, _ = F.step(st, g, prm)
        for f in (st.u, st.v, st.w, st.c):
            assert np.all(f[solid] == 0.0)
    assert np.max(np.abs(st.u)) > 0.1


def test_scalar_budget_closes():
    """the flux-form scalar transport is conservative: over one step the change of the total inventory equals
    the RK-weighted forcing inventory minus what the re-mask after the filter removes from solid cells."""
    prm, g, st = small_room_case()
    for _ in range(3):
        st, _ = F.step(st, g, prm)
    before = prm.cell_volume * float(np.sum(st.c))
    new, rec = F.step(st, g, prm, with_budget=True)
    after = rec['c_total']
    assert abs(rec['c_star_total'] - before - rec['forcing']) < 1e-12 * before
    assert abs(after - rec['c_star_total'] + rec['mask_loss']) < 1e-12 * before
    assert rec['forcing'] != 0.0
    # the re-mask after the filter is the only loss: with the filter off nothing is removed from the solids
    prm_nofilter = prm.with_(filter=False)
    _, rec2 = F.step(st, g, prm_nofilter, with_budget=True)
    assert rec2['mask_loss'] == 0.0


def test_room_outflow_closed_form():
    """outflow rate of a slab room x in [a, b) across a uniform flow U along x: c = 1 in the room, c_L in the
    cell before it and c_R in the cell after it.  Per (y, z) row the two x faces give
    A [U (c_R - c_L) / 2 + alpha (2 - c_R - c_L) / h] (face area A = dV / h); the slab spans y and z, so no other
    face leaves it.  A solid cell behind a face closes that face."""
    prm = F.Params(nx=16, ny=6, nz=5, lx=1.6, ly=0.9, lz=1.0, nu=0.0, alpha_c=0.003, dt=1e-3)
    a, b, U, cL, cR = 5, 11, 0.7, 0.25, -0.4
    room = np.zeros(prm.shape)
    room[:, :, a:b] = 1.0
    c = np.full(prm.shape, 3.0)              # cells away from the room's faces do not count
    c[:, :, a:b] = 1.0
    c[:, :, a - 1] = cL
    c[:, :, b] = cR
    u = np.full(prm.shape, U)
    z = np.zeros(prm.shape)
    g = F.Geometry(np.ones(prm.shape), np.zeros(prm.shape), room)
    hx = prm.h[0]
    A = prm.cell_volume / hx
    rows = prm.ny * prm.nz
    want = rows * A * (U * (cR - cL) / 2 + prm.alpha * (2 - cR - cL) / hx)
    got = F.room_outflow_rate(c, u, z, z, g, prm)
    assert abs(got - want) < 1e-13 * abs(want)
    # the same room with the cells behind its right face solid: only the left face is left
    beta = np.ones(prm.shape)
    beta[:, :, b] = 0.0
    g2 = F.Geometry(beta, np.zeros(prm.shape), room)
    want2 = rows * A * (-U * (cL + 1) / 2 + prm.alpha * (1 - cL) / hx)
    assert abs(F.room_outflow_rate(c * beta, u * beta, z, z, g2, prm) - want2) < 1e-13 * abs(want2)


def test_room_budget_closes():
    """over one step the room inventory changes by the forcing inside the room, minus what leaves the room
    through its openings, plus what the filter moves across the room's boundary: the flux form makes every
    interior face cancel.  A wrong sign, area or diffusive term of the outflow breaks the balance."""
    prm, g, st = small_room_case()
    u, v, w = rooms.random_fields(prm.shape, 4, count=3, scale=0.3, beta=g.beta)
    st = F.State(u, v, w, st.c, st.p)
    for _ in range(2):
        st, rec0 = F.step(st, g, prm)
    new, rec = F.step(st, g, prm, with_budget=True)
    change = rec['c_room'] - rec0['c_room']
    balance = rec['forcing_room'] - rec['outflow'] + rec['filter_room']
    assert abs(change - balance) < 1e-12 * rec['c_room']
    assert abs(rec['outflow']) > 1e-6 * rec['c_room'] and rec['forcing_room'] == 0.0
    # with the inlet region counted as room the forcing acts inside it, and the balance still closes
    g2 = F.Geometry(g.beta, g.S, np.maximum(g.room, g.S))
    _, r1 = F.step(st, g2, prm, with_budget=True)
    assert r1['forcing_room'] != 0.0
    before = prm.cell_volume * float(np.sum(g2.room * st.c))
    assert abs(r1['c_room'] - before - (r1['forcing_room'] - r1['outflow'] + r1['filter_room'])) < 1e-12 * before


def test_histogram_brute_force():
    rng = np.random.default_rng(7)
    c = rng.uniform(-0.2, 1.2, size=(5, 6, 7))
    c.flat[3] = 1.0
    c.flat[4] = 0.0
    room = (rng.random(c.shape) < 0.7).astype(np.float64)
    counts, under, over = F.histogram(c, room)
    ref = [0] * 64
    ru = ro = 0
    for val, inside in zip(c.ravel(), room.ravel()):
        if not inside:
            continue
        if val < 0:
            ru += 1
        elif val > 1:
            ro += 1
        else:
            ref[min(int(val * 64), 63)] += 1
    assert list(counts) == ref and under == ru and over == ro


def test_region_force_closed_forms():
    """Force on a region from the unmasked right-hand side: a uniform pressure gradient G over a fluid at rest
    pushes a region of V cells with -G V dV; a Couette-like shear profile u = a y^2 (diffusion only) gives
    2 nu a per cell.  Checks the sign, the cell volume and the pressure scaling p = dt p_phys."""
    prm = F.Params(nx=8, ny=10, nz=6, lx=0.8, ly=1.0, lz=0.6, nu=0.01, dt=0.05)
    geom = F.open_geometry(prm)
    st = F.zero_state(prm)
    region = np.zeros(prm.shape, dtype=bool)
    region[2:4, 3:6, 2:5] = True                       # 2 x 3 x 3 = 18 cells away from the periodic seams
    x = np.arange(prm.nx) * prm.h[0]
    st.p = prm.dt * np.broadcast_to(0.7 * x[None, None, :], prm.shape).copy()   # p_phys = 0.7 x in the middle
    f = F.region_force(st, geom, prm, region)
    assert f[0] == pytest.approx(-0.7 * 18 * prm.cell_volume, rel=1e-12)
    assert abs(f[1]) < 1e-14 and abs(f[2]) < 1e-14
    st = F.zero_state(prm)
    y = np.arange(prm.ny) * prm.h[1]
    st.u = np.broadcast_to(3.0 * (y ** 2)[None, :, None], prm.shape).copy()
    f = F.region_force(st, geom, prm, region)
    # convection of u(y) alone vanishes (v = w = 0, d/dx u = 0); diffusion: nu * 2 * 3.0 per cell
    assert f[0] == pytest.approx(prm.nu * 6.0 * 18 * prm.cell_volume, rel=1e-10)


def test_reductions_closed_forms():
    """The diagnostics (Sec. 3.3) of a state whose sums have closed forms over whole periods: u = A sin(2 pi x/lx),
    v = B cos(2 pi z/lz), w = C; c = c0 everywhere except three room cells at -0.01, 1.0 and 1.02.  Then
    KE = V (A^2/2 + B^2/2 + C^2) / 2, D u = a cos(2 pi x/lx) with a = A sin(2 pi/nx)/hx (v and w carry no
    divergence), so div_max = |a| and div_l2 = |a| sqrt(V/2); u_max = max(|A|, |B|, |C|); the scalar sums are
    counts times the values, and every room cell falls in bin floor(64 c0) except c = 1 (last bin, by the min rule)
    and the two cells outside [0, 1]."""
    nx, ny, nz = 16, 12, 10
    prm = F.Params(nx=nx, ny=ny, nz=nz, lx=1.6, ly=0.9, lz=1.3, nu=0.0, dt=1.0)
    hx, hy, hz = prm.h
    dV = hx * hy * hz
    vol = prm.lx * prm.ly * prm.lz
    A, B, C, c0 = 0.7, -0.45, 0.2, 0.41
    i = np.arange(nx)
    k = np.arange(nz)
    u = np.broadcast_to(A * np.sin(2 * math.pi * i / nx)[None, None, :], prm.shape).copy()
    v = np.broadcast_to(B * np.cos(2 * math.pi * k / nz)[:, None, None], prm.shape).copy()
    w = np.full(prm.shape, C)
    c = np.full(prm.shape, c0)
    room = np.zeros(prm.shape)
    room[:, :, : nx // 2] = 1.0                       # x < 8: the room
    c[3, 4, 2], c[5, 6, 1], c[7, 2, 5] = -0.01, 1.0, 1.02
    st = F.State(u, v, w, c, np.zeros(prm.shape))
    rec = F.reductions(st, F.Geometry(np.ones(prm.shape), np.zeros(prm.shape), room), prm)
    a = A * math.sin(2 * math.pi / nx) / hx
    n_room = (nx // 2) * ny * nz
    v_room = n_room * dV
    assert rec['ke'] == pytest.approx(0.5 * vol * (A * A / 2 + B * B / 2 + C * C), rel=1e-13)
    assert rec['div_max'] == pytest.approx(abs(a), rel=1e-13)
    assert rec['div_l2'] == pytest.approx(abs(a) * math.sqrt(vol / 2), rel=1e-13)
    assert rec['u_max'] == pytest.approx(max(abs(A), abs(B), abs(C)), rel=1e-15)
    odd = [-0.01, 1.0, 1.02]
    assert rec['v_room'] == pytest.approx(v_room, rel=1e-14)
    assert rec['c_total'] == pytest.approx(dV * ((nx * ny * nz - 3) * c0 + sum(odd)), rel=1e-13)
    assert rec['c_room'] == pytest.approx(dV * ((n_room - 3) * c0 + sum(odd)), rel=1e-13)
    assert rec['c2_room'] == pytest.approx(dV * ((n_room - 3) * c0 * c0 + sum(x * x for x in odd)), rel=1e-13)
    want = np.zeros(64, dtype=np.int64)
    want[int(64 * c0)] = n_room - 3
    want[63] = 1
    assert np.array_equal(rec['hist'], want)
    assert (rec['hist_under'], rec['hist_over']) == (1, 1)
