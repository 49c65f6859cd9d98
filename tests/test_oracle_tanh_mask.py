"""Pins of the smooth source mask of Eq. 5 (the paper's general inlet model).

Fixed by the formula's closed-form points and limits: 1 at the centre (the limit of the singular bracket), 1/2 per
axis at half the window width, 1/8 at the window's corners, symmetry, monotone decay, the binary window as the
sharpness grows, and the periodic wrap; and by the flow: a smooth window drives the flow like the binary one where
it is 1 and not at all where it is 0."""
import math

import numpy as np
import pytest

from oracle import flow as F


def prm_box(nx=20, ny=16, nz=12, h=0.1):
    return F.Params(nx=nx, ny=ny, nz=nz, lx=nx * h, ly=ny * h, lz=nz * h, nu=1e-3, dt=0.01)


def test_factor_closed_form_points():
    hw, B = 0.3, 2.0
    assert F.tanh_window_factor(0.0, hw, B) == 1.0
    assert F.tanh_window_factor(hw, hw, B) == 0.5
    d = 0.45
    assert F.tanh_window_factor(d, hw, B) == pytest.approx(0.5 * (1 - math.tanh(B * (d / hw - hw / d))), rel=1e-15)
    tiny = 1e-12
    assert F.tanh_window_factor(tiny, hw, B) == 1.0      # continuous at the singular point


def test_mask_at_centre_half_width_and_corner():
    prm = prm_box()
    c = (1.0, 0.8, 0.6)          # cell centres: x_10, y_8, z_6
    W = (0.4, 0.2, 0.4)          # half widths 0.2, 0.1, 0.2: two, one and two cells
    S = F.tanh_source_mask(prm, c, W, (3.0, 3.0, 3.0))
    assert S[6, 8, 10] == 1.0
    assert S[6, 8, 12] == pytest.approx(0.5, rel=1e-15)             # x at half width, y and z at the centre
    assert S[8, 9, 12] == pytest.approx(0.125, rel=1e-15)           # every axis at half width
    assert np.all((S >= 0.0) & (S <= 1.0))


def test_symmetric_and_monotone():
    prm = prm_box()
    S = F.tanh_source_mask(prm, (1.0, 0.8, 0.6), (0.6, 0.6, 0.6), (1.5, 1.5, 1.5))
    row = S[6, 8, :]
    for k in range(1, 10):
        assert row[10 - k] == pytest.approx(row[10 + k], rel=1e-14)
    assert np.all(np.diff(row[10:]) <= 0.0) and np.all(np.diff(row[:11]) >= 0.0)


def test_sharp_limit_is_the_binary_window():
    prm = prm_box()
    S = F.tanh_source_mask(prm, (1.0, 0.8, 0.6), (0.5, 0.5, 0.5), (200.0, 200.0, 200.0))
    x = np.arange(prm.nx) * prm.h[0]
    y = np.arange(prm.ny) * prm.h[1]
    z = np.arange(prm.nz) * prm.h[2]
    inside = ((np.abs(z - 0.6) < 0.25)[:, None, None] & (np.abs(y - 0.8) < 0.25)[None, :, None]
              & (np.abs(x - 1.0) < 0.25)[None, None, :])
    assert np.allclose(S, inside.astype(float), atol=1e-12)


def test_periodic_wrap():
    """A window centred on the x = 0 face is split across the wrap: cell nx - k mirrors cell k."""
    prm = prm_box()
    S = F.tanh_source_mask(prm, (0.0, 0.8, 0.6), (0.6, 0.4, 0.4), (1.0, 1.0, 1.0))
    for k in range(1, 5):
        assert S[6, 8, prm.nx - k] == pytest.approx(S[6, 8, k], rel=1e-14)


def test_smooth_window_drives_flow_like_binary_where_it_is_one():
    """With a sharp window the forced velocity after one step equals the binary window's to the mask difference;
    far outside the window the smooth forcing is exactly zero."""
    prm = prm_box().with_(u_set=(0.5, 0.0, 0.0), filter=False)
    st = F.zero_state(prm)
    smooth = F.tanh_source_mask(prm, (1.0, 0.8, 0.6), (0.5, 0.5, 0.5), (200.0, 200.0, 200.0))
    binary = (smooth > 0.5).astype(float)
    a, _ = F.step(st.copy(), F.Geometry(np.ones(prm.shape), smooth), prm)
    b, _ = F.step(st.copy(), F.Geometry(np.ones(prm.shape), binary), prm)
    assert np.max(np.abs(a.u - b.u)) < 1e-10
    assert np.max(np.abs(a.u)) > 0.1
