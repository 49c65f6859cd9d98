"""Plain FP64 oracle of the host-side ventilation metrics derived from the reduction series (Sec. 3.3, 3.4).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and the bench's CPU-baseline leg, never by the library path.

* Theoretical ACH (Eq. 14): ACH = V_dot / V with V_dot = inflow area * inflow speed, in 1/h.
* ACH from the mean-CO2 history: the paper fits f(t) = C0 exp(-ACH t) + C1 (Sec. 3.3.2).  For short runs where
  ACH * t_end << 1 that fit is ill-posed, so the log-slope estimate ACH = -d ln c_bar / dt (C1 = 0) is provided
  too; the three-parameter fit uses variable projection (golden-section search over ACH, linear least squares for
  C0 and C1).
* Time-dependent Wells-Riley (Eqs. 17-18): P = 1 - exp(-Q), Q(t) = (C0 p / ACH) (1 - exp(-ACH t)), and the same Q
  integrated by the trapezoid rule from a sampled concentration history c_q(t) = C0 c_bar(t) / c_bar(0).
* CO2 in ppm from the passive scalar: the paper starts from 1000 ppm stale air and fresh air at 400 ppm, so
  CO2 = 400 + 600 c (the printed perfect-mixing curve has its two constants swapped).
"""
from __future__ import annotations

import math

import numpy as np

SECONDS_PER_HOUR = 3600.0


def ach_theory(inflow_area_m2, inflow_speed_m_s, room_volume_m3):
    """Eq. 14 with V_dot = A U: air changes per hour."""
    return inflow_area_m2 * inflow_speed_m_s * SECONDS_PER_HOUR / room_volume_m3


def co2_ppm(c):
    """Map the passive scalar (1 = stale, 0 = fresh) to CO2 in ppm: 400 + 600 c."""
    return 400.0 + 600.0 * np.asarray(c, dtype=np.float64)


def ach_log_slope(t_seconds, c_mean):
    """ACH (1/h) from the least-squares slope of ln c_mean(t) against t (fresh air has c = 0, so C1 = 0)."""
    t = np.asarray(t_seconds, dtype=np.float64)
    y = np.log(np.asarray(c_mean, dtype=np.float64))
    tm = t.mean()
    slope = float(np.sum((t - tm) * (y - y.mean())) / np.sum((t - tm) ** 2))
    return -slope * SECONDS_PER_HOUR


def _linear_fit_for_rate(t, y, rate):
    """For a fixed decay rate a, the least-squares (C0, C1) of y = C0 exp(-a t) + C1 and the residual norm^2."""
    e = np.exp(-rate * t)
    A = np.stack([e, np.ones_like(t)], axis=1)
    coef, *_ = np.linalg.lstsq(A, y, rcond=None)
    res = y - A @ coef
    return coef, float(res @ res)


def ach_fit3(t_seconds, c_mean, rate_bounds_per_hour=(1e-3, 1e3), iters=200):
    """Three-parameter fit f(t) = C0 exp(-ACH t) + C1 (Sec. 3.3.2), returning (ACH per hour, C0, C1).

    Golden-section search on log(ACH) over ``rate_bounds_per_hour``; C0 and C1 by linear least squares."""
    t = np.asarray(t_seconds, dtype=np.float64) / SECONDS_PER_HOUR
    y = np.asarray(c_mean, dtype=np.float64)
    lo, hi = math.log(rate_bounds_per_hour[0]), math.log(rate_bounds_per_hour[1])
    g = (math.sqrt(5.0) - 1.0) / 2.0
    a = hi - g * (hi - lo)
    b = lo + g * (hi - lo)
    fa = _linear_fit_for_rate(t, y, math.exp(a))[1]
    fb = _linear_fit_for_rate(t, y, math.exp(b))[1]
    for _ in range(iters):
        if fa < fb:
            hi, b, fb = b, a, fa
            a = hi - g * (hi - lo)
            fa = _linear_fit_for_rate(t, y, math.exp(a))[1]
        else:
            lo, a, fa = a, b, fb
            b = lo + g * (hi - lo)
            fb = _linear_fit_for_rate(t, y, math.exp(b))[1]
    rate = math.exp(0.5 * (lo + hi))
    (c0, c1), _ = _linear_fit_for_rate(t, y, rate)
    return rate, float(c0), float(c1)


def wells_riley_dose(c0_quanta_m3, breathing_m3_h, ach_per_hour, t_hours):
    """Eq. 18: Q(t) = (C0 p / ACH) (1 - exp(-ACH t)); the limit ACH -> 0 is C0 p t."""
    if ach_per_hour == 0.0:
        return c0_quanta_m3 * breathing_m3_h * t_hours
    # 1 - exp(-x) written as -expm1(-x) so that the small-ACH limit keeps full precision
    return c0_quanta_m3 * breathing_m3_h / ach_per_hour * -math.expm1(-ach_per_hour * t_hours)


def infection_probability(dose):
    """Eq. 17: P = 1 - exp(-Q)."""
    return 1.0 - math.exp(-dose)


def wells_riley_dose_series(t_seconds, c_mean, c0_quanta_m3, breathing_m3_h):
    """Q(t_k) = p int_0^t_k C0 c_mean(t)/c_mean(0) dt by the trapezoid rule (t in seconds, Q dimensionless)."""
    t = np.asarray(t_seconds, dtype=np.float64) / SECONDS_PER_HOUR
    cq = c0_quanta_m3 * np.asarray(c_mean, dtype=np.float64) / float(c_mean[0])
    q = np.zeros_like(t)
    q[1:] = np.cumsum(0.5 * (cq[1:] + cq[:-1]) * np.diff(t))
    return breathing_m3_h * q
