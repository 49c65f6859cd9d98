// Host-side ventilation metrics derived from the per-step reduction series (Sec. 3.3.2 and 3.4).
#include <cmath>
#include <cstdint>

#include "../../include/ventflow.h"

namespace {

constexpr double kSecondsPerHour = 3600.0;

// Least-squares (c0, c1) of y = c0 * exp(-a t) + c1 for a fixed rate a, from the 2 x 2 normal equations, and the
// residual sum of squares.
double fit_linear(const double* t, const double* y, int64_t n, double a, double* c0, double* c1)
{
    double see = 0, se = 0, sy = 0, sey = 0;
    for (int64_t i = 0; i < n; ++i) {
        const double e = std::exp(-a * t[i]);
        see += e * e;
        se += e;
        sy += y[i];
        sey += e * y[i];
    }
    const double det = see * (double)n - se * se;
    if (det == 0.0) {
        *c0 = 0.0;
        *c1 = sy / (double)n;
    } else {
        *c0 = (sey * (double)n - se * sy) / det;
        *c1 = (see * sy - se * sey) / det;
    }
    double rss = 0;
    for (int64_t i = 0; i < n; ++i) {
        const double r = y[i] - (*c0 * std::exp(-a * t[i]) + *c1);
        rss += r * r;
    }
    return rss;
}

}  // namespace

extern "C" {

int vf_ach_log_slope(const double* t_seconds, const double* c_mean, int64_t n, double* ach_per_hour)
{
    if (!t_seconds || !c_mean || !ach_per_hour || n < 2) return VF_EINVAL;
    double tm = 0, ym = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!(c_mean[i] > 0)) return VF_EINVAL;
        tm += t_seconds[i];
        ym += std::log(c_mean[i]);
    }
    tm /= (double)n;
    ym /= (double)n;
    double stt = 0, sty = 0;
    for (int64_t i = 0; i < n; ++i) {
        const double dt = t_seconds[i] - tm;
        stt += dt * dt;
        sty += dt * (std::log(c_mean[i]) - ym);
    }
    if (stt == 0.0) return VF_EINVAL;
    *ach_per_hour = -(sty / stt) * kSecondsPerHour;
    return VF_OK;
}

int vf_ach_fit3(const double* t_seconds, const double* c_mean, int64_t n, double* ach_per_hour, double* c0,
                double* c1)
{
    if (!t_seconds || !c_mean || !ach_per_hour || !c0 || !c1 || n < 3) return VF_EINVAL;
    // work in hours so the rate is ACH itself; golden-section search over log(ACH) in [1e-3, 1e3]
    double* th = new double[(size_t)n];
    for (int64_t i = 0; i < n; ++i) th[i] = t_seconds[i] / kSecondsPerHour;
    double lo = std::log(1e-3), hi = std::log(1e3);
    const double g = 0.5 * (std::sqrt(5.0) - 1.0);
    double a = hi - g * (hi - lo), b = lo + g * (hi - lo), p0, p1;
    double fa = fit_linear(th, c_mean, n, std::exp(a), &p0, &p1);
    double fb = fit_linear(th, c_mean, n, std::exp(b), &p0, &p1);
    for (int it = 0; it < 200; ++it) {
        if (fa < fb) {
            hi = b; b = a; fb = fa;
            a = hi - g * (hi - lo);
            fa = fit_linear(th, c_mean, n, std::exp(a), &p0, &p1);
        } else {
            lo = a; a = b; fa = fb;
            b = lo + g * (hi - lo);
            fb = fit_linear(th, c_mean, n, std::exp(b), &p0, &p1);
        }
    }
    const double rate = std::exp(0.5 * (lo + hi));
    fit_linear(th, c_mean, n, rate, c0, c1);
    delete[] th;
    *ach_per_hour = rate;
    return VF_OK;
}

int vf_wells_riley(double c0, double breathing_m3_h, double ach_per_hour, double t_hours, double* dose,
                   double* probability)
{
    if (!dose || !probability || ach_per_hour < 0 || t_hours < 0) return VF_EINVAL;
    double q;
    if (ach_per_hour == 0.0) q = c0 * breathing_m3_h * t_hours;   // no ventilation: dose grows linearly
    else q = c0 * breathing_m3_h * (-std::expm1(-ach_per_hour * t_hours)) / ach_per_hour;
    *dose = q;
    *probability = -std::expm1(-q);
    return VF_OK;
}

}  // extern "C"
